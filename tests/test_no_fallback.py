"""Without the compiled library the binding refuses to import (there is no CPU
path to fall back to): a copy of the Python package with no lib/ directory."""
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_binding_without_library_fails_loudly(tmp_path):
    pkg = os.path.join(ROOT, "paper_1905_02504_gb300")
    dst = tmp_path / "paper_1905_02504_gb300"
    dst.mkdir()
    for name in os.listdir(pkg):
        if name.endswith(".py"):
            shutil.copy(os.path.join(pkg, name), dst / name)
    code = "import sys; sys.path.insert(0, %r); from paper_1905_02504_gb300 import geomhd" % str(tmp_path)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode != 0
    assert "libgeomhd.so is not built" in r.stderr
