"""The library's prism nodes (geo_prism_nodes, host code, no GPU) against the
nodes the paper prints (Eqs. C.2-C.16, D.2-D.27) and the oracle's element, in
the same order."""
import numpy as np
import pytest

from oracle import prism as PR
from test_oracle_prism import printed_nodes, _same_set


@pytest.mark.parametrize("p", [2, 3, 4])
def test_library_prism_nodes(p):
    from paper_1905_02504_gb300 import geomhd
    n = geomhd.geo_prism_nodes(p)
    assert _same_set(n, printed_nodes(p))
    assert np.allclose(n, PR.prism_nodes(p), atol=1e-15)
