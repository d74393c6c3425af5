"""The library's prism element (geo_prism_nodes, geo_prism_derivatives: host
code, no GPU) against the nodes the paper prints (Eqs. C.2-C.16, D.2-D.27) and
the oracle's element, in the same order."""
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


@pytest.mark.parametrize("p", [2, 3, 4])
def test_library_prism_derivatives(p):
    """The library's D^alpha equals the oracle element's; the entries it sets to
    zero are exactly those the oracle has at rounding level (nonzeros 42 / 247 /
    580), and the nonzero pattern the predictor walks is the same."""
    from paper_1905_02504_gb300 import geomhd
    D = geomhd.geo_prism_derivatives(p)
    ref = PR.PrismElement(p).D
    scale = np.abs(ref).max()
    assert np.abs(D - ref).max() < 1e-12 * scale
    assert ((D != 0) == (np.abs(ref) > 1e-12 * scale)).all()
    assert int((D != 0).sum()) == {2: 42, 3: 247, 4: 580}[p]
