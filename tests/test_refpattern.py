"""The compiled structure of the serendipity element (refpattern.py, the build step
behind the variable-layout predictor schedule) against the oracle's element
(Sec. V.c, Eq. 5.3): the pattern holds every nonzero of the nodal derivative
matrices and nothing that is zero, the face and edge node lists are the nodes on
each face and edge, and the row groups cover the rows with balanced work.  The
kernels read D^alpha only at the compiled positions, so a missing entry would
drop a term of the flux difference."""
import numpy as np
import pytest

from oracle import refelem
from paper_1905_02504_gb300 import refpattern


@pytest.mark.parametrize("p", [2, 3, 4])
def test_derivative_pattern_is_the_nonzero_set(p):
    el = refelem.HexElement(p)
    np.testing.assert_allclose(np.array(refpattern.nodes(p), dtype=float), el.nodes, atol=0)
    pat = refpattern.derivative_pattern(p)
    for a in range(3):
        mask = np.zeros((el.N, el.N), bool)
        for i, j in pat[a]:
            mask[i, j] = True
        D = el.D[a]
        scale = np.abs(D).max()
        assert np.abs(D[~mask]).max() < 1e-12 * scale          # nothing nonzero left out
        assert np.abs(D[mask]).min() > 1e-8 * scale            # no structural zero compiled in


@pytest.mark.parametrize("p", [2, 3, 4])
def test_face_and_edge_node_lists(p):
    el = refelem.HexElement(p)
    for f, nodes in enumerate(refpattern.face_nodes(p)):
        on = np.nonzero(np.abs(el.nodes[:, refelem.FACE_AXIS[f]] - refelem.FACE_SIDE[f]) < 1e-14)[0]
        assert nodes == on.tolist()
    for e, nodes in enumerate(refpattern.edge_nodes(p)):
        fixed = [a for a in range(3) if a != refelem.EDGE_AXIS[e]]
        on = np.nonzero(np.all(np.abs(el.nodes[:, fixed] - refelem.EDGE_FIXED[e][fixed]) < 1e-14, axis=1))[0]
        assert nodes == on.tolist()


@pytest.mark.parametrize("p", [2, 3, 4])
def test_row_groups_partition_and_balance(p):
    pat = refpattern.derivative_pattern(p)
    rg = refpattern.row_groups(p, pat)
    N = len(refpattern.nodes(p))
    assert rg[0] == 0 and rg[-1] == N and all(a < b for a, b in zip(rg, rg[1:]))
    work = [sum(1 for ax in pat for i, _ in ax if a <= i < b) for a, b in zip(rg, rg[1:])]
    assert max(work) <= 1.15 * sum(work) / len(work)


def test_generated_header_is_current(tmp_path):
    """The header the build writes is a pure function of the generator."""
    out = tmp_path / "refpattern.h"
    refpattern.write(str(out))
    text = out.read_text()
    assert text == refpattern.header()
    for p, nnz in ((2, 16), (3, 96), (4, 192)):
        assert "struct RefPattern<%d>" % p in text and "NNZ = %d," % nnz in text
