"""Host tables of the library (no GPU) pinned directly to what the paper prints:
the predictor's time-coupling matrix R (Eqs. B.9, C.18, D.28)."""
import numpy as np
import pytest

from test_oracle_refelem import load_r_matrices


@pytest.mark.parametrize("p", [2, 3, 4])
def test_library_time_matrix_is_the_printed_R(p):
    from paper_1905_02504_gb300 import geomhd
    R = geomhd.geo_time_matrix(p)
    printed = load_r_matrices()[p]
    assert np.abs(R - printed).max() < 1e-14
