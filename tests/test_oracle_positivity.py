"""Pins of the oracle's positivity scaling (reading of Sec. I, see oracle/positivity.py)."""
import numpy as np

from oracle import positivity
from oracle.physics import conserved, primitives

G = 5.0 / 3.0


def states(rho, p, rng, n):
    v = rng.uniform(-1, 1, (n, 3))
    B = rng.uniform(-1, 1, (n, 3))
    return conserved(np.asarray(rho, float), v, np.asarray(p, float), B, G)


def test_positive_states_untouched():
    rng = np.random.default_rng(0)
    s = states(rng.uniform(0.5, 1.0, 9), rng.uniform(0.5, 1.0, 9), rng, 9)[None]
    mean = s.mean(axis=1)
    out, th = positivity.limit(s, mean, G)
    assert th[0] == 1.0 and np.array_equal(out, s)


def test_limited_states_are_positive_and_keep_the_mean():
    rng = np.random.default_rng(1)
    for _ in range(20):
        rho = rng.uniform(-0.5, 1.5, 12)
        p = rng.uniform(-0.5, 1.5, 12)
        s = states(np.abs(rho), np.abs(p), rng, 12)
        s[:, 0] = rho                                   # some negative densities
        s[:, 4] -= rng.uniform(0, 2, 12)                # and some negative pressures
        mean = states([1.0], [0.5], rng, 1)[0]
        out, th = positivity.limit(s[None], mean[None], G)
        r, v, pp, B = primitives(out[0], G)
        assert (r >= min(1e-13, 1.0) * (1 - 1e-12)).all()
        assert (pp >= -1e-12).all()
        assert 0.0 <= th[0] <= 1.0
        # the scaling is affine toward the mean: (out - mean) = theta (s - mean)
        assert np.allclose(out[0] - mean, th[0] * (s - mean), atol=1e-14)
