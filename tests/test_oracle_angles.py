"""Pins for the oracle's angle sets (sec. 3 of the paper)."""
import os

import numpy as np
import pytest

from oracle import angles

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("N", [2, 4, 6, 8])
def test_level_symmetric_invariants(N):
    # sec. 3: the scheme gives K_ii / J = 1/3 for isotropic I with any number
    # of angles; with sum W = 1 that is sum W n n = I/3, and sum W n = 0.
    n, w = angles.level_symmetric(N)
    assert len(w) == N * (N + 2)
    assert np.all(w > 0)
    np.testing.assert_allclose(np.linalg.norm(n, axis=1), 1.0, rtol=0, atol=1e-15)
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(n.T @ w, 0.0, atol=1e-16)
    np.testing.assert_allclose((n.T * w) @ n, np.eye(3) / 3.0, atol=2e-16)


def _golden_lq():
    rows = {}
    with open(os.path.join(GOLDEN, "lq_quadrature.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            left, right = line.split("|")
            vals = left.split()
            rows[int(vals[0])] = ([float(x) for x in vals[1:]], [float(x) for x in right.split()])
    return rows


@pytest.mark.parametrize("N", [4, 6, 8])
def test_level_symmetric_matches_published_lq_table(N):
    mus, ws = _golden_lq()[N]
    n, w = angles.level_symmetric(N)
    got_mu = sorted(set(np.round(np.abs(n[:, 0]), 9)))
    np.testing.assert_allclose(got_mu, mus, atol=1.5e-7)
    got_w = sorted(set(np.round(w * 8.0, 9)))  # octant-normalised
    # the tabulated mu_1 is rounded to 7 digits and dw/dmu_1 ~ 1.3, so the
    # weights carry a few 1e-7 of table rounding
    np.testing.assert_allclose(got_w, ws, atol=5e-7)


def test_paper_s4_cosines():
    # sec. 5.2 prints mu_z = 0.333 and 0.882 for its 3-angles-per-octant set
    vals = {}
    with open(os.path.join(GOLDEN, "paper_values.txt")) as f:
        for line in f:
            if not line.startswith("#") and line.strip():
                k, v = line.split()[:2]
                vals[k] = float(v)
    n, w = angles.paper_s4()
    got = sorted(set(np.round(np.abs(n[:, 2]), 3)))
    assert got == [vals["s4_mu_small"], vals["s4_mu_large"]]
    np.testing.assert_allclose((n.T * w) @ n, np.eye(3) / 3.0, atol=2e-16)


@pytest.mark.parametrize("M", [2, 4, 8, 16])
def test_gauss_legendre_exactness(M):
    # Gauss-Legendre with M nodes integrates mu^k exactly for k <= 2M - 1:
    # (1/2) int_{-1}^{1} mu^k dmu = 1/(k+1) for even k, 0 for odd k.
    n, w = angles.gauss_legendre_1d(M)
    mu = n[:, 0]
    for k in range(2 * M):
        exact = 1.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * mu ** k) - exact) < 1e-14
    np.testing.assert_allclose(np.linalg.norm(n, axis=1), 1.0, atol=1e-15)
