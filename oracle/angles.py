"""Angle sets for the oracle (TEST INFRASTRUCTURE ONLY: used by tests/, the
smoke check and the CPU-baseline leg of bench.py, never by the GPU library).

Sec. 3 of the paper: each angle is a unit vector n = (mu_x, mu_y, mu_z) with
a weight W; the quadrature is J = sum W I, H = sum W n I, K = sum W n n I.
The paper cites Carlson (1963) / Bruls et al. (1999) without listing values.
Readings used here:

* weights are normalised to sum 1, so J is the mean intensity and E_r = 4 pi J;
* level-symmetric S_N sets (N = 2, 4, 6, 8 -> 8, 24, 48, 80 angles): in each
  octant the points are (mu_i, mu_j, mu_k) with i + j + k = N/2 + 2 and
  mu_i^2 = mu_1^2 + (i - 1) * 2 (1 - 3 mu_1^2) / (N - 2); points that are
  permutations of one another share a weight.  mu_1 and the class weights are
  fixed by normalisation and the even moment conditions <mu^2k> = 1/(2k+1)
  (the LQ_N construction).  The paper's own 3-angle-per-octant set has
  mu_1 = 1/3 (mu_z = 0.333 and 0.882 in the moving-medium test, sec. 5.2) and
  is available as ``paper_s4``;
* 1-D slab sets: Gauss-Legendre nodes mu on (-1, 1) with weights w_GL / 2,
  represented as n = (mu, sqrt(1 - mu^2), 0).
"""
import itertools

import numpy as np
from scipy.optimize import brentq


def _octant_points(N, mu1):
    """Level indices and direction cosines of the S_N points in one octant."""
    L = N // 2
    if N == 2:
        levels = np.array([1.0 / np.sqrt(3.0)])
    else:
        delta = 2.0 * (1.0 - 3.0 * mu1 * mu1) / (N - 2)
        levels = np.sqrt(mu1 * mu1 + delta * np.arange(L))
    pts, cls = [], []
    classes = {}
    for i in range(1, L + 1):
        for j in range(1, L + 1):
            k = L + 2 - i - j
            if 1 <= k <= L:
                key = tuple(sorted((i, j, k)))
                classes.setdefault(key, len(classes))
                pts.append((levels[i - 1], levels[j - 1], levels[k - 1]))
                cls.append(classes[key])
    return np.array(pts), np.array(cls), len(classes)


def _moment_weights(pts, cls, ncls, nmom):
    """Class weights (per point, octant total 1/8) from normalisation and
    <mu_x^(2k)> = 1/(2k+1) for k = 2 .. ncls; returns the weights and the
    residual of the condition for k = ncls + 1 (nmom = ncls rows of moments)."""
    rows, rhs = [], []
    rows.append([np.sum(cls == c) for c in range(ncls)])
    rhs.append(1.0 / 8.0)
    for k in range(2, nmom + 2):
        rows.append([np.sum(pts[cls == c, 0] ** (2 * k)) for c in range(ncls)])
        rhs.append(1.0 / (2 * k + 1) / 8.0)
    A = np.array(rows[:ncls])
    b = np.array(rhs[:ncls])
    wc = np.linalg.solve(A, b)
    resid = np.dot(rows[ncls], wc) - rhs[ncls]
    return wc, resid


def _weights_at(N, mu1):
    p, c, nc = _octant_points(N, mu1)
    return _moment_weights(p, c, nc, nc)[0]


def level_symmetric(N, mu1=None):
    """S_N level-symmetric set over the full sphere: (n [M,3], w [M])."""
    if N == 2:
        pts, cls, ncls = _octant_points(2, None)
        wc = np.array([1.0 / 8.0])
    else:
        if mu1 is None:
            def f(x):
                p, c, nc = _octant_points(N, x)
                return _moment_weights(p, c, nc, nc)[1]
            # the residual has several roots on (0, 1/sqrt 3); keep the one
            # whose class weights are all positive
            grid = np.linspace(0.02, 1.0 / np.sqrt(3.0) - 1e-6, 400)
            vals = [f(x) for x in grid]
            roots = [brentq(f, grid[i], grid[i + 1], xtol=1e-16, rtol=1e-15, maxiter=500)
                     for i in range(len(grid) - 1) if vals[i] * vals[i + 1] < 0]
            good = [x for x in roots if np.all(_weights_at(N, x) > 0)]
            if len(good) != 1:
                raise ValueError("no unique positive-weight S_%d set" % N)
            mu1 = good[0]
        pts, cls, ncls = _octant_points(N, mu1)
        wc, _ = _moment_weights(pts, cls, ncls, ncls)
    n, w = [], []
    for sx, sy, sz in itertools.product((1.0, -1.0), repeat=3):
        for p, c in zip(pts, cls):
            n.append((sx * p[0], sy * p[1], sz * p[2]))
            w.append(wc[c])
    return np.array(n), np.array(w)


def paper_s4():
    """The 24-angle set of sec. 5.2 (mu_1 = 1/3, mu_2 = sqrt(7/9))."""
    return level_symmetric(4, mu1=1.0 / 3.0)


def gauss_legendre_1d(M):
    """Slab set: Gauss-Legendre mu (M nodes), weights w_GL/2, n = (mu, sqrt(1-mu^2), 0)."""
    mu, wg = np.polynomial.legendre.leggauss(M)
    n = np.stack([mu, np.sqrt(1.0 - mu * mu), np.zeros_like(mu)], axis=1)
    return n, wg / 2.0


def by_name(name):
    """'sN' (level-symmetric), 'paper_s4', or 'glM' (1-D Gauss-Legendre, M angles)."""
    if name == "paper_s4":
        return paper_s4()
    if name.startswith("gl"):
        return gauss_legendre_1d(int(name[2:]))
    if name.startswith("s"):
        return level_symmetric(int(name[1:]))
    raise ValueError(name)
