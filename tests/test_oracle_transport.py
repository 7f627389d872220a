"""Pins for the oracle's transport step (sec. 4.2) and boundary values."""
import numpy as np
import pytest

import oracle
from oracle import angles


def _two_rays(mu=1.0):
    s = np.sqrt(max(0.0, 1.0 - mu * mu))
    n = np.array([[mu, s, 0.0], [-mu, s, 0.0]])
    return n, np.array([0.5, 0.5])


def _zeros(N):
    return np.zeros(N)


@pytest.mark.parametrize("with_v", [False, True])
def test_flux_differencing_conserves_each_ray(with_v):
    # Abstract / sec. 4.2: conservative differencing keeps sum_cells I_m fixed
    # on a periodic grid with no sources (sigma = 0), for every angle.
    rng = np.random.default_rng(11)
    n, w = angles.level_symmetric(4)
    p = oracle.Problem((5, 6, 7), (0.1, 0.12, 0.09), n, w, C=10.0, P=1.0)
    N, M = p.N, p.M
    I = rng.uniform(0.1, 2.0, (M, N))
    v = rng.uniform(-0.5, 0.5, (3, N)) if with_v else np.zeros((3, N))
    dt = oracle.cfl_dt(p, 0.4)
    dF = oracle.transport(p, dt, I, v, _zeros(N), _zeros(N))
    scale = np.abs(dF).max()
    assert scale > 1e-3
    np.testing.assert_allclose(dF.sum(axis=1), 0.0, atol=1e-13 * scale * N)
    out = oracle.step(p, dt, I, np.ones(N), np.ones(N), v, _zeros(N), _zeros(N))
    np.testing.assert_allclose(out["I"].sum(axis=1), I.sum(axis=1), rtol=1e-13)


def test_unit_courant_number_shifts_one_cell():
    # With alpha = 1 (sigma = 0), v = 0, mu = +-1 and C dt = dx (nu = 1) the
    # van Leer face state is the upwind cell value, so each step moves every
    # ray exactly one cell (sec. 4.2 with Stone & Mihalas eq. 4 at nu = 1).
    n, w = _two_rays(1.0)
    nx = 16
    p = oracle.Problem((1, 1, nx), 1.0 / nx, n, w, C=10.0, P=1.0, dim=1)
    rng = np.random.default_rng(3)
    I = rng.uniform(0.0, 1.0, (2, nx))
    dt = (1.0 / nx) / 10.0
    out = oracle.step(p, dt, I, np.ones(nx), np.ones(nx), np.zeros((3, nx)), _zeros(nx), _zeros(nx))
    np.testing.assert_allclose(out["I"][0], np.roll(I[0], 1), rtol=0, atol=1e-15)
    np.testing.assert_allclose(out["I"][1], np.roll(I[1], -1), rtol=0, atol=1e-15)


@pytest.mark.parametrize("kind", [oracle.VACUUM, oracle.INFLOW, oracle.COPY])
def test_boundary_kinds_at_unit_courant(kind):
    # Ghost values (sec. 5.3 / 5.8 setups): vacuum zeroes incoming rays,
    # inflow sets them, copy repeats the last active cell.  At nu = 1 the first
    # cell takes the ghost value of the incoming ray after one step.
    n, w = _two_rays(1.0)
    nx = 8
    inflow = {(0, 0): np.array([7.0, 0.0])}
    p = oracle.Problem((1, 1, nx), 1.0 / nx, n, w, C=10.0, P=1.0, dim=1,
                       bc=((kind, oracle.VACUUM), (0, 0), (0, 0)), inflow=inflow)
    I = np.arange(1.0, 1.0 + 2 * nx).reshape(2, nx)
    dt = (1.0 / nx) / 10.0
    out = oracle.step(p, dt, I, np.ones(nx), np.ones(nx), np.zeros((3, nx)), _zeros(nx), _zeros(nx))
    expect_first = {oracle.VACUUM: 0.0, oracle.INFLOW: 7.0, oracle.COPY: I[0, 0]}[kind]
    assert out["I"][0, 0] == expect_first
    np.testing.assert_array_equal(out["I"][0, 1:], I[0, :-1])
    # the mu < 0 ray leaves through x_lo and enters through the vacuum x_hi
    np.testing.assert_array_equal(out["I"][1, :-1], I[1, 1:])
    assert out["I"][1, -1] == 0.0


def test_light_crossing_time_step_keeps_transport_bounded():
    # Step 1 (sec. 4.1): dt from the cell size and the speed of light with a
    # CFL number of 0.4.  Pinned by what it is for: at that dt the explicit,
    # unsplit van Leer transport of every ray of the 3-D S8 set (sigma = 0,
    # periodic, uneven cells) keeps each angle's values inside the range they
    # started in, step after step; at CFL 1 (a ray along the cube diagonal
    # then crosses sqrt(3) cells per step) the first step already leaves it.
    # Inactive axes do not limit dt.
    n, w = angles.level_symmetric(8)
    rng = np.random.default_rng(5)
    p = oracle.Problem((6, 7, 8), (0.1, 0.07, 0.13), n, w, C=3.0, P=1.0)
    N = p.N
    flat = lambda I: oracle.step(p, dt, I, np.ones(N), np.ones(N), np.zeros((3, N)), _zeros(N), _zeros(N))["I"]
    dt = oracle.cfl_dt(p, 0.4)
    assert dt * p.C / 0.07 == pytest.approx(0.4, rel=1e-15)
    I0 = rng.uniform(0.0, 1.0, (p.M, N))
    I = I0
    for _ in range(100):
        I = flat(I)
        assert (I.min(axis=1) >= I0.min(axis=1) - 1e-13).all() and (I.max(axis=1) <= I0.max(axis=1) + 1e-13).all()
    assert np.ptp(I, axis=1).max() < 0.5 * np.ptp(I0, axis=1).min()     # and it did move them
    dt = oracle.cfl_dt(p, 1.0)
    I = flat(I0)
    assert (I.min(axis=1) < I0.min(axis=1) - 0.1).any() or (I.max(axis=1) > I0.max(axis=1) + 0.1).any()
    p1 = oracle.Problem((1, 1, 8), (0.1, 1e-9, 1e-9), n, w, C=3.0, P=1.0, dim=1)
    assert oracle.cfl_dt(p1, 0.4) * 3.0 / 0.1 == pytest.approx(0.4, rel=1e-15)


def test_uniform_field_has_no_transport():
    # a constant intensity with uniform J and v gives zero flux divergence
    n, w = angles.level_symmetric(6)
    p = oracle.Problem((4, 4, 4), 0.25, n, w, C=5.0, P=1.0)
    N = p.N
    I = np.full((p.M, N), 0.3)
    v = np.tile(np.array([[0.2], [-0.1], [0.05]]), (1, N))
    dF = oracle.transport(p, 0.01, I, v, np.full(N, 2.0), np.full(N, 1.0))
    assert np.abs(dF).max() < 1e-15


def _advect_error(nx, steps_per_unit=None):
    # one ray along +x, sigma = 0, periodic, smooth profile; error after t = 1/C
    n, w = _two_rays(1.0)
    C = 1.0
    p = oracle.Problem((1, 1, nx), 1.0 / nx, n, w, C=C, P=1.0, dim=1)
    x = (np.arange(nx) + 0.5) / nx
    prof = lambda s: 1.0 + 0.5 * np.sin(2 * np.pi * s)
    I = np.stack([prof(x), prof(x)])
    dt = oracle.cfl_dt(p, 0.4)
    nsteps = int(round(0.5 / dt))
    dt = 0.5 / nsteps
    for _ in range(nsteps):
        I = oracle.step(p, dt, I, np.ones(nx), np.ones(nx), np.zeros((3, nx)), _zeros(nx), _zeros(nx))["I"]
    return np.mean(np.abs(I[0] - prof(x - 0.5)))


def test_second_order_convergence_on_smooth_profile():
    # van Leer reconstruction is second order away from extrema; in L1 over a
    # sine wave the observed order must be well above first order.
    e1, e2, e3 = (_advect_error(nx) for nx in (32, 64, 128))
    order = np.log2(e2 / e3)
    assert np.log2(e1 / e2) > 1.5 and order > 1.6, (e1, e2, e3)


def test_alpha_limits():
    # sec. 4.2: alpha -> 1 for an optically thin cell, alpha ~ 1/(10 dl sigma)
    # when the optical depth per cell is large.
    assert oracle.alpha(0.1, 0.0) == 1.0
    assert abs(oracle.alpha(0.1, 1e-5) - 1.0) < 1e-9
    for s in (10.0, 100.0, 1e4):
        a = oracle.alpha(0.1, s)
        assert abs(a * (10 * 0.1 * s) - 1.0) < 1e-12
    # tau = 1 exactly: sqrt(1 - e^-1)
    assert abs(oracle.alpha(0.1, 1.0) - np.sqrt(1 - np.exp(-1.0))) < 1e-15


def _beams_problem():
    """Sec. 5.4 crossing beams, as an initial-value problem: a periodic-in-x,
    vacuum-in-y box of 32 x 128 square cells, sigma = 0, S2 angles (every
    direction at 45 degrees to the x and y axes in the x-y plane).  Beam A is
    a 4 x 4-cell blob of I = 1 on the two angles with n_x > 0, n_y > 0, beam
    B one on the two angles with n_x < 0, n_y > 0, 12 cells to its right."""
    n, w = angles.level_symmetric(2)
    nx, ny = 32, 128
    p = oracle.Problem((1, ny, nx), (1.0 / nx, 4.0 / ny, 1.0), n, w, C=1.0, P=1.0, dim=2,
                       bc=((oracle.PERIODIC, oracle.PERIODIC), (oracle.VACUUM, oracle.VACUUM),
                           (oracle.PERIODIC, oracle.PERIODIC)), hold_T=True)
    a = np.where((n[:, 0] > 0) & (n[:, 1] > 0))[0]
    b = np.where((n[:, 0] < 0) & (n[:, 1] > 0))[0]
    IA, IB = np.zeros((p.M, ny, nx)), np.zeros((p.M, ny, nx))
    IA[a, 8:12, 8:12] = 1.0
    IB[b, 8:12, 20:24] = 1.0
    return p, n, a, b, IA.reshape(p.M, -1), IB.reshape(p.M, -1)


def _run_free(p, I, dt, steps):
    N = p.N
    out = None
    for _ in range(steps):
        out = oracle.step(p, dt, I, np.ones(N), np.ones(N), np.zeros((3, N)), _zeros(N), _zeros(N))
        I = out["I"]
    return out


def test_crossing_beams_pass_through_each_other():
    # Sec. 5.4: with the intensity split by angle, two beams that cross do
    # not interact (an angle-moment closure would merge them where they
    # cross): after they have crossed, each angle holds exactly what it holds
    # when its beam travels alone, and E_r is the sum.  Each angle's sum over
    # cells is conserved (sigma = 0, the blobs stay off the vacuum faces), and
    # each blob's centroid moves at C n.
    p, n, a, b, IA, IB = _beams_problem()
    dt = oracle.cfl_dt(p, 0.4)
    steps = 60                     # relative x speed 0.46 cells/step: they meet near step 26
    both = _run_free(p, IA + IB, dt, steps)
    onlyA = _run_free(p, IA, dt, steps)
    onlyB = _run_free(p, IB, dt, steps)
    np.testing.assert_array_equal(both["I"][a], onlyA["I"][a])
    np.testing.assert_array_equal(both["I"][b], onlyB["I"][b])
    assert np.abs(both["I"][a]).max() > 0.1 and np.abs(onlyA["I"][b]).max() == 0.0
    np.testing.assert_allclose(both["E"], onlyA["E"] + onlyB["E"], rtol=0, atol=1e-15 * both["E"].max())
    ny, nx = p.shape[1], p.shape[2]
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) * 4.0 / ny
    t = steps * dt
    for m in np.concatenate([a, b]):
        I0 = (IA + IB)[m].reshape(ny, nx)
        I1 = both["I"][m].reshape(ny, nx)
        assert abs(I1.sum() / I0.sum() - 1.0) < 1e-13
        # x: offsets from the expected centre wrapped into (-0.5, 0.5] (periodic)
        wx0, wx1 = I0.sum(axis=0), I1.sum(axis=0)
        x_expect = (wx0 * x).sum() / wx0.sum() + p.C * n[m, 0] * t
        dxw = (x - x_expect + 0.5) % 1.0 - 0.5
        assert abs((wx1 * dxw).sum() / wx1.sum()) < 0.05 / nx, m
        wy0, wy1 = I0.sum(axis=1), I1.sum(axis=1)
        y_expect = (wy0 * y).sum() / wy0.sum() + p.C * n[m, 1] * t
        assert abs((wy1 * y).sum() / wy1.sum() - y_expect) < 0.05 * 4.0 / ny, m


def test_outgoing_rays_see_the_same_ghost_at_every_open_face():
    # Boundary values (setups of secs. 5.3, 5.8): vacuum, copy and inflow
    # faces all copy the OUTGOING rays from the last active cell; they differ
    # only on the incoming ones.  Each angle's transport depends only on its
    # own intensities (v = 0), so an outgoing ray's Delta F is the same for
    # the three kinds, also where the cells are optically thick (alpha < 1:
    # the downwind ghost enters the face value).
    n, w = angles.level_symmetric(4)
    rng = np.random.default_rng(41)
    shape = (1, 6, 7)
    N, M = 42, len(w)
    I = rng.uniform(0.1, 2.0, (M, N))
    st = 10 ** rng.uniform(0, 3, N)                      # 10 dl sigma_t up to 1e3: alpha well below 1
    dFs = {}
    for kind in (oracle.VACUUM, oracle.COPY, oracle.INFLOW):
        p = oracle.Problem(shape, (0.1, 0.12, 1.0), n, w, C=10.0, P=1.0, dim=2,
                           bc=((kind, kind), (oracle.PERIODIC, oracle.PERIODIC), (0, 0)),
                           inflow={(0, 0): rng.uniform(0, 3, M), (0, 1): rng.uniform(0, 3, M)})
        dFs[kind] = oracle.transport(p, 0.4 * 0.1 / 10.0, I, np.zeros((3, N)), st, np.zeros(N))
    out_lo = n[:, 0] < 0          # leaving through x_lo
    out_hi = n[:, 0] > 0          # leaving through x_hi
    first = (np.arange(N) % 7) == 0
    last = (np.arange(N) % 7) == 6
    for kind in (oracle.COPY, oracle.INFLOW):
        np.testing.assert_allclose(dFs[kind][np.ix_(out_lo, first)], dFs[oracle.VACUUM][np.ix_(out_lo, first)],
                                   rtol=1e-14, atol=1e-14)
        np.testing.assert_allclose(dFs[kind][np.ix_(out_hi, last)], dFs[oracle.VACUUM][np.ix_(out_hi, last)],
                                   rtol=1e-14, atol=1e-14)
    # the incoming rays do see the face kind
    assert np.abs(dFs[oracle.COPY][np.ix_(out_hi, first)] - dFs[oracle.VACUUM][np.ix_(out_hi, first)]).max() > 1e-3


def test_pressure_tensor_component_order():
    # sec. 3: P_r = 4 pi sum W n n I, stored xx, yy, zz, xy, xz, yz.  One
    # ray along (1, 2, 3)/sqrt(14) carrying all the radiation.
    nvec = np.array([[1.0, 2.0, 3.0]]) / np.sqrt(14.0)
    p = oracle.Problem((1, 1, 2), 1.0, nvec, np.array([1.0]), C=1.0, P=1.0, dim=1)
    E, F, P = oracle.moments(p, np.full((1, 2), 0.5))
    s = 4 * np.pi * 0.5 / 14.0
    np.testing.assert_allclose(E, 4 * np.pi * 0.5, rtol=1e-15)
    np.testing.assert_allclose(F[:, 0] * np.sqrt(14.0) / (4 * np.pi * 0.5), [1, 2, 3], rtol=1e-15)
    np.testing.assert_allclose(P[:, 0] / s, [1, 4, 9, 2, 3, 6], rtol=1e-14)
