"""Pins for the oracle's implicit source steps (secs. 4.3-4.5) and quadrature."""
import zlib

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
from oracle import angles

FOURPI = 4.0 * np.pi


def _uniform(shape, name, C, P, **kw):
    n, w = angles.by_name(name)
    return oracle.Problem(shape, 1.0 / max(shape), n, w, C=C, P=P, **kw)


def test_pure_absorption_held_T_decays_geometrically():
    # Step 4 with v = 0, T held, no transport (uniform periodic medium):
    # d I_m = r_m + dt C s_a B with d = 1 + dt C s_a, so
    # I_m^n - B = (I_m^0 - B) (1 + dt C s_a)^-n exactly, -> exp(-C s_a t).
    p = _uniform((1, 4, 4), "s4", C=10.0, P=1.0, hold_T=True)
    N, M = p.N, p.M
    rng = np.random.default_rng(5)
    I0 = np.repeat(rng.uniform(0.01, 0.2, (M, 1)), N, axis=1)
    T = np.full(N, 1.3)
    B = T[0] ** 4 / FOURPI
    sa = 2.5
    dt = oracle.cfl_dt(p, 0.4)
    I = I0.copy()
    for k in range(1, 6):
        I = oracle.step(p, dt, I, T, np.ones(N), np.zeros((3, N)), np.full(N, sa), np.zeros(N))["I"]
        np.testing.assert_allclose(I - B, (I0 - B) * (1 + dt * 10.0 * sa) ** (-k), rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("E0,T4,sa", [(100.0, 1.0, 1.0), (100.0, 1.0, 100.0), (1.0, 1e8, 1.0), (1.0, 1e8, 100.0)])
def test_thermal_equilibrium_static_medium(E0, T4, sa):
    # sec. 5.1: 2D periodic, rho = 1, v = 0, P = 1, C = 10, R = 1, gamma = 5/3.
    # Each step conserves P E_r + rho R T / (gamma - 1) (to the Newton
    # tolerance; the paper quotes < 1e-10) and the end state has E_r = T^4.
    p = _uniform((1, 4, 4), "s4", C=10.0, P=1.0, hold_T=False)
    N, M = p.N, p.M
    I = np.full((M, N), E0 / FOURPI)
    T = np.full(N, T4 ** 0.25)
    kv = 1.0 / (5.0 / 3.0 - 1.0)
    total0 = E0 + kv * T[0]
    dt = oracle.cfl_dt(p, 0.4)
    for k in range(400):
        out = oracle.step(p, dt, I, T, np.ones(N), np.zeros((3, N)), np.full(N, sa), np.zeros(N))
        assert out["failures"] == 0
        I, T = out["I"], out["T"]
        total = out["E"] + kv * T
        assert np.abs(total - total0).max() <= 1e-10 * total0
        # the energy handed to the gas is the change of its internal energy
        if k == 0:
            np.testing.assert_allclose(out["dEgas"], kv * (T - T4 ** 0.25), rtol=1e-14)
    Teq = brentq(lambda t: t ** 4 + kv * t - total0, 0.0, total0 ** 0.25 + total0)
    np.testing.assert_allclose(T, Teq, rtol=1e-9)
    np.testing.assert_allclose(out["E"], Teq ** 4, rtol=1e-8)


@pytest.mark.parametrize("dense", [False, True])
def test_isotropic_equilibrium_is_a_fixed_point(dense):
    # secs. 4.2-4.4: a static medium (v = 0) at one temperature with
    # I = T^4 / (4 pi) on every angle is in radiative equilibrium whatever the
    # opacities and densities are cell by cell: transport moves nothing, the
    # emission balances the absorption and scattering keeps an isotropic
    # field.  Every step leaves I and T as they were and hands the gas no
    # energy or momentum (T live, periodic 3-D box, uneven random fields).
    # To round-off: the dense Gaussian elimination of systems whose diagonal
    # reaches 1 + dt C sigma ~ 700 keeps about 12 digits (measured 1.0e-12
    # after five steps), the reduced form about 15.
    rtol = 1e-11 if dense else 1e-13
    rng = np.random.default_rng(17)
    p = _uniform((4, 5, 6), "s6", C=30.0, P=3.0, hold_T=False, dense=dense)
    N, M = p.N, p.M
    T0 = 1.3
    I = np.full((M, N), T0 ** 4 / FOURPI)
    T = np.full(N, T0)
    rho = rng.uniform(0.2, 5.0, N)
    sa, ss = 10 ** rng.uniform(-2, 4, N), 10 ** rng.uniform(-2, 4, N)
    dt = oracle.cfl_dt(p, 0.4)
    for _ in range(5):
        out = oracle.step(p, dt, I, T, rho, np.zeros((3, N)), sa, ss)
        assert out["failures"] == 0
        I, T = out["I"], out["T"]
    np.testing.assert_allclose(I, T0 ** 4 / FOURPI, rtol=rtol)
    np.testing.assert_allclose(T, T0, rtol=rtol)
    np.testing.assert_allclose(out["dEgas"], 0.0, atol=10 * rtol * T0 ** 4)
    np.testing.assert_allclose(out["dMom"], 0.0, atol=10 * rtol * T0 ** 4)
    np.testing.assert_allclose(out["E"], T0 ** 4, rtol=rtol)


@pytest.mark.parametrize("dense", [False, True])
@pytest.mark.parametrize("sa", [1.0, 100.0])
def test_energy_exchange_is_backward_euler_in_both_unknowns(sa, dense):
    # secs. 4.3 and 5.1: Step 4 is backward Euler in I and T together.  For a
    # static uniform medium (no transport, v = 0) with an anisotropic field,
    # every angle obeys its own discrete transfer equation with the NEW
    # temperature's emission, I1 - I0 = dt C s_a (T1^4 / (4 pi) - I1), and the
    # gas takes what the radiation loses, rho R/(gamma-1) (T1 - T0) =
    # -P (E1 - E0).  An emission at T^n (a semi-implicit step) keeps the
    # second relation and the equilibrium but fails the first.
    rng = np.random.default_rng(23)
    p = _uniform((1, 2, 2), "s4", C=10.0, P=1.0, hold_T=False, dense=dense)
    N, M = p.N, p.M
    I0 = np.repeat(rng.uniform(1.0, 15.0, (M, 1)), N, axis=1)
    T0 = np.full(N, 1.0)
    kv = 1.0 / (5.0 / 3.0 - 1.0)
    dt = oracle.cfl_dt(p, 0.4)
    out = oracle.step(p, dt, I0, T0, np.ones(N), np.zeros((3, N)), np.full(N, sa), np.zeros(N))
    assert out["failures"] == 0
    I1, T1 = out["I"], out["T"]
    a = dt * p.C * sa
    np.testing.assert_allclose(I1, (I0 + a * T1 ** 4 / FOURPI) / (1.0 + a), rtol=1e-12)
    E0 = FOURPI * np.einsum("m,mc->c", p.w, I0)
    np.testing.assert_allclose(kv * (T1 - T0), -p.P * (out["E"] - E0), rtol=1e-11, atol=1e-12 * E0.max())
    assert (T1 > 1.0).all()                 # the field (E ~ 100) heats the gas


def test_large_opacity_reaches_equilibrium_in_about_one_step():
    # sec. 5.1: with s_a = 100 the step is much longer than the thermalisation
    # time and the equilibrium is reached within about one step.
    n, w = angles.level_symmetric(4)
    p = oracle.Problem((1, 2, 2), 1.0 / 32, n, w, C=10.0, P=1.0)  # 32^2 cells of sec. 5.1
    N, M = p.N, p.M
    I = np.full((M, N), 100.0 / FOURPI)
    T = np.ones(N)
    dt = oracle.cfl_dt(p, 0.4)
    out = oracle.step(p, dt, I, T, np.ones(N), np.zeros((3, N)), np.full(N, 100.0), np.zeros(N))
    out = oracle.step(p, dt, out["I"], out["T"], np.ones(N), np.zeros((3, N)), np.full(N, 100.0), np.zeros(N))
    assert np.abs(out["E"] / out["T"] ** 4 - 1).max() < 1e-2


def test_temperature_root_matches_bisection():
    # For v = 0 and an isotropic right-hand side r, eq. absorptionmatrix gives
    # k_v (T - T0) + P C s_a dt (T^4 - E0) / (1 + dt C s_a) = 0 with
    # E0 = 4 pi r; its positive root is unique.
    n, w = angles.level_symmetric(6)
    p = oracle.Problem((1, 1, 1), 1.0, n, w, C=30.0, P=7.0, gamma=1.4, R=2.0)
    rng = np.random.default_rng(9)
    for _ in range(20):
        rho, T0, sa, dt = rng.uniform(0.1, 3), rng.uniform(0.2, 3), 10 ** rng.uniform(-2, 3), 10 ** rng.uniform(-4, -1)
        E0 = rng.uniform(0.01, 50)
        r = np.full(p.M, E0 / FOURPI)
        kv = rho * 2.0 / 0.4
        g = lambda T: kv * (T - T0) + 7.0 * 30.0 * sa * dt * (T ** 4 - E0) / (1 + dt * 30.0 * sa)
        Tb = brentq(g, 0.0, 10.0 + T0 + E0, xtol=1e-15, rtol=1e-15)
        for dense in (False, True):
            p.dense = dense
            p._s.dense = int(dense)
            I, T1, st = oracle.absorption_cell(p, rho, T0, sa, dt, np.zeros(3), r)
            assert st == 0
            assert abs(T1 - Tb) <= 1e-13 * Tb


def test_pure_scattering_conserves_J_and_relaxes_anisotropy():
    # Step 5 with v = 0: J is conserved exactly and I_m - J is divided by
    # (1 + dt C s_s) each step.
    p = _uniform((1, 2, 2), "s6", C=10.0, P=1.0, hold_T=True)
    N, M = p.N, p.M
    rng = np.random.default_rng(2)
    I0 = np.repeat(rng.uniform(0.0, 1.0, (M, 1)), N, axis=1)
    J0 = p.w @ I0
    ss = 3.0
    dt = oracle.cfl_dt(p, 0.4)
    I = I0.copy()
    for k in range(1, 5):
        I = oracle.step(p, dt, I, np.ones(N), np.ones(N), np.zeros((3, N)), np.zeros(N), np.full(N, ss))["I"]
        np.testing.assert_allclose(p.w @ I, J0, rtol=1e-14)
        np.testing.assert_allclose(I - J0, (I0 - J0) * (1 + dt * 10.0 * ss) ** (-k), rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("name", ["gl8", "s4", "s6", "s8"])
@pytest.mark.parametrize("hold_T", [False, True])
def test_reduced_solvers_equal_dense_brute_force(name, hold_T):
    # The O(N) reductions of Steps 4 and 5 against Gaussian elimination on the
    # full (N+1)- and N-unknown systems, random cells with |v| up to 0.3 C.
    n, w = angles.by_name(name)
    C = 20.0
    pr = oracle.Problem((1, 1, 1), 1.0, n, w, C=C, P=3.0, hold_T=hold_T)
    pd = oracle.Problem((1, 1, 1), 1.0, n, w, C=C, P=3.0, hold_T=hold_T, dense=True)
    rng = np.random.default_rng(zlib.crc32(repr((name, hold_T)).encode()))
    for _ in range(25):
        v = rng.normal(size=3)
        v *= rng.uniform(0, 0.3 * C) / np.linalg.norm(v)
        r = rng.uniform(0.0, 2.0, pr.M)
        rho, T0, sa, ss = rng.uniform(0.1, 3), rng.uniform(0.3, 2), 10 ** rng.uniform(-1, 3), 10 ** rng.uniform(-1, 3)
        dt = 10 ** rng.uniform(-4, -2)
        Ir, Tr, s1 = oracle.absorption_cell(pr, rho, T0, sa, dt, v, r)
        Id, Td, s2 = oracle.absorption_cell(pd, rho, T0, sa, dt, v, r)
        assert s1 == 0 and s2 == 0
        assert abs(Tr - Td) <= 1e-12 * Td
        np.testing.assert_allclose(Ir, Id, rtol=1e-11, atol=1e-12 * np.abs(Id).max())
        Sr, s1 = oracle.scattering_cell(pr, ss, dt, v, r)
        Sd, s2 = oracle.scattering_cell(pd, ss, dt, v, r)
        assert s1 == 0 and s2 == 0
        np.testing.assert_allclose(Sr, Sd, rtol=1e-11, atol=1e-12 * np.abs(Sd).max())


@pytest.mark.parametrize("which", ["absorption", "scattering"])
def test_moving_medium_steady_state(which):
    # sec. 5.2: in a uniform medium with a fixed velocity the intensities reach
    # a beamed steady state in which the co-moving flux vanishes:
    # F_r = v (E_r + P_xx) / C (the paper's F_v = F_r), and for absorption
    # E_r = T^4.  The Eulerian Eddington factors split, f_xx > 1/3 > f_yy.
    n, w = angles.paper_s4()
    C = 10.0
    p = oracle.Problem((1, 2, 2), 0.5, n, w, C=C, P=1.0, hold_T=True)
    N, M = p.N, p.M
    v = np.zeros((3, N))
    v[0] = 0.3 * C
    sa = np.full(N, 100.0 if which == "absorption" else 0.0)
    ss = np.full(N, 100.0 if which == "scattering" else 0.0)
    I = np.full((M, N), 1.0 / FOURPI)
    dt = 0.05
    for _ in range(300):
        out = oracle.step(p, dt, I, np.ones(N), np.ones(N), v, sa, ss)
        I = out["I"]
    E, F, P = out["E"], out["F"], out["P"]
    np.testing.assert_allclose(F[0], v[0] * (E + P[0]) / C, rtol=1e-10)
    np.testing.assert_allclose(F[1:], 0.0, atol=1e-12)
    if which == "absorption":
        np.testing.assert_allclose(E, 1.0, rtol=1e-10)
    assert np.all(P[0] / E > 1 / 3 + 1e-3) and np.all(P[1] / E < 1 / 3 - 1e-3)


@pytest.mark.parametrize("sa,ss", [(100.0, 0.0), (0.0, 100.0)])
def test_moving_medium_energy_error(sa, ss):
    # sec. 5.2: v_x = 0.3 C, T = E_r = 1, 3 angles per octant; the relative
    # total-energy error is about 1e-4 (the source terms are conservative to
    # O(dt^2)).  Per step: P dE_r + Delta E_T + Delta E_K ~ 0.
    n, w = angles.paper_s4()
    C = 10.0
    p = oracle.Problem((1, 2, 2), 0.5, n, w, C=C, P=1.0)
    N, M = p.N, p.M
    v = np.zeros((3, N))
    v[0] = 0.3 * C
    I = np.full((M, N), 1.0 / FOURPI)
    T = np.ones(N)
    dt = oracle.cfl_dt(p, 0.4)
    e_tot = 1.0 + 1.5 + 0.5 * (0.3 * C) ** 2
    worst = 0.0
    for _ in range(10):
        E0 = oracle.moments(p, I)[0]
        out = oracle.step(p, dt, I, T, np.ones(N), v, np.full(N, sa), np.full(N, ss))
        err = np.abs(out["E"] - E0 + out["dEgas"]).max() / e_tot
        worst = max(worst, err)
        I, T = out["I"], out["T"]
    assert worst < 3e-4
    # and the momentum handed to the gas balances the photon momentum
    out = oracle.step(p, dt, I, T, np.ones(N), v, np.full(N, sa), np.full(N, ss))
    F0 = oracle.moments(p, I)[1]
    np.testing.assert_allclose(out["dMom"], -(1.0 / C) * (out["F"] - F0), rtol=1e-12, atol=1e-15)


def test_velocity_estimate_limits():
    # sec. 4.5: with s_t = 0 the estimate is v itself; with s_t -> infinity it
    # is the momentum-exchange equilibrium C rho v~ + P v~ (E + P_dd)/C =
    # C rho v + P F, per axis.
    n, w = angles.level_symmetric(2)
    p = oracle.Problem((1, 1, 1), 1.0, n, w, C=10.0, P=50.0)
    v = np.array([0.3, -0.2, 0.1])
    F = np.array([0.5, 0.1, -0.3])
    Pd = np.array([0.4, 0.3, 0.5])
    np.testing.assert_allclose(oracle.vtilde(p, 2.0, v, 0.0, 1.2, F, Pd, 0.01), v, rtol=0, atol=0)
    vt = oracle.vtilde(p, 2.0, v, 1e14, 1.2, F, Pd, 0.01)
    lim = (10.0 * 2.0 * v + 50.0 * F) / (10.0 * 2.0 + 50.0 * (1.2 + Pd) / 10.0)
    np.testing.assert_allclose(vt, lim, rtol=1e-11)


def _momentum_exchange_exact(rho, v, F, K, st, C, P, t):
    """Exact solution at time t of the sec. 4.5 ODE pair with E_r and P_dd
    held (K = E + P_dd per axis):
        rho dv/dt = P st (F - v K / C),   dF/dt = -C st (F - v K / C).
    The total rho v + (P/C) F is conserved, and g = F - v K / C obeys
    dg/dt = -lam g with lam = st (C + P K / (rho C)), so
    v(t) = v + (P st / rho) g0 (1 - exp(-lam t)) / lam."""
    g0 = F - v * K / C
    lam = st * (C + P * K / (rho * C))
    return v + (P * st / rho) * g0 * (-np.expm1(-lam * t)) / lam


def test_velocity_estimate_is_a_half_step_of_the_momentum_exchange():
    # sec. 4.5: v~ estimates the velocity at n + 1/2 from the ODE pair of
    # photon-gas momentum exchange (E_r, P_r held).  Two checks against the
    # ODE itself rather than against the implicit formula:
    #  (a) as dt -> 0, (v~ - v^n) / dt tends to 1/2 of the ODE's rate
    #      dv/dt = (P st / rho) (F - v (E + P_dd) / C): v~ advances half a step;
    #  (b) v~ agrees with the exact solution at t = dt/2 to second order in
    #      dt (the error falls by ~4x when dt halves), as a one-step implicit
    #      estimate of the half-step velocity must.
    # Taking the full step dt in place of dt/2 fails (a) by a factor 2 and
    # (b) at first order.
    n, w = angles.level_symmetric(2)
    C, P, rho, st = 10.0, 50.0, 2.0, 3.0
    p = oracle.Problem((1, 1, 1), 1.0, n, w, C=C, P=P)
    v = np.array([0.3, -0.2, 0.1])
    F = np.array([0.5, 0.1, -0.3])
    E = 1.2
    Pd = np.array([0.4, 0.3, 0.5])
    K = E + Pd
    rate = (P * st / rho) * (F - v * K / C)
    dt = 1e-7
    slope = (oracle.vtilde(p, rho, v, st, E, F, Pd, dt) - v) / dt
    np.testing.assert_allclose(slope, 0.5 * rate, rtol=1e-5)
    errs = []
    for dt in (2e-3, 1e-3, 5e-4):
        vt = oracle.vtilde(p, rho, v, st, E, F, Pd, dt)
        errs.append(np.abs(vt - _momentum_exchange_exact(rho, v, F, K, st, C, P, 0.5 * dt)).max())
    for e1, e2 in zip(errs, errs[1:]):
        assert 3.5 < e1 / e2 < 4.5, errs
    # with the exchange fast against the step (lam dt >> 1) both reach the
    # exchange equilibrium g = 0, the implicit estimate to O(1 / (lam dt))
    vt = oracle.vtilde(p, rho, v, 1e6, E, F, Pd, 1.0)
    vinf = _momentum_exchange_exact(rho, v, F, K, 1e6, C, P, 0.5)
    np.testing.assert_allclose(vt, vinf, rtol=1e-5)


def test_quadrature_of_isotropic_field():
    # sec. 3: for isotropic I, E_r = 4 pi I, F_r = 0, P_r = E_r / 3 * identity.
    for name in ("s2", "s4", "s6", "s8"):
        n, w = angles.by_name(name)
        p = oracle.Problem((1, 1, 3), 1.0, n, w, C=1.0, P=1.0)
        I = np.full((p.M, 3), 0.7)
        E, F, P = oracle.moments(p, I)
        np.testing.assert_allclose(E, FOURPI * 0.7, rtol=1e-15)
        np.testing.assert_allclose(F, 0.0, atol=1e-15)
        np.testing.assert_allclose(P[:3], FOURPI * 0.7 / 3, rtol=1e-14)
        np.testing.assert_allclose(P[3:], 0.0, atol=1e-15)


@pytest.mark.parametrize("estimate_v", [False, True])
def test_transparent_cells_exchange_nothing_with_the_gas(estimate_v):
    # secs. 2 and 4.3-4.4: the radiation acts on the gas only through the
    # opacities.  In a cell with sigma_a = sigma_s = 0 the beams pass through
    # (the transport changes I there) but the gas gets no momentum, no
    # energy and keeps its temperature; the momentum source counts only the
    # change made by the implicit steps (eq. momentumchange), not the
    # transport flux.  A random anisotropic field on a periodic 3-D box,
    # moving gas, every other cell transparent.
    rng = np.random.default_rng(31)
    p = _uniform((4, 4, 6), "s4", C=20.0, P=5.0, hold_T=False, estimate_v=estimate_v)
    N, M = p.N, p.M
    I = rng.uniform(0.05, 2.0, (M, N))
    T = rng.uniform(0.5, 1.5, N)
    rho = rng.uniform(0.5, 2.0, N)
    v = rng.uniform(-0.1, 0.1, (3, N)) * p.C
    clear = (np.arange(N) % 2) == 0
    sa = np.where(clear, 0.0, 10 ** rng.uniform(-1, 2, N))
    ss = np.where(clear, 0.0, 10 ** rng.uniform(-1, 2, N))
    dt = oracle.cfl_dt(p, 0.4)
    out = oracle.step(p, dt, I, T, rho, v, sa, ss, return_dF=True)
    assert out["failures"] == 0
    assert np.abs(out["dF"][:, clear]).max() > 1e-2          # the beams do move through them
    # zero to the rounding of the (identity) implicit solves
    mscale, escale = np.abs(out["dMom"]).max(), np.abs(out["dEgas"]).max()
    np.testing.assert_allclose(out["dMom"][:, clear], 0.0, atol=1e-13 * mscale)
    np.testing.assert_allclose(out["dEgas"][clear], 0.0, atol=1e-13 * escale)
    np.testing.assert_array_equal(out["T"][clear], T[clear])
    np.testing.assert_allclose(out["I"][:, clear], (I + out["dF"])[:, clear], rtol=1e-14, atol=0)
    assert np.abs(out["dMom"][:, ~clear]).min() > 0 and np.abs(out["dEgas"][~clear]).min() > 0
