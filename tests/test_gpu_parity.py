"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on
identical seeded inputs.  FP64 path: 1e-12 norm-relative on every output.
Mixed path (FP32 intensities): 1e-5 on E_r and |F_r|, the bar for the
mixed-precision path; the other outputs are reported against looser
bounds derived from float32 storage."""
import numpy as np
import pytest

import oracle
from paper_1403_6126_gb300 import workloads as wlmod

from _helpers import field_err, flux_magnitude, gpu_context, initial_state, rel_err, run_both

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 1e-5


def _check_fp64(g, o):
    for k in ("I", "E", "F", "P", "T", "dEgas", "dMom"):
        err = field_err(g, o, k, o["wl"])
        assert err <= FP64_TOL, (k, err)


def _check_mixed(g, o):
    errE = rel_err(g["E"], o["E"])
    errF = field_err({"F": flux_magnitude(g["F"])}, {"F": flux_magnitude(o["F"]), "E": o["E"]}, "F", o["wl"])
    assert errE <= MIXED_TOL, ("E", errE)
    assert errF <= MIXED_TOL, ("|F|", errF)
    assert rel_err(g["T"], o["T"]) <= MIXED_TOL
    assert rel_err(g["I"], o["I"]) <= 1e-4
    # derived from float storage: the sources are differences of float sums
    assert field_err(g, o, "dMom", o["wl"]) <= 1e-4
    assert field_err(g, o, "dEgas", o["wl"]) <= 1e-4


SMALL = [
    ("slab1d", dict(n=64, steps=0), 30),
    ("slab1d", dict(n=37, M=16, steps=0), 20),            # ragged tile, 16 angles
    ("shadow2d", dict(nx=40, ny=24, angles="s4", steps=0), 15),
    ("shadow2d", dict(nx=33, ny=17, angles="s8", steps=0), 6),
    ("box3d", dict(n=12, angles="s4", steps=0), 5),
    ("box3d", dict(n=10, angles="s8", steps=0), 3),
]


@pytest.mark.parametrize("name,kw,nsteps", SMALL)
def test_fp64_matches_oracle(name, kw, nsteps):
    wl = wlmod.by_name(name, **kw)
    g, o = run_both(wl, nsteps, "fp64")
    _check_fp64(g, o)


@pytest.mark.parametrize("name,kw,nsteps", SMALL)
def test_mixed_matches_oracle(name, kw, nsteps):
    wl = wlmod.by_name(name, **kw)
    g, o = run_both(wl, nsteps, "fp32")
    _check_mixed(g, o)


def test_box3d_ragged_many_tiles_fp64():
    # several tiles in every direction plus a ragged tail on each axis
    wl = wlmod.box3d(n=20, angles="s2", steps=0)
    g, o = run_both(wl, 4, "fp64")
    _check_fp64(g, o)


def test_box3d_ragged_many_tiles_mixed():
    wl = wlmod.box3d(n=37, angles="s4", steps=0)
    g, o = run_both(wl, 3, "fp32", threads=8)
    _check_mixed(g, o)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_velocity_zero_in_half_the_box(precision):
    # v = 0 for x < 18: every face there has zero velocity (the IV state at
    # the face is the mean of its two cells' states) while the box's random
    # flow moves the rest, so tiles with and without such faces, and ragged
    # tiles, run in the same step
    wl = wlmod.box3d(n=37, angles="s4", steps=0)
    v = wl["v"].reshape(3, 37, 37, 37).copy()
    v[:, :, :, :18] = 0.0
    wl["v"] = v.reshape(3, -1)
    g, o = run_both(wl, 3, precision, threads=8)
    if precision == "fp64":
        _check_fp64(g, o)
    else:
        _check_mixed(g, o)


def test_flow_along_one_axis_2d():
    # 2-D flow along x only: every y face has zero velocity
    wl = wlmod.shadow2d(nx=40, ny=24, angles="s4", steps=0)
    wl["v"] = np.zeros_like(wl["v"])
    wl["v"][0] = 0.04 * wl["C"]
    g, o = run_both(wl, 10, "fp32")
    _check_mixed(g, o)


def test_single_cell_and_single_angle():
    # degenerate sizes: one cell (periodic onto itself) and one angle (W = 1)
    wl = wlmod.slab1d(n=1, M=2, steps=0)
    wl["bc"] = ((0, 0), (0, 0), (0, 0))
    g, o = run_both(wl, 5, "fp64")
    _check_fp64(g, o)
    wl = wlmod.slab1d(n=19, M=2, steps=0)
    n = np.array([[1.0, 0.0, 0.0]])
    w = np.array([1.0])
    g, o = run_both(wl, 4, "fp64", n=n, w=w)
    _check_fp64(g, o)


def test_many_angles():
    # 256 random directions with random positive weights (the largest set)
    rng = np.random.default_rng(7)
    n = rng.normal(size=(256, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    w = rng.uniform(0.5, 1.5, 256)
    w /= w.sum()
    wl = wlmod.slab1d(n=70, steps=0)
    g, o = run_both(wl, 3, "fp64", n=n, w=w)
    _check_fp64(g, o)
    g, o = run_both(wl, 3, "fp32", n=n, w=w)
    _check_mixed(g, o)


def test_pure_transport():
    # sigma = 0 everywhere: transport alone, with the inflow beam
    wl = wlmod.shadow2d(nx=24, ny=20, angles="s4", steps=0)
    wl["sa"] = np.zeros_like(wl["sa"])
    g, o = run_both(wl, 10, "fp64")
    _check_fp64(g, o)


def test_opaque_limit():
    # sigma_a = 1e6, sigma_s = 3e5 with |v| up to 0.1 C: dt C sigma ~ 5e4.
    # The angle sums with velocity weights (sum W n.v / d) cancel to ~1e-4 of
    # their terms here, so any two correct double-precision evaluations
    # differ by ~1e4 ulp; the bound is scaled by that condition number.
    wl = wlmod.box3d(n=8, angles="s2", steps=0)
    wl["sa"] = np.full_like(wl["sa"], 1e6)
    wl["ss"] = np.full_like(wl["ss"], 3e5)
    g, o = run_both(wl, 3, "fp64")
    for k in ("I", "E", "F", "P", "T", "dEgas", "dMom"):
        err = field_err(g, o, k, o["wl"])
        assert err <= 1e4 * 2.2e-16 * 10, (k, err)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_crossing_beams(precision):
    # Sec. 5.4 as an initial-value problem (see test_oracle_transport): two
    # beams on the 45-degree S2 angles cross in a periodic, source-free box;
    # 60 steps take them through each other.
    from test_oracle_transport import _beams_problem, _run_free
    from _helpers import gpu_context
    p, n, a, b, IA, IB = _beams_problem()
    N = p.N
    wl = dict(shape=p.shape, dim=2, lo=(0.0, 0.0, 0.0), hi=(1.0, 4.0, 1.0), bc=p.bc, C=1.0, P=1.0, cfl=0.4,
              gamma=5.0 / 3.0, R=1.0, hold_T=True, estimate_v=False, inflow={})
    ctx = gpu_context(wl, n, p.w, precision)
    ctx.set_intensity(IA + IB)
    ctx.set_material(np.ones(N), np.ones(N), np.zeros((3, N)), np.zeros(N), np.zeros(N))
    dt = oracle.cfl_dt(p, 0.4)
    assert abs(ctx.cfl_dt() - dt) <= 1e-15 * dt
    for _ in range(60):
        ctx.step(dt)
    ctx.sync()
    E, F, _ = ctx.moments()
    I = ctx.intensity()
    ctx.close()
    o = _run_free(p, IA + IB, dt, 60)
    Emax = np.abs(o["E"]).max()
    if precision == "fp64":
        assert np.abs(I - o["I"]).max() <= FP64_TOL * np.abs(o["I"]).max()
        assert np.abs(E - o["E"]).max() <= FP64_TOL * Emax
        assert np.abs(F - o["F"]).max() <= FP64_TOL * Emax
    else:
        assert np.abs(E - o["E"]).max() <= MIXED_TOL * Emax
        assert np.abs(flux_magnitude(F) - flux_magnitude(o["F"])).max() <= MIXED_TOL * Emax


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_inflow_change_between_graph_runs(precision):
    # rt_run replays a captured CUDA graph of its steps; an inflow table set
    # between two runs must reach the second one (the float step carries the
    # table in its launch parameters, which a kept graph would replay):
    # the same steps as plain launches give bitwise the same result
    import torch
    wl = wlmod.shadow2d(nx=40, ny=24, angles="s4", steps=0)
    n, w = oracle.angles.by_name(wl["angles"])
    stream = torch.cuda.Stream()
    out = []
    for graph in (True, False):
        ctx = gpu_context(wl, n, w, precision, stream=stream.cuda_stream)
        ctx.set_intensity(initial_state(wl, len(w), precision))
        ctx.set_material(wl["rho"], wl["T"], wl["v"], wl["sa"], wl["ss"])
        for k, scale in enumerate((1.0, 3.0)):
            if k:
                for (axis, side), rule in wl["inflow"].items():
                    ctx.set_inflow(axis, side, scale * wlmod.inflow_values(rule, n))
            if graph:
                ctx.run(0.0, 4)
            else:
                for _ in range(4):
                    ctx.step(0.0)
        ctx.sync()
        out.append(ctx.moments())
        ctx.close()
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)
