"""The two-kernel 3-D path (transport marched along z over an x-y column,
then the per-cell implicit steps) against the fused kernel and the oracle.

Every column tile gives results bitwise equal to the fused kernel's (same
arithmetic in the same order), on a ragged grid that is not a multiple of
any tile, with vacuum, inflow, copy and periodic faces, an odd angle count
(the padded pair), with and without velocity terms; and the path matches the
FP64 oracle within the mixed-precision bound."""
import numpy as np
import pytest

import oracle
import paper_1403_6126_gb300 as rt
from paper_1403_6126_gb300 import workloads as wlmod

from _helpers import field_err, flux_magnitude, gpu_context, oracle_problem, rel_err

pytestmark = pytest.mark.gpu

SPLIT_TILES = [(32, 8, 0), (16, 16, 0), (16, 8, 0)]
P_, V_, C_, I_ = wlmod.PERIODIC, wlmod.VACUUM, wlmod.COPY, wlmod.INFLOW


def _odd_angles(M=7, seed=3):
    rng = np.random.default_rng(seed)
    n = rng.normal(size=(M, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    return n, np.full(M, 1.0 / M)


def _workload(shape, bc, velocity, seed=11):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    N = nx * ny * nz
    C = 10.0
    v = rng.normal(size=(3, N))
    v *= (0.05 * C * rng.uniform(0, 1, N)) / np.linalg.norm(v, axis=0)
    if not velocity:
        v[:] = 0.0
    wl = dict(name="box3d_custom", shape=shape, dim=3, lo=(0.0, 0.0, 0.0), hi=(nx / 32.0, ny / 32.0, nz / 32.0), bc=bc,
              angles=None, C=C, P=1.0, gamma=5.0 / 3.0, R=1.0, cfl=0.4, hold_T=False, estimate_v=velocity,
              rho=rng.uniform(0.5, 2.0, N), T=rng.uniform(0.8, 1.2, N), v=v, sa=10.0 ** rng.uniform(-1, 2, N),
              ss=10.0 ** rng.uniform(-1, 2, N), inflow={}, precision="fp32")
    if bc[0][0] == I_:
        wl["inflow"] = {(0, 0): ("beam", 2.0, 0)}
    return wlmod.rounded_to_float32(wl)


def _run(wl, n, w, tile, nsteps, I0):
    ctx = gpu_context(wl, n, w, "fp32")
    if tile is not None:
        ctx.set_tile(*tile)
    ctx.set_intensity(I0)
    ctx.set_material(wl["rho"], wl["T"], wl["v"], wl["sa"], wl["ss"])
    for _ in range(nsteps):
        ctx.step(0.0)
    ctx.sync()
    E, F, P = ctx.moments()
    dE, dM, T = ctx.sources()
    out = dict(I=ctx.intensity(), E=E, F=F, P=P, dEgas=dE, dMom=dM, T=T)
    ctx.close()
    return out


CASES = [
    ("periodic", ((P_, P_), (P_, P_), (P_, P_)), True, "s4"),
    ("open", ((I_, C_), (V_, V_), (C_, V_)), True, "s4"),
    ("open_static", ((I_, C_), (V_, V_), (C_, V_)), False, "s2"),
    ("odd_angles", ((P_, P_), (V_, C_), (P_, P_)), True, "odd"),
]


@pytest.mark.parametrize("name,bc,velocity,angles", CASES)
def test_split_equals_fused_bitwise(name, bc, velocity, angles):
    wl = _workload((11, 19, 37), bc, velocity)
    n, w = _odd_angles() if angles == "odd" else oracle.angles.by_name(angles)
    rng = np.random.default_rng(5)
    I0 = (rng.uniform(0.5, 1.5, (len(w), int(np.prod(wl["shape"])))) / (4 * np.pi)).astype(np.float32).astype(np.float64)
    ref = _run(wl, n, w, (16, 8, 4), 3, I0)
    for tile in SPLIT_TILES:
        got = _run(wl, n, w, tile, 3, I0)
        for k in ref:
            np.testing.assert_array_equal(got[k], ref[k], err_msg="%s %s %s" % (name, tile, k))


def test_split_matches_oracle():
    wl = _workload((11, 19, 37), ((I_, C_), (V_, V_), (C_, V_)), True)
    n, w = oracle.angles.by_name("s4")
    rng = np.random.default_rng(6)
    I0 = (rng.uniform(0.5, 1.5, (len(w), int(np.prod(wl["shape"])))) / (4 * np.pi)).astype(np.float32).astype(np.float64)
    g = _run(wl, n, w, (32, 8, 0), 4, I0)
    p = oracle_problem(wl, n, w)
    o = oracle.run(p, oracle.cfl_dt(p, wl["cfl"]), 4, I0, wl["T"], wl["rho"], wl["v"], wl["sa"], wl["ss"])
    o["wl"] = wl
    assert rel_err(g["E"], o["E"]) <= 1e-5
    errF = field_err({"F": flux_magnitude(g["F"])}, {"F": flux_magnitude(o["F"]), "E": o["E"]}, "F", wl)
    assert errF <= 1e-5
    assert rel_err(g["T"], o["T"]) <= 1e-5
    assert rel_err(g["I"], o["I"]) <= 1e-4


def test_split_tile_in_graph_and_autotune():
    # rt_run captures the three launches of the split path in one graph;
    # the autotuner times the split tiles beside the fused ones
    wl = _workload((16, 16, 32), ((P_, P_), (P_, P_), (P_, P_)), True)
    n, w = oracle.angles.by_name("s4")
    I0 = np.full((len(w), int(np.prod(wl["shape"]))), 1.0 / (4 * np.pi))
    ctx = gpu_context(wl, n, w, "fp32")
    ctx.set_intensity(I0)
    ctx.set_material(wl["rho"], wl["T"], wl["v"], wl["sa"], wl["ss"])
    times = ctx.autotune(2)
    assert {t[:3] for t in times} >= set(SPLIT_TILES)
    ctx.set_tile(32, 8, 0)
    ctx.run(0.0, 4)
    ctx.sync()
    E_graph = ctx.moments()[0]
    ctx.close()
    ref = _run(wl, n, w, (16, 8, 4), 4, I0)
    np.testing.assert_array_equal(E_graph, ref["E"])
