"""The allocation-free step (rt_step_noalloc) against the regular entry point.

rt_step_noalloc is for callers that cannot allocate device memory (a memory
pool owned by another framework, a fixed budget, a plugin limited to the
buffers it is given): they pass every field as a device buffer, the tables
travel in the launch parameters and the library uses only a fixed scratch
word.  Here the caller's buffers are torch tensors; the same problem also
runs through rt_create / rt_step, and two consecutive steps of each must be
bitwise equal (both run the same per-tile code with the same rounding).
The cases cover 1-D, 2-D and 3-D launch shapes, and a grid with more tiles
than resident CTAs, so that each CTA walks several tiles.  The file sorts
last so that a run stopping at the first failure has run every other test
first.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1403_6126_gb300 as rt
from paper_1403_6126_gb300 import build as rtbuild
from paper_1403_6126_gb300 import workloads as wlmod

from _helpers import gpu_context, initial_state

pytestmark = pytest.mark.gpu


def _structs(wl, n, w):
    g = rt.rt_grid()
    g.dim = wl["dim"]
    nz, ny, nx = wl["shape"]
    for d, nd in enumerate((nx, ny, nz)):
        g.n[d] = nd
        g.lo[d], g.hi[d] = wl["lo"][d], wl["hi"][d]
        g.bc[d][0], g.bc[d][1] = wl["bc"][d]
    a = rt.rt_angles()
    a.m = len(w)
    a.n = n.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    a.w = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    o = rt.rt_options_default()
    o.precision = rt.RT_FP32
    o.cfl, o.gamma, o.r_ideal = wl["cfl"], wl["gamma"], wl["R"]
    o.hold_T, o.estimate_v = int(wl["hold_T"]), int(wl["estimate_v"])
    return g, a, o


def to_quads(I, M, N, dev):
    """Angle-major (M, N) values into the float step's layout: ceil(M/4)
    planes of (N, 4), zero padding past M."""
    Q = (M + 3) // 4
    buf = np.zeros((4 * Q, N), dtype=np.float32)
    buf[:M] = np.asarray(I, dtype=np.float32).reshape(M, N)
    return torch.tensor(np.ascontiguousarray(buf.reshape(Q, 4, N).transpose(0, 2, 1)).reshape(-1), device=dev)


def from_quads(t, M, N):
    Q = (M + 3) // 4
    a = t.cpu().numpy().reshape(Q, N, 4).transpose(0, 2, 1).reshape(4 * Q, N)
    return a[:M].astype(np.float64)


CASES = [
    ("box3d", dict(n=12, angles="s4", steps=0)),
    ("shadow2d", dict(nx=40, ny=20, angles="s4", steps=0)),
    ("slab1d", dict(n=700, steps=0)),
    ("box3d", dict(n=64, angles="s4", steps=0)),   # 1024 tiles of 8x8x4: every CTA walks several
]


@pytest.mark.parametrize("name,kw", CASES, ids=["box3d_12", "shadow2d_40x20", "slab1d_700", "box3d_64"])
def test_noalloc_step_equals_rt_step(name, kw):
    rtbuild.build()
    wl = wlmod.rounded_to_float32(wlmod.by_name(name, **kw))
    if name in ("shadow2d", "slab1d"):
        wl["v"] = np.zeros_like(wl["v"])
        wl["v"][0] = 0.05 * wl["C"]     # velocity terms on in every case
        wl["v"] = wl["v"].astype(np.float32).astype(np.float64)
    n, w = oracle.angles.by_name(wl["angles"])
    n, w = np.ascontiguousarray(n), np.ascontiguousarray(w)
    N, M = int(np.prod(wl["shape"])), len(w)

    ctx = gpu_context(wl, n, w, "fp32")
    ctx.set_intensity(initial_state(wl, M, "fp32"))
    ctx.set_material(wl["rho"], wl["T"], wl["v"], wl["sa"], wl["ss"])
    dt = ctx.cfl_dt()

    dev = torch.device("cuda", 0)
    f32 = lambda x: torch.tensor(np.asarray(x, dtype=np.float32).reshape(-1), device=dev)
    I = [to_quads(ctx.intensity(), M, N, dev), torch.empty(4 * ((M + 3) // 4) * N, dtype=torch.float32, device=dev)]
    E, F, P = ctx.moments()
    mom = [torch.tensor(np.concatenate([E[None], F, P]).reshape(-1), device=dev),
           torch.empty(10 * N, dtype=torch.float64, device=dev)]
    rho, sa, ss, v = f32(wl["rho"]), f32(wl["sa"]), f32(wl["ss"]), f32(wl["v"])
    T = torch.tensor(np.asarray(wl["T"], dtype=np.float64), device=dev)
    dE = torch.empty(N, dtype=torch.float64, device=dev)
    dM = torch.empty(3 * N, dtype=torch.float64, device=dev)
    inflow = np.zeros((3, 2, M))
    for (axis, side), rule in wl["inflow"].items():
        inflow[axis, side] = wlmod.inflow_values(rule, n)
    g, a, o = _structs(wl, n, w)

    for call in range(2):
        f = rt.rt_noalloc_fields()
        f.I_in, f.I_out = I[call % 2].data_ptr(), I[(call + 1) % 2].data_ptr()
        f.rho, f.sigma_a, f.sigma_s, f.v = rho.data_ptr(), sa.data_ptr(), ss.data_ptr(), v.data_ptr()
        f.T = T.data_ptr()
        f.mom_in, f.mom_out = mom[call % 2].data_ptr(), mom[(call + 1) % 2].data_ptr()
        f.dE_gas, f.dMom = dE.data_ptr(), dM.data_ptr()
        f.inflow = inflow.ctypes.data
        failures = rt.rt_step_noalloc(g, a, wl["C"], wl["P"], o, dt, f)
        assert failures == 0
        ctx.step(dt)
        ctx.sync()
        Er, Fr, Pr = ctx.moments()
        dEr, dMr, Tr = ctx.sources()
        out = mom[(call + 1) % 2].cpu().numpy().reshape(10, N)
        got = dict(I=from_quads(I[(call + 1) % 2], M, N), E=out[0], F=out[1:4], P=out[4:10],
                   dEgas=dE.cpu().numpy(), dMom=dM.cpu().numpy().reshape(3, N), T=T.cpu().numpy())
        ref = dict(I=ctx.intensity(), E=Er, F=Fr, P=Pr, dEgas=dEr, dMom=dMr, T=Tr)
        for k in ("I", "E", "F", "P", "dEgas", "dMom", "T"):
            assert np.array_equal(got[k], ref[k]), (call, k, float(np.abs(got[k] - ref[k]).max()))
        # the padding angles of the layout stay zero
        Q = (M + 3) // 4
        pad = I[(call + 1) % 2].cpu().numpy().reshape(Q, N, 4)[Q - 1, :, M - 4 * (Q - 1):]
        assert not pad.any()
    ctx.close()


def test_noalloc_rejects_oversized_angle_sets():
    rtbuild.build()
    wl = wlmod.slab1d(n=16, steps=0)
    rng = np.random.default_rng(3)
    n = rng.normal(size=(257, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    w = np.full(257, 1.0 / 257)
    g, a, o = _structs(wl, n, w)
    f = rt.rt_noalloc_fields()
    for k, _ in f._fields_:
        setattr(f, k, 256 + 64 * len(k))   # distinct, never dereferenced: the size check comes first
    with pytest.raises(rt.RTError) as e:
        rt.rt_step_noalloc(g, a, wl["C"], wl["P"], o, 1e-3, f)
    assert e.value.status == rt.RT_E_INVALID
    assert "256" in rt.rt_last_error()
