"""Child process of test_gpu_bounds.py: steps a set of float-intensity
problems with the index-checking library (RT_BOUNDS_CHECK), through every
compiled tile shape of each (the autotuner's trials), the persistent batch
kernel's three tile sets and the allocation-free step.  Any out-of-range
shared- or global-memory index of the per-tile code counts as a step
failure, which rt_sync reports as an error; the child prints OK only when
none occurred."""
import ctypes
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import paper_1403_6126_gb300 as rt  # noqa: E402
from paper_1403_6126_gb300 import build as rtbuild  # noqa: E402
from paper_1403_6126_gb300 import workloads as wlmod  # noqa: E402

rt.LIB_PATH = rtbuild.build(check=True)

import oracle  # noqa: E402
from _helpers import gpu_context, initial_state  # noqa: E402


def problems():
    out = []
    wl = wlmod.slab1d(n=37, M=7, steps=0)            # ragged 1-D tile, padding angles
    wl["hold_T"] = False
    out.append(("slab1d 37 x 7", wl))
    wl = wlmod.slab1d(n=301, M=8, steps=0)
    wl["v"] = np.zeros_like(wl["v"])
    wl["v"][0] = 0.05 * wl["C"]                        # velocity terms on
    out.append(("slab1d 301 x 8, moving", wl))
    out.append(("shadow2d 33 x 17 s4", wlmod.shadow2d(nx=33, ny=17, angles="s4", steps=0)))
    out.append(("box2d 45 s6", wlmod.box2d(n=45, angles="s6", steps=0)))
    out.append(("box3d 13 s4", wlmod.box3d(n=13, angles="s4", steps=0)))
    wl = wlmod.box3d(n=11, angles="s10", steps=0)      # 120 angles: the table in shared memory
    out.append(("box3d 11 s10", wl))
    wl = wlmod.box3d(n=19, angles="s2", steps=0)       # open faces on two axes
    wl["bc"] = ((1, 2), (2, 1), (0, 0))
    out.append(("box3d 19 s2, vacuum/copy faces", wl))
    return [(name, wlmod.rounded_to_float32(w)) for name, w in out]


def make(wl):
    n, w = oracle.angles.by_name(wl["angles"])
    n, w = np.ascontiguousarray(n), np.ascontiguousarray(w)
    ctx = gpu_context(wl, n, w, "fp32")
    ctx.set_intensity(initial_state(wl, len(w), "fp32"))
    ctx.set_material(wl["rho"], wl["T"], wl["v"], wl["sa"], wl["ss"])
    return ctx, n, w


def main():
    probs = problems()
    for name, wl in probs:
        ctx, _, _ = make(wl)
        ctx.autotune(2)          # two steps on every compiled tile shape
        ctx.run(0.0, 3)
        ctx.sync()
        ctx.close()
        print("checked", name, flush=True)
    # the persistent batch kernel, every tile set
    members = [make(wl)[0] for _, wl in probs]
    b = rt.rt_batch_create(None)
    for c in members:
        rt.rt_batch_add(b, c.ctx)
    rt.rt_batch_autotune(b, 2)
    rt.rt_batch_step(b, 3)
    for c in members:
        c.sync()
    rt.rt_batch_destroy(b)
    for c in members:
        c.close()
    print("checked batch", flush=True)
    # the allocation-free step (cell centers formed in the kernel)
    import torch
    wl = dict(probs[4][1])
    n, w = oracle.angles.by_name(wl["angles"])
    n, w = np.ascontiguousarray(n), np.ascontiguousarray(w)
    N, M = int(np.prod(wl["shape"])), len(w)
    Q = (M + 3) // 4
    dev = torch.device("cuda", 0)
    I0 = np.zeros((4 * Q, N), dtype=np.float32)
    I0[:M] = initial_state(wl, M, "fp32")
    f32 = lambda x: torch.tensor(np.asarray(x, dtype=np.float32).reshape(-1), device=dev)
    I = [torch.tensor(np.ascontiguousarray(I0.reshape(Q, 4, N).transpose(0, 2, 1)).reshape(-1), device=dev),
         torch.zeros(4 * Q * N, dtype=torch.float32, device=dev)]
    E = 4.0 * np.pi * (w[:, None] * I0[:M].astype(np.float64)).sum(0)
    mom = [torch.zeros(10 * N, dtype=torch.float64, device=dev), torch.zeros(10 * N, dtype=torch.float64, device=dev)]
    mom[0][:N] = torch.tensor(E, device=dev)
    rho, sa, ss, v = f32(wl["rho"]), f32(wl["sa"]), f32(wl["ss"]), f32(wl["v"])
    T = torch.tensor(np.asarray(wl["T"], dtype=np.float64), device=dev)
    dE = torch.zeros(N, dtype=torch.float64, device=dev)
    dM = torch.zeros(3 * N, dtype=torch.float64, device=dev)
    g = rt.rt_grid()
    g.dim = wl["dim"]
    nz, ny, nx = wl["shape"]
    for d, nd in enumerate((nx, ny, nz)):
        g.n[d] = nd
        g.lo[d], g.hi[d] = wl["lo"][d], wl["hi"][d]
        g.bc[d][0], g.bc[d][1] = wl["bc"][d]
    a = rt.rt_angles()
    a.m = M
    a.n = n.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    a.w = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    o = rt.rt_options_default()
    o.precision = rt.RT_FP32
    o.cfl, o.gamma, o.r_ideal = wl["cfl"], wl["gamma"], wl["R"]
    o.hold_T, o.estimate_v = int(wl["hold_T"]), int(wl["estimate_v"])
    inflow = np.zeros((3, 2, M))
    dt = wl["cfl"] * (1.0 / wl["shape"][2]) / wl["C"]
    for call in range(2):
        f = rt.rt_noalloc_fields()
        f.I_in, f.I_out = I[call % 2].data_ptr(), I[(call + 1) % 2].data_ptr()
        f.rho, f.sigma_a, f.sigma_s, f.v = rho.data_ptr(), sa.data_ptr(), ss.data_ptr(), v.data_ptr()
        f.T = T.data_ptr()
        f.mom_in, f.mom_out = mom[call % 2].data_ptr(), mom[(call + 1) % 2].data_ptr()
        f.dE_gas, f.dMom = dE.data_ptr(), dM.data_ptr()
        f.inflow = inflow.ctypes.data
        failures = rt.rt_step_noalloc(g, a, wl["C"], wl["P"], o, dt, f)
        assert failures == 0, failures
    print("checked noalloc", flush=True)
    print("OK", flush=True)


if __name__ == "__main__":
    main()
