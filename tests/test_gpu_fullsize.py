"""Parity at the full sizes the benchmark times, in the launch shapes it uses.

3-D box, 128^3 cells x 80 angles, float intensities: the GPU takes two steps
from a seeded random intensity field (so the limiter and the alpha blend are
active everywhere).  The oracle then recomputes sampled cells on 9^3 windows
cut around each one, with the full grid's periodic wrap.  A step reads two
cells along each axis, so two steps move information at most four cells: the
centre of a window sees exactly the inputs it sees in the full grid, whatever
happens at the window's own edges.  The samples include tile corners and the
periodic seams.

Batched workload, 512 uneven problems in one persistent launch per step: a
sample of members (the largest 1-D and 2-D ones among them) is run whole by
the oracle.
"""
import numpy as np
import pytest

import oracle
import paper_1403_6126_gb300 as rt
from paper_1403_6126_gb300 import workloads as wlmod

from _helpers import field_err, flux_magnitude, gpu_context, initial_state, oracle_problem, rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-5          # mixed-precision bound on E_r and |F_r|
STEPS = 2
RAD = 2 * STEPS     # window radius: two cells of stencil per step


def _window(n, centre):
    """Grid indices (z, y, x) of the (2 RAD + 1)^3 window around centre
    (x, y, z) in a periodic n^3 grid."""
    x, y, z = centre
    off = np.arange(-RAD, RAD + 1)
    return (z + off) % n, (y + off) % n, (x + off) % n


def test_box3d_full_size_sampled_cells():
    n = 128
    wl = wlmod.rounded_to_float32(wlmod.box3d(n=n, angles="s8", steps=STEPS))
    nn, w = oracle.angles.by_name("s8")
    M, N = len(w), n ** 3
    rng = np.random.default_rng(1403)
    I0 = (1.0 + rng.uniform(-0.5, 0.5, size=(M, N)).astype(np.float32)) / np.float32(4 * np.pi)
    I0 = I0.astype(np.float32).astype(np.float64)

    ctx = gpu_context(wl, nn, w, "fp32")
    assert ctx.tile() == (8, 8, 4)           # the shape the benchmark times
    ctx.set_intensity(I0)
    ctx.set_material(wl["rho"], wl["T"], wl["v"], wl["sa"], wl["ss"])
    dt = ctx.cfl_dt()
    for _ in range(STEPS):
        ctx.step(dt)
    ctx.sync()
    E, F, P = ctx.moments()
    dE, dM, T = ctx.sources()
    I = ctx.intensity()
    ctx.close()

    picks = [(0, 0, 0), (n - 1, n - 1, n - 1), (7, 7, 3), (8, 8, 4), (15, 7, 3), (16, 8, 4), (n - 1, 0, 64),
             (64, 64, 64), (31, 127, 0), (0, 64, 127)]
    while len(picks) < 24:
        picks.append(tuple(int(v) for v in rng.integers(0, n, 3)))

    side = 2 * RAD + 1
    wwl = dict(wl, shape=(side, side, side), hi=(side / n, side / n, side / n))
    p = oracle_problem(wwl, nn, w)
    assert abs(oracle.cfl_dt(p, wl["cfl"]) - dt) <= 1e-15 * dt
    ctr = RAD + side * (RAD + side * RAD)
    I3 = I0.reshape(M, n, n, n)
    got = {k: [] for k in ("I", "E", "F", "T", "dEgas", "dMom")}
    ref = {k: [] for k in got}
    for (x, y, z) in picks:
        zi, yi, xi = _window(n, (x, y, z))
        cut = lambda f: np.asarray(f).reshape(n, n, n)[np.ix_(zi, yi, xi)].reshape(-1)
        Iw = I3[:, zi][:, :, yi][:, :, :, xi].reshape(M, -1)
        vw = np.stack([cut(wl["v"][d]) for d in range(3)])
        Tw = cut(wl["T"])
        out = None
        for _ in range(STEPS):
            out = oracle.step(p, dt, Iw, Tw, cut(wl["rho"]), vw, cut(wl["sa"]), cut(wl["ss"]))
            assert out["failures"] == 0
            Iw, Tw = out["I"], out["T"]
        c = x + n * (y + n * z)
        got["I"].append(I[:, c]); ref["I"].append(out["I"][:, ctr])
        got["E"].append(E[c]); ref["E"].append(out["E"][ctr])
        got["F"].append(F[:, c]); ref["F"].append(out["F"][:, ctr])
        got["T"].append(T[c]); ref["T"].append(out["T"][ctr])
        got["dEgas"].append(dE[c]); ref["dEgas"].append(out["dEgas"][ctr])
        got["dMom"].append(dM[:, c]); ref["dMom"].append(out["dMom"][:, ctr])
    got = {k: np.array(v) for k, v in got.items()}
    ref = {k: np.array(v) for k, v in ref.items()}
    # pointwise on E_r and |F_r| at every sampled cell
    assert np.max(np.abs(got["E"] - ref["E"]) / np.abs(ref["E"])) <= TOL
    fg, fo = flux_magnitude(got["F"].T), flux_magnitude(ref["F"].T)
    assert np.max(np.abs(fg - fo) / np.maximum(fo, 1e-3 * np.abs(ref["E"]))) <= TOL
    # every intensity of every sampled cell, the temperature and the sources
    for i in range(len(picks)):
        assert rel_err(got["I"][i], ref["I"][i]) <= TOL, (picks[i], rel_err(got["I"][i], ref["I"][i]))
    assert rel_err(got["T"], ref["T"]) <= TOL
    ref["wl"] = wl
    for k in ("dEgas", "dMom"):
        assert field_err(got, ref, k, wl) <= 1e-4, (k, field_err(got, ref, k, wl))


def test_batched_full_size_sampled_problems():
    import torch
    wls = wlmod.batched()
    assert len(wls) == 512
    stream = torch.cuda.Stream()
    ctxs = []
    for wl in wls:
        nn, w = oracle.angles.by_name(wl["angles"])
        c = gpu_context(wl, nn, w, "fp32", stream=stream.cuda_stream)
        c.set_intensity(initial_state(wl, len(w), "fp32"))
        c.set_material(wl["rho"], wl["T"], wl["v"], wl["sa"], wl["ss"])
        ctxs.append(c)
    b = rt.rt_batch_create(stream.cuda_stream)
    for c in ctxs:
        rt.rt_batch_add(b, c.ctx)
    nsteps = 3
    rt.rt_batch_step(b, nsteps)
    torch.cuda.synchronize()
    rt.rt_batch_destroy(b)

    size = [int(np.prod(wl["shape"])) * len(oracle.angles.by_name(wl["angles"])[1]) for wl in wls]
    one_d = [i for i, wl in enumerate(wls) if wl["dim"] == 1]
    two_d = [i for i, wl in enumerate(wls) if wl["dim"] == 2]
    sample = {max(one_d, key=lambda i: size[i]), max(two_d, key=lambda i: size[i]),
              min(one_d, key=lambda i: size[i]), min(two_d, key=lambda i: size[i])}
    sample |= set(np.random.default_rng(7).choice(len(wls), 6, replace=False).tolist())
    for i in sorted(sample):
        wl = wlmod.rounded_to_float32(wls[i])
        nn, w = oracle.angles.by_name(wl["angles"])
        c = ctxs[i]
        c.sync()
        E, F, _ = c.moments()
        p = oracle_problem(wl, nn, w)
        o = oracle.run(p, c.cfl_dt(), nsteps, initial_state(wl, len(w), "fp32"), wl["T"], wl["rho"], wl["v"],
                       wl["sa"], wl["ss"])
        assert rel_err(E, o["E"]) <= TOL, (i, rel_err(E, o["E"]))
        errF = field_err({"F": flux_magnitude(F)}, {"F": flux_magnitude(o["F"]), "E": o["E"]}, "F", wl)
        assert errF <= TOL, (i, errF)
    for c in ctxs:
        c.close()


def test_largest_grid_sampled_cells():
    # The largest grid the ABI accepts (just under 2^28 cells), 9 angles (an
    # odd count: the padded pair too): the intensity array holds 2.4e9
    # values, past 32-bit indexing.  Fields are
    # drawn on the device and passed as device pointers; one step from the
    # isotropic equilibrium of a non-uniform temperature; sampled cells
    # (including the last one) recomputed by the oracle on 5^3 windows.
    import torch
    nx, ny, nz = 1023, 512, 512
    N = nx * ny * nz
    M = 9
    assert N < 2 ** 28 and M * N > 2 ** 31
    dev = torch.device("cuda", 0)
    gen = torch.Generator(device=dev).manual_seed(1403)
    u = lambda: torch.rand(N, generator=gen, device=dev, dtype=torch.float64)
    C = 10.0
    f = dict(rho=1.0 + 0.5 * u(), T=1.0 + 0.2 * u(), sa=10.0 ** (2.0 * u()), ss=10.0 ** (2.0 * u()))
    f["v"] = (0.05 * C) * (2.0 * torch.rand(3 * N, generator=gen, device=dev, dtype=torch.float64) - 1.0)
    nn = np.random.default_rng(9).normal(size=(M, 3))
    nn /= np.linalg.norm(nn, axis=1, keepdims=True)
    w = np.full(M, 1.0 / M)
    wl = dict(name="largest", shape=(nz, ny, nx), dim=3, lo=(0.0, 0.0, 0.0), hi=(nx / 512.0, 1.0, 1.0),
              bc=((0, 0), (0, 0), (0, 0)), angles=None, C=C, P=1.0, gamma=5.0 / 3.0, R=1.0, cfl=0.4,
              hold_T=False, estimate_v=True, inflow={})
    ctx = gpu_context(wl, nn, w, "fp32", device_ptrs=True)
    ctx.set_material(f["rho"], f["T"], f["v"], f["sa"], f["ss"])
    ctx.set_intensity(None)                      # T^4 / (4 pi) of each cell
    picks = [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (nx - 1, 0, nz // 2), (511, 255, 300)]
    rng = np.random.default_rng(4)
    while len(picks) < 12:
        picks.append((int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz))))
    rad, side = 2, 5
    off = np.arange(-rad, rad + 1)
    wins = []
    for (x, y, z) in picks:
        zi, yi, xi = (z + off) % nz, (y + off) % ny, (x + off) % nx
        idx = (xi[None, None, :] + nx * (yi[None, :, None] + ny * zi[:, None, None])).reshape(-1)
        wins.append(torch.as_tensor(idx, device=dev))
    # inputs of each window as the device holds them (float-rounded fields)
    I0 = torch.empty(M * N, dtype=torch.float64, device=dev)
    rt.rt_get_intensity(ctx.ctx, I0)
    torch.cuda.synchronize()
    I0 = I0.view(M, N)
    host = []
    for idx in wins:
        r = lambda t: t[idx].to(torch.float32).double().cpu().numpy()
        host.append(dict(I=I0[:, idx].cpu().numpy(), T=f["T"][idx].cpu().numpy(), rho=r(f["rho"]), sa=r(f["sa"]),
                         ss=r(f["ss"]), v=np.stack([r(f["v"][d * N:(d + 1) * N]) for d in range(3)])))
    ctx._keep = None            # the library holds its own copies once the stream is done
    del I0, f
    torch.cuda.empty_cache()
    dt = ctx.cfl_dt()
    ctx.step(dt)
    ctx.sync()
    I1 = torch.empty(M * N, dtype=torch.float64, device=dev)
    rt.rt_get_intensity(ctx.ctx, I1)
    E = torch.empty(N, dtype=torch.float64, device=dev)
    Fm = torch.empty(3 * N, dtype=torch.float64, device=dev)
    Pm = torch.empty(6 * N, dtype=torch.float64, device=dev)
    rt.rt_moments(ctx.ctx, E, Fm, Pm)
    Tn = torch.empty(N, dtype=torch.float64, device=dev)
    dE = torch.empty(N, dtype=torch.float64, device=dev)
    dM = torch.empty(3 * N, dtype=torch.float64, device=dev)
    rt.rt_sources(ctx.ctx, dE, dM, Tn)
    torch.cuda.synchronize()
    ctx.close()
    wwl = dict(wl, shape=(side, side, side), hi=(side / 512.0, side / 512.0, side / 512.0))
    p = oracle_problem(wwl, nn, w)
    assert abs(oracle.cfl_dt(p, wl["cfl"]) - dt) <= 1e-15 * dt
    ctr = rad + side * (rad + side * rad)
    for (x, y, z), h in zip(picks, host):
        out = oracle.step(p, dt, h["I"], h["T"], h["rho"], h["v"], h["sa"], h["ss"])
        assert out["failures"] == 0
        c = x + nx * (y + ny * z)
        gI = I1.view(M, N)[:, c].cpu().numpy()
        assert rel_err(gI, out["I"][:, ctr]) <= 1e-4, (x, y, z)
        assert abs(E[c].item() - out["E"][ctr]) <= TOL * abs(out["E"][ctr]), (x, y, z)
        gF = np.array([Fm[d * N + c].item() for d in range(3)])
        assert np.linalg.norm(gF - out["F"][:, ctr]) <= TOL * max(np.linalg.norm(out["F"][:, ctr]),
                                                                 1e-3 * out["E"][ctr]), (x, y, z)
        assert abs(Tn[c].item() - out["T"][ctr]) <= TOL * out["T"][ctr], (x, y, z)


@pytest.mark.parametrize("index,nsteps", [(247, 100), (483, 190)])
def test_float_newton_settles_near_the_root(index, nsteps):
    # Requests 247 (192^3 x 80) and 483 (160^3 x 24) of the 500-request
    # serving stream: at steps 98 and 187 the float T^4 Newton of one cell
    # cycled between two iterates two float ulps of T apart, and a stopping
    # test of 2e-7 T (1.7 ulps) was never met.  With the test at 1e-6 T the
    # cell settles, and the double step that follows gives T to ~1e-12: no
    # failure, T finite and positive.
    wl = wlmod.serving_request(index)
    n, w = oracle.angles.by_name(wl["angles"])
    ctx = gpu_context(wl, n, w, "fp32")
    ctx.set_material(wl["rho"], wl["T"], wl["v"], wl["sa"], wl["ss"])
    ctx.set_intensity(None)
    for _ in range(nsteps // 10):
        ctx.run(0.0, 10)
        ctx.sync()                     # raises RT_E_NONFINITE on a Newton failure
    T = ctx.sources()[2]
    ctx.close()
    assert np.all(np.isfinite(T)) and T.min() > 0
