"""Shared test helpers: run one workload through the GPU library and through
the CPU oracle on the same inputs, and compare them."""
import numpy as np

import oracle
from paper_1403_6126_gb300 import workloads as wlmod


def oracle_problem(wl, n, w, dense=False):
    inflow = {}
    for face, rule in wl["inflow"].items():
        inflow[face] = wlmod.inflow_values(rule, n)
    dx = tuple((wl["hi"][d] - wl["lo"][d]) / (wl["shape"][2 - d]) for d in range(3))
    return oracle.Problem(wl["shape"], dx, n, w, C=wl["C"], P=wl["P"], dim=wl["dim"], bc=wl["bc"],
                          inflow=inflow, gamma=wl["gamma"], R=wl["R"], hold_T=wl["hold_T"],
                          estimate_v=wl["estimate_v"], dense=dense)


def gpu_context(wl, n, w, precision, inflow=True, **kw):
    """A context for the workload; with inflow=False its inflow faces are
    left without incoming intensities (zero until set)."""
    import paper_1403_6126_gb300 as rt
    prec = {"fp64": rt.RT_FP64, "fp32": rt.RT_FP32, "bf16": rt.RT_BF16}[precision]
    ctx = rt.Context(wl["shape"], n, w, wl["C"], wl["P"], dim=wl["dim"], lo=wl["lo"], hi=wl["hi"], bc=wl["bc"],
                     precision=prec, cfl=wl["cfl"], gamma=wl["gamma"], r_ideal=wl["R"], hold_T=wl["hold_T"],
                     estimate_v=wl["estimate_v"], **kw)
    for (axis, side), rule in (wl["inflow"].items() if inflow else ()):
        ctx.set_inflow(axis, side, wlmod.inflow_values(rule, n))
    return ctx


def initial_state(wl, M, precision):
    I0 = wlmod.initial_intensity(wl, M)
    if precision == "fp32":
        I0 = I0.astype(np.float32).astype(np.float64)
    return I0


def run_both(wl, nsteps, precision, n=None, w=None, threads=None):
    """Runs nsteps on the GPU and in the oracle from identical inputs.
    Returns (gpu dict, oracle dict); the oracle dict also carries the
    workload under "wl" for the error scales."""
    if n is None:
        n, w = oracle.angles.by_name(wl["angles"])
    if precision == "fp32":
        wl = wlmod.rounded_to_float32(wl)
    M = len(w)
    I0 = initial_state(wl, M, precision)
    ctx = gpu_context(wl, n, w, precision)
    ctx.set_intensity(I0)
    ctx.set_material(wl["rho"], wl["T"], wl["v"], wl["sa"], wl["ss"])
    p = oracle_problem(wl, n, w)
    dt = oracle.cfl_dt(p, wl["cfl"])
    assert abs(dt - ctx.cfl_dt()) <= 1e-15 * dt
    for _ in range(nsteps):
        ctx.step(dt)
    ctx.sync()
    E, F, P = ctx.moments()
    dE, dM, T = ctx.sources()
    g = dict(I=ctx.intensity(), E=E, F=F, P=P, dEgas=dE, dMom=dM, T=T)
    ctx.close()
    if threads:
        oracle.set_threads(threads)
    o = oracle.run(p, dt, nsteps, I0, wl["T"], wl["rho"], wl["v"], wl["sa"], wl["ss"])
    o["wl"] = wl
    return g, o


def rel_err(a, b):
    """Norm-relative error max|a - b| / max|b| (0 when both vanish)."""
    a, b = np.asarray(a), np.asarray(b)
    scale = np.abs(b).max()
    if scale == 0:
        return float(np.abs(a).max())
    return float(np.abs(a - b).max() / scale)


def natural_scale(o, key, wl):
    """Magnitude a field would have if it were not small by cancellation:
    the radiation energy scale for E, F, P (|F_r| <= E_r), (P/C) E for the
    momentum source, P E for the gas energy source, the field itself for
    I and T."""
    if key in ("I", "T"):
        return float(np.abs(o[key]).max())
    E0 = float(np.abs(o["E"]).max())
    return {"E": E0, "F": E0, "P": E0, "dMom": wl["P"] / wl["C"] * E0, "dEgas": wl["P"] * E0}[key]


def field_err(g, o, key, wl, floor=1e-3):
    """max|g - o| / max(max|o|, floor * natural scale): norm-relative, except
    for a field that is pure round-off (F with isotropic I, the momentum
    source with v = 0), which is measured against 1e-3 of its natural
    scale instead of against its own noise."""
    a, b = np.asarray(g[key]), np.asarray(o[key])
    scale = max(float(np.abs(b).max()), floor * natural_scale(o, key, wl))
    if scale == 0:
        return float(np.abs(a).max())
    return float(np.abs(a - b).max() / scale)


def flux_magnitude(F):
    return np.sqrt((np.asarray(F) ** 2).sum(axis=0))
