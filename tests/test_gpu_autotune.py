"""Tile autotuners: rt_autotune (one context) and rt_batch_autotune (the
persistent multi-problem kernel).  Both time their candidates on the real
problem, keep the fastest, and leave the state bitwise as it was.  With
float intensities the results after tuning are bitwise those of an untuned
run (the tile changes speed, never arithmetic); the double-precision kernel
lets the compiler fuse multiply-adds per tile shape, so there they agree to
a few units in the last place."""
import numpy as np
import pytest
import torch

import oracle
import paper_1403_6126_gb300 as rt
from paper_1403_6126_gb300 import workloads as wlmod

from _helpers import field_err, gpu_context, initial_state

pytestmark = pytest.mark.gpu


def _snapshot(ctx):
    E, F, P = ctx.moments()
    dE, dM, T = ctx.sources()
    return dict(I=ctx.intensity(), E=E, F=F, P=P, dEgas=dE, dMom=dM, T=T)


def _make(wl, precision, stream=None):
    n, w = oracle.angles.by_name(wl["angles"])
    ctx = gpu_context(wl, n, w, precision, stream=stream)
    ctx.set_intensity(initial_state(wl, len(w), precision))
    ctx.set_material(wl["rho"], wl["T"], wl["v"], wl["sa"], wl["ss"])
    return ctx


@pytest.mark.parametrize("name,kw,precision", [
    ("box3d", dict(n=20, angles="s4"), "fp32"),
    ("box3d", dict(n=12, angles="s2"), "fp64"),
    ("shadow2d", dict(nx=70, ny=36, angles="s4"), "fp32"),
    ("slab1d", dict(n=700, M=16), "fp32"),
])
def test_autotune_keeps_state_and_picks_fastest(name, kw, precision):
    wl = wlmod.by_name(name, steps=0, **kw)
    ctx = _make(wl, precision)
    ctx.step(0.0)                      # non-trivial sources and moments to preserve
    ctx.sync()
    before = _snapshot(ctx)
    times = ctx.autotune(2)
    assert len(times) >= 2 and all(t[3] > 0 for t in times)
    best = min(times, key=lambda t: t[3])
    assert ctx.tile() == best[:3]
    ctx.sync()
    after = _snapshot(ctx)
    for k in before:
        np.testing.assert_array_equal(after[k], before[k], err_msg=k)
    # the next steps are bitwise those of a context that was never tuned
    ref = _make(wl, precision)
    ref.step(0.0)
    for c in (ctx, ref):
        c.step(0.0)
        c.step(0.0)
        c.sync()
    a, b = _snapshot(ctx), _snapshot(ref)
    for k in a:
        if precision == "fp32":
            np.testing.assert_array_equal(a[k], b[k], err_msg=k)
        else:
            assert field_err(a, b, k, wl) <= 1e-13, (k, field_err(a, b, k, wl))
    ctx.close()
    ref.close()


def test_batch_autotune_keeps_state_and_results():
    stream = torch.cuda.Stream()
    h = stream.cuda_stream
    probs = []
    for n, M in ((64, 8), (700, 24), (37, 48), (3000, 16)):
        wl = wlmod.slab1d(n=n, M=M, steps=0)
        wl["hold_T"] = False
        probs.append(wl)
    for nx, ny, ang in ((40, 24, "s2"), (65, 33, "s4"), (130, 97, "s6")):
        probs.append(wlmod.shadow2d(nx=nx, ny=ny, angles=ang, steps=0))
    members = [_make(wl, "fp32", h) for wl in probs]
    b = rt.rt_batch_create(h)
    for c in members:
        rt.rt_batch_add(b, c.ctx)
    rt.rt_batch_step(b, 1)
    for c in members:
        c.sync()
    before = [_snapshot(c) for c in members]
    ms, chosen = rt.rt_batch_autotune(b, 2)
    assert len(ms) == 3 and all(t > 0 for t in ms)
    assert chosen == int(np.argmin(ms))
    for c, s in zip(members, before):
        c.sync()
        after = _snapshot(c)
        for k in s:
            np.testing.assert_array_equal(after[k], s[k], err_msg=k)
    rt.rt_batch_step(b, 3)
    for c in members:
        c.sync()
    got = [_snapshot(c) for c in members]
    rt.rt_batch_destroy(b)
    for wl, g in zip(probs, got):
        alone = _make(wl, "fp32", h)
        for _ in range(4):
            alone.step(0.0)
        alone.sync()
        ref = _snapshot(alone)
        alone.close()
        for k in ref:
            np.testing.assert_array_equal(g[k], ref[k], err_msg=k)
    for c in members:
        c.close()
