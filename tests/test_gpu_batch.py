"""Many problems in one persistent launch per step: each problem's result is
bitwise what it gets when stepped alone, and matches the FP64 oracle within
the mixed-precision bound."""
import numpy as np
import pytest
import torch

import oracle
import paper_1403_6126_gb300 as rt
from paper_1403_6126_gb300 import workloads as wlmod

from _helpers import field_err, flux_magnitude, gpu_context, initial_state, oracle_problem, rel_err

pytestmark = pytest.mark.gpu


def _mixed_problems(with_velocity=False):
    rng = np.random.default_rng(21)
    probs = []
    for n, M in ((64, 8), (700, 24), (37, 48), (1500, 16)):
        wl = wlmod.slab1d(n=n, M=M, seed=int(rng.integers(1000)), steps=0)
        wl["hold_T"] = False
        probs.append(wl)
    for nx, ny, ang in ((40, 24, "s2"), (65, 33, "s4"), (32, 32, "s6"), (100, 17, "s4")):
        probs.append(wlmod.shadow2d(nx=nx, ny=ny, angles=ang, steps=0))
    if with_velocity:
        probs.append(wlmod.box3d(n=12, angles="s4", steps=0))
    return [wlmod.rounded_to_float32(w) for w in probs]


def _make(wl, stream):
    n, w = oracle.angles.by_name(wl["angles"])
    ctx = gpu_context(wl, n, w, "fp32", stream=stream)
    ctx.set_intensity(initial_state(wl, len(w), "fp32"))
    ctx.set_material(wl["rho"], wl["T"], wl["v"], wl["sa"], wl["ss"])
    return ctx


def _outputs(ctx):
    E, F, P = ctx.moments()
    dE, dM, T = ctx.sources()
    return dict(I=ctx.intensity(), E=E, F=F, P=P, dEgas=dE, dMom=dM, T=T)


@pytest.mark.parametrize("use_graph,with_velocity", [(True, False), (False, False), (True, True)])
def test_batch_equals_each_problem_alone(use_graph, with_velocity):
    # Without velocity terms the batch runs the same per-tile code as the
    # single-problem kernel: bitwise equal.  A member with velocity switches
    # the whole batch to the velocity-capable code, which computes the same
    # arithmetic with extra zero terms for the members without velocity:
    # bitwise equal too (every sum both variants share is an explicit fused
    # multiply-add, so the compiler cannot round them differently).
    stream = torch.cuda.Stream() if use_graph else None
    handle = stream.cuda_stream if use_graph else None
    probs = _mixed_problems(with_velocity)
    nsteps = 5
    batch = rt.rt_batch_create(handle)
    members = [_make(wl, handle) for wl in probs]
    for c in members:
        rt.rt_batch_add(batch, c.ctx)
    assert rt.rt_batch_size(batch) == len(probs)
    rt.rt_batch_step(batch, 2)
    rt.rt_batch_step(batch, nsteps - 2)   # odd then even counts: parity bookkeeping
    for c in members:
        c.sync()
    with pytest.raises(rt.RTError) as e:
        members[0].step(0.0)
    assert e.value.status == rt.RT_E_STATE
    got = [_outputs(c) for c in members]
    for wl, g in zip(probs, got):
        alone = _make(wl, handle)
        for _ in range(nsteps):
            alone.step(0.0)
        alone.sync()
        ref = _outputs(alone)
        alone.close()
        for k in list(ref):
            np.testing.assert_array_equal(g[k], ref[k], err_msg=k)
    rt.rt_batch_destroy(batch)
    for c in members:
        c.close()


def test_batch_matches_oracle():
    stream = torch.cuda.Stream()
    probs = _mixed_problems(True)[::2]
    batch = rt.rt_batch_create(stream.cuda_stream)
    members = [_make(wl, stream.cuda_stream) for wl in probs]
    for c in members:
        rt.rt_batch_add(batch, c.ctx)
    rt.rt_batch_step(batch, 4)
    for wl, c in zip(probs, members):
        c.sync()
        g = _outputs(c)
        n, w = oracle.angles.by_name(wl["angles"])
        p = oracle_problem(wl, n, w)
        o = oracle.run(p, oracle.cfl_dt(p, wl["cfl"]), 4, initial_state(wl, len(w), "fp32"), wl["T"], wl["rho"],
                       wl["v"], wl["sa"], wl["ss"])
        assert rel_err(g["E"], o["E"]) <= 1e-5
        errF = field_err({"F": flux_magnitude(g["F"])}, {"F": flux_magnitude(o["F"]), "E": o["E"]}, "F", wl)
        assert errF <= 1e-5
    rt.rt_batch_destroy(batch)
    for c in members:
        c.close()


def test_batch_membership_changes():
    stream = torch.cuda.Stream()
    probs = _mixed_problems()[:4]
    batch = rt.rt_batch_create(stream.cuda_stream)
    members = [_make(wl, stream.cuda_stream) for wl in probs]
    for c in members[:2]:
        rt.rt_batch_add(batch, c.ctx)
    rt.rt_batch_step(batch, 3)
    rt.rt_batch_remove(batch, members[0].ctx)
    rt.rt_batch_add(batch, members[2].ctx)   # joins with a different buffer parity
    rt.rt_batch_step(batch, 2)
    rt.rt_batch_destroy(batch)
    # member 1: 5 steps, member 2: 2 steps, member 0: 3 steps
    for idx, steps in ((0, 3), (1, 5), (2, 2)):
        members[idx].sync()
        g = _outputs(members[idx])
        alone = _make(probs[idx], stream.cuda_stream)
        for _ in range(steps):
            alone.step(0.0)
        alone.sync()
        ref = _outputs(alone)
        alone.close()
        np.testing.assert_array_equal(g["I"], ref["I"])
        np.testing.assert_array_equal(g["T"], ref["T"])
    for c in members:
        c.close()
