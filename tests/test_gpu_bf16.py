"""bf16 intensity storage (RT_BF16), the measured experiment: intensities
held as bf16 deviations from the cell's mean intensity, float arithmetic.

Against the FP64 oracle the error is bounded by what the format allows: each
step rounds every stored delta_m = I_m / J - 1 by at most 2^-8 |delta_m|, so
after n steps |E - E_oracle| <= n 2^-8 max|delta| E plus the float path's own
~1e-6.  A round trip through rt_set_intensity / rt_get_intensity loses at
most 2^-8 |delta| J per value; checkpoints resume bitwise; batches refuse
bf16 contexts."""
import numpy as np
import pytest

import oracle
import paper_1403_6126_gb300 as rt
from paper_1403_6126_gb300 import workloads as wlmod

from _helpers import gpu_context, initial_state, oracle_problem

pytestmark = pytest.mark.gpu

U = 2.0 ** -8   # largest relative rounding error of a bf16 value


def _deviation(I, w):
    J = (w[:, None] * I).sum(axis=0)
    return np.abs(I / J[None, :] - 1.0).max()


@pytest.mark.parametrize("name,kw,nsteps", [
    ("box3d", dict(n=12, angles="s4"), 6),
    ("shadow2d", dict(nx=40, ny=24, angles="s4"), 6),
    ("slab1d", dict(n=64, M=8), 10),
])
def test_bf16_error_within_format_bound(name, kw, nsteps):
    wl = wlmod.rounded_to_float32(wlmod.by_name(name, steps=0, **kw))
    n, w = oracle.angles.by_name(wl["angles"])
    I0 = initial_state(wl, len(w), "fp32")
    ctx = gpu_context(wl, n, w, "bf16")
    ctx.set_intensity(I0)
    ctx.set_material(wl["rho"], wl["T"], wl["v"], wl["sa"], wl["ss"])
    dt = ctx.cfl_dt()
    for _ in range(nsteps):
        ctx.step(dt)
    ctx.sync()
    E, F, _ = ctx.moments()
    I = ctx.intensity()
    ctx.close()
    p = oracle_problem(wl, n, w)
    o = oracle.run(p, dt, nsteps, I0, wl["T"], wl["rho"], wl["v"], wl["sa"], wl["ss"])
    dmax = max(_deviation(o["I"], w), _deviation(I0, w))
    bound = nsteps * U * dmax + 1e-5
    errE = np.abs(E - o["E"]).max() / np.abs(o["E"]).max()
    assert errE <= bound, (errE, bound)
    errI = np.abs(I - o["I"]).max() / np.abs(o["I"]).max()
    assert errI <= nsteps * U * max(dmax, 1.0) + 1e-4, errI


def test_bf16_round_trip():
    wl = wlmod.box3d(n=10, angles="s4", steps=0)
    n, w = oracle.angles.by_name("s4")
    rng = np.random.default_rng(8)
    I0 = rng.uniform(0.5, 1.5, (len(w), 1000)) / (4 * np.pi)
    ctx = gpu_context(wl, n, w, "bf16")
    ctx.set_intensity(I0)
    I = ctx.intensity()
    ctx.close()
    J = (w[:, None] * I0).sum(axis=0)[None, :]
    dev = np.abs(I0 / J - 1.0)
    # float moments, then the 16-bit deviation: within the format's rounding
    assert np.all(np.abs(I - I0) <= (U * dev + 1e-6) * J)


def test_bf16_resume_bitwise_and_batch_refusal():
    wl = wlmod.box3d(n=9, angles="s2", steps=0)
    n, w = oracle.angles.by_name("s2")
    ref = gpu_context(wl, n, w, "bf16")
    ref.set_intensity(initial_state(wl, len(w), "fp32"))
    ref.set_material(wl["rho"], wl["T"], wl["v"], wl["sa"], wl["ss"])
    for _ in range(4):
        ref.step(0.0)
    ref.sync()
    a = gpu_context(wl, n, w, "bf16")
    a.set_intensity(initial_state(wl, len(w), "fp32"))
    a.set_material(wl["rho"], wl["T"], wl["v"], wl["sa"], wl["ss"])
    a.step(0.0)
    a.step(0.0)
    buf = a.save_state()
    f32 = gpu_context(wl, n, w, "fp32")
    with pytest.raises(rt.RTError):
        f32.load_state(buf)                 # another storage precision
    b = gpu_context(wl, n, w, "bf16")
    b.load_state(buf)
    b.step(0.0)
    b.step(0.0)
    b.sync()
    np.testing.assert_array_equal(b.intensity(), ref.intensity())
    np.testing.assert_array_equal(b.moments()[0], ref.moments()[0])
    batch = rt.rt_batch_create(None)
    with pytest.raises(rt.RTError) as e:
        rt.rt_batch_add(batch, a.ctx)
    assert e.value.status == rt.RT_E_INVALID
    rt.rt_batch_destroy(batch)
    for c in (ref, a, f32, b):
        c.close()
