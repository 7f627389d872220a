"""Checkpoint / resume: a context saved after k steps and loaded into a fresh
context continues bitwise as the original run, for both precisions and with
inflow boundaries; a state from another grid, angle set or precision is
refused."""
import numpy as np
import pytest

import oracle
import paper_1403_6126_gb300 as rt
from paper_1403_6126_gb300 import workloads as wlmod

from _helpers import gpu_context, initial_state

pytestmark = pytest.mark.gpu


def _make(wl, precision, set_material=True, inflow=True):
    n, w = oracle.angles.by_name(wl["angles"])
    ctx = gpu_context(wl, n, w, precision, inflow=inflow)
    if set_material:
        ctx.set_intensity(initial_state(wl, len(w), precision))
        ctx.set_material(wl["rho"], wl["T"], wl["v"], wl["sa"], wl["ss"])
    return ctx


def _snapshot(ctx):
    E, F, P = ctx.moments()
    dE, dM, T = ctx.sources()
    return dict(I=ctx.intensity(), E=E, F=F, P=P, dEgas=dE, dMom=dM, T=T)


@pytest.mark.parametrize("name,kw,precision", [
    ("box3d", dict(n=12, angles="s4"), "fp32"),
    ("box3d", dict(n=10, angles="s2"), "fp64"),
    ("shadow2d", dict(nx=40, ny=24, angles="s4"), "fp32"),
])
def test_resume_is_bitwise(name, kw, precision):
    wl = wlmod.by_name(name, steps=0, **kw)
    straight = _make(wl, precision)
    for _ in range(6):
        straight.step(0.0)
    straight.sync()
    ref = _snapshot(straight)
    straight.close()

    first = _make(wl, precision)
    for _ in range(3):
        first.step(0.0)
    buf = first.save_state()
    first.close()
    # a fresh context: same grid, angles and options, no inflow and no
    # material set before the load (both come from the state)
    second = _make(wl, precision, set_material=False, inflow=False)
    second.load_state(buf)
    for _ in range(3):
        second.step(0.0)
    second.sync()
    got = _snapshot(second)
    second.close()
    for k in ref:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)


def test_load_refuses_other_problems():
    wl = wlmod.box3d(n=8, angles="s2", steps=0)
    a = _make(wl, "fp32")
    buf = a.save_state()
    for other, prec in ((wlmod.box3d(n=9, angles="s2", steps=0), "fp32"),
                        (wlmod.box3d(n=8, angles="s4", steps=0), "fp32"),
                        (wl, "fp64")):
        b = _make(other, prec, set_material=False)
        with pytest.raises(rt.RTError) as e:
            b.load_state(buf)
        assert e.value.status == rt.RT_E_INVALID
        b.close()
    with pytest.raises(rt.RTError) as e:
        a.load_state(buf[:100])
    assert e.value.status == rt.RT_E_INVALID
    a.close()
