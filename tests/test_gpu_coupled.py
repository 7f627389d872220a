"""rt_step_coupled: the gas-coupling loop (fields in, one step, sources out)
in one call, with the transfers of one slab of the grid overlapping the
step of the next.  Every output and the state afterwards are bitwise those of
rt_set_material + rt_step + rt_sources."""
import numpy as np
import pytest

import oracle
import paper_1403_6126_gb300 as rt
from paper_1403_6126_gb300 import workloads as wlmod

from _helpers import gpu_context

pytestmark = pytest.mark.gpu


def _box(shape, seed, bc=None, estimate_v=True):
    wl = wlmod.box3d(n=4, angles="s4", steps=0)
    rho, v, sa, ss = wlmod._gas_fields(shape, wl["C"], seed, 4.0)
    N = rho.size
    wl.update(shape=shape, rho=rho, v=v, sa=sa, ss=ss, T=np.ones(N), estimate_v=estimate_v,
              hi=(1.0, shape[1] / shape[2], shape[0] / shape[2]))
    if bc is not None:
        wl["bc"] = bc
        wl["inflow"] = {(a, s): ("beam", 2.0, a) for a in range(3) for s in range(2) if bc[a][s] == wlmod.INFLOW}
    return wl


def _fields(wl, k, T):
    """Fields of coupled step k: the caller's gas update changes rho and v a
    little every step; T is the previous step's T_new."""
    f = 1.0 + 0.01 * k
    return [wl["rho"] * f, T, wl["v"] * (2.0 - f), wl["sa"], wl["ss"]]


def _outputs(ctx):
    E, F, P = ctx.moments()
    return dict(I=ctx.intensity(), E=E, F=F, P=P)


def _twins(wl, precision):
    n, w = oracle.angles.by_name(wl["angles"])
    a, b = gpu_context(wl, n, w, precision), gpu_context(wl, n, w, precision)
    for c in (a, b):
        c.set_material(wl["rho"], wl["T"], wl["v"], wl["sa"], wl["ss"])
    return a, b


def _run_pair(wl, precision, steps, fields=_fields):
    """The coupled call on one context, the three calls on its twin, from
    identical states; returns both histories of sources and final outputs."""
    a, b = _twins(wl, precision)
    N = int(np.prod(wl["shape"]))
    Ta, Tb = wl["T"].copy(), wl["T"].copy()
    hist = []
    for k in range(steps):
        dEa, dMa = np.zeros(N), np.zeros((3, N))
        fa = fields(wl, k, Ta)
        a.step_coupled(0.0, *fa, dE_gas=dEa, dMom=dMa, T_new=Ta)   # T_new written over T
        fb = fields(wl, k, Tb)
        b.set_material(*fb)
        b.step(0.0)
        dEb, dMb, Tb = b.sources()
        hist.append(((dEa.copy(), dMa.copy(), Ta.copy()), (dEb, dMb, Tb.copy())))
    a.sync(); b.sync()
    out = (_outputs(a), _outputs(b))
    a.close(); b.close()
    return hist, out


def _assert_same(hist, out):
    for k, (ga, gb) in enumerate(hist):
        for name, x, y in zip(("dE_gas", "dMom", "T_new"), ga, gb):
            np.testing.assert_array_equal(x, y, err_msg="step %d %s" % (k, name))
    for key in out[0]:
        np.testing.assert_array_equal(out[0][key], out[1][key], err_msg=key)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_coupled_equals_three_calls_periodic(precision):
    # 40 planes: 10 tile layers of 4 in eight slabs (1, 1, 1, 2, 2, 1, 1, 1
    # layers) on two alternating streams; the periodic wrap
    # makes slab 0 read the top planes
    _assert_same(*_run_pair(_box((40, 24, 32), 31), precision, 4))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_coupled_equals_three_calls_ragged_open_faces(precision):
    bc = ((wlmod.INFLOW, wlmod.COPY), (wlmod.VACUUM, wlmod.COPY), (wlmod.COPY, wlmod.VACUUM))
    _assert_same(*_run_pair(_box((37, 29, 50), 32, bc=bc), precision, 3))


def test_coupled_velocity_switch_steps_again():
    # without the velocity estimate the kernel follows v: zero in the first
    # step, nonzero in the second, zero again in the third
    wl = _box((24, 16, 16), 33, estimate_v=False)

    def fields(wl, k, T):
        return [wl["rho"], T, wl["v"] * (k % 2), wl["sa"], wl["ss"]]

    _assert_same(*_run_pair(wl, "fp32", 3, fields))


def test_coupled_first_call_and_small_grids_fall_back():
    # the first call (no fields yet) and a grid of one tile layer run the
    # three calls in turn: same results
    wl = _box((4, 16, 16), 34)
    n, w = oracle.angles.by_name(wl["angles"])
    a, b = gpu_context(wl, n, w, "fp32"), gpu_context(wl, n, w, "fp32")
    dEa, dMa, Ta = a.step_coupled(0.0, wl["rho"], wl["T"], wl["v"], wl["sa"], wl["ss"])
    b.set_material(wl["rho"], wl["T"], wl["v"], wl["sa"], wl["ss"])
    b.step(0.0)
    dEb, dMb, Tb = b.sources()
    for x, y in ((dEa, dEb), (dMa, dMb), (Ta, Tb)):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(a.intensity(), b.intensity())
    a.close(); b.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_coupled_2d_slabs_along_y(precision):
    # 2-D: slabs of tile rows along y (periodic, so slab 0 reads the top rows)
    wl = wlmod.box2d(n=80, angles="s4", steps=0)
    _assert_same(*_run_pair(wl, precision, 3))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_coupled_1d_slabs_along_x(precision):
    # 1-D: slabs of tiles along x, open ends (copy below, vacuum above)
    wl = wlmod.slab1d(n=3000, M=16, steps=0)
    wl["hold_T"] = False

    def fields(wl, k, T):
        return [wl["rho"] * (1.0 + 0.01 * k), T, wl["v"], wl["sa"], wl["ss"]]

    _assert_same(*_run_pair(wl, precision, 3, fields))


def test_coupled_bad_field_leaves_intensity():
    wl = _box((40, 16, 16), 35)
    n, w = oracle.angles.by_name(wl["angles"])
    ctx = gpu_context(wl, n, w, "fp32")
    ctx.set_material(wl["rho"], wl["T"], wl["v"], wl["sa"], wl["ss"])
    ctx.step_coupled(0.0, wl["rho"], wl["T"].copy(), wl["v"], wl["sa"], wl["ss"])
    I0 = ctx.intensity()
    rho = wl["rho"].copy()
    rho[-5] = np.nan                     # in the last slab
    with pytest.raises(rt.RTError) as e:
        ctx.step_coupled(0.0, rho, wl["T"].copy(), wl["v"], wl["sa"], wl["ss"])
    assert e.value.status == rt.RT_E_NONFINITE
    np.testing.assert_array_equal(ctx.intensity(), I0)
    with pytest.raises(rt.RTError) as e:
        ctx.step(0.0)                    # the gas fields must be set again
    assert e.value.status == rt.RT_E_STATE
    ctx.set_material(wl["rho"], wl["T"], wl["v"], wl["sa"], wl["ss"])
    ctx.step(0.0)
    ctx.sync()
    ctx.close()
