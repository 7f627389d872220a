"""Host-side checks of the C ABI (no GPU work): the library loads, exports
every entry point include/rt.h declares, validates its arguments before
touching the device, and its angle-set generator matches the oracle's."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_1403_6126_gb300 as rt
from paper_1403_6126_gb300 import build as rtbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    rtbuild.build()


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(rt_[a-z_0-9]+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported():
    names = _declared()
    assert {"rt_create", "rt_set_material", "rt_step", "rt_moments", "rt_destroy"} <= names
    L = ctypes.CDLL(rt.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing


@pytest.mark.parametrize("kind,order,name", [
    (rt.RT_ANGLES_LEVEL_SYMMETRIC, 2, "s2"), (rt.RT_ANGLES_LEVEL_SYMMETRIC, 4, "s4"),
    (rt.RT_ANGLES_LEVEL_SYMMETRIC, 6, "s6"), (rt.RT_ANGLES_LEVEL_SYMMETRIC, 8, "s8"),
    (rt.RT_ANGLES_PAPER_S4, 4, "paper_s4"), (rt.RT_ANGLES_GAUSS_LEGENDRE, 8, "gl8"),
    (rt.RT_ANGLES_GAUSS_LEGENDRE, 16, "gl16"), (rt.RT_ANGLES_GAUSS_LEGENDRE, 1, "gl1"),
])
def test_angle_sets_match_oracle(kind, order, name):
    n, w = rt.rt_angle_set(kind, order)
    no, wo = oracle.angles.by_name(name)
    np.testing.assert_allclose(n, no, atol=2e-15)
    np.testing.assert_allclose(w, wo, rtol=1e-13)


def test_angle_set_rejects_bad_orders():
    for kind, order in ((rt.RT_ANGLES_LEVEL_SYMMETRIC, 3), (rt.RT_ANGLES_LEVEL_SYMMETRIC, 10),
                        (rt.RT_ANGLES_GAUSS_LEGENDRE, 0), (rt.RT_ANGLES_GAUSS_LEGENDRE, 65), (7, 4)):
        with pytest.raises(rt.RTError) as e:
            rt.rt_angle_set(kind, order)
        assert e.value.status == rt.RT_E_INVALID


def _grid(dim=1, n=(8, 1, 1), bc=0):
    g = rt.rt_grid()
    g.dim = dim
    for d in range(3):
        g.n[d] = n[d]
        g.lo[d], g.hi[d] = 0.0, 1.0
        g.bc[d][0] = g.bc[d][1] = bc
    return g


def _angles(n, w):
    a = rt.rt_angles()
    a.m = len(w)
    a.n = n.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    a.w = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return a


def _expect(status, fn, *args):
    with pytest.raises(rt.RTError) as e:
        fn(*args)
    assert e.value.status == status, rt.rt_last_error()


def test_create_validates_before_touching_the_device():
    n, w = oracle.angles.by_name("s2")
    n, w = np.ascontiguousarray(n), np.ascontiguousarray(w)
    o = rt.rt_options_default()
    assert o.precision == rt.RT_FP32 and abs(o.cfl - 0.4) < 1e-15 and o.estimate_v == 1
    _expect(rt.RT_E_INVALID, rt.rt_create, _grid(dim=4), _angles(n, w), 10.0, 1.0, o)
    _expect(rt.RT_E_INVALID, rt.rt_create, _grid(n=(0, 1, 1)), _angles(n, w), 10.0, 1.0, o)
    _expect(rt.RT_E_INVALID, rt.rt_create, _grid(n=(0, 4, 4), dim=3), _angles(n, w), 10.0, 1.0, o)
    # 2^28 cells is one more than the largest grid the ABI accepts
    _expect(rt.RT_E_INVALID, rt.rt_create, _grid(n=(1024, 1024, 256), dim=3), _angles(n, w), 10.0, 1.0, o)
    empty = _angles(n, w)
    empty.m = 0
    _expect(rt.RT_E_INVALID, rt.rt_create, _grid(), empty, 10.0, 1.0, o)
    many = np.random.default_rng(0).normal(size=(257, 3))
    many = np.ascontiguousarray(many / np.linalg.norm(many, axis=1, keepdims=True))
    _expect(rt.RT_E_INVALID, rt.rt_create, _grid(), _angles(many, np.full(257, 1.0 / 257)), 10.0, 1.0, o)
    _expect(rt.RT_E_INVALID, rt.rt_create, _grid(), _angles(n, w), -1.0, 1.0, o)
    _expect(rt.RT_E_INVALID, rt.rt_create, _grid(), _angles(n, w * 1.01), 10.0, 1.0, o)
    bad = n.copy()
    bad[0] *= 1.001
    _expect(rt.RT_E_INVALID, rt.rt_create, _grid(), _angles(bad, w), 10.0, 1.0, o)
    g = _grid()
    g.bc[0][0], g.bc[0][1] = rt.RT_BC_PERIODIC, rt.RT_BC_VACUUM
    _expect(rt.RT_E_INVALID, rt.rt_create, g, _angles(n, w), 10.0, 1.0, o)
    for field, value in (("cfl", 0.0), ("cfl", float("inf")), ("gamma", 1.0), ("gamma", float("nan")),
                         ("r_ideal", float("inf"))):
        bad_o = rt.rt_options_default()
        setattr(bad_o, field, value)
        _expect(rt.RT_E_INVALID, rt.rt_create, _grid(), _angles(n, w), 10.0, 1.0, bad_o)
        assert "finite cfl" in rt.rt_last_error()
    o.precision = 7
    _expect(rt.RT_E_INVALID, rt.rt_create, _grid(), _angles(n, w), 10.0, 1.0, o)
    assert "precision" in rt.rt_last_error()


def test_null_context_calls_are_rejected():
    for fn in (lambda: rt.rt_step(None, 0.1), lambda: rt.rt_sync(None), lambda: rt.rt_run(None, 0.1, 2),
               lambda: rt.rt_set_intensity(None, None),
               lambda: rt.rt_step_coupled(None, 0.1, *([np.ones(4)] * 5), None, None, None)):
        with pytest.raises(rt.RTError) as e:
            fn()
        assert e.value.status == rt.RT_E_INVALID
    rt.rt_destroy(None)


def test_fault_inject_arguments():
    with pytest.raises(rt.RTError) as e:
        rt.rt_fault_inject(99, 0)
    assert e.value.status == rt.RT_E_INVALID
    with pytest.raises(rt.RTError) as e:
        rt.rt_fault_inject(rt.RT_FAULT_ALLOC, -1)
    assert e.value.status == rt.RT_E_INVALID
    rt.rt_fault_inject(rt.RT_FAULT_NONE)


def test_newton_options_defaults_and_validation():
    # the T^4 Newton solve of sec. 4.3: defaults are the FP64 reference's rule
    # (1e-13 relative step, at most 60 steps); out-of-range settings are
    # refused by every entry point that takes options, before device work
    o = rt.rt_options_default()
    assert o.newton_max_it == 60 and o.newton_rtol == 1e-13
    n, w = oracle.angles.by_name("s2")
    n, w = np.ascontiguousarray(n), np.ascontiguousarray(w)
    for it, tol in ((0, 1e-13), (1001, 1e-13), (60, 0.0), (60, 1e-2), (60, float("nan"))):
        o = rt.rt_options_default()
        o.newton_max_it, o.newton_rtol = it, tol
        _expect(rt.RT_E_INVALID, rt.rt_create, _grid(), _angles(n, w), 10.0, 1.0, o)
        assert "newton" in rt.rt_last_error()
        _expect(rt.RT_E_INVALID, rt.rt_server_create, 1 << 30, o)
        f = rt.rt_noalloc_fields()
        for i, (k, _) in enumerate(f._fields_):
            setattr(f, k, 4096 * (i + 1))   # never dereferenced: validation comes first
        _expect(rt.RT_E_INVALID, rt.rt_step_noalloc, _grid(), _angles(n, w), 10.0, 1.0, o, 1e-3, f)


def test_noalloc_refuses_in_place_buffers_on_the_host():
    # rt_step_noalloc reads the step-n intensity and moments of neighbouring
    # cells while it writes the new ones: one buffer for both is refused
    n, w = oracle.angles.by_name("gl8")
    n, w = np.ascontiguousarray(n), np.ascontiguousarray(w)
    o = rt.rt_options_default()
    for same in ("I", "mom"):
        f = rt.rt_noalloc_fields()
        for i, (k, _) in enumerate(f._fields_):
            setattr(f, k, 4096 * (i + 1))
        if same == "I":
            f.I_out = f.I_in
        else:
            f.mom_out = f.mom_in
        _expect(rt.RT_E_INVALID, rt.rt_step_noalloc, _grid(), _angles(n, w), 10.0, 1.0, o, 1e-3, f)
        assert "different buffers" in rt.rt_last_error()


def test_noalloc_refuses_non_finite_scalars_on_the_host():
    # every scalar is checked before the device is touched (the field
    # pointers here are distinct dummies that are never dereferenced)
    n, w = oracle.angles.by_name("gl8")
    n, w = np.ascontiguousarray(n), np.ascontiguousarray(w)
    f = rt.rt_noalloc_fields()
    for i, (k, _) in enumerate(f._fields_):
        setattr(f, k, 4096 * (i + 1))
    for C, P, dt, field, value in ((float("inf"), 1.0, 1e-3, None, None), (10.0, float("inf"), 1e-3, None, None),
                                   (10.0, 1.0, float("nan"), None, None), (10.0, 1.0, 1e-3, "gamma", float("inf")),
                                   (10.0, 1.0, 1e-3, "r_ideal", float("nan"))):
        o = rt.rt_options_default()
        if field:
            setattr(o, field, value)
        _expect(rt.RT_E_INVALID, rt.rt_step_noalloc, _grid(), _angles(n, w), C, P, o, dt, f)
        assert "need finite" in rt.rt_last_error()
