"""Failure paths, driven by host-side fault injection (rt_fault_inject): a
device allocation that fails inside rt_create, a batch rebuild and a server
admission.  Each entry point reports the error, frees what it had
allocated, and the library keeps working afterwards.  No fault reaches the
GPU: the failing allocation is never requested."""
import numpy as np
import pytest
import torch

import oracle
import paper_1403_6126_gb300 as rt
from paper_1403_6126_gb300 import workloads as wlmod

from _helpers import gpu_context, initial_state

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def clear_faults():
    yield
    rt.rt_fault_inject(rt.RT_FAULT_NONE)


def _wl():
    return wlmod.box3d(n=12, angles="s4", steps=0)


def _ready(wl, stream=None):
    n, w = oracle.angles.by_name(wl["angles"])
    c = gpu_context(wl, n, w, "fp32", stream=stream)
    c.set_intensity(initial_state(wl, len(w), "fp32"))
    c.set_material(wl["rho"], wl["T"], wl["v"], wl["sa"], wl["ss"])
    return c


def test_create_fails_cleanly_at_every_allocation():
    wl = _wl()
    n, w = oracle.angles.by_name(wl["angles"])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    for k in range(64):
        rt.rt_fault_inject(rt.RT_FAULT_ALLOC, k)
        try:
            c = gpu_context(wl, n, w, "fp32")
        except rt.RTError as e:
            assert e.status == rt.RT_E_NOMEM
            failures += 1
            continue
        c.close()
        break
    assert failures >= 10                 # every allocation of rt_create was hit in turn
    rt.rt_fault_inject(rt.RT_FAULT_NONE)
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < 64 << 20     # nothing leaked
    c = _ready(wl)
    c.step(0.0)
    c.sync()
    assert np.all(np.isfinite(c.moments()[0]))
    c.close()


def test_batch_rebuild_failure_then_recovery():
    stream = torch.cuda.Stream()
    wl = _wl()
    members = [_ready(wl, stream.cuda_stream) for _ in range(3)]
    b = rt.rt_batch_create(stream.cuda_stream)
    for c in members:
        rt.rt_batch_add(b, c.ctx)
    rt.rt_fault_inject(rt.RT_FAULT_ALLOC, 0)       # the work list's allocation
    with pytest.raises(rt.RTError):
        rt.rt_batch_step(b, 2)
    rt.rt_fault_inject(rt.RT_FAULT_NONE)
    rt.rt_batch_step(b, 2)                          # rebuilds and runs
    torch.cuda.synchronize()
    alone = _ready(wl, stream.cuda_stream)
    alone.step(0.0)
    alone.step(0.0)
    alone.sync()
    for c in members:
        c.sync()
        np.testing.assert_array_equal(c.moments()[0], alone.moments()[0])
    rt.rt_batch_destroy(b)
    for c in members + [alone]:
        c.close()


def test_server_request_fails_others_continue():
    import ctypes
    wl = wlmod.box3d(n=10, angles="s2", steps=0)
    wl["v"] = np.zeros_like(wl["v"])
    n, w = oracle.angles.by_name(wl["angles"])
    g = rt.rt_grid()
    g.dim = 3
    for d in range(3):
        g.n[d] = 10
        g.lo[d], g.hi[d] = 0.0, 1.0
        g.bc[d][0] = g.bc[d][1] = rt.RT_BC_PERIODIC
    a = rt.rt_angles()
    a.m = len(w)
    a.n = n.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    a.w = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    f = [np.ascontiguousarray(wl[k], dtype=np.float64).reshape(-1) for k in ("rho", "T", "v", "sa", "ss")]
    o = rt.rt_options_default()
    server = rt.rt_server_create(1 << 30, o)
    rt.rt_fault_inject(rt.RT_FAULT_ALLOC, 0)        # the first request's context
    t_bad = rt.rt_submit(server, g, a, wl["C"], wl["P"], *f, 3)
    rt.rt_server_wait(server, t_bad, 60.0)
    with pytest.raises(rt.RTError) as e:
        rt.rt_poll(server, t_bad)
    assert e.value.status == rt.RT_E_NOMEM
    t_ok = rt.rt_submit(server, g, a, wl["C"], wl["P"], *f, 3)
    rt.rt_server_wait(server, t_ok, 60.0)
    E = np.zeros(1000)
    assert rt.rt_poll(server, t_ok, E) is not None
    assert np.all(np.isfinite(E)) and E.min() > 0
    rt.rt_server_destroy(server)
