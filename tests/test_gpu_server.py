"""Serving loop: continuous batching.  Requests that arrive while others run
are admitted as memory frees up, share the persistent launches, and each
result is bitwise the one the problem gets alone."""
import ctypes
import os
import sys
import time

import numpy as np
import pytest

import oracle
import paper_1403_6126_gb300 as rt
from paper_1403_6126_gb300 import workloads as wlmod

from _helpers import gpu_context

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))

pytestmark = pytest.mark.gpu


def _request(wl):
    n, w = oracle.angles.by_name(wl["angles"])
    n, w = np.ascontiguousarray(n), np.ascontiguousarray(w)
    g = rt.rt_grid()
    g.dim = wl["dim"]
    nz, ny, nx = wl["shape"]
    for d, nd in enumerate((nx, ny, nz)):
        g.n[d] = nd
        g.lo[d], g.hi[d] = wl["lo"][d], wl["hi"][d]
        g.bc[d][0], g.bc[d][1] = wl["bc"][d]
    a = rt.rt_angles()
    a.m = len(w)
    a.n = n.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    a.w = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    fields = [np.ascontiguousarray(wl[k], dtype=np.float64).reshape(-1) for k in ("rho", "T", "v", "sa", "ss")]
    return g, a, (n, w), fields


def _problems():
    out = []
    for n, ang in ((10, "s4"), (12, "s2"), (8, "s6"), (14, "s2")):
        out.append(wlmod.box3d(n=n, angles=ang, seed=n, steps=0))
    for nx, ny, ang in ((40, 24, "s4"), (33, 17, "s2")):
        wl = wlmod.shadow2d(nx=nx, ny=ny, angles=ang, steps=0)
        wl["bc"] = ((0, 0), (0, 0), (0, 0))   # periodic: the server takes no inflow tables
        wl["inflow"] = {}
        wl["v"][0] = 0.04 * wl["C"]
        out.append(wl)
    for wl in out:
        wl["estimate_v"], wl["hold_T"] = True, False
    return out


def _opts():
    o = rt.rt_options_default()
    o.estimate_v, o.hold_T = 1, 0
    return o


def _alone(wl, nsteps):
    n, w = oracle.angles.by_name(wl["angles"])
    ctx = gpu_context(wl, n, w, "fp32")
    ctx.set_material(wl["rho"], wl["T"], wl["v"], wl["sa"], wl["ss"])
    for _ in range(nsteps):
        ctx.step(0.0)
    ctx.sync()
    out = ctx.moments()
    ctx.close()
    return out


def test_server_results_equal_each_problem_alone():
    probs = _problems()
    steps = [3, 5, 2, 4, 6, 1]
    # budget: room for the two largest requests at a time, so the rest queue
    N = [int(np.prod(p["shape"])) for p in probs]
    M = [len(oracle.angles.by_name(p["angles"])[1]) for p in probs]
    per = sorted((Ni * (8 * Mi + 240) * 2 for Ni, Mi in zip(N, M)), reverse=True)
    server = rt.rt_server_create(per[0] + per[1], _opts())
    keep, tickets = [], []
    for i, wl in enumerate(probs[:3]):
        g, a, angs, fields = _request(wl)
        keep.append((g, a, angs, fields))
        tickets.append(rt.rt_submit(server, g, a, wl["C"], wl["P"], *fields, steps[i]))
    rt.rt_server_wait(server, tickets[0], 60.0)
    for i, wl in enumerate(probs[3:], start=3):   # arrive while others run
        g, a, angs, fields = _request(wl)
        keep.append((g, a, angs, fields))
        tickets.append(rt.rt_submit(server, g, a, wl["C"], wl["P"], *fields, steps[i]))
    results = []
    for i, t in enumerate(tickets):
        rt.rt_server_wait(server, t, 120.0)
        E, F, P = np.zeros(N[i]), np.zeros((3, N[i])), np.zeros((6, N[i]))
        lat = rt.rt_poll(server, t, E, F, P)
        assert lat is not None and lat > 0
        results.append((E, F, P))
    stats = rt.rt_server_stats(server)
    assert stats["queued"] == 0 and stats["running"] == 0 and stats["bytes_in_use"] == 0
    assert stats["steps"] >= max(steps)
    rt.rt_server_destroy(server)
    for wl, s, (E, F, P) in zip(probs, steps, results):
        Ea, Fa, Pa = _alone(wl, s)
        np.testing.assert_array_equal(E, Ea)
        np.testing.assert_array_equal(F, Fa)
        np.testing.assert_array_equal(P, Pa)


def test_server_errors_and_timeouts():
    # a long request in a static medium (no velocity: stays in equilibrium)
    wl = wlmod.box3d(n=32, angles="s8", steps=0)
    wl["v"] = np.zeros_like(wl["v"])
    g, a, angs, fields = _request(wl)
    small = rt.rt_server_create(1 << 20, _opts())
    with pytest.raises(rt.RTError) as e:
        rt.rt_submit(small, g, a, wl["C"], wl["P"], *fields, 10)
    assert e.value.status == rt.RT_E_BUDGET
    rt.rt_server_destroy(small)
    server = rt.rt_server_create(8 << 30, _opts())
    t = rt.rt_submit(server, g, a, wl["C"], wl["P"], *fields, 400)
    with pytest.raises(rt.RTError) as e:
        rt.rt_server_wait(server, t, 0.0)
    assert e.value.status == rt.RT_E_TIMEOUT
    assert rt.rt_poll(server, t) is None          # still pending
    rt.rt_server_wait(server, t, 300.0)
    assert rt.rt_poll(server, t) > 0
    with pytest.raises(rt.RTError) as e:
        rt.rt_poll(server, t)                      # ticket released
    assert e.value.status == rt.RT_E_INVALID
    rt.rt_server_destroy(server)


def test_process_exit_with_a_live_server():
    # a program that exits with a server still running (requests in flight,
    # no rt_server_destroy) ends cleanly: the library stops its servers
    # before the CUDA runtime shuts down
    import os
    import subprocess
    import sys
    code = """
import ctypes, numpy as np, oracle, paper_1403_6126_gb300 as rt
from paper_1403_6126_gb300 import workloads as wlmod
wl = wlmod.box3d(n=16, angles="s4", steps=0)
wl["v"] = np.zeros_like(wl["v"])
n, w = oracle.angles.by_name("s4")
g = rt.rt_grid(); g.dim = 3
for d in range(3):
    g.n[d] = 16; g.lo[d], g.hi[d] = 0.0, 1.0; g.bc[d][0] = g.bc[d][1] = rt.RT_BC_PERIODIC
a = rt.rt_angles(); a.m = len(w)
a.n = n.ctypes.data_as(ctypes.POINTER(ctypes.c_double)); a.w = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
f = [np.ascontiguousarray(wl[k], dtype=np.float64).reshape(-1) for k in ("rho", "T", "v", "sa", "ss")]
s = rt.rt_server_create(1 << 30, rt.rt_options_default())
for _ in range(4):
    rt.rt_submit(s, g, a, wl["C"], wl["P"], *f, 1000)
print("leaving")
"""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.returncode, r.stderr[-2000:])
    assert "leaving" in r.stdout


@pytest.mark.parametrize("req", [8, 41])
def test_served_result_matches_the_oracle(req):
    # Requests of the serving stream (8: 96^2 box2d, 41: 64^3 box3d, both 24
    # angles, 200 steps) submitted through rt_submit, alongside another
    # request so that they share the persistent launches, against the FP64
    # oracle's stored values (tests/golden/stated_serving_req*.txt, written
    # by make_stated_steps.py from the oracle alone): E_r and |F_r| within
    # the 1e-5 bound of the float path, at the stored cells, relative to the
    # whole-grid maxima.
    import make_stated_steps as golden
    name = "serving_req%d" % req
    dt, steps, scal, cells, Eo, Fo = golden.read(name)
    wl, n, w, I0, _, _ = golden.inputs(name)
    g, a, angs, fields = _request(wl)
    other = _problems()[0]
    og, oa, oangs, ofields = _request(other)
    server = rt.rt_server_create(8 << 30, _opts())
    try:
        # a few steps only: the 10^3 box's velocity field (spectrum to the
        # grid scale) drives the method past its positivity limit by ~40 steps
        t_other = rt.rt_submit(server, og, oa, other["C"], other["P"], *ofields, 5)
        t = rt.rt_submit(server, g, a, wl["C"], wl["P"], *fields, steps)
        rt.rt_server_wait(server, t, 600.0)
        N = int(np.prod(wl["shape"]))
        E, F = np.zeros(N), np.zeros((3, N))
        rt.rt_poll(server, t, E, F, None)
        rt.rt_server_wait(server, t_other, 600.0)
        rt.rt_poll(server, t_other)
    finally:
        rt.rt_server_destroy(server)
    dim = wl["dim"]
    Fg = golden.active_flux(F[:, cells], dim)
    Fa = golden.active_flux(Fo, dim)
    eE = np.abs(E[cells] - Eo).max() / scal["E_max"]
    eF = np.abs(Fg - Fa).max() / max(scal["F_max"], 1e-3 * scal["E_max"])
    assert eE <= 1e-5 and eF <= 1e-5, (eE, eF)


def test_served_beam_with_inflow():
    # The shadow problem (sec. 5.8: a beam entering through the lower x face,
    # 256x128 cells x 80 angles, 4000 steps) submitted with its inflow table
    # through rt_submit_inflow beside a periodic request: bitwise the problem
    # stepped alone with rt_set_inflow, and within the float path's 1e-5 of
    # the FP64 oracle's stored values (tests/golden/stated_shadow2d.txt).
    import make_stated_steps as golden
    name = "shadow2d"
    dt, steps, scal, cells, Eo, Fo = golden.read(name)
    wl, n, w, I0, _, _ = golden.inputs(name)
    g, a, angs, fields = _request(wl)
    M, N = len(w), int(np.prod(wl["shape"]))
    inflow = np.zeros((3, 2, M))
    for (axis, side), rule in wl["inflow"].items():
        inflow[axis, side] = wlmod.inflow_values(rule, n)
    assert inflow.any()
    o = rt.rt_options_default()
    o.hold_T, o.estimate_v = int(wl["hold_T"]), int(wl["estimate_v"])
    o.gamma, o.r_ideal, o.cfl = wl["gamma"], wl["R"], wl["cfl"]
    other = wlmod.shadow2d(nx=40, ny=24, angles="s4", steps=0)
    other["bc"] = ((0, 0), (0, 0), (0, 0))
    other["inflow"] = {}
    og, oa, oangs, ofields = _request(other)
    with pytest.raises(rt.RTError) as e:           # the table is checked at submission
        bad = inflow.copy()
        bad[0, 0, 0] = -1.0
        server = rt.rt_server_create(1 << 30, o)
        try:
            rt.rt_submit_inflow(server, g, a, wl["C"], wl["P"], *fields, bad, 1)
        finally:
            rt.rt_server_destroy(server)
    assert e.value.status == rt.RT_E_NONFINITE
    server = rt.rt_server_create(8 << 30, o)
    try:
        t_other = rt.rt_submit(server, og, oa, other["C"], other["P"], *ofields, 50)
        t = rt.rt_submit_inflow(server, g, a, wl["C"], wl["P"], *fields, inflow, steps)
        rt.rt_server_wait(server, t, 600.0)
        E, F, P = np.zeros(N), np.zeros((3, N)), np.zeros((6, N))
        rt.rt_poll(server, t, E, F, P)
        rt.rt_server_wait(server, t_other, 600.0)
        rt.rt_poll(server, t_other)
    finally:
        rt.rt_server_destroy(server)
    # alone: the same problem through rt_step, its inflow set face by face
    ctx = gpu_context(wl, n, w, "fp32")
    ctx.set_material(wl["rho"], wl["T"], wl["v"], wl["sa"], wl["ss"])
    for _ in range(steps):
        ctx.step(0.0)
    ctx.sync()
    Ea, Fa, Pa = ctx.moments()
    ctx.close()
    np.testing.assert_array_equal(E, Ea)
    np.testing.assert_array_equal(F, Fa)
    np.testing.assert_array_equal(P, Pa)
    dim = wl["dim"]
    Fg = golden.active_flux(F[:, cells], dim)
    Fs = golden.active_flux(Fo, dim)
    eE = np.abs(E[cells] - Eo).max() / scal["E_max"]
    eF = np.abs(Fg - Fs).max() / max(scal["F_max"], 1e-3 * scal["E_max"])
    assert eE <= 1e-5 and eF <= 1e-5, (eE, eF)
