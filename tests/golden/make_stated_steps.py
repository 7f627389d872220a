"""Writes the FP64 oracle's E_r and F_r after the full step count of each
single-problem workload (the 1-D slab: 2000 steps, the 2-D shadow problem:
4000 steps, the 3-D box: 500 steps), at full size, and of requests 8 and 41
of the serving stream (a 96^2 box2d and a 64^3 box3d problem, 24 angles,
200 steps each), for tests/test_gpu_stated_steps.py, tests/test_gpu_server.py
and the accuracy report of bench.py.

Only the CPU oracle (oracle/) computes anything here; the inputs come from
the seeded generators of paper_1403_6126_gb300.workloads, rounded to float32
(fields and initial intensity) so that one oracle run serves the FP64 and the
float32 GPU paths alike.  Each file holds the time step, the whole-grid
scales max E_r, max |F_r| (over the active axes) and sum E_r, and E_r, F_r
at a seeded sample of cells (every cell of the slab) plus the cells of
largest and smallest E_r and of largest |F_r|.

usage: python tests/golden/make_stated_steps.py [slab1d] [shadow2d] [box3d] [serving_req8] [serving_req41]
(the box takes a few CPU-hours on eight cores; the others minutes)
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1403_6126_gb300 import workloads as wlmod  # noqa: E402

# workload name -> (generator keywords, steps, sampled cells)
CASES = {
    "slab1d": (dict(), 2000, None),
    "shadow2d": (dict(), 4000, 600),
    "box3d": (dict(n=128), 500, 600),
    "serving_req8": (dict(index=8), 200, 600),
    "serving_req41": (dict(index=41), 200, 600),
}


def inputs(name):
    """The float32-rounded workload, its angle set, I0 and the oracle problem."""
    kw, steps, _ = CASES[name]
    base = wlmod.serving_request(**kw) if name.startswith("serving") else wlmod.by_name(name, **kw)
    assert base.get("steps", steps) == steps
    wl = wlmod.rounded_to_float32(base)
    n, w = oracle.angles.by_name(wl["angles"])
    I0 = wlmod.initial_intensity(wl, len(w)).astype(np.float32).astype(np.float64)
    dx = tuple((wl["hi"][d] - wl["lo"][d]) / wl["shape"][2 - d] for d in range(3))
    inflow = {face: wlmod.inflow_values(rule, n) for face, rule in wl["inflow"].items()}
    p = oracle.Problem(wl["shape"], dx, n, w, C=wl["C"], P=wl["P"], dim=wl["dim"], bc=wl["bc"], inflow=inflow,
                       gamma=wl["gamma"], R=wl["R"], hold_T=wl["hold_T"], estimate_v=wl["estimate_v"])
    return wl, n, w, I0, p, steps


def active_flux(F, dim):
    """|F_r| over the grid's active axes: a 1-D slab set is written as
    n = (mu, sqrt(1 - mu^2), 0), whose F_y is a by-product of that choice."""
    return np.sqrt((np.asarray(F)[:dim] ** 2).sum(axis=0))


def sample_cells(name, E, Fabs):
    N = E.size
    nsamp = CASES[name][2]
    if nsamp is None or nsamp >= N:
        return np.arange(N)
    rng = np.random.default_rng(1234)
    cells = set(rng.choice(N, size=nsamp, replace=False).tolist())
    cells.update([int(np.argmax(E)), int(np.argmin(E)), int(np.argmax(Fabs))])
    return np.array(sorted(cells))


def write(name):
    wl, n, w, I0, p, steps = inputs(name)
    dt = oracle.cfl_dt(p, wl["cfl"])
    oracle.set_threads(os.cpu_count() or 1)
    t0 = time.time()
    o = oracle.run(p, dt, steps, I0, wl["T"], wl["rho"], wl["v"], wl["sa"], wl["ss"])
    E, F = o["E"], o["F"]
    Fabs = active_flux(F, wl["dim"])
    cells = sample_cells(name, E, Fabs)
    path = os.path.join(HERE, "stated_%s.txt" % name)
    with open(path, "w") as f:
        f.write("# %s %s x %d angles (%s), %d steps, float32-rounded inputs; FP64 oracle\n"
                % (name, "x".join(str(s) for s in wl["shape"][::-1]), len(w), wl["angles"], steps))
        f.write("# written by tests/golden/make_stated_steps.py (oracle only)\n")
        f.write("dt %.17g\n" % dt)
        f.write("steps %d\n" % steps)
        f.write("E_max %.17g\n" % np.abs(E).max())
        f.write("F_max %.17g\n" % Fabs.max())
        f.write("E_sum %.17g\n" % E.sum())
        f.write("# cell E Fx Fy Fz\n")
        for c in cells:
            f.write("%d %.17g %.17g %.17g %.17g\n" % (c, E[c], F[0, c], F[1, c], F[2, c]))
    print("%s: %d steps in %.0f s, %d cells -> %s" % (name, steps, time.time() - t0, len(cells), path), flush=True)


def read(name):
    """(dt, steps, scales dict, cells, E, F[3, k]) from a written file."""
    path = os.path.join(HERE, "stated_%s.txt" % name)
    scal, rows = {}, []
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if len(parts) == 2:
                scal[parts[0]] = float(parts[1])
            else:
                rows.append([float(x) for x in parts])
    a = np.array(rows)
    return scal["dt"], int(scal["steps"]), scal, a[:, 0].astype(np.int64), a[:, 1], a[:, 2:5].T


if __name__ == "__main__":
    for name in sys.argv[1:] or list(CASES):
        write(name)
