"""The stored oracle values under tests/golden/ are what the committed
script computes: the cheaper cases are run again here from the same seeded
inputs through the oracle alone and compared with the files, cell by cell.
(The 3-D box and the shadow problem take CPU-hours and CPU-minutes; they
come from the same code path.)"""
import os
import sys

import numpy as np
import pytest

import oracle

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_stated_steps as golden  # noqa: E402


@pytest.mark.parametrize("name", ["slab1d", "serving_req8"])
def test_stored_values_are_reproduced_by_the_oracle(name):
    dt_s, steps_s, scal, cells, E_s, F_s = golden.read(name)
    wl, n, w, I0, p, steps = golden.inputs(name)
    dt = oracle.cfl_dt(p, wl["cfl"])
    assert steps == steps_s
    assert dt == pytest.approx(dt_s, rel=1e-15)
    o = oracle.run(p, dt, steps, I0, wl["T"], wl["rho"], wl["v"], wl["sa"], wl["ss"])
    E, F = o["E"], o["F"]
    Fabs = golden.active_flux(F, wl["dim"])
    # the same cells are drawn, and the same values come out (to the rounding
    # that thread counts and another libm may reorder)
    np.testing.assert_array_equal(golden.sample_cells(name, E, Fabs), cells)
    Es, Fs = scal["E_max"], max(scal["F_max"], 1e-3 * scal["E_max"])
    np.testing.assert_allclose(E[cells], E_s, rtol=0, atol=1e-12 * Es)
    np.testing.assert_allclose(F[:, cells], F_s, rtol=0, atol=1e-12 * Fs)
    assert abs(np.abs(E).max() - scal["E_max"]) <= 1e-12 * Es
    assert abs(Fabs.max() - scal["F_max"]) <= 1e-12 * Fs
    assert abs(E.sum() - scal["E_sum"]) <= 1e-12 * abs(scal["E_sum"])
