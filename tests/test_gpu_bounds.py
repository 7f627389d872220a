"""The index-checking build of the library (RT_BOUNDS_CHECK, built by
paper_1403_6126_gb300/build.py with check=True): every shared- and
global-memory index of the float step's per-tile code is range checked,
and a violation counts as a step failure instead of an access.  A child
process steps ragged 1-D/2-D/3-D grids (open, inflow and periodic faces,
padding angles, velocity on and off, 120 angles with the table in shared
memory) through every compiled tile shape, the batch kernel's tile sets and
the allocation-free step with that library, and must report none.  This
stands in for a memory checker, which this setup does not run."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_no_index_out_of_range_in_the_float_step():
    r = subprocess.run([sys.executable, os.path.join(HERE, "_bounds_child.py")], capture_output=True, text=True,
                       timeout=1500)
    assert r.returncode == 0 and r.stdout.rstrip().endswith("OK"), (r.stdout[-3000:], r.stderr[-3000:])
