"""Host-side logic of bench.py (no GPU): the workload description both arms
print, and the reading and scoring of the oracle's stored samples."""
import os
import sys
import types

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_arm_config_describes_the_timed_box():
    cfg = bench.arm_config(types.SimpleNamespace(workload="box3d", n=0), 1)
    assert cfg["cells"] == 128 ** 3 and cfg["angles"] == 80
    # sec. 4.1 Step 1: dt = CFL min dx / Crat with CFL 0.4, dx = 1/128, Crat = 100
    assert abs(cfg["dt"] - 0.4 / 128 / 100) <= 1e-18
    assert "128x128x128" in cfg["workload"] and cfg["parallelism"] == "single GPU"
    assert bench.arm_config(types.SimpleNamespace(workload="box3d", n=0), 4)["parallelism"] == "replicas"


def test_arm_config_other_workloads():
    slab = bench.arm_config(types.SimpleNamespace(workload="slab1d", n=0), 1)
    assert slab["cells"] == 512 and slab["angles"] == 8
    shadow = bench.arm_config(types.SimpleNamespace(workload="shadow2d", n=0), 1)
    assert shadow["cells"] == 256 * 128 and shadow["angles"] == 80


def test_stated_samples_read_and_score():
    for name in ("slab1d", "shadow2d", "box3d", "serving_req8", "serving_req41"):
        ref = bench._stated_sample(name)
        assert ref is not None, name
        dt, steps, scal, cells, Eo, Fo = ref
        wl = bench._stated_workload(name)
        N = int(np.prod(wl["shape"]))
        assert steps > 0 and dt > 0 and cells.max() < N and Fo.shape == (3, len(cells))
        assert scal["E_max"] >= np.abs(Eo).max() and scal["E_sum"] > 0
        E, F = np.zeros(N), np.zeros((3, N))
        E[cells], F[:, cells] = Eo, Fo
        err = bench._stated_errors(E, F, ref, wl["dim"])
        assert err["E_r"] == 0.0 and err["abs_F_r"] == 0.0
        E[cells[0]] += 1e-6 * scal["E_max"]
        assert abs(bench._stated_errors(E, F, ref, wl["dim"])["E_r"] - 1e-6) < 1e-12


def test_cpu_baseline_reports_the_threads_it_used():
    # the oracle timed on a tiny box: the line must say how many threads ran
    # and what was timed (grid, angles, steps)
    from paper_1403_6126_gb300 import workloads as wlmod
    wl = wlmod.box3d(n=6, angles="s2")
    one = bench.cpu_baseline("box3d", 1, 0, wl=wl, threads=1)
    assert one["cores"] == 1 and one["value"] > 0 and one["steps"] == 1
    assert "6x6x6 cells x 8 angles" in one["sample"] and "1 thread" in one["sample"]
    two = bench.cpu_baseline("box3d", 2, 1, wl=wl, threads=2)
    assert two["cores"] == 2 and "2 timed steps (+1 warm-up)" in two["sample"]


def test_roofline_bytes_and_profile_traffic():
    # 848 bytes per cell at 80 float angles with T live and velocity on:
    # I in and out 640, rho sigma_a sigma_s v 24, T in and out 16, E F P_dd
    # of step n 56, moments and sources out 112
    assert bench.algorithmic_bytes_per_cell(80, 4, True, True) == 848
    assert bench.algorithmic_bytes_per_cell(80, 4, True, True) * 128 ** 3 == 1778384896
    assert bench.algorithmic_bytes_per_cell(8, 8, False, False) == 2 * 8 * 8 + 48 + 8 + 112
    # the ncu figure is reported only while the summary's kernel hash matches
    text = open(bench.PROFILE).read()
    assert "algorithmic_bytes_per_launch: `1778384896`" in text
    traffic = bench._profile_traffic()
    if ("kernel_source_sha256_16: `%s`" % bench.kernel_sha()) in text:
        assert traffic is not None and traffic > 1778384896
    else:
        assert traffic is None


def test_clock_summary_reads_nvidia_smi_rows():
    s = bench.ClockSampler(0)
    s.rows = [["0", "2070", "2070", "900.1", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
              ["0", "2055", "2070", "1100.5", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
              ["0", "1980", "2070", "1390.0", "0x4", "Not Active", "Not Active", "Not Active", "Active"]]
    out = s.summary()
    assert out["sm_mhz"] == 2055.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    s.rows = [["0", "[N/A]", "[N/A]", "[N/A]", "[N/A]", "Active", "Not Active", "Not Active", "Not Active"]]
    out = s.summary()
    assert out["sm_mhz"] is None and out["reasons"] == ["hw_slowdown"]
    assert bench.ClockSampler(0).summary()["reasons"] == ["unsampled"]


def test_reference_arm_line(capsys):
    # the reference arm's JSON line (the FP64 oracle on the host cores) on a
    # small box: the contract's keys, its own cpu_baseline and an e2e entry
    # with no host-device bytes
    import json
    args = types.SimpleNamespace(workload="box3d", n=8, steps=2, warmup=3, ref_steps=5)
    assert bench.run_reference(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["dtype"] == "f64" and line["steps"] == 2 and line["warmup"] == 1
    assert line["config"]["cells"] == 8 ** 3 and line["config"]["angles"] == 80
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
