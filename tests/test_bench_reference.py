"""bench.py on CPU.  The reference arm (the FP64 oracle on host cores): one JSON line with the
headline's metric and unit, a cpu_baseline and an e2e object; under a launcher only rank 0
runs it and the other ranks exit without work.  The clock summary of the timed region."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=300, check=True)


def test_reference_arm_prints_one_line():
    out = _run({"RANK": "0", "WORLD_SIZE": "1"}).stdout.strip().splitlines()
    assert len(out) == 1
    line = json.loads(out[0])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "MLUPS" and line["higher_is_better"] is True and line["value"] > 0
    assert line["steps"] == 2 and line["warmup"] == 3 and line["n_gpus"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["config"]["workload"].startswith("quadrants_2d_1024")


def test_reference_arm_other_ranks_do_nothing():
    res = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert res.stdout.strip() == ""


def test_clock_summary_reads_the_samples_of_the_timed_region():
    c = bench.ClockSampler(0)
    c.lines = ["0, 1980, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",   # before the region
               "0, 2070, 2070, 1200.5, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2055, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active",
               "garbage"]
    c.skip = 1
    d = c.summary(2070.0)
    assert d["sm_mhz"] == 2062.5 and d["sm_max_mhz"] == 2070.0
    assert d["reasons"] == ["sw_power_cap"] and d["samples"] == 2 and d["samples_in_region"] == 3
    c.lines = c.lines[:1]                       # region shorter than one interval
    d = c.summary(2070.0)
    assert d["sm_mhz"] == 1980.0 and d["samples_in_region"] == 0
    c.lines = []
    assert bench.ClockSampler(0).summary(2070.0)["reasons"] == ["unsampled"]
