"""The JSON line bench.py prints: the reference arm (the oracle, on the CPU)
and the GB300 arm (on a GPU), on the small solitary-wave workload."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BASE_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
             "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"}


def run(args, timeout):
    out = subprocess.run([sys.executable, "bench.py"] + args, cwd=ROOT, capture_output=True,
                         text=True, timeout=timeout)
    assert out.returncode == 0, out.stderr[-3000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-3000:]
    return json.loads(lines[0])


def test_reference_arm_line():
    d = run(["--impl", "reference", "--workload", "solitary_1d", "--steps", "1", "--warmup", "1"], 600)
    assert BASE_KEYS <= d.keys() and d["impl"] == "reference"
    assert d["metric"] == "grid-point RK4 steps/s" and d["unit"] == "pt-steps/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["config"]["workload"] == "solitary_1d"
    # the config dict both arms print (same keys and values for the same flags)
    assert {"parallelism", "integrator", "diagnostic", "points", "members"} <= d["config"].keys()
    assert d["config"]["parallelism"] == "single GPU"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    # every host core, one single-threaded oracle process each, and the host named
    assert cb["cores"] == cb["threads"] == os.cpu_count() == cb["nproc"] and cb["cpu_model"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


@pytest.mark.gpu
def test_gb300_arm_line():
    d = run(["--workload", "solitary_1d", "--steps", "5", "--warmup", "3", "--no-cpu-baseline"], 900)
    assert BASE_KEYS <= d.keys()
    assert d["metric"] == "grid-point RK4 steps/s" and d["unit"] == "pt-steps/s" and d["value"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 5 and d["warmup"] == 3 and d["scaling"] == "weak"
    assert d["config"]["workload"] == "solitary_1d" and d["data"] == "synthetic"
    ref = run(["--impl", "reference", "--workload", "solitary_1d", "--steps", "1", "--warmup", "1"], 600)
    assert ref["config"] == d["config"]
    r = d["roofline"]
    assert {"bound", "achieved", "peak", "unit", "frac", "traffic"} <= r.keys()
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= d["clocks"].keys()
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] > 0
    assert d["schedule"]["chosen"]


def test_schedule_summary_parses_the_report():
    # the step-schedule report of the library, as bench.py summarises it
    sys.path.insert(0, ROOT)
    import bench
    rep = ("default 6.0500 ms per step: split total/3 [concurrent] 3 units: 256x256[0:64] "
           "512x512[0:16] 512x512[16:32]\n"
           "chosen 5.9000 ms per step: split total/6 [concurrent] 6 units: 256x256[0:32] "
           "256x256[32:64] 512x512[0:8] 512x512[8:16] 512x512[16:24] 512x512[24:32]\n"
           "tried 6.4000 ms per step: serial groups [serial] 2 units: 256x256[0:64] 512x512[0:32]\n"
           "default split total/3 [concurrent] 3 units: 256x256[0:64] 512x512[0:16] 512x512[16:32]\n")
    s = bench.schedule_summary(rep)
    assert s["chosen"] == "split total/6" and s["candidates"][2]["mode"] == "serial"
    assert [c["role"] for c in s["candidates"]] == ["default", "chosen", "tried", "default"]
    assert s["candidates"][1]["ms_per_step"] == 5.9 and len(s["candidates"][1]["units"]) == 6
    assert s["candidates"][3]["ms_per_step"] is None
    only = bench.schedule_summary("default split total/3 [concurrent] 1 units: 256x1[0:1]\n")
    assert only["chosen"] == "split total/3" and only["candidates"][0]["units"] == ["256x1[0:1]"]


def test_streamed_split_summary():
    sys.path.insert(0, ROOT)
    import bench
    rep = ("chosen 6.0300 ms per step: split total/3 [concurrent] 3 units: 256x256[0:64] "
           "512x512[0:16] 512x512[16:32]\n"
           "streamed-tried 7.6000 ms per step: streamed split x1 [concurrent] 3 units: 256x256[0:64] "
           "512x512[0:16] 512x512[16:32]\n"
           "streamed-chosen 7.2000 ms per step: streamed split x2 [concurrent] 6 units: 256x256[0:32] "
           "256x256[32:64] 512x512[0:8] 512x512[8:16] 512x512[16:24] 512x512[24:32]\n")
    s = bench.streamed_split(rep)
    assert s["chosen_units"] == 6 and [c["units"] for c in s["candidates"]] == [3, 6]
    assert bench.schedule_summary(rep)["chosen"] == "split total/3"
    assert bench.streamed_split("")["chosen_units"] is None
