"""bench.py's CPU baseline legs on a tiny workload (no GPU).

The single-thread leg and the all-cores leg (one oracle process per core, all
started together) must count the same events per copy: every copy runs the
same deterministic sample, so the all-cores rate is the copies' events over
the slowest copy's time.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_all_cores_leg_runs_one_oracle_per_core(orc):
    import bench

    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    r = bench._cpu_all_cores("cols2x2_f32w", 20)
    assert r is not None
    assert r["cores"] == cores and r["kind"] == "oracle" and r["unit"] == bench.UNIT
    assert r["value"] > 0
    assert "20 steps of cols2x2_f32w" in r["sample"]


def test_single_thread_leg_reports_both(orc):
    import bench

    cb = bench._cpu_baseline("cols2x2_f32w", seconds_target=0.3)
    assert cb["cores"] == 1 and cb["value"] > 0 and cb["kind"] == "oracle"
    assert cb["all_cores"] is not None and cb["all_cores"]["cores"] >= 1
