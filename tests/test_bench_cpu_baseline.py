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


def test_batch_bytes_match_the_per_net_formula():
    """The batched form's algorithmic bytes: 26 B per neuron and step, and per
    spike 12 B + k_out records of 8 B + 6 B per delay bucket, summed over nets."""
    import bench
    from paper_1511_09325_gb300 import workloads as W

    grids = [(1, 1), (2, 3)]
    neurons = [W.neuron_params(), W.neuron_params(nu_ext_kHz=3.0)]
    synapses = [W.synapse_params(), W.synapse_params(k_out=150, d_min=2, d_max=7)]
    events = [1240.0 * 10, 150.0 * 4]  # 10 and 4 spikes
    got = bench._batch_bytes(grids, neurons, synapses, events, 5)
    want = (26 * 1240 * 5 + 10 * (12 + 8 * 1240 + 6 * 20)
            + 26 * 6 * 1240 * 5 + 4 * (12 + 8 * 150 + 6 * 6))
    assert got == want


def test_clock_samples_parse_median_max_and_reasons():
    """nvidia-smi lines (uuid, SM MHz, max MHz, power, active mask, then the
    four throttle flags): the median clock under load, the maximum, the
    reasons that were ever active, other GPUs' and garbled lines ignored."""
    import bench

    u = "GPU-0a1b2c3d-4e5f-6789-abcd-ef0123456789"
    other = "GPU-ffffffff-0000-0000-0000-000000000000"
    na = "Not Active"
    lines = [
        "%s, 1995, 2070, 880.1, 0x0, %s, %s, %s, %s" % (u, na, na, na, na),
        "%s, 2070, 2070, 910.0, 0x4, %s, %s, %s, Active" % (u, na, na, na),
        "%s, 2025, 2070, 905.2, 0x0, %s, %s, %s, %s" % (u, na, na, na, na),
        "%s, 705, 2070, 90.0, 0x8, Active, %s, %s, %s" % (other, na, na, na),
        "%s, [N/A], 2070, 0, 0x0, %s, %s, %s, %s" % (u, na, na, na, na),
        "garbage",
    ]
    r = bench.parse_clocks("\n".join(lines), u)
    assert r == {"sm_mhz": 2025.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                 "samples": 3}
    assert bench.parse_clocks("", u) is None
    assert bench.parse_clocks("\n".join(lines))["samples"] == 4  # every GPU's lines


def test_clock_records_that_disqualify_a_timing():
    import bench

    ok = {"sm_mhz": 2025.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 9}
    assert not bench.clocks_rejected(ok)
    assert not bench.clocks_rejected(None)
    assert not bench.clocks_rejected(dict(ok, reasons=["sw_power_cap"], sm_mhz=1500.0))
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.clocks_rejected(dict(ok, reasons=[r]))
    assert bench.clocks_rejected(dict(ok, sm_mhz=1200.0))  # locked low, no reason
    assert not bench.any_rank(None, False, "cpu") and bench.any_rank(None, True, "cpu")


def test_reference_arm_line_on_a_tiny_workload(orc, capsys):
    """The reference arm times the oracle for exactly K steps after W warm-up
    steps and prints the same config object as the GPU arm."""
    import argparse
    import json

    import bench
    from paper_1511_09325_gb300 import workloads as W

    args = argparse.Namespace(workload="cols2x2_f32w", steps=4, warmup=2, gpus=1, settle=0)
    bench.run_reference(args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 4 and line["warmup"] == 2
    assert line["value"] > 0 and line["unit"] == bench.UNIT
    assert line["config"] == bench._config(args, W.WORKLOADS["cols2x2_f32w"], None, 1)
    assert line["cpu_baseline"]["value"] == line["value"]
    assert "steps 2..5" in line["cpu_baseline"]["sample"]
