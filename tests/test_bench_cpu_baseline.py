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
