"""Population statistics of the GPU paths against the FP64 model.

Criterion: over 10 s of model time, population rates within 2 % and ISI CV
within 5 % of the FP64 model.  The exact paths (FP32 weights; FP16 weights)
cannot follow the FP64 trajectory -- one threshold crossing decided
differently is amplified by the network -- and a single 10 s run of the
adopted 2x2 workload alternates Up and Down states, so its rates spread by
about 10 % from seed to seed.  The criterion is therefore applied to the
ensemble mean over the seeds of tests/golden/fp64_ensemble_2x2.json, whose
FP64 statistics the oracle wrote: the GPU runs exactly those networks (same
seeds: same synapses, initial state and external-input draws) through the
batched form, and the paired differences give the standard error of each
comparison, which is printed and must itself be small enough for the 2 % /
5 % bounds to mean something.
"""
import json
import os
import sys

import numpy as np
import pytest

from paper_1511_09325_gb300 import build as B
from paper_1511_09325_gb300 import snn
from paper_1511_09325_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import fp64_ensemble as F  # noqa: E402

pytestmark = pytest.mark.gpu

GOLD = os.path.join(HERE, "golden", "fp64_ensemble_2x2.json")


def _gpu_rows(prec, seeds, steps, chunk=256, drain_every=1000):
    """Per-seed statistics of the GPU path, members of one batch at a time."""
    n, s = W.neuron_params(), W.synapse_params()
    ncols = F.GRID[0] * F.GRID[1]
    rows = []
    for k0 in range(0, len(seeds), chunk):
        part = seeds[k0:k0 + chunk]
        grids = [F.GRID] * len(part)
        with snn.Batch(grids, [n] * len(part), [s] * len(part), part, prec) as b:
            for m in b.members:
                m.set_record_capacity(1 << 20)
            ts = [[] for _ in part]
            ids = [[] for _ in part]
            done = 0
            while done < steps:
                k = min(drain_every, steps - done)
                b.step(k)
                done += k
                for j, m in enumerate(b.members):
                    t, i, over = m.spikes()
                    assert not over
                    ts[j].append(t)
                    ids[j].append(i)
            for j, seed in enumerate(part):
                r = F.stats(np.concatenate(ts[j]), np.concatenate(ids[j]), n["n_per_col"],
                            n["n_exc"], ncols, F.TRANSIENT, F.TRANSIENT + F.STEPS)
                r["seed"] = seed
                rows.append(r)
    return rows


def _observables(rows, n):
    ncols = F.GRID[0] * F.GRID[1]
    secs = F.STEPS / 1000.0
    rate_e = np.array([r["spikes_e"] for r in rows]) / (n["n_exc"] * ncols * secs)
    rate_i = np.array([r["spikes_i"] for r in rows]) / ((n["n_per_col"] - n["n_exc"]) * ncols * secs)
    return {"rate_e": rate_e, "rate_i": rate_i,
            "cv_e": np.array([r["cv_e"] for r in rows]),
            "cv_i": np.array([r["cv_i"] for r in rows])}


@pytest.fixture(scope="module")
def gold():
    if not os.path.exists(GOLD):
        pytest.fail("missing %s (written by tests/golden/fp64_ensemble.py)" % GOLD)
    with open(GOLD) as f:
        return json.load(f)


@pytest.mark.parametrize("prec", ["f32w", "f16w"])
def test_ensemble_rates_and_isi_cv_against_fp64(gold, prec):
    B.build()
    snn.load()
    n = W.neuron_params()
    seeds = [r["seed"] for r in gold["rows"]]
    assert gold["steps"] == F.STEPS and gold["transient"] == F.TRANSIENT
    got = _observables(_gpu_rows(prec, seeds, F.TRANSIENT + F.STEPS), n)
    ref = _observables(gold["rows"], n)
    bounds = {"rate_e": 0.02, "rate_i": 0.02, "cv_e": 0.05, "cv_i": 0.05}
    report = {}
    for k, bound in bounds.items():
        g, f = got[k], ref[k]
        ok = np.isfinite(g) & np.isfinite(f)
        rel = g[ok].mean() / f[ok].mean() - 1.0
        se = np.std(g[ok] - f[ok], ddof=1) / np.sqrt(ok.sum()) / f[ok].mean()
        report[k] = (float(g[ok].mean()), float(f[ok].mean()), float(rel), float(se))
        # the comparison must resolve the bound: its standard error is well below it
        assert se < bound / 2.5, (prec, k, report[k])
        assert abs(rel) < bound, (prec, k, report[k])
    print("\n%s vs FP64 over %d seeds x %d ms: %s" % (
        prec, len(seeds), F.STEPS,
        ", ".join("%s %.4g/%.4g (%+.2f%% +- %.2f%%)" % (k, a, b, 100 * r, 100 * e)
                  for k, (a, b, r, e) in report.items())))


def test_rates_are_in_the_expected_regime(gold):
    """The Up/Down regime of the adopted workload: FP64 mean rates of a few
    to a few tens of Hz and bursty spike trains (ISI CV above 1)."""
    ref = _observables(gold["rows"], W.neuron_params())
    for k in ("rate_e", "rate_i"):
        assert 2.0 < ref[k].mean() < 40.0, (k, ref[k].mean())
    for k in ("cv_e", "cv_i"):
        assert np.nanmean(ref[k]) > 1.0, (k, np.nanmean(ref[k]))
