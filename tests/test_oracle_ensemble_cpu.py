"""The FP64 ensemble statistics (tests/golden/fp64_ensemble_2x2.json) and the
observable that computes them, checked without a GPU.

* `stats` on hand-made rasters: spike counts per population and the ISI CV
  (population standard deviation over mean of a neuron's intervals, averaged
  over the neurons with at least 5 intervals) against values worked out by
  hand, the window bounds, and neurons with too few intervals left out.
* The stored file: one row per seed, and the first seed's row recomputed by
  the oracle equals the stored one exactly (the file was written by the
  oracle, deterministically).
"""
import json
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import fp64_ensemble as F  # noqa: E402

GOLD = os.path.join(HERE, "golden", "fp64_ensemble_2x2.json")


def test_stats_by_hand():
    # 2 columns of 4 neurons, 3 excitatory per column; window [10, 100)
    # neuron 0 (E): spikes 10, 20, 30, 40, 50, 60 -> 5 ISIs of 10: CV 0
    # neuron 3 (I): spikes 10, 12, 20, 22, 30, 32 -> ISIs 2,8,2,8,2: mean 4.4,
    #               population sd sqrt(((2.4^2)*3 + (3.6^2)*2)/5) = 2.939..
    # neuron 5 (E): spikes 11, 31, 61, 91 -> 3 ISIs: left out of the CV
    # neuron 1 (E): one spike at 5 (outside the window) and one at 100 (outside)
    t = [10, 20, 30, 40, 50, 60, 10, 12, 20, 22, 30, 32, 11, 31, 61, 91, 5, 100]
    i = [0] * 6 + [3] * 6 + [5] * 4 + [1, 1]
    r = F.stats(t, i, 4, 3, 2, 10, 100)
    assert r["spikes_e"] == 10 and r["spikes_i"] == 6
    assert r["n_cv_e"] == 1 and r["cv_e"] == 0.0
    isi = np.array([2, 8, 2, 8, 2], float)
    assert r["n_cv_i"] == 1
    assert r["cv_i"] == pytest.approx(isi.std() / isi.mean(), rel=1e-12)
    assert r["cv_i"] == pytest.approx(np.sqrt((3 * 2.4 ** 2 + 2 * 3.6 ** 2) / 5) / 4.4, rel=1e-12)


def test_stats_unordered_input_and_means_over_neurons():
    # two E neurons with CV 0 and 0.5; input in random order
    a = [0, 10, 20, 30, 40, 50]                # ISIs all 10
    b = [0, 10, 30, 40, 60, 70]                # ISIs 10,20,10,20,10: mean 14, sd 4.899
    t = np.array(a + b)
    i = np.array([0] * 6 + [1] * 6)
    p = np.random.default_rng(3).permutation(len(t))
    r = F.stats(t[p], i[p], 10, 8, 1, 0, 1000)
    isi_b = np.diff(b).astype(float)
    assert r["cv_e"] == pytest.approx((0.0 + isi_b.std() / isi_b.mean()) / 2, rel=1e-12)
    assert np.isnan(r["cv_i"]) and r["n_cv_i"] == 0


@pytest.mark.skipif(not os.path.exists(GOLD), reason="ensemble file not written yet")
def test_stored_ensemble_reproduces(orc):
    with open(GOLD) as f:
        g = json.load(f)
    assert g["mode"] == "f64" and g["n_seeds"] == len(g["rows"]) >= 256
    assert [r["seed"] for r in g["rows"]] == list(range(g["seed0"], g["seed0"] + g["n_seeds"]))
    assert g["steps"] == F.STEPS and g["transient"] == F.TRANSIENT
    row = F._one(g["seed0"])
    assert row == g["rows"][0]
