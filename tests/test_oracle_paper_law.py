"""Pins of the oracle's second connectivity law: Sec. 2's own description
(a synapse to every other neuron of the column with probability 0.8; to
every neuron of a column at grid distance r with probability
0.05 exp(-r^2 / 2), offsets where that is below 1/1000 dropped).

The law is a reading (the paper's numbers do not add up: its "7x7" stencil is
a 5x5 one without corners under its own cut-off, and the expected out-degree
is ~1307, not 1239-1245), so the pins check the oracle against the law as
stated: the kept offsets and thresholds, the binomial statistics of rows, and
a dense brute-force restatement of the network step on such rows.
"""
import numpy as np
import pytest

from paper_1511_09325_gb300 import workloads as W

from dense_model import _reference

PAPER = dict(connectivity=1)


def _params(orc, gw, gh, seed, **nov):
    return orc.make_params(gw, gh, W.neuron_params(**nov), W.synapse_params(**PAPER), seed)


def test_kept_offsets_and_thresholds(orc):
    """The 20 offsets with 0.05 exp(-r^2/2) >= 1e-3 (r <= sqrt 5), dy-major,
    and floor(P 2^32) thresholds."""
    t = orc.paper_tables(_params(orc, 3, 3, 1))
    want = [(dx, dy) for dy in range(-3, 4) for dx in range(-3, 4)
            if (dx, dy) != (0, 0) and 0.05 * np.exp(-(dx * dx + dy * dy) / 2.0) >= 1e-3]
    assert list(zip(t["dx"].tolist(), t["dy"].tolist())) == want and len(want) == 20
    a = np.float64(np.float32(0.05))  # the parameter is a float
    p = a * np.exp(-(t["dx"].astype(float) ** 2 + t["dy"].astype(float) ** 2) / 2.0)
    assert np.all(np.abs(t["thr"].astype(np.float64) - np.floor(p * 2.0 ** 32)) <= 1)
    assert t["local_thr"] == int(np.floor(np.float64(np.float32(0.8)) * 2.0 ** 32))
    assert t["n_cand"] == 1239 + 20 * 1240


def test_row_statistics(orc):
    """1000 rows of a 5x5 grid: local, per-offset and total counts against
    their binomial means (4 standard errors), no autapse, delays uniform."""
    p = _params(orc, 5, 5, 4)
    t = orc.paper_tables(p)
    n_rows = 1000
    j0 = 7 * 1240 + 17
    s = orc.paper_synapses(p, "f32w", j0, n_rows)
    cnt = s["count"]
    src = np.repeat(np.arange(j0, j0 + n_rows), cnt)
    local = (s["dx"] == 0) & (s["dy"] == 0)
    assert not np.any(s["target"][local] == src[local])
    assert np.all(s["target"][local] // 1240 == src[local] // 1240)
    pl = np.float64(np.float32(0.8))
    n_loc = np.bincount(np.repeat(np.arange(n_rows), cnt)[local], minlength=n_rows)
    se = np.sqrt(1239 * pl * (1 - pl) / n_rows)
    assert abs(n_loc.mean() - 1239 * pl) < 4 * se
    pr = t["thr"].astype(np.float64) / 2.0 ** 32
    mean_deg = 1239 * pl + 1240 * pr.sum()
    var_deg = 1239 * pl * (1 - pl) + 1240 * np.sum(pr * (1 - pr))
    assert abs(cnt.mean() - mean_deg) < 4 * np.sqrt(var_deg / n_rows)
    assert abs(cnt.var() - var_deg) < 0.25 * var_deg
    # every remote offset with its own probability (one-sided 4-sigma each)
    for m in range(len(pr)):
        k = np.sum((s["dx"] == t["dx"][m]) & (s["dy"] == t["dy"][m]))
        mu = n_rows * 1240 * pr[m]
        assert abs(k - mu) < 4 * np.sqrt(mu * (1 - pr[m])) + 1, (m, k, mu)
    # targets of a remote offset land in the right column
    rem = ~local
    col = src[rem] // 1240
    cx, cy = col % 5, col // 5
    tcol = s["target"][rem] // 1240
    assert np.array_equal(tcol, ((cy + s["dy"][rem]) % 5) * 5 + (cx + s["dx"][rem]) % 5)
    d = np.bincount(s["delay"] - 1, minlength=20)
    e = d.sum() / 20
    assert np.sum((d - e) ** 2 / e) < 50  # chi2, 19 dof: p ~ 1e-4


def test_rows_are_reproducible_and_independent(orc):
    p = _params(orc, 2, 2, 9)
    a = orc.paper_synapses(p, "f32w", 100, 3)
    b = orc.paper_synapses(p, "f32w", 101, 1)
    n0 = a["count"][0]
    assert b["count"][0] == a["count"][1]
    assert np.array_equal(b["target"], a["target"][n0:n0 + a["count"][1]])
    c = orc.paper_synapses(_params(orc, 2, 2, 10), "f32w", 101, 1)
    assert not np.array_equal(c["target"][:100], b["target"][:100])


def test_network_matches_dense_reference(orc):
    """The event-driven oracle under the paper law equals the dense per-delay
    restatement bit for bit (100 neurons per column, 2x3 grid, 80 steps)."""
    n = W.neuron_params(n_per_col=100, n_exc=80, nu_ext_kHz=3.0)
    s = W.synapse_params(connectivity=1)
    p = orc.make_params(2, 3, n, s, 19)
    raster, V, c, r = _reference(orc, p, "f32w", 80)
    o = orc.run(p, "f32w", 80)
    assert len(raster) > 100
    assert list(zip(o["t"].tolist(), o["i"].tolist())) == raster
    assert np.array_equal(o["v"], V)
