"""Pins of the oracle's network construction (Sec. 2 connectivity).

Sec. 2: columns of 1240 neurons (80 % excitatory) on a 2-D grid; each neuron
projects about 1240 synapses, part inside its own column and part to nearby
columns with a probability that decreases with distance, cut off to a 7x7
stencil.  The oracle's reading: exactly 1240 synapses, the first half local,
the rest over the stencil with P ~ exp(-r / 1.5), periodic boundaries, integer
delays uniform in 1..20, weights normal(mu, 0.25 mu) clipped to the source's
sign.  These tests check counts, ranges and distributions (chi-square), not
the oracle's own formulas.
"""
import math

import numpy as np
import pytest
import scipy.stats

from paper_1511_09325_gb300 import workloads as W

NPC = 1240


def _p(orc, gw, gh, seed=11):
    return orc.make_params(gw, gh, W.neuron_params(), W.synapse_params(), seed)


@pytest.fixture(scope="module")
def sample7(orc):
    """Synapses of 8 blocks of 24 neurons spread over a 7x7 grid (offsets never
    alias there); every block straddles an excitatory/inhibitory boundary."""
    p = _p(orc, 7, 7)
    starts = [c * NPC + 980 for c in (0, 6, 17, 24, 30, 41, 45, 48)]
    rows = [orc.synapses(p, "f64", j0, 24) for j0 in starts]
    out = {k: np.concatenate([r[k] for r in rows]) for k in rows[0]}
    out["j"] = np.concatenate([np.arange(j0, j0 + 24) for j0 in starts])
    return out


def test_row_structure(sample7):
    K, KL = 1240, 620
    for n, j in enumerate(sample7["j"]):
        tgt = sample7["target"][n]
        col_j, l_j = divmod(int(j), NPC)
        cx, cy = col_j % 7, col_j // 7
        tcol, tl = np.divmod(tgt, NPC)
        assert len(tgt) == K
        # local half: own column, no autapse
        assert np.all(tcol[:KL] == col_j)
        assert np.all(tl[:KL] != l_j)
        assert np.all((sample7["dx"][n][:KL] == 0) & (sample7["dy"][n][:KL] == 0))
        # remote half: the column drawn by the stencil offset, periodic
        dx, dy = sample7["dx"][n][KL:], sample7["dy"][n][KL:]
        assert np.all((np.abs(dx) <= 3) & (np.abs(dy) <= 3) & ((dx != 0) | (dy != 0)))
        assert np.all(tcol[KL:] == ((cy + dy) % 7) * 7 + (cx + dx) % 7)
        assert np.all((tl >= 0) & (tl < NPC))


def test_delays_uniform(sample7):
    d = sample7["delay"].ravel()
    assert d.min() == 1 and d.max() == 20
    counts = np.bincount(d, minlength=21)[1:]
    _, pval = scipy.stats.chisquare(counts)
    assert pval > 1e-4


def test_remote_offsets_follow_exponential_law(sample7):
    dx, dy = sample7["dx"][:, 620:].ravel(), sample7["dy"][:, 620:].ravel()
    idx = (dy + 3) * 7 + (dx + 3)
    counts = np.bincount(idx, minlength=49)
    ex = np.array([math.exp(-math.hypot(a - 3, b - 3) / 1.5) if (a, b) != (3, 3) else 0.0
                   for b in range(7) for a in range(7)])
    keep = ex > 0
    assert counts[~keep].sum() == 0
    exp_counts = ex[keep] / ex[keep].sum() * counts.sum()
    _, pval = scipy.stats.chisquare(counts[keep], exp_counts)
    assert pval > 1e-4


def test_local_targets_uniform(sample7):
    tl = (sample7["target"][:, :620] % NPC).ravel()
    counts = np.bincount(tl // 62, minlength=20)  # 20 bins of 62 neurons
    _, pval = scipy.stats.chisquare(counts)
    assert pval > 1e-4


def test_weight_distribution_and_dale(sample7):
    w = sample7["w"]
    exc = (sample7["j"] % NPC) < 992
    we, wi = w[exc].ravel(), w[~exc].ravel()
    assert np.all(we >= 0) and np.all(wi <= 0)
    for ws, mu in ((we, 0.4), (wi, -1.6)):
        mu32 = float(np.float32(mu))
        sd = abs(mu32) * 0.25
        assert abs(ws.mean() - mu32) < 5 * sd / math.sqrt(len(ws))
        assert ws.std() / abs(mu32) == pytest.approx(0.25, rel=0.02)
    # quantiles of Q span about +-4.3 sigma: the clip at zero never bites
    assert we.min() > 0.4 * (1 - 0.25 * 4.4)


def test_fixed_point_and_half_weights(orc):
    p = _p(orc, 3, 2)
    s64 = orc.synapses(p, "f64", 100, 3)
    s32 = orc.synapses(p, "f32w", 100, 3)
    s16 = orc.synapses(p, "f16w", 100, 3)
    assert np.array_equal(s64["target"], s32["target"])
    assert np.array_equal(s64["delay"], s16["delay"])
    w32 = s64["w"].astype(np.float32)
    assert np.array_equal(s32["w"], w32.astype(np.float64))
    assert np.array_equal(s32["wfx"], np.rint(w32 * np.float32(65536)).astype(np.int32))
    w16 = s64["w"].astype(np.float16)  # numpy rounds double -> half to nearest even
    assert np.array_equal(s16["w"], w16.astype(np.float64))
    assert np.array_equal(s16["wfx"], np.rint(w16.astype(np.float32) * np.float32(65536)).astype(np.int32))


def test_single_column_grid_keeps_every_target_local(orc):
    s = orc.synapses(_p(orc, 1, 1), "f32w", 0, 40)
    assert np.all((s["target"] >= 0) & (s["target"] < NPC))


def test_small_grid_wraps_offsets(orc):
    p = _p(orc, 2, 3)
    s = orc.synapses(p, "f32w", 5 * NPC + 7, 1)  # column 5 = (x 1, y 2)
    tcol = s["target"][0] // NPC
    dx, dy = s["dx"][0], s["dy"][0]
    assert np.all(tcol[620:] == ((2 + dy[620:]) % 3) * 2 + (1 + dx[620:]) % 2)


def test_construction_is_deterministic_and_seeded(orc):
    a = orc.synapses(_p(orc, 3, 3, seed=4), "f32w", 500, 2)
    b = orc.synapses(_p(orc, 3, 3, seed=4), "f32w", 500, 2)
    c = orc.synapses(_p(orc, 3, 3, seed=5), "f32w", 500, 2)
    assert np.array_equal(a["target"], b["target"]) and np.array_equal(a["wfx"], b["wfx"])
    assert not np.array_equal(a["target"], c["target"])


def test_external_counts_are_poisson(orc):
    p = _p(orc, 2, 2)
    k = orc.ext_counts(p, 0, 4960, 0, 20).ravel()
    lam = 2.5
    assert abs(k.mean() - lam) < 5 * math.sqrt(lam / len(k))
    hist = np.bincount(k, minlength=12)[:12]
    pk = scipy.stats.poisson.pmf(np.arange(12), lam)
    pk[-1] += scipy.stats.poisson.sf(11, lam)
    hist[-1] += int((k >= 12).sum())
    _, pval = scipy.stats.chisquare(hist, pk * len(k))
    assert pval > 1e-4
