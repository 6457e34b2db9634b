"""Pins of the oracle's random generator and FP64 tables.

Each check compares the oracle with something other than itself: published
known-answer vectors (Philox4x32-10), library routines (scipy's normal
quantile, Poisson CDF and matrix exponential) and closed-form invariants of
the stencil distribution.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.special
import scipy.stats

from paper_1511_09325_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _params(orc, gw=2, gh=2, seed=1, **over):
    n = W.neuron_params(**{k: v for k, v in over.items() if k in W.NEURON})
    s = W.synapse_params(**{k: v for k, v in over.items() if k in W.SYNAPSE})
    return orc.make_params(gw, gh, n, s, seed)


def test_philox_known_answers(orc):
    """Philox4x32-10 against the Random123 known-answer vectors (SC'11 generator)."""
    rows = [l.split() for l in open(os.path.join(GOLD, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = orc.philox(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_stencil_distribution(orc):
    """Remote offsets (Sec. 2: probability decreasing with column distance).

    Invariants: 48 offsets of the 7x7 cut-off without the centre, dy-major and
    dx ascending; shares depend on distance only (the 8 symmetries of the
    square); the share ratio between distances r1 and r2 is exp(-(r1-r2)/1.5);
    the shares sum to one.
    """
    t = orc.tables(_params(orc))
    dx, dy, thr = t["off_dx"], t["off_dy"], t["stencil_thr"].astype(np.float64)
    assert len(dx) == 48
    order = [(int(a), int(b)) for a, b in zip(dy, dx)]
    assert order == sorted(order)
    assert (0, 0) not in order
    assert max(abs(dx).max(), abs(dy).max()) == 3
    share = np.diff(np.concatenate([[0.0], thr])) / 2.0 ** 32
    assert abs(share.sum() - 1.0) < 1e-12
    assert np.all(np.diff(thr) > 0)
    r = np.hypot(dx, dy)
    by = {}
    for i in range(48):
        key = (min(abs(dx[i]), abs(dy[i])), max(abs(dx[i]), abs(dy[i])))
        by.setdefault(key, []).append(share[i])
    for vals in by.values():
        assert max(vals) - min(vals) < 2.0 ** -31
    i1 = int(np.argmin(np.where(r == 1.0, 0, 1)))
    for i in range(48):
        # shares are quantised to 2^-32
        assert abs(share[i] - share[i1] * math.exp(-(r[i] - 1.0) / 1.5)) < 3.0 * 2.0 ** -32


def test_stencil_flat_limit(orc):
    """With a very long length constant every remote column is equally likely."""
    t = orc.tables(_params(orc, lambda_cols=1e30))
    share = np.diff(np.concatenate([[0.0], t["stencil_thr"].astype(np.float64)])) / 2.0 ** 32
    assert np.allclose(share, 1.0 / 48.0, atol=2.0 ** -31)


@pytest.mark.parametrize("nu", [2.5, 1.5, 3.5, 0.0, 25.0])
def test_poisson_table(orc, nu):
    """External input counts: Poisson(nu_ext * 1 ms) by CDF inversion.

    The quantised CDF equals scipy's Poisson CDF to 2^-32; mean and variance of
    the quantised law equal lambda; the table saturates at 2^32.
    """
    t = orc.tables(_params(orc, nu_ext_kHz=nu))
    thr = t["pois_thr"].astype(np.float64)
    lam = float(np.float32(nu))
    assert thr[-1] == 2.0 ** 32
    assert np.all(np.diff(thr) >= 0)
    ks = np.arange(len(thr))
    ref = scipy.stats.poisson.cdf(ks[:-1], lam) if lam > 0 else np.ones(len(thr) - 1)
    assert np.all(np.abs(thr[:-1] / 2.0 ** 32 - ref) < 2.0 ** -32 + 1e-13)
    pk = np.diff(np.concatenate([[0.0], thr])) / 2.0 ** 32
    mean = float((pk * ks).sum())
    var = float((pk * ks * ks).sum()) - mean ** 2
    assert abs(mean - lam) < 1e-7 * max(lam, 1)
    assert abs(var - lam) < 1e-6 * max(lam, 1)
    if nu == 2.5:
        assert len(thr) == 18  # k_max = 17 for lambda = 2.5


def test_normal_quantiles(orc):
    """Q[m] = Phi^-1((m + 0.5) / 65536) against scipy.special.ndtri; symmetric."""
    q = orc.tables(_params(orc))["q"]
    m = np.arange(65536)
    ref = scipy.special.ndtri((m + 0.5) / 65536.0)
    # the quantile's slope grows in the tails, where one ulp of erfc moves z most
    assert np.max(np.abs(q - ref)) < 5e-12
    assert np.max(np.abs(q[1000:-1000] - ref[1000:-1000])) < 1e-13
    assert np.max(np.abs(q + q[::-1])) < 5e-12
    assert q[0] == pytest.approx(-4.3249, abs=1e-4)  # the table spans +-4.32 sigma


def test_propagators_match_matrix_exponential(orc):
    """Exact 1 ms propagator of dV/dt = -V/tau_m - g_c c, dc/dt = -c/tau_c.

    The oracle's closed form against scipy.linalg.expm of the system matrix.
    """
    for gc, tc in [(0.02, 500.0), (0.5, 37.0), (0.0, 500.0)]:
        p = _params(orc, gc_exc=gc, tau_c=tc)
        t = orc.tables(p)
        tm = float(np.float32(20.0))
        g = float(np.float32(gc))
        tcf = float(np.float32(tc))
        A = np.array([[-1.0 / tm, -g], [0.0, -1.0 / tcf]])
        M = scipy.linalg.expm(A * 1.0)
        assert t["pvv"] == pytest.approx(M[0, 0], rel=1e-14)
        assert t["pcc"] == pytest.approx(M[1, 1], rel=1e-14)
        assert t["pvc_e"] == pytest.approx(M[0, 1], rel=1e-12, abs=1e-300)
        assert t["pvc_i"] == 0.0


def test_fixed_point_constants(orc):
    t = orc.tables(_params(orc))
    assert t["jx"] == 26214          # rint(0.4 mV * 2^16)
    assert t["nref"] == 2            # 2 ms refractory at h = 1 ms
    assert t["k_local"] == 620       # half of 1240 synapses local


def test_paper_table1_sizes():
    """Sec. 2, Table 1: neurons and synapses of the three grids.

    N = W * H * 1240; recurrent synapses N * 1240; total equivalent synapses
    N * (1240 + 540).  The paper rounds to one decimal (its 'total' column is
    rounded inconsistently, e.g. 20.34 G printed as 20.4 G), so the printed
    values are matched to within 0.1 of their unit.
    """
    rows = [l.split() for l in open(os.path.join(GOLD, "table1_problem_sizes.txt"))
            if l.strip() and not l.startswith("#")]
    for gw, gh, cols, nM, recG, totG in rows:
        gw, gh, cols = int(gw), int(gh), int(cols)
        n = W.n_neurons(gw, gh)
        assert gw * gh == cols
        assert abs(n / 1e6 - float(nM)) <= 0.05 + 1e-9
        assert abs(n * 1240 / 1e9 - float(recG)) <= 0.05 + 1e-9
        assert abs(n * (1240 + 540) / 1e9 - float(totG)) <= 0.1 + 1e-9
    assert W.n_neurons(96, 96) * 1240 == 14170521600
    assert W.n_neurons(48, 48) * 1240 == 3542630400
    assert W.n_neurons(24, 24) * 1240 == 885657600
