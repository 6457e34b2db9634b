"""Brute-force pin of the oracle's event-driven network step.

On one column (1240 neurons) the recurrent input of step t is written out as a
dense sum over delays, I(t) = sum_d A_d s(t - d), with A_d the synapse matrix of
delay d (scipy sparse) and s the spike vector, and the neuron update is
restated in numpy float32 with an exactly rounded fused multiply-add.  The
synapse list and the external counts come from the oracle's generator, which
the table and construction tests pin separately.  The event-driven oracle
(ring buffer of d_max + 1 slots, synapses regenerated per spike) must match
this bit for bit in the fixed-point modes and to rounding in FP64.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_1511_09325_gb300 import workloads as W

NPC = 1240


def fma32(a, b, c):
    """float32 fma(a, b, c) with a single rounding, vectorised.

    a*b is exact in float64; the float64 sum s can only round the float32
    result the wrong way when it lands exactly on a float32 midpoint, which is
    resolved with the two-sum error term.
    """
    a = a.astype(np.float64)
    b = np.float64(b)
    p = a * b
    cc = c.astype(np.float64)
    s = p + cc
    bb = s - p
    err = (p - (s - bb)) + (cc - bb)
    r = s.astype(np.float32)
    d = s - r.astype(np.float64)
    toward = np.where(d > 0, np.float32(np.inf), np.float32(-np.inf)).astype(np.float32)
    nb = np.nextafter(r, toward)
    mid = (d != 0) & (2.0 * d == nb.astype(np.float64) - r.astype(np.float64))
    fix = mid & (err != 0)
    up = np.maximum(r, nb)
    lo = np.minimum(r, nb)
    r = np.where(fix & (err > 0), up, np.where(fix & (err < 0), lo, r))
    return r.astype(np.float32)


def _reference(orc, p, mode, T):
    N = p.grid_w * p.grid_h * p.n_per_col
    syn = orc.synapses(p, mode, 0, N)
    tb = orc.tables(p)
    D = p.d_max
    src = np.repeat(np.arange(N), p.k_out)
    A = []
    for d in range(1, D + 1):
        m = syn["delay"].ravel() == d
        vals = syn["wfx"].ravel()[m] if mode != "f64" else syn["w"].ravel()[m]
        A.append(sp.csr_matrix((vals.astype(np.int64 if mode != "f64" else np.float64),
                                (syn["target"].ravel()[m], src[m])), shape=(N, N)))
    # initial potentials: uniform [0, theta) with 24-bit resolution (INIT stream)
    key = [p.seed & 0xFFFFFFFF, p.seed >> 32]
    u = np.array([orc.philox([i >> 2, 0, 3, 0], key)[i & 3] for i in range(N)], np.uint64)
    exc = (np.arange(N) % p.n_per_col) < p.n_exc
    if mode == "f64":
        V = float(np.float32(p.theta)) * ((u >> 8).astype(np.float64) * 2.0 ** -24)
        c = np.zeros(N)
    else:
        V = np.float32(p.theta) * ((u >> 8).astype(np.float32) * np.float32(2.0 ** -24))
        c = np.zeros(N, np.float32)
    r = np.zeros(N, np.int64)
    hist = [np.zeros(N, bool) for _ in range(D)]  # hist[d-1] = spikes of step t-d
    raster = []
    kall = orc.ext_counts(p, 0, N, 0, T).astype(np.int64)
    for t in range(T):
        k = kall[t]
        if mode == "f64":
            I = sum(A[d] @ hist[d].astype(np.float64) for d in range(D)) + k * float(np.float32(p.j_ext))
        else:
            I = sum(A[d] @ hist[d].astype(np.int64) for d in range(D)) + k * tb["jx"]
            assert np.all(np.abs(I) < 2 ** 31)
        refr = r > 0
        r = np.where(refr, r - 1, r)
        if mode == "f64":
            Vn = np.where(refr, float(np.float32(p.v_reset)), V + I)
            spk = (~refr) & (Vn >= float(np.float32(p.theta)))
            Vn = np.where(spk, float(np.float32(p.v_reset)), Vn)
            c = np.where(spk, c + float(np.float32(p.dc)), c)
            pvc = np.where(exc, tb["pvc_e"], tb["pvc_i"])
            V = pvc * c + tb["pvv"] * Vn
            c = c * tb["pcc"]
        else:
            add = V + (I.astype(np.float32) * np.float32(2.0 ** -16))
            Vn = np.where(refr, np.float32(p.v_reset), add).astype(np.float32)
            spk = (~refr) & (Vn >= np.float32(p.theta))
            Vn = np.where(spk, np.float32(p.v_reset), Vn).astype(np.float32)
            c = np.where(spk, c + np.float32(p.dc), c).astype(np.float32)
            pvc_e, pvc_i = np.float32(tb["pvc_e"]), np.float32(tb["pvc_i"])
            prod = (Vn * np.float32(tb["pvv"])).astype(np.float32)
            V = np.where(exc, fma32(c, pvc_e, prod), fma32(c, pvc_i, prod)).astype(np.float32)
            c = (c * np.float32(tb["pcc"])).astype(np.float32)
        r = np.where(spk, tb["nref"], r)
        raster.extend((t, int(i)) for i in np.flatnonzero(spk))
        hist = [spk] + hist[:-1]
    return raster, np.asarray(V, np.float64), np.asarray(c, np.float64), r


@pytest.mark.parametrize("mode", ["f32w", "f16w", "f64"])
def test_one_column_matches_dense_reference(orc, mode):
    p = orc.make_params(1, 1, W.neuron_params(), W.synapse_params(), 7)
    T = 160
    raster, V, c, r = _reference(orc, p, mode, T)
    o = orc.run(p, mode, T)
    got = list(zip(o["t"].tolist(), o["i"].tolist()))
    assert len(raster) > 500  # the initial volley and its echoes
    assert got == raster
    if mode == "f64":
        assert np.allclose(o["v"], V, rtol=0, atol=1e-9)
        assert np.allclose(o["c"], c, rtol=0, atol=1e-12)
    else:
        assert np.array_equal(o["v"], V)
        assert np.array_equal(o["c"], c)
    assert np.array_equal(o["r"].astype(np.int64), r)


def test_two_by_three_grid_matches_dense_reference(orc):
    """Periodic wrap on a grid narrower than the stencil, delays over the ring."""
    n = W.neuron_params(n_per_col=100, n_exc=80, nu_ext_kHz=3.0)
    s = W.synapse_params(k_out=120)
    p = orc.make_params(2, 3, n, s, 19)
    raster, V, c, r = _reference(orc, p, "f32w", 120)
    o = orc.run(p, "f32w", 120)
    assert len(raster) > 100
    assert list(zip(o["t"].tolist(), o["i"].tolist())) == raster
    assert np.array_equal(o["v"], V)


def test_fma32_emulation_against_known_midpoint():
    """The fma emulation resolves a double-rounding midpoint correctly."""
    a = np.array([1.0 + 2.0 ** -12], np.float32)
    b = np.float32(1.0 + 2.0 ** -12)
    # a*b = 1 + 2^-11 + 2^-24 exactly, a float32 midpoint; 2^-60 is lost in
    # the float64 sum but must still push the single rounding upwards
    c = np.array([2.0 ** -60], np.float32)
    got = fma32(a, b, c)[0]
    want = np.nextafter(np.float32(1.0 + 2.0 ** -11), np.float32(2.0))
    assert got == want
