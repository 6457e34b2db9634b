"""Dense restatement of the network step, used by the brute-force and the
partitioned (multi-rank) pins of the oracle.

The recurrent input of step t is written out as a sum over delays,
I(t) = sum_d A_d s(t - d), with A_d the synapse matrix of delay d (scipy
sparse, rows = targets) and s the spike vector; the neuron update is restated
in numpy float32 with an exactly rounded fused multiply-add.  The synapse list
and the external counts come from the oracle's generator, which the table and
construction tests pin separately.
"""
import numpy as np
import scipy.sparse as sp


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


class DenseNet:
    """Per-delay synapse matrices, tables and initial state of a network."""

    def __init__(self, orc, p, mode):
        self.p, self.mode = p, mode
        N = p.grid_w * p.grid_h * p.n_per_col
        self.N = N
        if p.connectivity == 1:   # the paper's law: variable out-degree
            syn = orc.paper_synapses(p, mode, 0, N)
            src = np.repeat(np.arange(N), syn["count"])
        else:
            syn = orc.synapses(p, mode, 0, N)
            src = np.repeat(np.arange(N), p.k_out)
        self.tb = orc.tables(p)
        self.D = p.d_max
        self.A = []
        for d in range(1, self.D + 1):
            m = syn["delay"].ravel() == d
            vals = syn["wfx"].ravel()[m] if mode != "f64" else syn["w"].ravel()[m]
            self.A.append(sp.csr_matrix((vals.astype(np.int64 if mode != "f64" else np.float64),
                                         (syn["target"].ravel()[m], src[m])), shape=(N, N)))
        key = [p.seed & 0xFFFFFFFF, p.seed >> 32]
        self.u = np.array([orc.philox([i >> 2, 0, 3, 0], key)[i & 3] for i in range(N)], np.uint64)
        self.exc = (np.arange(N) % p.n_per_col) < p.n_exc


def _reference(orc, p, mode, T):
    return simulate(orc, DenseNet(orc, p, mode), T)


def simulate(orc, net, T, rows=None, exchange=None):
    """Run T steps for the neurons `rows` (all if None).  `exchange(spk)`
    turns the local spike vector into the global one (identity when one
    process owns every neuron)."""
    p, mode, N, D, A, tb = net.p, net.mode, net.N, net.D, net.A, net.tb
    rows = np.arange(N) if rows is None else np.asarray(rows)
    A = [a[rows] for a in A]
    u = net.u[rows]
    exc = net.exc[rows]
    M = len(rows)
    # initial potentials: uniform [0, theta) with 24-bit resolution (INIT stream)
    if mode == "f64":
        V = float(np.float32(p.theta)) * ((u >> 8).astype(np.float64) * 2.0 ** -24)
        c = np.zeros(M)
    else:
        V = np.float32(p.theta) * ((u >> 8).astype(np.float32) * np.float32(2.0 ** -24))
        c = np.zeros(M, np.float32)
    r = np.zeros(M, np.int64)
    hist = [np.zeros(N, bool) for _ in range(D)]  # hist[d-1] = global spikes of step t-d
    raster = []
    kall = orc.ext_counts(p, 0, N, 0, T).astype(np.int64)[:, rows]
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
        raster.extend((t, int(rows[i])) for i in np.flatnonzero(spk))
        local = np.zeros(N, bool)
        local[rows[spk]] = True
        glob = local if exchange is None else exchange(local)
        hist = [glob] + hist[:-1]
    return raster, np.asarray(V, np.float64), np.asarray(c, np.float64), r


