"""FP64 oracle of the relaxed (differentiable) network and of its gradient.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper has nothing on gradients (arxiv 1511.09325 describes the spiking
simulator only, Sec. 2).  This file restates the reading adopted for a
surrogate-gradient extension of the Sec. 2 network, in plain numpy/scipy:

  per neuron i of population p_i (E: l < n_exc), step t = 0 .. T-1:
    X_E,i(t) = sum over synapses (j -> i, delay d, weight w), j in E, of w s_j(t-d)
    X_I,i(t) = the same over inhibitory sources j
    I_i(t)   = a[E][p_i] X_E,i + a[I][p_i] X_I,i + J (lam + sqrt(lam) xi_i(t))
    g_i(t)   = max(0, 1 - s_i(t-1) - s_i(t-2))                 refractory gate
    U_i(t)   = g (V_i + I_i) + (1 - g) V_reset
    s_i(t)   = sigmoid(beta (U_i - theta))                       soft spike
    V'       = U - s (U - V_reset);  c' = c + dc s               soft reset, calcium
    V_i(t+1) = P_VV V' + P_VC,i c';  c_i(t+1) = P_CC c'
  with lam = nu_ext h, J = j_ext, P_VC,E = g_c kappa, P_VC,I = gc_inh kappa and
  kappa = -tau_m tau_c / (tau_c - tau_m) (P_CC - P_VV) (the exact 1 ms propagator
  of Sec. 2's LIF + calcium SFA, as in the spiking oracle).  s(t < 0) = 0,
  V(0) is the spiking network's initial state, c(0) = 0.  xi_i(t) is the normal
  draw of Philox stream SURR (``oracle.surr_xi``).  When beta -> infinity and
  the external input is the spiking network's Poisson input, the recursion is
  the spiking model itself (the gate then clamps refractory neurons to V_reset).

  loss = (r_E - r_E*)^2 + (r_I - r_I*)^2,  r_X = 1000 / (T N_X) sum_t sum_{i in X} s_i(t)
  parameters theta = (a_EE, a_EI, a_IE, a_II, g_c, nu_ext); a_XY scales the
  synapses from population X onto population Y.

``forward`` runs the recursion and keeps every intermediate; ``backward`` is
the reverse-mode recursion (adjoint of every line above, in reverse order),
written out by hand; the adjoint of the delayed delivery is the transposed
matrix product, i.e. a gather over each neuron's outgoing synapses.

Pins (tests, no GPU): soft-mode gradient = central finite differences; the
beta -> infinity limit = the spiking C oracle's raster; reverse recursion =
forward-mode tangents in both modes.  The hard mode's surrogate derivative
itself is a choice, not a derivative of the forward: the paper has no
gradient to compare with (parity unpinned by the paper).
"""
import numpy as np
import scipy.sparse as sp

from . import init_v, surr_xi, synapses, tables

PARAMS = ("a_EE", "a_EI", "a_IE", "a_II", "g_c", "nu_ext")


def fma32(a, b, c):
    """float32 fma(a, b, c) with one rounding (vectorised): a * b is exact in
    float64, and a float64 sum that lands on a float32 rounding midpoint is
    resolved with its two-sum error term."""
    a = np.asarray(a, np.float64)
    p = a * np.float64(b)
    cc = np.asarray(c, np.float64)
    s = p + cc
    bb = s - p
    err = (p - (s - bb)) + (cc - bb)
    r = s.astype(np.float32)
    d = s - r.astype(np.float64)
    toward = np.where(d > 0, np.float32(np.inf), np.float32(-np.inf)).astype(np.float32)
    nb = np.nextafter(r, toward)
    mid = (d != 0) & (2.0 * d == nb.astype(np.float64) - r.astype(np.float64))
    fix = mid & (err != 0)
    r = np.where(fix & (err > 0), np.maximum(r, nb), np.where(fix & (err < 0), np.minimum(r, nb), r))
    return r.astype(np.float32)


def _sigmoid(x):
    e = np.exp(-np.abs(x))
    return np.where(x >= 0, 1.0 / (1.0 + e), e / (1.0 + e))


class SoftNet:
    """Synapse matrices, tables and initial state of one network.

    weights: "fixed" (the spiking F32W path's round(w * 2^16) / 2^16, what the
    GPU delivers) or "exact" (the unrounded FP64 weights of the F64 mode).
    """

    def __init__(self, p, weights="fixed"):
        self.p = p
        npc, nexc = p.n_per_col, p.n_exc
        N = p.grid_w * p.grid_h * npc
        self.N, self.D = N, p.d_max
        syn = synapses(p, "f32w" if weights == "fixed" else "f64", 0, N)
        w = syn["wfx"].ravel() / 65536.0 if weights == "fixed" else syn["w"].ravel()
        tgt = syn["target"].ravel()
        dly = syn["delay"].ravel().astype(np.int64)
        src = np.repeat(np.arange(N), p.k_out)
        self.exc = (np.arange(N) % npc) < nexc
        sexc = self.exc[src]
        D = self.D
        # forward: hstack over delays, column (d - 1) N + j holds source j at delay d
        cols = (dly - 1) * N + src
        self.M = {pop: sp.csr_matrix((w[m], (tgt[m], cols[m])), shape=(N, D * N))
                  for pop, m in (("E", sexc), ("I", ~sexc))}
        # backward: per-delay transposes (sources x targets)
        self.WT = [sp.csr_matrix((w[dly == d], (src[dly == d], tgt[dly == d])), shape=(N, N))
                   for d in range(1, D + 1)]
        tb = tables(p)
        self.pvv, self.pcc = tb["pvv"], tb["pcc"]
        tm, tc = float(np.float32(p.tau_m)), float(np.float32(p.tau_c))
        self.kappa = -tm * tc / (tc - tm) * (self.pcc - self.pvv)
        self.v0 = init_v(p, "f64", 0, N)

    def forward(self, theta, T, beta=5.0, targets=(3.0, 8.0), ext=None, hard=False):
        """Loss, rates and the tape of the recursion.  ext: None for the
        Gaussian input, else an explicit [T, N] array of external input (mV).
        hard: spikes are s = [U >= theta] (the spiking model) and the backward
        uses the surrogate derivative 1 / (1 + beta |U - theta|)^2."""
        p, N, D, exc = self.p, self.N, self.D, self.exc
        aEE, aEI, aIE, aII, gc, nu = (float(x) for x in theta)
        aE = np.where(exc, aEE, aEI)   # scale of excitatory sources onto i
        aI = np.where(exc, aIE, aII)   # scale of inhibitory sources onto i
        h = float(p.h)
        lam = nu * h
        J = float(np.float32(p.j_ext))
        vr, th, dc = (float(np.float32(x)) for x in (p.v_reset, p.theta, p.dc))
        pvc = np.where(exc, gc * self.kappa, float(np.float32(p.gc_inh)) * self.kappa)
        xi = surr_xi(p, 0, N, 0, T) if ext is None else None
        hist = np.zeros((D, N))       # hist[d - 1] = s(t - d)
        s1, s2 = np.zeros(N), np.zeros(N)   # s(t - 1), s(t - 2)
        V, c = self.v0.copy(), np.zeros(N)
        keys = ("V", "I", "U", "g", "s", "cp", "XE", "XI", "act")
        tape = {k: np.zeros((T, N)) for k in keys}
        for t in range(T):
            stacked = hist.reshape(-1)
            XE = self.M["E"] @ stacked
            XI = self.M["I"] @ stacked
            e = J * (lam + np.sqrt(lam) * xi[t]) if ext is None else ext[t]
            I = aE * XE + aI * XI + e
            gate = 1.0 - s1 - s2
            g = np.maximum(gate, 0.0)
            U = g * (V + I) + (1.0 - g) * vr
            s = (U >= th).astype(np.float64) if hard else _sigmoid(beta * (U - th))
            Vp = U - s * (U - vr)
            cp = c + dc * s
            for k, v in zip(keys, (V, I, U, g, s, cp, XE, XI, gate > 0)):
                tape[k][t] = v
            V = self.pvv * Vp + pvc * cp
            c = self.pcc * cp
            hist[1:] = hist[:-1].copy()
            hist[0] = s
            s1, s2 = s, s1
        NE = int(exc.sum())
        NI = N - NE
        rE = 1000.0 * tape["s"][:, exc].sum() / (T * NE)
        rI = 1000.0 * tape["s"][:, ~exc].sum() / (T * NI) if NI else 0.0
        loss = (rE - targets[0]) ** 2 + (rI - targets[1]) ** 2
        st = dict(theta=(aEE, aEI, aIE, aII, gc, nu), T=T, beta=beta, targets=targets, hard=hard,
                  th=th,
                  aE=aE, aI=aI, pvc=pvc, lam=lam, J=J, vr=vr, dc=dc, xi=xi,
                  rates=(rE, rI), NE=NE, NI=NI, V_end=V, c_end=c)
        st.update(tape)
        return loss, st

    def forward32(self, theta, T, beta=5.0, targets=(3.0, 8.0)):
        """The hard-spike recursion in FP32 with the operation order of the
        device path (reading: one IEEE float32 rounding per operation, the
        propagation as one fused multiply-add), so its spikes can be compared
        bit for bit.  Returns (loss, tape) like ``forward``; the tape holds the
        float32 values as float64 for ``backward``."""
        p, N, D, exc = self.p, self.N, self.D, self.exc
        f = np.float32
        aEE, aEI, aIE, aII, gc, nu = (float(x) for x in theta)
        aE = np.where(exc, f(aEE), f(aEI)).astype(f)
        aI = np.where(exc, f(aIE), f(aII)).astype(f)
        h = float(p.h)
        lam64 = nu * h
        lam, sqlam = f(lam64), f(np.sqrt(lam64))
        J, vr, th, dc = (f(x) for x in (p.j_ext, p.v_reset, p.theta, p.dc))
        pvv, pcc = f(self.pvv), f(self.pcc)
        pvc = np.where(exc, f(gc * self.kappa), f(float(np.float32(p.gc_inh)) * self.kappa)).astype(f)
        xi = surr_xi(p, 0, N, 0, T).astype(f)
        hist = np.zeros((D, N))
        s1, s2 = np.zeros(N, f), np.zeros(N, f)
        V, c = self.v0.astype(f), np.zeros(N, f)
        keys = ("V", "I", "U", "g", "s", "cp", "XE", "XI", "act")
        tape = {k: np.zeros((T, N)) for k in keys}
        for t in range(T):
            stacked = hist.reshape(-1)
            XE = (self.M["E"] @ stacked).astype(f)   # exact sums of multiples of 2^-16
            XI = (self.M["I"] @ stacked).astype(f)
            e = J * (lam + sqlam * xi[t])
            I = (aE * XE + aI * XI) + e
            g = (s1 + s2 == 0).astype(f)
            U = np.where(g > 0, V + I, vr).astype(f)
            s = (U >= th).astype(f)
            Vp = np.where(s > 0, vr, U).astype(f)
            cp = np.where(s > 0, c + dc, c).astype(f)
            for k, v in zip(keys, (V, I, U, g, s, cp, XE, XI, g > 0)):
                tape[k][t] = v
            V = fma32(cp, pvc, Vp * pvv)
            c = (cp * pcc).astype(f)
            hist[1:] = hist[:-1].copy()
            hist[0] = s
            s1, s2 = s, s1
        NE = int(exc.sum())
        NI = N - NE
        rE = 1000.0 * tape["s"][:, exc].sum() / (T * NE)
        rI = 1000.0 * tape["s"][:, ~exc].sum() / (T * NI) if NI else 0.0
        loss = (rE - targets[0]) ** 2 + (rI - targets[1]) ** 2
        st = dict(theta=(aEE, aEI, aIE, aII, gc, nu), T=T, beta=beta, targets=targets, hard=True,
                  th=float(th), aE=aE.astype(np.float64), aI=aI.astype(np.float64),
                  pvc=pvc.astype(np.float64), lam=lam64, J=float(J), vr=float(vr), dc=float(dc),
                  xi=xi.astype(np.float64), rates=(rE, rI), NE=NE, NI=NI,
                  V_end=V.astype(np.float64), c_end=c.astype(np.float64))
        st.update(tape)
        return loss, st

    def backward(self, st):
        """Gradient of the loss with respect to theta (6 values)."""
        N, D, exc = self.N, self.D, self.exc
        T, beta = st["T"], st["beta"]
        rE, rI = st["rates"]
        dE = 2.0 * (rE - st["targets"][0]) * 1000.0 / (T * st["NE"])
        dI = 2.0 * (rI - st["targets"][1]) * 1000.0 / (T * st["NI"]) if st["NI"] else 0.0
        dlds = np.where(exc, dE, dI)
        aE, aI, pvc = st["aE"], st["aI"], st["pvc"]
        vr, dc, lam, J = st["vr"], st["dc"], st["lam"], st["J"]
        grad = np.zeros(6)
        Vbar, cbar = np.zeros(N), np.zeros(N)
        Ibar = np.zeros((T + D + 1, N))     # adjoint of I(t); zero beyond T - 1
        gb = np.zeros((T + 3, N))           # -gbar(t) act(t): goes to s(t-1), s(t-2)
        for t in range(T - 1, -1, -1):
            s, U, g, cp = st["s"][t], st["U"][t], st["g"][t], st["cp"][t]
            # s(t) feeds the input of steps t + d through its outgoing synapses
            yE = np.zeros(N)
            yI = np.zeros(N)
            for d in range(1, D + 1):
                if t + d < T:
                    yE += self.WT[d - 1] @ (aE * Ibar[t + d])
                    yI += self.WT[d - 1] @ (aI * Ibar[t + d])
            sbar = dlds + np.where(exc, yE, yI) + gb[t + 1] + gb[t + 2]
            # V(t+1) = P_VV V' + P_VC c',  c(t+1) = P_CC c'
            Vpbar = self.pvv * Vbar
            cpbar = self.pcc * cbar + pvc * Vbar
            grad[4] += np.sum((Vbar * cp * self.kappa)[exc])
            # V' = U - s (U - V_reset),  c' = c + dc s
            Ubar = Vpbar * (1.0 - s)
            sbar = sbar - Vpbar * (U - vr) + cpbar * dc
            # s = sigmoid(beta (U - theta)), or the surrogate of the hard threshold
            if st["hard"]:
                dsdU = 1.0 / (1.0 + beta * np.abs(U - st["th"])) ** 2
            else:
                dsdU = beta * s * (1.0 - s)
            Ubar = Ubar + sbar * dsdU
            # U = g (V + I) + (1 - g) V_reset
            Vbar = Ubar * g
            Ib = Ubar * g
            gbar = Ubar * (st["V"][t] + st["I"][t] - vr)
            gb[t] = -gbar * st["act"][t]
            cbar = cpbar
            Ibar[t] = Ib
            # I = aE X_E + aI X_I + J (lam + sqrt(lam) xi)
            XE, XI = st["XE"][t], st["XI"][t]
            grad[0] += np.sum((Ib * XE)[exc])
            grad[1] += np.sum((Ib * XE)[~exc])
            grad[2] += np.sum((Ib * XI)[exc])
            grad[3] += np.sum((Ib * XI)[~exc])
            if st["xi"] is not None:
                h = float(self.p.h)
                grad[5] += np.sum(Ib * J * h * (1.0 + st["xi"][t] / (2.0 * np.sqrt(lam))))
        return grad
