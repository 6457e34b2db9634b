"""Pins of the FP64 oracle of the differentiable form (oracle/surrogate.py).

The paper has no gradient (its Sec. 2 network is simulated, not trained), so
the relaxed recursion is a reading; these tests pin the oracle's code against
things other than itself:
  - its reverse-mode gradient against central finite differences of its own
    forward pass (soft spikes, where the derivative is exact), all six
    parameters;
  - its forward pass, in the limit of a step-like sigmoid and with the
    spiking model's Poisson input, against the independent C oracle of the
    spiking network (same raster, same final potentials);
  - the exact-FP32 forward against the FP64 one (same spikes);
  - its reverse recursion against forward-mode tangents of the same step, in
    hard mode (where finite differences do not apply) and in soft mode.
"""
import numpy as np
import pytest

import oracle
from oracle import surrogate as S
from paper_1511_09325_gb300 import workloads as W

THETA = np.array([1.0, 1.0, 1.0, 1.0, 0.02, 2.5])


@pytest.fixture(scope="module")
def net1():
    p = oracle.make_params(1, 1, W.neuron_params(), W.synapse_params(), 7)
    return S.SoftNet(p)


def test_gradient_matches_finite_differences(net1):
    """Soft spikes, 12 steps: the reverse recursion equals central differences
    to 1e-6 on every parameter (steps 1e-7, and 1e-6 for g_c, whose loss
    derivative is 20x smaller: both well above the loss's rounding and below
    its curvature)."""
    T = 12
    loss, st = net1.forward(THETA, T)
    g = net1.backward(st)
    assert loss > 0 and np.all(np.isfinite(g))
    steps = (1e-7, 1e-7, 1e-7, 1e-7, 1e-6, 1e-7)
    for k in range(6):
        e = steps[k]
        tp, tm = THETA.copy(), THETA.copy()
        tp[k] += e
        tm[k] -= e
        fd = (net1.forward(tp, T)[0] - net1.forward(tm, T)[0]) / (2 * e)
        assert abs(g[k] - fd) <= 1e-6 * max(abs(fd), 1.0), (S.PARAMS[k], g[k], fd)


def test_one_step_gradient_is_the_external_drive_only(net1):
    """After one step no spike has been delivered yet (d_min = 1) and no
    neuron has adapted its potential through c, so only nu_ext moves the
    loss: the other five derivatives are exactly zero."""
    loss, st = net1.forward(THETA, 1)
    g = net1.backward(st)
    assert np.all(g[:5] == 0.0) and g[5] != 0.0


@pytest.mark.parametrize("grid,seed", [((1, 1), 3), ((2, 2), 5)])
def test_step_limit_is_the_spiking_model(grid, seed):
    """beta = 1e9 with the spiking model's Poisson input and unrounded weights:
    the relaxed recursion's spikes (s > 1/2) are the C oracle's F64 raster and
    the final potentials agree to 1e-9 mV, over 150 steps."""
    n, s = W.neuron_params(), W.synapse_params()
    p = oracle.make_params(grid[0], grid[1], n, s, seed)
    net = S.SoftNet(p, weights="exact")
    T = 150
    N = net.N
    ext = oracle.ext_counts(p, 0, N, 0, T).astype(np.float64) * float(np.float32(p.j_ext))
    th = np.array([1.0, 1.0, 1.0, 1.0, float(np.float32(p.gc_exc)), 2.5])
    for hard in (False, True):
        _, st = net.forward(th, T, beta=1e9, ext=ext, hard=hard)
        spk = st["s"] > 0.5
        o = oracle.run(p, "f64", T)
        key = np.sort(o["t"].astype(np.int64) * N + o["i"])
        t_, i_ = np.nonzero(spk)
        assert len(key) > 100
        assert np.array_equal(np.sort(t_.astype(np.int64) * N + i_), key)
        assert np.max(np.abs(st["V_end"] - o["v"])) < 1e-9


def test_normal_draws_are_standard_normal_and_keyed_as_stated(orc):
    """xi_i(t) = Q[word >> 16], word = word i mod 4 of Philox(seed; i/4, t, 4):
    the wiring against the oracle's own generator and table, and the draws
    against N(0, 1) (moments and a Kolmogorov-Smirnov test)."""
    from scipy import stats

    p = orc.make_params(1, 1, W.neuron_params(), W.synapse_params(), 77)
    xi = orc.surr_xi(p, 0, 1240, 0, 40)
    q = orc.tables(p)["q"]
    key = [77, 0]
    for i, t in ((0, 0), (5, 3), (1239, 39), (402, 17)):
        w = orc.philox([i >> 2, t, 4, 0], key)[i & 3]
        assert xi[t, i] == q[int(w) >> 16]
    x = xi.ravel()
    assert abs(x.mean()) < 4 / np.sqrt(x.size) and abs(x.var() - 1) < 0.03
    assert stats.kstest(x, "norm").pvalue > 1e-4


def test_fp32_forward_has_the_fp64_spikes(net1):
    """Hard spikes, 100 steps: the exact-FP32 recursion fires exactly where the
    FP64 one does, and its gradient agrees to 1e-3."""
    T = 100
    l64, s64 = net1.forward(THETA, T, hard=True)
    l32, s32 = net1.forward32(THETA, T)
    assert np.array_equal(s64["s"], s32["s"]) and s64["s"].sum() > 1000
    assert l64 == l32
    g64, g32 = net1.backward(s64), net1.backward(s32)
    assert np.allclose(g32, g64, rtol=1e-3, atol=1e-6 * np.abs(g64).max())


def _forward_mode(net, theta, T, beta=5.0, targets=(3.0, 8.0), hard=True):
    """Loss and its six derivatives by forward-mode accumulation: each state
    variable carries its tangent with respect to every parameter (arrays of
    6 x N) through the step, with ds/dU taken as the fast-sigmoid surrogate
    (hard spikes) or the sigmoid's own derivative (soft).  The refractory gate
    max(0, 1 - s(t-1) - s(t-2)) passes tangents only where it is positive.
    This accumulates the derivative in the opposite direction to the oracle's
    hand-written adjoint recursion, so the two agree only if every adjoint
    there is the transpose of the corresponding step here."""
    p, N, D, exc = net.p, net.N, net.D, net.exc
    aEE, aEI, aIE, aII, gc, nu = (float(x) for x in theta)
    aE, aI = np.where(exc, aEE, aEI), np.where(exc, aIE, aII)
    daE, daI, dpvc = np.zeros((6, N)), np.zeros((6, N)), np.zeros((6, N))
    daE[0], daE[1] = exc, ~exc
    daI[2], daI[3] = exc, ~exc
    dpvc[4] = np.where(exc, net.kappa, 0.0)
    h = float(p.h)
    lam = nu * h
    J = float(np.float32(p.j_ext))
    vr, th, dc = (float(np.float32(x)) for x in (p.v_reset, p.theta, p.dc))
    pvc = np.where(exc, gc * net.kappa, float(np.float32(p.gc_inh)) * net.kappa)
    xi = oracle.surr_xi(p, 0, N, 0, T)
    hist, dhist = np.zeros((D, N)), np.zeros((D, 6, N))
    s1, s2 = np.zeros(N), np.zeros(N)
    ds1, ds2 = np.zeros((6, N)), np.zeros((6, N))
    V, c = net.v0.copy(), np.zeros(N)
    dV, dc_ = np.zeros((6, N)), np.zeros((6, N))
    sums, dsums = np.zeros(2), np.zeros((2, 6))
    for t in range(T):
        XE, XI = net.M["E"] @ hist.reshape(-1), net.M["I"] @ hist.reshape(-1)
        dstk = dhist.transpose(1, 0, 2).reshape(6, D * N)
        dXE, dXI = (net.M["E"] @ dstk.T).T, (net.M["I"] @ dstk.T).T
        I = aE * XE + aI * XI + J * (lam + np.sqrt(lam) * xi[t])
        dI = daE * XE + aE * dXE + daI * XI + aI * dXI
        dI[5] += J * h * (1.0 + xi[t] / (2.0 * np.sqrt(lam)))
        gate = 1.0 - s1 - s2
        g = np.maximum(gate, 0.0)
        dg = np.where(gate > 0, -(ds1 + ds2), 0.0)
        U = g * (V + I) + (1.0 - g) * vr
        dU = dg * (V + I - vr) + g * (dV + dI)
        if hard:
            s = (U >= th).astype(np.float64)
            slope = 1.0 / (1.0 + beta * np.abs(U - th)) ** 2
        else:
            s = 1.0 / (1.0 + np.exp(-beta * (U - th)))
            slope = beta * s * (1.0 - s)
        ds = slope * dU
        Vp, dVp = U - s * (U - vr), (1.0 - s) * dU - ds * (U - vr)
        cp, dcp = c + dc * s, dc_ + dc * ds
        V, dV = net.pvv * Vp + pvc * cp, net.pvv * dVp + pvc * dcp + dpvc * cp
        c, dc_ = net.pcc * cp, net.pcc * dcp
        hist[1:], dhist[1:] = hist[:-1].copy(), dhist[:-1].copy()
        hist[0], dhist[0] = s, ds
        s1, s2, ds1, ds2 = s, s1, ds, ds1
        sums += (s[exc].sum(), s[~exc].sum())
        dsums += (ds[:, exc].sum(1), ds[:, ~exc].sum(1))
    n = np.array([exc.sum(), N - exc.sum()], np.float64)
    r = 1000.0 * sums / (T * n)
    loss = float(((r - np.array(targets)) ** 2).sum())
    dloss = (2.0 * (r - np.array(targets)) * 1000.0 / (T * n)) @ dsums
    return loss, dloss


@pytest.mark.parametrize("hard,T", [(True, 40), (False, 10)])
def test_reverse_gradient_equals_forward_mode_tangents(net1, hard, T):
    """The hard mode's surrogate gradient has no finite-difference check (the
    spiking loss is piecewise constant), so its adjoint recursion is pinned
    against forward-mode tangents of the same linearised step: all six
    derivatives agree to FP64 rounding.  Soft spikes too, for the record."""
    loss, st = net1.forward(THETA, T, hard=hard)
    g = net1.backward(st)
    lf, gf = _forward_mode(net1, THETA, T, hard=hard)
    assert lf == pytest.approx(loss, rel=1e-12)
    assert st["s"].sum() > 100  # spikes (or spike mass) on the path
    scale = np.abs(gf).max()
    assert np.all(np.abs(g - gf) <= 1e-9 * np.maximum(np.abs(gf), 1e-3 * scale)), (g, gf)
