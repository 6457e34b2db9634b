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
  - the exact-FP32 forward against the FP64 one (same spikes).
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
