"""Pins of the oracle's LIF + SFA neuron update against closed forms.

Sec. 2 of the paper names the neuron model (leaky integrate-and-fire with
spike-frequency adaptation from a calcium-dependent after-hyperpolarisation
current) without equations.  The oracle integrates
    dV/dt = -V / tau_m - g_c c,   dc/dt = -c / tau_c
exactly over each step, adds the step's input as a jump, and on a threshold
crossing resets V, clamps it for the refractory steps and increments c.
These tests check it against solutions written independently of its loop.
"""
import math

import numpy as np
import pytest

from paper_1511_09325_gb300 import workloads as W


def _p(orc, h=1.0, **over):
    n = W.neuron_params(**over)
    return orc.make_params(1, 1, n, W.synapse_params(), 1, h=h)


# parameters enter the model as float32 numbers
GC = float(np.float32(0.02))


def _analytic(v0, c0, t, tm=20.0, tc=500.0, gc=GC):
    c = c0 * np.exp(-t / tc)
    v = v0 * np.exp(-t / tm) - gc * c0 * tm * tc / (tc - tm) * (np.exp(-t / tc) - np.exp(-t / tm))
    return v, c


@pytest.mark.parametrize("v0,c0", [(10.0, 5.0), (19.9, 0.0), (-3.0, 12.5)])
def test_subthreshold_f64_closed_form(orc, v0, c0):
    n = 400
    v, c, s = orc.neuron_trace(_p(orc), "f64", 0, v0, c0, np.zeros(n))
    t = np.arange(1, n + 1, dtype=np.float64)
    va, ca = _analytic(v0, c0, t)
    assert not s.any()
    assert np.allclose(v, va, rtol=1e-12, atol=1e-12)
    assert np.allclose(c, ca, rtol=1e-12, atol=1e-14)


def test_subthreshold_f32_few_ulp(orc):
    n = 400
    v, c, s = orc.neuron_trace(_p(orc), "f32w", 0, 10.0, 5.0, np.zeros(n, np.int32))
    t = np.arange(1, n + 1, dtype=np.float64)
    va, ca = _analytic(10.0, 5.0, t)
    # a few ulp of float32 per step, accumulated over 400 steps
    assert np.max(np.abs(v - va)) < 400 * 4 * 2.0 ** -23 * 10.0
    assert np.max(np.abs(c - ca) / ca) < 400 * 4 * 2.0 ** -23


def test_inhibitory_neuron_has_no_adaptation_current(orc):
    v, c, _ = orc.neuron_trace(_p(orc), "f64", 1, 10.0, 5.0, np.zeros(50))
    t = np.arange(1, 51, dtype=np.float64)
    assert np.allclose(v, 10.0 * np.exp(-t / 20.0), rtol=1e-13)


def _discrete_isi(I, vr=15.0, theta=20.0, tm=20.0, nref=2):
    """Inter-spike interval (steps) of the step rule under constant input I.

    After a spike at step s the two refractory steps leave V = vr e^{-1/tm};
    the n-th integrating step then sees
        pre_n = P^{n-1} V0 + I (1 - P^n) / (1 - P),  P = e^{-1/tm},
    (geometric sum, no recursion) and fires at the first n with pre_n >= theta.
    """
    P = math.exp(-1.0 / tm)
    V0 = vr * P
    for n in range(1, 100000):
        pre = P ** (n - 1) * V0 + I * (1.0 - P ** n) / (1.0 - P)
        if pre >= theta:
            return n + nref
    return None


@pytest.mark.parametrize("I", [1.2, 1.5, 2.0, 3.0, 6.0])
def test_constant_drive_discrete_period(orc, I):
    p = _p(orc, gc_exc=0.0)
    n = 600
    _, _, s = orc.neuron_trace(p, "f64", 0, 15.0, 0.0, np.full(n, I))
    spk = np.flatnonzero(s)
    assert len(spk) >= 3
    isi = np.diff(spk)
    assert np.all(isi == _discrete_isi(I))


@pytest.mark.parametrize("mu", [1.2, 1.5, 3.0])
def test_constant_drive_continuous_limit(orc, mu):
    """At h = 0.01 ms the period approaches t_ref + tau ln((mu tau - Vr)/(mu tau - theta))."""
    h = 0.01
    p = _p(orc, h=h, gc_exc=0.0)
    n = int(200 / h)
    _, _, s = orc.neuron_trace(p, "f64", 0, 15.0, 0.0, np.full(n, mu * h))
    isi = np.diff(np.flatnonzero(s)) * h
    T = 2.0 + 20.0 * math.log((mu * 20.0 - 15.0) / (mu * 20.0 - 20.0))
    assert len(isi) >= 3
    assert abs(isi.mean() - T) / T < 0.01


def test_adaptation_steady_state(orc):
    """Periodic firing with SFA: just after each spike c = dc / (1 - P_cc^ISI)."""
    p = _p(orc, gc_exc=0.02)
    n = 20000
    v, c, s = orc.neuron_trace(p, "f64", 0, 15.0, 0.0, np.full(n, 3.0))
    spk = np.flatnonzero(s)
    isi = np.diff(spk)
    late = isi[len(isi) // 2:]
    assert late.min() == late.max(), "firing should settle to a fixed period"
    n_isi = int(late[0])
    # the update decays c once in the spike step itself
    c_after = c[spk[-1]] / math.exp(-1.0 / 500.0)
    assert c_after == pytest.approx(1.0 / (1.0 - math.exp(-n_isi / 500.0)), rel=1e-9)
    # adaptation lengthens the intervals
    assert isi[-1] > isi[0]


def test_refractory_clamp(orc):
    """Input in the two steps after a spike is discarded; V restarts from V_reset."""
    p = _p(orc, gc_exc=0.0)
    inp = np.array([30.0, 50.0, 50.0, 0.0, 0.0])
    v, _, s = orc.neuron_trace(p, "f64", 0, 0.0, 0.0, inp)
    P = math.exp(-1.0 / 20.0)
    assert list(s) == [True, False, False, False, False]
    assert v[0] == pytest.approx(15.0 * P)
    assert v[1] == pytest.approx(15.0 * P)
    assert v[2] == pytest.approx(15.0 * P)
    assert v[3] == pytest.approx(15.0 * P * P)


def test_f32_fixed_point_input_scale(orc):
    """One fixed-point unit is 2^-16 mV: 65536 units raise V by exactly 1 mV."""
    p = _p(orc, gc_exc=0.0)
    v, _, _ = orc.neuron_trace(p, "f32w", 0, 0.0, 0.0, np.array([65536 * 5], np.int32))
    assert v[0] == np.float32(np.float32(5.0) * np.float32(math.exp(-1.0 / 20.0)))
