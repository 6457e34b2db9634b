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

from paper_1511_09325_gb300 import workloads as W

from dense_model import _reference, fma32

NPC = 1240


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
