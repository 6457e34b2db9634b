"""Inconsistent delivery counts are reported, not silently dropped.

The item counts a delivery splits over its blocks (per column and per group
of 32 columns) are kept by the update kernel; a bookkeeping fault would make
them disagree with the step's spike lists.  The fault is made on the host
(snn_debug_offset_count adds to a count; no device fault is involved): the
next delivery must set the net's status word, snn_step and the reads must then
return SNN_ESTATE, and the device must stay usable for other nets.
"""
import numpy as np
import pytest

from paper_1511_09325_gb300 import build as B
from paper_1511_09325_gb300 import snn
from paper_1511_09325_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    snn.load()


@pytest.mark.parametrize("group_only", [False, True])
@pytest.mark.parametrize("prec", ["f32w", "f16w"])
def test_offset_count_sets_status(prec, group_only):
    n, s = W.neuron_params(), W.synapse_params()
    with snn.Net(3, 2, n, s, 5, prec) as net:
        net.step(20)
        net.spikes()
        assert net.stats()[2] == 20
        snn.snn_debug_offset_count(net.handle, 4, 37, group_only)
        net.step(1)  # asynchronous: returns before the delivery has run
        with pytest.raises(snn.SnnError) as e:
            net.spikes()
        assert e.value.code == snn.SNN_ESTATE
        with pytest.raises(snn.SnnError) as e:
            net.step(1)
        assert e.value.code == snn.SNN_ESTATE
        with pytest.raises(snn.SnnError) as e:
            net.stats()
        assert e.value.code == snn.SNN_ESTATE
        assert "disagree" in snn.snn_last_error(net.handle)
    # another net on the same device is unaffected
    with snn.Net(1, 1, n, s, 6, prec) as other:
        other.step(30)
        t, i, over = other.spikes()
        assert not over and len(t) > 0 and other.stats()[2] == 30


def test_consistent_counts_leave_status_clear():
    n, s = W.neuron_params(), W.synapse_params()
    with snn.Net(2, 2, n, s, 1, "f16w") as net:
        net.step(300)
        t, i, over = net.spikes()
        assert not over and len(t) > 0
        snn.snn_debug_offset_count(net.handle, 0, 0)
        net.step(10)
        assert net.stats()[2] == 310


def test_offset_count_rejects_bad_column():
    with snn.Net(1, 1, W.neuron_params(), W.synapse_params(), 1, "f32w") as net:
        with pytest.raises(snn.SnnError) as e:
            snn.snn_debug_offset_count(net.handle, 1, 1)
        assert e.value.code == snn.SNN_EINVAL
