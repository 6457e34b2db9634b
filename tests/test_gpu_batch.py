"""The batched form (many independent nets, one persistent launch per call).

Every member is held to the CPU oracle directly: its raster, final
potentials, calcium and refractory counters equal the oracle's run of the
same network (bit for bit, as in the single-net parity tests), whatever the
other members are.
The grid barrier between the phases waits a bounded number of polls; the
timeout path is exercised by a barrier that waits for one more block than
the launch has, which must end the call with SNN_ETIMEOUT.
"""
import numpy as np
import pytest

import oracle
from oracle_pool import OraclePool
from paper_1511_09325_gb300 import build as B
from paper_1511_09325_gb300 import snn
from paper_1511_09325_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    oracle.build()
    B.build()
    snn.load()


@pytest.fixture(scope="module")
def pool():
    p = OraclePool()
    yield p
    p.close()


def _key(t, i):
    return np.sort(np.asarray(t, np.int64) * (1 << 32) + np.asarray(i, np.int64))


def _check_members(batch, grids, neurons, synapses, seeds, prec, steps, pool):
    want = pool.map([(g, n, sy, sd, prec, steps) for g, n, sy, sd in
                      zip(grids, neurons, synapses, seeds)])
    for k, m in enumerate(batch.members):
        t, i, over = m.spikes()
        assert not over
        o = want[k]
        assert len(o["key"]) > 0, k
        assert np.array_equal(_key(t, i), o["key"]), k
        mv, mc, mr = m.state()
        assert np.array_equal(mv.astype(np.float64), o["v"]), k
        assert np.array_equal(mc.astype(np.float64), o["c"]), k
        assert np.array_equal(mr, o["r"]), k
        assert m.stats()[2] == steps


GRIDS = [(1, 1), (2, 3), (3, 1), (4, 4), (1, 2), (8, 2)]


@pytest.mark.parametrize("prec", ["f32w", "f16w"])
def test_members_match_oracle(prec, pool):
    n = len(GRIDS)
    neurons = [W.neuron_params(nu_ext_kHz=1.5 + 2.0 * k / (n - 1)) for k in range(n)]
    synapses = [W.synapse_params() for _ in range(n)]
    seeds = [100 + k for k in range(n)]
    with snn.Batch(GRIDS, neurons, synapses, seeds, prec) as b:
        for m in b.members:
            m.set_record_capacity(1 << 22)
        b.step(1)
        b.step(99)
        b.step(200)
        _check_members(b, GRIDS, neurons, synapses, seeds, prec, 300, pool)


def test_mixed_neuron_counts_and_delays(pool):
    """Members with different column sizes, delay ranges and stencils."""
    grids = [(2, 2), (3, 2), (1, 1)]
    neurons = [W.neuron_params(n_per_col=101, n_exc=81, nu_ext_kHz=3.0), W.neuron_params(),
               W.neuron_params(nu_ext_kHz=2.0)]
    synapses = [W.synapse_params(k_out=150, d_min=2, d_max=7, stencil_radius=2),
                W.synapse_params(d_max=32), W.synapse_params(d_min=3, d_max=5)]
    seeds = [7, 8, 9]
    with snn.Batch(grids, neurons, synapses, seeds, "f32w") as b:
        for m in b.members:
            m.set_record_capacity(1 << 22)
        b.step(250)
        _check_members(b, grids, neurons, synapses, seeds, "f32w", 250, pool)


def test_tuned_schedule_keeps_results(pool):
    grids, neurons, synapses, seeds = W.batch_workload(n_nets=8)
    with snn.Batch(grids, neurons, synapses, seeds, "f32w") as b:
        for m in b.members:
            m.set_record_capacity(1 << 22)
        choice = b.tune(10)  # 2 stages x 2 rounds x 4 candidates x 10 steps
        assert 0 <= choice < 16
        b.step(40)
        _check_members(b, grids, neurons, synapses, seeds, "f32w", 200, pool)


def test_member_cannot_be_stepped_alone():
    with snn.Batch([(1, 1)], [W.neuron_params()], [W.synapse_params()], [1]) as b:
        h = b.members[0].handle
        assert snn.load().snn_step(h, 1) == snn.SNN_ESTATE


def test_barrier_wait_gives_up_with_timeout():
    """A barrier that waits for one block too many must return SNN_ETIMEOUT
    after its bounded polls, and the context stays usable."""
    with snn.Batch([(2, 2), (1, 1)], [W.neuron_params()] * 2, [W.synapse_params()] * 2,
                   [3, 4]) as b:
        b.set_wait(spin_limit=2000, extra_arrivals=1)
        with pytest.raises(snn.SnnError) as e:
            b.step(3)
        assert e.value.code == snn.SNN_ETIMEOUT
    # the device still works
    with snn.Net(1, 1, W.neuron_params(), W.synapse_params(), 5, "f32w") as net:
        net.step(10)
        assert net.stats()[2] == 10
