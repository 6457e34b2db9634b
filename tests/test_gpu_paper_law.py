"""The paper's own connectivity law (SNN_CONN_PAPER) on the GPU against the
oracle (oracle/snn_oracle.c, pinned by tests/test_oracle_paper_law.py):
the same rows synapse for synapse, bit-identical rasters, exact counters."""
import numpy as np
import pytest

import oracle
from paper_1511_09325_gb300 import build as B
from paper_1511_09325_gb300 import snn
from paper_1511_09325_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PAPER = dict(connectivity=1)


@pytest.fixture(scope="module", autouse=True)
def lib():
    B.build()
    snn.load()


def _keys(tgt, dly, w):
    return np.sort(tgt.astype(np.int64) * 64 * 2 ** 24 + dly.astype(np.int64) * 2 ** 24
                   + (w.astype(np.int64) & 0xFFFFFF))


@pytest.mark.parametrize("prec,gw,gh,seed", [("f32w", 2, 2, 3), ("f16w", 3, 5, 4)])
def test_rows_match_oracle(prec, gw, gh, seed):
    n, s = W.neuron_params(), W.synapse_params(**PAPER)
    p = oracle.make_params(gw, gh, n, s, seed)
    with snn.Net(gw, gh, n, s, seed, prec) as net:
        N = net.n
        rng = np.random.default_rng(seed)
        starts = sorted(set(rng.choice(N - 40, 5, replace=False).tolist() + [0, N - 40]))
        total = 0
        for j0 in starts:
            o = oracle.paper_synapses(p, prec, j0, 40)
            lens = net.row_lengths(j0, 40)
            assert np.array_equal(lens, o["count"])
            tg, dl, wf = net.synapses(j0, 40)
            cut = np.concatenate([[0], np.cumsum(lens)])
            ocut = np.concatenate([[0], np.cumsum(o["count"])])
            for r in range(40):
                a, b = slice(cut[r], cut[r + 1]), slice(ocut[r], ocut[r + 1])
                assert np.array_equal(_keys(tg[a], dl[a], wf[a]),
                                      _keys(o["target"][b], o["delay"][b], o["wfx"][b]))
            total += int(lens.sum())
        info = net.info()
        assert abs(info["synapses"] / N - 1307.5) < 5  # mean out-degree of the law
        assert total > 0


@pytest.mark.parametrize("prec,steps", [("f32w", 300), ("f16w", 150)])
def test_cols2x2_paper_law_bit_exact(prec, steps):
    n, s = W.neuron_params(), W.synapse_params(**PAPER)
    p = oracle.make_params(2, 2, n, s, 1)
    with snn.Net(2, 2, n, s, 1, prec) as net:
        net.step(steps)
        st, ids, over = net.spikes()
        v, c, r = net.state()
        rec, _, nsteps = net.stats()
        deg = net.row_lengths(0, net.n)
    o = oracle.run(p, prec, steps)
    assert not over and len(o["t"]) > 1000
    key = lambda t, i: np.sort(np.asarray(t, np.int64) * 10 ** 7 + np.asarray(i, np.int64))
    assert np.array_equal(key(st, ids), key(o["t"], o["i"]))
    assert np.array_equal(v.astype(np.float64), o["v"])
    assert np.array_equal(c.astype(np.float64), o["c"])
    assert nsteps == steps
    # every spike counts its own neuron's out-degree
    assert rec == float(deg[ids].astype(np.int64).sum())


def test_batch_members_with_both_laws_match_standalone():
    n = W.neuron_params()
    sf, spp = W.synapse_params(), W.synapse_params(**PAPER)
    grids, syns, seeds = [(2, 1), (1, 2)], [sf, spp], [5, 6]
    ref = []
    for g, s, sd in zip(grids, syns, seeds):
        with snn.Net(g[0], g[1], n, s, sd, "f32w") as net:
            net.step(120)
            st, ids, _ = net.spikes()
            ref.append(np.sort(st.astype(np.int64) * 10 ** 7 + ids))
    with snn.Batch(grids, [n, n], syns, seeds, "f32w") as b:
        b.step(120)
        for k, m in enumerate(b.members):
            st, ids, _ = m.spikes()
            assert np.array_equal(np.sort(st.astype(np.int64) * 10 ** 7 + ids), ref[k])


def test_full_size_24x24_paper_law_rows():
    """24x24 columns under the paper law: ~933 M synapses; sampled rows
    against the oracle and a few steps run."""
    n, s = W.neuron_params(), W.synapse_params(**PAPER)
    p = oracle.make_params(24, 24, n, s, 2)
    with snn.Net(24, 24, n, s, 2, "f32w") as net:
        info = net.info()
        assert abs(info["synapses"] / net.n - 1307.5) < 1
        rng = np.random.default_rng(9)
        for j0 in rng.choice(net.n - 4, 4, replace=False).tolist() + [net.n - 4]:
            o = oracle.paper_synapses(p, "f32w", int(j0), 4)
            assert np.array_equal(net.row_lengths(int(j0), 4), o["count"])
            tg, dl, wf = net.synapses(int(j0), 4)
            assert np.array_equal(_keys(tg, dl, wf), _keys(o["target"], o["delay"], o["wfx"]))
        net.step(20)
        assert net.stats()[2] == 20


def test_gradient_view_of_a_paper_law_net():
    n, s = W.neuron_params(), W.synapse_params(**PAPER)
    with snn.Net(2, 2, n, s, 1, "f32w") as net, snn.Grad(net, 40, checkpoint_every=16) as g:
        loss, rates, grad = g.loss_and_grad([1, 1, 1, 1, 0.02, 2.5])
    assert np.isfinite(loss) and np.all(np.isfinite(grad)) and rates[0] > 0
