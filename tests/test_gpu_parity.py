"""GPU path against the CPU oracle, through the C ABI.

The bar: the synapse table, the spike raster and the final neuron state are
bit-identical to the oracle's fixed-point/FP32 modes (integer accumulation
makes the delivery order irrelevant, every float operation is rounded as the
oracle rounds it).  Rasters are compared as sorted (step, neuron) lists: the
order of spikes within one step is not defined.
"""
import numpy as np
import pytest

import oracle
from paper_1511_09325_gb300 import build as B
from paper_1511_09325_gb300 import snn
from paper_1511_09325_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    snn.load()
    oracle.build()


def _sorted_raster(t, i):
    t = np.asarray(t, np.int64)
    i = np.asarray(i, np.int64)
    key = t * (1 << 32) + i
    return np.sort(key)


def _row_keys(tgt, dly, wfx):
    """Per-row sorted keys of (delay, target, weight) for multiset comparison."""
    key = (dly.astype(np.int64) << 56) + (tgt.astype(np.int64) << 20) + (wfx.astype(np.int64) + (1 << 19))
    return np.sort(key, axis=1)


def _compare_rows(net, p, mode, j0, n):
    tg, dg, wg = net.synapses(j0, n)
    o = oracle.synapses(p, mode, j0, n)
    assert np.array_equal(_row_keys(tg, dg, wg), _row_keys(o["target"], o["delay"], o["wfx"]))


@pytest.mark.parametrize("gw,gh,prec,seed", [
    (1, 1, "f32w", 7), (2, 2, "f32w", 1), (3, 5, "f16w", 4), (2, 2, "f16w", 1),
])
def test_synapse_table_matches_oracle(gw, gh, prec, seed):
    n, s = W.neuron_params(), W.synapse_params()
    with snn.Net(gw, gh, n, s, seed, prec) as net:
        p = oracle.make_params(gw, gh, n, s, seed)
        for j0 in range(0, net.n, 2480):
            _compare_rows(net, p, prec, j0, min(2480, net.n - j0))


def _run_both(gw, gh, n, s, seed, prec, steps, chunks=None):
    with snn.Net(gw, gh, n, s, seed, prec) as net:
        net.set_record_capacity(max(1 << 20, net.n * 4))
        if chunks:
            for c in chunks:
                net.step(c)
        else:
            net.step(steps)
        st, ids, over = net.spikes()
        assert not over
        v, c, r = net.state()
        stats = net.stats()
        _, pop = net.rates()
    p = oracle.make_params(gw, gh, n, s, seed)
    o = oracle.run(p, prec, steps)
    return dict(t=st, i=ids, v=v, c=c, r=r, stats=stats, pop=pop), o


def _assert_same(g, o, n_neurons):
    assert np.array_equal(_sorted_raster(g["t"], g["i"]), _sorted_raster(o["t"], o["i"]))
    assert np.array_equal(g["v"].astype(np.float64), o["v"])
    assert np.array_equal(g["c"].astype(np.float64), o["c"])
    assert np.array_equal(g["r"], o["r"])


def test_cols2x2_f32w_1000_steps_bit_exact():
    """The 2x2 parity workload (4960 neurons, seed 1, 1000 steps)."""
    cfg = W.WORKLOADS["cols2x2_f32w"]
    n, s = W.neuron_params(), W.synapse_params()
    g, o = _run_both(2, 2, n, s, cfg["seed"], "f32w", cfg["steps"])
    assert len(o["t"]) > 10000
    _assert_same(g, o, 4960)
    rec, ext, steps = g["stats"]
    assert steps == cfg["steps"]
    assert rec == len(o["t"]) * 1240
    assert ext == float(o["step_ext"].sum())


VARIANTS = {
    # FP16 weights on a grid narrower than the stencil in x, wider in y
    "f16w_3x5": (3, 5, {}, {}, 4, "f16w", 300),
    # ragged sizes: 101 neurons per column (N = 303, not a multiple of 4),
    # a short delay range starting at 2, a 5x5 stencil
    "ragged_f32w": (3, 1, dict(n_per_col=101, n_exc=81, nu_ext_kHz=3.0),
                    dict(k_out=150, d_min=2, d_max=7, stencil_radius=2), 9, "f32w", 400),
    "ragged_f16w": (3, 1, dict(n_per_col=101, n_exc=81, nu_ext_kHz=3.0),
                    dict(k_out=150, d_min=2, d_max=7, stencil_radius=2), 9, "f16w", 400),
    # strong drive: most neurons fire every refractory period
    "saturated": (2, 1, dict(nu_ext_kHz=30.0), {}, 3, "f32w", 60),
    # no external input: silence
    "silent": (2, 2, dict(nu_ext_kHz=0.0), {}, 3, "f32w", 50),
    # one column, FP16
    "one_column_f16w": (1, 1, {}, {}, 7, "f16w", 400),
    # the longest delay range, a 64-bit seed
    "dmax32_seed64": (2, 2, {}, dict(d_max=32), (1 << 40) + 12345, "f32w", 200),
    # inhibitory adaptation switched on, single-delay network
    "gc_inh_single_delay": (2, 2, dict(gc_inh=0.01), dict(d_min=3, d_max=3), 21, "f32w", 200),
}


@pytest.mark.parametrize("name", sorted(VARIANTS))
def test_variants_bit_exact(name):
    gw, gh, nov, sov, seed, prec, steps = VARIANTS[name]
    n, s = W.neuron_params(**nov), W.synapse_params(**sov)
    g, o = _run_both(gw, gh, n, s, seed, prec, steps)
    if name == "silent":
        assert len(o["t"]) == 0
    else:
        assert len(o["t"]) > 0
    _assert_same(g, o, gw * gh * n["n_per_col"])


def test_step_chunking_does_not_change_the_run():
    """Whole-graph replays (64 steps) and single steps give the same raster."""
    n, s = W.neuron_params(), W.synapse_params()
    g, o = _run_both(2, 2, n, s, 1, "f32w", 300, chunks=[1, 7, 64, 129, 0, 99])
    _assert_same(g, o, 4960)


def test_profiled_steps_match_graph_steps():
    n, s = W.neuron_params(), W.synapse_params()
    with snn.Net(2, 2, n, s, 1, "f32w") as a, snn.Net(2, 2, n, s, 1, "f32w") as b:
        a.step(200)
        ms, by = b.step_profiled(200)
        assert ms[0] > 0 and ms[1] > 0 and by[0] > 0 and by[1] > 0
        ta, ia, _ = a.spikes()
        tb, ib, _ = b.spikes()
        assert np.array_equal(_sorted_raster(ta, ia), _sorted_raster(tb, ib))
        assert np.array_equal(a.state()[0], b.state()[0])


def test_record_overflow_keeps_counters_exact():
    n, s = W.neuron_params(), W.synapse_params()
    p = oracle.make_params(2, 2, n, s, 1)
    o = oracle.run(p, "f32w", 100, want_state=False)
    with snn.Net(2, 2, n, s, 1, "f32w") as net:
        net.set_record_capacity(50)
        net.step(100)
        st, ids, over = net.spikes()
        assert over and len(st) == 50
        rec, ext, steps = net.stats()
        assert rec == len(o["t"]) * 1240 and steps == 100
        # the drain reset the buffer: the next window is complete again
        net.set_record_capacity(1 << 20)
        net.step(10)
        st2, _, over2 = net.spikes()
        assert not over2 and np.all(st2 >= 100)


def test_rates_match_raster():
    n, s = W.neuron_params(), W.synapse_params()
    with snn.Net(2, 2, n, s, 1, "f32w") as net:
        net.step(400)
        st, ids, _ = net.spikes()
        hz, pop = net.rates()
    col, l = np.divmod(ids, 1240)
    for c in range(4):
        ne = int(((col == c) & (l < 992)).sum())
        ni = int(((col == c) & (l >= 992)).sum())
        assert hz[c, 0] == pytest.approx(ne / (992 * 0.4), rel=1e-6)
        assert hz[c, 1] == pytest.approx(ni / (248 * 0.4), rel=1e-6)
    assert pop[0] == pytest.approx(int((l < 992).sum()) / (3968 * 0.4), rel=1e-6)


def test_zero_steps_is_a_noop():
    n, s = W.neuron_params(), W.synapse_params()
    with snn.Net(1, 1, n, s, 1, "f32w") as net:
        net.step(0)
        assert net.stats()[2] == 0
        with pytest.raises(snn.SnnError):
            net.step(-1)


def test_full_size_24x24_f32w():
    """The 24x24 workload (714 240 neurons, 885.7 M synapses, seed 2) in the
    benchmark's launch configuration: sampled rows of the synapse table and
    the first 6 steps' raster against the oracle."""
    cfg = W.WORKLOADS["cols24x24_f32w"]
    n, s = W.neuron_params(), W.synapse_params()
    p = oracle.make_params(24, 24, n, s, cfg["seed"])
    with snn.Net(24, 24, n, s, cfg["seed"], "f32w") as net:
        info = net.info()
        assert info["synapses"] == 885657600
        rng = np.random.default_rng(1)
        for j0 in rng.choice(net.n - 8, 6, replace=False):
            _compare_rows(net, p, "f32w", int(j0), 8)
        _compare_rows(net, p, "f32w", net.n - 8, 8)
        net.step(6)
        st, ids, over = net.spikes()
        v, c, r = net.state()
    o = oracle.run(p, "f32w", 6)
    assert not over and len(o["t"]) > 1000
    assert np.array_equal(_sorted_raster(st, ids), _sorted_raster(o["t"], o["i"]))
    assert np.array_equal(v.astype(np.float64), o["v"])


@pytest.fixture(scope="module")
def full_size_oracle():
    """The oracle's 3-step runs of the 96x96 F16W and 48x48 F32W workloads,
    started in parallel processes when the first full-size test asks for
    them (each takes minutes on one core)."""
    from oracle_pool import OraclePool

    n, s = W.neuron_params(), W.synapse_params()
    pool = OraclePool(workers=2)
    jobs = {}
    for name, gw, prec in (("cols96x96_f16w", 96, "f16w"), ("cols48x48_f32w", 48, "f32w")):
        N = gw * gw * n["n_per_col"]
        jobs[name] = pool.submit((gw, gw), n, s, W.WORKLOADS[name]["seed"], prec, 3, N)
    yield jobs
    pool.close()


def _full_size_steps(name, rows_seed, job):
    """Build the workload in the benchmark's launch configuration, compare
    sampled rows of the table, run 3 steps, and compare the whole raster and
    the whole final state with the oracle's."""
    cfg = W.WORKLOADS[name]
    gw, prec, seed = cfg["grid_w"], cfg["precision"], cfg["seed"]
    n, s = W.neuron_params(), W.synapse_params()
    p = oracle.make_params(gw, gw, n, s, seed)
    with snn.Net(gw, gw, n, s, seed, prec) as net:
        N = net.n
        assert net.info()["synapses"] == N * 1240
        rng = np.random.default_rng(rows_seed)
        for j0 in rng.choice(N - 4, 6, replace=False):
            _compare_rows(net, p, prec, int(j0), 4)
        _compare_rows(net, p, prec, N - 4, 4)
        net.set_record_capacity(N)
        net.step(3)
        st, ids, over = net.spikes()
        v, c, r = net.state()
        rec, _, done = net.stats()
    o = job.get()
    assert not over and done == 3
    assert np.array_equal(_sorted_raster(st, ids), o["key"])
    assert rec == len(o["key"]) * 1240
    assert np.array_equal(v.astype(np.float64), o["v"])
    assert np.array_equal(c.astype(np.float64), o["c"])
    assert np.array_equal(r, o["r"])
    return o


def test_full_size_96x96_f16w_three_steps(full_size_oracle):
    """The 96x96 workload (11.43 M neurons, 14.17 G synapses, FP16 weights,
    seed 3): the whole raster and every neuron's state after 3 steps equal
    the oracle's.  Rows j >= 2^32 / row capacity (~3.1 M) start beyond slot
    2^32 of the table, so the deliveries of steps 0 and 1 (delays 1 and 2)
    run through the 64-bit slot arithmetic on most spikers."""
    o = _full_size_steps("cols96x96_f16w", 2, full_size_oracle["cols96x96_f16w"])
    assert o["step_spikes"][0] > 100000 and o["step_spikes"][2] > 0
    assert o["i_max"] > (1 << 32) // 1384


def test_full_size_48x48_f32w_three_steps(full_size_oracle):
    """The 48x48 FP32-weight comparison network (2.86 M neurons, 3.54 G
    synapses, seed 3): whole raster and state after 3 steps."""
    o = _full_size_steps("cols48x48_f32w", 3, full_size_oracle["cols48x48_f32w"])
    assert o["step_spikes"][0] > 10000
