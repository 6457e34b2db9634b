"""Column-tile shards against the CPU oracle, through the C ABI.

The paper distributes the grid's columns over processes that exchange the
step's spikes every step (Sec. 2, Sec. 3).  Here the grid is split into
tiles; each tile is a shard (its columns plus the rows of the halo that end in
them), stepped as update -> read own spikes -> exchange -> deliver.  The union
of the shards' rasters and the tiles' final states must equal the oracle's
single network bit for bit.  Shards of one process share the GPU one after
the other (no kernel waits on another shard); the two-process case exchanges
over gloo through host memory.
"""
import os
import socket
import sys

import numpy as np
import pytest

import oracle
from paper_1511_09325_gb300 import build as B
from paper_1511_09325_gb300 import snn
from paper_1511_09325_gb300 import workloads as W

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    snn.load()
    oracle.build()


def _sorted_raster(t, i):
    return np.sort(np.asarray(t, np.int64) * (1 << 32) + np.asarray(i, np.int64))


def _run_shards(gw, gh, n, s, seed, prec, steps, nx, ny, device_ids=False):
    """Step the shards of an nx x ny split together; the union raster and the
    tiles' states placed at their global neuron indices."""
    npc = n["n_per_col"]
    N = gw * gh * npc
    shards = [snn.Shard(gw, gh, t, n, s, seed, prec) for t in snn.split_grid(gw, gh, nx, ny)]
    ts, ids = [], []
    try:
        for t in range(steps):
            mine = []
            for sh in shards:
                sh.update()
            for sh in shards:
                st, i, over = sh.spikes()
                assert not over
                assert np.all(st == t)
                mine.append(i)
            got = np.concatenate(mine) if mine else np.zeros(0, np.int32)
            ts.append(np.full(got.size, t, np.int64))
            ids.append(got.astype(np.int64))
            if device_ids:
                import torch
                dev = torch.from_numpy(got.astype(np.int32)).cuda()
                torch.cuda.synchronize()  # the copy is on torch's stream
                for sh in shards:
                    sh.deliver(dev)
                torch.cuda.synchronize()
            else:
                for sh in shards:
                    sh.deliver(got)
        v = np.full(N, np.nan, np.float64)
        c = np.full(N, np.nan, np.float64)
        r = np.full(N, 255, np.int64)
        rec = ext = 0.0
        for sh in shards:
            lv, lc, lr = sh.state()
            loc = sh.tile_local_neurons()
            glo = sh.local_to_global(loc)
            assert np.all(np.isnan(v[glo])), "tiles overlap"
            v[glo] = lv[loc]
            c[glo] = lc[loc]
            r[glo] = lr[loc]
            a, b, k = sh.stats()
            assert k == steps
            rec += a
            ext += b
    finally:
        for sh in shards:
            sh.close()
    return dict(t=np.concatenate(ts), i=np.concatenate(ids), v=v, c=c, r=r, rec=rec, ext=ext)


def _check(g, o, k_out):
    assert np.array_equal(_sorted_raster(g["t"], g["i"]), _sorted_raster(o["t"], o["i"]))
    assert np.array_equal(g["v"], o["v"])
    assert np.array_equal(g["c"], o["c"])
    assert np.array_equal(g["r"], o["r"])
    assert g["rec"] == len(o["t"]) * k_out
    assert g["ext"] == float(o["step_ext"].sum())


SMALL_N = dict(n_per_col=100, n_exc=80, nu_ext_kHz=3.0)
SMALL_S = dict(k_out=150, d_min=2, d_max=7, stencil_radius=2)

CASES = {
    # the grids of the two-rank acceptance case, default (paper-sized) columns
    "4x2_f32w_2x1": (4, 2, {}, {}, 1, "f32w", 150, 2, 1),
    "6x6_f16w_2x1": (6, 6, {}, {}, 5, "f16w", 60, 2, 1),
    "6x6_f32w_2x2": (6, 6, {}, {}, 5, "f32w", 60, 2, 2),
    # tile + halo narrower than the grid: the local grid wraps around the
    # global edge (width 13 of 14)
    "14x2_f16w_halo_wraps": (14, 2, {}, {}, 3, "f16w", 60, 2, 1),
    # radius-2 stencil, d_min = 2, three tiles of a 9-wide grid (local grids
    # 7 wide, wrapping), uneven tile heights
    "9x5_small_3x2": (9, 5, SMALL_N, SMALL_S, 9, "f32w", 300, 3, 2),
    "9x5_small_3x2_f16w": (9, 5, SMALL_N, SMALL_S, 9, "f16w", 300, 3, 2),
    # one shard holding the whole grid
    "3x3_one_shard": (3, 3, {}, {}, 2, "f32w", 80, 1, 1),
    # d_min = 1 with a single delay, one-column-wide tiles
    "5x1_single_delay": (5, 1, SMALL_N, dict(k_out=150, d_min=1, d_max=1), 4, "f32w", 300, 5, 1),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_shards_match_oracle(name):
    gw, gh, nov, sov, seed, prec, steps, nx, ny = CASES[name]
    n, s = W.neuron_params(**nov), W.synapse_params(**sov)
    g = _run_shards(gw, gh, n, s, seed, prec, steps, nx, ny)
    o = oracle.run(oracle.make_params(gw, gh, n, s, seed), prec, steps)
    assert len(o["t"]) > 100
    _check(g, o, s["k_out"])


def test_shards_take_device_spike_lists():
    n, s = W.neuron_params(**SMALL_N), W.synapse_params(**SMALL_S)
    g = _run_shards(9, 5, n, s, 9, "f16w", 120, 3, 2, device_ids=True)
    o = oracle.run(oracle.make_params(9, 5, n, s, 9), "f16w", 120)
    _check(g, o, s["k_out"])


def test_shard_rows_hold_the_synapses_into_the_tile():
    """Row lengths of a shard = the oracle's synapses of the neuron that end
    in the tile (every one of them, halo neurons included)."""
    n, s = W.neuron_params(**SMALL_N), W.synapse_params(**SMALL_S)
    gw, gh = 9, 5
    p = oracle.make_params(gw, gh, n, s, 9)
    with snn.Shard(gw, gh, (3, 0, 3, 3), n, s, 9, "f32w") as sh:
        g = sh.geo
        assert (g["local_w"], g["local_h"]) == (7, 5)
        assert (g["ex0"], g["tx0"], g["ey0"], g["ty0"]) == (1, 2, 0, 0)
        own = set(int(x) for x in sh.local_to_global(sh.tile_local_neurons()))
        lens = snn.snn_row_lengths(sh.handle, 0, sh.n)
        glo = sh.local_to_global(np.arange(sh.n))
        for j_loc in range(0, sh.n, 37):
            o = oracle.synapses(p, "f32w", int(glo[j_loc]), 1)
            want = sum(1 for t in o["target"].reshape(-1) if int(t) in own)
            assert lens[j_loc] == want


def test_shard_call_order_and_bad_indices_are_errors():
    n, s = W.neuron_params(**SMALL_N), W.synapse_params(**SMALL_S)
    with snn.Shard(9, 5, (0, 0, 3, 5), n, s, 9, "f32w") as sh:
        with pytest.raises(snn.SnnError) as e:
            sh.deliver(np.zeros(0, np.int32))  # update is due first
        assert e.value.code == snn.SNN_ESTATE
        sh.update()
        with pytest.raises(snn.SnnError) as e:
            sh.update()  # delivery is due first
        assert e.value.code == snn.SNN_ESTATE
        with pytest.raises(snn.SnnError) as e:
            snn.snn_step(sh.handle, 1)  # a shard does not step as a whole net
        assert e.value.code == snn.SNN_ESTATE
        sh.spikes()
        # an index beyond the network: skipped by the kernel, status set
        sh.deliver(np.array([9 * 5 * 100 + 7], np.int32))
        with pytest.raises(snn.SnnError) as e:
            sh.spikes()
        assert e.value.code == snn.SNN_ESTATE
    with snn.Shard(9, 5, (0, 0, 3, 5), n, s, 9, "f32w") as sh:
        sh.update()
        sh.spikes()
        # neuron 0 of halo column (8, 0) listed 101 times: more spikes than
        # the column has neurons
        sh.deliver(np.full(101, 8 * 100, np.int32))
        with pytest.raises(snn.SnnError) as e:
            sh.spikes()
        assert e.value.code == snn.SNN_ESTATE


def _free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def _rank_worker(rank, world, port, out_dir, gw, gh, prec, steps):
    sys.path[:0] = [ROOT, HERE]
    import torch
    import torch.distributed as dist

    from paper_1511_09325_gb300 import snn as S
    from paper_1511_09325_gb300 import workloads as WL

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    n, s = WL.neuron_params(), WL.synapse_params()
    nx, ny = S.shard_layout(world, gw, gh)
    tile = S.split_grid(gw, gh, nx, ny)[rank]
    ts, ids = [], []
    with S.Shard(gw, gh, tile, n, s, 1, prec) as sh:
        for t in range(steps):
            sh.update()
            st, i, over = sh.spikes()
            assert not over and np.all(st == t)
            got = S.exchange_spikes(torch.from_numpy(i.astype(np.int32)))
            sh.deliver(got.numpy())
            ts.append(st.astype(np.int64))
            ids.append(i.astype(np.int64))
        v, c, r = sh.state()
        loc = sh.tile_local_neurons()
        glo = sh.local_to_global(loc)
        np.savez(os.path.join(out_dir, "rank%d.npz" % rank), t=np.concatenate(ts),
                 i=np.concatenate(ids), glo=glo, v=v[loc], c=c[loc], r=r[loc])
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("gw,gh,prec,steps", [(4, 2, "f32w", 100), (6, 6, "f16w", 40)])
def test_two_ranks_over_gloo_match_oracle(tmp_path, gw, gh, prec, steps):
    """world_size 2: two processes, one shard each, on the same GPU; the
    exchange is an all-gather of spike index lists over gloo."""
    import torch.multiprocessing as mp

    mp.start_processes(_rank_worker, args=(2, _free_port(), str(tmp_path), gw, gh, prec, steps),
                       nprocs=2, join=True, start_method="spawn")
    n, s = W.neuron_params(), W.synapse_params()
    o = oracle.run(oracle.make_params(gw, gh, n, s, 1), prec, steps)
    N = gw * gh * n["n_per_col"]
    v = np.full(N, np.nan)
    c = np.full(N, np.nan)
    r = np.full(N, 255, np.int64)
    ts, ids = [], []
    for k in range(2):
        z = np.load(os.path.join(str(tmp_path), "rank%d.npz" % k))
        ts.append(z["t"])
        ids.append(z["i"])
        v[z["glo"]] = z["v"]
        c[z["glo"]] = z["c"]
        r[z["glo"]] = z["r"]
    assert np.array_equal(_sorted_raster(np.concatenate(ts), np.concatenate(ids)),
                          _sorted_raster(o["t"], o["i"]))
    assert np.array_equal(v, o["v"]) and np.array_equal(c, o["c"]) and np.array_equal(r, o["r"])
