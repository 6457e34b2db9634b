"""Multi-process paths on CPU ranks (gloo, world sizes 2, 4 and 9).

1. The paper distributes the columns of the grid over MPI processes that
   exchange spikes every step (Sec. 2).  Here each rank owns a tile of
   columns, integrates only its own neurons (the dense restatement of the
   step) and all-gathers its spike index list once per step with the
   library's exchange helper (the minimum delay is one step, so one exchange
   per step suffices); the union of the ranks' rasters must equal the
   single-process oracle's raster bit for bit.  The helper itself is checked
   with uneven and empty lists, and the tiling helpers on their own.
2. bench.py's whole-job reduction over N replicas takes the slowest rank's
   time and the sum of the ranks' events.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


def _partitioned_worker(rank, world, port, steps, out_dir, gw, gh):
    sys.path[:0] = [ROOT, HERE]
    import torch

    import oracle
    from dense_model import DenseNet, simulate
    from paper_1511_09325_gb300 import workloads as W

    dist = _init(rank, world, port)
    n = W.neuron_params(n_per_col=100, n_exc=80, nu_ext_kHz=3.0)
    s = W.synapse_params(k_out=120, d_max=6)
    p = oracle.make_params(gw, gh, n, s, 23)
    net = DenseNet(oracle, p, "f32w")
    ncol = gw * gh  # rank r owns columns [r ncol / world, (r + 1) ncol / world)
    c0, c1 = rank * ncol // world, (rank + 1) * ncol // world
    rows = np.arange(c0 * 100, c1 * 100)

    from paper_1511_09325_gb300 import snn

    def exchange(local):
        mine = torch.from_numpy(np.flatnonzero(local).astype(np.int32))
        got = snn.exchange_spikes(mine).numpy()
        fired = np.zeros(local.size, bool)
        fired[got] = True
        return fired

    raster, v, _, _ = simulate(oracle, net, steps, rows=rows, exchange=exchange)
    np.save(os.path.join(out_dir, "raster%d.npy" % rank), np.array(raster, np.int64).reshape(-1, 2))
    np.save(os.path.join(out_dir, "v%d.npy" % rank), v)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,gw,gh", [(2, 2, 1), (4, 2, 2), (9, 3, 3)])
def test_column_partition_with_spike_exchange_matches_oracle(tmp_path, orc, world, gw, gh):
    from paper_1511_09325_gb300 import workloads as W

    steps = 120
    mp.spawn(_partitioned_worker, args=(world, _free_port(), steps, str(tmp_path), gw, gh),
             nprocs=world, join=True)
    got = np.concatenate([np.load(tmp_path / ("raster%d.npy" % r)) for r in range(world)])
    n = W.neuron_params(n_per_col=100, n_exc=80, nu_ext_kHz=3.0)
    s = W.synapse_params(k_out=120, d_max=6)
    o = orc.run(orc.make_params(gw, gh, n, s, 23), "f32w", steps)
    key = lambda a: np.sort(a[:, 0] * 100000 + a[:, 1])
    want = np.stack([o["t"], o["i"]], 1).astype(np.int64)
    assert len(want) > 200
    assert np.array_equal(key(got), key(want))
    v = np.concatenate([np.load(tmp_path / ("v%d.npy" % r)) for r in range(world)])
    assert np.array_equal(v, o["v"])


def _reduce_worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import bench

    dist = _init(rank, world, port)
    ms, rec, ext = bench.reduce_ranks(dist, 10.0 + rank, 100.0 * (rank + 1), 7.0, "cpu")
    np.save(os.path.join(out_dir, "red%d.npy" % rank), np.array([ms, rec, ext]))
    dist.destroy_process_group()


def test_bench_reduction_over_replicas(tmp_path):
    mp.spawn(_reduce_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        ms, rec, ext = np.load(tmp_path / ("red%d.npy" % r))
        assert ms == 11.0 and rec == 300.0 and ext == 14.0


class _SleepyNet:
    """Stands in for a net in bench._e2e: each step takes `dt` seconds and
    adds `ev` recurrent events; a read drains nothing."""

    def __init__(self, dt, ev):
        self.n, self.dt, self.ev, self.events = 4, dt, ev, 0.0

    def spikes(self):
        return None

    def step(self, k):
        import time

        time.sleep(self.dt * k)
        self.events += self.ev * k

    def spikes_into(self, steps, ids):
        return 0, False

    def stats(self):
        return self.events, 0.0, 0


class _NoCuda:
    class cuda:
        @staticmethod
        def synchronize():
            pass


def _e2e_worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import bench

    dist = _init(rank, world, port)
    net = _SleepyNet(0.01 * (rank + 1), 100.0 * (rank + 1))
    r = bench._e2e(net, _NoCuda, 3, dist, "cpu")
    np.save(os.path.join(out_dir, "e2e%d.npy" % rank), np.array([r["value"]]))
    dist.destroy_process_group()


def test_bench_e2e_is_whole_job_over_ranks(tmp_path):
    """The end-to-end rate of N ranks is the events of all ranks (here 300 +
    600) over the slowest rank's time (3 steps of 20 ms), on every rank."""
    mp.spawn(_e2e_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    v = [float(np.load(tmp_path / ("e2e%d.npy" % r))[0]) for r in range(2)]
    assert v[0] == v[1]
    assert 900.0 / 0.5 < v[0] <= 900.0 / 0.06


def _any_rank_worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import bench

    dist = _init(rank, world, port)
    got = [bench.any_rank(dist, rank == 1, "cpu"), bench.any_rank(dist, False, "cpu")]
    np.save(os.path.join(out_dir, "any%d.npy" % rank), np.array(got))
    dist.destroy_process_group()


def test_bench_remeasure_decision_is_taken_by_all_ranks(tmp_path):
    """One rank's disqualified clock record makes every rank time again (the
    timed region holds barriers, so the ranks must take the same branch)."""
    mp.spawn(_any_rank_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        assert list(np.load(tmp_path / ("any%d.npy" % r))) == [True, False]


def _exchange_worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch

    from paper_1511_09325_gb300 import snn

    dist = _init(rank, world, port)
    # rank r sends r * 3 ids (rank 0 sends none), values 1000 r + k
    mine = torch.arange(rank * 3, dtype=torch.int32) + 1000 * rank
    got = snn.exchange_spikes(mine)
    empty = snn.exchange_spikes(torch.zeros(0, dtype=torch.int32))
    np.save(os.path.join(out_dir, "ex%d.npy" % rank), got.numpy())
    assert empty.numel() == 0
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_spike_exchange_gathers_every_rank_in_order(tmp_path, world):
    mp.spawn(_exchange_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    want = np.concatenate([np.arange(r * 3, dtype=np.int32) + 1000 * r for r in range(world)])
    for r in range(world):
        assert np.array_equal(np.load(tmp_path / ("ex%d.npy" % r)), want)


def test_split_grid_covers_the_grid_once():
    sys.path.insert(0, ROOT)
    from paper_1511_09325_gb300 import snn

    for gw, gh, nx, ny in [(4, 2, 2, 1), (9, 5, 3, 2), (96, 96, 4, 2), (7, 3, 7, 3), (1, 1, 1, 1)]:
        tiles = snn.split_grid(gw, gh, nx, ny)
        assert len(tiles) == nx * ny
        cover = np.zeros((gh, gw), np.int32)
        for x0, y0, w, h in tiles:
            assert w >= 1 and h >= 1
            cover[y0:y0 + h, x0:x0 + w] += 1
        assert np.all(cover == 1)
        ws = sorted(set(w for _, _, w, _ in tiles))
        assert ws[-1] - ws[0] <= 1
    with pytest.raises(ValueError):
        snn.split_grid(2, 2, 3, 1)
    assert snn.shard_layout(2, 96, 96) in [(2, 1), (1, 2)]
    assert snn.shard_layout(4, 96, 96) == (2, 2)
    assert snn.shard_layout(8, 96, 96) in [(4, 2), (2, 4)]
    assert snn.shard_layout(2, 4, 2) == (2, 1)
    assert snn.shard_layout(3, 1, 9) == (1, 3)
