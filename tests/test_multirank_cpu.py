"""Multi-process paths on CPU ranks (gloo, world sizes 2, 4 and 9).

1. The paper distributes the columns of the grid over MPI processes that
   exchange spikes every step (Sec. 2).  Here each rank owns a tile of
   columns, integrates only its own neurons (the dense restatement of the
   step) and all-gathers the spike vector once per step (the minimum delay is
   one step, so one exchange per step suffices); the union of the ranks'
   rasters must equal the single-process oracle's raster bit for bit.
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

    def exchange(local):
        mine = torch.from_numpy(local.astype(np.uint8))
        parts = [torch.zeros_like(mine) for _ in range(world)]
        dist.all_gather(parts, mine)
        return np.logical_or.reduce([q.numpy().astype(bool) for q in parts])

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
