"""Oracle runs in parallel processes, for the GPU tests that compare several
networks (or one large one) with the oracle.

The workers are started with the "spawn" method (a process forked after the
CUDA context exists can hang), each builds its network's parameters from
plain dictionaries and returns the sorted raster keys and the final state.
"""
import multiprocessing as mp
import os

import numpy as np


def raster_key(t, i):
    return np.sort(np.asarray(t, np.int64) * (1 << 32) + np.asarray(i, np.int64))


def _job(args):
    grid, neuron, synapse, seed, prec, steps, cap = args
    import oracle

    oracle.build()
    p = oracle.make_params(grid[0], grid[1], neuron, synapse, seed)
    o = oracle.run(p, prec, steps, cap=cap)
    return dict(key=raster_key(o["t"], o["i"]), v=o["v"], c=o["c"], r=o["r"],
                step_spikes=o["step_spikes"], i_max=int(o["i"].max()) if len(o["i"]) else -1)


class OraclePool:
    """Submit oracle runs; results arrive in submission order."""

    def __init__(self, workers=None):
        n = workers or max(1, min(8, os.cpu_count() or 1))
        self.pool = mp.get_context("spawn").Pool(n)

    def submit(self, grid, neuron, synapse, seed, prec, steps, cap=None):
        return self.pool.apply_async(_job, ((tuple(grid), dict(neuron), dict(synapse), seed, prec,
                                              steps, cap),))

    def map(self, jobs):
        handles = [self.submit(*j) for j in jobs]
        return [h.get() for h in handles]

    def close(self):
        self.pool.close()
        self.pool.join()
