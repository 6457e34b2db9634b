"""FP64 reference statistics of the population-rate / ISI-CV criterion.

The criterion: over 10 s of model time, the population rates of the exact
fixed-point paths (FP32 and FP16 weights) lie within 2 % of the FP64 model's
and their ISI CV within 5 %.  A single 10 s run of these networks alternates
Up and Down states and its rates spread by about 10 % from seed to seed, so
the comparison is made between ensembles: the same seeds (the same networks,
initial states and external input draws) simulated by the FP64 oracle here
and by the GPU paths in the test.

This script runs the oracle only (FP64 mode) and writes
fp64_ensemble_2x2.json: per seed, the E and I spike counts and ISI CVs over
steps [transient, transient + steps).  `stats` is the observable both sides
use (the GPU test imports it; it holds none of the model's arithmetic).

  python tests/golden/fp64_ensemble.py [n_seeds] [workers]
"""
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))

GRID = (2, 2)
SEED0 = 10000
TRANSIENT = 500       # steps (ms) discarded: the initial synchronous volley
STEPS = 10000         # the 10 s window that is measured
MIN_ISIS = 5          # neurons with at least this many ISIs enter the CV mean
OUT = os.path.join(HERE, "fp64_ensemble_2x2.json")


def stats(t, i, n_per_col, n_exc, n_cols, t0, t1):
    """Spike counts and mean ISI CV per population over steps [t0, t1).

    ISI CV of a neuron: population standard deviation over mean of the
    intervals between its consecutive spikes in the window; the population
    value is the mean over its neurons with at least MIN_ISIS intervals."""
    t = np.asarray(t, np.int64)
    i = np.asarray(i, np.int64)
    keep = (t >= t0) & (t < t1)
    t, i = t[keep], i[keep]
    exc = (i % n_per_col) < n_exc
    out = {"spikes_e": int(exc.sum()), "spikes_i": int((~exc).sum())}
    order = np.lexsort((t, i))
    ts, is_ = t[order], i[order]
    same = is_[1:] == is_[:-1]
    isi = (ts[1:] - ts[:-1])[same].astype(np.float64)
    who = is_[1:][same]
    N = n_per_col * n_cols
    cnt = np.bincount(who, minlength=N)
    s1 = np.bincount(who, weights=isi, minlength=N)
    s2 = np.bincount(who, weights=isi * isi, minlength=N)
    ok = cnt >= MIN_ISIS
    mean = np.where(ok, s1 / np.maximum(cnt, 1), 1.0)
    var = np.where(ok, s2 / np.maximum(cnt, 1) - mean * mean, 0.0)
    cv = np.sqrt(np.maximum(var, 0.0)) / mean
    pop_e = (np.arange(N) % n_per_col) < n_exc
    for name, sel in (("e", pop_e), ("i", ~pop_e)):
        m = ok & sel
        out["cv_" + name] = float(cv[m].mean()) if m.any() else float("nan")
        out["n_cv_" + name] = int(m.sum())
    return out


def _one(seed):
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1511_09325_gb300 import workloads as W

    n, s = W.neuron_params(), W.synapse_params()
    p = oracle.make_params(GRID[0], GRID[1], n, s, seed)
    o = oracle.run(p, "f64", TRANSIENT + STEPS, want_state=False)
    r = stats(o["t"], o["i"], n["n_per_col"], n["n_exc"], GRID[0] * GRID[1], TRANSIENT,
              TRANSIENT + STEPS)
    r["seed"] = seed
    return r


def main():
    n_seeds = int(sys.argv[1]) if len(sys.argv) > 1 else 512
    workers = int(sys.argv[2]) if len(sys.argv) > 2 else max(1, (os.cpu_count() or 2) - 2)
    sys.path.insert(0, ROOT)
    import oracle

    oracle.build()
    t0 = time.time()
    with mp.get_context("spawn").Pool(workers) as pool:
        rows = pool.map(_one, range(SEED0, SEED0 + n_seeds), chunksize=1)
    doc = {
        "what": "FP64 oracle: per-seed E/I spike counts and mean ISI CV of 2x2-column "
                "networks (1240 neurons per column, default parameters), steps "
                "[%d, %d)" % (TRANSIENT, TRANSIENT + STEPS),
        "grid": list(GRID), "seed0": SEED0, "n_seeds": n_seeds, "transient": TRANSIENT,
        "steps": STEPS, "min_isis": MIN_ISIS, "mode": "f64",
        "writer": "tests/golden/fp64_ensemble.py (oracle only)",
        "seconds": time.time() - t0, "rows": rows,
    }
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=0)
    print("wrote", OUT, "in %.0f s" % doc["seconds"])


if __name__ == "__main__":
    main()
