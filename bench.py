"""Benchmark: synaptic events/s of the column-network step on GB300.

A bench step is one 1 ms simulation step (neuron update + spike delivery) of
the 96x96-column network (11.43 M neurons, 14.17 G synapses, FP16 weights,
seed 3) unless --workload names another one.  The network first runs
--settle untimed steps (past the initial synchronous volley), then W warm-up
steps, then the K timed steps; the line reports that window's own activity.
Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--settle S]
                  [--workload NAME] [--impl ours|reference] [--no-extra]

N > 1 runs N independent replicas (one network per GPU, seed + rank), launched
with torch.distributed.run; rank 0 prints the whole-job line.
--sharded runs ONE network split into N x M column tiles instead (M =
--shards-per-gpu shards per rank, stepped in turn; the step's spike index
lists are gathered on each rank and all-gathered over torch.distributed every
step; with N = M = 1 the single shard holds the whole grid and nothing is
exchanged, which times the split step's host round trip).
--impl reference times the CPU oracle on a bounded sample of the workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1511_09325_gb300 import workloads as W  # noqa: E402

METRIC = "synaptic events/s and wall-s per model-s on 1 GB300; FP16-weight vs plain FP32 path"
UNIT = "events/s"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--workload", default="cols96x96_f16w")
    ap.add_argument("--settle", type=int, default=2000,
                    help="untimed steps after the build, before the warm-up")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the 96x96 FP16-vs-FP32 comparison and the batched form")
    ap.add_argument("--profile-steps", type=int, default=None,
                    help="steps of the per-kernel timing pass (default: all timed steps)")
    ap.add_argument("--e2e-steps", type=int, default=1000)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--sharded", action="store_true",
                    help="one network split into column tiles over the ranks")
    ap.add_argument("--shards-per-gpu", type=int, default=1,
                    help="--sharded: tiles each rank holds (stepped in turn on its GPU)")
    return ap.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _traffic(workload, window, kernel):
    """DRAM bytes per launch of a kernel over exactly this window (workload,
    settle, warm-up and timed steps) from the committed ncu summary, or None
    when there is none or the kernel source changed since it was taken."""
    import hashlib

    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            t = json.load(f)
        src = os.path.join(ROOT, "paper_1511_09325_gb300", "csrc", "snn_step.cu")
        with open(src, "rb") as f:
            digest = hashlib.sha256(f.read()).hexdigest()
        if not digest.startswith(t.get("kernel_sha256", "-")):
            return None
        w = t.get(workload, {})
        if [w.get("settle"), w.get("warmup"), w.get("steps")] != list(window):
            return None
        return w.get(kernel)
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons while running."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.out = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        return parse_clocks(out, self.uuid)


def parse_clocks(text, uuid=""):
    """Median SM clock, its maximum and the throttle reasons seen, from the
    CSV lines of Clocks.FIELDS (no header, no units) of the GPU `uuid` (all
    lines when empty).  None when no line parses."""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in text.splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9 or (uuid and not uuid.startswith(f[0][:12]) and uuid not in f[0]):
            continue
        try:
            sm.append(float(f[1]))
            mx.append(float(f[2]))
        except ValueError:
            continue
        for n, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
            "reasons": sorted(reasons), "samples": len(sm)}


def clocks_rejected(clk, floor=0.85):
    """True when a clock record disqualifies the timing it covers: a hardware
    or thermal slowdown was active, or the median SM clock sat below `floor`
    of its maximum with no reason given (a clock lock left by someone else).
    A power cap alone is kept (and shows in the record)."""
    if not clk:
        return False
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    if bad & set(clk["reasons"]):
        return True
    return not clk["reasons"] and clk["sm_mhz"] < floor * clk["sm_max_mhz"]


def any_rank(dist, flag, device):
    """The flag of every rank or-ed together (so that all ranks take the same
    branch around a collective)."""
    if not dist:
        return bool(flag)
    import torch

    t = torch.tensor([1 if flag else 0], device=device, dtype=torch.int32)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return bool(t.item())


# The oracle's sample of each workload: the same construction on a grid the
# oracle steps in seconds (one oracle step of the 96x96 network takes about a
# minute).
CPU_SLICE = {"cols96x96_f16w": "cols48x48_f16w", "cols96x96_f32w": "cols48x48_f32w"}


def _cpu_baseline(workload, seconds_target=15.0):
    """The oracle, as it stands, on a bounded sample of the workload: the
    first steps of its CPU slice from the initial state."""
    import oracle

    sample = CPU_SLICE.get(workload, workload)
    cfg = W.WORKLOADS[sample]
    n, s = W.neuron_params(), W.synapse_params(**cfg.get("synapse", {}))
    p = oracle.make_params(cfg["grid_w"], cfg["grid_h"], n, s, cfg["seed"])
    mode = cfg["precision"]
    oracle.build()
    steps = 1
    while True:
        t0 = time.perf_counter()
        o = oracle.run(p, mode, steps, want_state=False)
        dt = time.perf_counter() - t0
        if dt > seconds_target / 3 or steps >= 64:
            break
        steps *= 2
    events = float(len(o["t"])) * s["k_out"]
    return {"value": events / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%s, first %d steps from the initial state (%d spikes), single thread"
                      % (sample, steps, len(o["t"])),
            "seconds": dt, "all_cores": _cpu_all_cores(sample, steps)}


# One oracle process: set up, report ready, wait for the start line, run the
# sample and print its recurrent events and seconds.
_ORACLE_REPLICA = r"""
import sys, time
sys.path.insert(0, sys.argv[1])
import oracle
from paper_1511_09325_gb300 import workloads as W
cfg = W.WORKLOADS[sys.argv[2]]
n, s = W.neuron_params(), W.synapse_params(**cfg.get("synapse", {}))
p = oracle.make_params(cfg["grid_w"], cfg["grid_h"], n, s, cfg["seed"])
print("ready", flush=True)
sys.stdin.readline()
t0 = time.perf_counter()
o = oracle.run(p, cfg["precision"], int(sys.argv[3]), want_state=False)
print(len(o["t"]) * s["k_out"], time.perf_counter() - t0, flush=True)
"""


def _cpu_all_cores(workload, steps):
    """The same sample on every host core at once: one single-thread oracle
    process per core, started together (the oracle itself is serial, so the
    host's aggregate rate is that of independent copies).  Each copy holds
    only the neuron state and the delay ring (the synapses are regenerated
    on the fly), ~60 MB at 24x24.  Returns None if any copy fails."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    procs = []
    try:
        for _ in range(cores):
            procs.append(subprocess.Popen(
                [sys.executable, "-c", _ORACLE_REPLICA, ROOT, workload, str(steps)],
                stdin=subprocess.PIPE, stdout=subprocess.PIPE, text=True))
        if any(q.stdout.readline().strip() != "ready" for q in procs):
            return None
        for q in procs:
            q.stdin.write("go\n")
            q.stdin.flush()
        res = [q.stdout.readline().split() for q in procs]
        events = sum(float(r[0]) for r in res)
        slowest = max(float(r[1]) for r in res)
    except (OSError, ValueError, IndexError):
        return None
    finally:
        for q in procs:
            if q.poll() is None:
                q.kill()
            q.wait()
    return {"value": events / slowest, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d single-thread oracle processes at once, each on the first %d "
                      "steps of %s; events of all over the slowest one's time"
                      % (cores, steps, workload)}


# Reference arm: the oracle on the workload's CPU slice; each bench step is one
# oracle step, so the driver's K and W set the length of the run.
REF_SLICE = {"cols96x96_f16w": "cols24x24_f16w", "cols96x96_f32w": "cols24x24_f32w",
             "cols48x48_f16w": "cols24x24_f16w", "cols48x48_f32w": "cols24x24_f32w"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle

    sample = REF_SLICE.get(args.workload, args.workload)
    cfg = W.WORKLOADS[sample]
    n, s = W.neuron_params(), W.synapse_params(**cfg.get("synapse", {}))
    p = oracle.make_params(cfg["grid_w"], cfg["grid_h"], n, s, cfg["seed"])
    oracle.build()
    wu = max(args.warmup, 0)
    t0 = time.perf_counter()
    if wu:
        oracle.run(p, cfg["precision"], wu, want_state=False)
    t1 = time.perf_counter()
    o2 = oracle.run(p, cfg["precision"], wu + args.steps, want_state=False)
    t2 = time.perf_counter()
    # timed: the K steps after the W warm-up ones (the second run repeats the
    # warm-up, whose time the first run measured)
    secs = max((t2 - t1) - (t1 - t0), 1e-9)
    spikes = int(o2["step_spikes"][wu:].sum())
    value = spikes * s["k_out"] / secs
    main = W.WORKLOADS[args.workload]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": secs * 1e3 / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+i32" if main["precision"] == "f32w" else "f16+i32",
        "data": "synthetic", "config": _config(args, main, None, args.gpus),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "%s (the workload's construction at %dx%d), steps %d..%d "
                                   "from the initial state, single thread"
                                   % (sample, cfg["grid_w"], cfg["grid_h"], wu,
                                      wu + args.steps - 1)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _config(args, cfg, info=None, ws=1):
    """The config object of the JSON line (the same for both arms)."""
    return {"workload": args.workload, "grid": [cfg["grid_w"], cfg["grid_h"]],
            "precision": cfg["precision"], "seed": cfg["seed"], "parallelism": "replicas%d" % ws,
            "settle_steps": getattr(args, "settle", 0),
            "l2": "inputs larger than L2 (the synapse table)"}


def reduce_ranks(dist, ms, rec_ev, ext_ev, device):
    """Whole-job numbers of N replicas: the slowest rank's time, the sum of
    every rank's events (value = events of all ranks / that time)."""
    import torch

    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ev = torch.tensor([rec_ev, ext_ev], device=device, dtype=torch.float64)
    dist.all_reduce(ev)
    return float(t.item()), float(ev[0].item()), float(ev[1].item())


def _build_net(snn, torch, cfg, seed, stream):
    n, s = W.neuron_params(), W.synapse_params(**cfg.get("synapse", {}))
    t0 = time.perf_counter()
    net = snn.Net(cfg["grid_w"], cfg["grid_h"], n, s, seed, cfg["precision"],
                  stream=stream.cuda_stream)
    torch.cuda.synchronize()
    return net, time.perf_counter() - t0


def _timed(net, torch, stream, steps, barrier=None):
    """Device time of `steps` graph-replayed steps, barrier + sync on both sides."""
    torch.cuda.synchronize()
    if barrier:
        barrier()
    r0, e0, _ = net.stats()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    net.step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    ms = ev0.elapsed_time(ev1)
    r1, e1, _ = net.stats()
    return ms, r1 - r0, e1 - e0


def _kernel_roofline(snn, torch, cfg, seed, stream, lead, P, workload, window):
    """Per-kernel device time and algorithmic bytes over the timed window.

    A second net with the same seed replays the identical window (the
    simulation is deterministic: `lead` untimed steps, then the P timed ones)
    with every kernel bracketed by CUDA events on the net's stream."""
    twin, _ = _build_net(snn, torch, cfg, seed, stream)
    twin.step(lead)
    twin.spikes()
    kms, kbytes = twin.step_profiled(P)
    twin.close()
    torch.cuda.empty_cache()
    hbm, peak_kind = _peaks()
    dom = 0 if kms[0] >= kms[1] else 1
    kname = ["update_kernel", "deliver_kernel"][dom]
    achieved = kbytes[dom] / (kms[dom] * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm,
            "unit": "GB/s", "frac": achieved / hbm, "peak_kind": peak_kind,
            "traffic": _traffic(workload, window, kname), "launches": P,
            "kernel_ms": {"update": kms[0] / P, "deliver": kms[1] / P},
            "kernel_gbs": {"update": kbytes[0] / (kms[0] * 1e-3) / 1e9,
                           "deliver": kbytes[1] / (kms[1] * 1e-3) / 1e9},
            "kernel_frac": {"update": kbytes[0] / (kms[0] * 1e-3) / 1e9 / hbm,
                            "deliver": kbytes[1] / (kms[1] * 1e-3) / 1e9 / hbm},
            "algorithmic_bytes_per_launch": {"update": kbytes[0] / P, "deliver": kbytes[1] / P},
            "bytes_model": "update 26 B per neuron + 12 B per spike; deliver per spike k_out x "
                           "record bytes (4 B FP16 record: 15-bit weight + 17-bit target; 8 B "
                           "FP32 record) + 6 B per delay bucket (descriptor id and bucket end)"}


def _e2e(net, torch, E, dist=None, device="cuda"):
    """Same metric through the public API with host buffers: every step is
    one snn_step call followed by one drain of that step's spike records into
    host arrays (device -> host copies and stream sync inside the region).
    With several ranks: the events of all ranks over the slowest rank's time."""
    import numpy as np

    net.spikes()
    torch.cuda.synchronize()
    steps_buf = np.zeros(net.n, np.int32)
    ids_buf = np.zeros(net.n, np.int32)
    r0, _, _ = net.stats()
    d2h = 0
    t0 = time.perf_counter()
    for _ in range(E):
        net.step(1)
        n, _ = net.spikes_into(steps_buf, ids_buf)
        d2h += 8 * n + 16  # records, plus the drain header
    dt = time.perf_counter() - t0
    r1, _, _ = net.stats()
    ms, ev = dt * 1e3, r1 - r0
    if dist:
        ms, ev, _ = reduce_ranks(dist, ms, ev, 0.0, device)
    return {"value": ev / (ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": 0,
            "d2h_bytes_per_step": d2h / E, "steps": E}


def run_ours(args):
    import torch

    from paper_1511_09325_gb300 import build as B
    from paper_1511_09325_gb300 import snn

    ws, rank, local = _dist()
    dist = None
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if rank == 0:
        B.build()
    if dist:
        dist.barrier()
    snn.load()
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    uuid = str(getattr(props, "uuid", "") or "")
    if uuid and not uuid.startswith("GPU-"):
        uuid = "GPU-" + uuid
    cfg = W.WORKLOADS[args.workload]
    stream = torch.cuda.Stream()
    seed = cfg["seed"] + rank
    K, Wm, S = args.steps, args.warmup, args.settle

    clocks = Clocks(uuid)
    clocks.start()
    net, build_s = _build_net(snn, torch, cfg, seed, stream)
    net.step(S)
    net.spikes()
    net.step(Wm)
    net.spikes()
    net.rates()  # opens the rate window of the timed steps
    ms, rec_ev, ext_ev = _timed(net, torch, stream, K, dist.barrier if dist else None)
    clk = clocks.stop()
    remeasured = False
    if any_rank(dist, clocks_rejected(clk), "cuda"):
        # a slowed or locked clock disqualifies the window: time the next one
        remeasured = True
        net.rates()
        clocks = Clocks(uuid)
        clocks.start()
        ms, rec_ev, ext_ev = _timed(net, torch, stream, K, dist.barrier if dist else None)
        clk = clocks.stop()
    if clk is not None:
        clk["remeasured"] = remeasured
        clk["rejected"] = bool(clocks_rejected(clk))
    _, pop_hz = net.rates()
    spikes_window = rec_ev / W.SYNAPSE["k_out"]
    if dist:
        ms, rec_ev, ext_ev = reduce_ranks(dist, ms, rec_ev, ext_ev, "cuda")
    info = net.info()
    e2e = _e2e(net, torch, max(1, min(args.e2e_steps, max(K, 1))), dist)
    net.close()
    torch.cuda.empty_cache()
    P = K if args.profile_steps is None else min(args.profile_steps, K)
    lead = S + Wm + (K if remeasured else 0)
    roofline = _kernel_roofline(snn, torch, cfg, seed, stream, lead, max(1, P), args.workload,
                                (S, Wm, K))

    extra = batched = surrogate = paper = crit = None
    if not args.no_extra and ws == 1:
        extra = _precision_form(snn, torch, stream, S)
        crit = _fp64_criterion(snn, torch, stream)
        batched = _batched_form(snn, torch, stream)
        surrogate = _surrogate_form(snn, torch, stream)
        paper = _paper_form(snn, torch, stream, Wm)
    cpu = None
    if ws == 1 and not args.no_cpu:
        cb = _cpu_baseline(args.workload)
        cpu = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "all_cores")}

    if dist:
        dist.barrier()
    if rank == 0:
        line = {
            "metric": METRIC, "value": rec_ev / (ms * 1e-3), "unit": UNIT, "n_gpus": ws,
            "steps": K, "warmup": Wm, "ms_per_step": ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+i32" if cfg["precision"] == "f32w" else "f16+i32",
            "data": "synthetic",
            "config": _config(args, cfg, None, args.gpus),
            "window": {"first_step": lead, "steps": K,
                       "state": "after %d settle and %d warm-up steps (model time %.3f s)"
                                % (S, Wm, lead * 1e-3),
                       "spikes_per_step": spikes_window / K,
                       "pop_hz": [float(pop_hz[0]), float(pop_hz[1])]},
            "neurons": info["neurons"], "synapses": info["synapses"],
            "synapse_table_gb": info["synapse_bytes"] / 1e9,
            "wall_s_per_model_s": ms / K,
            "paper_convention_events_per_s": (rec_ev + ext_ev) / (ms * 1e-3),
            "build_s": build_s,
            "gpu_launches": 2 * K,
            "roofline": roofline,
            "e2e": e2e,
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        if extra:
            line["precision_form"] = extra
        if crit:
            line["fp64_criterion"] = crit
        if batched:
            line["batched_form"] = batched
        if surrogate:
            line["surrogate_gradient"] = surrogate
        if paper:
            line["paper_connectivity"] = paper
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def _surrogate_form(snn, torch, stream, steps=500, ckpt=50):
    """The differentiable form on 4x4 columns (19 840 neurons, 24.6 M
    synapses, seed 11): 500 steps, checkpoints every 50, hard spikes with the
    surrogate derivative; time of the forward pass alone and of forward plus
    checkpointed backward (the library call synchronises)."""
    theta = [1.0, 1.0, 1.0, 1.0, 0.02, 2.5]
    n, s = W.neuron_params(), W.synapse_params()
    out = {"workload": "cols4x4", "steps": steps, "checkpoint_every": ckpt, "mode": "hard"}
    net = snn.Net(4, 4, n, s, 11, "f32w", stream=stream.cuda_stream)
    g = snn.Grad(net, steps, checkpoint_every=ckpt, hard=True)
    g.loss_and_grad(theta)  # warm-up
    t0 = time.perf_counter()
    for _ in range(3):
        loss, rates = g.loss(theta)
    fwd = (time.perf_counter() - t0) / 3
    t0 = time.perf_counter()
    for _ in range(3):
        loss, rates, grad = g.loss_and_grad(theta)
    both = (time.perf_counter() - t0) / 3
    g.close()
    net.close()
    out.update(forward_ms=fwd * 1e3, forward_backward_ms=both * 1e3,
               forward_backward_ms_per_step=both * 1e3 / steps, loss=loss,
               rates_hz=[float(x) for x in rates], grad=[float(x) for x in grad])
    return out


def _batched_form(snn, torch, stream, steps=2000, n_nets=64):
    """64 independent nets (grids 1x1..8x8, seeds 100-163, external rates
    1.5-3.5 kHz) advanced by one persistent launch per call, against the same
    nets stepped one after the other with their own graphs."""
    grids, neurons, synapses, seeds = W.batch_workload(n_nets)
    out = {"workload": "batch64", "nets": n_nets, "steps": steps,
           "neurons": int(sum(g[0] * g[1] for g in grids) * 1240)}
    t0 = time.perf_counter()
    b = snn.Batch(grids, neurons, synapses, seeds, "f32w", stream=stream.cuda_stream)
    torch.cuda.synchronize()
    out["build_s"] = time.perf_counter() - t0
    choice = b.tune(25)
    out["tuned_choice"] = choice
    out["tuned_schedule"] = {"sector_rounds_in_flight": [2, 2, 1, 1][choice % 4],
                             "windows": choice % 2 == 0,
                             "delivery_blocks_per_column": [8, 4, 2, 1][choice // 4]}
    tuned_steps = 2 * 2 * 4 * 25  # two stages of two rounds of four candidates
    r0 = [m.stats()[0] for m in b.members]
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    b.step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    r1 = [m.stats()[0] for m in b.members]
    b.close()
    hbm, _ = _peaks()
    alg = _batch_bytes(grids, neurons, synapses, [c - a for a, c in zip(r0, r1)], steps)
    out["events_per_s"] = (sum(r1) - sum(r0)) / (ms * 1e-3)
    out["ms_per_step"] = ms / steps
    out["algorithmic_bytes_per_step"] = alg / steps
    out["step_gbs"] = alg / (ms * 1e-3) / 1e9
    out["step_frac_hbm"] = out["step_gbs"] / hbm
    # the same nets, one by one, same steps after the same warm-up
    total_ms, ev_seq = 0.0, []
    for g, n, s, sd in zip(grids, neurons, synapses, seeds):
        net = snn.Net(g[0], g[1], n, s, sd, "f32w", stream=stream.cuda_stream)
        net.step(tuned_steps)
        torch.cuda.synchronize()
        a0 = net.stats()[0]
        ev0.record(stream)
        net.step(steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        total_ms += ev0.elapsed_time(ev1)
        ev_seq.append(net.stats()[0] - a0)
        net.close()
    alg_seq = _batch_bytes(grids, neurons, synapses, ev_seq, steps)
    out["sequential_ms_per_step"] = total_ms / steps
    out["sequential_events_per_s"] = sum(ev_seq) / (total_ms * 1e-3)
    out["sequential_step_gbs"] = alg_seq / (total_ms * 1e-3) / 1e9
    out["batch_speedup"] = total_ms / ms
    return out


def _batch_bytes(grids, neurons, synapses, events, steps):
    """Algorithmic bytes of `steps` steps of several FP32-weight nets with
    `events` recurrent synaptic events each: per neuron and step 26 B (state
    and input), per spike 12 B (list entry and record) + k_out 8-byte records
    + 6 B per delay bucket (list entry and bucket end), as for one net."""
    total = 0.0
    for g, n, s, ev in zip(grids, neurons, synapses, events):
        N = g[0] * g[1] * n["n_per_col"]
        spikes = ev / s["k_out"]
        ndel = s["d_max"] - s["d_min"] + 1
        total += 26.0 * N * steps + spikes * (12.0 + 8.0 * s["k_out"] + 6.0 * ndel)
    return total


def _precision_form(snn, torch, stream, settle, steps=2000):
    """96x96 columns (14.17 G synapses), FP16 weights vs FP32 weights: the
    same network (seed 3) after `settle` untimed steps, then `steps` timed
    graph-replayed steps (about two Up/Down cycles), then the first 500 of the
    following steps with per-kernel events."""
    out = {"workload": "cols96x96", "settle": settle, "steps": steps}
    free, _ = torch.cuda.mem_get_info()
    for prec in ("f16w", "f32w"):
        cfg = W.WORKLOADS["cols96x96_" + prec]
        need = 11427840 * (1384 * (4 if prec == "f16w" else 8) + 140 + 21 * 32)
        if need > free * 0.97:
            out[prec] = {"skipped": "needs %.0f GB of %.0f GB free" % (need / 1e9, free / 1e9)}
            continue
        net, build_s = _build_net(snn, torch, cfg, cfg["seed"], stream)
        net.step(settle)
        net.spikes()
        net.rates()
        ms, rec_ev, ext_ev = _timed(net, torch, stream, steps)
        _, pop = net.rates()
        net.spikes()
        kms, kb = net.step_profiled(min(steps, 500))
        hbm, _ = _peaks()
        gbs = (kb[0] + kb[1]) / ((kms[0] + kms[1]) * 1e-3) / 1e9
        out[prec] = {"events_per_s": rec_ev / (ms * 1e-3), "wall_s_per_model_s": ms / steps,
                     "ms_per_step": ms / steps, "build_s": build_s,
                     "spikes_per_step": rec_ev / W.SYNAPSE["k_out"] / steps,
                     "pop_rates_hz": [float(pop[0]), float(pop[1])],
                     "step_gbs": gbs, "step_frac_hbm": gbs / hbm,
                     "deliver_gbs": kb[1] / (kms[1] * 1e-3) / 1e9,
                     "deliver_frac_hbm": kb[1] / (kms[1] * 1e-3) / 1e9 / hbm,
                     "update_gbs": kb[0] / (kms[0] * 1e-3) / 1e9}
        net.close()
        torch.cuda.empty_cache()
    if "events_per_s" in out.get("f16w", {}) and "events_per_s" in out.get("f32w", {}):
        out["fp16_speedup_wall"] = out["f32w"]["ms_per_step"] / out["f16w"]["ms_per_step"]
    return out


def _fp64_criterion(snn, torch, stream, n_seeds=256):
    """The rate / ISI-CV criterion against the FP64 model on the first
    n_seeds networks of the stored FP64 ensemble (2x2 columns, 10 s after a
    0.5 s transient; tests/golden/fp64_ensemble_2x2.json, written by the
    oracle): each path runs the same networks through the batched form, and
    the ensemble-mean relative errors come with their paired standard
    errors."""
    import numpy as np

    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    import fp64_ensemble as F

    path = os.path.join(ROOT, "tests", "golden", "fp64_ensemble_2x2.json")
    with open(path) as f:
        gold = json.load(f)
    rows_ref = gold["rows"][:n_seeds]
    seeds = [r["seed"] for r in rows_ref]
    n, s = W.neuron_params(), W.synapse_params()
    ncols = F.GRID[0] * F.GRID[1]
    secs = F.STEPS / 1000.0

    def obs(rows):
        return {"rate_e": np.array([r["spikes_e"] for r in rows]) / (n["n_exc"] * ncols * secs),
                "rate_i": np.array([r["spikes_i"] for r in rows])
                          / ((n["n_per_col"] - n["n_exc"]) * ncols * secs),
                "cv_e": np.array([r["cv_e"] for r in rows]),
                "cv_i": np.array([r["cv_i"] for r in rows])}

    ref = obs(rows_ref)
    out = {"networks": len(seeds), "model_s": secs, "transient_s": F.TRANSIENT / 1000.0,
           "reference": "FP64 oracle, %s" % os.path.relpath(path, ROOT),
           "bounds": {"rates": 0.02, "isi_cv": 0.05}}
    for prec in ("f16w", "f32w"):
        rows = []
        t0 = time.perf_counter()
        with snn.Batch([F.GRID] * len(seeds), [n] * len(seeds), [s] * len(seeds), seeds, prec,
                       stream=stream.cuda_stream) as b:
            for m in b.members:
                m.set_record_capacity(1 << 20)
            ts = [[] for _ in seeds]
            ids = [[] for _ in seeds]
            done, total = 0, F.TRANSIENT + F.STEPS
            while done < total:
                k = min(1000, total - done)
                b.step(k)
                done += k
                for j, m in enumerate(b.members):
                    t, i, _ = m.spikes()
                    ts[j].append(t)
                    ids[j].append(i)
        for j in range(len(seeds)):
            rows.append(F.stats(np.concatenate(ts[j]), np.concatenate(ids[j]), n["n_per_col"],
                                n["n_exc"], ncols, F.TRANSIENT, F.TRANSIENT + F.STEPS))
        got = obs(rows)
        res = {"seconds": time.perf_counter() - t0}
        for k in ref:
            g, f = got[k], ref[k]
            ok = np.isfinite(g) & np.isfinite(f)
            res[k] = {"rel_error": float(g[ok].mean() / f[ok].mean() - 1.0),
                      "paired_se": float(np.std(g[ok] - f[ok], ddof=1) / np.sqrt(ok.sum())
                                         / f[ok].mean())}
        out[prec] = res
    return out


def _paper_form(snn, torch, stream, warmup, steps=2000):
    """24x24 columns under the paper's own connectivity law (Bernoulli local,
    Gaussian remote, variable out-degree): same metric, same timing."""
    cfg = W.WORKLOADS["cols24x24_paper_f32w"]
    net, build_s = _build_net(snn, torch, cfg, cfg["seed"], stream)
    info = net.info()
    net.step(warmup)
    net.spikes()
    ms, rec_ev, _ = _timed(net, torch, stream, steps)
    _, pop = net.rates()
    kms, kb = net.step_profiled(min(steps, 500))
    net.close()
    torch.cuda.empty_cache()
    return {"workload": "cols24x24_paper_f32w", "steps": steps, "warmup": warmup,
            "synapses": info["synapses"], "build_s": build_s,
            "events_per_s": rec_ev / (ms * 1e-3), "ms_per_step": ms / steps,
            "pop_rates_hz": [float(pop[0]), float(pop[1])],
            "deliver_gbs": kb[1] / (kms[1] * 1e-3) / 1e9,
            "update_gbs": kb[0] / (kms[0] * 1e-3) / 1e9}


def run_sharded(args):
    """One network of the workload split into column tiles, M per rank.  A
    step: update of every own tile, drain of their spike records (global
    indices, device -> host), the concatenated lists all-gathered over the
    ranks (one rank: nothing to send), delivery of the received spikes into
    each tile.  Timed on the host clock (the step waits for the exchange)
    with a barrier and a device sync on both sides; value = synaptic events
    of all ranks / the slowest rank's time."""
    import numpy as np
    import torch

    from paper_1511_09325_gb300 import build as B
    from paper_1511_09325_gb300 import snn

    ws, rank, local = _dist()
    dist = None
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if rank == 0:
        B.build()
    if dist:
        dist.barrier()
    snn.load()
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    uuid = str(getattr(props, "uuid", "") or "")
    if uuid and not uuid.startswith("GPU-"):
        uuid = "GPU-" + uuid
    cfg = W.WORKLOADS[args.workload]
    n, s = W.neuron_params(), W.synapse_params(**cfg.get("synapse", {}))
    M = max(1, args.shards_per_gpu)
    nx, ny = snn.shard_layout(ws * M, cfg["grid_w"], cfg["grid_h"])
    tiles = snn.split_grid(cfg["grid_w"], cfg["grid_h"], nx, ny)[rank * M:(rank + 1) * M]
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    shards = [snn.Shard(cfg["grid_w"], cfg["grid_h"], t, n, s, cfg["seed"], cfg["precision"],
                        stream=stream.cuda_stream) for t in tiles]
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    nbytes = {"h2d": 0, "d2h": 0}
    alone = ws == 1 and M == 1

    def step():
        for sh in shards:
            sh.update()
        mine = []
        for sh in shards:
            _, ids, over = sh.spikes()
            if over:
                raise RuntimeError("spike records dropped")
            nbytes["d2h"] += 8 * ids.size + 16
            mine.append(ids.astype(np.int32))
        if alone:
            shards[0].deliver(np.zeros(0, np.int32))
            return
        mine = np.concatenate(mine)
        if dist:
            with torch.cuda.stream(stream):
                dev = torch.from_numpy(mine).to("cuda")
                got = snn.exchange_spikes(dev)
            nbytes["h2d"] += 4 * mine.size
            for sh in shards:
                sh.deliver(got)
        else:
            nbytes["h2d"] += 4 * mine.size * len(shards)
            for sh in shards:
                sh.deliver(mine)

    def stats():
        r = e = 0.0
        for sh in shards:
            a, b, _ = sh.stats()
            r += a
            e += b
        return r, e

    K, Wm, S = args.steps, args.warmup, args.settle
    for _ in range(S + Wm):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(uuid)
    clocks.start()
    r0, e0 = stats()
    nbytes["h2d"] = nbytes["d2h"] = 0
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(K):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = (time.perf_counter() - t0) * 1e3
    clk = clocks.stop()
    if clk is not None:
        clk["rejected"] = bool(clocks_rejected(clk))
    r1, e1 = stats()
    rec_ev, ext_ev = r1 - r0, e1 - e0
    own_ms = ms
    if dist:
        ms, rec_ev, ext_ev = reduce_ranks(dist, ms, rec_ev, ext_ev, "cuda")
    kept = sum(sh.info()["synapses"] for sh in shards)
    geo = [[sh.geo["local_w"], sh.geo["local_h"]] for sh in shards]
    for sh in shards:
        sh.close()
    if rank == 0:
        value = rec_ev / (ms * 1e-3)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K,
            "warmup": Wm, "ms_per_step": ms / K, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "mode": "sharded",
            "dtype": "f32+i32" if cfg["precision"] == "f32w" else "f16+i32",
            "data": "synthetic",
            "config": dict(_config(args, cfg, None, ws), parallelism="tiles%dx%d" % (nx, ny),
                           shards_per_gpu=M,
                           exchange=("all-gather of spike index lists" if dist else
                                     "host concatenation" if not alone else "none (1 shard)")),
            "rank0": {"tiles": [list(t) for t in tiles], "local_grids": geo,
                      "synapses_kept": kept, "ms": own_ms},
            "build_s": build_s,
            # per shard: update, record drain, ingest of the received list
            # (when one is sent), delivery
            "gpu_launches": (3 if alone else 4) * M * K,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": nbytes["h2d"] / K,
                    "d2h_bytes_per_step": nbytes["d2h"] / K,
                    "note": "the sharded step itself crosses the host every step"},
            "roofline": None,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    elif args.sharded:
        run_sharded(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
