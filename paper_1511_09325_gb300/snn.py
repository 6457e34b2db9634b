"""ctypes binding of the C ABI declared in ``include/snn.h``.

Argument marshalling only: every step of the simulation runs in the CUDA
library ``libsnn_gb300.so``.  There is no CPU fallback -- if the library is
missing or no GPU is present the calls raise.  Function names follow the C
ABI (``snn_build``, ``snn_step``, ...); :class:`Net` wraps them for Python.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsnn_gb300.so")

SNN_OK, SNN_EINVAL, SNN_ENOMEM, SNN_ECUDA, SNN_EOVERFLOW, SNN_ETIMEOUT, SNN_ESTATE = (
    0, -1, -2, -3, -4, -5, -6)
SNN_EXACT_F32W, SNN_EXACT_F16W = 0, 1
PRECISIONS = {"f32w": SNN_EXACT_F32W, "f16w": SNN_EXACT_F16W}

# every symbol the header declares
EXPORTS = ("snn_build", "snn_step", "snn_read_spikes", "snn_pending_spikes",
           "snn_set_record_capacity", "snn_read_rates", "snn_stats", "snn_get_state",
           "snn_read_synapses", "snn_row_lengths", "snn_info", "snn_step_profiled", "snn_update_noalloc",
           "snn_debug_offset_count",
           "snn_build_shard", "snn_shard_update", "snn_shard_deliver", "snn_shard_info",
           "snn_shard_geometry",
           "snn_batch_build", "snn_batch_step", "snn_batch_net", "snn_batch_tune",
           "snn_batch_set_wait", "snn_batch_last_error", "snn_batch_destroy",
           "snn_grad_build", "snn_grad_run", "snn_grad_last_error", "snn_grad_destroy",
           "snn_last_error", "snn_destroy")


class SnnError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("snn error %d: %s" % (code, msg))
        self.code = code


class NeuronParams(ctypes.Structure):
    _fields_ = [("n_per_col", ctypes.c_int32), ("n_exc", ctypes.c_int32),
                ("tau_m", ctypes.c_float), ("theta", ctypes.c_float),
                ("v_reset", ctypes.c_float), ("t_ref", ctypes.c_float),
                ("tau_c", ctypes.c_float), ("dc", ctypes.c_float),
                ("gc_exc", ctypes.c_float), ("gc_inh", ctypes.c_float),
                ("j_ext_mV", ctypes.c_float), ("nu_ext_kHz", ctypes.c_float)]


class SynapseParams(ctypes.Structure):
    _fields_ = [("k_out", ctypes.c_int32), ("frac_local", ctypes.c_float),
                ("lambda_cols", ctypes.c_float), ("stencil_radius", ctypes.c_int32),
                ("w_exc_mV", ctypes.c_float), ("w_inh_mV", ctypes.c_float),
                ("w_cv", ctypes.c_float), ("d_min", ctypes.c_int32),
                ("d_max", ctypes.c_int32), ("periodic", ctypes.c_int32),
                ("connectivity", ctypes.c_int32), ("p_local", ctypes.c_float),
                ("remote_a", ctypes.c_float), ("remote_sigma", ctypes.c_float),
                ("remote_cutoff", ctypes.c_float)]


_lib = None


def load(path=LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("CUDA library %s not built (run __graft_entry__.build())" % path)
    L = ctypes.CDLL(path)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    P = ctypes.POINTER
    L.snn_build.argtypes = [i32, i32, P(NeuronParams), P(SynapseParams), ctypes.c_uint64,
                            i32, vp, P(vp)]
    L.snn_step.argtypes = [vp, i64]
    L.snn_build_shard.argtypes = [i32, i32, i32, i32, i32, i32, P(NeuronParams),
                                  P(SynapseParams), ctypes.c_uint64, i32, vp, P(vp)]
    L.snn_shard_update.argtypes = [vp]
    L.snn_shard_deliver.argtypes = [vp, vp, i64, ctypes.c_int32]
    L.snn_shard_info.argtypes = [vp, vp, i32]
    L.snn_shard_geometry.argtypes = [i32, i32, i32, i32, i32, i32, i32, vp, i32]
    L.snn_read_spikes.argtypes = [vp, vp, vp, i64, P(i64)]
    L.snn_pending_spikes.argtypes = [vp, P(i64)]
    L.snn_set_record_capacity.argtypes = [vp, i64]
    L.snn_read_rates.argtypes = [vp, vp, i64, vp]
    L.snn_stats.argtypes = [vp, P(ctypes.c_double), P(ctypes.c_double), P(i64)]
    L.snn_get_state.argtypes = [vp, vp, vp, vp]
    L.snn_read_synapses.argtypes = [vp, i64, i64, vp, vp, vp]
    L.snn_row_lengths.argtypes = [vp, i64, i64, vp]
    L.snn_info.argtypes = [vp, vp, i32]
    L.snn_step_profiled.argtypes = [vp, i64, vp, vp]
    L.snn_debug_offset_count.argtypes = [vp, i64, ctypes.c_int32, ctypes.c_int32]
    L.snn_update_noalloc.argtypes = [i32, i32, P(NeuronParams), ctypes.c_uint64, i64,
                                     vp, vp, vp, vp, vp, P(i64), P(i64), vp, vp]
    L.snn_batch_build.argtypes = [i32, vp, vp, vp, vp, vp, i32, vp, P(vp)]
    L.snn_batch_step.argtypes = [vp, i64]
    L.snn_batch_net.argtypes = [vp, i32]
    L.snn_batch_net.restype = vp
    L.snn_batch_tune.argtypes = [vp, i64, P(ctypes.c_int32)]
    L.snn_batch_set_wait.argtypes = [vp, i64, ctypes.c_int32]
    L.snn_batch_last_error.argtypes = [vp]
    L.snn_batch_last_error.restype = ctypes.c_char_p
    L.snn_batch_destroy.argtypes = [vp]
    L.snn_batch_destroy.restype = None
    L.snn_grad_build.argtypes = [vp, i64, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, vp,
                                 P(vp)]
    L.snn_grad_run.argtypes = [vp, vp, P(ctypes.c_double), vp, vp]
    L.snn_grad_last_error.argtypes = [vp]
    L.snn_grad_last_error.restype = ctypes.c_char_p
    L.snn_grad_destroy.argtypes = [vp]
    L.snn_grad_destroy.restype = None
    L.snn_last_error.argtypes = [vp]
    L.snn_last_error.restype = ctypes.c_char_p
    L.snn_destroy.argtypes = [vp]
    L.snn_destroy.restype = None
    for f in EXPORTS:
        if f not in ("snn_last_error", "snn_destroy", "snn_batch_net", "snn_batch_last_error",
                     "snn_batch_destroy", "snn_grad_last_error", "snn_grad_destroy"):
            getattr(L, f).restype = i32
    _lib = L
    return L


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def neuron_struct(d):
    return NeuronParams(**{k: d[k] for k, _ in NeuronParams._fields_})


SNN_CONN_FIXED, SNN_CONN_PAPER = 0, 1
_SYN_DEFAULTS = dict(connectivity=SNN_CONN_FIXED, p_local=0.8, remote_a=0.05, remote_sigma=1.0,
                     remote_cutoff=0.001)


def synapse_struct(d):
    return SynapseParams(**{k: d.get(k, _SYN_DEFAULTS.get(k)) for k, _ in SynapseParams._fields_})


def snn_last_error(handle=None):
    return load().snn_last_error(handle).decode()


def _check(rc, handle, ok=(SNN_OK,)):
    if rc not in ok:
        raise SnnError(rc, snn_last_error(handle))
    return rc


def snn_build(grid_w, grid_h, neuron, synapse, seed, precision, stream=None):
    """Build a net; returns the opaque handle (an int)."""
    L = load()
    h = ctypes.c_void_p()
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    n = neuron_struct(neuron)
    s = synapse_struct(synapse)
    rc = L.snn_build(int(grid_w), int(grid_h), ctypes.byref(n), ctypes.byref(s),
                     int(seed), prec, stream, ctypes.byref(h))
    _check(rc, None)
    return h.value


def snn_step(handle, n_steps):
    _check(load().snn_step(handle, int(n_steps)), handle)


def snn_build_shard(grid_w, grid_h, x0, y0, w, h, neuron, synapse, seed, precision,
                    stream=None):
    """Build the shard of tile (x0, y0, w, h); returns the opaque handle."""
    L = load()
    hd = ctypes.c_void_p()
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    n = neuron_struct(neuron)
    s = synapse_struct(synapse)
    rc = L.snn_build_shard(int(grid_w), int(grid_h), int(x0), int(y0), int(w), int(h),
                           ctypes.byref(n), ctypes.byref(s), int(seed), prec, stream,
                           ctypes.byref(hd))
    _check(rc, None)
    return hd.value


def snn_shard_update(handle):
    _check(load().snn_shard_update(handle), handle)


def snn_shard_deliver(handle, ids):
    """Deliver step t with the received global spike indices `ids`: a numpy
    int32 array (host) or a contiguous int32 CUDA tensor (device; it must
    stay unchanged until the net's stream has passed the delivery)."""
    if hasattr(ids, "is_cuda") and ids.is_cuda:
        import torch
        if ids.dtype != torch.int32 or not ids.is_contiguous():
            raise TypeError("device ids must be a contiguous int32 tensor")
        rc = load().snn_shard_deliver(handle, ctypes.c_void_p(ids.data_ptr()), int(ids.numel()), 1)
    else:
        a = np.ascontiguousarray(np.asarray(ids, dtype=np.int32))
        rc = load().snn_shard_deliver(handle, _p(a), int(a.size), 0)
    _check(rc, handle)


_GEO_KEYS = ("grid_w", "grid_h", "local_w", "local_h", "ex0", "ey0", "tx0", "ty0", "w", "h")


def snn_shard_info(handle):
    g = np.zeros(10, np.int32)
    _check(load().snn_shard_info(handle, _p(g), 10), handle)
    return {k: int(v) for k, v in zip(_GEO_KEYS, g)}


def snn_shard_geometry(grid_w, grid_h, tile, stencil_radius):
    """The geometry of the shard of `tile` = (x0, y0, w, h) (host only)."""
    x0, y0, w, h = tile
    g = np.zeros(10, np.int32)
    _check(load().snn_shard_geometry(int(grid_w), int(grid_h), int(x0), int(y0), int(w), int(h),
                                     int(stencil_radius), _p(g), 10), None)
    return {k: int(v) for k, v in zip(_GEO_KEYS, g)}


def shard_local_to_global(geo, npc, local_ids):
    """Global neuron indices of a shard's local neuron indices."""
    j = np.asarray(local_ids, np.int64)
    c, l = j // npc, j % npc
    ly, lx = c // geo["local_w"], c % geo["local_w"]
    gx = (geo["ex0"] + lx) % geo["grid_w"]
    gy = (geo["ey0"] + ly) % geo["grid_h"]
    return (gy * geo["grid_w"] + gx) * npc + l


def shard_tile_neurons(geo, npc):
    """Local indices of a shard's tile neurons: tile rows, then columns, then l."""
    ly, lx = np.meshgrid(np.arange(geo["ty0"], geo["ty0"] + geo["h"]),
                         np.arange(geo["tx0"], geo["tx0"] + geo["w"]), indexing="ij")
    c = (ly * geo["local_w"] + lx).reshape(-1, 1)
    return (c * npc + np.arange(npc)).reshape(-1)


def snn_pending_spikes(handle):
    n = ctypes.c_int64()
    _check(load().snn_pending_spikes(handle, ctypes.byref(n)), handle)
    return n.value


def snn_read_spikes(handle, cap=None):
    """Drain the spike records: (steps, ids, overflowed)."""
    if cap is None:
        cap = snn_pending_spikes(handle)
    st = np.zeros(max(cap, 1), np.int32)
    ids = np.zeros(max(cap, 1), np.int32)
    n = ctypes.c_int64()
    rc = _check(load().snn_read_spikes(handle, _p(st), _p(ids), int(cap), ctypes.byref(n)),
                handle, ok=(SNN_OK, SNN_EOVERFLOW))
    return st[:n.value], ids[:n.value], rc == SNN_EOVERFLOW


def _int32_out(a, name):
    """A caller's output array must be writeable, C-contiguous int32: the
    library writes that many int32 values through its pointer."""
    if not (isinstance(a, np.ndarray) and a.dtype == np.int32 and a.flags.c_contiguous
            and a.flags.writeable):
        raise TypeError("%s must be a writeable C-contiguous int32 numpy array" % name)


def snn_read_spikes_into(handle, steps, ids):
    """Drain into preallocated int32 arrays; returns (count, overflowed)."""
    _int32_out(steps, "steps")
    _int32_out(ids, "ids")
    n = ctypes.c_int64()
    rc = _check(load().snn_read_spikes(handle, _p(steps), _p(ids), int(min(len(steps), len(ids))),
                                       ctypes.byref(n)), handle, ok=(SNN_OK, SNN_EOVERFLOW))
    return n.value, rc == SNN_EOVERFLOW


def snn_set_record_capacity(handle, capacity):
    _check(load().snn_set_record_capacity(handle, int(capacity)), handle)


def snn_read_rates(handle, n_cols):
    hz = np.zeros(2 * n_cols, np.float32)
    pop = np.zeros(2, np.float32)
    _check(load().snn_read_rates(handle, _p(hz), hz.size, _p(pop)), handle)
    return hz.reshape(n_cols, 2), pop


def snn_stats(handle):
    r, e, s = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    _check(load().snn_stats(handle, ctypes.byref(r), ctypes.byref(e), ctypes.byref(s)), handle)
    return r.value, e.value, s.value


def snn_get_state(handle, n):
    v = np.zeros(n, np.float32)
    c = np.zeros(n, np.float32)
    r = np.zeros(n, np.uint8)
    _check(load().snn_get_state(handle, _p(v), _p(c), _p(r)), handle)
    return v, c, r


def snn_row_lengths(handle, j0, n):
    c = np.zeros(max(n, 1), np.int32)
    _check(load().snn_row_lengths(handle, int(j0), int(n), _p(c)), handle)
    return c[:n]


def snn_read_synapses(handle, j0, n, k_out=None):
    """Rows j0..j0+n-1: (target, delay, wfx) as [n, k_out] arrays when every
    row has k_out synapses (pass k_out), else flat arrays in row order (see
    snn_row_lengths)."""
    total = int(snn_row_lengths(handle, j0, n).sum())
    tgt = np.zeros(max(total, 1), np.int64)
    d = np.zeros(max(total, 1), np.int32)
    w = np.zeros(max(total, 1), np.int32)
    _check(load().snn_read_synapses(handle, int(j0), int(n), _p(tgt), _p(d), _p(w)), handle)
    tgt, d, w = tgt[:total], d[:total], w[:total]
    if k_out is not None and total == n * k_out:
        sh = (n, k_out)
        return tgt.reshape(sh), d.reshape(sh), w.reshape(sh)
    return tgt, d, w


def snn_info(handle):
    info = np.zeros(9, np.int64)
    _check(load().snn_info(handle, _p(info), 9), handle)
    keys = ("neurons", "synapses", "device_bytes", "synapse_bytes", "row_capacity", "precision",
            "tile", "deliver_blocks", "update_blocks")
    return dict(zip(keys, (int(x) for x in info)))


def snn_debug_offset_count(handle, column, delta, group_only=False):
    """Testing aid: offset one column's delivery item count (see snn.h)."""
    _check(load().snn_debug_offset_count(handle, int(column), int(delta), 1 if group_only else 0),
           handle)


def snn_step_profiled(handle, n_steps):
    """Eager step loop with CUDA events: (ms[update, deliver], bytes[update, deliver])."""
    ms = np.zeros(2, np.float64)
    by = np.zeros(2, np.float64)
    _check(load().snn_step_profiled(handle, int(n_steps), _p(ms), _p(by)), handle)
    return ms, by


def snn_update_noalloc(grid_w, grid_h, neuron, seed, step, v, c, refractory, input_fx,
                       spikes, col_counts=None, stream=None):
    """One neuron-update step on caller-owned device buffers (raw pointers).

    No allocation happens inside the library; see include/snn.h for the buffer
    sizes and alignment.  Returns (n_spikes, ext_events)."""
    n = neuron_struct(neuron)
    ns, ne = ctypes.c_int64(), ctypes.c_int64()
    rc = load().snn_update_noalloc(int(grid_w), int(grid_h), ctypes.byref(n), int(seed), int(step),
                                   v, c, refractory, input_fx, spikes, ctypes.byref(ns),
                                   ctypes.byref(ne), col_counts, stream)
    _check(rc, None)
    return ns.value, ne.value


def snn_destroy(handle):
    if handle:
        load().snn_destroy(handle)


def _bcheck(rc, handle, ok=(SNN_OK,)):
    if rc not in ok:
        raise SnnError(rc, load().snn_batch_last_error(handle).decode())
    return rc


GRAD_PARAMS = ("a_EE", "a_EI", "a_IE", "a_II", "g_c", "nu_ext")


def snn_grad_build(handle, n_steps, checkpoint_every=50, hard=True, beta=5.0,
                   target_rates=(3.0, 8.0)):
    """Differentiable view of an F32W net; returns the opaque handle."""
    h = ctypes.c_void_p()
    tr = np.array(target_rates, np.float64)
    _check(load().snn_grad_build(handle, int(n_steps), int(checkpoint_every), 1 if hard else 0,
                                 float(beta), _p(tr), ctypes.byref(h)), None)
    return h.value


def snn_grad_run(handle, theta, want_grad=True):
    """(loss, rates[2], grad[6] or None) for theta[6]."""
    th = np.ascontiguousarray(theta, np.float64)
    loss = ctypes.c_double()
    rates = np.zeros(2, np.float64)
    grad = np.zeros(6, np.float64) if want_grad else None
    rc = load().snn_grad_run(handle, _p(th), ctypes.byref(loss), _p(rates), _p(grad))
    if rc != SNN_OK:
        raise SnnError(rc, load().snn_grad_last_error(handle).decode())
    return loss.value, rates, grad


def snn_grad_destroy(handle):
    if handle:
        load().snn_grad_destroy(handle)


class Grad:
    """Loss and gradient of the net's differentiable form (see include/snn.h)."""

    def __init__(self, net, n_steps, checkpoint_every=50, hard=True, beta=5.0,
                 target_rates=(3.0, 8.0)):
        self.net = net  # the view reads the net's synapse table: keep it alive
        self.handle = snn_grad_build(net.handle, n_steps, checkpoint_every, hard, beta,
                                     target_rates)

    def loss(self, theta):
        return snn_grad_run(self.handle, theta, want_grad=False)[:2]

    def loss_and_grad(self, theta):
        return snn_grad_run(self.handle, theta, want_grad=True)

    def close(self):
        if self.handle:
            snn_grad_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rate_loss(grad_view, theta):
    """The differentiable form as a torch function of a 6-element parameter
    tensor: forward and backward both run in the CUDA library."""
    import torch

    class _RateLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, th):
            loss, _, g = grad_view.loss_and_grad(th.detach().double().cpu().numpy())
            ctx.save_for_backward(torch.as_tensor(g, dtype=th.dtype, device=th.device))
            return torch.as_tensor(loss, dtype=th.dtype, device=th.device)

        @staticmethod
        def backward(ctx, gout):
            (g,) = ctx.saved_tensors
            return gout * g

    return _RateLoss.apply(theta)


class Member:
    """A net owned by a Batch: every read-only call of Net, no stepping."""

    def __init__(self, handle, grid_w, grid_h, neuron, synapse):
        self.handle = handle
        self.grid_w, self.grid_h = grid_w, grid_h
        self.n_cols = grid_w * grid_h
        self.n = self.n_cols * neuron["n_per_col"]
        self.k_out = synapse["k_out"]

    def spikes(self, cap=None):
        return snn_read_spikes(self.handle, cap)

    def rates(self):
        return snn_read_rates(self.handle, self.n_cols)

    def stats(self):
        return snn_stats(self.handle)

    def state(self):
        return snn_get_state(self.handle, self.n)

    def info(self):
        return snn_info(self.handle)

    def set_record_capacity(self, cap):
        snn_set_record_capacity(self.handle, cap)


class Batch:
    """Independent nets advanced together by one persistent launch."""

    def __init__(self, grids, neurons, synapses, seeds, precision="f32w", stream=None):
        L = load()
        n = len(grids)
        gw = np.array([g[0] for g in grids], np.int32)
        gh = np.array([g[1] for g in grids], np.int32)
        nps = (NeuronParams * n)(*[neuron_struct(x) for x in neurons])
        sps = (SynapseParams * n)(*[synapse_struct(x) for x in synapses])
        sd = np.array(seeds, np.uint64)
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        h = ctypes.c_void_p()
        _bcheck(L.snn_batch_build(n, _p(gw), _p(gh), ctypes.cast(nps, ctypes.c_void_p),
                                  ctypes.cast(sps, ctypes.c_void_p), _p(sd), prec, stream,
                                  ctypes.byref(h)), None)
        self.handle = h.value
        self.members = [Member(L.snn_batch_net(self.handle, k), grids[k][0], grids[k][1],
                               neurons[k], synapses[k]) for k in range(n)]

    def step(self, n_steps):
        _bcheck(load().snn_batch_step(self.handle, int(n_steps)), self.handle)

    def tune(self, steps_per_trial):
        c = ctypes.c_int32()
        _bcheck(load().snn_batch_tune(self.handle, int(steps_per_trial), ctypes.byref(c)), self.handle)
        return c.value

    def set_wait(self, spin_limit, extra_arrivals=0):
        _bcheck(load().snn_batch_set_wait(self.handle, int(spin_limit), int(extra_arrivals)),
                self.handle)

    def close(self):
        if self.handle:
            load().snn_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Net:
    """A grid of cortical columns living on the current CUDA device."""

    def __init__(self, grid_w, grid_h, neuron, synapse, seed, precision="f32w", stream=None):
        self.grid_w, self.grid_h = grid_w, grid_h
        self.neuron, self.synapse = dict(neuron), dict(synapse)
        self.n_cols = grid_w * grid_h
        self.n = self.n_cols * neuron["n_per_col"]
        self.k_out = synapse["k_out"]
        self.handle = snn_build(grid_w, grid_h, neuron, synapse, seed, precision, stream)

    def step(self, n_steps):
        snn_step(self.handle, n_steps)

    def spikes(self, cap=None):
        return snn_read_spikes(self.handle, cap)

    def spikes_into(self, steps, ids):
        return snn_read_spikes_into(self.handle, steps, ids)

    def rates(self):
        return snn_read_rates(self.handle, self.n_cols)

    def stats(self):
        return snn_stats(self.handle)

    def state(self):
        return snn_get_state(self.handle, self.n)

    def synapses(self, j0, n):
        return snn_read_synapses(self.handle, j0, n, self.k_out)

    def row_lengths(self, j0, n):
        return snn_row_lengths(self.handle, j0, n)

    def info(self):
        return snn_info(self.handle)

    def set_record_capacity(self, cap):
        snn_set_record_capacity(self.handle, cap)

    def step_profiled(self, n_steps):
        return snn_step_profiled(self.handle, n_steps)

    def close(self):
        if self.handle:
            snn_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def split_grid(grid_w, grid_h, nx, ny):
    """Tiles (x0, y0, w, h) of an nx x ny partition of a grid_w x grid_h grid,
    row-major; tile sides differ by at most one column."""
    if not (1 <= nx <= grid_w and 1 <= ny <= grid_h):
        raise ValueError("need 1 <= nx <= grid_w and 1 <= ny <= grid_h")
    xs = [grid_w * i // nx for i in range(nx + 1)]
    ys = [grid_h * j // ny for j in range(ny + 1)]
    return [(xs[i], ys[j], xs[i + 1] - xs[i], ys[j + 1] - ys[j])
            for j in range(ny) for i in range(nx)]


def shard_layout(world_size, grid_w, grid_h):
    """nx x ny for world_size shards: the factorisation whose tiles are the
    most nearly square (least halo per tile)."""
    best = None
    for nx in range(1, world_size + 1):
        if world_size % nx:
            continue
        ny = world_size // nx
        if nx > grid_w or ny > grid_h:
            continue
        cost = grid_w / nx + grid_h / ny  # half the perimeter of a tile
        if best is None or cost < best[0]:
            best = (cost, nx, ny)
    if best is None:
        raise ValueError("cannot split a %dx%d grid into %d tiles" % (grid_w, grid_h, world_size))
    return best[1], best[2]


def exchange_spikes(ids, group=None):
    """All-gather of every rank's spike indices of one step over
    torch.distributed: the ranks' counts first, then the id lists padded to
    the largest count.  `ids` is an int32 tensor (CPU for gloo, CUDA for
    NCCL); returns the concatenation over all ranks (rank order)."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size(group)
    n = torch.tensor([ids.numel()], dtype=torch.int64, device=ids.device)
    counts = [torch.zeros_like(n) for _ in range(ws)]
    dist.all_gather(counts, n, group=group)
    counts = [int(c.item()) for c in counts]
    m = max(counts)
    if m == 0:
        return ids.new_zeros(0)
    buf = ids.new_zeros(m)
    buf[:ids.numel()] = ids
    parts = [ids.new_zeros(m) for _ in range(ws)]
    dist.all_gather(parts, buf, group=group)
    return torch.cat([p[:c] for p, c in zip(parts, counts)])


class Shard:
    """The part of a grid_w x grid_h network that one process holds: tile
    (x0, y0, w, h) and the halo rows that target it.  A step is
    update() -> spikes() -> exchange -> deliver(received)."""

    def __init__(self, grid_w, grid_h, tile, neuron, synapse, seed, precision="f32w",
                 stream=None):
        x0, y0, w, h = tile
        self.tile = (int(x0), int(y0), int(w), int(h))
        self.neuron, self.synapse = dict(neuron), dict(synapse)
        self.npc = neuron["n_per_col"]
        self.handle = snn_build_shard(grid_w, grid_h, x0, y0, w, h, neuron, synapse, seed,
                                      precision, stream)
        self.geo = snn_shard_info(self.handle)
        g = self.geo
        self.n_cols = g["local_w"] * g["local_h"]
        self.n = self.n_cols * self.npc

    def local_to_global(self, local_ids):
        """Global neuron indices of local neuron indices."""
        return shard_local_to_global(self.geo, self.npc, local_ids)

    def tile_local_neurons(self):
        """Local indices of the tile's neurons, tile row-major, then l."""
        return shard_tile_neurons(self.geo, self.npc)

    def update(self):
        snn_shard_update(self.handle)

    def spikes(self, cap=None):
        return snn_read_spikes(self.handle, cap)

    def deliver(self, ids):
        snn_shard_deliver(self.handle, ids)

    def state(self):
        return snn_get_state(self.handle, self.n)

    def rates(self):
        return snn_read_rates(self.handle, self.n_cols)

    def stats(self):
        return snn_stats(self.handle)

    def info(self):
        return snn_info(self.handle)

    def close(self):
        if self.handle:
            snn_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
