"""ctypes front end of the CPU oracle (``oracle/snn_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users.  The GPU library never
imports this package and shares no code with it.

``build()`` compiles the C file with gcc (``-ffp-contract=off`` so that the
float operations stay exactly as written).  All functions take the parameter
dictionaries of :mod:`paper_1511_09325_gb300.workloads`.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "snn_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MODE_F32W, MODE_F16W, MODE_F64 = 0, 1, 2
MODES = {"f32w": MODE_F32W, "f16w": MODE_F16W, "f64": MODE_F64}
Q_SIZE = 65536
POIS_CAP = 128


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("grid_w", ctypes.c_int32), ("grid_h", ctypes.c_int32),
        ("n_per_col", ctypes.c_int32), ("n_exc", ctypes.c_int32),
        ("tau_m", ctypes.c_float), ("theta", ctypes.c_float),
        ("v_reset", ctypes.c_float), ("t_ref", ctypes.c_float),
        ("tau_c", ctypes.c_float), ("dc", ctypes.c_float),
        ("gc_exc", ctypes.c_float), ("gc_inh", ctypes.c_float),
        ("j_ext", ctypes.c_float), ("nu_ext_khz", ctypes.c_float),
        ("k_out", ctypes.c_int32), ("frac_local", ctypes.c_float),
        ("lambda_cols", ctypes.c_float), ("stencil_radius", ctypes.c_int32),
        ("w_exc", ctypes.c_float), ("w_inh", ctypes.c_float),
        ("w_cv", ctypes.c_float), ("d_min", ctypes.c_int32),
        ("d_max", ctypes.c_int32), ("h", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("connectivity", ctypes.c_int32),
        ("p_local", ctypes.c_float), ("remote_a", ctypes.c_float),
        ("remote_sigma", ctypes.c_float), ("remote_cutoff", ctypes.c_float),
    ]


def build(force=False):
    """Compile liboracle.so next to the source (idempotent)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call([
        "gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared",
        "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        vp = ctypes.c_void_p
        L.orc_philox4x32_10.argtypes = [vp, vp, vp]
        L.orc_philox4x32_10.restype = None
        L.orc_validate.argtypes = [P(OrcParams)]
        L.orc_tables_export.argtypes = [P(OrcParams)] + [vp] * 9
        L.orc_synapses.argtypes = [P(OrcParams), ctypes.c_int, ctypes.c_int64,
                                   ctypes.c_int64] + [vp] * 6
        L.orc_ext_counts.argtypes = [P(OrcParams), ctypes.c_int64, ctypes.c_int64,
                                     ctypes.c_int64, ctypes.c_int64, vp]
        L.orc_neuron_trace.argtypes = [P(OrcParams), ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int64, vp, vp, vp, vp, vp]
        L.orc_init_v.argtypes = [P(OrcParams), ctypes.c_int, ctypes.c_int64, ctypes.c_int64, vp]
        L.orc_surr_xi.argtypes = [P(OrcParams), ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                  ctypes.c_int64, vp]
        L.orc_paper_tables.argtypes = [P(OrcParams)] + [vp] * 6
        L.orc_paper_synapses.argtypes = [P(OrcParams), ctypes.c_int, ctypes.c_int64,
                                         ctypes.c_int64, ctypes.c_int64] + [vp] * 7
        L.orc_run.argtypes = [P(OrcParams), ctypes.c_int, ctypes.c_int64,
                              ctypes.c_int64] + [vp] * 8
        for f in ("orc_validate", "orc_tables_export", "orc_synapses", "orc_init_v",
                  "orc_ext_counts", "orc_neuron_trace", "orc_run", "orc_surr_xi",
                  "orc_paper_tables", "orc_paper_synapses"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def make_params(grid_w, grid_h, neuron, synapse, seed, h=1.0):
    """Fill the oracle's parameter struct from workload dictionaries."""
    p = OrcParams()
    p.grid_w, p.grid_h = grid_w, grid_h
    p.n_per_col, p.n_exc = neuron["n_per_col"], neuron["n_exc"]
    p.tau_m, p.theta, p.v_reset = neuron["tau_m"], neuron["theta"], neuron["v_reset"]
    p.t_ref, p.tau_c, p.dc = neuron["t_ref"], neuron["tau_c"], neuron["dc"]
    p.gc_exc, p.gc_inh = neuron["gc_exc"], neuron["gc_inh"]
    p.j_ext, p.nu_ext_khz = neuron["j_ext_mV"], neuron["nu_ext_kHz"]
    p.k_out, p.frac_local = synapse["k_out"], synapse["frac_local"]
    p.lambda_cols, p.stencil_radius = synapse["lambda_cols"], synapse["stencil_radius"]
    p.w_exc, p.w_inh, p.w_cv = synapse["w_exc_mV"], synapse["w_inh_mV"], synapse["w_cv"]
    p.d_min, p.d_max = synapse["d_min"], synapse["d_max"]
    p.h = h
    p.seed = seed
    p.connectivity = synapse.get("connectivity", 0)
    p.p_local = synapse.get("p_local", 0.8)
    p.remote_a = synapse.get("remote_a", 0.05)
    p.remote_sigma = synapse.get("remote_sigma", 1.0)
    p.remote_cutoff = synapse.get("remote_cutoff", 0.001)
    return p


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed with status %d" % (what, rc))


def philox(counter, key):
    """Philox4x32-10 of one 128-bit counter under a 64-bit key (4 + 2 words)."""
    c = np.asarray(counter, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def tables(p):
    """The oracle's FP64 tables: dict of stencil, Poisson, quantile, propagators."""
    n_off = ctypes.c_int32()
    n_pois = ctypes.c_int32()
    dx = np.zeros(64, np.int32)
    dy = np.zeros(64, np.int32)
    sthr = np.zeros(64, np.uint64)
    pthr = np.zeros(POIS_CAP, np.uint64)
    q = np.zeros(Q_SIZE, np.float64)
    props = np.zeros(4, np.float64)
    ints = np.zeros(3, np.int32)
    _check(lib().orc_tables_export(ctypes.byref(p), ctypes.byref(n_off), _ptr(dx), _ptr(dy),
                                   _ptr(sthr), ctypes.byref(n_pois), _ptr(pthr), _ptr(q),
                                   _ptr(props), _ptr(ints)), "tables")
    n, m = n_off.value, n_pois.value
    return dict(off_dx=dx[:n], off_dy=dy[:n], stencil_thr=sthr[:n],
                pois_thr=pthr[:m], q=q, pvv=props[0], pcc=props[1],
                pvc_e=props[2], pvc_i=props[3], jx=int(ints[0]),
                nref=int(ints[1]), k_local=int(ints[2]))


def synapses(p, mode, j0, n):
    """Outgoing synapses of neurons j0..j0+n-1, k order: dict of arrays [n, k_out]."""
    K = p.k_out
    tot = n * K
    tgt = np.zeros(tot, np.int64)
    dly = np.zeros(tot, np.int32)
    wfx = np.zeros(tot, np.int32)
    w = np.zeros(tot, np.float64)
    dx = np.zeros(tot, np.int32)
    dy = np.zeros(tot, np.int32)
    _check(lib().orc_synapses(ctypes.byref(p), MODES[mode] if isinstance(mode, str) else mode,
                              j0, n, _ptr(tgt), _ptr(dly), _ptr(wfx), _ptr(w),
                              _ptr(dx), _ptr(dy)), "synapses")
    sh = (n, K)
    return dict(target=tgt.reshape(sh), delay=dly.reshape(sh), wfx=wfx.reshape(sh),
                w=w.reshape(sh), dx=dx.reshape(sh), dy=dy.reshape(sh))


def paper_tables(p):
    """The paper law's kept remote offsets, their thresholds, the local
    threshold and the number of candidates per neuron."""
    n_off = ctypes.c_int32()
    dx = np.zeros(64, np.int32)
    dy = np.zeros(64, np.int32)
    thr = np.zeros(64, np.uint64)
    lthr = ctypes.c_uint64()
    nc = ctypes.c_int64()
    _check(lib().orc_paper_tables(ctypes.byref(p), ctypes.byref(n_off), _ptr(dx), _ptr(dy),
                                  _ptr(thr), ctypes.byref(lthr), ctypes.byref(nc)),
           "paper_tables")
    n = n_off.value
    return dict(dx=dx[:n], dy=dy[:n], thr=thr[:n], local_thr=lthr.value, n_cand=nc.value)


def paper_synapses(p, mode, j0, n):
    """Synapses of neurons j0..j0+n-1 under the paper law: dict of count[n]
    and flat arrays (row r's synapses follow those of rows < r, in k order)."""
    cap = paper_tables(p)["n_cand"]
    tot = n * cap
    cnt = np.zeros(n, np.int64)
    tgt = np.zeros(tot, np.int64)
    dly = np.zeros(tot, np.int32)
    wfx = np.zeros(tot, np.int32)
    w = np.zeros(tot, np.float64)
    dx = np.zeros(tot, np.int32)
    dy = np.zeros(tot, np.int32)
    _check(lib().orc_paper_synapses(ctypes.byref(p), MODES[mode] if isinstance(mode, str) else mode,
                                    j0, n, cap, _ptr(cnt), _ptr(tgt), _ptr(dly), _ptr(wfx),
                                    _ptr(w), _ptr(dx), _ptr(dy)), "paper_synapses")
    keep = (np.arange(cap)[None, :] < cnt[:, None]).ravel()
    return dict(count=cnt, target=tgt[keep], delay=dly[keep], wfx=wfx[keep], w=w[keep],
                dx=dx[keep], dy=dy[keep])


def ext_counts(p, i0, n, t0, n_steps=None):
    """External event counts k_i(t): shape [n] for one step, [n_steps, n] else."""
    nt = 1 if n_steps is None else n_steps
    k = np.zeros(nt * n, np.int32)
    _check(lib().orc_ext_counts(ctypes.byref(p), i0, n, t0, nt, _ptr(k)), "ext_counts")
    return k if n_steps is None else k.reshape(nt, n)


def surr_xi(p, i0, n, t0, n_steps):
    """Normal draws xi[t][i] of the relaxed network (Philox stream SURR)."""
    xi = np.zeros(n_steps * n, np.float64)
    _check(lib().orc_surr_xi(ctypes.byref(p), i0, n, t0, n_steps, _ptr(xi)), "surr_xi")
    return xi.reshape(n_steps, n)


def init_v(p, mode, i0, n):
    """Initial membrane potentials of neurons i0..i0+n-1."""
    mode = MODES[mode] if isinstance(mode, str) else mode
    v = np.zeros(n, np.float64)
    _check(lib().orc_init_v(ctypes.byref(p), mode, i0, n, _ptr(v)), "init_v")
    return v


def neuron_trace(p, mode, pop, v0, c0, inputs):
    """Single neuron under an explicit input sequence (fx ints or mV doubles)."""
    mode = MODES[mode] if isinstance(mode, str) else mode
    n = len(inputs)
    v = np.zeros(n, np.float64)
    c = np.zeros(n, np.float64)
    s = np.zeros(n, np.uint8)
    if mode == MODE_F64:
        inp = np.ascontiguousarray(inputs, dtype=np.float64)
        _check(lib().orc_neuron_trace(ctypes.byref(p), mode, pop, v0, c0, n, None,
                                      _ptr(inp), _ptr(v), _ptr(c), _ptr(s)), "trace")
    else:
        inp = np.ascontiguousarray(inputs, dtype=np.int32)
        _check(lib().orc_neuron_trace(ctypes.byref(p), mode, pop, v0, c0, n, _ptr(inp),
                                      None, _ptr(v), _ptr(c), _ptr(s)), "trace")
    return v, c, s.astype(bool)


def run(p, mode, n_steps, cap=None, want_state=True):
    """Simulate n_steps; returns raster (t, i), per-step counts and final state."""
    mode = MODES[mode] if isinstance(mode, str) else mode
    N = p.grid_w * p.grid_h * p.n_per_col
    if cap is None:
        cap = max(1 << 20, N * n_steps // 8)
    st = np.zeros(cap, np.int32)
    si = np.zeros(cap, np.int32)
    ns = ctypes.c_int64()
    sspk = np.zeros(max(n_steps, 1), np.int64)
    sext = np.zeros(max(n_steps, 1), np.int64)
    v = np.zeros(N, np.float64) if want_state else None
    c = np.zeros(N, np.float64) if want_state else None
    r = np.zeros(N, np.uint8) if want_state else None
    _check(lib().orc_run(ctypes.byref(p), mode, n_steps, cap, _ptr(st), _ptr(si),
                         ctypes.byref(ns), _ptr(sspk), _ptr(sext), _ptr(v), _ptr(c),
                         _ptr(r)), "run")
    n = ns.value
    if n > cap:
        raise RuntimeError("raster capacity %d exceeded (%d spikes)" % (cap, n))
    return dict(t=st[:n].copy(), i=si[:n].copy(), step_spikes=sspk[:n_steps],
                step_ext=sext[:n_steps], v=v, c=c, r=r)
