"""The C-ABI library builds, loads and exports every declared symbol (no GPU).

Only host-side behaviour is exercised here: argument validation happens before
any CUDA call, so invalid parameters are rejected without a device.
"""
import os
import re

import pytest

from paper_1511_09325_gb300 import build as B
from paper_1511_09325_gb300 import snn
from paper_1511_09325_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return snn.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "snn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(snn_[a-z_]+)\s*\(", src)))


def test_header_declares_the_binding_exports():
    assert _declared() == sorted(snn.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_library_is_built_for_sm103a():
    # the fatbin of the in-tree library carries sm_103a code (cuobjdump-free
    # check: the architecture string the linker records)
    B.build()
    data = open(B.LIB, "rb").read()
    assert b"sm_103a" in data or b"sm_103" in data


@pytest.mark.parametrize("field,value", [
    ("n_per_col", 1), ("n_per_col", 4096), ("n_exc", 2000), ("tau_m", 0.0),
    ("nu_ext_kHz", 41.0), ("nu_ext_kHz", -1.0), ("theta", float("nan")),
])
def test_invalid_neuron_params_rejected(lib, field, value):
    n = W.neuron_params(**{field: value})
    with pytest.raises(snn.SnnError) as e:
        snn.snn_build(2, 2, n, W.synapse_params(), 1, "f32w")
    assert e.value.code == snn.SNN_EINVAL
    assert snn.snn_last_error()


@pytest.mark.parametrize("field,value", [
    ("k_out", 0), ("k_out", 4000), ("stencil_radius", 4), ("d_min", 0), ("d_max", 33),
    ("frac_local", 1.5), ("periodic", 0), ("lambda_cols", 0.0),
])
def test_invalid_synapse_params_rejected(lib, field, value):
    s = W.synapse_params(**{field: value})
    with pytest.raises(snn.SnnError) as e:
        snn.snn_build(2, 2, W.neuron_params(), s, 1, "f32w")
    assert e.value.code == snn.SNN_EINVAL


@pytest.mark.parametrize("over", [
    dict(connectivity=2), dict(connectivity=1, p_local=1.5), dict(connectivity=1, remote_a=-0.1),
    dict(connectivity=1, remote_sigma=0.0), dict(connectivity=1, remote_cutoff=0.0),
    # sigma 2 keeps offsets at r = 4 (0.05 e^-2 = 0.0068 > 1e-3): wider than 7x7
    dict(connectivity=1, remote_sigma=2.0),
])
def test_invalid_paper_law_rejected(lib, over):
    s = W.synapse_params(**over)
    with pytest.raises(snn.SnnError) as e:
        snn.snn_build(2, 2, W.neuron_params(), s, 1, "f32w")
    assert e.value.code == snn.SNN_EINVAL


def test_invalid_grid_and_precision_rejected(lib):
    for gw, gh, prec in ((0, 2, 0), (2, -1, 0), (2, 2, 7)):
        with pytest.raises(snn.SnnError) as e:
            snn.snn_build(gw, gh, W.neuron_params(), W.synapse_params(), 1, prec)
        assert e.value.code == snn.SNN_EINVAL


def test_destroy_null_is_noop(lib):
    lib.snn_destroy(None)


def test_calls_on_null_net_fail_cleanly(lib):
    assert lib.snn_step(None, 1) == snn.SNN_EINVAL
    assert lib.snn_stats(None, None, None, None) == snn.SNN_EINVAL
    assert lib.snn_last_error(None) is not None
    assert lib.snn_row_lengths(None, 0, 1, None) == snn.SNN_EINVAL


def test_shard_entry_points_validate_before_touching_a_device(lib):
    n, s = W.neuron_params(), W.synapse_params()
    # tiles outside the grid, n_per_col not a multiple of 4, the paper law:
    # refused before any stream exists
    for args in [(4, 2, (0, 0, 0, 1), n, s), (4, 2, (3, 0, 2, 1), n, s),
                 (4, 2, (-1, 0, 1, 1), n, s), (4, 2, (0, 1, 1, 2), n, s),
                 (4, 2, (0, 0, 2, 2), W.neuron_params(n_per_col=102, n_exc=80), s),
                 (4, 2, (0, 0, 2, 2), n, W.synapse_params(connectivity=1)),
                 (0, 2, (0, 0, 1, 1), n, s)]:
        gw, gh, tile, nn, ss = args
        with pytest.raises(snn.SnnError) as e:
            snn.snn_build_shard(gw, gh, *tile, nn, ss, 1, "f32w")
        assert e.value.code == snn.SNN_EINVAL
    assert lib.snn_shard_update(None) == snn.SNN_EINVAL
    assert lib.snn_shard_deliver(None, None, 0, 0) == snn.SNN_EINVAL
    assert lib.snn_shard_info(None, None, 0) == snn.SNN_EINVAL


def test_gradient_entry_points_refuse_null_arguments(lib):
    import ctypes

    out = ctypes.c_void_p()
    assert lib.snn_grad_build(None, 10, 5, 1, 5.0, None, ctypes.byref(out)) == snn.SNN_EINVAL
    assert out.value is None
    assert lib.snn_grad_build(None, 10, 5, 1, 5.0, None, None) == snn.SNN_EINVAL
    loss = ctypes.c_double()
    assert lib.snn_grad_run(None, None, ctypes.byref(loss), None, None) == snn.SNN_EINVAL
    assert lib.snn_grad_last_error(None) == b""
    lib.snn_grad_destroy(None)


def test_batch_entry_points_validate_before_touching_a_device(lib):
    import ctypes

    grids = [(2, 2), (1, 1)]
    good_n, good_s = [W.neuron_params()] * 2, [W.synapse_params()] * 2
    # no nets, too many nets, a bad member: refused before any stream exists
    for grids_, ns, ss in (([], [], []), ([(1, 1)] * 257, [W.neuron_params()] * 257,
                                          [W.synapse_params()] * 257),
                           (grids, [W.neuron_params(), W.neuron_params(n_exc=5000)], good_s),
                           (grids, good_n, [W.synapse_params(), W.synapse_params(d_min=0)])):
        with pytest.raises(snn.SnnError) as e:
            snn.Batch(grids_, ns, ss, list(range(len(grids_))))
        assert e.value.code == snn.SNN_EINVAL
    with pytest.raises(snn.SnnError) as e:
        snn.Batch([(0, 3)], [W.neuron_params()], [W.synapse_params()], [1])
    assert e.value.code == snn.SNN_EINVAL
    out = ctypes.c_void_p()
    assert lib.snn_batch_build(1, None, None, None, None, None, 0, None,
                               ctypes.byref(out)) == snn.SNN_EINVAL
    assert out.value is None
    assert lib.snn_batch_build(1, None, None, None, None, None, 0, None, None) == snn.SNN_EINVAL
    assert lib.snn_batch_step(None, 1) == snn.SNN_EINVAL
    assert lib.snn_batch_tune(None, 1, None) == snn.SNN_EINVAL
    assert lib.snn_batch_set_wait(None, 1, 0) == snn.SNN_EINVAL
    assert lib.snn_batch_net(None, 0) is None
    assert lib.snn_batch_last_error(None)  # the last refusal's message
    lib.snn_batch_destroy(None)


def test_noalloc_update_validates_before_touching_a_device(lib):
    import numpy as np

    n = W.neuron_params()
    buf = np.zeros(64, np.float32)
    p = buf.ctypes.data  # 16-byte aligned host memory: never dereferenced here

    def call(**kw):
        a = dict(grid_w=1, grid_h=1, neuron=n, seed=1, step=0, v=p, c=p, refractory=p,
                 input_fx=p, spikes=p)
        a.update(kw)
        with pytest.raises(snn.SnnError) as e:
            snn.snn_update_noalloc(**a)
        return e.value.code

    assert call(neuron=W.neuron_params(n_exc=2000)) == snn.SNN_EINVAL
    assert call(grid_w=0) == snn.SNN_EINVAL
    assert call(grid_w=129, grid_h=128) == snn.SNN_EINVAL  # 16 512 columns > 16 384
    assert call(step=-1) == snn.SNN_EINVAL
    assert call(step=1 << 32) == snn.SNN_EINVAL
    assert call(v=None) == snn.SNN_EINVAL
    assert call(spikes=None) == snn.SNN_EINVAL
    assert call(v=p + 4) == snn.SNN_EINVAL  # V must be 16-byte aligned
    assert call(refractory=p + 2) == snn.SNN_EINVAL  # refractory must be 4-byte aligned
    assert call(spikes=p + 2) == snn.SNN_EINVAL  # spike ids are stored as u32
    assert call(col_counts=p + 4) == snn.SNN_EINVAL  # u64 counters


def test_spike_readback_refuses_unsafe_output_arrays(lib):
    """The library writes int32 records through the arrays' pointers, so a
    wrong dtype, a strided view or a read-only array is refused before the
    call (the handle is never used)."""
    import numpy as np

    good = np.zeros(8, np.int32)
    ro = np.zeros(8, np.int32)
    ro.flags.writeable = False
    for bad in (np.zeros(8, np.int16), np.zeros(8, np.int64), np.zeros(16, np.int32)[::2], ro,
                [0] * 8):
        with pytest.raises(TypeError):
            snn.snn_read_spikes_into(None, bad, good)
        with pytest.raises(TypeError):
            snn.snn_read_spikes_into(None, good, bad)
