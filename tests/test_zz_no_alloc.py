"""snn_update_noalloc against the regular entry points, through the C ABI.

snn_update_noalloc serves callers that cannot let the library allocate device
memory (graph capture, memory pre-reserved by another framework's allocator,
real-time loops); it runs the neuron-update kernel on buffers the caller owns
and keeps its scratch in a fixed array inside the library.  Here its two
first steps must reproduce what snn_build + snn_step compute for the same
network: the same spikes, potentials, calcium and refractory counters.  The
network has d_min = 2, so no recurrent input arrives before step 2 and the
caller's input buffer is zero for both calls.  Tolerance: exact, as in the
other parity tests.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

from paper_1511_09325_gb300 import build as B
from paper_1511_09325_gb300 import snn
from paper_1511_09325_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_update_noalloc_matches_snn_step_two_calls():
    import torch

    B.build()
    snn.load()
    torch.cuda.set_device(0)
    gw, gh = 3, 2
    n = W.neuron_params(nu_ext_kHz=3.5)
    s = W.synapse_params(d_min=2)
    N = gw * gh * n["n_per_col"]
    npad = (N + 3) // 4 * 4
    seed = 11
    stream = torch.cuda.current_stream()

    with snn.Net(gw, gh, n, s, seed, "f32w", stream=stream.cuda_stream) as net:
        v0, c0, r0 = net.state()
        ref_states, ref_spikes = [], []
        for step in range(2):
            net.step(1)
            st, ids, over = net.spikes()
            assert not over
            ref_spikes.append(np.sort(ids))
            ref_states.append(net.state())
            assert np.all(st == step)
        _, pop = net.rates()

    dev = torch.device("cuda", 0)
    v = torch.zeros(npad, dtype=torch.float32, device=dev)
    c = torch.zeros(npad, dtype=torch.float32, device=dev)
    r = torch.zeros(npad, dtype=torch.uint8, device=dev)
    inp = torch.zeros(npad, dtype=torch.int32, device=dev)
    spikes = torch.zeros(N, dtype=torch.int32, device=dev)
    cols = torch.zeros(2 * gw * gh, dtype=torch.int64, device=dev)
    v[:N] = torch.from_numpy(v0).to(dev)
    c[:N] = torch.from_numpy(c0).to(dev)
    r[:N] = torch.from_numpy(r0).to(dev)
    torch.cuda.synchronize()

    total = 0
    for step in range(2):
        ns, ne = snn.snn_update_noalloc(
            gw, gh, n, seed, step, v.data_ptr(), c.data_ptr(), r.data_ptr(), inp.data_ptr(),
            spikes.data_ptr(), cols.data_ptr(), stream.cuda_stream)
        got = np.sort(spikes[:ns].cpu().numpy().astype(np.int64))
        assert ns > 0 and ne > 0
        assert np.array_equal(got, ref_spikes[step].astype(np.int64))
        rv, rc, rr = ref_states[step]
        assert np.array_equal(v[:N].cpu().numpy(), rv)
        assert np.array_equal(c[:N].cpu().numpy(), rc)
        assert np.array_equal(r[:N].cpu().numpy(), rr)
        assert int(inp.abs().sum().item()) == 0
        col = cols.cpu().numpy().reshape(-1, 2)
        assert int(col.sum()) == ns
        ids = spikes[:ns].cpu().numpy().astype(np.int64)
        assert np.array_equal(col[:, 0], np.bincount(ids // 1240, weights=(ids % 1240 < 992),
                                                     minlength=gw * gh).astype(np.int64))
        total += ns
    assert total > 0


def test_update_noalloc_rejects_oversized_grid():
    B.build()
    snn.load()
    with pytest.raises(snn.SnnError) as e:
        snn.snn_update_noalloc(129, 128, W.neuron_params(), 1, 0, 16, 16, 16, 16, 16)
    assert e.value.code == snn.SNN_EINVAL
    assert "16384" in snn.snn_last_error()
