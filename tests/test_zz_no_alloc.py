"""snn_update_noalloc against the regular entry points and the oracle, through
the C ABI.

snn_update_noalloc serves callers that cannot let the library allocate device
memory -- a process whose device memory is already reserved by another
framework's allocator, or a real-time loop that cannot afford an allocation's
implicit synchronisation.  It runs the neuron-update kernel on buffers the
caller owns and keeps its scratch in a fixed array inside the library.

* Two calls in a row must reproduce what snn_build + snn_step compute for the
  same network: the same spikes, potentials, calcium and refractory counters
  (a network with d_min = 2, so that the caller's input is zero for both).
* Two calls in a row with a nonzero input pattern in the caller's input
  buffer must give, neuron by neuron, the oracle's single-neuron trace under
  that input plus the external Poisson input of the step, and must leave the
  input buffer cleared; the grid has 1238 neurons per column, so N is not a
  multiple of 4 and the padded tail is exercised.
* After a warm-up call, a call must not change the device's free memory.

Tolerance: exact, as in the other parity tests.  This file is collected last
so that a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

import oracle
from paper_1511_09325_gb300 import build as B
from paper_1511_09325_gb300 import snn
from paper_1511_09325_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    snn.load()
    oracle.build()


def test_update_noalloc_matches_snn_step_two_calls():
    import torch

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


def test_update_noalloc_nonzero_input_matches_oracle_trace():
    import torch

    torch.cuda.set_device(0)
    gw, gh = 1, 1
    n = W.neuron_params(n_per_col=1238, n_exc=990)
    N = gw * gh * n["n_per_col"]
    npad = (N + 3) // 4 * 4
    seed, t0 = 23, 40
    p = oracle.make_params(gw, gh, n, W.synapse_params(), seed)
    v0 = oracle.init_v(p, "f32w", 0, N)
    # caller input of two steps: deterministic values in about -4 .. +5 mV
    rng = np.random.default_rng(5)
    inputs = rng.integers(-4 * 65536, 5 * 65536, size=(2, N)).astype(np.int32)
    k = oracle.ext_counts(p, 0, N, t0, 2)

    stream = torch.cuda.current_stream()
    dev = torch.device("cuda", 0)
    v = torch.zeros(npad, dtype=torch.float32, device=dev)
    c = torch.zeros(npad, dtype=torch.float32, device=dev)
    r = torch.zeros(npad, dtype=torch.uint8, device=dev)
    inp = torch.zeros(npad, dtype=torch.int32, device=dev)
    spikes = torch.zeros(N, dtype=torch.int32, device=dev)
    v[:N] = torch.from_numpy(v0.astype(np.float32)).to(dev)
    torch.cuda.synchronize()

    want_v = np.zeros((2, N))
    want_c = np.zeros((2, N))
    want_s = np.zeros((2, N), bool)
    for i in range(N):
        pop = 0 if i < n["n_exc"] else 1
        tot = inputs[:, i].astype(np.int64) + k[:, i].astype(np.int64) * 26214
        vo, co, so = oracle.neuron_trace(p, "f32w", pop, float(np.float32(v0[i])), 0.0,
                                         tot.astype(np.int32))
        want_v[:, i], want_c[:, i], want_s[:, i] = vo, co, so

    for step in range(2):
        inp[:N] = torch.from_numpy(inputs[step]).to(dev)
        torch.cuda.synchronize()
        ns, ne = snn.snn_update_noalloc(gw, gh, n, seed, t0 + step, v.data_ptr(), c.data_ptr(),
                                        r.data_ptr(), inp.data_ptr(), spikes.data_ptr(), None,
                                        stream.cuda_stream)
        assert ne == int(k[step].sum())
        got = np.sort(spikes[:ns].cpu().numpy().astype(np.int64))
        assert np.array_equal(got, np.flatnonzero(want_s[step]))
        assert np.array_equal(v[:N].cpu().numpy().astype(np.float64), want_v[step])
        assert np.array_equal(c[:N].cpu().numpy().astype(np.float64), want_c[step])
        assert int(inp.abs().sum().item()) == 0  # read, then cleared
    assert want_s.sum() > 0


def test_update_noalloc_allocates_nothing():
    import torch

    torch.cuda.set_device(0)
    gw, gh = 2, 2
    n = W.neuron_params()
    N = gw * gh * n["n_per_col"]
    dev = torch.device("cuda", 0)
    bufs = [torch.zeros(N, dtype=dt, device=dev)
            for dt in (torch.float32, torch.float32, torch.uint8, torch.int32, torch.int32)]
    stream = torch.cuda.current_stream()
    args = [b.data_ptr() for b in bufs]
    snn.snn_update_noalloc(gw, gh, n, 1, 0, *args, None, stream.cuda_stream)  # warm-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for step in range(1, 4):
        snn.snn_update_noalloc(gw, gh, n, 1, step, *args, None, stream.cuda_stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_update_noalloc_rejects_oversized_grid():
    with pytest.raises(snn.SnnError) as e:
        snn.snn_update_noalloc(129, 128, W.neuron_params(), 1, 0, 16, 16, 16, 16, 16)
    assert e.value.code == snn.SNN_EINVAL
    assert "16384" in snn.snn_last_error()
