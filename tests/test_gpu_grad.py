"""The differentiable form on the GPU (snn_grad_*) against the FP64 oracle of
oracle/surrogate.py, which tests/test_oracle_surrogate.py pins.

Hard spikes: the device recursion is the oracle's exact-FP32 one, so both fire
the same spikes and the losses (functions of the spike counts) are equal; the
surrogate gradients then differ only by the FP32 (device) vs FP64 (oracle)
arithmetic of the adjoint recursion.  Soft spikes: the sigmoid is evaluated
with different exponential functions, so loss and gradient agree to a
tolerance over a short horizon (the exact gradient of this chaotic recursion
grows by orders of magnitude within tens of steps).
"""
import numpy as np
import pytest

import oracle
from oracle import surrogate as S
from paper_1511_09325_gb300 import build as B
from paper_1511_09325_gb300 import snn
from paper_1511_09325_gb300 import workloads as W

pytestmark = pytest.mark.gpu

THETA = np.array([1.0, 1.0, 1.0, 1.0, 0.02, 2.5])


@pytest.fixture(scope="module", autouse=True)
def lib():
    B.build()
    snn.load()


def _run(gw, gh, seed, T, ckpt=50, hard=True, theta=THETA):
    n, s = W.neuron_params(), W.synapse_params()
    with snn.Net(gw, gh, n, s, seed, "f32w") as net:
        with snn.Grad(net, T, checkpoint_every=ckpt, hard=hard) as g:
            return g.loss_and_grad(theta)


def _oracle(gw, gh, seed, T, hard=True, theta=THETA):
    p = oracle.make_params(gw, gh, W.neuron_params(), W.synapse_params(), seed)
    net = S.SoftNet(p)
    loss, st = net.forward32(theta, T) if hard else net.forward(theta, T)
    return loss, st["rates"], net.backward(st)


def _close(g, go, rtol):
    scale = np.abs(go).max()
    assert np.all(np.abs(g - go) <= rtol * np.maximum(np.abs(go), 1e-2 * scale)), (g, go)


def test_hard_mode_2x2_matches_oracle():
    """2x2 columns, 120 steps, checkpoints every 50 (a partial last segment)."""
    loss, rates, g = _run(2, 2, 5, 120)
    lo, ro, go = _oracle(2, 2, 5, 120)
    assert rates[0] > 1.0 and np.array_equal(rates, np.array(ro))
    assert loss == lo
    _close(g, go, 2e-3)


def test_soft_mode_2x2_matches_oracle():
    """8 steps: FP32 rounding grows through the relaxed recursion (its exact
    gradient grows ~10x every few steps), so 1e-4 on the loss, 5e-3 on the
    gradient."""
    loss, rates, g = _run(2, 2, 5, 8, hard=False)
    lo, ro, go = _oracle(2, 2, 5, 8, hard=False)
    assert abs(loss - lo) <= 1e-4 * lo
    assert np.allclose(rates, ro, rtol=1e-4)
    _close(g, go, 5e-3)


def test_checkpoint_interval_and_repeats_do_not_change_results():
    """Recomputation from checkpoints is exact: any interval, any repeat, the
    same bits (every reduction has a fixed order)."""
    a = _run(2, 2, 9, 80, ckpt=7)
    b = _run(2, 2, 9, 80, ckpt=80)
    c = _run(2, 2, 9, 80, ckpt=7)
    for x, y in ((a, b), (a, c)):
        assert x[0] == y[0] and np.array_equal(x[1], y[1]) and np.array_equal(x[2], y[2])


def test_cols4x4_500_steps_matches_oracle():
    """The 4x4 workload (19 840 neurons, 24.6 M synapses), 500 steps,
    checkpoints every 50: same spikes, so the same loss; gradient to 5e-3."""
    loss, rates, g = _run(4, 4, 11, 500)
    lo, ro, go = _oracle(4, 4, 11, 500)
    assert loss == lo and np.array_equal(rates, np.array(ro))
    _close(g, go, 5e-3)


def test_torch_function_and_parameter_changes():
    """rate_loss as a torch function: backward returns the library gradient;
    a different theta changes the loss; the forward-only call agrees."""
    torch = pytest.importorskip("torch")
    n, s = W.neuron_params(), W.synapse_params()
    with snn.Net(2, 2, n, s, 5, "f32w") as net, snn.Grad(net, 60) as g:
        th = torch.tensor(THETA, dtype=torch.float64, requires_grad=True)
        L = snn.rate_loss(g, th)
        L.backward()
        loss, rates, grad = g.loss_and_grad(THETA)
        assert float(L.detach()) == loss and np.array_equal(th.grad.numpy(), grad)
        assert g.loss(THETA)[0] == loss
        th2 = THETA.copy()
        th2[0] = 0.5
        assert g.loss(th2)[0] != loss


def test_invalid_arguments():
    n, s = W.neuron_params(), W.synapse_params()
    with snn.Net(1, 1, n, s, 1, "f16w") as net:
        with pytest.raises(snn.SnnError) as e:
            snn.Grad(net, 10)
        assert e.value.code == snn.SNN_EINVAL
    with snn.Net(1, 1, n, s, 1, "f32w") as net:
        for bad in ((0, 5), (10, 0)):
            with pytest.raises(snn.SnnError):
                snn.Grad(net, bad[0], checkpoint_every=bad[1])
        with snn.Grad(net, 10) as g:
            th = THETA.copy()
            th[5] = 0.0
            with pytest.raises(snn.SnnError) as e:
                g.loss(th)
            assert e.value.code == snn.SNN_EINVAL
            th[5] = np.nan
            with pytest.raises(snn.SnnError):
                g.loss(th)
            assert np.isfinite(g.loss(THETA)[0])
