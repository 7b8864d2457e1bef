"""GPU parity of the surrogate network (libzda tensor-core kernels) against
the FP64 oracle in oracle/surrogate.py, which rounds to bfloat16 at the same
points as the kernels.

Tolerances.  Both sides round every stored activation to bfloat16 (relative
step 2^-8); they differ only in the accumulation (FP32 in tensor memory vs
FP64), about 1e-7 relative before rounding.  A rounding decision therefore
flips on roughly 1e-4 of the elements of a layer, by one bfloat16 step, and
the flips feed the next layers.  On 16 x 16 images the cascade stays
negligible (an FP32-accumulating copy of the oracle differs from the FP64
one by ~4e-8 in the output), so the small case is held to 1e-3; on larger
images the cascade reaches ~4e-3 in the output and ~2e-2 in the weight
gradients (the same copy at 64 x 64), so larger cases are held to 2e-2 /
5e-2 / 1e-1 (output / weight gradients / input gradient).  A wrong tap, a
transposed operand, a lost bias or mask moves these by O(1).
"""
import numpy as np
import pytest
import torch

from oracle import surrogate as S

pytestmark = pytest.mark.gpu


def _net(H, W, ic, oc, B):
    from paper_2501_07979_gb300.surrogate import Surrogate
    return Surrogate(H, W, ic, oc, B, device=0)


def _params(ic, oc, seed):
    ps = S.init_params(ic, oc, seed=seed)
    r = np.random.default_rng(seed + 1)
    return [(w, r.standard_normal(b.shape) * 0.05) for w, b in ps]


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


CASES = {
    # name: (H, W, in_ch, out_ch, batch, forward tol, weight-grad tol, input-grad tol)
    "small": (16, 16, 2, 8, 2, 1e-3, 1e-2, 1e-2),
    "ragged": (24, 40, 1, 24, 3, 2e-2, 5e-2, 1e-1),
}


@pytest.mark.parametrize("name", list(CASES))
def test_forward_and_backward_match_oracle(name):
    H, W, ic, oc, B, tf, tg, tx = CASES[name]
    ps = _params(ic, oc, seed=11)
    r = np.random.default_rng(12)
    x = r.uniform(0, 1, (B, H, W, ic))
    t = r.standard_normal((B, H, W, oc))
    net = _net(H, W, ic, oc, B)
    net.set_params(S.flatten(ps).astype(np.float32))
    y = net.forward(torch.tensor(x, dtype=torch.float32, device="cuda:0"))
    loss, dy = net.mse(y, torch.tensor(t, dtype=torch.float32, device="cuda:0"))
    dx = net.backward(dy, want_dx=True)
    g = net.grads().cpu().numpy()
    net.check()

    y0, cache = S.forward(ps, x, rounding=True)
    assert _rel(y.cpu().numpy(), y0) < tf
    l0, dy0 = S.mse(y.cpu().numpy().astype(np.float64), t)         # the loss of the GPU's own output
    assert abs(float(loss.item()) - l0) <= 1e-6 * l0
    assert _rel(dy.cpu().numpy(), dy0) < 1e-6
    grads, dx0 = S.backward(ps, cache, dy.cpu().numpy().astype(np.float64), want_dx=True)
    off = 0
    for (lname, *_), (gw, gb) in zip(S.layer_table(ic, oc), grads):
        n = gw.size + gb.size
        gl = g[off:off + n]
        off += n
        assert _rel(gl[:gw.size], gw.ravel()) < tg, lname
        assert _rel(gl[gw.size:], gb) < tg, lname
    assert off == g.size
    assert _rel(dx.cpu().numpy(), dx0) < tx


def test_adam_step_matches_oracle():
    H, W, ic, oc, B = 16, 16, 1, 8, 2
    ps = _params(ic, oc, seed=21)
    r = np.random.default_rng(22)
    x = torch.tensor(r.uniform(0, 1, (B, H, W, ic)), dtype=torch.float32, device="cuda:0")
    t = torch.tensor(r.standard_normal((B, H, W, oc)), dtype=torch.float32, device="cuda:0")
    net = _net(H, W, ic, oc, B)
    p0 = S.flatten(ps).astype(np.float32)
    net.set_params(p0)
    m = np.zeros(p0.size)
    v = np.zeros(p0.size)
    p = p0.astype(np.float64)
    for step in (1, 2):
        y = net.forward(x)
        _, dy = net.mse(y, t)
        net.backward(dy)
        g = net.grads().cpu().numpy().astype(np.float64)
        p, m, v = S.adam(p, g, m, v, step, lr=1e-3)
        net.adam(1e-3)
        assert np.allclose(net.params().cpu().numpy(), p, rtol=1e-5, atol=1e-7)
    net.check()


def test_full_size_batch_forward_sampled_against_oracle():
    """128 x 128 patches, batch 256 (the inference batch): two sampled items
    against the oracle run on that item alone (samples are independent)."""
    H = W = 128
    ic, oc, B = 1, 24, 256
    ps = _params(ic, oc, seed=31)
    r = np.random.default_rng(32)
    x = r.uniform(0, 1, (B, H, W, ic)).astype(np.float32)
    net = _net(H, W, ic, oc, B)
    net.set_params(S.flatten(ps).astype(np.float32))
    y = net.forward(torch.tensor(x, device="cuda:0")).cpu().numpy()
    net.check()
    for i in (0, 173):
        y0, _ = S.forward(ps, x[i:i + 1].astype(np.float64), rounding=True)
        assert _rel(y[i:i + 1], y0) < 2e-2


def test_training_reduces_the_loss():
    H, W, ic, oc, B = 16, 16, 1, 8, 4
    r = np.random.default_rng(41)
    x = r.uniform(0, 1, (B, H, W, ic))
    # a smooth target: a fixed linear filter of the input
    t = np.concatenate([np.roll(x, s, axis=2) * (0.5 + 0.1 * s) for s in range(oc)], axis=3)
    net = _net(H, W, ic, oc, B)
    net.set_params(S.flatten(S.init_params(ic, oc, seed=42)).astype(np.float32))
    xt = torch.tensor(x, dtype=torch.float32, device="cuda:0")
    tt = torch.tensor(t, dtype=torch.float32, device="cuda:0")
    losses = [float(net.train_step(xt, tt, lr=2e-3).item()) for _ in range(60)]
    net.check()
    assert losses[-1] < 0.2 * losses[0]
    assert net.launches > 60 * 40
