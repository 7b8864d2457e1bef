"""Pins of the surrogate oracle (oracle/surrogate.py) against definitions
that do not come from its own code: library convolution and rounding
routines, adjoint identities, finite differences, closed forms of the U-Net
with hand-set weights, and Adam's textbook first step."""
import numpy as np
import pytest

from oracle import surrogate as S


def _rng(seed=0):
    return np.random.default_rng(seed)


def test_bf16_matches_torch_rounding_including_ties():
    torch = pytest.importorskip("torch")
    r = _rng(1)
    x = np.concatenate([r.standard_normal(5000) * 10 ** r.uniform(-6, 6, 5000),
                        [0.0, -0.0, 1.0, 65504.0, 1e-38, 3.0e38]]).astype(np.float32)
    # exact ties: lower 16 bits = 0x8000, with even and odd kept parts
    base = r.integers(0x3F800000, 0x40800000, 256, dtype=np.uint32) & 0xFFFF0000
    ties = (base | 0x8000).view(np.float32)
    x = np.concatenate([x, ties, -ties])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(S.bf16(x), ref)


def test_conv_matches_scipy_correlate2d():
    signal = pytest.importorskip("scipy.signal")
    r = _rng(2)
    x = r.standard_normal((2, 7, 9, 3))
    for k in (1, 3):
        w = r.standard_normal((4, k, k, 3))
        b = r.standard_normal(4)
        y = S.conv(x, w, b)
        for n in range(2):
            for o in range(4):
                ref = b[o] + sum(signal.correlate2d(x[n, :, :, c], w[o, :, :, c], mode="same",
                                                    boundary="fill") for c in range(3))
                assert np.allclose(y[n, :, :, o], ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("k", [1, 3])
def test_conv_transposes_satisfy_adjoint_identities(k):
    r = _rng(3)
    x = r.standard_normal((2, 8, 6, 5))
    w = r.standard_normal((3, k, k, 5))
    g = r.standard_normal((2, 8, 6, 3))
    lhs = np.sum(S.conv(x, w) * g)
    assert np.isclose(lhs, np.sum(x * S.conv_dgrad(g, w)), rtol=1e-12)
    assert np.isclose(lhs, np.sum(w * S.conv_wgrad(x, g, k)), rtol=1e-12)


def test_pool_and_upsample_values_and_transposes():
    x = np.arange(16, dtype=float).reshape(1, 4, 4, 1)
    assert np.array_equal(S.avgpool2(x)[0, :, :, 0], [[2.5, 4.5], [10.5, 12.5]])
    assert np.array_equal(S.up2(np.array([[[[1.0], [2.0]]]]))[0, :, :, 0], [[1, 1, 2, 2], [1, 1, 2, 2]])
    r = _rng(4)
    f = r.standard_normal((2, 8, 4, 3))
    c = r.standard_normal((2, 4, 2, 3))
    assert np.isclose(np.sum(S.avgpool2(f) * c), np.sum(f * S.avgpool2_T(c)), rtol=1e-12)
    assert np.isclose(np.sum(S.up2(c) * f), np.sum(c * S.up2_T(f)), rtol=1e-12)


def _identity_net(in_ch, width, take_skip):
    """Weights that make every conv the identity on the first channels (centre
    tap), with the decoder's first conv taking either the skip half or the
    upsampled half of its concatenated input."""
    ps = []
    for name, k, ci, co in S.layer_table(in_ch, in_ch, width):
        w = np.zeros((co, k, k, ci))
        c = k // 2
        off = 0
        if name.startswith("dec") and name.endswith("a"):
            off = width if take_skip else 0
        for o in range(min(co, in_ch)):
            w[o, c, c, off + o] = 1.0
        ps.append((w, np.zeros(co)))
    return ps


def test_unet_wiring_closed_forms():
    """With identity convolutions the U-Net reduces to closed forms: taking
    the skip path at every decoder level returns the input; taking the
    upsampled path returns the 8 x 8 block means (three poolings, three
    nearest upsamplings)."""
    r = _rng(5)
    x = r.uniform(0, 1, (2, 16, 24, 2))
    y, _ = S.forward(_identity_net(2, 8, True), x, rounding=False)
    assert np.allclose(y, x, atol=1e-14)
    y, _ = S.forward(_identity_net(2, 8, False), x, rounding=False)
    blocks = x.reshape(2, 2, 8, 3, 8, 2).mean(axis=(2, 4))
    ref = np.repeat(np.repeat(blocks, 8, axis=1), 8, axis=2)
    assert np.allclose(y, ref, atol=1e-14)


def test_unet_backward_matches_central_differences():
    """Directional derivatives of L = sum(r * y) in FP64 (no rounding) against
    central differences, for the weights and for the input."""
    r = _rng(6)
    in_ch, out_ch, width = 2, 3, 4
    ps = S.init_params(in_ch, out_ch, seed=7, width=width)
    ps = [(w, r.standard_normal(b.shape) * 0.1) for w, b in ps]
    x = r.uniform(0, 1, (1, 16, 16, in_ch))
    rr = r.standard_normal((1, 16, 16, out_ch))
    y, cache = S.forward(ps, x, rounding=False)
    grads, dx = S.backward(ps, cache, rr, want_dx=True)
    vec = S.flatten(ps)
    gvec = S.flatten(grads)
    d = r.standard_normal(vec.size)
    h = 1e-6

    def L(v, xx):
        return float(np.sum(rr * S.forward(S.unflatten(v, in_ch, out_ch, width), xx, rounding=False)[0]))

    fd = (L(vec + h * d, x) - L(vec - h * d, x)) / (2 * h)
    assert np.isclose(fd, gvec @ d, rtol=1e-6)
    dxx = r.standard_normal(x.shape)
    fd = (L(vec, x + h * dxx) - L(vec, x - h * dxx)) / (2 * h)
    assert np.isclose(fd, np.sum(dx * dxx), rtol=1e-6)
    # per-layer: the bias gradient of every layer (each is one directional test)
    o = 0
    for (w, b), (gw, gb) in zip(ps, grads):
        o += w.size
        e = np.zeros(vec.size)
        e[o] = 1.0
        fd = (L(vec + h * e, x) - L(vec - h * e, x)) / (2 * h)
        assert np.isclose(fd, gb[0], rtol=1e-5, atol=1e-9)
        o += b.size


def test_adam_first_steps_are_sign_steps():
    """Bias correction makes Adam's step -lr * g / (|g| + eps) while the
    gradient is constant (m_hat = g, v_hat = g^2)."""
    r = _rng(8)
    g = r.standard_normal(100)
    p = r.standard_normal(100)
    m = np.zeros(100)
    v = np.zeros(100)
    p0 = p.copy()
    for t in range(1, 4):
        p, m, v = S.adam(p, g, m, v, t, lr=0.01, eps=1e-8)
        assert np.allclose(p, p0 - 0.01 * t * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-12)


def test_rounded_forward_is_close_to_exact_forward():
    """bf16 storage perturbs the output by a few bf16 epsilons (2^-8), not more."""
    r = _rng(9)
    ps = S.init_params(2, 8, seed=10, width=16)
    x = r.uniform(0, 1, (1, 32, 32, 2))
    y0, _ = S.forward(ps, x, rounding=False)
    y1, _ = S.forward(ps, x, rounding=True)
    rel = np.linalg.norm(y1 - y0) / np.linalg.norm(y0)
    assert 1e-4 < rel < 3e-2


def test_monitor_target_round_trip_and_layer_count():
    r = _rng(11)
    mon = r.standard_normal((6, 2, 20, 8)) + 1j * r.standard_normal((6, 2, 20, 8))
    t = S.target_from_monitor(mon, 3, 15, 2.0)
    assert t.shape == (12, 8, 24)
    assert t[4, 5, ((3 * 2 + 1) * 2 + 1)] == mon[3, 1, 7, 5].imag / 2.0
    assert np.allclose(S.monitor_from_output(t, 6, 2.0), mon[:, :, 3:15, :])
    tab = S.layer_table(16, 24)
    assert len(tab) == 15 and sum(1 for t_ in tab if t_[1] == 3) == 14
    # forward FLOPs of the 128 x 128, 64-channel network (16 input, 24 output channels)
    f = S.forward_flops(128, 128, 16, 24)
    assert abs(f - 7.08e9) / 7.08e9 < 0.01
