"""ORACLE -- test infrastructure, not the product: the learned surrogate.

A plain FP64 NumPy statement of the zone surrogate: a 4-level convolutional
U-Net (Ronneberger, Fischer and Brox, MICCAI 2015) that maps a zone's
density patch rho (the design layer, n_r x n_phi pixels) to the zone's
monitor-plane DFT over the design annulus (the near field that the focal
transform of "Results and Discussion" integrates), its mean-squared-error
training loss, the hand-written backward pass, and the Adam update (Kingma
and Ba, ICLR 2015, Algorithm 1).  The paper itself has no learned component;
the network is the warm start of each zone's topology optimisation.

Architecture (H, W multiples of 8, width C = 64):

    level l = 0, 1, 2:  e_la = relu(conv3(in_l)),  e_lb = relu(conv3(e_la)),
                        in_{l+1} = avgpool2(e_lb)          (in_0 = x)
    bottleneck:         b_a = relu(conv3(in_3)),  b_b = relu(conv3(b_a))
    level l = 2, 1, 0:  d_la = relu(conv3(concat(up2(d_{l+1}), e_lb))),
                        d_lb = relu(conv3(d_la))            (d_3 = b_b)
    head:               y = conv1(d_0b)   (no activation)

conv3 is a 3x3 cross-correlation with zero padding ("same" size) plus bias;
avgpool2 the mean of each 2 x 2 block; up2 nearest-neighbour doubling.

Precision model (the CUDA path's; the oracle applies the same rounding
points so that both sides take every rounding decision on the same value up
to the accumulation order): weights, the input and every stored activation
and activation gradient are bfloat16; convolutions accumulate their bf16
products in FP32 on the GPU, FP64 here; biases, the head output, the loss,
weight/bias gradients and the optimiser state are FP32 (FP64 here).
With rounding=False every function is exact FP64 arithmetic (used by the
finite-difference pins).

Only tests/, the smoke check and the benchmark's CPU-baseline leg may import
this module; it shares no code with the CUDA library.
"""
from __future__ import annotations

import numpy as np

WIDTH = 64
LEVELS = 3          # pooled levels below the input level (4 resolution levels)

# layer table: (name, kind, input channels (symbolic), output channels)
#   'in' = input channels, 'C' = width, '2C' = concat width, 'out' = outputs


def layer_table(in_ch, out_ch, width=WIDTH):
    """Names and shapes of the 15 parameterised layers, in parameter order."""
    C = width
    t = []
    for l in range(LEVELS):
        t.append(("enc%da" % l, 3, in_ch if l == 0 else C, C))
        t.append(("enc%db" % l, 3, C, C))
    t.append(("bota", 3, C, C))
    t.append(("botb", 3, C, C))
    for l in reversed(range(LEVELS)):
        t.append(("dec%da" % l, 3, 2 * C, C))
        t.append(("dec%db" % l, 3, C, C))
    t.append(("head", 1, C, out_ch))
    return t


def param_count(in_ch, out_ch, width=WIDTH):
    return sum(k * k * ci * co + co for _, k, ci, co in layer_table(in_ch, out_ch, width))


def forward_flops(H, W, in_ch, out_ch, width=WIDTH):
    """Multiply-add FLOPs (2 per MAC) of one sample's forward pass, counted on
    the H x W output pixels of every convolution."""
    f = 0
    for name, k, ci, co in layer_table(in_ch, out_ch, width):
        lev = int(name[3]) if name[3].isdigit() else LEVELS
        if name == "head":
            lev = 0
        f += 2 * (H >> lev) * (W >> lev) * k * k * ci * co
    return f


# --------------------------------------------------------------------------
# rounding
# --------------------------------------------------------------------------
def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64.

    bfloat16 keeps the top 16 bits of an IEEE binary32; rounding first to
    binary32 is exact for every value this module rounds (they are binary32
    results on the GPU side too)."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) >> 16
    out = (u.astype(np.uint32) << 16).view(np.float32)
    nan = np.isnan(a)
    if nan.any():
        out = np.where(nan, np.float32(np.nan), out)
    return out.astype(np.float64)


def _r(x, rounding):
    return bf16(x) if rounding else np.asarray(x, dtype=np.float64)


# --------------------------------------------------------------------------
# layers (NHWC arrays: [batch][H][W][channels])
# --------------------------------------------------------------------------
def conv(x, w, b=None):
    """Cross-correlation with zero padding ('same' output size):
    y[n,i,j,o] = b[o] + sum_{dy,dx,c} w[o,dy,dx,c] x[n, i+dy-k//2, j+dx-k//2, c]."""
    k = w.shape[1]
    p = k // 2
    n, H, W_, _ = x.shape
    xp = np.pad(x, ((0, 0), (p, p), (p, p), (0, 0)))
    y = np.zeros((n, H, W_, w.shape[0]))
    for dy in range(k):
        for dx in range(k):
            y += xp[:, dy:dy + H, dx:dx + W_, :] @ w[:, dy, dx, :].T
    if b is not None:
        y += b
    return y


def conv_dgrad(g, w):
    """Transpose of conv with respect to its input: dx[n,i,j,c] =
    sum_{dy,dx,o} w[o,dy,dx,c] g[n, i-dy+k//2, j-dx+k//2, o]."""
    k = w.shape[1]
    p = k // 2
    n, H, W_, _ = g.shape
    gp = np.pad(g, ((0, 0), (p, p), (p, p), (0, 0)))
    dx_ = np.zeros((n, H, W_, w.shape[3]))
    for dy in range(k):
        for dx in range(k):
            dx_ += gp[:, 2 * p - dy:2 * p - dy + H, 2 * p - dx:2 * p - dx + W_, :] @ w[:, dy, dx, :]
    return dx_


def conv_wgrad(x, g, k):
    """Gradient of sum(g * conv(x, w)) with respect to w:
    dw[o,dy,dx,c] = sum_{n,i,j} g[n,i,j,o] x[n, i+dy-k//2, j+dx-k//2, c]."""
    p = k // 2
    n, H, W_, ci = x.shape
    co = g.shape[3]
    xp = np.pad(x, ((0, 0), (p, p), (p, p), (0, 0)))
    dw = np.zeros((co, k, k, ci))
    g2 = g.reshape(-1, co)
    for dy in range(k):
        for dx in range(k):
            dw[:, dy, dx, :] = g2.T @ xp[:, dy:dy + H, dx:dx + W_, :].reshape(-1, ci)
    return dw


def relu(x):
    return np.maximum(x, 0.0)


def avgpool2(x):
    n, H, W_, c = x.shape
    return x.reshape(n, H // 2, 2, W_ // 2, 2, c).mean(axis=(2, 4))


def avgpool2_T(g):
    """Transpose of avgpool2: every fine pixel receives a quarter of its block's value."""
    return 0.25 * np.repeat(np.repeat(g, 2, axis=1), 2, axis=2)


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_T(g):
    """Transpose of up2: the sum over each 2 x 2 block."""
    n, H, W_, c = g.shape
    return g.reshape(n, H // 2, 2, W_ // 2, 2, c).sum(axis=(2, 4))


# --------------------------------------------------------------------------
# parameters
# --------------------------------------------------------------------------
def init_params(in_ch, out_ch, seed, width=WIDTH):
    """He-normal weights (std sqrt(2 / fan_in)), zero biases; the head is
    scaled by 0.1 so that the untrained output starts small.  Layout per
    layer: w [c_out][k][k][c_in], b [c_out]."""
    rng = np.random.default_rng(seed)
    ps = []
    for name, k, ci, co in layer_table(in_ch, out_ch, width):
        std = np.sqrt(2.0 / (k * k * ci)) * (0.1 if name == "head" else 1.0)
        ps.append((rng.standard_normal((co, k, k, ci)) * std, np.zeros(co)))
    return ps


def flatten(params):
    """Flat FP64 vector in layer order: each layer's w (row-major) then b."""
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in params])


def unflatten(vec, in_ch, out_ch, width=WIDTH):
    ps, o = [], 0
    for _, k, ci, co in layer_table(in_ch, out_ch, width):
        nw = co * k * k * ci
        ps.append((np.asarray(vec[o:o + nw], dtype=np.float64).reshape(co, k, k, ci),
                   np.asarray(vec[o + nw:o + nw + co], dtype=np.float64)))
        o += nw + co
    return ps


# --------------------------------------------------------------------------
# network
# --------------------------------------------------------------------------
def forward(params, x, rounding=True):
    """U-Net forward pass. x: [n][H][W][in_ch].  Returns (y, cache) with y
    [n][H][W][out_ch] and cache the stored activations of the backward pass."""
    P = {name: (_r(w, rounding), b) for (name, *_), (w, b) in
         zip(layer_table(x.shape[3], params[-1][0].shape[0], params[0][0].shape[0]), params)}
    a = {"x": _r(x, rounding)}

    def cr(name, inp):
        w, b = P[name]
        return _r(relu(conv(inp, w, b)), rounding)

    inp = a["x"]
    for l in range(LEVELS):
        a["enc%da" % l] = cr("enc%da" % l, inp)
        a["enc%db" % l] = cr("enc%db" % l, a["enc%da" % l])
        inp = a["in%d" % (l + 1)] = _r(avgpool2(a["enc%db" % l]), rounding)
    a["bota"] = cr("bota", inp)
    a["botb"] = cr("botb", a["bota"])
    d = a["botb"]
    for l in reversed(range(LEVELS)):
        a["cat%d" % l] = np.concatenate([up2(d), a["enc%db" % l]], axis=3)
        a["dec%da" % l] = cr("dec%da" % l, a["cat%d" % l])
        d = a["dec%db" % l] = cr("dec%db" % l, a["dec%da" % l])
    w, b = P["head"]
    y = conv(d, w, b)
    a["P"] = P
    a["rounding"] = rounding
    return y, a


def backward(params, cache, dy, want_dx=False):
    """Backward pass of forward(): dy = dL/dy [n][H][W][out_ch] ->
    (grads, dx) with grads a list of (dw, db) in parameter order and dx the
    input gradient (None unless want_dx)."""
    a = cache
    P = a["P"]
    rd = a["rounding"]
    names = list(P.keys())
    G = {}

    def mask(t):
        return (t > 0).astype(np.float64)

    def layer_bwd(name, inp, g):
        """g: gradient w.r.t. this conv's pre-activation output (already masked)."""
        w, _ = P[name]
        G[name] = (conv_wgrad(inp, g, w.shape[1]), g.sum(axis=(0, 1, 2)))
        return conv_dgrad(g, w)

    g = _r(dy, rd)
    g = _r(mask(a["dec0b"]) * layer_bwd("head", a["dec0b"], g), rd)
    skip_part = {}
    for l in range(LEVELS):
        g = _r(mask(a["dec%da" % l]) * layer_bwd("dec%db" % l, a["dec%da" % l], g), rd)
        gc = layer_bwd("dec%da" % l, a["cat%d" % l], g)
        C = gc.shape[3] // 2
        gu = _r(gc[..., :C], rd)
        skip_part[l] = _r(gc[..., C:], rd)
        below = a["botb"] if l == LEVELS - 1 else a["dec%db" % (l + 1)]
        g = _r(mask(below) * up2_T(gu), rd)
    g = _r(mask(a["bota"]) * layer_bwd("botb", a["bota"], g), rd)
    g_in = _r(layer_bwd("bota", a["in%d" % LEVELS], g), rd)
    dx = None
    for l in reversed(range(LEVELS)):
        g = _r(mask(a["enc%db" % l]) * (skip_part[l] + avgpool2_T(g_in)), rd)
        g = _r(mask(a["enc%da" % l]) * layer_bwd("enc%db" % l, a["enc%da" % l], g), rd)
        inp = a["x"] if l == 0 else a["in%d" % l]
        gi = layer_bwd("enc%da" % l, inp, g)
        if l > 0:
            g_in = _r(gi, rd)
        elif want_dx:
            dx = gi
    return [G[n] for n in names], dx


def mse(y, t):
    """Mean squared error over all elements and its gradient with respect to y."""
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size


def adam(params, grads, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, Algorithm 1) on flat vectors: returns
    (params', m', v') with bias-corrected moments; step counts from 1."""
    m = b1 * m + (1 - b1) * grads
    v = b2 * v + (1 - b2) * grads * grads
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


# --------------------------------------------------------------------------
# zone data <-> network tensors
# --------------------------------------------------------------------------
def target_from_monitor(mon, i_d0, i_d1, scale):
    """Monitor DFT [Q][2][n_r][n_phi] (complex) -> network target
    [n_rd][n_phi][4Q] over the design columns: channel ((q*2 + comp)*2 + part)
    with part 0 = real, 1 = imaginary, divided by `scale`."""
    m = np.asarray(mon)[:, :, i_d0:i_d1, :] / scale
    Q = m.shape[0]
    t = np.stack([m.real, m.imag], axis=2)           # [Q][2][2][nr][nphi]
    return t.reshape(Q * 4, m.shape[2], m.shape[3]).transpose(1, 2, 0)


def monitor_from_output(y, Q, scale):
    """Inverse of target_from_monitor for one sample: [n_rd][n_phi][4Q] ->
    complex [Q][2][n_rd][n_phi] times `scale`."""
    t = np.asarray(y).transpose(2, 0, 1).reshape(Q, 2, 2, y.shape[0], y.shape[1])
    return (t[:, :, 0] + 1j * t[:, :, 1]) * scale
