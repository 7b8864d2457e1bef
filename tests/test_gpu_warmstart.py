"""The learned warm start, end to end on the GPU (the network's gain over the
method without it): FDTD-generated data, training by the library's own
kernels, surrogate-driven ascent, then adjoint-FDTD refinement compared
with the cold start.  Also parity of the focal transform on the surrogate's
output layout (and its transpose) against the oracle's focal weights."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import surrogate as S
from zda_inputs import smoothed_rho, zone_tiny

pytestmark = pytest.mark.gpu

SPEC = zone_tiny(n_phi=16, n_fold=20, eps_hi=4.0, n_steps=800, filter_radius=0.2, beta=4.0)


def test_focal_transform_on_surrogate_layout_matches_oracle():
    import ctypes
    from paper_2501_07979_gb300 import _lib
    from paper_2501_07979_gb300.zone import Zone
    spec = SPEC.replace(wavelengths=(0.9, 1.1))
    g = O.Geometry(spec)
    z = Zone(spec, device=0)
    Q = z.n_freq
    r = np.random.default_rng(3)
    mon = r.standard_normal((Q, 2, spec.n_r, spec.n_phi)) + 1j * r.standard_normal((Q, 2, spec.n_r, spec.n_phi))
    scale = 0.37
    y = np.stack([S.target_from_monitor(mon, g.i_d0, g.i_d1, scale), S.target_from_monitor(2 * mon, g.i_d0, g.i_d1, scale)])
    yt = torch.tensor(np.ascontiguousarray(y), dtype=torch.float32, device="cuda:0").contiguous()
    Sd = torch.empty((2, Q, 2), dtype=torch.float64, device="cuda:0")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _lib.check(_lib.lib().zda_focal_transform_nn(z.handle, ctypes.c_void_p(yt.data_ptr()), 2, scale,
                                                 ctypes.c_void_p(Sd.data_ptr()), st))
    Sg = Sd[..., 0].cpu().numpy() + 1j * Sd[..., 1].cpu().numpy()
    wr, wp, _ = O.focal_weights(spec, g)
    rows = slice(g.i_d0, g.i_d1)
    m32 = S.monitor_from_output(y[0].astype(np.float32), Q, scale)          # what the kernel reads
    ref = np.einsum("qij,qij->q", wr[:, rows], m32[:, 0]) + np.einsum("qij,qij->q", wp[:, rows], m32[:, 1])
    assert np.allclose(Sg[0], ref, rtol=1e-6, atol=1e-12)
    assert np.allclose(Sg[1], 2 * ref, rtol=1e-6, atol=1e-12)
    # transpose: dobj/dy for G = dobj/dRe S + i dobj/dIm S
    G = r.standard_normal((2, Q)) + 1j * r.standard_normal((2, Q))
    Gd = torch.tensor(np.stack([G.real, G.imag], -1), dtype=torch.float64, device="cuda:0").contiguous()
    dy = torch.empty(tuple(yt.shape), dtype=torch.float32, device="cuda:0")
    _lib.check(_lib.lib().zda_focal_transform_nn_transpose(z.handle, ctypes.c_void_p(Gd.data_ptr()), 2, scale,
                                                   ctypes.c_void_p(dy.data_ptr()), st))
    dy = dy.cpu().numpy()
    for b in range(2):
        for q in range(Q):
            for comp, w in ((0, wr[q, rows]), (1, wp[q, rows])):
                ch = (q * 2 + comp) * 2
                assert np.allclose(dy[b, :, :, ch], scale * np.real(np.conj(G[b, q]) * w), rtol=1e-5, atol=1e-9)
                assert np.allclose(dy[b, :, :, ch + 1], scale * np.imag(G[b, q] * np.conj(w)), rtol=1e-5, atol=1e-9)
    # and the two are adjoint: <T(G), dy'> = Re sum conj(G) S(dy')
    assert np.isclose(np.sum(dy[0] * y[0]), np.real(np.sum(np.conj(G[0]) * Sg[0])), rtol=1e-5)


def test_surrogate_warm_start_beats_cold_start():
    from paper_2501_07979_gb300.warmstart import WarmStart
    ws = WarmStart(SPEC, batch=64, lens_width=16)
    rhos = [smoothed_rho(ws.H, ws.W, 1000 + i, sigma=1.0 + (i % 3), mode="minmax") for i in range(640)]
    X, M = ws.generate(rhos)
    ws.init_params(0)
    hist = ws.fit(X[64:], M[64:], steps=800, lr=2e-3)
    assert hist[-1] < 0.05 * hist[0]
    err = ws.field_error(X[:64], M[:64])                 # held-out samples, against the FDTD
    assert err < 0.2, err
    rho0 = np.full((ws.H, ws.W), 0.5)
    I0, _ = ws.zone.iteration(torch.tensor(rho0, dtype=torch.float32, device="cuda:0"))
    rw, hs = ws.optimize_surrogate(rho0, steps=60, lr=0.02)
    Iw, _ = ws.zone.iteration(torch.tensor(rw, dtype=torch.float32, device="cuda:0"))
    assert hs[-1] > 3 * hs[0]
    assert Iw > 3 * I0, (I0, Iw)                          # the FDTD confirms the surrogate's design
    _, cold, _ = ws.fdtd_topopt(rho0, 30)
    _, warm, _ = ws.fdtd_topopt(rw, 5)
    # 5 warm-started FDTD iterations reach what 30 cold ones reach
    assert max(warm) >= 0.99 * max(cold), (max(warm), max(cold))
