"""Surrogate warm start of a zone's topology optimisation.

Pipeline (every numerical step runs in libzda kernels; this module moves
tensors between calls):

1. Data: random smoothed densities rho -> rho~ = projection(filter(rho))
   (zda_filter_project) -> FDTD forward run of the zone (a lens of identical
   zones per CUDA graph launch, zda_lens_forward) -> monitor-plane DFT over
   the design rows, the network target (divided by one global scale).
2. Training: the U-Net (include/zda_nn.h) on (rho~, target) pairs, MSE loss,
   Adam, tensor-core forward and backward kernels.
3. Warm start: Adam ascent of rho on the surrogate's focal intensity
   I_s(rho) = 2 sum_q |S_q|^2, S = focal transform of the predicted monitor
   DFT (zda_focal_transform_nn), gradient through the transposed focal
   transform, the network's backward pass and the transposed filter chain.
4. The FDTD (zda_iteration) then refines rho and checks the result; the
   surrogate's field error against the FDTD is reported on held-out samples.
"""
import ctypes
import time

import numpy as np

from . import _lib
from ._lib import check
from .lens import Lens
from .surrogate import Surrogate
from .topopt import Adam
from .zone import Zone


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class WarmStart:
    def __init__(self, spec, batch=64, device=0, lens_width=16, seed=0):
        import torch
        self.torch = torch
        self.spec = spec
        self.device = torch.device("cuda", device)
        self.zone = Zone(spec, device=device)
        self.Q = self.zone.n_freq
        self.H, self.W = self.zone.n_r_design, spec.n_phi
        self.i_d0 = spec.pml_r_in
        self.net = Surrogate(self.H, self.W, 1, 4 * self.Q, batch, device=device)
        self.lens_width = lens_width
        self.scale = None
        self._pools = {}
        self.seed = seed

    def set_target(self, spec):
        """Optimise another zone of the same design grid (the network is shared)."""
        assert spec.n_r - spec.pml_r_in - spec.pml_r_out == self.H and spec.n_phi == self.W
        self.spec = spec
        self.zone = Zone(spec, device=self.device.index)

    # ------------------------------------------------------------ data
    def _lens(self, spec=None):
        """A lens of lens_width identical zones (one graph launch runs them all)."""
        spec = spec or self.spec
        key = spec.to_json()
        if key not in self._pools:
            zones = [Zone(spec, device=self.device.index) for _ in range(self.lens_width)]
            self._pools[key] = (zones, Lens(zones, use_graph=True))
        return self._pools[key]

    def release_pools(self):
        self._pools = {}

    def _target(self, mon):
        torch = self.torch
        m = mon[:, :, self.i_d0:self.i_d0 + self.H, :]
        t = torch.stack([m.real, m.imag], dim=2)              # [Q][2][2][H][W]
        return t.reshape(4 * self.Q, self.H, self.W).permute(1, 2, 0)

    def generate(self, rhos, spec=None):
        """FDTD data for a list of densities: (X [n][H][W][1] = rho~, M [n][H][W][4Q]
        unscaled monitor DFT channels).  spec: another zone of the same design
        grid (e.g. at another radius) whose runs give the data; default the
        target zone."""
        torch = self.torch
        zones, lens = self._lens(spec)
        X, M = [], []
        for k in range(0, len(rhos), len(zones)):
            chunk = list(rhos[k:k + len(zones)])
            pad = len(zones) - len(chunk)
            batch = [torch.as_tensor(r, dtype=torch.float32, device=self.device) for r in chunk]
            batch += [batch[-1]] * pad
            lens.forward(batch)
            for z, r in zip(zones[:len(chunk)], batch[:len(chunk)]):
                X.append(z.filter_project(r))
                M.append(self._target(z.monitor_dft()))
        return torch.stack(X)[..., None].contiguous(), torch.stack(M).contiguous()

    # ------------------------------------------------------------ training
    def init_params(self, seed):
        self.net.init_params(seed)

    def fit(self, X, M, steps=400, batch=None, lr=2e-3, seed=0):
        """Train on (X, M); the target scale is the RMS of M.  Returns the loss history."""
        torch = self.torch
        if self.scale is None:
            self.scale = float(torch.sqrt(torch.mean(M * M)).item())
        Y = M / self.scale
        n = X.shape[0]
        b = min(batch or self.net.batch, self.net.batch, n)
        g = torch.Generator(device="cpu").manual_seed(seed)
        hist = []
        for s in range(steps):
            idx = torch.randperm(n, generator=g)[:b].to(self.device)
            loss = self.net.train_step(X[idx], Y[idx], lr=lr)
            if s % 20 == 0 or s == steps - 1:
                hist.append(float(loss.item()))
        self.net.check()
        return hist

    def field_error(self, X, M):
        """Relative L2 error of the surrogate's monitor DFT against the FDTD's."""
        torch = self.torch
        errs = []
        for k in range(0, X.shape[0], self.net.batch):
            y = self.net.forward(X[k:k + self.net.batch]) * self.scale
            ref = M[k:k + self.net.batch]
            errs.append((torch.linalg.vector_norm(y - ref) / torch.linalg.vector_norm(ref)).item())
        return float(np.mean(errs))

    # ------------------------------------------------------------ surrogate objective
    def surrogate_value_and_grad(self, rho):
        """(I_s, dI_s/drho) of the surrogate's focal intensity for one density."""
        torch = self.torch
        L = _lib.lib()
        r = torch.as_tensor(rho, dtype=torch.float32, device=self.device).contiguous()
        rt = self.zone.filter_project(r)
        y = self.net.forward(rt[None, :, :, None].contiguous())
        S = torch.empty((1, self.Q, 2), dtype=torch.float64, device=self.device)
        stream = ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
        check(L.zda_focal_transform_nn(self.zone.handle, _ptr(y), 1, float(self.scale), _ptr(S), stream))
        Sc = S[..., 0] + 1j * S[..., 1]
        I = 2.0 * float((Sc.abs() ** 2).sum().item())
        G = torch.stack([4.0 * Sc.real, 4.0 * Sc.imag], dim=-1).contiguous()      # dI/dRe S + i dI/dIm S
        dy = torch.empty_like(y)
        check(L.zda_focal_transform_nn_transpose(self.zone.handle, _ptr(G), 1, float(self.scale), _ptr(dy), stream))
        drt = self.net.backward(dy, want_dx=True)[0, :, :, 0].contiguous()
        return I, self.zone.filter_project_backward(r, drt)

    def optimize_surrogate(self, rho0, steps=200, lr=0.02):
        opt = Adam([rho0.shape], lr=lr)
        rho = [np.asarray(rho0, dtype=np.float64)]
        hist = []
        for _ in range(steps):
            I, g = self.surrogate_value_and_grad(rho[0])
            hist.append(I)
            rho = opt.step(rho, [g.cpu().numpy()])
        return rho[0], hist

    def fdtd_topopt(self, rho0, iters, lr=0.02):
        """Plain adjoint-FDTD ascent from rho0; returns (rho, [I per iteration], seconds)."""
        opt = Adam([rho0.shape], lr=lr)
        rho = [np.asarray(rho0, dtype=np.float64)]
        hist = []
        t0 = time.perf_counter()
        for _ in range(iters):
            I, g = self.zone.iteration(self.torch.as_tensor(rho[0], dtype=self.torch.float32, device=self.device))
            hist.append(float(I))
            rho = opt.step(rho, [g.cpu().numpy()])
        return rho[0], hist, time.perf_counter() - t0
