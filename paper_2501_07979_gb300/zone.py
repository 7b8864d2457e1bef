"""Python binding of one ZDA zone (argument marshalling over the C ABI).

PyTorch provides device memory (the workspace and the density / gradient
tensors) and the stream; every step of the solve runs in libzda's kernels.
"""
import ctypes
import math

import numpy as np
import torch

from . import _lib
from ._lib import check


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def make_desc(spec):
    """Pack a zone description (any object with the ZoneSpec attributes)."""
    d = _lib.ZoneDesc()
    d.r_lo, d.dr, d.dz = float(spec.r_lo), float(spec.dr), float(spec.dz)
    d.n_r, d.n_phi, d.n_z = int(spec.n_r), int(spec.n_phi), int(spec.n_z)
    d.n_fold, d.m = int(spec.n_fold), int(spec.m)
    d.pml_r_in, d.pml_r_out, d.pml_z = int(spec.pml_r_in), int(spec.pml_r_out), int(spec.pml_z)
    if len(spec.layer_k0) > _lib.MAX_LAYERS:
        raise ValueError("at most %d layers" % _lib.MAX_LAYERS)
    d.n_layers = len(spec.layer_k0)
    for l, (k0, e) in enumerate(zip(spec.layer_k0, spec.layer_eps)):
        d.layer_k0[l] = int(k0)
        d.layer_eps[l] = float(e)
    d.design_k0, d.design_k1 = int(spec.design_k0), int(spec.design_k1)
    d.eps_lo, d.eps_hi = float(spec.eps_lo), float(spec.eps_hi)
    d.source_k, d.monitor_k = int(spec.source_k), int(spec.monitor_k)
    d.courant, d.n_steps = float(spec.courant), int(spec.n_steps)
    d.filter_radius, d.beta, d.eta = float(spec.filter_radius), float(spec.beta), float(spec.eta)
    d.focal = float(spec.focal)
    return d


class Context:
    def __init__(self, device=0):
        self.device = int(device)
        h = ctypes.c_void_p()
        check(_lib.lib().zda_ctx_create(ctypes.byref(h), self.device))
        self.handle = h

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            _lib.lib().zda_ctx_destroy(h)
            self.handle = None


_CTX = {}


def context(device=0):
    if device not in _CTX:
        _CTX[device] = Context(device)
    return _CTX[device]


def zone_info(spec, device=0):
    """The derived quantities of a zone description (dt, dphi, tau, n_freq,
    n_r_design, design_nk, workspace_bytes, cells) from zda_zone_query,
    without binding a workspace (nothing is allocated on the device)."""
    ctx = context(device)
    L = _lib.lib()
    h = ctypes.c_void_p()
    check(L.zda_zone_create(ctx.handle, ctypes.byref(make_desc(spec)), ctypes.byref(h)))
    try:
        lam = (ctypes.c_double * len(spec.wavelengths))(*[float(x) for x in spec.wavelengths])
        check(L.zda_set_wavelengths(h, lam, len(spec.wavelengths)))
        info = _lib.ZoneInfo()
        check(L.zda_zone_query(h, ctypes.byref(info)))
        return {f: getattr(info, f) for f, _ in _lib.ZoneInfo._fields_}
    finally:
        L.zda_zone_destroy(h)


class Zone:
    """One annular zone's n-fold wedge on one GPU (see include/zda.h)."""

    def __init__(self, spec, device=0):
        self.spec = spec
        self.device = torch.device("cuda", device)
        self.ctx = context(device)
        L = _lib.lib()
        h = ctypes.c_void_p()
        check(L.zda_zone_create(self.ctx.handle, ctypes.byref(make_desc(spec)), ctypes.byref(h)))
        self.handle = h
        lam = (ctypes.c_double * len(spec.wavelengths))(*[float(x) for x in spec.wavelengths])
        check(L.zda_set_wavelengths(h, lam, len(spec.wavelengths)))
        check(L.zda_set_pulse(h, float(spec.pulse_f0), float(spec.pulse_sigma), float(spec.pulse_t0)))
        info = _lib.ZoneInfo()
        check(L.zda_zone_query(h, ctypes.byref(info)))
        self.info = {f: getattr(info, f) for f, _ in _lib.ZoneInfo._fields_}
        self.n_freq = info.n_freq
        self.n_r_design = info.n_r_design
        self.design_nk = info.design_nk
        self.dt = info.dt
        self.workspace = torch.empty(int(info.workspace_bytes), dtype=torch.uint8, device=self.device)
        check(L.zda_zone_bind_workspace(h, _ptr(self.workspace), self.workspace.numel()))
        self.version = 0

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            _lib.lib().zda_zone_destroy(h)
            self.handle = None

    # ------------------------------------------------------------------
    def _rho(self, rho):
        if not (isinstance(rho, torch.Tensor) and rho.is_cuda):
            raise TypeError("rho must be a CUDA tensor")
        if tuple(rho.shape) != (self.n_r_design, self.spec.n_phi):
            raise ValueError("rho must have shape (%d, %d)" % (self.n_r_design, self.spec.n_phi))
        return rho.detach().to(torch.float32).contiguous()

    def forward(self, rho):
        """Forward run; returns the focal phasors S (complex128, n_freq)."""
        r = self._rho(rho)
        out = (ctypes.c_double * (2 * self.n_freq))()
        check(_lib.lib().zda_forward(self.handle, _ptr(r), out, _stream()))
        self.version += 1
        self._last_rho = r
        a = np.frombuffer(out, dtype=np.float64).copy()
        return a[0::2] + 1j * a[1::2]

    def adjoint(self, dI_dS):
        """Adjoint run for g_q = dI/dRe S_q + i dI/dIm S_q; returns dI/drho."""
        g = np.asarray(dI_dS, dtype=np.complex128)
        buf = (ctypes.c_double * (2 * self.n_freq))(*np.stack([g.real, g.imag], 1).ravel().tolist())
        grad = torch.empty((self.n_r_design, self.spec.n_phi), dtype=torch.float32, device=self.device)
        check(_lib.lib().zda_adjoint(self.handle, buf, _ptr(grad), _stream()))
        return grad

    def iteration(self, rho, host=False):
        """One TopOpt iteration of I = 2 sum |S|^2: returns (I, dI/drho).
        host=True takes and returns host (CPU) float32 tensors; the call copies
        them to / from the device itself."""
        I = ctypes.c_double()
        if host:
            r = rho.detach().to(torch.float32).contiguous()
            assert not r.is_cuda
            g = torch.empty_like(r)
            check(_lib.lib().zda_iteration(self.handle, _ptr(r), ctypes.byref(I), _ptr(g), 1, _stream()))
        else:
            r = self._rho(rho)
            g = torch.empty_like(r)
            check(_lib.lib().zda_iteration(self.handle, _ptr(r), ctypes.byref(I), _ptr(g), 0, _stream()))
        self.version += 1
        return I.value, g

    def filter_project(self, rho):
        r = self._rho(rho)
        out = torch.empty_like(r)
        check(_lib.lib().zda_filter_project(self.handle, _ptr(r), _ptr(out), _stream()))
        return out

    def filter_project_backward(self, rho, g_tilde):
        r = self._rho(rho)
        g = g_tilde.detach().to(torch.float32).contiguous()
        out = torch.empty_like(r)
        check(_lib.lib().zda_filter_project_backward(self.handle, _ptr(r), _ptr(g), _ptr(out), _stream()))
        return out

    def focal_transform(self, monitor_dft):
        m = monitor_dft.detach().to(torch.complex64).contiguous()
        assert tuple(m.shape) == (self.n_freq, 2, self.spec.n_r, self.spec.n_phi)
        out = (ctypes.c_double * (2 * self.n_freq))()
        check(_lib.lib().zda_focal_transform(self.handle, _ptr(m), out, _stream()))
        a = np.frombuffer(out, dtype=np.float64).copy()
        return a[0::2] + 1j * a[1::2]

    def fields(self):
        s = self.spec
        out = torch.empty((6, s.n_r, s.n_phi, s.n_z), dtype=torch.complex64, device=self.device)
        check(_lib.lib().zda_copy_fields(self.handle, _ptr(out), _stream()))
        return out

    def monitor_dft(self):
        s = self.spec
        out = torch.empty((self.n_freq, 2, s.n_r, s.n_phi), dtype=torch.complex64, device=self.device)
        check(_lib.lib().zda_copy_monitor_dft(self.handle, _ptr(out), _stream()))
        return out

    def design_dft(self, which=0):
        """[n_freq][3][n_r][n_phi][design_nk] complex64 (which: 0 forward, 1 adjoint)."""
        s = self.spec
        out = torch.empty((self.n_freq, 3, s.n_r, s.n_phi, self.design_nk), dtype=torch.complex64,
                          device=self.device)
        check(_lib.lib().zda_copy_design_dft(self.handle, int(which), _ptr(out), _stream()))
        return out

    def set_kernel(self, variant=1, tile_phi=2, i_ranges=0):
        """Time-step kernel (zda_zone_set_kernel): 0 split H/E (tile_phi = phi
        rows per block), 1 fused streaming (tile_phi 2 or 4), 2 split one cell
        per thread, 3 fused TMA tiles (tile_phi 4, 8 or 16; i_ranges radius
        ranges), 4 split with the E half on TMA tiles (tile_phi 8, 16 or 32;
        i_ranges radius ranges), 5 the same with both halves on TMA tiles."""
        check(_lib.lib().zda_zone_set_kernel(self.handle, int(variant), int(tile_phi), int(i_ranges)))

    def set_radial_pml(self, form):
        """r-PML form: 0 convolutional PML with the real radius (default),
        1 stretched coordinates (split radial curl, stretched outer radius)."""
        check(_lib.lib().zda_zone_set_radial_pml(self.handle, int(form)))

    def radial_pml(self):
        f = ctypes.c_int()
        check(_lib.lib().zda_zone_get_radial_pml(self.handle, ctypes.byref(f)))
        return f.value

    def time_steps(self, steps):
        """Milliseconds for `steps` steps of the current step kernel (no
        source, no DFT); overwrites the fields."""
        ms = ctypes.c_double()
        check(_lib.lib().zda_zone_time_steps(self.handle, int(steps), ctypes.byref(ms), _stream()))
        return ms.value

    def set_projection(self, beta, eta=0.5):
        check(_lib.lib().zda_zone_set_projection(self.handle, float(beta), float(eta)))

    def set_wait_limit(self, polls, inject_timeout=False):
        check(_lib.lib().zda_zone_set_wait_limit(self.handle, int(polls), int(bool(inject_timeout))))

    def get_kernel(self):
        v, t, r = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(_lib.lib().zda_zone_get_kernel(self.handle, ctypes.byref(v), ctypes.byref(t), ctypes.byref(r)))
        return v.value, t.value, r.value

    def set_timing(self, every):
        """Sample every `every`-th time step's launches with CUDA events (0: off)."""
        check(_lib.lib().zda_zone_set_timing(self.handle, int(every)))

    def timing(self):
        """([ms of launch 1, 2, 3 summed over the samples], sampled steps) since
        the last call; split step: H update, E update, DFT update (one z-cell
        per thread: the DFT is inside the E update); fused step: streaming
        kernel, 0, DFT kernel."""
        ms = (ctypes.c_double * 3)()
        n = ctypes.c_longlong()
        check(_lib.lib().zda_zone_timing(self.handle, ms, ctypes.byref(n)))
        return list(ms), n.value

    def set_energy_probe(self, every):
        """Record the field energy W and the energy of the one-step difference
        Wdot after every `every`-th step of each forward run (0: off)."""
        check(_lib.lib().zda_zone_set_energy_probe(self.handle, int(every)))
        self._probe_every = int(every)

    def energy_trace(self, max_samples=1 << 20):
        """(steps, W, Wdot) of the last forward run's decay probe."""
        n = ctypes.c_int()
        m = int(min(max_samples, max(1, self.spec.n_steps)))
        w = (ctypes.c_double * m)()
        wd = (ctypes.c_double * m)()
        check(_lib.lib().zda_zone_energy_trace(self.handle, w, wd, m, ctypes.byref(n)))
        k = n.value
        every = self._probe_every if getattr(self, "_probe_every", 0) else 1
        steps = every * (np.arange(k) + 1)
        return steps, np.array(w[:k]), np.array(wd[:k])

    @property
    def launches(self):
        return int(_lib.lib().zda_zone_launch_count(self.handle))


def intensity(S):
    """Summed focal-spot intensity I = 2 sum_q |S_q|^2 of the m = +-1 runs."""
    return 2.0 * float(np.sum(np.abs(S) ** 2))


class ZoneFocal(torch.autograd.Function):
    """rho -> focal phasors S (float64 tensor [n_freq, 2] = (Re, Im)) with the
    adjoint run as the hand-written backward; compose with any objective of
    S, e.g. I = 2 * (S ** 2).sum()."""

    @staticmethod
    def forward(ctx, rho, zone):
        S = zone.forward(rho)
        ctx.zone = zone
        ctx.version = zone.version
        ctx.save_for_backward(rho)
        return torch.from_numpy(np.stack([S.real, S.imag], 1)).to(rho.device)

    @staticmethod
    def backward(ctx, grad_S):
        zone = ctx.zone
        (rho,) = ctx.saved_tensors
        if zone.version != ctx.version:        # another forward ran on this zone since
            zone.forward(rho)
        g = grad_S.detach().to("cpu", torch.float64).numpy()
        grad = zone.adjoint(g[:, 0] + 1j * g[:, 1])
        return grad.to(rho.dtype), None


def zone_focal(rho, zone):
    return ZoneFocal.apply(rho, zone)
