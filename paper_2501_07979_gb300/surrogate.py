"""Zone surrogate: a 4-level U-Net behind include/zda_nn.h (libzda).

The network maps a zone's density patch (n_r_design x n_phi pixels, plus
optional conditioning channels) to the zone's monitor-plane DFT over the
design annulus, the near field that the on-axis focal transform integrates.
It is trained on the GPU by the library's own tensor-core kernels on data
the FDTD solver generates, and serves only as a warm start: the zone's
topology optimisation is then refined with the adjoint FDTD, which also
measures the surrogate's error.

This module only marshals arguments; every step runs in libzda.
"""
import ctypes

import numpy as np

from . import _lib
from ._lib import check


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class Surrogate:
    """One network instance with its device workspace (a torch uint8 tensor).

    x, y tensors: float32 CUDA tensors [n][H][W][channels], n <= batch."""

    def __init__(self, height, width, in_ch, out_ch, batch, device=0):
        import torch
        self.device = torch.device("cuda", device)
        self.shape = (int(height), int(width))
        self.in_ch, self.out_ch, self.batch = int(in_ch), int(out_ch), int(batch)
        L = _lib.lib()
        d = _lib.NnDesc(batch=self.batch, height=self.shape[0], width=self.shape[1], in_ch=self.in_ch,
                        out_ch=self.out_ch)
        h = ctypes.c_void_p()
        check(L.zda_nn_create(int(device), ctypes.byref(d), ctypes.byref(h)))
        self.handle = h
        n = ctypes.c_size_t()
        check(L.zda_nn_param_count(h, ctypes.byref(n)))
        self.n_params = int(n.value)
        f = ctypes.c_double()
        check(L.zda_nn_forward_flops(h, ctypes.byref(f)))
        self.flops_per_sample = float(f.value)
        nb = ctypes.c_size_t()
        check(L.zda_nn_workspace_bytes(h, ctypes.byref(nb)))
        self.workspace = torch.empty(int(nb.value), dtype=torch.uint8, device=self.device)
        check(L.zda_nn_bind_workspace(h, _ptr(self.workspace), self.workspace.numel()))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                _lib.lib().zda_nn_destroy(h)
            except ImportError:
                pass
            self.handle = None

    def _stream(self):
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def _f32(self, t, shape=None):
        import torch
        t = torch.as_tensor(t, dtype=torch.float32, device=self.device).contiguous()
        if shape is not None and tuple(t.shape) != tuple(shape):
            raise ValueError("expected shape %s, got %s" % (shape, tuple(t.shape)))
        return t

    # ------------------------------------------------------------ parameters
    def layer_shapes(self):
        """(k, c_in, c_out) of the 15 layers in parameter order (include/zda_nn.h)."""
        C = 64
        layers = []
        for lev in range(3):
            layers += [(3, self.in_ch if lev == 0 else C, C), (3, C, C)]
        layers += [(3, C, C), (3, C, C)]
        for _ in range(3):
            layers += [(3, 2 * C, C), (3, C, C)]
        return layers + [(1, C, self.out_ch)]

    def init_params(self, seed):
        """He-normal weights (std sqrt(2 / fan_in)), zero biases, the head
        scaled by 0.1; sets them (and resets Adam)."""
        rng = np.random.default_rng(seed)
        shapes = self.layer_shapes()
        parts = []
        for i, (k, ci, co) in enumerate(shapes):
            std = np.sqrt(2.0 / (k * k * ci)) * (0.1 if i == len(shapes) - 1 else 1.0)
            parts += [rng.standard_normal(co * k * k * ci) * std, np.zeros(co)]
        v = np.concatenate(parts).astype(np.float32)
        assert v.size == self.n_params
        self.set_params(v)

    def set_params(self, vec):
        v = self._f32(np.asarray(vec, dtype=np.float32) if not hasattr(vec, "data_ptr") else vec)
        if v.numel() != self.n_params:
            raise ValueError("expected %d parameters" % self.n_params)
        check(_lib.lib().zda_nn_set_params(self.handle, _ptr(v), 0, self._stream()))

    def params(self):
        import torch
        out = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        check(_lib.lib().zda_nn_get_params(self.handle, _ptr(out), 0, self._stream()))
        return out

    def grads(self):
        import torch
        out = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        check(_lib.lib().zda_nn_get_grads(self.handle, _ptr(out), 0, self._stream()))
        return out

    # ------------------------------------------------------------ passes
    def forward(self, x):
        import torch
        x = self._f32(x)
        n = x.shape[0]
        if tuple(x.shape[1:]) != (*self.shape, self.in_ch):
            raise ValueError("x must be [n][%d][%d][%d]" % (*self.shape, self.in_ch))
        y = torch.empty((n, *self.shape, self.out_ch), dtype=torch.float32, device=self.device)
        check(_lib.lib().zda_nn_forward(self.handle, _ptr(x), int(n), _ptr(y), self._stream()))
        self._n = n
        return y

    def backward(self, dy, want_dx=False):
        """Gradient of the last forward: parameters (see grads()) and, with
        want_dx, the input gradient (returned)."""
        import torch
        dy = self._f32(dy, (self._n, *self.shape, self.out_ch))
        dx = torch.empty((self._n, *self.shape, self.in_ch), dtype=torch.float32,
                         device=self.device) if want_dx else None
        check(_lib.lib().zda_nn_backward(self.handle, _ptr(dy), _ptr(dx) if want_dx else None, self._stream()))
        return dx

    def mse(self, y, target):
        """(loss as a 1-element device tensor, dL/dy)."""
        import torch
        y = self._f32(y)
        t = self._f32(target, tuple(y.shape))
        dy = torch.empty_like(y)
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        check(_lib.lib().zda_nn_mse(self.handle, _ptr(y), _ptr(t), int(y.shape[0]), _ptr(dy), _ptr(loss),
                                    self._stream()))
        return loss, dy

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        check(_lib.lib().zda_nn_adam(self.handle, float(lr), float(beta1), float(beta2), float(eps), self._stream()))

    def train_step(self, x, target, lr=1e-3):
        """forward + MSE + backward + Adam; returns the loss tensor (device)."""
        y = self.forward(x)
        loss, dy = self.mse(y, target)
        self.backward(dy)
        self.adam(lr)
        return loss

    def set_timing(self, on=True):
        check(_lib.lib().zda_nn_set_timing(self.handle, int(bool(on))))

    def timing(self):
        """(summed ms, useful FLOPs, launches) of the timed forward convolutions."""
        ms, fl, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        check(_lib.lib().zda_nn_timing(self.handle, ctypes.byref(ms), ctypes.byref(fl), ctypes.byref(n)))
        return ms.value, fl.value, n.value

    def check(self):
        check(_lib.lib().zda_nn_check(self.handle, self._stream()))

    @property
    def launches(self):
        return int(_lib.lib().zda_nn_launch_count(self.handle))
