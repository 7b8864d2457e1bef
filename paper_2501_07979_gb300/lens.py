"""A lens = concentric zones (section "Zoned discrete axisymmetry (ZDA)").

Zones are independent FDTD problems; the only coupling of a whole-lens
iteration is the focal field, the sum of the zones' focal phasors
(2 x wavelengths complex numbers), whose sensitivity every zone needs for its
adjoint run.  With several processes (one GPU each) the zones are assigned
by longest-processing-time-first on their cost n_r n_phi n_z n_steps and the
phasor sum is one all-reduce of a few hundred bytes.

The zone solver is pluggable (any object with forward(rho) -> S and
adjoint(dI_dS) -> grad): `Zone` on a GPU, or any stand-in.
"""
import ctypes
import warnings

import numpy as np

ORDER_BOUND_TOL = 1e-3


def order_bound(spec, pts):
    """Bound on the azimuthal orders the lens-field transforms neglect for
    one zone at points (x, y) or (x, y, h) (zda_zone_order_bound)."""
    from . import _lib
    from ._lib import check
    from .zone import make_desc
    pts = np.ascontiguousarray(np.asarray(pts, dtype=np.float64))
    stride = pts.shape[-1]
    pts = pts.reshape(-1, stride)
    lam = np.ascontiguousarray(np.asarray(spec.wavelengths, dtype=np.float64))
    d = make_desc(spec)
    out = ctypes.c_double()
    check(_lib.lib().zda_zone_order_bound(ctypes.byref(d), lam.ctypes.data, lam.size, pts.ctypes.data,
                                          pts.shape[0], stride, ctypes.byref(out)))
    return out.value


def zone_cost(spec):
    return float(spec.n_r) * spec.n_phi * spec.n_z * spec.n_steps


def assign_zones(specs, world):
    """Longest-processing-time-first: returns owner rank per zone (list)."""
    order = sorted(range(len(specs)), key=lambda z: -zone_cost(specs[z]))
    load = [0.0] * world
    owner = [0] * len(specs)
    for z in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[z] = r
        load[r] += zone_cost(specs[z])
    return owner


class ShardedLens:
    """Zones of one lens spread over the ranks of a torch.distributed group.

    solvers: {zone index: solver} for the zones this rank owns.
    forward(rhos) -> S_lens (complex, summed over all zones of all ranks).
    adjoint(dI_dS) -> {zone index: dI/drho} for the local zones, with dI_dS
    the objective's sensitivity to the lens phasors (the same for every zone:
    dS_lens/dS_zone = 1).
    """

    def __init__(self, specs, solvers, group=None):
        self.specs = specs
        self.solvers = solvers
        self.group = group

    def _allreduce(self, x):
        """Sum of the ranks' phasors (2 x n_freq float64).  NCCL reduces device
        tensors only: under it the buffer goes to this rank's current CUDA
        device; gloo reduces it on the host."""
        import torch
        import torch.distributed as dist
        if not dist.is_available() or not dist.is_initialized():
            return x
        t = torch.from_numpy(np.ascontiguousarray(np.stack([x.real, x.imag], 1)))
        if dist.get_backend(self.group) == "nccl":
            t = t.to("cuda:%d" % torch.cuda.current_device())
        dist.all_reduce(t, group=self.group)
        a = t.cpu().numpy()
        return a[:, 0] + 1j * a[:, 1]

    def forward(self, rhos):
        S = None
        for z, solver in sorted(self.solvers.items()):
            s = np.asarray(solver.forward(rhos[z]), dtype=np.complex128)
            S = s if S is None else S + s
        if S is None:
            nq = 2 * len(self.specs[0].wavelengths)
            S = np.zeros(nq, np.complex128)
        return self._allreduce(S)

    def adjoint(self, dI_dS):
        return {z: solver.adjoint(dI_dS) for z, solver in sorted(self.solvers.items())}


class Lens:
    """All zones of a lens on one GPU through the C ABI (zda_lens_*): one
    CUDA graph launch runs every zone's forward (or adjoint) run, the zones'
    focal phasors are summed on the device."""

    def __init__(self, zones, use_graph=True):
        import torch
        from . import _lib
        from ._lib import check
        self.zones = list(zones)
        L = _lib.lib()
        arr = (ctypes.c_void_p * len(self.zones))(*[z.handle.value for z in self.zones])
        h = ctypes.c_void_p()
        check(L.zda_lens_create(self.zones[0].ctx.handle, arr, len(self.zones), ctypes.byref(h)))
        self.handle = h
        nb = ctypes.c_size_t()
        check(L.zda_lens_workspace_bytes(h, ctypes.byref(nb)))
        self.workspace = torch.empty(max(int(nb.value), 256), dtype=torch.uint8, device=self.zones[0].device)
        check(L.zda_lens_bind_workspace(h, ctypes.c_void_p(self.workspace.data_ptr()), self.workspace.numel()))
        check(L.zda_lens_set_graph(h, int(bool(use_graph))))
        self.n_freq = self.zones[0].n_freq

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                from . import _lib
                _lib.lib().zda_lens_destroy(h)
            except ImportError:          # interpreter shutting down
                pass
            self.handle = None

    def _stream(self):
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def forward(self, rhos):
        """rhos: list of CUDA float32 tensors (one per zone) -> lens phasors S."""
        from . import _lib
        from ._lib import check
        rs = [z._rho(r) for z, r in zip(self.zones, rhos)]
        self._rhos = rs
        arr = (ctypes.c_void_p * len(rs))(*[r.data_ptr() for r in rs])
        out = (ctypes.c_double * (2 * self.n_freq))()
        check(_lib.lib().zda_lens_forward(self.handle, arr, out, self._stream()))
        a = np.frombuffer(out, dtype=np.float64).copy()
        return a[0::2] + 1j * a[1::2]

    def zone_focal(self, z):
        from . import _lib
        from ._lib import check
        out = (ctypes.c_double * (2 * self.n_freq))()
        check(_lib.lib().zda_lens_zone_focal(self.handle, int(z), out))
        a = np.frombuffer(out, dtype=np.float64).copy()
        return a[0::2] + 1j * a[1::2]

    def adjoint(self, dI_dS):
        """dI_dS: n_freq complex (dI/dRe S + i dI/dIm S of the lens phasors)
        -> list of dI/drho tensors, one per zone."""
        import torch
        from . import _lib
        from ._lib import check
        g = np.asarray(dI_dS, dtype=np.complex128)
        buf = (ctypes.c_double * (2 * self.n_freq))(*np.stack([g.real, g.imag], 1).ravel().tolist())
        grads = [torch.empty((z.n_r_design, z.spec.n_phi), dtype=torch.float32, device=z.device)
                 for z in self.zones]
        arr = (ctypes.c_void_p * len(grads))(*[t.data_ptr() for t in grads])
        check(_lib.lib().zda_lens_adjoint(self.handle, buf, arr, self._stream()))
        return grads

    @property
    def launches(self):
        from . import _lib
        return int(_lib.lib().zda_lens_launch_count(self.handle))

    def focal_plane(self, pts_xy, n_phi_samples=128):
        """Focal-plane field of the last forward at points (x, y) (n x 2):
        returns (E_x, E_y) as complex arrays [n_lambda][n_pts] and the
        transmitted power per wavelength."""
        import torch
        from . import _lib
        from ._lib import check
        pts = torch.tensor(np.asarray(pts_xy, dtype=np.float64).reshape(-1, 2), device=self.zones[0].device)
        n = pts.shape[0]
        nl = self.n_freq // 2
        out = torch.empty((2, nl, n, 2), dtype=torch.float64, device=pts.device)
        pt = (ctypes.c_double * nl)()
        check(_lib.lib().zda_lens_focal_plane(self.handle, ctypes.c_void_p(pts.data_ptr()), int(n), int(n_phi_samples),
                                              ctypes.c_void_p(out.data_ptr()), pt, self._stream()))
        o = out.cpu().numpy()
        self._check_orders(pts_xy)
        return o[0, ..., 0] + 1j * o[0, ..., 1], o[1, ..., 0] + 1j * o[1, ..., 1], np.array(pt[:])

    def order_bound(self, pts):
        """Largest zda_zone_order_bound over the lens's zones at these points."""
        return max(order_bound(z.spec, pts) for z in self.zones)

    def _check_orders(self, pts):
        b = self.order_bound(pts)
        if b > ORDER_BOUND_TOL:
            warnings.warn("lens field: the neglected azimuthal orders may reach %.2g of the kept ones at these "
                          "points (zones with small n far off axis)" % b, RuntimeWarning, stacklevel=3)

    def field_points(self, pts_xyh, n_phi_samples=128):
        """Field of the last forward at points (x, y, h), h = height above the
        focal plane: returns (E_x, E_y) as complex arrays [n_lambda][n_pts]."""
        import torch
        from . import _lib
        from ._lib import check
        pts = torch.tensor(np.asarray(pts_xyh, dtype=np.float64).reshape(-1, 3), device=self.zones[0].device)
        n = pts.shape[0]
        nl = self.n_freq // 2
        out = torch.empty((2, nl, n, 2), dtype=torch.float64, device=pts.device)
        check(_lib.lib().zda_lens_field_points(self.handle, ctypes.c_void_p(pts.data_ptr()), int(n),
                                               int(n_phi_samples), ctypes.c_void_p(out.data_ptr()), self._stream()))
        o = out.cpu().numpy()
        self._check_orders(np.asarray(pts_xyh, dtype=np.float64).reshape(-1, 3))
        return o[0, ..., 0] + 1j * o[0, ..., 1], o[1, ..., 0] + 1j * o[1, ..., 1]
