"""ctypes declarations of the libzda C ABI (include/zda.h).

Argument marshalling only.  If libzda.so has not been built this module
raises at import: there is no CPU fallback.
"""
import ctypes
import os

from . import build as _build

MAX_LAYERS = 8
MAX_FREQ = 16

OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_TIMEOUT, ERR_NONFINITE, ERR_STATE = 0, -1, -2, -3, -4, -5, -6
_NAMES = {ERR_ARG: "ZDA_ERR_ARG", ERR_CUDA: "ZDA_ERR_CUDA", ERR_OOM: "ZDA_ERR_OOM",
          ERR_TIMEOUT: "ZDA_ERR_TIMEOUT", ERR_NONFINITE: "ZDA_ERR_NONFINITE", ERR_STATE: "ZDA_ERR_STATE"}


class ZdaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_NAMES.get(status, str(status)), msg))
        self.status = status


class ZoneDesc(ctypes.Structure):
    _fields_ = [
        ("r_lo", ctypes.c_double), ("dr", ctypes.c_double), ("dz", ctypes.c_double),
        ("n_r", ctypes.c_int), ("n_phi", ctypes.c_int), ("n_z", ctypes.c_int),
        ("n_fold", ctypes.c_int), ("m", ctypes.c_int),
        ("pml_r_in", ctypes.c_int), ("pml_r_out", ctypes.c_int), ("pml_z", ctypes.c_int),
        ("n_layers", ctypes.c_int),
        ("layer_k0", ctypes.c_int * MAX_LAYERS),
        ("layer_eps", ctypes.c_double * MAX_LAYERS),
        ("design_k0", ctypes.c_int), ("design_k1", ctypes.c_int),
        ("eps_lo", ctypes.c_double), ("eps_hi", ctypes.c_double),
        ("source_k", ctypes.c_int), ("monitor_k", ctypes.c_int),
        ("courant", ctypes.c_double),
        ("n_steps", ctypes.c_int),
        ("filter_radius", ctypes.c_double), ("beta", ctypes.c_double), ("eta", ctypes.c_double),
        ("focal", ctypes.c_double),
    ]


class ZoneInfo(ctypes.Structure):
    _fields_ = [
        ("dt", ctypes.c_double), ("dphi", ctypes.c_double), ("tau", ctypes.c_double),
        ("n_freq", ctypes.c_int), ("n_r_design", ctypes.c_int), ("design_nk", ctypes.c_int),
        ("workspace_bytes", ctypes.c_size_t), ("cells", ctypes.c_longlong),
    ]


_vp = ctypes.c_void_p
_i = ctypes.c_int
_dp = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes); every symbol include/zda.h declares
SIGNATURES = {
    "zda_ctx_create": (_i, [ctypes.POINTER(_vp), _i]),
    "zda_ctx_destroy": (None, [_vp]),
    "zda_zone_create": (_i, [_vp, ctypes.POINTER(ZoneDesc), ctypes.POINTER(_vp)]),
    "zda_zone_destroy": (None, [_vp]),
    "zda_set_wavelengths": (_i, [_vp, _dp, _i]),
    "zda_set_pulse": (_i, [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    "zda_zone_query": (_i, [_vp, ctypes.POINTER(ZoneInfo)]),
    "zda_zone_set_projection": (_i, [_vp, ctypes.c_double, ctypes.c_double]),
    "zda_zone_workspace_bytes": (_i, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "zda_zone_bind_workspace": (_i, [_vp, _vp, ctypes.c_size_t]),
    "zda_forward": (_i, [_vp, _vp, _dp, _vp]),
    "zda_adjoint": (_i, [_vp, _dp, _vp, _vp]),
    "zda_iteration": (_i, [_vp, _vp, _dp, _vp, _i, _vp]),
    "zda_filter_project": (_i, [_vp, _vp, _vp, _vp]),
    "zda_filter_project_backward": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "zda_focal_transform": (_i, [_vp, _vp, _dp, _vp]),
    "zda_copy_fields": (_i, [_vp, _vp, _vp]),
    "zda_copy_monitor_dft": (_i, [_vp, _vp, _vp]),
    "zda_copy_design_dft": (_i, [_vp, _i, _vp, _vp]),
    "zda_zone_launch_count": (ctypes.c_longlong, [_vp]),
    "zda_zone_set_kernel": (_i, [_vp, _i, _i, _i]),
    "zda_zone_get_kernel": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "zda_zone_set_radial_pml": (_i, [_vp, _i]),
    "zda_zone_get_radial_pml": (_i, [_vp, ctypes.POINTER(_i)]),
    "zda_zone_set_wait_limit": (_i, [_vp, _i, _i]),
    "zda_zone_time_steps": (_i, [_vp, _i, _dp, _vp]),
    "zda_zone_set_timing": (_i, [_vp, _i]),
    "zda_zone_timing": (_i, [_vp, _dp, ctypes.POINTER(ctypes.c_longlong)]),
    "zda_zone_set_energy_probe": (_i, [_vp, _i]),
    "zda_zone_energy_trace": (_i, [_vp, _dp, _dp, _i, ctypes.POINTER(_i)]),
    "zda_filter_project_noalloc": (_i, [ctypes.POINTER(ZoneDesc), _vp, _vp, _vp]),
    "zda_lens_create": (_i, [_vp, ctypes.POINTER(_vp), _i, ctypes.POINTER(_vp)]),
    "zda_lens_destroy": (None, [_vp]),
    "zda_lens_workspace_bytes": (_i, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "zda_lens_bind_workspace": (_i, [_vp, _vp, ctypes.c_size_t]),
    "zda_lens_set_graph": (_i, [_vp, _i]),
    "zda_lens_forward": (_i, [_vp, ctypes.POINTER(_vp), _dp, _vp]),
    "zda_lens_adjoint": (_i, [_vp, _dp, ctypes.POINTER(_vp), _vp]),
    "zda_lens_zone_focal": (_i, [_vp, _i, _dp]),
    "zda_lens_launch_count": (ctypes.c_longlong, [_vp]),
    "zda_lens_focal_plane": (_i, [_vp, _vp, _i, _i, _vp, _dp, _vp]),
    "zda_lens_field_points": (_i, [_vp, _vp, _i, _i, _vp, _vp]),
    "zda_lens_evaluate_scratch_bytes": (_i, [_vp, _i, _i, _i, ctypes.POINTER(ctypes.c_size_t)]),
    "zda_lens_evaluate": (_i, [_vp, ctypes.c_double, ctypes.c_double, _dp, ctypes.c_double, _i, ctypes.c_double, _i,
                               _i, _i, _vp, ctypes.c_size_t, _dp, _vp, _vp]),
    "zda_zone_incident_intensity": (_i, [_vp, _vp, _vp]),
    "zda_field_intensity": (_i, [_vp, _i, _i, ctypes.c_double, _vp, _vp]),
    "zda_encircled_power": (_i, [_vp, _vp, _i, _i, _vp, _vp]),
    "zda_zone_order_bound": (_i, [_vp, _vp, _i, _vp, _i, _i, ctypes.POINTER(ctypes.c_double)]),
    "zda_last_error": (ctypes.c_char_p, []),
    "zda_focal_transform_nn": (_i, [_vp, _vp, _i, ctypes.c_float, _vp, _vp]),
    "zda_focal_transform_nn_transpose": (_i, [_vp, _vp, _i, ctypes.c_float, _vp, _vp]),
    # surrogate network (include/zda_nn.h)
    "zda_nn_create": (_i, [_i, _vp, _vp]),
    "zda_nn_destroy": (None, [_vp]),
    "zda_nn_param_count": (_i, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "zda_nn_forward_flops": (_i, [_vp, _dp]),
    "zda_nn_workspace_bytes": (_i, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "zda_nn_bind_workspace": (_i, [_vp, _vp, ctypes.c_size_t]),
    "zda_nn_set_params": (_i, [_vp, _vp, _i, _vp]),
    "zda_nn_get_params": (_i, [_vp, _vp, _i, _vp]),
    "zda_nn_get_grads": (_i, [_vp, _vp, _i, _vp]),
    "zda_nn_forward": (_i, [_vp, _vp, _i, _vp, _vp]),
    "zda_nn_backward": (_i, [_vp, _vp, _vp, _vp]),
    "zda_nn_mse": (_i, [_vp, _vp, _vp, _i, _vp, _vp, _vp]),
    "zda_nn_adam": (_i, [_vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _vp]),
    "zda_nn_launch_count": (ctypes.c_longlong, [_vp]),
    "zda_nn_set_timing": (_i, [_vp, _i]),
    "zda_nn_timing": (_i, [_vp, _dp, _dp, ctypes.POINTER(ctypes.c_int)]),
    "zda_nn_check": (_i, [_vp, _vp]),
}


class NnDesc(ctypes.Structure):
    """zda_nn_desc of include/zda_nn.h."""
    _fields_ = [("batch", ctypes.c_int), ("height", ctypes.c_int), ("width", ctypes.c_int),
                ("in_ch", ctypes.c_int), ("out_ch", ctypes.c_int)]


def load(path=None):
    path = path or _build.lib_path()
    if not os.path.exists(path):
        raise ImportError("libzda.so not found at %s: build it first "
                          "(python -c 'import __graft_entry__ as g; g.build()')" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        _LIB = load()
    return _LIB


def check(status):
    if status != OK:
        raise ZdaError(status, lib().zda_last_error().decode(errors="replace"))
