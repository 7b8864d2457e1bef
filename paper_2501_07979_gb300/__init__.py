"""GB300-native zone solver of the zoned-discrete-axisymmetry metalens method.

The compute path is libzda (CUDA, sm_103a) behind the C ABI in
include/zda.h; this package is its Python binding.  Importing it loads the
library and fails if it has not been built -- there is no CPU fallback.
"""
from ._lib import ZdaError, lib  # noqa: F401  (loads libzda.so or raises)
from .zone import Zone, ZoneFocal, zone_focal, intensity, make_desc  # noqa: F401

lib()
