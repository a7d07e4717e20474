"""GB300-native Flux Reconstruction right-hand side (PyFR v2.0.3 hot path).

The compute path is the CUDA library ``lib/libfrgb.so`` (sources in
``csrc/``, C ABI in ``include/frgb.h``); this package only marshals
arguments to it.
"""
from ._binding import (ERRORS, ETYPES, AdaptCtl, FRError, FRGroup, FRMesh, load,  # noqa: F401
                       check_conversions, mlp_loss_grad, mlp_train, probe_fma)
from .build import build  # noqa: F401
