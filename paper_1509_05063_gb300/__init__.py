"""GB300 (sm_103a) Lippmann-Schwinger Nystrom solver: thin Python binding of the
C ABI in include/ls.h.  Every step of the apply and solve runs in the library's
CUDA kernels; this package only marshals arguments."""
from .ls import (LS_FP64, LS_MIXED, LS_MIXED32, Batch, HostAccel3, HostBall3, HostPlan, LSError, Plan, Plan3,
                 build_library, geometry_from, interior_window3, lib_path, load_library, measure_peaks,
                 options_from)

__all__ = ["Plan", "Plan3", "measure_peaks", "Batch", "HostPlan", "HostAccel3", "HostBall3", "LSError", "LS_FP64", "LS_MIXED", "LS_MIXED32",
           "load_library", "build_library", "lib_path", "geometry_from", "options_from", "interior_window3"]
