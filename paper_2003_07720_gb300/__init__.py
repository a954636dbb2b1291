"""GB300-native RPM-FFT: the Lippmann-Schwinger fixed-point map and the
recursive projection method as sm_103a CUDA kernels behind a C ABI
(include/rpm.h), plus a learned warm start (a spectral neural operator with
its own forward, backward and Adam kernels, include/rpm_fno.h).  This package
holds the kernels (csrc/), their build step and the ctypes bindings (rpm.py,
fno.py) and the training driver of the warm start (fno_train.py); it has no
other implementation of the method."""
from . import rpm  # noqa: F401
from .rpm import (Context, RpmError, rpm_apply_gamma, rpm_create, rpm_default_options,  # noqa: F401
                  rpm_destroy, rpm_effective_stiffness, rpm_effective_stiffness_batch,
                  rpm_grid_supported, rpm_pencil_tile, rpm_set_materials, rpm_set_options,
                  rpm_set_phase, rpm_solve)
