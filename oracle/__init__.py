"""FP64 CPU oracle for the RPM-FFT method - test infrastructure only.

Imported by the tests, by the package smoke check and by the benchmark's CPU
baseline leg; never by the library's compute path.
"""
from .rpm_oracle import *  # noqa: F401,F403
from . import rpm_oracle  # noqa: F401
