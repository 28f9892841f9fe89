"""GB300 (sm_103a) Fourier-domain jerk search.

The search runs in the hand-written CUDA kernels of ``libjerk.so`` behind
the C ABI in ``include/jerk.h``; ``jerk`` is its ctypes binding.
"""
from .jerk import (THRESH_ABS, THRESH_SIGMA, Candidate, Info, JerkError, Params, Plan, Refined,  # noqa: F401
                   lib, make_params, measure_packed_fma, measure_peaks)
