"""GB300-native HOTRG for the 4D Ising model (arXiv:1911.12954, Sec. 2 and 3.1).

The compute path is libhotrg.so (CUDA for sm_103a, C ABI in include/hotrg.h); this
package holds its sources (csrc/), its build script and a thin ctypes binding.
"""

from .hotrg import (FP32, FP64, IMPURE_NONE, IMPURE_SIGMA, IMPURE_SIGMASIGMA, OPT_AUTOTUNE,  # noqa: F401
                    OPT_GEMM_VARIANT, OPT_GRAPHS, OPT_GROUP, OPT_JACOBI_SWEEPS, OPT_MAXNORM, PRECISIONS, SYMBOLS,
                    TF32X3, HOTRG, HotrgError, library_path)
