"""GB300-native batched element-local contraction (dG FEM volume, Table 1).

    out[f, e, i] = sum_j D_f[i, j] * u[e, j]

The CUDA library (csrc/, built by build.py into _build/liblc.so) implements the
C ABI of include/lc.h; ``lc`` is its ctypes binding.
"""

from . import lc  # noqa: F401
from .build import build  # noqa: F401
