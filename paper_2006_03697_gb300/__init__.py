"""GB300 (sm_103a) infinite-cell Clenshaw-Curtis Spectral Quadrature: density, energies and
density-matrix stress (arXiv 2006.03697, Sec. 4). The compute path is the CUDA library
libsq_gb300.so (C ABI in include/sq_api.h); `sq` is its ctypes binding."""
from . import sq  # noqa: F401
