"""GB300 library for updating a rank-k truncated SVD of a sparse matrix with
the SV-LCOV method (arXiv 2401.09703): C ABI in include/svlcov.h, CUDA
kernels in csrc/, this package binds them for Python callers."""
from ._abi import SvlcovError, lib  # noqa: F401
from .svlcov import (SVLCOV, DeviceCSR, add_cols_with_grad, batch_run, dgemm, kernel_launches,  # noqa: F401
                     small_svd, small_svd_arrow)
