"""GB300-native singular value soft-thresholding via the polar decomposition.

A_tau = U max(Sigma - tau I, 0) V^T (Eq. 1) computed without an SVD as
1/2 (A - tau P)(I + S) with P = polar(A), S = polar(A^T A - tau^2 I)
(Proposition 1), all on tcgen05 tensor cores of one GB300 (sm_103a).

The compute path is the C-ABI library libsvt.so (include/svt.h); this package
is its Python binding.
"""
from .binding import (BF16, FP32, FP64, Context, Matrix, Options, SVTError,  # noqa: F401
                      EXPORTS, lib, make_options, polar_noalloc, read_completion_stats,
                      fp8_policy, schedule_coeffs, status_str, workspace_bytes,
                      workspace_bytes_fp8)
