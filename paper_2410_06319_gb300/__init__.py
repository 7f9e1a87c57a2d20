"""GB300 (sm_103a) mixed-precision sketch-and-precondition least squares.

Python binding of the C ABI in ``include/lsq.h`` (Carson & Dauzickaite,
arXiv 2410.06319: Algorithm 1 -- sketch and Householder R; Algorithm 2 --
R-preconditioned LSQR and FGMRES-based augmented-system refinement).

The functions ``lsq_sketch``, ``lsq_qr_r``, ``lsq_lsqr``, ``lsq_lsir`` and
``lsq_omega`` keep the C names and arguments; they only marshal arguments
(torch CUDA tensors or raw device pointers; host arrays for
``lsq_lsir_host``) and call the library, whose
kernels do all the work.  Importing this module fails loudly if the CUDA
library has not been built; there is no fallback.
"""
from ._lib import (  # noqa: F401
    KERNELS, PREC, STATUS, Handle, Info, LsqError, Opts, Problem, lib, lsq_ir_step, lsq_lsir, lsq_lsir_batched,
    lsq_lsir_host,
    lsq_lsqr, lsq_omega, lsq_probe_fma_rate, lsq_qr_r, lsq_qr_r_noalloc, lsq_residual, lsq_sketch, library_path,
    declared_functions,
)
