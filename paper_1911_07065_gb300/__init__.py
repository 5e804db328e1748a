"""GB300 (sm_103a) polynomial-preconditioned GMRES (Loe & Morgan).

The hot path -- the GMRES polynomial in root form applied as a chain of
fused CSR SpMV-root kernels (Algorithms 1 and 3) inside restarted GMRES(m)
with CGS2 and Givens least squares (Algorithm 4) -- lives in the CUDA
library ``_lib/libppgmres.so`` behind the C ABI of ``include/ppgmres.h``.
This package is its Python binding; importing it without the built library
raises ImportError.  On import the library is (re)built in-tree when it is
missing or older than its sources (set PPG_NO_AUTOBUILD=1 to skip that).
"""
import os as _os

if not _os.environ.get("PPG_NO_AUTOBUILD"):
    from .build import build as _build
    _build()

from ._binding import (EXPORTS, PPGError, Roots, add_roots, csr_validate_host,  # noqa: F401
                       harmonic_ritz, leja_order, lib, roots_from_hessenberg, STATUS)

try:  # the device API needs torch; the host-only steps above do not
    from .api import (CSR, PPGMRESFunction, adjoint_vals_grad, apply_phi,  # noqa: F401
                      apply_poly, apply_poly_noalloc, build_poly, build_poly_checked, build_poly_composite, solve, solve_batched, solve_chpoly, solve_double, solve_flex, solve_host, spmv,
                      stability_check, SweepPlan, solve_flex_sweep)
except ImportError:  # pragma: no cover
    pass

__version__ = "0.1.0"
