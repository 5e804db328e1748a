"""Plain CPU FP64 oracle for polynomial-preconditioned GMRES (Loe & Morgan).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` use it.  It shares no code with
the CUDA library; the only thing both sides use is the seeded input module
``synth``.

Modules
-------
``oracle.poly``   Arnoldi / GMRES(d) polynomial construction, harmonic Ritz
                  values (Algorithm 4 step 1(b)), modified Leja ordering and
                  the pof root-adding rule (Algorithm 2), phi(A) v
                  (Algorithm 1) and p(A) v (Algorithm 3), plus their scalar
                  versions.
``oracle.gmres``  Restarted GMRES(m) on phi(A) with x = p(A) y (Algorithm 4
                  step 2), the FP32-inner flexible form, the stability check
                  StCh (Section 3.5) and the adjoint gradients.

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms
(dense matrix polynomials, brute-force least squares over an explicit Krylov
basis, a second eigenvalue route), hand-derived golden fixtures and numbers
printed in the paper.  Iteration counts of the full solver against the
paper's tables are "parity unpinned" (the paper's runs used MGS and an
unstated random stream); they are pinned only as trends.
"""
from . import poly, gmres  # noqa: F401
