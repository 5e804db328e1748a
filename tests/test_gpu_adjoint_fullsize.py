"""Differentiation form at its full size (run with -m gpu): 2-D
convection-diffusion 512 x 512 with a per-node convection field, loss
L = 1/2 ||x - x*||^2.  The adjoint gradient (A^T solve with the same roots,
p(A^T) = p(A)^T) is checked three ways:

* against central finite differences (h = 1e-6) of device solves on the 20
  seeded random directions of the workload, each direction unit-norm over
  (b, vals) and scaled by ||b|| and ||vals||.  The solves run to relative
  residual 1e-13, or to the attainable level StCh predicts when that is
  higher (Section 3.5).  The difference quotient then carries a relative
  error of order 1e-7 from the solves and 1e-12 from truncation, so
  agreement within 1e-5 is required;
* against the oracle's adjoint (its own PP-GMRES on A^T, same roots, same
  dL/dx), lambda and dL/dvals within 1e-7 relative: both adjoint solves
  stop at relative residual 1e-13, and with kappa(A) of order 1e5 the two
  lambdas may differ by about kappa * 1e-13 relative;
* lambda against the host: A^T lambda = dL/dx.
"""
import numpy as np
import pytest

import synth
from oracle import gmres

from gpu_util import dev_csr, ppg_or_skip, to_dev

pytestmark = pytest.mark.gpu

N_DIRECTIONS = 20
H_FD = 1e-6


def test_adjoint_512_against_central_differences_and_the_oracle():
    p, torch = ppg_or_skip()
    P = synth.problem("cd2d_field_512")
    A = dev_csr(p, torch, P.A)
    R = p.build_poly(A, P.d, to_dev(torch, P.v0))
    xstar = to_dev(torch, P.extra["xstar"])
    b0 = to_dev(torch, P.b)
    # the attainable relative residual of this polynomial (Section 3.5)
    stch = p.stability_check(A, R, b0 / torch.linalg.norm(b0))
    tol = max(1e-13, 10.0 * stch)
    assert tol < 1e-12
    bt = b0.clone().requires_grad_(True)
    vt = A.vals.clone().requires_grad_(True)
    x = p.PPGMRESFunction.apply(bt, vt, A, R, P.m, tol, None, 400)
    loss = 0.5 * torch.sum((x - xstar) ** 2)
    loss.backward()
    gb = bt.grad.cpu().numpy()
    gv = vt.grad.cpu().numpy()
    As = P.A.to_scipy()
    g = (x - xstar).detach().cpu().numpy()
    # lambda = dL/db solves A^T lambda = x - x*
    assert np.linalg.norm(As.T @ gb - g) <= 1e-11 * np.linalg.norm(g)

    # the oracle's adjoint from the same dL/dx and the same roots
    AT = As.T.tocsr()
    lam_o, gv_o, st_o = gmres.adjoint_grads(As, AT, R.complex(), x.detach().cpu().numpy(),
                                            g, P.m, 1e-13, P.A.rowptr, P.A.colind)
    assert st_o.converged
    assert np.linalg.norm(gb - lam_o) <= 1e-7 * np.linalg.norm(lam_o)
    assert np.linalg.norm(gv - gv_o) <= 1e-7 * np.linalg.norm(gv_o)

    def L(bb, vv):
        xx, st = p.solve(A.with_vals(vv), bb, P.m, tol, roots=R, max_cycles=400)
        assert st["converged"] == 1
        return 0.5 * torch.sum((xx - xstar) ** 2).item()

    rng = np.random.default_rng(105)
    worst = 0.0
    for _ in range(N_DIRECTIONS):
        db = rng.standard_normal(P.A.n)
        dv = rng.standard_normal(P.A.nnz)
        sc = np.sqrt(db @ db + dv @ dv)
        db, dv = db / sc * np.linalg.norm(P.b), dv / sc * np.linalg.norm(P.A.vals)
        tb, tv = to_dev(torch, db), to_dev(torch, dv)
        fd = (L(b0 + H_FD * tb, A.vals + H_FD * tv)
              - L(b0 - H_FD * tb, A.vals - H_FD * tv)) / (2 * H_FD)
        an = gb @ db + gv @ dv
        rel = abs(fd - an) / max(abs(an), 1e-300)
        worst = max(worst, rel)
        assert rel <= 1e-5, (fd, an, rel)
    print("adjoint 512^2: %d directions, worst relative FD gap %.2e, tol %.1e"
          % (N_DIRECTIONS, worst, tol))
