"""Differentiation form at its full size (run with -m gpu): 2-D
convection-diffusion 512 x 512 with a per-node convection field, loss
L = 1/2 ||x - x*||^2.  The adjoint gradient (A^T solve with the same roots)
is checked against central finite differences of device solves on seeded
random directions, and lambda against the host: A^T lambda = dL/dx.

The solves run to relative residual 1e-12 (the attainable level here is
about 1e-13); with h = 1e-6 on directions scaled to ||b|| and ||vals|| the
difference quotient carries a relative error of order 1e-6 from the solves
and 1e-8 from truncation, so 1e-4 is the acceptance bound."""
import numpy as np
import pytest

import synth

from gpu_util import dev_csr, ppg_or_skip, to_dev

pytestmark = pytest.mark.gpu


def test_adjoint_512_against_central_differences():
    p, torch = ppg_or_skip()
    P = synth.problem("cd2d_field_512")
    A = dev_csr(p, torch, P.A)
    R = p.build_poly(A, P.d, to_dev(torch, P.v0))
    xstar = to_dev(torch, P.extra["xstar"])
    b0 = to_dev(torch, P.b)
    bt = b0.clone().requires_grad_(True)
    vt = A.vals.clone().requires_grad_(True)
    x = p.PPGMRESFunction.apply(bt, vt, A, R, P.m, 1e-12, None, 200)
    loss = 0.5 * torch.sum((x - xstar) ** 2)
    loss.backward()
    gb = bt.grad.cpu().numpy()
    gv = vt.grad.cpu().numpy()
    # lambda = dL/db solves A^T lambda = x - x*
    As = P.A.to_scipy()
    g = (x - xstar).detach().cpu().numpy()
    assert np.linalg.norm(As.T @ gb - g) <= 1e-10 * np.linalg.norm(g)

    def L(bb, vv):
        xx, st = p.solve(A.with_vals(vv), bb, P.m, 1e-12, roots=R, max_cycles=200)
        assert st["converged"] == 1
        return 0.5 * torch.sum((xx - xstar) ** 2).item()

    rng = np.random.default_rng(105)
    h = 1e-6
    for _ in range(6):
        db = rng.standard_normal(P.A.n)
        dv = rng.standard_normal(P.A.nnz)
        sc = np.sqrt(db @ db + dv @ dv)
        db, dv = db / sc * np.linalg.norm(P.b), dv / sc * np.linalg.norm(P.A.vals)
        tb, tv = to_dev(torch, db), to_dev(torch, dv)
        fd = (L(b0 + h * tb, A.vals + h * tv) - L(b0 - h * tb, A.vals - h * tv)) / (2 * h)
        an = gb @ db + gv @ dv
        assert abs(fd - an) <= 1e-4 * max(abs(an), 1e-12), (fd, an)
