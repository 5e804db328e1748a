"""Iteration-count parity on reduced versions of the benchmark workloads (run
with -m gpu): the same seeds and generator recipes, smaller grid sides, so
that the oracle runs the whole solve.

* 2-D convection-diffusion 200 x 200 (recipe of the 1000 x 1000 workload,
  d = 40, GMRES(50), tol 1e-10): device roots against the oracle's, then
  PP-GMRES with the device roots on both sides: iterations (+-2), cycles,
  mvps (consistent with the iteration difference), true residual, solution.
* 3-D convection-diffusion 40^3 (recipe of 160^3, d = 60, m = 50): the
  FP32-inner flexible solve against the oracle's float32-inner FGMRES, and
  the FP64 PP-GMRES against the oracle's.
* Per-node convection field 64 x 64 (recipe of the 512 x 512 adjoint
  workload, d = 30, GMRES(50)): forward and adjoint iteration counts, the
  adjoint gradients against the oracle's (lambda = A^{-T} dL/dx,
  dL/dvals = -lambda_i x_j), and central differences of device solves run
  to 1e-13 (h = 1e-6: difference-quotient noise ~1e-7 relative, accepted
  at 1e-5).
"""
import numpy as np
import pytest

import synth
from oracle import gmres, poly

from gpu_util import dev_csr, ppg_or_skip, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return ppg_or_skip()


def _roots_match(got, ref, tol):
    from scipy.optimize import linear_sum_assignment
    C = np.abs(got[:, None] - ref[None, :])
    r, c = linear_sum_assignment(C)
    return np.max(C[r, c] / np.abs(ref[c]))


def test_cd2d_200_iteration_parity(env):
    p, torch = env
    P = synth.problem("cd2d_1000", scale=200)
    As = P.A.to_scipy()
    A = dev_csr(p, torch, P.A)
    R = p.build_poly(A, P.d, to_dev(torch, P.v0))
    orc = poly.build_poly(As, P.d, P.v0)
    assert R.n_total == orc.roots.size
    assert _roots_match(R.complex(), orc.roots, 1e-8) <= 1e-8
    x, st = p.solve(A, to_dev(torch, P.b), P.m, P.tol, roots=R)
    xo, so = gmres.pp_gmres(As, R.complex(), P.b, P.m, P.tol)
    assert st["converged"] == 1 and so.converged
    assert abs(st["iters"] - so.iters) <= 2
    assert st["cycles"] == so.cycles
    assert st["mvps"] - so.mvps == (st["iters"] - so.iters) * R.n_total
    xg = x.cpu().numpy()
    rel = np.linalg.norm(P.b - As @ xg) / np.linalg.norm(P.b)
    assert rel <= P.tol
    assert abs(st["true_relres"] - rel) <= 1e-3 * rel
    assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)
    # CGS2 with its middle passes fused (one pass over the basis, the same
    # multiply-adds in another order): the same solve within the same bounds
    xf, sf = p.solve(A, to_dev(torch, P.b), P.m, P.tol, roots=R, cgs2_fused=True)
    assert sf["converged"] == 1 and abs(sf["iters"] - so.iters) <= 2
    assert sf["cycles"] == so.cycles
    xfg = xf.cpu().numpy()
    assert np.linalg.norm(P.b - As @ xfg) / np.linalg.norm(P.b) <= P.tol
    assert np.linalg.norm(xfg - xo) <= 1e-6 * np.linalg.norm(xo)


@pytest.mark.parametrize("inner", ["f32", "f64"])
def test_cd3d_40_iteration_parity(env, inner):
    p, torch = env
    P = synth.problem("cd3d_160", scale=40)
    As = P.A.to_scipy()
    A64 = dev_csr(p, torch, P.A)
    R = p.build_poly(A64, P.d, to_dev(torch, P.v0))
    if inner == "f32":
        x, st = p.solve_flex(A64, A64.astype(torch.float32), to_dev(torch, P.b), R, P.m, P.tol)
        xo, so = gmres.fgmres_p(As, R.complex(), P.b, P.m, P.tol, inner="f32")
    else:
        x, st = p.solve(A64, to_dev(torch, P.b), P.m, P.tol, roots=R)
        xo, so = gmres.pp_gmres(As, R.complex(), P.b, P.m, P.tol)
    assert st["converged"] == 1 and so.converged
    assert abs(st["iters"] - so.iters) <= 2
    xg = x.cpu().numpy()
    rel = np.linalg.norm(P.b - As @ xg) / np.linalg.norm(P.b)
    assert rel <= P.tol
    assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)


def test_field_64_adjoint_parity_and_finite_differences(env):
    p, torch = env
    P = synth.problem("cd2d_field_512", scale=64)
    As = P.A.to_scipy()
    ATs = As.T.tocsr()
    A = dev_csr(p, torch, P.A)
    R = p.build_poly(A, P.d, to_dev(torch, P.v0))
    roots = R.complex()
    xstar = P.extra["xstar"]
    tol = 1e-13
    # forward and adjoint solves, iteration counts against the oracle
    x, st = p.solve(A, to_dev(torch, P.b), P.m, tol, roots=R, max_cycles=200)
    xo, so = gmres.pp_gmres(As, roots, P.b, P.m, tol, max_cycles=200)
    assert st["converged"] == 1 and so.converged
    assert abs(st["iters"] - so.iters) <= 2
    xg = x.cpu().numpy()
    gx = xg - xstar
    AT = A.transpose()
    lam, sl = p.solve(AT, to_dev(torch, gx), P.m, tol, roots=R, max_cycles=200)
    lam_o, gv_o, sao = gmres.adjoint_grads(As, ATs, roots, xg, gx, P.m, tol,
                                           P.A.rowptr, P.A.colind, max_cycles=200)
    assert sl["converged"] == 1 and sao.converged
    assert abs(sl["iters"] - sao.iters) <= 2
    # the gradients through the autograd path
    bt = to_dev(torch, P.b).requires_grad_(True)
    vt = A.vals.clone().requires_grad_(True)
    xa = p.PPGMRESFunction.apply(bt, vt, A, R, P.m, tol, AT, 200)
    loss = 0.5 * torch.sum((xa - to_dev(torch, xstar)) ** 2)
    loss.backward()
    gb = bt.grad.cpu().numpy()
    gv = vt.grad.cpu().numpy()
    assert np.linalg.norm(gb - lam_o) <= 1e-8 * np.linalg.norm(lam_o)
    assert np.linalg.norm(gv - gv_o) <= 1e-8 * np.linalg.norm(gv_o)
    assert np.linalg.norm(gb - lam.cpu().numpy()) <= 1e-8 * np.linalg.norm(gb)

    def L(bb, vv):
        xx, s2 = p.solve(A.with_vals(vv), bb, P.m, tol, roots=R, max_cycles=200)
        assert s2["converged"] == 1
        return 0.5 * torch.sum((xx - to_dev(torch, xstar)) ** 2).item()

    rng = np.random.default_rng(105)
    h = 1e-6
    b0 = to_dev(torch, P.b)
    for _ in range(4):
        db = rng.standard_normal(P.A.n)
        dv = rng.standard_normal(P.A.nnz)
        sc = np.sqrt(db @ db + dv @ dv)
        db, dv = db / sc * np.linalg.norm(P.b), dv / sc * np.linalg.norm(P.A.vals)
        tb, tv = to_dev(torch, db), to_dev(torch, dv)
        fd = (L(b0 + h * tb, A.vals + h * tv) - L(b0 - h * tb, A.vals - h * tv)) / (2 * h)
        an = gb @ db + gv @ dv
        assert abs(fd - an) <= 1e-5 * max(abs(an), 1e-12), (fd, an)
