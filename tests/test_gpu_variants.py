"""Double polynomial preconditioning (Section 6) and the changing
polynomial (Section 5.2) through the C ABI against the oracle (run with
-m gpu).  Sizes span several row tiles with a ragged tail."""
import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

import synth
from oracle import gmres, poly

from gpu_util import dev_csr, ppg_or_skip, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return ppg_or_skip()


def _close(got, ref, tol):
    C = np.abs(got[:, None] - ref[None, :])
    r, c = linear_sum_assignment(C)
    return np.max(C[r, c] / np.abs(ref[c])) <= tol


def test_composite_construction_and_double_solve(env):
    p, torch = env
    A = synth.cd2d(37, 1.0)          # n = 1369
    As = A.to_scipy()
    rs = synth.streams(15)
    b = synth.uniform_rhs(rs[1], A.n)
    v1 = synth.gaussian_v0(rs[0], A.n)
    v2 = synth.gaussian_v0(rs[0], A.n)
    Ad = dev_csr(p, torch, A)
    R1 = p.build_poly(Ad, 6, to_dev(torch, v1))
    r1 = R1.complex()
    R2 = p.build_poly_composite(Ad, R1, 5, to_dev(torch, v2))
    orc2 = poly.build_poly(gmres.Composite(As, r1), 5, v2)
    assert R2.n_total == orc2.roots.size
    assert _close(R2.complex(), orc2.roots, 1e-9)
    x, st = p.solve_double(Ad, to_dev(torch, b), R1, R2, 30, 1e-10)
    rel = np.linalg.norm(b - As @ x.cpu().numpy()) / np.linalg.norm(b)
    assert st["converged"] == 1 and rel <= 1e-10
    xo, so = gmres.double_pp_gmres(As, r1, R2.complex(), b, 30, 1e-10)
    assert abs(st["iters"] - so.iters) <= 2
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-6 * np.linalg.norm(xo)
    # every SpMV counted: d1 per product with phi_1(A)
    assert st["mvps"] >= st["iters"] * R1.n_total * R2.n_total


def test_chpoly_matches_oracle(env):
    p, torch = env
    A = synth.cd2d(33, 0.6)          # n = 1089
    As = A.to_scipy()
    b = synth.uniform_rhs(synth.streams(16)[1], A.n)
    x, st = p.solve_chpoly(dev_csr(p, torch, A), to_dev(torch, b), 6, 20, 1e-10)
    rel = np.linalg.norm(b - As @ x.cpu().numpy()) / np.linalg.norm(b)
    assert st["converged"] == 1 and rel <= 1e-10
    _, so = gmres.chpoly_gmres(As, 6, b, 20, 1e-10)
    assert abs(st["iters"] - so.iters) <= 2
    assert st["cycles"] == so.cycles
