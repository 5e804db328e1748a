"""Pins for the oracle's restarted GMRES, the FP32-inner flexible form, the
stability check and the adjoint."""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import gmres, poly

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _paper_numbers():
    out = {}
    for line in open(os.path.join(GOLDEN, "paper_numbers.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def _krylov_min_residual(Op, r0, j):
    """min ||r0 - Op K c|| over c, K = [r0, Op r0, ..., Op^{j-1} r0], by
    brute-force least squares on the explicit (normalised) Krylov basis."""
    n = r0.shape[0]
    K = np.empty((n, j))
    K[:, 0] = r0 / np.linalg.norm(r0)
    for i in range(1, j):
        K[:, i] = Op @ K[:, i - 1]
        K[:, i] /= np.linalg.norm(K[:, i])
    M = Op @ K
    c, *_ = np.linalg.lstsq(M, r0, rcond=None)
    return np.linalg.norm(r0 - M @ c)


def test_first_cycle_residuals_equal_krylov_least_squares_plain():
    P = synth.problem("cd2d_50", scale=8)
    A = P.A.dense()
    b = P.b
    _, st = gmres.pp_gmres(P.A.to_scipy(), None, b, m=8, tol=1e-30, max_cycles=1)
    for j in range(1, 8):
        ref = _krylov_min_residual(A, b, j) / np.linalg.norm(b)
        assert abs(st.history[j - 1] - ref) <= 1e-9 * max(ref, 1e-3)


def test_first_cycle_residuals_equal_krylov_least_squares_pp():
    """GMRES on phi(A): the shortcut residuals equal the Krylov least-squares
    minimum for the dense operator I - prod(I - A/theta_i)."""
    P = synth.problem("cd2d_50", scale=8)
    As = P.A.to_scipy()
    pp = poly.build_poly(As, 5, P.v0)
    n = P.A.n
    Pi = np.eye(n, dtype=complex)
    for t in pp.roots:
        Pi = Pi @ (np.eye(n) - P.A.dense() / t)
    Phi = np.eye(n) - Pi.real
    _, st = gmres.pp_gmres(As, pp.roots, P.b, m=6, tol=1e-30, max_cycles=1)
    for j in range(1, 6):
        ref = _krylov_min_residual(Phi, P.b, j) / np.linalg.norm(P.b)
        assert abs(st.history[j - 1] - ref) <= 1e-8 * max(ref, 1e-3)


def test_pp_gmres_converges_to_the_exact_solution():
    P = synth.problem("cd2d_50")
    As = P.A.to_scipy()
    pp = poly.build_poly(As, P.d, P.v0)
    x, st = gmres.pp_gmres(As, pp.roots, P.b, P.m, P.tol)
    assert st.converged
    r = P.b - As @ x
    assert np.linalg.norm(r) / np.linalg.norm(P.b) <= P.tol
    xe = spla.spsolve(As.tocsc(), P.b)
    assert np.linalg.norm(x - xe) / np.linalg.norm(xe) < 1e-5
    # mvps accounting: d per phi, d-1 per p, 1 per true residual
    d = pp.roots.size
    assert st.mvps == st.iters * d + st.cycles * (d - 1) + st.cycles


def test_degree_one_is_plain_gmres():
    """d = 1: phi(A) = A/theta_1, and GMRES is invariant to scaling the
    operator, so the residual history equals plain GMRES (Section 3.2)."""
    P = synth.problem("cd2d_50", scale=20)
    As = P.A.to_scipy()
    pp = poly.build_poly(As, 1, P.v0)
    assert pp.roots.size == 1 and pp.roots[0].imag == 0
    _, s1 = gmres.pp_gmres(As, pp.roots, P.b, 20, 1e-8)
    _, s0 = gmres.pp_gmres(As, None, P.b, 20, 1e-8)
    assert s1.iters == s0.iters
    k = min(len(s1.history), 40)
    assert np.allclose(s1.history[:k], s0.history[:k], rtol=1e-6)


def test_fgmres_with_fp64_inner_equals_pp_gmres():
    """With a fixed preconditioner, flexible GMRES builds the same iterates
    as right-preconditioned GMRES."""
    P = synth.problem("cd2d_50", scale=30)
    As = P.A.to_scipy()
    pp = poly.build_poly(As, 8, P.v0)
    _, s1 = gmres.fgmres_p(As, pp.roots, P.b, 20, 1e-10, inner="f64")
    _, s0 = gmres.pp_gmres(As, pp.roots, P.b, 20, 1e-10)
    k = min(len(s0.history), len(s1.history), 15)
    assert np.allclose(s1.history[:k], s0.history[:k], rtol=1e-6)


def test_fgmres_fp32_inner_reaches_fp64_accuracy():
    P = synth.problem("cd3d_160", scale=12)
    As = P.A.to_scipy()
    pp = poly.build_poly(As, 12, P.v0)
    x, st = gmres.fgmres_p(As, pp.roots, P.b, 30, 1e-10, inner="f32")
    assert st.converged and st.true_relres <= 1e-10
    # the float32 inner product really ran in float32
    r32 = gmres._roots32(pp.roots)
    z32 = gmres.apply_p32(As.astype(np.float32), r32, P.b)
    z64 = poly.apply_p(As, pp.roots, P.b)
    rel = np.linalg.norm(z32 - z64) / np.linalg.norm(z64)
    assert 1e-9 < rel < 1e-3


def test_stability_check_small_for_stable_and_large_for_unstable():
    """Section 3.5: StCh is at rounding level for a tame polynomial and
    large for a high-degree one without root adding on a matrix with an
    outlying eigenvalue."""
    P = synth.problem("cd2d_50")
    As = P.A.to_scipy()
    pp = poly.build_poly(As, P.d, P.v0)
    b = P.b / np.linalg.norm(P.b)
    assert gmres.stability_check(As, pp.roots, b) < 1e-12
    lam = np.concatenate([np.linspace(1.0, 2.0, 400), [1e4]])
    Ad = synth.diag_csr(lam).to_scipy()
    v0 = np.random.default_rng(1).standard_normal(401)
    bad = poly.build_poly(Ad, 40, v0, stability=False)
    good = poly.build_poly(Ad, 40, v0, stability=True)
    bb = np.random.default_rng(2).standard_normal(401)
    bb /= np.linalg.norm(bb)
    assert good.n_added >= 1
    s_bad = gmres.stability_check(Ad, bad.roots, bb)
    s_good = gmres.stability_check(Ad, good.roots, bb)
    assert s_good < s_bad


def _outlier_cd2d(value=1e4):
    """20 x 20 convection-diffusion with one outlying diagonal entry: the
    high-degree GMRES polynomial without root adding is unstable on it."""
    A = synth.cd2d(20, 0.5)
    k = A.rowptr[137] + 2
    assert A.colind[k] == 137
    A.vals[k] = value
    return A


def test_checked_construction_lowers_the_degree_until_stch_passes():
    """Section 3.5: the check runs once the polynomial is built and before
    the solve; the degree is lowered (halved, the reading taken) while StCh
    is above tol.  Pins: with a loose tol nothing changes; every degree it
    rejects has StCh above tol and makes PP-GMRES fail to reach tol (the
    instability is detected before the solve), the degree it keeps has StCh
    at or below tol and PP-GMRES converges with it; the kept polynomial is
    GMRES(d') from the same v0."""
    A = _outlier_cd2d()
    As = A.to_scipy()
    v0 = np.random.default_rng(1).standard_normal(A.n)
    b = np.random.default_rng(2).standard_normal(A.n)
    b /= np.linalg.norm(b)
    loose, tried = gmres.build_poly_checked(As, 40, v0, b, 1e300, stability=False)
    assert tried[0][0] == 40 and len(tried) == 1
    assert np.array_equal(loose.roots, poly.build_poly(As, 40, v0, stability=False).roots)
    tol = 1e-10
    pp, tried = gmres.build_poly_checked(As, 40, v0, b, tol, d_min=2, stability=False)
    degs = [t[0] for t in tried]
    assert degs == [40, 20, 10, 5]
    assert all(s > tol for _, s in tried[:-1]) and tried[-1][1] <= tol
    assert pp.d == 5
    assert np.array_equal(pp.roots, poly.build_poly(As, 5, v0, stability=False).roots)
    for deg, _ in tried[:-1]:
        bad = poly.build_poly(As, deg, v0, stability=False)
        _, st = gmres.pp_gmres(As, bad.roots, b, 50, tol, max_cycles=10)
        assert not st.converged
    _, st = gmres.pp_gmres(As, pp.roots, b, 50, tol, max_cycles=50)
    assert st.converged and st.true_relres <= tol
    # with root adding (Algorithm 2) the degree-40 polynomial passes at once
    good, tried = gmres.build_poly_checked(As, 40, v0, b, tol, stability=True)
    assert len(tried) == 1 and good.n_added >= 1
    # the floor stops the lowering even when StCh stays above tol
    _, tried = gmres.build_poly_checked(As, 40, v0, b, 1e-30, d_min=20, stability=False)
    assert [t[0] for t in tried] == [40, 20]


def test_adjoint_matches_dense_solve_and_finite_differences():
    N = 10
    fld = synth.smooth_field(N, synth.streams(105)[2])
    A = synth.cd2d(N, 1.0 + 0.5 * fld)
    As = A.to_scipy()
    AT = As.T.tocsr()
    rng = np.random.default_rng(3)
    b = rng.uniform(-1, 1, A.n)
    xstar = rng.standard_normal(A.n)
    pp = poly.build_poly(As, 6, rng.standard_normal(A.n))
    x, _ = gmres.pp_gmres(As, pp.roots, b, 30, 1e-13)
    gx = x - xstar
    lam, gvals, _ = gmres.adjoint_grads(As, AT, pp.roots, x, gx, 30, 1e-13,
                                        A.rowptr, A.colind)
    Ad = A.dense()
    lam_ref = np.linalg.solve(Ad.T, gx)
    assert np.linalg.norm(lam - lam_ref) <= 1e-10 * np.linalg.norm(lam_ref)
    # central differences of L = 1/2 ||x(b, vals) - x*||^2 on random directions
    def loss(bb, vv):
        M = sp.csr_matrix((vv, A.colind, A.rowptr), shape=(A.n, A.n))
        xx = spla.spsolve(M.tocsc(), bb)
        return 0.5 * np.sum((xx - xstar) ** 2)
    h = 1e-6
    for k in range(3):
        db = rng.standard_normal(A.n)
        dv = rng.standard_normal(A.nnz)
        s = math.sqrt(db @ db + dv @ dv)
        db /= s
        dv /= s
        fd = (loss(b + h * db, A.vals + h * dv) - loss(b - h * db, A.vals - h * dv)) / (2 * h)
        an = lam @ db + gvals @ dv
        assert abs(fd - an) <= 1e-5 * max(abs(an), 1e-8)


@pytest.mark.slow
def test_example5_pp50_cuts_mvps_about_threefold():
    """Table 3.6 row 1: on the 200x200 Laplacian GMRES(50) takes 3050 mvps
    and PP(50)-GMRES(50) 1051.  The random streams and the orthogonalisation
    differ from the paper's, so the pin is the ratio and the magnitude."""
    nums = _paper_numbers()
    A = synth.cd2d(200, 0.0)
    As = A.to_scipy()
    rs = synth.streams(5)
    b = rs[1].standard_normal(A.n)
    b /= np.linalg.norm(b)
    pp = poly.build_poly(As, 50, synth.gaussian_v0(rs[0], A.n))
    _, spp = gmres.pp_gmres(As, pp.roots, b, 50, 1e-8)
    _, s0 = gmres.pp_gmres(As, None, b, 50, 1e-8, max_cycles=200)
    assert spp.converged and s0.converged
    ratio_paper = nums["ex5_pp_mvps"] / nums["ex5_gmres_mvps"]
    ratio = (spp.mvps + 50) / s0.mvps     # + 50: the construction's GMRES(50)
    assert 0.5 * ratio_paper < ratio < 2.0 * ratio_paper
    assert 0.5 < s0.mvps / nums["ex5_gmres_mvps"] < 2.0


def test_estimate_4_1_doubling_the_degree_about_halves_the_mvps():
    """Estimate 4.1 (Section 4, from the Chebyshev model of a composed
    polynomial): for a real spectrum in [a, b] with 0 < a << b, PP(d)-GMRES(m)
    needs about 1/d of the matrix-vector products of GMRES(m), so doubling d
    about halves them; Example 11 / Table 4.1 (A = diag(i^2/n)) shows ratios
    a little above one half.  Orthogonalisation (dot products) falls faster
    than the mvps.  Here n = 2000 (the paper: 20,000), GMRES(50), tol 1e-10,
    d = 8, 16, 32, 64 (measured ratios about 0.58, 0.57, 0.45)."""
    n = 2000
    As = sp.diags(synth.ex11_diagonal(n)).tocsr()
    rng = np.random.default_rng(1)
    b = rng.standard_normal(n)
    b /= np.linalg.norm(b)
    v0 = rng.standard_normal(n)
    runs = []
    for d in (8, 16, 32, 64):
        roots = poly.build_poly(As, d, v0).roots
        _, st = gmres.pp_gmres(As, roots, b, 50, 1e-10, max_cycles=5000)
        assert st.converged and st.true_relres <= 1e-10
        runs.append(st)
    for lo, hi in zip(runs[:-1], runs[1:]):
        r_mvps = hi.mvps / lo.mvps
        assert 0.35 <= r_mvps <= 0.75, r_mvps
        assert hi.dots / lo.dots < r_mvps
