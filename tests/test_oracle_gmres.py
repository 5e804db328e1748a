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


def _alg3_coef64(A, coef, v):
    """Algorithm 3 in FP64 arithmetic on given coefficients (the float32
    ones, widened): with the float32 matrix and vector it isolates the
    effect of rounding the DATA to float32 from that of float32 ARITHMETIC."""
    d = len(coef)
    prod = v.copy()
    p = np.zeros_like(v)
    i = 0
    while i < d - 1:
        kind, c1, c2 = coef[i]
        c1, c2 = float(c1), float(c2)
        if kind == "r":
            p = p + c1 * prod
            prod = prod - c1 * (A @ prod)
            i += 1
        else:
            tmp = c1 * prod - A @ prod
            p = p + c2 * tmp
            if i <= d - 3:
                prod = prod - c2 * (A @ tmp)
            i += 2
    if coef[d - 1][0] == "r" and i == d - 1:
        p = p + float(coef[d - 1][1]) * prod
    return p


def _alg3_magnitudes(Aabs, coef, vabs):
    """The same recurrence on magnitudes: |A|, |coefficients|, |v|, every
    subtraction an addition.  Each intermediate of a float32 evaluation is
    bounded in magnitude by the matching quantity here."""
    d = len(coef)
    prod = vabs.copy()
    p = np.zeros_like(vabs)
    i = 0
    while i < d - 1:
        kind, c1, c2 = coef[i]
        c1, c2 = abs(float(c1)), abs(float(c2))
        if kind == "r":
            p = p + c1 * prod
            prod = prod + c1 * (Aabs @ prod)
            i += 1
        else:
            tmp = c1 * prod + Aabs @ prod
            p = p + c2 * tmp
            if i <= d - 3:
                prod = prod + c2 * (Aabs @ tmp)
            i += 2
    if coef[d - 1][0] == "r" and i == d - 1:
        p = p + abs(float(coef[d - 1][1])) * prod
    return p


def _slip(coef, k, rel):
    """coef with entry k's coefficient scaled by (1 + rel) (a planted mistake)."""
    coef = list(coef)
    kind, c1, c2 = coef[k]
    coef[k] = (kind, np.float32(float(c1) * (1 + rel)), c2) if kind == "r" else \
        (kind, c1, np.float32(float(c2) * (1 + rel)))
    return coef


def test_apply_p32_short_chains_within_the_rounding_bound():
    """Rigorous first-order bound (running error analysis) on chains of one
    to three roots, where it is tight: with the float32 data fixed, every
    rounded float32 operation adds at most u |result| (u = 2^-24) and along
    any path there are at most N = steps x (longest row + 3) roundings, so
    |z32 - z| <= gamma_N S elementwise, S from the magnitude recurrence and
    z the same data in FP64 arithmetic.  A coefficient 1e-4 off breaks it."""
    P = synth.problem("cd3d_160", scale=10)
    As = P.A.to_scipy()
    A32 = As.astype(np.float32)
    A32d = A32.astype(np.float64)
    v32 = P.b.astype(np.float32)
    u = 2.0 ** -24
    kmax = int(np.diff(As.indptr).max())
    for roots in (np.array([4.0, 6.5], dtype=complex),
                  np.array([5 + 1j, 5 - 1j, 3.0]),
                  np.array([5 + 1j, 5 - 1j]),
                  np.array([2.5, 5 + 1j, 5 - 1j, 3.0])):
        coef = gmres._roots32(roots)
        z32 = gmres.apply_p32(A32, coef, v32).astype(np.float64)
        z = _alg3_coef64(A32d, coef, v32.astype(np.float64))
        N = len(roots) * (kmax + 3) + 1
        bound = N * u / (1 - N * u) * _alg3_magnitudes(abs(A32d), coef, np.abs(v32))
        err = np.abs(z32 - z)
        assert np.all(err <= bound), float(np.max(err / bound))
        assert np.max(err) > 0.0
        bad = gmres.apply_p32(A32, _slip(coef, 0, 1e-4), v32).astype(np.float64)
        assert np.any(np.abs(bad - z) > bound)


def test_apply_p32_arithmetic_error_comparable_to_data_rounding():
    """Whole chains (degrees 6 to 30): the float32 ARITHMETIC of the oracle's
    Algorithm 3 adds an error within 10x of the error that rounding the data
    alone (matrix, coefficients, v) to float32 causes, and within 1e-6 of
    ||p(A) v|| -- so a float32 path less accurate than its data rounding
    warrants fails here (a coefficient 1e-3 off does)."""
    P = synth.problem("cd3d_160", scale=12)
    As = P.A.to_scipy()
    A32 = As.astype(np.float32)
    A32d = A32.astype(np.float64)
    v = P.b
    v32d = v.astype(np.float32).astype(np.float64)
    for deg, stab in ((6, True), (12, True), (20, False), (30, True)):
        roots = poly.build_poly(As, deg, P.v0, stability=stab).roots
        coef = gmres._roots32(roots)
        z64 = poly.apply_p(As, roots, v)
        zd = _alg3_coef64(A32d, coef, v32d)
        z32 = gmres.apply_p32(A32, coef, v).astype(np.float64)
        e_arith = np.linalg.norm(z32 - zd)
        e_data = np.linalg.norm(zd - z64)
        nz = np.linalg.norm(z64)
        assert 0.0 < e_arith <= 10.0 * e_data, (deg, e_arith / e_data)
        assert np.linalg.norm(z32 - z64) <= 1e-6 * nz
        bad = gmres.apply_p32(A32, _slip(coef, 0, 1e-3), v).astype(np.float64)
        assert np.linalg.norm(bad - zd) > 10.0 * e_data


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
