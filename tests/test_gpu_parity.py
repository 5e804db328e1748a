"""GPU-vs-oracle parity through the C ABI (run with -m gpu).

Systems of at most 32,768 rows run the direct root-step kernel (one row per
thread, no staging); larger ones the staged, tiled kernel.  The matrices
below cover both: small stencils and a random matrix with long and empty
rows, and stencils and a random matrix of 36,100-40,001 rows (ragged last
tiles; the random one with rows longer than a staging chunk, and in FP32
most of its 512-row tiles in several chunks).

Tolerances (FP64): SpMV within 1e-15 of the row's absolute sum; p(A) v and
phi(A) v within 1e-11 ||p(A)||_2 ||v|| in norm and per element; Hbar within
1e-10 relative; roots within 1e-10 max(1, kappa_i); solve: true residual
<= tol and iteration count within 2 of the oracle.  FP32 (precision form):
the device's float32 Algorithm 3 is as accurate as the oracle's float32 run
(error against FP64 at most 3x the oracle's, difference at most 4x), and
within 1e-5 ||p(A)||_2 ||v|| of it on the small cases.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import gmres, poly

from gpu_util import dev_csr, p_norm_estimate, ppg_or_skip, random_csr, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return ppg_or_skip()


ROOT_SETS = {
    "real": np.array([2.5, 3.1, 4.0, 2.2, 3.7, 5.5], dtype=complex),
    "ends_in_pair": np.array([4.0, 3 + 1j, 3 - 1j, 2.5, 2 + 0.5j, 2 - 0.5j]),
    "pair_then_real": np.array([3 + 1j, 3 - 1j, 2.5, 2 + 0.5j, 2 - 0.5j, 3.3]),
    "pair_pair_real": np.array([3 + 1j, 3 - 1j, 2 + 0.5j, 2 - 0.5j, 3.3]),
    "single_real": np.array([3.0 + 0j]),
    "single_pair": np.array([3 + 1j, 3 - 1j]),
    "real_real": np.array([3.0, 4.5], dtype=complex),
    "repeated": np.array([3.0, 2.0, 3.0, 3 + 1j, 3 - 1j, 3 + 1j, 3 - 1j], dtype=complex),
}


def _matrices():
    yield "cd2d_37", synth.cd2d(37, 0.7)            # n = 1369, ragged tail
    yield "cd3d_13", synth.cd3d(13, (0.8, 0.4, 0.2))  # n = 2197, 7-point
    yield "random_long_empty", random_csr(3001, 1, long_rows={5: 2500, 700: 4100},
                                          empty_rows={17, 1000, 3000})


def _large_matrices():
    # staged kernel: 36100 = 141 * 256 + 4 rows, 39304 = 76 * 512 + 392
    yield "cd2d_190", synth.cd2d(190, 0.7)
    yield "cd3d_34", synth.cd3d(34, (0.8, 0.4, 0.2))


def _large_random():
    return random_csr(40001, 3, long_rows={5: 2500, 700: 4100, 33000: 9000},
                      empty_rows={17, 1000, 40000})


@pytest.mark.parametrize("mname,A", list(_matrices()) + list(_large_matrices())
                         + [("random_long_empty_40k", _large_random())])
def test_spmv_matches_oracle(env, mname, A):
    p, torch = env
    As = A.to_scipy()
    x = np.random.default_rng(3).standard_normal(A.n)
    y = p.spmv(dev_csr(p, torch, A), to_dev(torch, x)).cpu().numpy()
    ref = As @ x
    scale = abs(As) @ np.abs(x) + 1e-300
    assert np.all(np.abs(y - ref) <= 1e-15 * scale * 8)


def _scaled_err(y, ref, pnorm, v):
    scale = pnorm * np.linalg.norm(v)
    return np.linalg.norm(y - ref) / scale, np.max(np.abs(y - ref)) / scale


@pytest.mark.parametrize("rname", list(ROOT_SETS))
@pytest.mark.parametrize("mname,A", list(_matrices())[:2] + list(_large_matrices()))
def test_apply_p_and_phi_fp64_match_oracle(env, rname, mname, A):
    p, torch = env
    roots = ROOT_SETS[rname]
    As = A.to_scipy()
    Ad = dev_csr(p, torch, A)
    R = p.Roots.from_complex(roots)
    v = np.random.default_rng(4).standard_normal(A.n)
    yp = p.apply_poly(Ad, R, to_dev(torch, v)).cpu().numpy()
    yf = p.apply_phi(Ad, R, to_dev(torch, v)).cpu().numpy()
    rp = poly.apply_p(As, roots, v)
    rf = poly.apply_phi(As, roots, v)
    ATs = As.T.tocsr()
    pn = p_norm_estimate(lambda u: poly.apply_p(As, roots, u),
                         lambda u: poly.apply_p(ATs, roots, u), A.n)
    e2, einf = _scaled_err(yp, rp, pn, v)
    assert e2 <= 1e-11 and einf <= 1e-11
    phin = p_norm_estimate(lambda u: poly.apply_phi(As, roots, u),
                           lambda u: poly.apply_phi(ATs, roots, u), A.n)
    e2, einf = _scaled_err(yf, rf, phin, v)
    assert e2 <= 1e-11 and einf <= 1e-11


@pytest.mark.parametrize("side", [13, 34])
@pytest.mark.parametrize("rname", ["real", "ends_in_pair", "pair_then_real", "single_real"])
def test_apply_p_fp32_matches_float32_oracle(env, rname, side):
    p, torch = env
    roots = ROOT_SETS[rname]
    A = synth.cd3d(side, (0.8, 0.4, 0.2))
    As32 = A.to_scipy().astype(np.float32)
    Ad = dev_csr(p, torch, A, dtype=torch.float32)
    R = p.Roots.from_complex(roots)
    v = np.random.default_rng(5).standard_normal(A.n).astype(np.float32)
    y = p.apply_poly(Ad, R, to_dev(torch, v, torch.float32)).cpu().numpy().astype(np.float64)
    ref = gmres.apply_p32(As32, gmres._roots32(roots), v).astype(np.float64)
    As = A.to_scipy()
    ref64 = poly.apply_p(As, roots, v.astype(np.float64))
    e_orc = np.linalg.norm(ref - ref64)
    assert np.linalg.norm(y - ref64) <= 3.0 * e_orc
    assert np.linalg.norm(y - ref) <= 4.0 * e_orc
    pn = p_norm_estimate(lambda u: poly.apply_p(As, roots, u),
                         lambda u: poly.apply_p(As.T.tocsr(), roots, u), A.n)
    e2, einf = _scaled_err(y, ref, pn, v.astype(np.float64))
    assert e2 <= 1e-5 and einf <= 1e-5


@pytest.mark.parametrize("n", [3001, 40001])
def test_apply_on_matrix_with_long_and_empty_rows(env, n):
    p, torch = env
    if n == 3001:
        A = random_csr(3001, 2, long_rows={5: 2500, 700: 4100}, empty_rows={17, 1000, 3000})
    else:
        A = _large_random()
    As = A.to_scipy()
    roots = ROOT_SETS["ends_in_pair"] * 2.0
    R = p.Roots.from_complex(roots)
    v = np.random.default_rng(6).standard_normal(A.n)
    y = p.apply_poly(dev_csr(p, torch, A), R, to_dev(torch, v))
    ref = poly.apply_p(As, roots, v)
    assert np.linalg.norm(y.cpu().numpy() - ref) <= 1e-11 * np.linalg.norm(ref) * 10
    yf = p.apply_phi(dev_csr(p, torch, A), R, to_dev(torch, v))
    reff = poly.apply_phi(As, roots, v)
    assert np.linalg.norm(yf.cpu().numpy() - reff) <= 1e-11 * np.linalg.norm(reff) * 10
    # FP32: as accurate as the oracle's float32 Algorithm 3 on the same data
    As32 = As.astype(np.float32)
    v32 = v.astype(np.float32)
    y32 = p.apply_poly(dev_csr(p, torch, A, dtype=torch.float32), R,
                       to_dev(torch, v32, torch.float32)).cpu().numpy().astype(np.float64)
    r32 = gmres.apply_p32(As32, gmres._roots32(roots), v32).astype(np.float64)
    r64 = poly.apply_p(As, roots, v32.astype(np.float64))
    e_orc = np.linalg.norm(r32 - r64)
    assert np.linalg.norm(y32 - r64) <= 3.0 * e_orc
    assert np.linalg.norm(y32 - r32) <= 4.0 * e_orc


def test_build_poly_matches_oracle_hbar_and_roots(env):
    p, torch = env
    P = synth.problem("cd2d_50")
    As = P.A.to_scipy()
    Ad = dev_csr(p, torch, P.A)
    R, H = p.build_poly(Ad, P.d, to_dev(torch, P.v0), return_hbar=True)
    orc = poly.build_poly(As, P.d, P.v0)
    assert np.linalg.norm(H - orc.Hbar) <= 1e-10 * np.linalg.norm(orc.Hbar)
    assert R.n_orig == P.d and R.n_added == orc.n_added
    got = R.complex()
    from scipy.optimize import linear_sum_assignment
    C = np.abs(got[:, None] - orc.roots[None, :])
    r, c = linear_sum_assignment(C)
    assert np.max(C[r, c] / np.abs(orc.roots[c])) <= 1e-10
    # the library's roots from the SAME Hbar agree to 1e-12
    R2 = p.roots_from_hessenberg(orc.Hbar)
    C = np.abs(R2.complex()[:, None] - orc.roots[None, :])
    r, c = linear_sum_assignment(C)
    assert np.max(C[r, c] / np.abs(orc.roots[c])) <= 1e-12


def test_build_poly_residual_identity(env):
    """||pi(A) v0|| / ||v0|| equals the GMRES(d) residual: the last |g| of a
    d-step GMRES from v0 (Section 2)."""
    p, torch = env
    P = synth.problem("cd2d_50")
    Ad = dev_csr(p, torch, P.A)
    R = p.build_poly(Ad, P.d, to_dev(torch, P.v0), stability_control=False)
    v0 = to_dev(torch, P.v0)
    phi = p.apply_phi(Ad, R, v0)
    pi_norm = torch.linalg.norm(v0 - phi).item() / torch.linalg.norm(v0).item()
    _, st = gmres.pp_gmres(P.A.to_scipy(), None, P.v0, P.d, 1e-30, max_cycles=1)
    assert abs(pi_norm - st.history[P.d - 1]) <= 1e-9 * st.history[P.d - 1] + 1e-14


def test_build_poly_breakdown_is_reported(env):
    p, torch = env
    A = synth.diag_csr(np.arange(1.0, 301.0))
    v0 = np.zeros(300)
    v0[:4] = 1.0
    Ad = dev_csr(p, torch, A)
    import ctypes as C
    from paper_1911_07065_gb300._binding import default_opts, lib
    r = p.Roots(64)
    H = np.zeros(11 * 10)
    rc = lib.ppg_build_poly(Ad.ref(), 10, C.c_void_p(to_dev(torch, v0).data_ptr()),
                            C.byref(default_opts()), r.ref(),
                            H.ctypes.data_as(C.POINTER(C.c_double)),
                            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 2   # PPG_LUCKY_BREAKDOWN
    assert r.n_orig == 4
    assert np.allclose(np.sort(r.complex().real[:4]), [1, 2, 3, 4], rtol=1e-10)


def _oracle_solve(P, roots):
    return gmres.pp_gmres(P.A.to_scipy(), roots, P.b, P.m, P.tol)


def test_solve_config_cd2d_50(env):
    """PP(10)-GMRES(50) on 50 x 50 convection-diffusion, tol 1e-8."""
    p, torch = env
    P = synth.problem("cd2d_50")
    As = P.A.to_scipy()
    Ad = dev_csr(p, torch, P.A)
    orc = poly.build_poly(As, P.d, P.v0)
    R = p.Roots.from_complex(orc.roots)
    x, st = p.solve(Ad, to_dev(torch, P.b), P.m, P.tol, roots=R)
    xo, so = _oracle_solve(P, orc.roots)
    xh = x.cpu().numpy()
    rel = np.linalg.norm(P.b - As @ xh) / np.linalg.norm(P.b)
    assert st["converged"] == 1 and rel <= P.tol
    assert abs(st["iters"] - so.iters) <= 2
    assert st["mvps"] == so.mvps or abs(st["iters"] - so.iters) > 0
    assert np.linalg.norm(xh - xo) <= 1e-6 * np.linalg.norm(xo)


@pytest.mark.parametrize("beta_h,d", [(3.0, 12), (0.0, 16)])
def test_solve_with_complex_roots_and_added_roots(env, beta_h, d):
    """beta*h = 3 gives a complex spectrum (conjugate-pair kernels);
    beta*h = 0 (Laplacian) at d = 16 stresses the real chain."""
    p, torch = env
    A = synth.cd2d(48, beta_h)
    As = A.to_scipy()
    rs = synth.streams(11)
    b = synth.uniform_rhs(rs[1], A.n)
    v0 = synth.gaussian_v0(rs[0], A.n)
    Ad = dev_csr(p, torch, A)
    R = p.build_poly(Ad, d, to_dev(torch, v0))
    orc = poly.build_poly(As, d, v0)
    if beta_h > 0:
        assert np.any(orc.roots.imag != 0)
    x, st = p.solve(Ad, to_dev(torch, b), 40, 1e-10, roots=R)
    _, so = gmres.pp_gmres(As, orc.roots, b, 40, 1e-10)
    rel = np.linalg.norm(b - As @ x.cpu().numpy()) / np.linalg.norm(b)
    assert st["converged"] == 1 and rel <= 1e-10
    assert abs(st["iters"] - so.iters) <= 2


def test_plain_gmres_matches_oracle(env):
    p, torch = env
    P = synth.problem("cd2d_50", scale=30)
    As = P.A.to_scipy()
    x, st = p.solve(dev_csr(p, torch, P.A), to_dev(torch, P.b), 30, 1e-9)
    _, so = gmres.pp_gmres(As, None, P.b, 30, 1e-9)
    rel = np.linalg.norm(P.b - As @ x.cpu().numpy()) / np.linalg.norm(P.b)
    assert st["converged"] == 1 and rel <= 1e-9
    assert abs(st["iters"] - so.iters) <= 2


def test_solve_flex_fp32_inner_reaches_1e10(env):
    p, torch = env
    P = synth.problem("cd3d_160", scale=20)
    As = P.A.to_scipy()
    A64 = dev_csr(p, torch, P.A)
    A32 = A64.astype(torch.float32)
    R = p.build_poly(A64, 20, to_dev(torch, P.v0))
    x, st = p.solve_flex(A64, A32, to_dev(torch, P.b), R, 50, 1e-10)
    xh = x.cpu().numpy()
    rel = np.linalg.norm(P.b - As @ xh) / np.linalg.norm(P.b)
    assert st["converged"] == 1 and rel <= 1e-10
    _, so = gmres.fgmres_p(As, R.complex(), P.b, 50, 1e-10, inner="f32")
    assert abs(st["iters"] - so.iters) <= 2


def test_stability_check_matches_oracle(env):
    """StCh (Section 3.5) on a 20 x 20 convection-diffusion matrix with one
    outlying diagonal entry: without root adding the degree-40 polynomial is
    unstable (StCh huge on both sides), with it StCh is at rounding level.
    StCh measures rounding, so only its magnitude class is compared.  (On a
    diagonal matrix the fused multiply-add can cancel the outlier's
    component exactly, which makes the unstable case look stable: a
    non-diagonal matrix avoids that.)"""
    p, torch = env
    A = synth.cd2d(20, 0.5)
    k = A.rowptr[137] + 2
    assert A.colind[k] == 137
    A.vals[k] = 1e4
    As = A.to_scipy()
    v0 = np.random.default_rng(1).standard_normal(A.n)
    bb = np.random.default_rng(2).standard_normal(A.n)
    bb /= np.linalg.norm(bb)
    Ad = dev_csr(p, torch, A)
    for stab in (False, True):
        orc = poly.build_poly(As, 40, v0, stability=stab)
        s_orc = gmres.stability_check(As, orc.roots, bb)
        s_gpu = p.stability_check(Ad, p.Roots.from_complex(orc.roots), to_dev(torch, bb))
        if stab:
            assert s_orc < 1e-10 and s_gpu < 1e-10
        else:
            assert s_orc > 1e-4 and s_gpu > 1e-4


def test_build_poly_checked_lowers_the_degree_like_the_oracle(env):
    """Section 3.5 inside the construction: on the outlier matrix without
    root adding, StCh rejects degrees 40, 20 and 10 and keeps 5 on both sides;
    the kept roots match the oracle's within 1e-10; with root adding the
    degree-40 polynomial passes at once; and StCh values agree with the
    oracle's within a relative factor where StCh sums many rounding errors
    (StCh measures rounding, which the two sides do in different orders)."""
    p, torch = env
    A = synth.cd2d(20, 0.5)
    k = A.rowptr[137] + 2
    assert A.colind[k] == 137
    A.vals[k] = 1e4
    As = A.to_scipy()
    v0 = np.random.default_rng(1).standard_normal(A.n)
    bb = np.random.default_rng(2).standard_normal(A.n)
    Ad = dev_csr(p, torch, A)
    tol = 1e-10
    orc, tried = gmres.build_poly_checked(As, 40, v0, bb, tol, d_min=2, stability=False)
    R, info = p.build_poly_checked(Ad, 40, to_dev(torch, v0), tol, b=to_dev(torch, bb),
                                   d_min=2, stability_control=False)
    assert info["d_requested"] == 40
    assert info["n_tried"] == len(tried) == 4
    assert info["d_chosen"] == orc.d == 5 == R.n_orig
    assert info["stch"] <= tol
    # first degree: hugely unstable on both sides; kept degree: rounding level
    assert tried[0][1] > 1e6 and info["stch_first"] > 1e6
    assert tried[-1][1] <= 1e-12 and info["stch"] <= 1e-12
    # StCh values within a relative factor, the same roots on both sides so
    # that only the rounding of Algorithms 1 and 3 differs.  Chosen where
    # StCh sums many rounding errors (a relative rescaling of b by 2^-30
    # moves the oracle's own value by at most a factor 3 here); on the 1e4
    # outlier StCh is a single ulp of a huge cancelled component (a power of
    # two that the fused multiply-add may cancel outright), so only its
    # class is compared above.
    cases = []
    A2 = synth.cd2d(20, 0.5)
    A2.vals[A2.rowptr[137] + 2] = 20.0          # moderately unstable: StCh ~ 1e-8
    cases.append((A2, 15, 30.0))
    cases.append((synth.cd2d(30, 0.5), 60, 10.0))   # stable: StCh ~ 1e-13
    for Ac, deg, factor in cases:
        Acs = Ac.to_scipy()
        v0c = np.random.default_rng(1).standard_normal(Ac.n)
        uc = np.random.default_rng(2).standard_normal(Ac.n)
        uc /= np.linalg.norm(uc)
        roots = poly.build_poly(Acs, deg, v0c, stability=False).roots
        s_orc = gmres.stability_check(Acs, roots, uc)
        s_dev = p.stability_check(dev_csr(p, torch, Ac), p.Roots.from_complex(roots),
                                  to_dev(torch, uc))
        assert s_orc > 1e-15 and s_dev > 0.0
        assert abs(np.log10(s_dev / s_orc)) <= np.log10(factor), (deg, s_dev, s_orc)
    got = R.complex()
    assert got.size == orc.roots.size
    assert np.max(np.abs(np.sort_complex(got) - np.sort_complex(orc.roots))) <= \
        1e-10 * np.max(np.abs(orc.roots))
    # the lowered polynomial is the one ppg_build_poly gives at that degree
    R5 = p.build_poly(Ad, 5, to_dev(torch, v0), stability_control=False)
    assert np.array_equal(R5.complex(), got)
    # with Algorithm 2's added roots the requested degree passes
    R40, info40 = p.build_poly_checked(Ad, 40, to_dev(torch, v0), tol, b=to_dev(torch, bb))
    assert info40["n_tried"] == 1 and info40["d_chosen"] == 40 and R40.n_added >= 1
    assert info40["stch"] <= tol


def test_transpose_and_adjoint_gradient(env):
    p, torch = env
    N = 24
    fld = synth.smooth_field(N, synth.streams(105)[2])
    A = synth.cd2d(N, 1.0 + 0.5 * fld)
    Ad = dev_csr(p, torch, A)
    T, perm = Ad.transpose(with_perm=True)
    ATs = A.to_scipy().T.tocsr()
    ATs.sort_indices()
    assert np.array_equal(T.rowptr.cpu().numpy(), ATs.indptr)
    assert np.array_equal(T.colind.cpu().numpy(), ATs.indices)
    assert np.array_equal(T.vals.cpu().numpy(), ATs.data)
    assert np.array_equal(A.vals[perm.cpu().numpy()], ATs.data)
    rng = np.random.default_rng(7)
    b = rng.uniform(-1, 1, A.n)
    xstar = rng.standard_normal(A.n)
    R = p.build_poly(Ad, 8, to_dev(torch, rng.standard_normal(A.n)))
    bt = to_dev(torch, b).requires_grad_(True)
    vt = Ad.vals.clone().requires_grad_(True)
    x = p.PPGMRESFunction.apply(bt, vt, Ad, R, 40, 1e-13, None)
    loss = 0.5 * torch.sum((x - to_dev(torch, xstar)) ** 2)
    loss.backward()
    Ads = A.dense()
    xe = np.linalg.solve(Ads, b)
    lam = np.linalg.solve(Ads.T, xe - xstar)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    gv = -lam[rows] * xe[A.colind]
    assert np.linalg.norm(bt.grad.cpu().numpy() - lam) <= 1e-9 * np.linalg.norm(lam)
    assert np.linalg.norm(vt.grad.cpu().numpy() - gv) <= 1e-9 * np.linalg.norm(gv)


def test_error_paths_are_reported_not_crashed(env):
    p, torch = env
    A = synth.cd2d(10, 0.3)
    Ad = dev_csr(p, torch, A)
    v = to_dev(torch, np.ones(A.n))
    bad = p.Roots.from_complex(np.array([1 + 1j, 2 - 1j]))   # not conjugates
    with pytest.raises(p.PPGError) as ei:
        p.apply_poly(Ad, bad, v)
    assert ei.value.code == -1
    with pytest.raises(p.PPGError):
        p.apply_poly(Ad, p.Roots.from_complex(np.array([0.0 + 0j])), v)
    with pytest.raises(p.PPGError):
        p.solve(Ad, v, 0, 1e-8)
    with pytest.raises(p.PPGError) as ei:
        p.solve(Ad, v, 10, 1e-8, out=v)          # b aliases x
    nanb = v.clone()
    nanb[3] = float("nan")
    with pytest.raises(p.PPGError) as ei:
        p.solve(Ad, nanb, 10, 1e-8)
    assert ei.value.code == -4
    x, st = p.solve(Ad, torch.zeros_like(v), 10, 1e-8)
    assert st["converged"] == 1 and torch.all(x == 0)
    x, st = p.solve(Ad, v, 5, 1e-14, max_cycles=2)
    assert st["status"] == 1 and st["cycles"] == 2   # PPG_NOT_CONVERGED
