"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times (run with -m gpu).

* 2-D convection-diffusion 1000 x 1000 (n = 1e6): p(A) v against the oracle
  on seeded vectors with the oracle's own roots, the device-built roots
  against the oracle's, the full PP-GMRES solve checked by its true
  residual computed on the host, and the residual history of the first two
  restart cycles against the oracle's.
* 3-D convection-diffusion 160^3 (n = 4.1e6): the device-built roots against
  the oracle's (degree 60), FP32 p(A) v on three seeded vectors against the
  oracle's float32 Algorithm 3 (as accurate as it, both against FP64), and
  the FP32-inner flexible solve checked by its true residual.
* 3-D convection-diffusion 100^3 (n = 1e6): in FP64 a matrix whose chains
  hold their leading rows in L2 and stream the rest, in FP32 one held in L2
  entirely: p(A) v and phi(A) v against the oracle.
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


@pytest.fixture(scope="module")
def cd2d(env):
    p, torch = env
    P = synth.problem("cd2d_1000")
    As = P.A.to_scipy()
    orc = poly.build_poly(As, P.d, P.v0)
    return P, As, orc, dev_csr(p, torch, P.A)


def _assert_roots_match_oracle(R, orc):
    """Device-built roots against the oracle's end to end (GPU Arnoldi vs
    CPU Arnoldi): the same count, and each root within 1e-10 relative,
    relaxed by the eigenvalue condition number of the harmonic-Ritz matrix
    (computed on the oracle side)."""
    import scipy.linalg as sla
    assert R.n_total == orc.roots.size
    H = orc.Hbar
    d = H.shape[1]
    e = np.zeros(d); e[-1] = 1
    f = np.linalg.solve(H[:d, :d].T, e)
    G = H[:d, :d].copy(); G[:, -1] += H[d, d - 1] ** 2 * f
    w, vl, vr = sla.eig(G, left=True, right=True)
    kappa = 1.0 / np.abs(np.sum(vl.conj() * vr, axis=0))
    for t in R.complex():
        i = int(np.argmin(np.abs(w - t)))
        assert abs(w[i] - t) / abs(w[i]) <= 1e-10 * max(1.0, kappa[i])


def _pnorm_lower(As, roots, n, iters=3):
    """A lower bound of ||p(A)||_2 (a few power steps): using it as the
    error scale makes the check stricter, not looser."""
    ATs = As.T.tocsr()
    v = np.random.default_rng(0).standard_normal(n)
    v /= np.linalg.norm(v)
    est = 0.0
    for _ in range(iters):
        w = poly.apply_p(As, roots, v)
        est = np.linalg.norm(w)
        v = poly.apply_p(ATs, roots, w)
        v /= np.linalg.norm(v)
    return est


def test_cd2d_1000_apply_p_and_phi(env, cd2d):
    p, torch = env
    P, As, orc, Ad = cd2d
    R = p.Roots.from_complex(orc.roots)
    pn = _pnorm_lower(As, orc.roots, P.A.n)
    for seed in (1, 2):
        v = np.random.default_rng(seed).standard_normal(P.A.n)
        y = p.apply_poly(Ad, R, to_dev(torch, v)).cpu().numpy()
        ref = poly.apply_p(As, orc.roots, v)
        scale = pn * np.linalg.norm(v)
        assert np.linalg.norm(y - ref) <= 1e-11 * scale
        assert np.max(np.abs(y - ref)) <= 1e-11 * scale
    v = np.random.default_rng(3).standard_normal(P.A.n)
    y = p.apply_phi(Ad, R, to_dev(torch, v)).cpu().numpy()
    ref = poly.apply_phi(As, orc.roots, v)
    assert np.linalg.norm(y - ref) <= 1e-11 * np.linalg.norm(v) * max(1.0, np.linalg.norm(ref) / np.linalg.norm(v))


def test_cd2d_1000_roots_and_solve(env, cd2d):
    p, torch = env
    P, As, orc, Ad = cd2d
    R = p.build_poly(Ad, P.d, to_dev(torch, P.v0))
    _assert_roots_match_oracle(R, orc)
    x, st = p.solve(Ad, to_dev(torch, P.b), P.m, P.tol, roots=R)
    rel = np.linalg.norm(P.b - As @ x.cpu().numpy()) / np.linalg.norm(P.b)
    assert st["converged"] == 1 and rel <= P.tol


def test_cd2d_1000_residual_history_first_two_cycles(env, cd2d):
    """The whole 1000 x 1000 solve with the oracle's roots on both sides: the
    true residual and the shortcut estimate after the first restart cycle
    (a device solve capped at one cycle), then iterations, cycles and mvps
    of the converged solve, against the oracle's PP-GMRES."""
    p, torch = env
    P, As, orc, Ad = cd2d
    R = p.Roots.from_complex(orc.roots)
    xo, so = gmres.pp_gmres(As, orc.roots, P.b, P.m, P.tol, max_cycles=2)
    assert len(so.true_history) >= 1
    b = to_dev(torch, P.b)
    _, s1 = p.solve(Ad, b, P.m, P.tol, roots=R, max_cycles=1)
    if so.cycles > 1:
        assert s1["converged"] == 0 and s1["cycles"] == 1
        assert abs(s1["true_relres"] - so.true_history[0]) <= 1e-6 * so.true_history[0]
        assert abs(s1["est_relres"] - so.history[P.m - 1]) <= 1e-6 * so.history[P.m - 1]
    x, st = p.solve(Ad, b, P.m, P.tol, roots=R, max_cycles=2)
    assert st["converged"] == 1 and so.converged
    assert st["cycles"] == so.cycles
    assert abs(st["iters"] - so.iters) <= 2
    assert st["mvps"] - so.mvps == (st["iters"] - so.iters) * R.n_total
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)


@pytest.fixture(scope="module")
def cd3d(env):
    p, torch = env
    P = synth.problem("cd3d_160")
    orc = poly.build_poly(P.A.to_scipy(), P.d, P.v0)
    return P, orc


def test_cd3d_160_roots(env, cd3d):
    p, torch = env
    P, orc = cd3d
    R = p.build_poly(dev_csr(p, torch, P.A), P.d, to_dev(torch, P.v0))
    _assert_roots_match_oracle(R, orc)


@pytest.mark.parametrize("seed", [4, 5, 6])
def test_cd3d_160_fp32_apply_p(env, cd3d, seed):
    p, torch = env
    P, orc = cd3d
    roots = orc.roots
    A32 = dev_csr(p, torch, P.A, dtype=torch.float32)
    As32 = P.A.to_scipy().astype(np.float32)
    v = np.random.default_rng(seed).standard_normal(P.A.n).astype(np.float32)
    y = p.apply_poly(A32, p.Roots.from_complex(roots), to_dev(torch, v, torch.float32))
    y = y.cpu().numpy().astype(np.float64)
    ref = gmres.apply_p32(As32, gmres._roots32(roots), v).astype(np.float64)
    # Two float32 runs of Algorithm 3 differ by rounding order only, so the
    # device result must be about as accurate as the oracle's float32 run,
    # both measured against the FP64 oracle.
    ref64 = poly.apply_p(P.A.to_scipy(), roots, v.astype(np.float64))
    e_orc = np.linalg.norm(ref - ref64)
    e_gpu = np.linalg.norm(y - ref64)
    assert e_gpu <= 3.0 * e_orc
    assert np.linalg.norm(y - ref) <= 4.0 * e_orc
    assert e_gpu <= 1e-3 * np.linalg.norm(ref64)


def test_cd3d_160_flex_solve(env, cd3d):
    p, torch = env
    P, _ = cd3d
    A64 = dev_csr(p, torch, P.A)
    A32 = A64.astype(torch.float32)
    R = p.build_poly(A64, P.d, to_dev(torch, P.v0))
    x, st = p.solve_flex(A64, A32, to_dev(torch, P.b), R, P.m, P.tol)
    rel = np.linalg.norm(P.b - P.A.to_scipy() @ x.cpu().numpy()) / np.linalg.norm(P.b)
    assert st["converged"] == 1 and rel <= P.tol


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_cd3d_100_apply_with_leading_rows_held_in_l2(env, dtype):
    """3-D convection-diffusion 100^3 (n = 1e6, 7e6 nonzeros).  In FP64 the
    matrix and three vectors are too large for L2, so a chain streams the
    matrix and holds the nonzeros of its leading rows (about half of them)
    in an L2 set-aside; in FP32 they fit, and the whole matrix is held in L2
    (the direct-read step).  p(A) v and phi(A) v against the oracle element
    by element: FP64 within 1e-11 ||p(A)||_2 ||v||; FP32 as accurate as the
    oracle's float32 Algorithm 3 (error against FP64 at most 3x the
    oracle's)."""
    p, torch = env
    from gpu_util import p_norm_estimate
    A = synth.cd3d(100, (0.8, 0.4, 0.2))
    As = A.to_scipy()
    roots = np.array([4.0, 3 + 1j, 3 - 1j, 2.5, 2 + 0.5j, 2 - 0.5j, 3.3], dtype=complex)
    R = p.Roots.from_complex(roots)
    v = np.random.default_rng(17).standard_normal(A.n)
    if dtype == "f64":
        Ad = dev_csr(p, torch, A)
        yp = p.apply_poly(Ad, R, to_dev(torch, v)).cpu().numpy()
        yf = p.apply_phi(Ad, R, to_dev(torch, v)).cpu().numpy()
        rp = poly.apply_p(As, roots, v)
        rf = poly.apply_phi(As, roots, v)
        ATs = As.T.tocsr()
        pn = p_norm_estimate(lambda u: poly.apply_p(As, roots, u),
                             lambda u: poly.apply_p(ATs, roots, u), A.n, iters=15)
        phin = p_norm_estimate(lambda u: poly.apply_phi(As, roots, u),
                               lambda u: poly.apply_phi(ATs, roots, u), A.n, iters=15)
        nv = np.linalg.norm(v)
        assert np.max(np.abs(yp - rp)) <= 1e-11 * pn * nv
        assert np.linalg.norm(yp - rp) <= 1e-11 * pn * nv
        assert np.max(np.abs(yf - rf)) <= 1e-11 * phin * nv
        assert np.linalg.norm(yf - rf) <= 1e-11 * phin * nv
    else:
        Ad = dev_csr(p, torch, A, dtype=torch.float32)
        v32 = v.astype(np.float32)
        y = p.apply_poly(Ad, R, to_dev(torch, v32, torch.float32)).cpu().numpy().astype(np.float64)
        r32 = gmres.apply_p32(As.astype(np.float32), gmres._roots32(roots), v32).astype(np.float64)
        r64 = poly.apply_p(As, roots, v32.astype(np.float64))
        e_orc = np.linalg.norm(r32 - r64)
        assert np.linalg.norm(y - r64) <= 3.0 * e_orc
        assert np.linalg.norm(y - r32) <= 4.0 * e_orc
