"""Pins for the oracle's double polynomial (Section 6) and changing
polynomial (Section 5.2) variants."""
import math
import os

import numpy as np
import pytest

import synth
from oracle import gmres, poly

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dense_pi(M, roots):
    n = M.shape[0]
    P = np.eye(n, dtype=complex)
    for t in roots:
        P = P @ (np.eye(n) - M / t)
    return P.real


def _small():
    A = synth.cd2d(6, 0.8)          # n = 36
    rng = np.random.default_rng(3)
    r1 = poly.build_poly(A.to_scipy(), 4, rng.standard_normal(36)).roots
    M = gmres.Composite(A.to_scipy(), r1)
    r2 = poly.build_poly(M, 4, rng.standard_normal(36)).roots
    return A, r1, r2


def test_composite_operator_is_phi1_of_A():
    A, r1, r2 = _small()
    Ad = A.dense()
    Phi1 = np.eye(36) - _dense_pi(Ad, r1)
    v = np.random.default_rng(4).standard_normal(36)
    M = gmres.Composite(A.to_scipy(), r1)
    assert np.allclose(M @ v, Phi1 @ v, rtol=1e-12, atol=1e-12)
    # phi_2(phi_1(A)) v by Algorithm 1 on M equals the dense composition
    Phi2 = np.eye(36) - _dense_pi(Phi1, r2)
    assert np.allclose(poly.apply_phi(M, r2, v), Phi2 @ v, rtol=1e-10, atol=1e-11)


def test_double_solution_identity():
    """A p_1(A) p_2(phi_1(A)) = phi_2(phi_1(A)): so x = p_1(A) p_2(M) z solves
    A x = b whenever phi_2(M) z = b (Section 6)."""
    A, r1, r2 = _small()
    Ad = A.dense()
    Phi1 = np.eye(36) - _dense_pi(Ad, r1)
    P1 = np.linalg.solve(Ad, np.eye(36) - _dense_pi(Ad, r1))
    P2 = np.linalg.solve(Phi1, np.eye(36) - _dense_pi(Phi1, r2))
    Phi2 = np.eye(36) - _dense_pi(Phi1, r2)
    assert np.allclose(Ad @ P1 @ P2, Phi2, atol=1e-9)


def test_outer_roots_are_the_gmres_residual_polynomial_of_phi1():
    """pi_2(M) v0 equals the GMRES(d_2) residual for the operator M = phi_1(A),
    found by least squares over the explicit Krylov basis of M."""
    A, r1, _ = _small()
    Ad = A.dense()
    Phi1 = np.eye(36) - _dense_pi(Ad, r1)
    v0 = np.random.default_rng(5).standard_normal(36)
    M = gmres.Composite(A.to_scipy(), r1)
    d2 = 4
    V, H, _ = poly.arnoldi(M, v0, d2)
    theta = poly.harmonic_ritz(H)
    K = np.empty((36, d2))
    K[:, 0] = v0
    for j in range(1, d2):
        K[:, j] = Phi1 @ K[:, j - 1]
    c, *_ = np.linalg.lstsq(Phi1 @ K, v0, rcond=None)
    r_ls = v0 - Phi1 @ (K @ c)
    assert np.linalg.norm(_dense_pi(Phi1, theta) @ v0 - r_ls) <= 1e-8 * np.linalg.norm(v0)


def test_double_pp_gmres_converges():
    A = synth.cd2d(30, 1.0)
    As = A.to_scipy()
    rs = synth.streams(13)
    b = synth.uniform_rhs(rs[1], A.n)
    r1 = poly.build_poly(As, 6, synth.gaussian_v0(rs[0], A.n)).roots
    r2 = poly.build_poly(gmres.Composite(As, r1), 6, synth.gaussian_v0(rs[0], A.n)).roots
    x, st = gmres.double_pp_gmres(As, r1, r2, b, 30, 1e-10)
    assert st.converged
    assert np.linalg.norm(b - As @ x) / np.linalg.norm(b) <= 1e-10


def test_chpoly_first_cycle_is_pp_gmres_with_roots_from_b():
    A = synth.cd2d(20, 0.6)
    As = A.to_scipy()
    b = synth.uniform_rhs(synth.streams(14)[1], A.n)
    _, s_ch = gmres.chpoly_gmres(As, 6, b, 15, 1e-30, max_cycles=1)
    roots = poly.build_poly(As, 6, b).roots
    _, s_pp = gmres.pp_gmres(As, roots, b, 15, 1e-30, max_cycles=1)
    assert np.allclose(s_ch.history, s_pp.history, rtol=1e-12)


def _paper():
    out = {}
    for line in open(os.path.join(GOLDEN, "paper_numbers.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def test_chpoly_beats_fixed_polynomial_at_low_degree():
    """Table 5.1: at degree 5 the changing polynomial needs far fewer mvps
    than PP-GMRES (580k vs 5765k at n = 10000).  The same trend at n = 1000
    (random streams and orthogonalisation differ from the paper's): ChPoly
    needs at most half the mvps."""
    nums = _paper()
    assert nums["ex12_d5_chpoly_mvps"] < 0.5 * nums["ex12_d5_ppg_mvps"]
    n = 1000
    A = synth.diag_csr(synth.ex11_diagonal(n)).to_scipy()
    rs = synth.streams(12)
    b = rs[1].standard_normal(n)
    b /= np.linalg.norm(b)
    pp = poly.build_poly(A, 5, rs[0].standard_normal(n))
    _, s1 = gmres.pp_gmres(A, pp.roots, b, 50, 1e-10, max_cycles=3000)
    _, s2 = gmres.chpoly_gmres(A, 5, b, 50, 1e-10, max_cycles=3000)
    assert s1.converged and s2.converged
    assert s2.mvps < 0.5 * s1.mvps
