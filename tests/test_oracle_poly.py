"""Pins for the oracle's polynomial construction and application.

Each test checks the oracle against something other than itself: a dense
closed form, a brute-force least-squares problem, a second eigenvalue route,
hand-worked golden fixtures, or numbers printed in the paper.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import poly

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_matrix(n, seed, shift=None):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n)) / math.sqrt(n)
    return M + (shift if shift is not None else 3.0) * np.eye(n)


def _dense_pi(A, roots):
    """pi(A) = prod (I - A/theta_i) as a dense complex product (eq 2.1)."""
    n = A.shape[0]
    P = np.eye(n, dtype=np.complex128)
    for t in roots:
        P = P @ (np.eye(n) - A / t)
    return P


def _root_sets():
    yield "real", np.array([2.5, 3.1, 4.0, 2.2, 3.7], dtype=complex)
    yield "ends_in_pair", np.array([4.0, 3 + 1j, 3 - 1j, 2.5, 2 + 0.5j, 2 - 0.5j])
    yield "pair_then_real", np.array([3 + 1j, 3 - 1j, 2.5, 2 + 0.5j, 2 - 0.5j, 3.3])
    yield "single_real", np.array([3.0 + 0j])
    yield "single_pair", np.array([3 + 1j, 3 - 1j])
    yield "repeated", np.array([3.0, 2.0, 3.0, 3 + 1j, 3 - 1j, 3 + 1j, 3 - 1j], dtype=complex)


@pytest.mark.parametrize("name,roots", list(_root_sets()))
def test_apply_phi_and_p_match_dense_closed_form(name, roots):
    """Alg 1 = I - prod(I - A/theta) and Alg 3 = A^{-1}(I - pi(A))."""
    A = _rand_matrix(24, 1)
    rng = np.random.default_rng(2)
    v = rng.standard_normal(24)
    Pi = _dense_pi(A, roots)
    assert np.abs(Pi.imag).max() < 1e-10
    Pi = Pi.real
    phi_ref = v - Pi @ v
    p_ref = np.linalg.solve(A, v - Pi @ v)
    phi = poly.apply_phi(A, roots, v)
    p = poly.apply_p(A, roots, v)
    assert np.linalg.norm(phi - phi_ref) <= 1e-12 * max(1, np.linalg.norm(phi_ref))
    Pmat = np.linalg.solve(A, np.eye(24) - Pi)
    assert np.linalg.norm(p - p_ref) <= 1e-12 * np.linalg.norm(Pmat, 2) * np.linalg.norm(v)
    # consistency of the two algorithms: v - A p(A) v = pi(A) v (Section 3.5)
    assert np.linalg.norm((v - A @ p) - (v - phi)) <= 1e-11 * np.linalg.norm(v)


def test_scalar_p_gives_one_over_alpha_at_roots():
    """1 - theta_i p(theta_i) = pi(theta_i) = 0 for every root (eq 3.1)."""
    roots = np.array([4.0, 3 + 1j, 3 - 1j, 2.5, 2 + 0.5j, 2 - 0.5j])
    for t in roots:
        assert abs(1.0 - t * poly.p_scalar(roots, t)) < 1e-12
        assert abs(1.0 - poly.phi_scalar(roots, t)) < 1e-12


def test_pair_factor_eq_2_2():
    """(1 - a/t)(1 - a/conj t) = 1 + (a^2 - 2 a Re t)/|t|^2, via Alg 1 with a
    single pair against the complex product."""
    t = 1.7 + 0.6j
    roots = np.array([t, t.conjugate()])
    for alpha in (0.3, 1.1, -2.0, 0.5 + 0.5j):
        pi_direct = (1 - alpha / t) * (1 - alpha / t.conjugate())
        assert abs((1 - poly.phi_scalar(roots, alpha)) - pi_direct) < 1e-13


def test_diagonal_matrix_is_scalar_evaluation():
    lam = np.linspace(0.5, 5.0, 40)
    A = synth.diag_csr(lam).to_scipy()
    roots = np.array([4.5, 3 + 1j, 3 - 1j, 1.0, 2.0], dtype=complex)
    v = np.random.default_rng(3).standard_normal(40)
    pi = np.ones(40, dtype=complex)
    for t in roots:
        pi *= 1 - lam / t
    expect = (1 - pi.real) / lam * v
    got = poly.apply_p(A, roots, v)
    assert np.allclose(got, expect, rtol=1e-12, atol=1e-13)


def test_arnoldi_relation_and_orthogonality():
    A = _rand_matrix(60, 4, shift=1.0)
    v0 = np.random.default_rng(5).standard_normal(60)
    for ortho in ("cgs2", "mgs"):
        V, H, d = poly.arnoldi(A, v0, 12, ortho)
        assert d == 12
        assert np.linalg.norm(A @ V[:, :12] - V @ H) < 1e-12 * np.linalg.norm(A)
        assert np.linalg.norm(V.T @ V - np.eye(13)) < 1e-13
        assert np.allclose(V[:, 0], v0 / np.linalg.norm(v0))
    V1, H1, _ = poly.arnoldi(A, v0, 12, "cgs2")
    V2, H2, _ = poly.arnoldi(A, v0, 12, "mgs")
    assert np.allclose(H1, H2, atol=1e-11)


def test_arnoldi_breakdown_on_invariant_subspace():
    A = np.diag([1.0, 2.0, 3.0, 4.0, 5.0, 6.0])
    v0 = np.array([1.0, 1.0, 1.0, 0, 0, 0])
    V, H, d = poly.arnoldi(A, v0, 5)
    assert d == 3
    theta = np.sort(poly.harmonic_ritz(H[:4, :3]).real)
    assert np.allclose(theta, [1, 2, 3])


@pytest.mark.parametrize("seed,d", [(6, 5), (7, 8), (8, 10)])
def test_harmonic_ritz_roots_are_the_gmres_residual_polynomial(seed, d):
    """pi(A) v0 with pi built from the harmonic Ritz values equals the
    GMRES(d) residual, found by brute-force least squares over the explicit
    Krylov basis [v0, A v0, ..., A^{d-1} v0] (Section 2, Algorithm 4)."""
    n = 40
    A = _rand_matrix(n, seed, shift=2.0)
    v0 = np.random.default_rng(seed + 100).standard_normal(n)
    K = np.empty((n, d))
    K[:, 0] = v0
    for j in range(1, d):
        K[:, j] = A @ K[:, j - 1]
    c, *_ = np.linalg.lstsq(A @ K, v0, rcond=None)
    r_ls = v0 - A @ (K @ c)
    V, H, _ = poly.arnoldi(A, v0, d)
    theta = poly.harmonic_ritz(H)
    r_pi = (_dense_pi(A, theta) @ v0).real
    assert np.linalg.norm(r_pi - r_ls) <= 1e-8 * np.linalg.norm(v0)
    # and the oracle's own root-form loop gives the same vector
    r_loop = poly.apply_pi(A, poly.leja_order(theta), v0)
    assert np.linalg.norm(r_loop - r_ls) <= 1e-8 * np.linalg.norm(v0)


@pytest.mark.parametrize("seed", [9, 10, 11])
def test_harmonic_ritz_two_routes_agree(seed):
    A = _rand_matrix(80, seed, shift=1.5)
    v0 = np.random.default_rng(seed).standard_normal(80)
    _, H, _ = poly.arnoldi(A, v0, 15)
    t1 = poly.harmonic_ritz(H)
    t2 = poly.harmonic_ritz_pencil(H)
    # match as multisets
    from scipy.optimize import linear_sum_assignment
    C = np.abs(t1[:, None] - t2[None, :])
    r, c = linear_sum_assignment(C)
    assert np.max(C[r, c] / np.abs(t1[r])) < 1e-8


def _parse_roots(s):
    return np.array([complex(x.strip()) for x in s.split(",")])


def _golden_lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                yield [part.strip() for part in line.split(";")]


def test_leja_golden_cases():
    n = 0
    for inp, out in _golden_lines("leja_cases.txt"):
        got = poly.leja_order(_parse_roots(inp))
        assert np.array_equal(got, _parse_roots(out)), (inp, got)
        n += 1
    assert n >= 4


def test_leja_invariants_on_random_sets():
    rng = np.random.default_rng(12)
    for _ in range(20):
        nr = rng.integers(0, 6)
        npair = rng.integers(0, 5)
        re = list(rng.uniform(-1, 5, nr))
        z = rng.uniform(0, 5, npair) + 1j * rng.uniform(0.1, 3, npair)
        theta = np.array(re + list(z) + list(z.conjugate()), dtype=complex)
        if theta.size == 0:
            continue
        rng.shuffle(theta)
        o = poly.leja_order(theta)
        assert sorted(o.tolist(), key=lambda c: (c.real, c.imag)) == \
            sorted(theta.tolist(), key=lambda c: (c.real, c.imag))
        assert np.abs(o[0]) >= np.abs(theta).max() * (1 - 1e-14)
        i = 0
        while i < o.size:
            if o[i].imag != 0:
                assert o[i].imag > 0 and o[i + 1] == o[i].conjugate()
                i += 2
            else:
                i += 1


def test_root_adding_golden_cases():
    for inp, out, nadd in _golden_lines("root_adding_cases.txt"):
        roots, n_added, _ = poly.add_roots(_parse_roots(inp))
        assert n_added == int(nadd)
        assert np.allclose(roots, _parse_roots(out), rtol=0, atol=0), (inp, roots)


def test_copies_threshold_rule():
    """Algorithm 2: one copy above pof 1e4, one more per factor 1e14."""
    assert poly.n_copies(4.0) == 0
    assert poly.n_copies(3.0) == 0
    assert poly.n_copies(4.0001) == 1
    assert poly.n_copies(18.0) == 1
    assert poly.n_copies(18.001) == 2
    assert poly.n_copies(32.001) == 3
    assert poly.n_copies(-math.inf) == 0


def _paper_numbers():
    out = {}
    for line in open(os.path.join(GOLDEN, "paper_numbers.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def test_example7_two_roots_added_at_30_and_60():
    """Example 7: PP(125) on the diagonal test matrix adds one root at 30
    (pof 5.79e5) and one at 60 (pof 3.12e4)."""
    nums = _paper_numbers()
    A = synth.diag_csr(synth.ex7_diagonal()).to_scipy()
    v0 = synth.gaussian_v0(synth.streams(7)[0], 5000)
    P = poly.build_poly(A, int(nums["ex7_d"]), v0)
    assert P.n_added == int(nums["ex7_added"])
    added = np.sort(P.roots[P.roots.size - P.n_added:].real)
    assert np.allclose(added, [30.0, 60.0], rtol=1e-6)
    led = poly.leja_order(P.theta)
    k30 = int(np.argmin(np.abs(led - 30)))
    k60 = int(np.argmin(np.abs(led - 60)))
    assert abs(P.lpof[k30] - math.log10(nums["ex7_pof_30"])) < 0.3
    assert abs(P.lpof[k60] - math.log10(nums["ex7_pof_60"])) < 0.3


def test_spd_smallest_root_never_gets_a_copy():
    """Section 3.4: for SPD A the smallest harmonic Ritz value has pof < 1."""
    rng = np.random.default_rng(13)
    for trial in range(5):
        lam = np.sort(rng.uniform(0.01, 10.0, 300))
        lam[-1] = 200.0  # an outlier that does get copies
        A = synth.diag_csr(lam).to_scipy()
        P = poly.build_poly(A, 30, rng.standard_normal(300))
        led = poly.leja_order(P.theta)
        k = int(np.argmin(np.abs(led)))
        assert P.lpof[k] < 0.0


def test_theorem_3_1_richardson_step():
    """Theorem 3.1: SPD A, theta_k >= lambda_n / 2 gives
    ||(I - A/theta_k) pi(A) b|| <= ||pi(A) b||."""
    rng = np.random.default_rng(14)
    lam = np.sort(rng.uniform(0.1, 10.0, 200))
    A = synth.diag_csr(lam).to_scipy()
    P = poly.build_poly(A, 20, rng.standard_normal(200), stability=False)
    b = rng.standard_normal(200)
    pib = poly.apply_pi(A, P.roots, b)
    checked = 0
    for t in P.roots:
        if t.imag == 0 and t.real >= lam[-1] / 2:
            assert np.linalg.norm(pib - (A @ pib) / t.real) <= np.linalg.norm(pib) * (1 + 1e-12)
            checked += 1
    assert checked > 0


@pytest.mark.slow
def test_example11_degree512_adds_about_four_roots():
    """Table 4.1: degree 512 on diag(i^2/n), n = 20000, gets 512+4."""
    nums = _paper_numbers()
    n = int(nums["ex11_n"])
    A = synth.diag_csr(synth.ex11_diagonal(n)).to_scipy()
    v0 = synth.gaussian_v0(synth.streams(11)[0], n)
    P = poly.build_poly(A, 512, v0)
    assert abs(P.n_added - int(nums["ex11_d512_added"])) <= 3
