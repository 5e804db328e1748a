"""Oracle: construction and application of the GMRES polynomial.

TEST INFRASTRUCTURE ONLY (see the package docstring).

References are to Loe & Morgan, "Toward Efficient Polynomial Preconditioning
for GMRES": eq (2.1) the residual polynomial in root form, eq (2.2) the
conjugate-pair factor, Algorithm 1 (phi(A) v), Algorithm 2 (root adding),
eq (3.1) the expansion of p, Algorithm 3 (p(A) v), Algorithm 4 (the method).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Tuple

import numpy as np
import scipy.linalg as sla

# ---------------------------------------------------------------------------
# Arnoldi / GMRES(d) -- Algorithm 4 step 1(a)
# ---------------------------------------------------------------------------

BREAKDOWN_RTOL = 1e-13


def arnoldi(A, v0: np.ndarray, d: int, ortho: str = "cgs2"):
    """d steps of Arnoldi from v0: A V_d = V_{d+1} Hbar.

    ``A`` is anything with ``A @ x``.  ``ortho`` is "cgs2" (classical
    Gram-Schmidt applied twice) or "mgs" (modified Gram-Schmidt, the choice
    of the paper's experiments, Section 3.2).  Returns (V, Hbar, d_eff) where
    d_eff < d after a breakdown (h_{j+1,j} = 0: the Krylov space is
    invariant).  The breakdown test is relative: h_{j+1,j} <= 1e-13 ||A v_j||
    (the paper does not state one; an exact-zero test never fires in
    floating point).
    """
    n = v0.shape[0]
    V = np.zeros((n, d + 1))
    H = np.zeros((d + 1, d))
    beta = np.linalg.norm(v0)
    V[:, 0] = v0 / beta
    for j in range(d):
        w = A @ V[:, j]
        wnorm0 = np.linalg.norm(w)
        if ortho == "cgs2":
            for _ in range(2):
                h = V[:, : j + 1].T @ w
                w = w - V[:, : j + 1] @ h
                H[: j + 1, j] += h
        elif ortho == "mgs":
            for i in range(j + 1):
                hij = V[:, i] @ w
                w = w - hij * V[:, i]
                H[i, j] = hij
        else:
            raise ValueError(ortho)
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] <= BREAKDOWN_RTOL * wnorm0:
            H[j + 1, j] = 0.0
            return V[:, : j + 1], H[: j + 2, : j + 1], j + 1
        V[:, j + 1] = w / H[j + 1, j]
    return V, H, d


# ---------------------------------------------------------------------------
# Harmonic Ritz values -- Algorithm 4 step 1(b)
# ---------------------------------------------------------------------------


def harmonic_ritz(Hbar: np.ndarray) -> np.ndarray:
    """Roots of the GMRES polynomial from the (d+1) x d Hessenberg matrix.

    theta = eig(H_dd + h_{d+1,d}^2 f e_d^T) with H_dd^T f = e_d (H is real,
    so H^{-*} = H^{-T}).  Returned as a complex array; real eigenvalues have
    an imaginary part of exactly 0 and complex ones come in exact conjugate
    pairs (LAPACK's real Schur form).
    """
    d = Hbar.shape[1]
    Hdd = Hbar[:d, :d]
    hlast = Hbar[d, d - 1] if Hbar.shape[0] > d else 0.0
    e = np.zeros(d)
    e[-1] = 1.0
    f = np.linalg.solve(Hdd.T, e)
    G = Hdd.copy()
    G[:, -1] += hlast * hlast * f
    theta = np.linalg.eigvals(G).astype(np.complex128)
    return theta


def harmonic_ritz_pencil(Hbar: np.ndarray) -> np.ndarray:
    """Second route to the same values: the pencil (Hbar^T Hbar, H_dd^T).

    Multiplying (H_dd + h^2 f e_d^T) g = theta g by H_dd^T gives
    (H_dd^T H_dd + h^2 e_d e_d^T) g = theta H_dd^T g, and the left matrix is
    Hbar^T Hbar.
    """
    d = Hbar.shape[1]
    return sla.eigvals(Hbar.T @ Hbar, Hbar[:d, :d].T).astype(np.complex128)


# ---------------------------------------------------------------------------
# Modified Leja ordering (Section 2, Algorithm 2 step 1)
# ---------------------------------------------------------------------------


def _units(theta: np.ndarray) -> List[complex]:
    """Representatives of the root units: each real root, and the +Im member
    of each conjugate pair (the -Im member is implied)."""
    out = []
    for t in theta:
        if t.imag >= 0:
            out.append(complex(t))
    n_real = sum(1 for t in theta if t.imag == 0)
    n_pos = sum(1 for t in theta if t.imag > 0)
    n_neg = sum(1 for t in theta if t.imag < 0)
    if n_pos != n_neg:
        raise ValueError("roots are not closed under conjugation")
    assert len(out) == n_real + n_pos
    return out


def _expand(units: List[complex]) -> np.ndarray:
    out = []
    for u in units:
        out.append(u)
        if u.imag != 0:
            out.append(u.conjugate())
    return np.array(out, dtype=np.complex128)


def leja_order(theta: np.ndarray) -> np.ndarray:
    """Modified Leja ordering of a conjugation-closed set of roots.

    Reading of the ordering the paper cites (modified Leja points of Bai, Hu
    and Reichel): the first point has the largest modulus; each next point
    maximises the product of distances to the points already chosen
    (computed as a sum of logarithms, against overflow and underflow); when a
    non-real point is chosen its conjugate follows at once, +Im member first.
    Ties go to the larger real part, then the larger imaginary part.  A
    point equal to a chosen one scores -inf and so goes last.
    """
    units = _units(np.asarray(theta, dtype=np.complex128))
    chosen: List[complex] = []
    order: List[complex] = []
    remaining = list(units)
    while remaining:
        best = None
        best_key = None
        for z in remaining:
            if not chosen:
                score = math.log(abs(z)) if z != 0 else -math.inf
            else:
                score = 0.0
                for c in chosen:
                    dist = abs(z - c)
                    score += math.log(dist) if dist > 0 else -math.inf
            key = (score, z.real, z.imag)
            if best_key is None or key > best_key:
                best_key = key
                best = z
        remaining.remove(best)
        order.append(best)
        chosen.append(best)
        if best.imag != 0:
            chosen.append(best.conjugate())
    return _expand(order)


# ---------------------------------------------------------------------------
# pof and root adding -- Algorithm 2
# ---------------------------------------------------------------------------


def log10_pof(theta: np.ndarray) -> np.ndarray:
    """log10 pof(k) = sum_{i != k} log10 |1 - theta_k / theta_i|."""
    d = theta.shape[0]
    out = np.empty(d)
    for k in range(d):
        s = 0.0
        for i in range(d):
            if i == k:
                continue
            m = abs(1.0 - theta[k] / theta[i])
            s += math.log10(m) if m > 0 else -math.inf
        out[k] = s
    return out


def n_copies(lpof: float, threshold_log10: float = 4.0,
             step_log10: float = 14.0) -> int:
    """Extra copies of a root: least integer above (log10 pof - 4)/14.

    At an exact integer the rule "least integer greater than x" and the
    statement "add one when pof > 1e4" disagree; the reading taken is
    ceil(x) for x > 0 and 0 otherwise, which keeps pof = 1e4 at no copies.
    """
    x = (lpof - threshold_log10) / step_log10
    if not (x > 0):
        return 0
    return int(math.ceil(x))


def add_roots(theta_leja: np.ndarray, threshold_log10: float = 4.0,
              step_log10: float = 14.0) -> Tuple[np.ndarray, int, np.ndarray]:
    """Algorithm 2 steps 2-3 on Leja-ordered roots.

    For each original root unit k in order (a conjugate pair is one unit
    and shares one pof), with c_k = n_copies(pof(k)) > 0: one copy goes to
    the end of the current list; the other c_k - 1 copies go evenly between
    the unit's own position p and the end: copy j (j = 1..c_k-1) is inserted
    before index p + max(1, floor(j * (L - 1 - p) / c_k + 1/2)), where L is
    the current list length after the first copy was appended.  Pairs stay
    together because positions count units.  Returns (roots, n_added,
    log10 pof per original root).
    """
    theta_leja = np.asarray(theta_leja, dtype=np.complex128)
    lpof = log10_pof(theta_leja)
    # build the unit list with its pof
    units: List[Tuple[complex, int]] = []   # (representative, original index)
    k = 0
    unit_pof = []
    while k < theta_leja.shape[0]:
        t = theta_leja[k]
        if t.imag != 0:
            if not (k + 1 < theta_leja.shape[0] and theta_leja[k + 1] == t.conjugate()):
                raise ValueError("conjugate pair not adjacent")
            units.append((complex(t), k))
            unit_pof.append(lpof[k])
            k += 2
        else:
            units.append((complex(t), k))
            unit_pof.append(lpof[k])
            k += 1
    lst: List[Tuple[complex, int]] = [(u, idx) for idx, (u, _) in enumerate(units)]
    tags = list(range(len(units)))       # tag = original unit id, -1 for copies
    n_added = 0
    for uid, (u, _) in enumerate(units):
        c = n_copies(unit_pof[uid], threshold_log10, step_log10)
        if c == 0:
            continue
        lst.append((u, -1))
        tags.append(-1)
        p = tags.index(uid)
        L = len(lst)
        span = (L - 1) - p
        for j in range(c - 1, 0, -1):
            q = p + max(1, int(math.floor(j * span / c + 0.5)))
            lst.insert(q, (u, -1))
            tags.insert(q, -1)
        n_added += c * (2 if u.imag != 0 else 1)
    roots = _expand([u for u, _ in lst])
    return roots, n_added, lpof


# ---------------------------------------------------------------------------
# Whole construction -- Algorithm 4 step 1
# ---------------------------------------------------------------------------


@dataclass
class Poly:
    roots: np.ndarray        # Leja-ordered roots with added copies (complex)
    theta: np.ndarray        # harmonic Ritz values as computed (complex)
    Hbar: np.ndarray
    V: np.ndarray
    d: int                   # original degree actually reached
    n_added: int
    lpof: np.ndarray


def build_poly(A, d: int, v0: np.ndarray, ortho: str = "cgs2",
               stability: bool = True) -> Poly:
    """GMRES(d) from v0, harmonic Ritz values, Leja order, root adding."""
    V, Hbar, d_eff = arnoldi(A, v0, d, ortho)
    theta = harmonic_ritz(Hbar)
    led = leja_order(theta)
    if stability:
        roots, n_added, lpof = add_roots(led)
    else:
        roots, n_added, lpof = led, 0, log10_pof(led)
    return Poly(roots, theta, Hbar, V, d_eff, n_added, lpof)


# ---------------------------------------------------------------------------
# Application -- Algorithms 1 and 3
# ---------------------------------------------------------------------------


def apply_phi(A, roots: np.ndarray, v: np.ndarray) -> np.ndarray:
    """phi(A) v = v - pi(A) v with pi in root form (Algorithm 1)."""
    d = roots.shape[0]
    pi = v.copy()
    i = 0
    while i < d:
        t = roots[i]
        if t.imag == 0:
            prod = A @ pi
            pi = pi - (1.0 / t.real) * prod
            i += 1
        else:
            a, b = t.real, t.imag
            prod = A @ pi
            tmp = A @ prod - 2.0 * a * prod
            pi = pi + (1.0 / (a * a + b * b)) * tmp
            i += 2
    return v - pi


def apply_pi(A, roots: np.ndarray, v: np.ndarray) -> np.ndarray:
    """pi(A) v, the residual polynomial, by the same loop as Algorithm 1."""
    return v - apply_phi(A, roots, v)


def apply_p(A, roots: np.ndarray, v: np.ndarray) -> np.ndarray:
    """p(A) v by Algorithm 3 (sum of the terms u_k of eq (3.1))."""
    d = roots.shape[0]
    prod = v.copy()
    p = np.zeros_like(v)
    i = 0
    while i < d - 1:       # 0-based: roots[0 .. d-2]
        t = roots[i]
        if t.imag == 0:
            p = p + (1.0 / t.real) * prod
            prod = prod - (1.0 / t.real) * (A @ prod)
            i += 1
        else:
            a, b = t.real, t.imag
            c2 = 1.0 / (a * a + b * b)
            tmp = 2.0 * a * prod - A @ prod
            p = p + c2 * tmp
            if i <= d - 3:     # 1-based i <= d-2
                prod = prod - c2 * (A @ tmp)
            i += 2
    if roots[d - 1].imag == 0 and i == d - 1:
        p = p + (1.0 / roots[d - 1].real) * prod
    return p


def spmv_count_phi(roots: np.ndarray) -> int:
    """SpMVs in one Algorithm 1 application (= d)."""
    return int(roots.shape[0])


def spmv_count_p(roots: np.ndarray) -> int:
    """SpMVs in one Algorithm 3 application (= d - 1)."""
    return max(int(roots.shape[0]) - 1, 0)


class _Scalar:
    """A 1x1 'matrix' alpha so that Algorithms 1 and 3 evaluate the scalar
    polynomials phi(alpha), p(alpha)."""

    def __init__(self, alpha):
        self.alpha = alpha

    def __matmul__(self, x):
        return self.alpha * x


def p_scalar(roots: np.ndarray, alpha: complex) -> complex:
    return complex(apply_p(_Scalar(alpha), roots, np.array([1.0 + 0j]))[0])


def phi_scalar(roots: np.ndarray, alpha: complex) -> complex:
    return complex(apply_phi(_Scalar(alpha), roots, np.array([1.0 + 0j]))[0])
