"""Oracle: restarted GMRES with the polynomial preconditioner.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Algorithm 4 step 2 of Loe & Morgan: restarted GMRES(m) on phi(A) y = b with
phi(A) applied by Algorithm 1, then x = p(A) y by Algorithm 3.  Each restart
here starts from the true residual b - A x of the current x (x0 = 0, as in
Section 3.2); this is the same Krylov method, since b - phi(A) y =
b - A p(A) y, and costs the same d SpMVs per restart.

A cycle stops at m steps or when the shortcut residual |g_{j+1}| (the
least-squares residual ||beta e_1 - Hbar y||, Section 3.2 Example 3) falls to
tol ||b||; the solve is declared converged on the TRUE relative residual.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from .poly import apply_p, apply_phi


@dataclass
class SolveStats:
    iters: int = 0
    cycles: int = 0
    mvps: int = 0
    dots: int = 0
    converged: bool = False
    true_relres: float = float("nan")
    est_relres: float = float("nan")
    history: List[float] = field(default_factory=list)   # shortcut, per step
    true_history: List[float] = field(default_factory=list)  # per cycle end


def _givens(a: float, b: float):
    r = np.hypot(a, b)
    if r == 0.0:
        return 1.0, 0.0, 0.0
    return a / r, b / r, r


def _cycle(apply_op, r: np.ndarray, beta: float, m: int, bnorm: float,
           tol: float, ortho: str, st: SolveStats):
    """One GMRES(m) cycle from residual r: returns (V, y, k) with k steps."""
    n = r.shape[0]
    V = np.zeros((n, m + 1))
    H = np.zeros((m + 1, m))
    cs = np.zeros(m)
    sn = np.zeros(m)
    g = np.zeros(m + 1)
    g[0] = beta
    V[:, 0] = r / beta
    k = 0
    for j in range(m):
        w = apply_op(V[:, j])
        if ortho == "cgs2":
            for _ in range(2):
                h = V[:, : j + 1].T @ w
                w = w - V[:, : j + 1] @ h
                H[: j + 1, j] += h
            st.dots += 2 * (j + 1)
        else:
            for i in range(j + 1):
                hij = V[:, i] @ w
                w = w - hij * V[:, i]
                H[i, j] = hij
            st.dots += j + 1
        hn = np.linalg.norm(w)
        st.dots += 1
        H[j + 1, j] = hn
        # apply the earlier rotations to the new column
        for i in range(j):
            t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
            H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
            H[i, j] = t
        cs[j], sn[j], H[j, j] = _givens(H[j, j], H[j + 1, j])
        H[j + 1, j] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        k = j + 1
        st.iters += 1
        est = abs(g[j + 1]) / bnorm
        st.history.append(est)
        st.est_relres = est
        if est <= tol or hn == 0.0:
            break
        V[:, j + 1] = w / hn
    y = np.linalg.solve(np.triu(H[:k, :k]), g[:k]) if k > 0 else np.zeros(0)
    return V[:, :k], y, k


def pp_gmres(A, roots: Optional[np.ndarray], b: np.ndarray, m: int,
             tol: float, max_cycles: int = 1000, x0: Optional[np.ndarray] = None,
             ortho: str = "cgs2"):
    """PP(d)-GMRES(m) (roots given) or plain GMRES(m) (roots None).

    Returns (x, SolveStats).  mvps counts every SpMV: d per phi(A) v,
    d - 1 per p(A) v and 1 per true residual.
    """
    st = SolveStats()
    bnorm = np.linalg.norm(b)
    if x0 is None:
        x = np.zeros_like(b)
        r = b.copy()
    else:
        x = x0.copy()
        r = b - A @ x
        st.mvps += 1
    if roots is None:
        def op(v):
            st.mvps += 1
            return A @ v
    else:
        d = roots.shape[0]

        def op(v):
            st.mvps += d
            return apply_phi(A, roots, v)
    beta = np.linalg.norm(r)
    st.true_relres = beta / bnorm
    if st.true_relres <= tol:
        st.converged = True
        return x, st
    for _ in range(max_cycles):
        st.cycles += 1
        V, y, k = _cycle(op, r, beta, m, bnorm, tol, ortho, st)
        u = V @ y
        if roots is None:
            x = x + u
        else:
            x = x + apply_p(A, roots, u)
            st.mvps += max(roots.shape[0] - 1, 0)
        r = b - A @ x
        st.mvps += 1
        beta = np.linalg.norm(r)
        st.true_relres = beta / bnorm
        st.true_history.append(st.true_relres)
        if st.true_relres <= tol:
            st.converged = True
            break
        if not np.isfinite(beta):
            break
    return x, st


def fgmres_p(A, roots: np.ndarray, b: np.ndarray, m: int, tol: float,
             inner: str = "f32", max_cycles: int = 1000,
             A32=None):
    """Flexible GMRES(m) with z_j = p(A) v_j (right preconditioning).

    ``inner="f64"``: p(A) v in FP64 (then the iterates equal those of
    pp_gmres in exact arithmetic).  ``inner="f32"``: p(A) v runs in float32
    (matrix values, vectors, the root coefficients 1/theta, 2a and
    1/(a^2+b^2) rounded to float32, float32 accumulation), with the FP64
    Arnoldi, Givens least squares and true residual around it.
    """
    st = SolveStats()
    n = b.shape[0]
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b)
    r = b.copy()
    beta = np.linalg.norm(r)
    d = roots.shape[0]
    if inner == "f32":
        if A32 is None:
            A32 = A.astype(np.float32)
        r32 = _roots32(roots)

        def prec(v):
            return apply_p32(A32, r32, v.astype(np.float32)).astype(np.float64)
    else:
        def prec(v):
            return apply_p(A, roots, v)
    for _ in range(max_cycles):
        st.cycles += 1
        V = np.zeros((n, m + 1))
        Z = np.zeros((n, m))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[:, 0] = r / beta
        k = 0
        for j in range(m):
            Z[:, j] = prec(V[:, j])
            w = A @ Z[:, j]
            st.mvps += d          # (d - 1) inside p(A) v plus one A z
            for _ in range(2):
                h = V[:, : j + 1].T @ w
                w = w - V[:, : j + 1] @ h
                H[: j + 1, j] += h
            st.dots += 2 * (j + 1) + 1
            hn = np.linalg.norm(w)
            H[j + 1, j] = hn
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            cs[j], sn[j], H[j, j] = _givens(H[j, j], H[j + 1, j])
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            st.iters += 1
            est = abs(g[j + 1]) / bnorm
            st.history.append(est)
            st.est_relres = est
            if est <= tol or hn == 0.0:
                break
            V[:, j + 1] = w / hn
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        x = x + Z[:, :k] @ y
        r = b - A @ x
        st.mvps += 1
        beta = np.linalg.norm(r)
        st.true_relres = beta / bnorm
        st.true_history.append(st.true_relres)
        if st.true_relres <= tol:
            st.converged = True
            break
        if not np.isfinite(beta):
            break
    return x, st


def _roots32(roots: np.ndarray):
    """Per-step float32 coefficients for Algorithm 3 in float32."""
    out = []
    for t in roots:
        if t.imag == 0:
            out.append(("r", np.float32(1.0 / t.real), np.float32(0.0)))
        else:
            a, b = t.real, t.imag
            out.append(("c", np.float32(2.0 * a), np.float32(1.0 / (a * a + b * b))))
    return out


def apply_p32(A32, coef, v: np.ndarray) -> np.ndarray:
    """Algorithm 3 in float32 arithmetic (coefficients from _roots32)."""
    d = len(coef)
    prod = v.astype(np.float32).copy()
    p = np.zeros_like(prod)
    i = 0
    while i < d - 1:
        kind, c1, c2 = coef[i]
        if kind == "r":
            p = p + c1 * prod
            prod = prod - c1 * (A32 @ prod)
            i += 1
        else:
            tmp = c1 * prod - A32 @ prod
            p = p + c2 * tmp
            if i <= d - 3:
                prod = prod - c2 * (A32 @ tmp)
            i += 2
    if coef[d - 1][0] == "r" and i == d - 1:
        p = p + coef[d - 1][1] * prod
    return p


def stability_check(A, roots: np.ndarray, b: np.ndarray) -> float:
    """StCh = ||r1 - r2|| (Section 3.5): r1 = b - A p(A) b by Algorithm 3,
    r2 = pi(A) b = b - phi(A) b by Algorithm 1."""
    r1 = b - A @ apply_p(A, roots, b)
    r2 = b - apply_phi(A, roots, b)
    return float(np.linalg.norm(r1 - r2))


def build_poly_checked(A, d: int, v0: np.ndarray, b: Optional[np.ndarray], tol: float,
                       d_min: int = 1, stability: bool = True):
    """The polynomial with the stability check of Section 3.5 applied before
    the solve: build the degree-d polynomial from v0 (Algorithm 4 step 1),
    compute StCh with the unit vector b / ||b|| (v0 / ||v0|| when b is None),
    and while StCh > tol and the degree is above d_min, lower the degree and
    check again.  The paper says only that the degree "can be lowered"; the
    reading taken here halves it, d <- max(d_min, d // 2), and the lower-degree
    polynomial is GMRES(d) from the same v0.  Returns (Poly, tried) with
    tried = [(original degree, StCh), ...] largest degree first."""
    from .poly import build_poly
    u = v0 if b is None else b
    u = u / np.linalg.norm(u)
    tried = []
    deg = d
    while True:
        pp = build_poly(A, deg, v0, stability=stability)
        s = stability_check(A, pp.roots, u)
        tried.append((pp.d, s))
        if s <= tol or pp.d <= d_min:
            return pp, tried
        deg = max(d_min, pp.d // 2)


def adjoint_grads(A, AT, roots, x: np.ndarray, gx: np.ndarray, m: int,
                  tol: float, rowptr: np.ndarray, colind: np.ndarray,
                  max_cycles: int = 1000):
    """Gradients of L(x(b, vals)) with A x = b, given gx = dL/dx.

    lambda solves A^T lambda = gx; since p(A^T) = p(A)^T the same roots
    precondition the transposed system.  dL/db = lambda and
    dL/dvals[k] = -lambda[row(k)] * x[colind[k]].
    """
    lam, st = pp_gmres(AT, roots, gx, m, tol, max_cycles=max_cycles)
    rows = np.repeat(np.arange(rowptr.shape[0] - 1), np.diff(rowptr))
    gvals = -lam[rows] * x[colind]
    return lam, gvals, st


def batched_solve(problems, d: int, m: int, tol: float, inner: str = "f32",
                  max_cycles: int = 1000):
    """The batching form, defined as what it computes: for every system
    (A, B, v0) its own polynomial from GMRES(d) on v0, then FGMRES(m) with
    p(A) applied in float32 for every right-hand side, independently.
    Returns per-system (roots, [x per rhs], [stats per rhs])."""
    from .poly import build_poly
    out = []
    for A, B, v0 in problems:
        As = A.to_scipy() if hasattr(A, "to_scipy") else A
        pp = build_poly(As, d, v0)
        xs, sts = [], []
        for b in B:
            x, st = fgmres_p(As, pp.roots, b, m, tol, inner=inner, max_cycles=max_cycles)
            xs.append(x)
            sts.append(st)
        out.append((pp.roots, xs, sts))
    return out


class Composite:
    """The operator M = phi_1(A) (Algorithm 1 with the inner roots), usable
    wherever the oracle takes a matrix (``M @ v``): Arnoldi on M gives the
    outer polynomial of double polynomial preconditioning (Section 6)."""

    def __init__(self, A, roots1):
        self.A = A
        self.roots1 = roots1
        self.shape = A.shape

    def __matmul__(self, v):
        return apply_phi(self.A, self.roots1, v)


def double_pp_gmres(A, roots1: np.ndarray, roots2: np.ndarray, b: np.ndarray, m: int,
                    tol: float, max_cycles: int = 1000):
    """Section 6: GMRES on phi_2(phi_1(A)) z = b, x = p_1(A) p_2(phi_1(A)) z.
    Restarts from the true residual of x' = p_2(M) z for M = phi_1(A), then
    x = p_1(A) x' (A x = A p_1(A) x' = M x')."""
    M = Composite(A, roots1)
    xp, st = pp_gmres(M, roots2, b, m, tol, max_cycles=max_cycles)
    x = apply_p(A, roots1, xp)
    return x, st


def chpoly_gmres(A, d: int, b: np.ndarray, m: int, tol: float, max_cycles: int = 1000):
    """Section 5.2: PP-GMRES(m) with the polynomial rebuilt at the start of
    every cycle by GMRES(d) from the current residual."""
    from .poly import build_poly
    st = SolveStats()
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b)
    r = b.copy()
    beta = bnorm
    st.true_relres = 1.0
    for _ in range(max_cycles):
        st.cycles += 1
        roots = build_poly(A, d, r).roots
        st.mvps += d
        nd = roots.shape[0]

        def op(v):
            st.mvps += nd
            return apply_phi(A, roots, v)
        V, y, k = _cycle(op, r, beta, m, bnorm, tol, "cgs2", st)
        x = x + apply_p(A, roots, V @ y)
        st.mvps += nd - 1
        r = b - A @ x
        st.mvps += 1
        beta = np.linalg.norm(r)
        st.true_relres = beta / bnorm
        st.true_history.append(st.true_relres)
        if st.true_relres <= tol:
            st.converged = True
            break
        if not np.isfinite(beta):
            break
    return x, st
