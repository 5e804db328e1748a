"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the polynomial-preconditioning method.  It
only builds the problems the method is run on: finite-difference
convection-diffusion matrices in CSR form (the family of Example 5, Section
3.2 of Loe & Morgan, "Toward Efficient Polynomial Preconditioning for
GMRES"), the diagonal test matrices of Examples 7, 11 and 12, and the seeded
random vectors (right-hand sides and the random starting vector v0 that
Algorithm 4 step 1(a) asks for).

Conventions
-----------
* CSR: ``rowptr`` int32 [n+1], ``colind`` int32 [nnz] sorted within each
  row, ``vals`` float64 [nnz].
* Grids are interior nodes of the unit square / cube with zero Dirichlet
  boundary, ``h = 1/(N+1)``, lexicographic order with x fastest.
* The stencil is scaled by h^2: the centred 5-point (7-point in 3-D)
  Laplacian has diagonal 4 (6), and a first-derivative term ``beta * u_x``
  with cell value ``c = beta*h/2`` gives the lower x-neighbour ``-1 - c``
  and the upper x-neighbour ``-1 + c``.
* Random streams: ``numpy.random.Generator(PCG64)`` seeded through
  ``SeedSequence(seed).spawn(4)`` in the fixed order (v0, b, field, batch).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "CSRHost", "cd2d", "cd3d", "diag_csr", "smooth_field", "streams", "batch_problem",
    "ProblemSpec", "problem", "PROBLEMS", "batch_specs", "uniform_rhs",
    "gaussian_v0", "ex7_diagonal", "ex11_diagonal",
]


@dataclass
class CSRHost:
    """Host CSR matrix (int32 indices, float64 values)."""
    n: int
    rowptr: np.ndarray
    colind: np.ndarray
    vals: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.colind.shape[0])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.vals, self.colind, self.rowptr),
                             shape=(self.n, self.n))

    def dense(self) -> np.ndarray:
        out = np.zeros((self.n, self.n))
        for i in range(self.n):
            lo, hi = self.rowptr[i], self.rowptr[i + 1]
            out[i, self.colind[lo:hi]] += self.vals[lo:hi]
        return out


def _assemble(n: int, offsets: Sequence[int], coeffs: np.ndarray,
              valid: np.ndarray) -> CSRHost:
    """Pack a banded stencil into CSR.

    ``coeffs`` and ``valid`` are (n, len(offsets)) arrays; column ``k`` of a
    row ``i`` is ``i + offsets[k]``.  ``offsets`` must be increasing so that
    each row's column indices come out sorted.
    """
    offs = np.asarray(offsets, dtype=np.int64)
    assert np.all(np.diff(offs) > 0)
    rows = np.arange(n, dtype=np.int64)[:, None]
    cols = rows + offs[None, :]
    counts = valid.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32 CSR indices")
    colind = cols[valid].astype(np.int32)
    vals = coeffs[valid].astype(np.float64)
    return CSRHost(n, rowptr.astype(np.int32), colind, vals)


def cd2d(N: int, beta_h, ) -> CSRHost:
    """2-D convection-diffusion ``-u_xx - u_yy + beta u_x`` on an N x N grid.

    ``beta_h`` is the cell value beta*h: a scalar, or an array of N*N
    per-node values (each row then uses its own node's value).
    """
    n = N * N
    c = np.broadcast_to(np.asarray(beta_h, dtype=np.float64) / 2.0, (n,))
    idx = np.arange(n, dtype=np.int64)
    ix = idx % N
    iy = idx // N
    coeffs = np.empty((n, 5))
    valid = np.empty((n, 5), dtype=bool)
    # column order S, W, C, E, N  (offsets -N, -1, 0, +1, +N)
    coeffs[:, 0] = -1.0; valid[:, 0] = iy > 0
    coeffs[:, 1] = -1.0 - c; valid[:, 1] = ix > 0
    coeffs[:, 2] = 4.0; valid[:, 2] = True
    coeffs[:, 3] = -1.0 + c; valid[:, 3] = ix < N - 1
    coeffs[:, 4] = -1.0; valid[:, 4] = iy < N - 1
    return _assemble(n, (-N, -1, 0, 1, N), coeffs, valid)


def cd3d(N: int, beta_h: Tuple[float, float, float]) -> CSRHost:
    """3-D convection-diffusion ``-lap u + b . grad u`` on an N^3 grid.

    ``beta_h`` is the cell value (bx*h, by*h, bz*h).
    """
    n = N * N * N
    cx, cy, cz = (float(b) / 2.0 for b in beta_h)
    idx = np.arange(n, dtype=np.int64)
    ix = idx % N
    iy = (idx // N) % N
    iz = idx // (N * N)
    coeffs = np.empty((n, 7))
    valid = np.empty((n, 7), dtype=bool)
    NN = N * N
    coeffs[:, 0] = -1.0 - cz; valid[:, 0] = iz > 0
    coeffs[:, 1] = -1.0 - cy; valid[:, 1] = iy > 0
    coeffs[:, 2] = -1.0 - cx; valid[:, 2] = ix > 0
    coeffs[:, 3] = 6.0; valid[:, 3] = True
    coeffs[:, 4] = -1.0 + cx; valid[:, 4] = ix < N - 1
    coeffs[:, 5] = -1.0 + cy; valid[:, 5] = iy < N - 1
    coeffs[:, 6] = -1.0 + cz; valid[:, 6] = iz < N - 1
    return _assemble(n, (-NN, -N, -1, 0, 1, N, NN), coeffs, valid)


def block_order(dims: Tuple[int, ...], block: Tuple[int, ...]) -> np.ndarray:
    """Row ordering of a lexicographic grid (x fastest) by blocks: the
    blocks of ``block`` nodes (the last ones clipped) in lexicographic block
    order, the nodes of a block lexicographic inside it.  Returns perm with
    perm[new] = old (grid structure of the inputs; no arithmetic of the
    method)."""
    dims = tuple(int(d) for d in dims)
    block = tuple(int(b) for b in block)
    grids = np.meshgrid(*[np.arange(d) for d in reversed(dims)], indexing="ij")
    # coordinates per old index (lexicographic, x fastest): reversed dims
    coords = [g.ravel() for g in reversed(grids)]
    old = np.zeros_like(coords[0])
    stride = 1
    for c, d in zip(coords, dims):
        old = old + c * stride
        stride *= d
    bkey = np.zeros_like(old)
    inkey = np.zeros_like(old)
    bstride = 1
    istride = 1
    for c, d, b in zip(coords, dims, block):
        nb = -(-d // b)
        bkey = bkey + (c // b) * bstride
        bstride *= nb
        inkey = inkey + (c % b) * istride
        istride *= b
    key = bkey * istride + inkey
    return old[np.argsort(key, kind="stable")].astype(np.int32)


def diag_csr(d: np.ndarray) -> CSRHost:
    """Diagonal matrix diag(d) in CSR."""
    d = np.asarray(d, dtype=np.float64)
    n = d.shape[0]
    return CSRHost(n, np.arange(n + 1, dtype=np.int32),
                   np.arange(n, dtype=np.int32), d.copy())


def ex7_diagonal() -> np.ndarray:
    """Diagonal entries of Example 7 (Section 3.4): n = 5000.

    0.01, 0.02, ..., 0.1 (ten values), 30, 60, and 100, 101, ..., 5087.
    """
    small = np.arange(1, 11) / 100.0
    big = np.arange(100, 5088, dtype=np.float64)
    out = np.concatenate([small, [30.0, 60.0], big])
    assert out.shape[0] == 5000
    return out


def ex11_diagonal(n: int) -> np.ndarray:
    """Diagonal entries i^2/n, i = 1..n (Examples 11 and 12, Sections 4-5)."""
    i = np.arange(1, n + 1, dtype=np.float64)
    return i * i / n


def streams(seed: int) -> List[np.random.Generator]:
    """Four independent generators for (v0, b, field, batch) draws."""
    ss = np.random.SeedSequence(seed)
    return [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(4)]


def uniform_rhs(rng: np.random.Generator, n: int) -> np.ndarray:
    return rng.uniform(-1.0, 1.0, size=n)


def gaussian_v0(rng: np.random.Generator, n: int) -> np.ndarray:
    return rng.standard_normal(n)


def smooth_field(N: int, rng: np.random.Generator, modes: int = 8) -> np.ndarray:
    """Smooth random field on the N x N interior nodes, max |field| = 1.

    sum_{k,l < modes} a_kl cos(2 pi k x + phi_kl) cos(2 pi l y + psi_kl),
    a_kl ~ N(0,1)/(1+k^2+l^2), phases ~ U[0, 2 pi).
    """
    h = 1.0 / (N + 1)
    x = (np.arange(N) + 1) * h
    a = rng.standard_normal((modes, modes))
    phi = rng.uniform(0.0, 2 * np.pi, (modes, modes))
    psi = rng.uniform(0.0, 2 * np.pi, (modes, modes))
    f = np.zeros((N, N))   # f[iy, ix]
    for k in range(modes):
        for l in range(modes):
            amp = a[k, l] / (1.0 + k * k + l * l)
            fx = np.cos(2 * np.pi * k * x + phi[k, l])
            fy = np.cos(2 * np.pi * l * x + psi[k, l])
            f += amp * np.outer(fy, fx)
    f /= np.abs(f).max()
    return f.reshape(-1)


@dataclass
class ProblemSpec:
    """One seeded workload: matrix, right-hand sides and solver settings."""
    name: str
    A: CSRHost
    b: np.ndarray               # (n,) or (nrhs, n)
    v0: np.ndarray              # random start vector of Algorithm 4 step 1(a)
    d: int                      # polynomial degree before added roots
    m: int                      # GMRES restart length
    tol: float
    inner: str = "f64"          # "f64" or "f32" (precision form)
    extra: dict = field(default_factory=dict)


def batch_specs(rng: np.random.Generator, nsys: int = 64,
                side_lo: int = 64, side_hi: int = 512,
                bh_lo: float = 0.1, bh_hi: float = 2.0):
    """Grid sides ~ U{side_lo..side_hi} and beta*h ~ U[bh_lo, bh_hi]."""
    sides = rng.integers(side_lo, side_hi + 1, size=nsys)
    bh = rng.uniform(bh_lo, bh_hi, size=nsys)
    return [(int(s), float(c)) for s, c in zip(sides, bh)]


def problem(name: str, scale: Optional[int] = None) -> ProblemSpec:
    """Seeded workload by name.

    ``cd2d_50``  : 50 x 50, beta*h = 0.5, d = 10, GMRES(50), tol 1e-8.
    ``cd2d_1000``: 1000 x 1000, beta*h = 1.0, d = 40, GMRES(50), tol 1e-10.
    ``cd3d_160`` : 160^3, beta*h = (0.8, 0.4, 0.2), d = 60, FGMRES(50) with
                   an FP32 inner polynomial, tol 1e-10.
    ``cd2d_field_512``: 512 x 512, per-node beta*h = 1 + 0.5 field, d = 30,
                   GMRES(50), tol 1e-10 (adjoint workload).
    ``scale`` overrides the grid side (same seeds, same recipe) for reduced
    versions of a workload.
    """
    if name == "cd2d_50":
        N = scale or 50
        rv, rb, _, _ = streams(101)
        A = cd2d(N, 0.5)
        return ProblemSpec(name, A, uniform_rhs(rb, A.n), gaussian_v0(rv, A.n),
                           d=10, m=50, tol=1e-8, extra={"N": N, "beta_h": 0.5})
    if name == "cd2d_1000":
        N = scale or 1000
        rv, rb, _, _ = streams(102)
        A = cd2d(N, 1.0)
        return ProblemSpec(name, A, uniform_rhs(rb, A.n), gaussian_v0(rv, A.n),
                           d=40, m=50, tol=1e-10, extra={"N": N, "beta_h": 1.0})
    if name == "cd3d_160":
        N = scale or 160
        rv, rb, _, _ = streams(103)
        A = cd3d(N, (0.8, 0.4, 0.2))
        return ProblemSpec(name, A, uniform_rhs(rb, A.n), gaussian_v0(rv, A.n),
                           d=60, m=50, tol=1e-10, inner="f32",
                           extra={"N": N, "beta_h": (0.8, 0.4, 0.2)})
    if name == "cd2d_field_512":
        N = scale or 512
        rv, rb, rf, _ = streams(105)
        fld = smooth_field(N, rf)
        A = cd2d(N, 1.0 + 0.5 * fld)
        xstar = rb.standard_normal(A.n)
        return ProblemSpec(name, A, uniform_rhs(rb, A.n), gaussian_v0(rv, A.n),
                           d=30, m=50, tol=1e-10,
                           extra={"N": N, "xstar": xstar, "field": fld})
    raise KeyError(name)


def batch_problem(nsys: int = 64, seed: int = 104, side_lo: int = 64, side_hi: int = 512,
                  nrhs: int = 4, bh_lo: float = 0.1, bh_hi: float = 2.0):
    """Batch of independent 2-D convection-diffusion systems (the batching
    workload): grid sides ~ U{side_lo..side_hi}, beta*h ~ U[bh_lo, bh_hi],
    nrhs right-hand sides ~ U[-1, 1] and one Gaussian v0 per system.
    Returns a list of (A, B (nrhs x n), v0)."""
    rv, rb, _, rbatch = streams(seed)
    out = []
    for side, bh in batch_specs(rbatch, nsys, side_lo, side_hi, bh_lo, bh_hi):
        A = cd2d(side, bh)
        B = np.stack([uniform_rhs(rb, A.n) for _ in range(nrhs)])
        out.append((A, B, gaussian_v0(rv, A.n)))
    return out


PROBLEMS = ("cd2d_50", "cd2d_1000", "cd3d_160", "cd2d_field_512", "batch_64x4")
