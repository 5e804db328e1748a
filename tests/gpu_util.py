"""Shared helpers for the GPU parity tests (imported by tests only)."""
import numpy as np
import pytest

import synth


def ppg_or_skip():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_07065_gb300 import build as B
    B.build()
    import paper_1911_07065_gb300 as p
    return p, torch


def dev_csr(p, torch, A: synth.CSRHost, dtype=None):
    dtype = dtype or torch.float64
    return p.CSR.from_host(A.rowptr, A.colind, A.vals, device="cuda", dtype=dtype)


def to_dev(torch, x, dtype=None):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype=dtype or torch.float64)


def p_norm_estimate(apply_fn, apply_t_fn, n, iters=30, seed=0):
    """||p(A)||_2 by power iteration on p(A)^T p(A) (oracle side)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(n)
    v /= np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = apply_t_fn(apply_fn(v))
        lam = np.linalg.norm(w)
        v = w / lam
    return np.sqrt(lam)


def random_csr(n, seed, max_row=12, long_rows=(), empty_rows=(), diag=4.0):
    """Random sparse matrix with variable row lengths, optional long rows
    (more nonzeros than one staging chunk) and empty rows.  Above 5000 rows
    the columns of a row are drawn with replacement and deduplicated (a row
    may then hold fewer than its drawn length)."""
    rng = np.random.default_rng(seed)
    rows = []
    for i in range(n):
        if i in empty_rows:
            rows.append(np.zeros(0, dtype=np.int64))
            continue
        k = int(long_rows[i]) if i in long_rows else int(rng.integers(1, max_row + 1))
        if n > 5000:
            cols = rng.integers(0, n, size=min(k, n))
        else:
            cols = rng.choice(n, size=min(k, n), replace=False)
        cols = np.unique(np.concatenate([cols, [i]]))
        rows.append(cols)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    colind = np.concatenate(rows).astype(np.int32)
    vals = rng.standard_normal(colind.size) * 0.1
    # strengthen the diagonal
    for i, r in enumerate(rows):
        j = np.searchsorted(r, i)
        if j < len(r) and r[j] == i:
            vals[rowptr[i] + j] = diag
    return synth.CSRHost(n, rowptr.astype(np.int32), colind, vals)
