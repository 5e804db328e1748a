"""Multi-root fused sweep (run with -m gpu): Algorithm 3 in FP32 with both
SpMV passes of every conjugate pair in one launch over compact row tiles of
a reordered matrix.  Each row keeps the unfused arithmetic and a symmetric
reordering keeps each row's entries in order, so p(A) v through a plan must
equal ppg_apply_poly bit for bit, and the precision-form solve through a
plan must take the same iterates as ppg_solve_flex."""
import numpy as np
import pytest

import synth
from oracle import poly

from gpu_util import dev_csr, ppg_or_skip, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return ppg_or_skip()


ROOTS = {
    # pairs, real roots between them, a final real root (fused final pair)
    "pairs_then_real": np.array([5 + 2j, 5 - 2j, 3.1, 7 + 1j, 7 - 1j, 2 + 0.5j, 2 - 0.5j,
                                 4.5]),
    # pairs only: the last pair's second pass is omitted (not fused)
    "pairs_only": np.array([5 + 2j, 5 - 2j, 7 + 1j, 7 - 1j, 2 + 0.5j, 2 - 0.5j]),
    # a pair fused with the final real root in its second pass
    "pair_final_real": np.array([6.0, 5 + 2j, 5 - 2j, 3.3]),
}


def _check_bitwise(p, torch, A, plan_kw, roots):
    A32 = dev_csr(p, torch, A, dtype=torch.float32)
    plan = p.SweepPlan(A32, **plan_kw)
    R = p.Roots.from_complex(roots)
    v = to_dev(torch, np.random.default_rng(5).standard_normal(A.n), torch.float32)
    ref = p.apply_poly(A32, R, v)
    got = plan.apply_poly(R, v)
    torch.cuda.synchronize()
    assert torch.isfinite(ref).all()
    assert torch.equal(got, ref)
    return plan.info()


@pytest.mark.parametrize("name", sorted(ROOTS))
def test_sweep_3d_blocked_bit_identical(env, name):
    """3-D 40^3 in 16^3 blocks (ragged last blocks; tiles of 4096 rows)."""
    p, torch = env
    A = synth.cd3d(40, (0.8, 0.4, 0.2))
    perm = synth.block_order((40, 40, 40), (16, 16, 16))
    info = _check_bitwise(p, torch, A, dict(tile_rows=4096, perm=perm), ROOTS[name])
    assert info["fused"] == 1 and info["halo_fraction"] <= 0.6


def test_sweep_breadth_first_ordering_and_ragged_tail(env):
    """No ordering given: breadth-first parts; n = 70^2 is not a multiple of
    the tile, a 2-D grid."""
    p, torch = env
    A = synth.cd2d(70, 1.0)
    info = _check_bitwise(p, torch, A, dict(tile_rows=1024), ROOTS["pairs_then_real"])
    assert info["ntiles"] == -(-A.n // 1024)
    assert info["fused"] == 1


def _banded_random(n, seed, band, long_row, long_len, empty_row):
    """Random banded pattern: rows of 1-12 nonzeros within +-band of the
    diagonal (unsorted draws, stored sorted), one long row, one empty row,
    a strong diagonal."""
    rng = np.random.default_rng(seed)
    rows = []
    for i in range(n):
        if i == empty_row:
            rows.append(np.zeros(0, dtype=np.int64))
            continue
        k = long_len if i == long_row else int(rng.integers(1, 13))
        lo, hi = max(0, i - band), min(n, i + band + 1)
        cols = rng.choice(np.arange(lo, hi), size=min(k, hi - lo), replace=False)
        rows.append(np.unique(np.concatenate([cols, [i]])))
    rowptr = np.zeros(n + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    colind = np.concatenate(rows).astype(np.int32)
    vals = rng.standard_normal(colind.size) * 0.1
    for i, r in enumerate(rows):
        j = np.searchsorted(r, i)
        if j < len(r) and r[j] == i:
            vals[rowptr[i] + j] = 4.0
    return synth.CSRHost(n, rowptr.astype(np.int32), colind, vals)


def test_sweep_irregular_rows_and_unfused_plan(env):
    """Banded random pattern with rows of 1-12 nonzeros, one row of 600
    nonzeros and an empty row: the fused plan and a plan with fuse = 0 (the
    plain chain on the reordered matrix) both equal ppg_apply_poly."""
    p, torch = env
    A = _banded_random(3000, 11, 40, 1700, 600, 5)
    infos = [_check_bitwise(p, torch, A, dict(tile_rows=256, fuse=f), ROOTS["pairs_then_real"])
             for f in (False, True)]
    assert infos[0]["fused"] == 0 and infos[1]["fused"] == 1


def test_sweep_halo_guard_falls_back_to_the_unfused_chain(env):
    """Lexicographic rows of a 3-D grid in 4096-row tiles: each tile reaches
    two whole planes beyond it, the halos exceed 60 % of n and the plan does
    not fuse (the result is still exact)."""
    p, torch = env
    A = synth.cd3d(40, (0.8, 0.4, 0.2))
    info = _check_bitwise(p, torch, A, dict(tile_rows=4096, perm=np.arange(A.n)),
                          ROOTS["pairs_only"])
    assert info["halo_fraction"] > 0.6 and info["fused"] == 0


def test_solve_flex_sweep_same_iterates_as_solve_flex(env):
    """The precision form at 40^3 with the workload's own degree-60
    polynomial: through a blocked plan the solve gives exactly what
    ppg_solve_flex gives."""
    p, torch = env
    P = synth.problem("cd3d_160", scale=40)
    A64 = dev_csr(p, torch, P.A)
    A32 = A64.astype(torch.float32)
    R = p.build_poly(A64, P.d, to_dev(torch, P.v0))
    plan = p.SweepPlan(A32, 4096, perm=synth.block_order((40, 40, 40), (16, 16, 16)))
    assert plan.info()["fused"] == 1
    b = to_dev(torch, P.b)
    x_ref, s_ref = p.solve_flex(A64, A32, b, R, P.m, P.tol)
    x, s = p.solve_flex_sweep(A64, plan, b, R, P.m, P.tol)
    torch.cuda.synchronize()
    assert s["iters"] == s_ref["iters"] and s["cycles"] == s_ref["cycles"]
    assert torch.equal(x, x_ref)
    assert s["true_relres"] <= P.tol


def test_sweep_full_size_160_bit_identical(env):
    """The precision workload's 160^3 matrix in 16^3 blocks with its own
    degree-60 polynomial: bit-identical to the unfused chain."""
    p, torch = env
    P = synth.problem("cd3d_160")
    A64 = dev_csr(p, torch, P.A)
    R = p.build_poly(A64, P.d, to_dev(torch, P.v0))
    A32 = A64.astype(torch.float32)
    del A64
    plan = p.SweepPlan(A32, 4096, perm=synth.block_order((160, 160, 160), (16, 16, 16)))
    info = plan.info()
    assert info["fused"] == 1 and info["ntiles"] == 1000
    v = to_dev(torch, np.random.default_rng(9).standard_normal(P.A.n), torch.float32)
    ref = p.apply_poly(A32, R, v)
    got = plan.apply_poly(R, v)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
