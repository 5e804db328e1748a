"""Edge cases of the device path (run with -m gpu).

* CSR arrays that do not start on a 16-byte boundary (views one element into
  a buffer): the staged root-step kernel (systems above 32,768 rows) then
  stages values and column indices one element at a time instead of in
  16-byte granules.  Staging only moves data,
  so y = A x, p(A) v and phi(A) v must be bit-identical to the aligned run,
  in FP64 and FP32, including matrices with rows longer than one staging
  chunk and empty rows.
* The batching form with a degree-one polynomial (p(A) = 1/theta, the
  elementwise step) against the oracle's FGMRES with the same root.
* The batching form on systems so small that the GMRES(d) construction
  breaks down (n < d): per-system degrees differ, the shorter step tables are
  padded with no-ops; roots, iteration counts and solutions against the
  oracle.
* The end-to-end call from host memory with NumPy or pinned inputs.
* Degenerate sizes: a matrix without nonzeros and a 1 x 1 matrix.
"""
import numpy as np
import pytest

import synth
from oracle import gmres, poly

from gpu_util import dev_csr, ppg_or_skip, random_csr, to_dev

pytestmark = pytest.mark.gpu

ROOTS = np.array([4.0, 3 + 1j, 3 - 1j, 2.5, 2 + 0.5j, 2 - 0.5j, 3.3], dtype=complex)


@pytest.fixture(scope="module")
def env():
    return ppg_or_skip()


def _unaligned(torch, t, offset=1):
    """The same values in a view that starts `offset` elements into a fresh
    buffer (4 or 8 bytes past a 256-byte aligned allocation)."""
    buf = torch.empty(t.numel() + offset, dtype=t.dtype, device=t.device)
    view = buf[offset:]
    view.copy_(t)
    assert view.data_ptr() % 16 != 0
    return view


def _matrices():
    # at most 32,768 rows: the direct kernel (no staging; alignment must not
    # matter either); above: the staged kernel, whose copies fall back to
    # one element at a time for arrays off a 16-byte boundary
    yield "cd2d_37", synth.cd2d(37, 0.7)
    yield "cd3d_13", synth.cd3d(13, (0.8, 0.4, 0.2))
    yield "random_long_empty", random_csr(3001, 1, long_rows={5: 2500, 700: 4100},
                                          empty_rows={17, 1000, 3000})
    yield "cd3d_34", synth.cd3d(34, (0.8, 0.4, 0.2))
    yield "random_long_empty_40k", random_csr(40001, 3, long_rows={5: 2500, 700: 4100,
                                                                   33000: 9000},
                                              empty_rows={17, 1000, 40000})


@pytest.mark.parametrize("which", ["vals", "colind", "both"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("mname,A", list(_matrices()))
def test_unaligned_csr_arrays_bitwise(env, mname, A, dtype, which):
    p, torch = env
    tdt = torch.float64 if dtype == "f64" else torch.float32
    Ad = dev_csr(p, torch, A, dtype=tdt)
    ci = _unaligned(torch, Ad.colind) if which in ("colind", "both") else Ad.colind
    vv = _unaligned(torch, Ad.vals) if which in ("vals", "both") else Ad.vals
    Au = p.CSR(Ad.rowptr, ci, vv)
    R = p.Roots.from_complex(ROOTS)
    v = to_dev(torch, np.random.default_rng(11).standard_normal(A.n), tdt)
    assert torch.equal(p.spmv(Ad, v), p.spmv(Au, v))
    assert torch.equal(p.apply_poly(Ad, R, v), p.apply_poly(Au, R, v))
    assert torch.equal(p.apply_phi(Ad, R, v), p.apply_phi(Au, R, v))


def _batched(p, torch, probs, d, m, tol):
    As = [dev_csr(p, torch, A) for A, _, _ in probs]
    Bs = [to_dev(torch, np.ascontiguousarray(B)) for _, B, _ in probs]
    v0s = [to_dev(torch, v0) for _, _, v0 in probs]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        Xs, info = p.solve_batched(As, Bs, v0s, d, m, tol)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in Xs], info


def _check_against_oracle(probs, Xs, info, d, m, tol):
    for s, (A, B, v0) in enumerate(probs):
        As = A.to_scipy()
        orc = poly.build_poly(As, d, v0)
        R = info["roots"][s]
        assert R.n_total == orc.roots.size, (s, A.n, R.n_total, orc.roots.size)
        got = R.complex()
        for t in orc.roots:
            assert np.min(np.abs(got - t)) <= 1e-8 * abs(t)
        for k in range(B.shape[0]):
            rel = np.linalg.norm(B[k] - As @ Xs[s][k]) / np.linalg.norm(B[k])
            assert rel <= tol, (s, k, rel)
            xo, so = gmres.fgmres_p(As, got, B[k], m, tol, inner="f32")
            assert abs(int(info["iters"][s, k]) - so.iters) <= 2, (s, k)
            assert np.linalg.norm(Xs[s][k] - xo) <= 1e-6 * np.linalg.norm(xo)


def test_batched_degree_one_polynomial(env):
    p, torch = env
    probs = synth.batch_problem(nsys=5, seed=21, side_lo=6, side_hi=12, nrhs=4)
    d, m, tol = 1, 20, 1e-10
    Xs, info = _batched(p, torch, probs, d, m, tol)
    assert info["status"] == 0
    assert all(info["roots"][s].n_total == 1 for s in range(len(probs)))
    _check_against_oracle(probs, Xs, info, d, m, tol)


def test_batched_mixed_degrees_with_breakdown(env):
    p, torch = env
    # sides 2..5 (n = 4..25) with d = 12: the smallest systems exhaust their
    # Krylov space before step d, so their polynomials are shorter
    probs = synth.batch_problem(nsys=8, seed=22, side_lo=2, side_hi=5, nrhs=4)
    d, m, tol = 12, 20, 1e-10
    Xs, info = _batched(p, torch, probs, d, m, tol)
    assert info["status"] == 0
    degrees = {info["roots"][s].n_orig for s in range(len(probs))}
    assert len(degrees) > 1, degrees
    _check_against_oracle(probs, Xs, info, d, m, tol)


def test_solve_host_numpy_and_pinned_inputs(env):
    """The end-to-end call from host memory: NumPy arrays (page-locked by
    the call) and tensors already in pinned memory give the same solution,
    whose true residual meets the tolerance; iterations against the
    oracle's PP-GMRES with the same roots."""
    p, torch = env
    P = synth.problem("cd2d_50")
    x1, R1, s1 = p.solve_host(P.A.rowptr, P.A.colind, P.A.vals, P.b, P.v0, P.d, P.m, P.tol)
    pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
              for a in (P.A.rowptr, P.A.colind, P.A.vals, P.b, P.v0)]
    x2, R2, s2 = p.solve_host(*pinned, P.d, P.m, P.tol)
    assert np.array_equal(x1, x2)
    assert np.array_equal(R1.complex(), R2.complex())
    As = P.A.to_scipy()
    rel = np.linalg.norm(P.b - As @ x1) / np.linalg.norm(P.b)
    assert s1["converged"] == 1 and rel <= P.tol
    _, so = gmres.pp_gmres(As, R1.complex(), P.b, P.m, P.tol)
    assert abs(s1["iters"] - so.iters) <= 2


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_empty_and_one_by_one_matrices(env, dtype):
    """Degenerate sizes: a 5 x 5 matrix with no nonzeros (y = A x = 0, and
    p(A) v reduces to the constant and linear terms the roots leave) and a
    1 x 1 matrix (p(A) v is the scalar polynomial); against the oracle's
    Algorithm 3 (float32 for FP32) and y = A x."""
    p, torch = env
    tdt = torch.float64 if dtype == "f64" else torch.float32
    R = p.Roots.from_complex(ROOTS)
    cases = [
        synth.CSRHost(5, np.zeros(6, np.int32), np.zeros(0, np.int32), np.zeros(0)),
        synth.CSRHost(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([3.0])),
    ]
    for A in cases:
        Ad = dev_csr(p, torch, A, dtype=tdt)
        v = np.random.default_rng(A.n).standard_normal(A.n)
        vd = to_dev(torch, v, tdt)
        As = A.to_scipy()
        y = p.spmv(Ad, vd).cpu().numpy().astype(np.float64)
        assert np.allclose(y, As @ v.astype(y.dtype), rtol=1e-6, atol=0)
        got = p.apply_poly(Ad, R, vd).cpu().numpy().astype(np.float64)
        if dtype == "f64":
            ref = poly.apply_p(As, ROOTS, v)
            assert np.allclose(got, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
        else:
            ref = gmres.apply_p32(As.astype(np.float32), gmres._roots32(ROOTS),
                                  v.astype(np.float32)).astype(np.float64)
            assert np.allclose(got, ref, rtol=1e-5, atol=1e-5 * np.abs(ref).max())


def _block_diag_with_identity(A, n_extra, scale=4.0):
    """A (+) scale I: the first block's rows read only the first block's
    entries of x, so they compute exactly what A alone computes."""
    n = A.n + n_extra
    rowptr = np.concatenate([A.rowptr, A.rowptr[-1] + np.arange(1, n_extra + 1)]).astype(np.int32)
    colind = np.concatenate([A.colind, A.n + np.arange(n_extra)]).astype(np.int32)
    vals = np.concatenate([A.vals, np.full(n_extra, scale)])
    return synth.CSRHost(n, rowptr, colind, vals)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("side", [50, 128])
def test_small_system_and_l2_resident_steps_are_bitwise(env, side, dtype):
    """Systems of up to 32,768 rows run the direct-read step with eight
    entries preloaded and no register bound; the same matrix as the first
    block of a 70,000-row block-diagonal system (held in L2) runs the
    direct-read step with three or four entries preloaded under a 32-register
    bound.  p(A) v and phi(A) v on the first block must agree bit for bit,
    for root sets with real roots, pairs and a final real root, and with a
    degree-one polynomial."""
    p, torch = env
    tdt = torch.float64 if dtype == "f64" else torch.float32
    A = synth.cd2d(side, 0.7)
    big = _block_diag_with_identity(A, 70000 - A.n)
    As, Ab = dev_csr(p, torch, A, dtype=tdt), dev_csr(p, torch, big, dtype=tdt)
    rng = np.random.default_rng(side)
    v = rng.standard_normal(A.n)
    vb = np.concatenate([v, rng.standard_normal(big.n - A.n)])
    for roots in (ROOTS, ROOTS[:6], np.array([3.0 + 0j]), np.array([3 + 1j, 3 - 1j])):
        R = p.Roots.from_complex(roots)
        ys = p.apply_poly(As, R, to_dev(torch, v, tdt))
        yb = p.apply_poly(Ab, R, to_dev(torch, vb, tdt))
        assert torch.equal(ys, yb[: A.n]), roots
        fs = p.apply_phi(As, R, to_dev(torch, v, tdt))
        fb = p.apply_phi(Ab, R, to_dev(torch, vb, tdt))
        assert torch.equal(fs, fb[: A.n]), roots
