"""Batching form through the C ABI (run with -m gpu): every system's roots
against the oracle's construction, every solve's true residual, iteration
counts against the oracle's float32-inner flexible GMRES, and the solution
against the oracle's.  Small batches span several 256-row tiles per system
with ragged ends; the full batch (64 systems x 4 right-hand sides) is
checked by its true residuals and sampled roots."""
import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

import synth
from oracle import gmres, poly

from gpu_util import dev_csr, ppg_or_skip, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return ppg_or_skip()


def _roots_close(got, ref, tol):
    C = np.abs(got[:, None] - ref[None, :])
    r, c = linear_sum_assignment(C)
    return np.max(C[r, c] / np.abs(ref[c])) <= tol


def _run(p, torch, probs, d, m, tol, nrhs, side_stream, **kw):
    As = [dev_csr(p, torch, A) for A, _, _ in probs]
    Bs = [to_dev(torch, np.ascontiguousarray(B[:nrhs])) for _, B, _ in probs]
    v0s = [to_dev(torch, v0) for _, _, v0 in probs]
    if side_stream:
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            Xs, info = p.solve_batched(As, Bs, v0s, d, m, tol, **kw)
        torch.cuda.current_stream().wait_stream(s)
    else:
        Xs, info = p.solve_batched(As, Bs, v0s, d, m, tol, **kw)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in Xs], info


@pytest.mark.parametrize("nrhs,side_stream", [(4, True), (1, False)])
def test_batched_small_matches_oracle_per_solve(env, nrhs, side_stream):
    p, torch = env
    probs = synth.batch_problem(nsys=6, seed=7, side_lo=9, side_hi=40, nrhs=4)
    d, m, tol = 8, 20, 1e-10
    Xs, info = _run(p, torch, probs, d, m, tol, nrhs, side_stream)
    assert info["status"] == 0
    for s, (A, B, v0) in enumerate(probs):
        As = A.to_scipy()
        orc = poly.build_poly(As, d, v0)
        R = info["roots"][s]
        assert R.n_total == orc.roots.size
        assert _roots_close(R.complex(), orc.roots, 1e-9)
        for k in range(nrhs):
            x = Xs[s][k]
            b = B[k]
            rel = np.linalg.norm(b - As @ x) / np.linalg.norm(b)
            assert rel <= tol
            assert abs(info["relres"][s, k] - rel) <= 1e-3 * tol + 0.5 * rel
            xo, so = gmres.fgmres_p(As, R.complex(), b, m, tol, inner="f32")
            assert abs(int(info["iters"][s, k]) - so.iters) <= 2
            assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)


def test_batched_full_size_64_systems_4_rhs(env):
    """The batching workload: 64 systems, sides ~ U{64..512}, beta*h ~
    U[0.1, 2], 4 right-hand sides, d = 20, FGMRES(30), tol 1e-10."""
    p, torch = env
    probs = synth.batch_problem(nsys=64, seed=104)
    d, m, tol = 20, 30, 1e-10
    Xs, info = _run(p, torch, probs, d, m, tol, 4, True)
    assert info["status"] == 0
    worst = 0.0
    for s, (A, B, _) in enumerate(probs):
        As = A.to_scipy()
        for k in range(4):
            rel = np.linalg.norm(B[k] - As @ Xs[s][k]) / np.linalg.norm(B[k])
            worst = max(worst, rel)
    assert worst <= tol
    # sampled roots: the two smallest systems against the oracle
    order = np.argsort([A.n for A, _, _ in probs])[:2]
    for s in order:
        A, _, v0 = probs[s]
        orc = poly.build_poly(A.to_scipy(), d, v0)
        assert _roots_close(info["roots"][s].complex(), orc.roots, 1e-8)


@pytest.mark.parametrize("side_stream", [True, False])
def test_batched_mid_size_persistent_launch_against_graph_and_oracle(env, side_stream):
    """Eight systems with sides 64-200 (full 8-tile CGS2 units, up to 157
    tiles per system), 4 right-hand sides: the persistent launch gives
    exactly the per-cycle graph's results (the same arithmetic, phase by
    phase), and every one of the 32 solves matches the oracle's float32-inner
    FGMRES: iterations within 2, solution within 1e-6."""
    p, torch = env
    probs = synth.batch_problem(nsys=8, seed=41, side_lo=64, side_hi=200, nrhs=4)
    d, m, tol = 12, 30, 1e-10
    Xp, ip = _run(p, torch, probs, d, m, tol, 4, side_stream, persistent=True)
    Xg, ig = _run(p, torch, probs, d, m, tol, 4, side_stream, persistent=False)
    assert ip["status"] == 0 and ig["status"] == 0
    assert ip["stats"]["cycles"] == ig["stats"]["cycles"]
    assert np.array_equal(ip["iters"], ig["iters"])
    for s in range(len(probs)):
        assert np.array_equal(Xp[s], Xg[s])
    for s, (A, B, v0) in enumerate(probs):
        As = A.to_scipy()
        R = ip["roots"][s]
        for k in range(4):
            rel = np.linalg.norm(B[k] - As @ Xp[s][k]) / np.linalg.norm(B[k])
            assert rel <= tol
            xo, so = gmres.fgmres_p(As, R.complex(), B[k], m, tol, inner="f32")
            assert abs(int(ip["iters"][s, k]) - so.iters) <= 2
            assert np.linalg.norm(Xp[s][k] - xo) <= 1e-6 * np.linalg.norm(xo)


def test_batched_persistent_wait_limit_returns_timeout(env):
    """Every grid-wide wait of the persistent launch is bounded: with a zero
    limit the first barrier's waits run out, every CTA returns and the call
    reports PPG_ERR_TIMEOUT; the context stays usable and the next call,
    with the default limit, solves the batch."""
    p, torch = env
    probs = synth.batch_problem(nsys=6, seed=7, side_lo=9, side_hi=40, nrhs=4)
    with pytest.raises(p.PPGError) as ei:
        _run(p, torch, probs, 8, 20, 1e-10, 4, True, wait_timeout_ms=0.0)
    assert ei.value.code == -10
    Xs, info = _run(p, torch, probs, 8, 20, 1e-10, 4, True)
    assert info["status"] == 0
    for s, (A, B, _) in enumerate(probs):
        for k in range(4):
            rel = np.linalg.norm(B[k] - A.to_scipy() @ Xs[s][k]) / np.linalg.norm(B[k])
            assert rel <= 1e-10
