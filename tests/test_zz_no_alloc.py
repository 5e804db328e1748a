"""ppg_apply_poly_noalloc: p(A) v for callers that cannot allocate device
memory at call time (their GPU memory is held by another allocator, or an
allocation would synchronise the device or could fail mid-work).  It must
give what ppg_apply_poly gives, call after call, from its fixed work area.

This file is named to be collected last, so a run that stops at the first
failure has already run every other test.  It also passes alone in a fresh
process (the first call on the device sets up the work area's address).
"""
import ctypes as C

import numpy as np
import pytest

import synth

from gpu_util import dev_csr, ppg_or_skip, to_dev

pytestmark = pytest.mark.gpu


def _call_noalloc(p, torch, Ad, R, v, y):
    from paper_1911_07065_gb300._binding import lib
    return lib.ppg_apply_poly_noalloc(Ad.ref(), R.ref(), C.c_void_p(v.data_ptr()),
                                      C.c_void_p(y.data_ptr()),
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_apply_poly_on_two_calls_in_a_row():
    p, torch = ppg_or_skip()
    A = synth.cd2d(400, 0.7)                  # n = 160,000: many row tiles
    Ad = dev_csr(p, torch, A)
    rng = np.random.default_rng(21)
    cases = [
        np.array([4.0, 3 + 1j, 3 - 1j, 2.5, 2 + 0.5j, 2 - 0.5j, 3.3, 1.7]),  # pairs, real end
        np.array([6.5, 0.4, 3.1, 5.2, 1.1, 7.3, 2.2], dtype=complex),        # all real
    ]
    for roots in cases:
        R = p.Roots.from_complex(roots)
        v = to_dev(torch, rng.standard_normal(A.n))
        ref = p.apply_poly(Ad, R, v)
        y = torch.full_like(v, float("nan"))
        rc = _call_noalloc(p, torch, Ad, R, v, y)
        assert rc == 0, p.lib.ppg_strerror(rc)
        torch.cuda.synchronize()
        # the same kernels in the same order: within the parity tolerance
        # of the test suite (1e-11 relative), in practice bit-identical
        err = torch.linalg.norm(y - ref).item()
        assert err <= 1e-11 * torch.linalg.norm(ref).item()
        assert torch.isfinite(y).all()


def test_noalloc_float32_and_size_limit():
    p, torch = ppg_or_skip()
    from paper_1911_07065_gb300._binding import NOALLOC_MAX_N
    A = synth.cd3d(30, (0.8, 0.4, 0.2))
    A32 = dev_csr(p, torch, A, dtype=torch.float32)
    R = p.Roots.from_complex(np.array([7.0, 4 + 2j, 4 - 2j, 1.5], dtype=complex))
    v = to_dev(torch, np.random.default_rng(22).standard_normal(A.n), torch.float32)
    ref = p.apply_poly(A32, R, v)
    y = torch.empty_like(v)
    assert _call_noalloc(p, torch, A32, R, v, y) == 0
    torch.cuda.synchronize()
    assert torch.linalg.norm(y - ref).item() <= 1e-6 * torch.linalg.norm(ref).item()
    # one row more than the work area holds: rejected before any launch
    n = NOALLOC_MAX_N + 1
    big = synth.diag_csr(np.full(n, 2.0))
    Bd = dev_csr(p, torch, big)
    vb = torch.ones(n, dtype=torch.float64, device="cuda")
    yb = torch.zeros_like(vb)
    assert _call_noalloc(p, torch, Bd, R, vb, yb) == -9     # PPG_ERR_TOO_LARGE
    torch.cuda.synchronize()
    assert torch.all(yb == 0)
