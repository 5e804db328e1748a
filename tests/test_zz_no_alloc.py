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


def test_noalloc_rejects_nonfinite_roots_like_apply_poly():
    p, torch = ppg_or_skip()
    A = synth.cd2d(20, 0.5)
    Ad = dev_csr(p, torch, A)
    v = to_dev(torch, np.random.default_rng(23).standard_normal(A.n))
    for bad in (np.inf, -np.inf, np.nan):
        R = p.Roots.from_complex(np.array([3.0, bad, 2.0], dtype=complex))
        R.im[1] = 0.0                        # a "real" root of +-inf or NaN
        y = torch.zeros_like(v)
        assert _call_noalloc(p, torch, Ad, R, v, y) == -1          # PPG_ERR_ARG
        y2 = torch.zeros_like(v)
        rc = p.lib.ppg_apply_poly(Ad.ref(), R.ref(), C.c_void_p(v.data_ptr()),
                                  C.c_void_p(y2.data_ptr()),
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == -1
        torch.cuda.synchronize()
        assert torch.all(y == 0) and torch.all(y2 == 0)


class _DefaultPool:
    """The device's default stream-ordered memory pool, read through the
    driver API: the pool the library's other entry points allocate from."""
    USED_MEM_CURRENT, USED_MEM_HIGH = 7, 8      # CUmemPool_attribute

    def __init__(self, torch):
        self.cu = C.CDLL("libcuda.so.1")
        dev = C.c_int(0)
        assert self.cu.cuDeviceGet(C.byref(dev), torch.cuda.current_device()) == 0
        self.pool = C.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(C.byref(self.pool), dev) == 0

    def get(self, attr):
        v = C.c_uint64(0)
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, C.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = C.c_uint64(0)     # resets the high-water mark to the current use
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH, C.byref(zero)) == 0


def test_noalloc_allocates_nothing():
    """The defining contract: around a synchronised call, the default pool's
    high-water mark of used memory does not rise and the device's free memory
    does not drop.  The allocating entry point, run the same way, does raise
    the mark, which shows that the probe sees stream-ordered allocations."""
    p, torch = ppg_or_skip()
    A = synth.cd2d(300, 0.7)
    Ad = dev_csr(p, torch, A)
    R = p.Roots.from_complex(np.array([4.0, 3 + 1j, 3 - 1j, 2.5, 1.7]))
    v = to_dev(torch, np.random.default_rng(24).standard_normal(A.n))
    y = torch.empty_like(v)
    stream = torch.cuda.current_stream()
    assert _call_noalloc(p, torch, Ad, R, v, y) == 0          # address set up
    torch.cuda.synchronize()
    pool = _DefaultPool(torch)

    pool.reset_high()
    used0 = pool.get(pool.USED_MEM_CURRENT)
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        assert _call_noalloc(p, torch, Ad, R, v, y) == 0
        stream.synchronize()
    assert pool.get(pool.USED_MEM_HIGH) == used0
    assert torch.cuda.mem_get_info()[0] == free0

    # positive control: ppg_apply_poly takes its work vectors from the pool
    pool.reset_high()
    y2 = torch.empty_like(v)
    rc = p.lib.ppg_apply_poly(Ad.ref(), R.ref(), C.c_void_p(v.data_ptr()),
                              C.c_void_p(y2.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert rc == 0
    stream.synchronize()
    assert pool.get(pool.USED_MEM_HIGH) >= used0 + 3 * 8 * A.n
    assert torch.equal(y, y2)


def test_noalloc_on_a_matrix_streamed_from_hbm():
    """3-D 100^3 in FP64 (n = 1e6, within the work area's limit): the
    matrix does not fit in L2 with the chain's vectors, so both entry points
    stream it; ppg_apply_poly sets the L2 set-aside for the chain's leading
    rows, the no-allocation call only uses the set-aside in place.  The L2
    hints differ, the arithmetic does not: the results are bit-identical."""
    p, torch = ppg_or_skip()
    A = synth.cd3d(100, (0.8, 0.4, 0.2))
    Ad = dev_csr(p, torch, A)
    R = p.Roots.from_complex(np.array([4.0, 3 + 1j, 3 - 1j, 2.5, 2 + 0.5j, 2 - 0.5j, 3.3]))
    v = to_dev(torch, np.random.default_rng(23).standard_normal(A.n))
    ref = p.apply_poly(Ad, R, v)
    y = torch.full_like(v, float("nan"))
    rc = _call_noalloc(p, torch, Ad, R, v, y)
    assert rc == 0, p.lib.ppg_strerror(rc)
    torch.cuda.synchronize()
    assert torch.equal(y, ref)
