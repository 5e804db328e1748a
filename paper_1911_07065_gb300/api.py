"""PyTorch-facing API over the C ABI (argument marshalling only).

Device vectors are torch tensors on a CUDA device; every computation is a
call into libppgmres on the current torch CUDA stream.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Tuple

import numpy as np
import torch

from ._binding import (PPG_F32, PPG_F64, Roots, check, default_opts, lib, ppg_roots,
                       ppg_csr, ppg_poly_check, ppg_stats, ppg_sweep_info, csr_validate_host,
                       _dp)


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t: torch.Tensor):
    return C.c_void_p(t.data_ptr())


def _need_cuda(*ts):
    for t in ts:
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
            raise ValueError("expected contiguous CUDA tensors")


class CSR:
    """CSR matrix on the device: int32 rowptr/colind, float64 or float32 vals."""

    def __init__(self, rowptr: torch.Tensor, colind: torch.Tensor, vals: torch.Tensor):
        _need_cuda(rowptr, colind, vals)
        if rowptr.dtype != torch.int32 or colind.dtype != torch.int32:
            raise ValueError("rowptr/colind must be int32")
        if vals.dtype not in (torch.float64, torch.float32):
            raise ValueError("vals must be float64 or float32")
        self.rowptr, self.colind, self.vals = rowptr, colind, vals
        self.n = rowptr.numel() - 1
        self.nnz = colind.numel()
        self.s = ppg_csr(self.n, self.nnz, rowptr.data_ptr(), colind.data_ptr(),
                         vals.data_ptr(), PPG_F64 if vals.dtype == torch.float64 else PPG_F32)

    @property
    def dtype(self):
        return self.vals.dtype

    @classmethod
    def from_host(cls, rowptr, colind, vals, device="cuda", dtype=torch.float64,
                  validate=True) -> "CSR":
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        colind = np.ascontiguousarray(colind, dtype=np.int32)
        if validate:
            rc = csr_validate_host(rowptr, colind)
            check(rc, "ppg_csr_validate_host")
        return cls(torch.from_numpy(rowptr).to(device), torch.from_numpy(colind).to(device),
                   torch.from_numpy(np.asarray(vals)).to(device=device, dtype=dtype))

    def with_vals(self, vals: torch.Tensor) -> "CSR":
        return CSR(self.rowptr, self.colind, vals)

    def astype(self, dtype) -> "CSR":
        return CSR(self.rowptr, self.colind, self.vals.to(dtype))

    def ref(self):
        return C.byref(self.s)

    def transpose(self, with_perm: bool = False, stream=None):
        rp = torch.empty(self.n + 1, dtype=torch.int32, device=self.vals.device)
        ci = torch.empty(self.nnz, dtype=torch.int32, device=self.vals.device)
        vv = torch.empty(self.nnz, dtype=self.vals.dtype, device=self.vals.device)
        perm = torch.empty(self.nnz, dtype=torch.int32, device=self.vals.device) if with_perm else None
        check(lib.ppg_csr_transpose(self.ref(), _ptr(rp), _ptr(ci), _ptr(vv),
                                    _ptr(perm) if perm is not None else None, _stream(stream)),
              "ppg_csr_transpose")
        T = CSR(rp, ci, vv)
        return (T, perm) if with_perm else T


def build_poly(A: CSR, d: int, v0: torch.Tensor, stability_control: bool = True,
               return_hbar: bool = False, capacity: Optional[int] = None, stream=None):
    """Algorithm 4 step 1 on the device; returns Roots (and Hbar)."""
    _need_cuda(v0)
    if v0.dtype != torch.float64:
        raise ValueError("v0 must be float64")
    cap = capacity or max(16, 4 * d)
    r = Roots(cap)
    H = np.zeros((d + 1) * d)
    o = default_opts(stability_control=int(bool(stability_control)))
    rc = lib.ppg_build_poly(A.ref(), d, _ptr(v0), C.byref(o), r.ref(), _dp(H), _stream(stream))
    if rc == -6 and capacity is None:
        return build_poly(A, d, v0, stability_control, return_hbar, r.s.n_total + 8, stream)
    check(rc, "ppg_build_poly")
    Hbar = H.reshape(d, d + 1).T.copy()
    return (r, Hbar) if return_hbar else r


def build_poly_checked(A: CSR, d: int, v0: torch.Tensor, stch_tol: float,
                       b: Optional[torch.Tensor] = None, d_min: int = 1,
                       stability_control: bool = True, capacity: Optional[int] = None,
                       stream=None):
    """Algorithm 4 step 1 with the stability check of Section 3.5 (degree
    halved while StCh > stch_tol, down to d_min).  Returns (Roots, info) with
    info = {d_requested, d_chosen, n_tried, stch, stch_first}."""
    _need_cuda(v0)
    if v0.dtype != torch.float64 or (b is not None and b.dtype != torch.float64):
        raise ValueError("v0 and b must be float64")
    cap = capacity or max(16, 4 * d)
    r = Roots(cap)
    info = ppg_poly_check()
    o = default_opts(stability_control=int(bool(stability_control)))
    rc = lib.ppg_build_poly_checked(A.ref(), d, _ptr(v0), _ptr(b) if b is not None else None,
                                    float(stch_tol), int(d_min), C.byref(o), r.ref(),
                                    C.byref(info), _stream(stream))
    if rc == -6 and capacity is None:
        return build_poly_checked(A, d, v0, stch_tol, b, d_min, stability_control,
                                  r.s.n_total + 8, stream)
    check(rc, "ppg_build_poly_checked")
    return r, info.as_dict()


def apply_poly(A: CSR, roots: Roots, v: torch.Tensor, out: Optional[torch.Tensor] = None,
               stream=None) -> torch.Tensor:
    """y = p(A) v (Algorithm 3) in A's dtype."""
    _need_cuda(v)
    y = torch.empty_like(v) if out is None else out
    check(lib.ppg_apply_poly(A.ref(), roots.ref(), _ptr(v), _ptr(y), _stream(stream)),
          "ppg_apply_poly")
    return y


def apply_poly_noalloc(A: CSR, roots: Roots, v: torch.Tensor, out: torch.Tensor,
                       stream=None) -> torch.Tensor:
    """y = p(A) v through the entry point that allocates no device memory
    (for callers that cannot allocate: see ppg_apply_poly_noalloc in the C
    header).  ``out`` must be given; n <= 1048576; calls must not overlap."""
    _need_cuda(v, out)
    check(lib.ppg_apply_poly_noalloc(A.ref(), roots.ref(), _ptr(v), _ptr(out), _stream(stream)),
          "ppg_apply_poly_noalloc")
    return out


def apply_phi(A: CSR, roots: Roots, v: torch.Tensor, out: Optional[torch.Tensor] = None,
              stream=None) -> torch.Tensor:
    """y = phi(A) v (Algorithm 1) in A's dtype."""
    _need_cuda(v)
    y = torch.empty_like(v) if out is None else out
    check(lib.ppg_apply_phi(A.ref(), roots.ref(), _ptr(v), _ptr(y), _stream(stream)),
          "ppg_apply_phi")
    return y


def spmv(A: CSR, x: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None):
    _need_cuda(x)
    y = torch.empty_like(x) if out is None else out
    check(lib.ppg_spmv(A.ref(), _ptr(x), _ptr(y), _stream(stream)), "ppg_spmv")
    return y


def solve(A: CSR, b: torch.Tensor, m: int = 50, tol: float = 1e-10,
          roots: Optional[Roots] = None, x0: Optional[torch.Tensor] = None,
          max_cycles: int = 10000, timing: bool = False, out: Optional[torch.Tensor] = None,
          stream=None, cgs2_fused: bool = False) -> Tuple[torch.Tensor, dict]:
    """PP-GMRES(m) (roots given) or GMRES(m); returns (x, stats)."""
    _need_cuda(b)
    x = torch.empty_like(b) if out is None else out
    if x0 is not None:
        x.copy_(x0)
    o = default_opts(max_cycles=max_cycles, timing=int(timing), x0_given=int(x0 is not None),
                     cgs2_fused=int(bool(cgs2_fused)))
    st = ppg_stats()
    rc = lib.ppg_solve(A.ref(), roots.ref() if roots is not None else None, _ptr(b), _ptr(x),
                       m, tol, C.byref(o), C.byref(st), _stream(stream))
    check(rc, "ppg_solve")
    s = st.as_dict()
    s["status"] = rc
    return x, s


def solve_flex(A64: CSR, A32: CSR, b: torch.Tensor, roots: Roots, m: int = 50,
               tol: float = 1e-10, max_cycles: int = 10000, timing: bool = False,
               out: Optional[torch.Tensor] = None, stream=None):
    """FGMRES(m) in FP64 with p(A) applied in FP32 on A32; returns (x, stats)."""
    _need_cuda(b)
    x = torch.empty_like(b) if out is None else out
    o = default_opts(max_cycles=max_cycles, timing=int(timing))
    st = ppg_stats()
    rc = lib.ppg_solve_flex(A64.ref(), A32.ref(), roots.ref(), _ptr(b), _ptr(x), m, tol,
                            C.byref(o), C.byref(st), _stream(stream))
    check(rc, "ppg_solve_flex")
    s = st.as_dict()
    s["status"] = rc
    return x, s


class SweepPlan:
    """Multi-root fused sweep plan of an FP32 CSR (ppg_sweep_plan_create):
    the matrix reordered into compact tiles of ``tile_rows`` rows (by
    ``perm``, new -> old, or breadth-first growth when None), with each
    tile's halo, so that a conjugate pair of Algorithm 3 runs in one pass."""

    def __init__(self, A32: "CSR", tile_rows: int = 4096, perm=None, fuse: bool = True,
                 stream=None):
        if A32.dtype != torch.float32:
            raise ValueError("the sweep plan takes the FP32 matrix")
        self._h = C.c_void_p()
        pp = None
        if perm is not None:
            self._perm = np.ascontiguousarray(perm, dtype=np.int32)
            pp = self._perm.ctypes.data_as(C.c_void_p)
        check(lib.ppg_sweep_plan_create(A32.ref(), pp, int(tile_rows), int(bool(fuse)),
                                        C.byref(self._h), _stream(stream)),
              "ppg_sweep_plan_create")
        self.n = A32.n

    def info(self) -> dict:
        i = ppg_sweep_info()
        check(lib.ppg_sweep_plan_info(self._h, C.byref(i)), "ppg_sweep_plan_info")
        return i.as_dict()

    def apply_poly(self, roots: Roots, v: torch.Tensor, out: Optional[torch.Tensor] = None,
                   stream=None) -> torch.Tensor:
        _need_cuda(v)
        if v.dtype != torch.float32:
            raise ValueError("v must be float32")
        y = torch.empty_like(v) if out is None else out
        check(lib.ppg_apply_poly_sweep(self._h, roots.ref(), _ptr(v), _ptr(y),
                                       _stream(stream)), "ppg_apply_poly_sweep")
        return y

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.ppg_sweep_plan_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_flex_sweep(A64: "CSR", plan: SweepPlan, b: torch.Tensor, roots: Roots,
                     m: int = 50, tol: float = 1e-10, max_cycles: int = 10000,
                     timing: bool = False, out: Optional[torch.Tensor] = None, stream=None):
    """The precision form with p(A) v_j through a fused-sweep plan."""
    _need_cuda(b)
    x = torch.empty_like(b) if out is None else out
    o = default_opts(max_cycles=max_cycles, timing=int(timing))
    st = ppg_stats()
    rc = lib.ppg_solve_flex_sweep(A64.ref(), plan._h, roots.ref(), _ptr(b), _ptr(x), m, tol,
                                  C.byref(o), C.byref(st), _stream(stream))
    check(rc, "ppg_solve_flex_sweep")
    s = st.as_dict()
    s["status"] = rc
    return x, s


def build_poly_composite(A: CSR, inner: Roots, d: int, v0: torch.Tensor,
                         stability_control: bool = True, capacity: Optional[int] = None,
                         stream=None) -> Roots:
    """Roots of phi_2 from GMRES(d) on phi_inner(A) (Section 6)."""
    _need_cuda(v0)
    cap = capacity or max(16, 4 * d)
    r = Roots(cap)
    o = default_opts(stability_control=int(bool(stability_control)))
    rc = lib.ppg_build_poly_composite(A.ref(), inner.ref(), d, _ptr(v0), C.byref(o), r.ref(),
                                      None, _stream(stream))
    if rc == -6 and capacity is None:
        return build_poly_composite(A, inner, d, v0, stability_control, r.s.n_total + 8, stream)
    check(rc, "ppg_build_poly_composite")
    return r


def solve_double(A: CSR, b: torch.Tensor, r1: Roots, r2: Roots, m: int = 50,
                 tol: float = 1e-10, max_cycles: int = 10000, out=None, stream=None):
    """Double polynomial preconditioning: GMRES(m) on phi_2(phi_1(A)) z = b,
    x = p_1(A) p_2(phi_1(A)) z.  Returns (x, stats)."""
    _need_cuda(b)
    x = torch.empty_like(b) if out is None else out
    o = default_opts(max_cycles=max_cycles)
    st = ppg_stats()
    rc = lib.ppg_solve_double(A.ref(), r1.ref(), r2.ref(), _ptr(b), _ptr(x), m, tol,
                              C.byref(o), C.byref(st), _stream(stream))
    check(rc, "ppg_solve_double")
    s = st.as_dict()
    s["status"] = rc
    return x, s


def solve_chpoly(A: CSR, b: torch.Tensor, d: int, m: int = 50, tol: float = 1e-10,
                 max_cycles: int = 10000, out=None, stream=None):
    """PP-GMRES with the degree-d polynomial rebuilt from the residual at
    every restart (Section 5.2).  Returns (x, stats)."""
    _need_cuda(b)
    x = torch.empty_like(b) if out is None else out
    o = default_opts(max_cycles=max_cycles)
    st = ppg_stats()
    rc = lib.ppg_solve_chpoly(A.ref(), d, _ptr(b), _ptr(x), m, tol, C.byref(o), C.byref(st),
                              _stream(stream))
    check(rc, "ppg_solve_chpoly")
    s = st.as_dict()
    s["status"] = rc
    return x, s


def solve_batched(As, Bs, v0s, d: int = 20, m: int = 30, tol: float = 1e-10,
                  max_cycles: int = 10000, Xs=None, stream=None, persistent: bool = True,
                  wait_timeout_ms: Optional[float] = None):
    """Batching form: systems As[s] (FP64 CSR) with right-hand sides Bs[s]
    (tensor (nrhs, n_s), nrhs = 1 or 4, same nrhs for all) and start vectors
    v0s[s]; each system gets its own polynomial; FGMRES(m) with FP32 p(A).
    persistent: the whole solve in one persistent cooperative launch (else
    one CUDA graph per restart cycle).  Returns (Xs, info) with info =
    {"roots", "relres", "iters", "stats", "status"}."""
    nsys = len(As)
    nrhs = Bs[0].shape[0] if Bs[0].dim() == 2 else 1
    csrs = (ppg_csr * nsys)(*[A.s for A in As])
    if Xs is None:
        Xs = [torch.empty_like(b) for b in Bs]
    for t in list(Bs) + list(Xs) + list(v0s):
        _need_cuda(t)
    bp = (C.c_void_p * nsys)(*[b.data_ptr() for b in Bs])
    xp = (C.c_void_p * nsys)(*[x.data_ptr() for x in Xs])
    vp = (C.c_void_p * nsys)(*[v.data_ptr() for v in v0s])
    roots = [Roots(4 * d + 8) for _ in range(nsys)]
    rarr = (ppg_roots * nsys)(*[r.s for r in roots])
    rel = np.zeros(nsys * nrhs)
    its = np.zeros(nsys * nrhs, dtype=np.int32)
    o = default_opts(max_cycles=max_cycles, batch_mode=0 if persistent else 1,
                     wait_timeout_ms=wait_timeout_ms)
    st = ppg_stats()
    rc = lib.ppg_solve_batched(nsys, csrs, nrhs, bp, xp, vp, d, m, tol, C.byref(o), rarr,
                               C.byref(st), _dp(rel),
                               its.ctypes.data_as(C.POINTER(C.c_int32)), _stream(stream))
    check(rc, "ppg_solve_batched")
    for r, rs in zip(roots, rarr):
        r.s.n_orig, r.s.n_added, r.s.n_total = rs.n_orig, rs.n_added, rs.n_total
    return Xs, {"roots": roots, "relres": rel.reshape(nsys, nrhs),
                "iters": its.reshape(nsys, nrhs), "stats": st.as_dict(), "status": rc}


def stability_check(A: CSR, roots: Roots, b: torch.Tensor, stream=None) -> float:
    """StCh = ||(b - A p(A) b) - pi(A) b|| (Section 3.5)."""
    _need_cuda(b)
    out = C.c_double(0.0)
    check(lib.ppg_stability_check(A.ref(), roots.ref(), _ptr(b), C.byref(out), _stream(stream)),
          "ppg_stability_check")
    return out.value


def adjoint_vals_grad(A: CSR, lam: torch.Tensor, x: torch.Tensor, out=None, stream=None):
    g = torch.empty_like(A.vals) if out is None else out
    check(lib.ppg_adjoint_vals_grad(A.ref(), _ptr(lam), _ptr(x), _ptr(g), _stream(stream)),
          "ppg_adjoint_vals_grad")
    return g


def solve_host(rowptr: np.ndarray, colind: np.ndarray, vals: np.ndarray, b: np.ndarray,
               v0: np.ndarray, d: int, m: int = 50, tol: float = 1e-10,
               device="cuda", timing: bool = False):
    """End-to-end call from host arrays: copy CSR, b and v0 to the device,
    build the polynomial, solve, copy x back.  Returns (x, roots, stats).

    The inputs may be NumPy arrays (page-locked here, on every call) or CPU
    tensors already in pinned memory (copied as they are: the fast path for
    repeated calls)."""
    def pinned(a, dt):
        if isinstance(a, torch.Tensor):
            tdt = torch.int32 if dt == np.int32 else torch.float64
            t = a if a.dtype == tdt else a.to(tdt)
            return t if t.is_pinned() else t.contiguous().pin_memory()
        t = torch.from_numpy(np.ascontiguousarray(a, dtype=dt))
        return t.pin_memory()
    rp = pinned(rowptr, np.int32).to(device, non_blocking=True)
    ci = pinned(colind, np.int32).to(device, non_blocking=True)
    vv = pinned(vals, np.float64).to(device, non_blocking=True)
    bd = pinned(b, np.float64).to(device, non_blocking=True)
    vd = pinned(v0, np.float64).to(device, non_blocking=True)
    A = CSR(rp, ci, vv)
    roots = build_poly(A, d, vd)
    x, st = solve(A, bd, m, tol, roots=roots, timing=timing)
    xh = torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
    xh.copy_(x, non_blocking=True)
    torch.cuda.current_stream().synchronize()
    return xh.numpy(), roots, st


class PPGMRESFunction(torch.autograd.Function):
    """x = A(vals)^{-1} b by PP-GMRES, differentiable in b and vals.

    Backward runs the adjoint PP-GMRES on A^T with the same roots
    (p(A^T) = p(A)^T): lambda = A^{-T} grad_x, dL/db = lambda and
    dL/dvals[k] = -lambda[row k] x[colind k].
    """

    @staticmethod
    def forward(ctx, b, vals, A: CSR, roots: Roots, m: int, tol: float, AT: Optional[CSR],
                max_cycles: int = 10000):
        Aw = A.with_vals(vals.detach().contiguous())
        x, st = solve(Aw, b.detach().contiguous(), m, tol, roots=roots, max_cycles=max_cycles)
        ctx.A, ctx.roots, ctx.m, ctx.tol, ctx.AT = Aw, roots, m, tol, AT
        ctx.max_cycles = max_cycles
        ctx.save_for_backward(x)
        ctx.stats = st
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        AT = ctx.AT
        if AT is None:
            AT = ctx.A.transpose()
        lam, _ = solve(AT, gx.contiguous(), ctx.m, ctx.tol, roots=ctx.roots,
                       max_cycles=ctx.max_cycles)
        gvals = adjoint_vals_grad(ctx.A, lam, x)
        return lam, gvals, None, None, None, None, None, None
