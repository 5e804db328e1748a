"""ctypes binding of libppgmres (argument marshalling only).

Every computation runs inside the shared library; PyTorch provides device
memory and the current CUDA stream.  The library must have been built
(``paper_1911_07065_gb300.build.build()``): importing this module without it
raises, there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os



import numpy as np

from .build import LIB

c_i32, c_i64, c_f64, c_vp = C.c_int32, C.c_int64, C.c_double, C.c_void_p
P_F64 = C.POINTER(C.c_double)

PPG_F64, PPG_F32 = 0, 1
STATUS = {
    0: "PPG_OK", 1: "PPG_NOT_CONVERGED", 2: "PPG_LUCKY_BREAKDOWN",
    -1: "PPG_ERR_ARG", -2: "PPG_ERR_CSR", -3: "PPG_ERR_SINGULAR_H",
    -4: "PPG_ERR_NONFINITE", -5: "PPG_ERR_CUDA", -6: "PPG_ERR_CAPACITY",
    -7: "PPG_ERR_EIG", -8: "PPG_ERR_NOMEM", -9: "PPG_ERR_TOO_LARGE", -10: "PPG_ERR_TIMEOUT",
}
NOALLOC_MAX_N = 1048576


class ppg_csr(C.Structure):
    _fields_ = [("n", c_i32), ("nnz", c_i32), ("rowptr", c_vp), ("colind", c_vp),
                ("vals", c_vp), ("dtype", c_i32)]


class ppg_roots(C.Structure):
    _fields_ = [("n_orig", c_i32), ("n_added", c_i32), ("n_total", c_i32),
                ("capacity", c_i32), ("re", P_F64), ("im", P_F64), ("log10_pof", P_F64)]


class ppg_opts(C.Structure):
    _fields_ = [("max_cycles", c_i32), ("stability_control", c_i32),
                ("pof_threshold_log10", c_f64), ("pof_step_log10", c_f64),
                ("timing", c_i32), ("x0_given", c_i32), ("batch_mode", c_i32),
                ("cgs2_fused", c_i32), ("wait_timeout_ms", c_f64)]


class ppg_stats(C.Structure):
    _fields_ = [("iters", c_i64), ("cycles", c_i64), ("mvps", c_i64), ("dots", c_i64),
                ("launches", c_i64), ("true_relres", c_f64), ("est_relres", c_f64),
                ("converged", c_i32), ("pad_", c_i32), ("poly_ms", c_f64),
                ("poly_launches", c_i64), ("poly_bytes", c_f64), ("ortho_ms", c_f64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


class ppg_poly_check(C.Structure):
    _fields_ = [("d_requested", c_i32), ("d_chosen", c_i32), ("n_tried", c_i32),
                ("pad_", c_i32), ("stch", c_f64), ("stch_first", c_f64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


class ppg_sweep_info(C.Structure):
    _fields_ = [("n", c_i32), ("nnz", c_i32), ("tile_rows", c_i32), ("ntiles", c_i32),
                ("max_halo", c_i32), ("fused", c_i32), ("halo_total", c_i64),
                ("halo_fraction", c_f64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PPGError(RuntimeError):
    def __init__(self, code, where):
        msg = lib.ppg_strerror(code).decode()
        if code == -5:
            msg += " (" + lib.ppg_last_cuda_error().decode() + ")"
        super().__init__("%s: %s [%s]" % (where, msg, STATUS.get(code, code)))
        self.code = code


def _load():
    if not os.path.exists(LIB):
        raise ImportError("libppgmres.so is not built (%s); run "
                          "paper_1911_07065_gb300.build.build()" % LIB)
    L = C.CDLL(LIB)
    sig = {
        "ppg_abi_version": (c_i32, []),
        "ppg_strerror": (C.c_char_p, [c_i32]),
        "ppg_last_cuda_error": (C.c_char_p, []),
        "ppg_default_opts": (None, [C.POINTER(ppg_opts)]),
        "ppg_launch_count": (c_i64, []),
        "ppg_harmonic_ritz": (c_i32, [P_F64, c_i32, c_i32, P_F64, P_F64]),
        "ppg_leja_order": (c_i32, [c_i32, P_F64, P_F64, P_F64, P_F64]),
        "ppg_add_roots": (c_i32, [c_i32, P_F64, P_F64, c_f64, c_f64, C.POINTER(ppg_roots)]),
        "ppg_roots_from_hessenberg": (c_i32, [P_F64, c_i32, c_i32, C.POINTER(ppg_opts),
                                              C.POINTER(ppg_roots)]),
        "ppg_csr_validate_host": (c_i32, [c_i32, c_i32, c_vp, c_vp]),
        "ppg_build_poly": (c_i32, [C.POINTER(ppg_csr), c_i32, c_vp, C.POINTER(ppg_opts),
                                   C.POINTER(ppg_roots), P_F64, c_vp]),
        "ppg_build_poly_checked": (c_i32, [C.POINTER(ppg_csr), c_i32, c_vp, c_vp, c_f64, c_i32,
                                           C.POINTER(ppg_opts), C.POINTER(ppg_roots),
                                           C.POINTER(ppg_poly_check), c_vp]),
        "ppg_sweep_plan_create": (c_i32, [C.POINTER(ppg_csr), c_vp, c_i32, c_i32,
                                          C.POINTER(c_vp), c_vp]),
        "ppg_sweep_plan_info": (c_i32, [c_vp, C.POINTER(ppg_sweep_info)]),
        "ppg_sweep_plan_destroy": (None, [c_vp]),
        "ppg_apply_poly_sweep": (c_i32, [c_vp, C.POINTER(ppg_roots), c_vp, c_vp, c_vp]),
        "ppg_solve_flex_sweep": (c_i32, [C.POINTER(ppg_csr), c_vp, C.POINTER(ppg_roots), c_vp,
                                         c_vp, c_i32, c_f64, C.POINTER(ppg_opts),
                                         C.POINTER(ppg_stats), c_vp]),
        "ppg_apply_poly": (c_i32, [C.POINTER(ppg_csr), C.POINTER(ppg_roots), c_vp, c_vp, c_vp]),
        "ppg_apply_phi": (c_i32, [C.POINTER(ppg_csr), C.POINTER(ppg_roots), c_vp, c_vp, c_vp]),
        "ppg_apply_poly_noalloc": (c_i32, [C.POINTER(ppg_csr), C.POINTER(ppg_roots), c_vp,
                                           c_vp, c_vp]),
        "ppg_spmv": (c_i32, [C.POINTER(ppg_csr), c_vp, c_vp, c_vp]),
        "ppg_solve": (c_i32, [C.POINTER(ppg_csr), C.POINTER(ppg_roots), c_vp, c_vp, c_i32,
                              c_f64, C.POINTER(ppg_opts), C.POINTER(ppg_stats), c_vp]),
        "ppg_solve_flex": (c_i32, [C.POINTER(ppg_csr), C.POINTER(ppg_csr),
                                   C.POINTER(ppg_roots), c_vp, c_vp, c_i32, c_f64,
                                   C.POINTER(ppg_opts), C.POINTER(ppg_stats), c_vp]),
        "ppg_stability_check": (c_i32, [C.POINTER(ppg_csr), C.POINTER(ppg_roots), c_vp,
                                        P_F64, c_vp]),
        "ppg_build_poly_composite": (c_i32, [C.POINTER(ppg_csr), C.POINTER(ppg_roots), c_i32,
                                             c_vp, C.POINTER(ppg_opts), C.POINTER(ppg_roots),
                                             P_F64, c_vp]),
        "ppg_solve_double": (c_i32, [C.POINTER(ppg_csr), C.POINTER(ppg_roots),
                                     C.POINTER(ppg_roots), c_vp, c_vp, c_i32, c_f64,
                                     C.POINTER(ppg_opts), C.POINTER(ppg_stats), c_vp]),
        "ppg_solve_chpoly": (c_i32, [C.POINTER(ppg_csr), c_i32, c_vp, c_vp, c_i32, c_f64,
                                     C.POINTER(ppg_opts), C.POINTER(ppg_stats), c_vp]),
        "ppg_solve_batched": (c_i32, [c_i32, C.POINTER(ppg_csr), c_i32, C.POINTER(c_vp),
                                      C.POINTER(c_vp), C.POINTER(c_vp), c_i32, c_i32, c_f64,
                                      C.POINTER(ppg_opts), C.POINTER(ppg_roots),
                                      C.POINTER(ppg_stats), P_F64, C.POINTER(c_i32), c_vp]),
        "ppg_csr_transpose": (c_i32, [C.POINTER(ppg_csr), c_vp, c_vp, c_vp, c_vp, c_vp]),
        "ppg_adjoint_vals_grad": (c_i32, [C.POINTER(ppg_csr), c_vp, c_vp, c_vp, c_vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


lib = _load()

# names the C header declares (checked by the CPU tests)
EXPORTS = (
    "ppg_abi_version", "ppg_strerror", "ppg_last_cuda_error", "ppg_default_opts",
    "ppg_launch_count",
    "ppg_harmonic_ritz", "ppg_leja_order", "ppg_add_roots", "ppg_roots_from_hessenberg",
    "ppg_csr_validate_host", "ppg_build_poly", "ppg_apply_poly", "ppg_apply_phi",
    "ppg_spmv", "ppg_solve", "ppg_solve_flex", "ppg_stability_check",
    "ppg_csr_transpose", "ppg_adjoint_vals_grad", "ppg_apply_poly_noalloc",
    "ppg_solve_batched", "ppg_build_poly_composite", "ppg_solve_double", "ppg_solve_chpoly",
    "ppg_build_poly_checked", "ppg_sweep_plan_create", "ppg_sweep_plan_info",
    "ppg_sweep_plan_destroy", "ppg_apply_poly_sweep", "ppg_solve_flex_sweep",
)


def check(code, where):
    if code < 0:
        raise PPGError(code, where)
    return code


def _dp(a: np.ndarray):
    return a.ctypes.data_as(P_F64)


def default_opts(**kw) -> ppg_opts:
    o = ppg_opts()
    lib.ppg_default_opts(C.byref(o))
    for k, v in kw.items():
        if v is not None:
            setattr(o, k, v)
    return o


# ---------------------------------------------------------------------------
# Roots (host arrays)
# ---------------------------------------------------------------------------


class Roots:
    """Leja-ordered roots of pi (with added copies), held on the host."""

    def __init__(self, capacity: int):
        self.capacity = int(capacity)
        self.re = np.zeros(self.capacity)
        self.im = np.zeros(self.capacity)
        self.log10_pof = np.zeros(self.capacity)
        self.s = ppg_roots(0, 0, 0, self.capacity, _dp(self.re), _dp(self.im),
                           _dp(self.log10_pof))

    @classmethod
    def from_complex(cls, theta) -> "Roots":
        theta = np.asarray(theta, dtype=np.complex128)
        r = cls(max(1, theta.size))
        r.re[: theta.size] = theta.real
        r.im[: theta.size] = theta.imag
        r.s.n_orig = theta.size
        r.s.n_added = 0
        r.s.n_total = theta.size
        return r

    @property
    def n_total(self):
        return self.s.n_total

    @property
    def n_orig(self):
        return self.s.n_orig

    @property
    def n_added(self):
        return self.s.n_added

    def complex(self) -> np.ndarray:
        k = self.s.n_total
        return self.re[:k] + 1j * self.im[:k]

    def pof(self) -> np.ndarray:
        return self.log10_pof[: self.s.n_orig].copy()

    def ref(self):
        return C.byref(self.s)


# ---------------------------------------------------------------------------
# Host-only steps
# ---------------------------------------------------------------------------


def harmonic_ritz(Hbar: np.ndarray) -> np.ndarray:
    """Harmonic Ritz values of a (d+1) x d Hessenberg matrix (HOST)."""
    H = np.asfortranarray(np.asarray(Hbar, dtype=np.float64))
    d = H.shape[1]
    re = np.zeros(d)
    im = np.zeros(d)
    check(lib.ppg_harmonic_ritz(_dp(H), H.shape[0], d, _dp(re), _dp(im)), "ppg_harmonic_ritz")
    return re + 1j * im


def leja_order(theta) -> np.ndarray:
    t = np.asarray(theta, dtype=np.complex128)
    re = np.ascontiguousarray(t.real)
    im = np.ascontiguousarray(t.imag)
    ro = np.zeros(t.size)
    io = np.zeros(t.size)
    check(lib.ppg_leja_order(t.size, _dp(re), _dp(im), _dp(ro), _dp(io)), "ppg_leja_order")
    return ro + 1j * io


def add_roots(theta_leja, thr_log10=4.0, step_log10=14.0, capacity=None) -> Roots:
    t = np.asarray(theta_leja, dtype=np.complex128)
    re = np.ascontiguousarray(t.real)
    im = np.ascontiguousarray(t.imag)
    cap = capacity or max(8, 4 * t.size)
    r = Roots(cap)
    rc = lib.ppg_add_roots(t.size, _dp(re), _dp(im), thr_log10, step_log10, r.ref())
    if rc == -6 and capacity is None:
        return add_roots(theta_leja, thr_log10, step_log10, capacity=r.s.n_total + 8)
    check(rc, "ppg_add_roots")
    return r


def roots_from_hessenberg(Hbar: np.ndarray, stability_control=True, capacity=None) -> Roots:
    H = np.asfortranarray(np.asarray(Hbar, dtype=np.float64))
    d = H.shape[1]
    cap = capacity or max(8, 4 * d)
    r = Roots(cap)
    o = default_opts(stability_control=int(bool(stability_control)))
    rc = lib.ppg_roots_from_hessenberg(_dp(H), H.shape[0], d, C.byref(o), r.ref())
    if rc == -6 and capacity is None:
        return roots_from_hessenberg(Hbar, stability_control, capacity=r.s.n_total + 8)
    check(rc, "ppg_roots_from_hessenberg")
    return r


def csr_validate_host(rowptr: np.ndarray, colind: np.ndarray) -> int:
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(colind, dtype=np.int32)
    return lib.ppg_csr_validate_host(rp.size - 1, ci.size, rp.ctypes.data, ci.ctypes.data)
