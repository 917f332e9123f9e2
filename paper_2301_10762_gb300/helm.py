"""Thin Python binding of libhelm (include/helm.h) over ctypes.

Argument marshalling only: tensors are checked (device, dtype, contiguity, shape) and
their device pointers passed to the C entry points, which run every step of the path
in CUDA kernels.  There is no CPU fallback: if libhelm.so is missing or no GPU is
visible, every call raises.

Function names follow the C ABI: helm_assemble, helm_factor, helm_solve,
helm_adjoint_solve, helm_sources, helm_restrict, fwi_misfit_grad, bilevel_hypergrad.
Right-hand-side blocks are complex128 tensors of shape [n_omega, nrhs, N] with
N = nx * nz and node index k = i * nz + j (z fastest).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhelm.so")

HELM_FP64, HELM_MIXED = 0, 1
_STATUS = {0: "HELM_OK", 1: "HELM_EINVAL", 2: "HELM_ENOMEM", 3: "HELM_ECUDA", 4: "HELM_ENOCONV",
           5: "HELM_ESINGULAR", 6: "HELM_ETIMEOUT"}


class HelmError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        super().__init__(f"{where}: {_STATUS.get(status, status)} {detail}".strip())


class helm_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("nz", C.c_int32), ("lx", C.c_double), ("lz", C.c_double),
                ("lumping", C.c_int32)]


HELM_LUMP_TENSOR, HELM_LUMP_UP, HELM_LUMP_DOWN = 0, 1, 2


class helm_acq(C.Structure):
    _fields_ = [("n_src", C.c_int32), ("n_rec", C.c_int32), ("src_xz", C.POINTER(C.c_double)),
                ("src_amp", C.POINTER(C.c_double)), ("rec_xz", C.POINTER(C.c_double)),
                ("rec_w", C.POINTER(C.c_double))]


class helm_solve_info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("max_relres", C.c_double)]


class helm_pcg_opts(C.Structure):
    _fields_ = [("max_iter", C.c_int32), ("fixed_iters", C.c_int32), ("rtol", C.c_double), ("x0", C.c_double),
                ("refine_rtol", C.c_double), ("concurrent_models", C.c_int32), ("factor_method", C.c_int32)]


class helm_factor_opts(C.Structure):
    _fields_ = [("method", C.c_int32)]


class helm_hyper_info(C.Structure):
    _fields_ = [("cg_matvecs", C.c_int32), ("cg_relres", C.c_double), ("solves", C.c_int64),
                ("data_solves", C.c_int64), ("max_refine_iters", C.c_int32)]


class helm_trace_event(C.Structure):
    _fields_ = [("kernel", C.c_int32), ("stream", C.c_int32), ("start_ms", C.c_double), ("end_ms", C.c_double)]


class helm_server_opts(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_uint64), ("max_batch_rhs", C.c_int32), ("workers", C.c_int32),
                ("max_iter", C.c_int32)]


class helm_request(C.Structure):
    _fields_ = [("model", C.c_int32), ("omega", C.c_double), ("prec", C.c_int32), ("adjoint", C.c_int32),
                ("nrhs", C.c_int32), ("B", C.c_void_p), ("X", C.c_void_p), ("rtol", C.c_double)]


class helm_request_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("cache_hit", C.c_int32), ("batch_rhs", C.c_int32), ("iters", C.c_int32),
                ("max_relres", C.c_double), ("queue_ms", C.c_double), ("total_ms", C.c_double)]


class helm_server_counters(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("refused", C.c_int64),
                ("rhs_solved", C.c_int64), ("batches", C.c_int64), ("factor_builds", C.c_int64),
                ("cache_hits", C.c_int64), ("evictions", C.c_int64), ("entries", C.c_int64),
                ("bytes_used", C.c_uint64), ("bytes_peak", C.c_uint64), ("bytes_budget", C.c_uint64)]


class helm_trace_entry(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("launches", C.c_int64), ("total_ms", C.c_double), ("timed", C.c_int64),
                ("flops", C.c_double)]


EXPORTED = ["helm_status_string", "helm_last_error", "helm_assemble", "helm_op_destroy", "helm_factor",
            "helm_factor_destroy", "helm_factor_fp64_blocks", "helm_factor_get_method", "helm_set_wait_tries",
            "helm_fault_mask",
            # include/helm_blas.h
            "helm_zgemm_batched", "helm_zinv_batched", "helm_solve", "helm_adjoint_solve", "helm_solve_noalloc", "helm_sources",
            "helm_restrict", "helm_restrict_adjoint", "helm_field_grad",
            "fwi_misfit_grad", "fwi_hessian_vec", "bilevel_hypergrad", "helm_gamma_solve",
            # include/helm_trace.h
            "helm_trace_enable", "helm_trace_reset", "helm_trace_read", "helm_launch_count",
            "helm_trace_timeline", "helm_trace_kernel_name", "helm_trace_select",
            # include/helm_server.h
            "helm_server_create", "helm_server_add_model", "helm_server_footprint", "helm_server_submit",
            "helm_server_wait", "helm_server_stats", "helm_server_destroy"]

_lib = None


def load(path: str = LIB_PATH):
    """Load libhelm.so (raises if it is missing; there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libhelm.so not found at {path}; build it with __graft_entry__.build()")
    lib = C.CDLL(path)
    vp, i32, dbl = C.c_void_p, C.c_int32, C.c_double
    P = C.POINTER
    lib.helm_status_string.restype = C.c_char_p
    lib.helm_status_string.argtypes = [C.c_int]
    lib.helm_last_error.restype = C.c_char_p
    lib.helm_last_error.argtypes = []
    lib.helm_assemble.restype = C.c_int
    lib.helm_assemble.argtypes = [P(helm_grid), vp, P(dbl), i32, vp, P(vp)]
    lib.helm_op_destroy.restype = None
    lib.helm_op_destroy.argtypes = [vp]
    lib.helm_factor.restype = C.c_int
    lib.helm_factor.argtypes = [vp, C.c_int, P(helm_factor_opts), P(vp)]
    lib.helm_zgemm_batched.restype = C.c_int
    lib.helm_zgemm_batched.argtypes = [i32, i32, i32, i32, vp, C.c_int64, i32, vp, C.c_int64, i32, C.c_float, vp, vp,
                                       C.c_int64, i32, vp]
    lib.helm_zinv_batched.restype = C.c_int
    lib.helm_zinv_batched.argtypes = [i32, i32, vp, C.c_int64, i32, vp, C.c_int64, i32, vp]
    lib.helm_set_wait_tries.restype = None
    lib.helm_set_wait_tries.argtypes = [C.c_int64]
    lib.helm_fault_mask.restype = C.c_uint32
    lib.helm_fault_mask.argtypes = []
    lib.helm_factor_get_method.restype = i32
    lib.helm_factor_get_method.argtypes = [vp]
    lib.helm_factor_fp64_blocks.restype = i32
    lib.helm_factor_fp64_blocks.argtypes = [vp]
    lib.helm_factor_destroy.restype = None
    lib.helm_factor_destroy.argtypes = [vp]
    for name in ("helm_solve", "helm_adjoint_solve"):
        fn = getattr(lib, name)
        fn.restype = C.c_int
        fn.argtypes = [vp, i32, vp, vp, dbl, i32, P(helm_solve_info)]
    lib.helm_solve_noalloc.restype = C.c_int
    lib.helm_solve_noalloc.argtypes = [vp, i32, vp, vp, dbl, i32, i32, P(helm_solve_info)]
    lib.helm_sources.restype = C.c_int
    lib.helm_sources.argtypes = [vp, P(helm_acq), vp]
    lib.helm_restrict.restype = C.c_int
    lib.helm_restrict.argtypes = [vp, P(helm_acq), i32, vp, vp]
    lib.helm_restrict_adjoint.restype = C.c_int
    lib.helm_restrict_adjoint.argtypes = [vp, P(helm_acq), i32, vp, vp]
    lib.helm_field_grad.restype = C.c_int
    lib.helm_field_grad.argtypes = [vp, i32, vp, vp, vp]
    lib.fwi_misfit_grad.restype = C.c_int
    lib.fwi_misfit_grad.argtypes = [vp, P(helm_acq), vp, dbl, dbl, dbl, P(dbl), vp, vp, vp]
    lib.fwi_hessian_vec.restype = C.c_int
    lib.fwi_hessian_vec.argtypes = [vp, P(helm_acq), vp, vp, vp, dbl, dbl, dbl, i32, vp]
    lib.helm_gamma_solve.restype = C.c_int
    lib.helm_gamma_solve.argtypes = [P(helm_grid), dbl, dbl, i32, vp, vp, vp]
    lib.bilevel_hypergrad.restype = C.c_int
    lib.bilevel_hypergrad.argtypes = [i32, P(helm_grid), P(vp), P(vp), P(helm_acq), P(helm_grid), P(vp), P(dbl), i32, dbl, dbl,
                                      dbl, C.c_int, P(helm_pcg_opts), vp, P(dbl), P(dbl), P(dbl), P(dbl),
                                      P(helm_hyper_info)]
    lib.helm_trace_enable.restype = None
    lib.helm_trace_enable.argtypes = [C.c_int]
    lib.helm_trace_reset.restype = None
    lib.helm_trace_reset.argtypes = []
    lib.helm_trace_read.restype = C.c_int32
    lib.helm_trace_read.argtypes = [P(helm_trace_entry), i32]
    lib.helm_trace_timeline.restype = C.c_int32
    lib.helm_trace_timeline.argtypes = [P(helm_trace_event), i32]
    lib.helm_trace_kernel_name.restype = C.c_char_p
    lib.helm_trace_kernel_name.argtypes = [i32]
    lib.helm_trace_select.restype = C.c_int32
    lib.helm_trace_select.argtypes = [C.c_char_p]
    lib.helm_launch_count.restype = C.c_int64
    lib.helm_launch_count.argtypes = []
    lib.helm_server_create.restype = C.c_int
    lib.helm_server_create.argtypes = [P(helm_server_opts), P(vp)]
    lib.helm_server_add_model.restype = C.c_int
    lib.helm_server_add_model.argtypes = [vp, P(helm_grid), P(dbl), P(i32)]
    lib.helm_server_footprint.restype = C.c_uint64
    lib.helm_server_footprint.argtypes = [vp, i32, i32, i32]
    lib.helm_server_submit.restype = C.c_int
    lib.helm_server_submit.argtypes = [vp, P(helm_request), P(C.c_int64)]
    lib.helm_server_wait.restype = C.c_int
    lib.helm_server_wait.argtypes = [vp, C.c_int64, P(helm_request_info)]
    lib.helm_server_stats.restype = C.c_int
    lib.helm_server_stats.argtypes = [vp, P(helm_server_counters)]
    lib.helm_server_destroy.restype = None
    lib.helm_server_destroy.argtypes = [vp]
    _lib = lib
    return lib


def _check(status, where):
    if status != 0:
        detail = _lib.helm_last_error().decode(errors="replace") if _lib is not None else ""
        raise HelmError(status, where, detail)


def _dev(t: torch.Tensor, dtype, name, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return C.c_void_p(t.data_ptr())


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dbuf(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


class Acq:
    """Host-side acquisition marshalled into a helm_acq struct (keeps the arrays alive)."""

    def __init__(self, src_xz, rec_xz, src_amp=None, rec_w=None):
        self._src, p_src = _dbuf(np.asarray(src_xz, dtype=np.float64).reshape(-1, 2))
        self._rec, p_rec = _dbuf(np.asarray(rec_xz, dtype=np.float64).reshape(-1, 2))
        self._amp = self._w = None
        p_amp = p_w = C.POINTER(C.c_double)()
        if src_amp is not None:
            self._amp, p_amp = _dbuf(src_amp)
        if rec_w is not None:
            self._w, p_w = _dbuf(rec_w)
        self.n_src, self.n_rec = self._src.shape[0], self._rec.shape[0]
        self.struct = helm_acq(self.n_src, self.n_rec, p_src, p_amp, p_rec, p_w)

    @classmethod
    def from_workload(cls, acq):
        return cls(acq.src_xz, acq.rec_xz, acq.src_amp, acq.rec_w)


class Op:
    def __init__(self, handle, nx, nz, lx, lz, omegas, stream):
        self.handle, self.nx, self.nz, self.lx, self.lz = handle, nx, nz, lx, lz
        self.omegas = np.asarray(omegas, dtype=np.float64)
        self.n_omega = len(self.omegas)
        self.N = nx * nz
        self.stream = stream

    def close(self):
        if self.handle:
            load().helm_op_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Factor:
    def __init__(self, handle, op, prec):
        self.handle, self.op, self.prec = handle, op, prec

    @property
    def fp64_blocks(self) -> int:
        """Pivot blocks of a mixed factor that were flagged and inverted in FP64."""
        return int(load().helm_factor_fp64_blocks(self.handle))

    @property
    def method(self) -> int:
        """HELM_FACTOR_LINE (1) or HELM_FACTOR_BCR (2): the method the factor was built with."""
        return int(load().helm_factor_get_method(self.handle))

    def close(self):
        if self.handle:
            load().helm_factor_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def helm_assemble(nx, nz, lx, lz, m: torch.Tensor, omegas, stream=None, lumping=HELM_LUMP_TENSOR) -> Op:
    """A(m, w) for every w; lumping: HELM_LUMP_TENSOR (tensor trapezoid) or HELM_LUMP_UP /
    HELM_LUMP_DOWN (vertex quadrature of the triangles of that orientation; include/helm.h)."""
    lib = load()
    pm = _dev(m, torch.float64, "m", (nx * nz,))
    om, p_om = _dbuf(np.atleast_1d(omegas))
    h = C.c_void_p()
    g = helm_grid(nx, nz, lx, lz, int(lumping))
    _check(lib.helm_assemble(C.byref(g), pm, p_om, len(om), _stream_ptr(stream), C.byref(h)), "helm_assemble")
    return Op(h, nx, nz, lx, lz, om, stream)


def helm_set_wait_tries(tries=-1):
    """Polls of a bounded device-side wait before it gives up, for later launches (< 0: the
    library default; 0: give up at the first wait that is not already complete)."""
    load().helm_set_wait_tries(int(tries))


HELM_FAULT_ALLOC, HELM_FAULT_PIVOT, HELM_FAULT_TIMEOUT, HELM_FAULT_NAN_RHS = 0x1, 0x2, 0x4, 0x8
HELM_FAULT_UNKNOWN = 0x80000000


def helm_fault_mask():
    """The HELM_FAULT_* bits that the HELM_FAULT environment variable selects now (host-side
    fault injection for tests: alloc, pivot, timeout, nan_rhs)."""
    return int(load().helm_fault_mask())


HELM_FACTOR_AUTO, HELM_FACTOR_LINE, HELM_FACTOR_BCR = 0, 1, 2


def helm_factor(op: Op, prec=HELM_FP64, method=HELM_FACTOR_AUTO) -> Factor:
    lib = load()
    h = C.c_void_p()
    opts = helm_factor_opts(int(method))
    _check(lib.helm_factor(op.handle, int(prec), C.byref(opts), C.byref(h)), "helm_factor")
    return Factor(h, op, prec)


def helm_zgemm_batched(A: torch.Tensor, Bt: torch.Tensor, C0: torch.Tensor | None = None, sign=1.0, C=None,
                       stream=None):
    """C[t] = C0[t] + sign * A[t] @ Bt[t].T on the tensor cores (complex64, [batch, rows, cols])."""
    lib = load()
    if A.dim() != 3 or Bt.dim() != 3 or A.shape[0] != Bt.shape[0] or A.shape[2] != Bt.shape[2]:
        raise ValueError("A [batch, M, K], Bt [batch, N, K]")
    b, M, K = A.shape
    N = Bt.shape[1]
    pa = _dev(A, torch.complex64, "A")
    pb = _dev(Bt, torch.complex64, "Bt")
    if C is None:
        C = torch.empty((b, M, N), dtype=torch.complex64, device=A.device)
    pc = _dev(C, torch.complex64, "C", (b, M, N))
    p0 = _dev(C0, torch.complex64, "C0", (b, M, N)) if C0 is not None else None
    _check(lib.helm_zgemm_batched(b, M, N, K, pa, M * K, K, pb, N * K, K, float(sign), p0, pc, M * N, N,
                                  _stream_ptr(stream)), "helm_zgemm_batched")
    return C


def helm_zinv_batched(A: torch.Tensor, X: torch.Tensor | None = None, stream=None):
    """X[t] = A[t]^{-1} for complex symmetric complex64 matrices [batch, n, n]."""
    lib = load()
    b, n, _ = A.shape
    pa = _dev(A, torch.complex64, "A", (b, n, n))
    if X is None:
        X = torch.empty_like(A)
    px = _dev(X, torch.complex64, "X", (b, n, n))
    _check(lib.helm_zinv_batched(b, n, pa, n * n, n, px, n * n, n, _stream_ptr(stream)), "helm_zinv_batched")
    return X


def _solve(name, f: Factor, B, X, rtol, max_iter):
    lib = load()
    op = f.op
    if B.dim() != 3 or B.shape[0] != op.n_omega or B.shape[2] != op.N:
        raise ValueError(f"B must be [n_omega={op.n_omega}, nrhs, N={op.N}]")
    nrhs = B.shape[1]
    pb = _dev(B, torch.complex128, "B")
    if X is None:
        X = torch.empty_like(B)
    px = _dev(X, torch.complex128, "X", B.shape)
    info = helm_solve_info()
    _check(getattr(lib, name)(f.handle, nrhs, pb, px, float(rtol), int(max_iter), C.byref(info)), name)
    return X, {"iters": info.iters, "max_relres": info.max_relres}


def helm_solve(f: Factor, B: torch.Tensor, X: torch.Tensor | None = None, rtol=1e-10, max_iter=8):
    return _solve("helm_solve", f, B, X, rtol, max_iter)


def helm_adjoint_solve(f: Factor, B: torch.Tensor, X: torch.Tensor | None = None, rtol=1e-10, max_iter=8):
    return _solve("helm_adjoint_solve", f, B, X, rtol, max_iter)


def helm_solve_noalloc(f: Factor, B: torch.Tensor, X: torch.Tensor, rtol=1e-10, max_iter=8, adjoint=False):
    """Same result as helm_solve / helm_adjoint_solve, but the library allocates nothing:
    its working memory is a fixed 32 MiB device array (see include/helm.h).  X must be
    passed in by the caller."""
    lib = load()
    op = f.op
    if B.dim() != 3 or B.shape[0] != op.n_omega or B.shape[2] != op.N:
        raise ValueError(f"B must be [n_omega={op.n_omega}, nrhs, N={op.N}]")
    pb = _dev(B, torch.complex128, "B")
    px = _dev(X, torch.complex128, "X", B.shape)
    info = helm_solve_info()
    _check(lib.helm_solve_noalloc(f.handle, B.shape[1], pb, px, float(rtol), int(max_iter), 1 if adjoint else 0,
                                  C.byref(info)), "helm_solve_noalloc")
    return X, {"iters": info.iters, "max_relres": info.max_relres}


def helm_sources(op: Op, acq: Acq, B: torch.Tensor | None = None) -> torch.Tensor:
    lib = load()
    if B is None:
        B = torch.empty((op.n_omega, acq.n_src, op.N), dtype=torch.complex128, device="cuda")
    _check(lib.helm_sources(op.handle, C.byref(acq.struct), _dev(B, torch.complex128, "B", (op.n_omega, acq.n_src, op.N))),
           "helm_sources")
    return B


def helm_restrict(op: Op, acq: Acq, X: torch.Tensor) -> torch.Tensor:
    lib = load()
    ncol = X.shape[1]
    px = _dev(X, torch.complex128, "X", (op.n_omega, ncol, op.N))
    Y = torch.empty((op.n_omega, ncol, acq.n_rec), dtype=torch.complex128, device="cuda")
    _check(lib.helm_restrict(op.handle, C.byref(acq.struct), ncol, px, _dev(Y, torch.complex128, "Y")),
           "helm_restrict")
    return Y


def helm_restrict_adjoint(op: Op, acq: Acq, Y: torch.Tensor) -> torch.Tensor:
    """X = R(P)^T Y, Y [n_omega, ncol, n_rec] -> X [n_omega, ncol, N]."""
    lib = load()
    ncol = Y.shape[1]
    py = _dev(Y, torch.complex128, "Y", (op.n_omega, ncol, acq.n_rec))
    X = torch.empty((op.n_omega, ncol, op.N), dtype=torch.complex128, device="cuda")
    _check(lib.helm_restrict_adjoint(op.handle, C.byref(acq.struct), ncol, py, _dev(X, torch.complex128, "X")),
           "helm_restrict_adjoint")
    return X


def helm_field_grad(op: Op, U: torch.Tensor, Lam: torch.Tensor) -> torch.Tensor:
    """grad_k = Re sum g_k U_k conj(Lam_k) over frequencies and columns (include/helm.h)."""
    lib = load()
    nrhs = U.shape[1]
    shape = (op.n_omega, nrhs, op.N)
    pu = _dev(U, torch.complex128, "U", shape)
    pl = _dev(Lam, torch.complex128, "Lam", shape)
    grad = torch.empty(op.N, dtype=torch.float64, device="cuda")
    _check(lib.helm_field_grad(op.handle, nrhs, pu, pl, C.c_void_p(grad.data_ptr())), "helm_field_grad")
    return grad


def fwi_misfit_grad(f: Factor, acq: Acq, data: torch.Tensor, alpha, mu, rtol=1e-10, want_fields=False):
    lib = load()
    op = f.op
    pd = _dev(data, torch.complex128, "data", (op.n_omega, acq.n_src, acq.n_rec))
    grad = torch.empty(op.N, dtype=torch.float64, device="cuda")
    U = Lam = None
    pu = pl = C.c_void_p()
    if want_fields:
        U = torch.empty((op.n_omega, acq.n_src, op.N), dtype=torch.complex128, device="cuda")
        Lam = torch.empty_like(U)
        pu, pl = C.c_void_p(U.data_ptr()), C.c_void_p(Lam.data_ptr())
    phi = C.c_double()
    _check(lib.fwi_misfit_grad(f.handle, C.byref(acq.struct), pd, float(alpha), float(mu), float(rtol),
                               C.byref(phi), C.c_void_p(grad.data_ptr()), pu, pl), "fwi_misfit_grad")
    return phi.value, grad, U, Lam


def fwi_hessian_vec(f: Factor, acq: Acq, U: torch.Tensor, Lam: torch.Tensor | None, mt: torch.Tensor, alpha, mu,
                    rtol=1e-10, gauss_newton=False):
    lib = load()
    op = f.op
    shape = (op.n_omega, acq.n_src, op.N)
    pu = _dev(U, torch.complex128, "U", shape)
    pl = _dev(Lam, torch.complex128, "Lam", shape) if Lam is not None else C.c_void_p()
    pm = _dev(mt, torch.float64, "mt", (op.N,))
    hv = torch.empty(op.N, dtype=torch.float64, device="cuda")
    _check(lib.fwi_hessian_vec(f.handle, C.byref(acq.struct), pu, pl, pm, float(alpha), float(mu), float(rtol),
                               1 if gauss_newton else 0, C.c_void_p(hv.data_ptr())), "fwi_hessian_vec")
    return hv


def helm_gamma_solve(nx, nz, alpha0, mu, R: torch.Tensor, Z: torch.Tensor | None = None, lx=1.0, lz=1.0,
                     stream=None) -> torch.Tensor:
    """Z = Gamma(alpha0, mu)^{-1} R; R [N] or [ncol, N] FP64 CUDA tensor."""
    lib = load()
    N = int(nx) * int(nz)
    if R.dim() not in (1, 2) or R.shape[-1] != N:
        raise ValueError(f"R must be [N={N}] or [ncol, N]")
    pr = _dev(R, torch.float64, "R")
    if Z is None:
        Z = torch.empty_like(R)
    pz = _dev(Z, torch.float64, "Z", tuple(R.shape))
    ncol = 1 if R.dim() == 1 else R.shape[0]
    g = helm_grid(int(nx), int(nz), float(lx), float(lz))
    _check(lib.helm_gamma_solve(C.byref(g), float(alpha0), float(mu), ncol, pr, pz, _stream_ptr(stream)),
           "helm_gamma_solve")
    return Z


def bilevel_hypergrad(grids, m_fwi, m_true, acq, omegas, alpha, alpha0, mu, prec=HELM_FP64,
                      cg_rtol=1e-13, cg_max_iter=500, cg_fixed_iters=0, x0=1.0, refine_rtol=1e-10,
                      stream=None, concurrent_models=0, factor_method=0, data_grids=None, m_data=None):
    """grids: list of (nx, nz, lx, lz); m_fwi, m_true: lists of CUDA float64 tensors; acq: one
    Acq for every model, or a list with one per model (the same number of receivers).
    data_grids, m_data: None, or per model the (nx, nz, lx, lz) of another grid of the same
    domain and m' sampled on it, from which the training data are computed."""
    lib = load()
    n = len(grids)
    acqs = list(acq) if isinstance(acq, (list, tuple)) else [acq] * n
    if len(acqs) != n:
        raise ValueError("one acquisition per model")
    A = (helm_acq * n)(*[a.struct for a in acqs])
    acq = acqs[0]
    G = (helm_grid * n)(*[helm_grid(*g) for g in grids])
    pf = (C.c_void_p * n)(*[_dev(t, torch.float64, "m_fwi", (g[0] * g[1],)).value for t, g in zip(m_fwi, grids)])
    pt = (C.c_void_p * n)(*[_dev(t, torch.float64, "m_true", (g[0] * g[1],)).value for t, g in zip(m_true, grids)])
    om, p_om = _dbuf(np.atleast_1d(omegas))
    if (data_grids is None) != (m_data is None):
        raise ValueError("data_grids and m_data go together")
    DG = pd = None
    if data_grids is not None:
        if len(data_grids) != n or len(m_data) != n:
            raise ValueError("one data grid and one m' per model")
        DG = (helm_grid * n)(*[helm_grid(*g) for g in data_grids])
        pd = (C.c_void_p * n)(*[_dev(t, torch.float64, "m_data", (g[0] * g[1],)).value
                                for t, g in zip(m_data, data_grids)])
    opts = helm_pcg_opts(int(cg_max_iter), int(cg_fixed_iters), float(cg_rtol), float(x0), float(refine_rtol),
                         int(concurrent_models), int(factor_method))
    psi, dalpha = C.c_double(), C.c_double()
    dp = np.zeros((acq.n_rec, 2))
    dw = np.zeros(acq.n_rec)
    info = helm_hyper_info()
    _check(lib.bilevel_hypergrad(n, G, pf, pt, A, DG, pd, p_om, len(om), float(alpha), float(alpha0),
                                 float(mu), int(prec), C.byref(opts), _stream_ptr(stream), C.byref(psi),
                                 C.byref(dalpha), dp.ctypes.data_as(C.POINTER(C.c_double)),
                                 dw.ctypes.data_as(C.POINTER(C.c_double)), C.byref(info)), "bilevel_hypergrad")
    return {"psi": psi.value, "dpsi_dalpha": dalpha.value, "dpsi_dp": dp, "dpsi_dw": dw,
            "cg_matvecs": info.cg_matvecs, "cg_relres": info.cg_relres, "solves": info.solves,
            "data_solves": info.data_solves, "max_refine_iters": info.max_refine_iters}


# ------------------------------------------------------------------ tracing (helm_trace.h)

def helm_trace_enable(on=True):
    load().helm_trace_enable(1 if on else 0)


def helm_trace_select(kernel_name=None):
    """Time only the launches of this kernel (None: every kernel)."""
    if load().helm_trace_select((kernel_name or "").encode()) != 0:
        raise ValueError(f"no kernel named {kernel_name!r}")


def helm_trace_reset():
    load().helm_trace_reset()


def helm_trace_read():
    """{kernel name: {"launches", "total_ms", "timed"}} since the last reset (synchronises)."""
    buf = (helm_trace_entry * 64)()
    n = load().helm_trace_read(buf, 64)
    if n < 0:
        raise HelmError(3, "helm_trace_read")
    return {buf[i].name.decode(): {"launches": buf[i].launches, "total_ms": buf[i].total_ms,
                                   "timed": buf[i].timed, "flops": buf[i].flops} for i in range(n)}


def helm_trace_timeline(max_events=200000):
    """[(kernel name, stream index, start_ms, end_ms)] of the timed launches since the last
    reset or read, in launch order (synchronises; the records stay for helm_trace_read)."""
    lib = load()
    buf = (helm_trace_event * max_events)()
    n = lib.helm_trace_timeline(buf, max_events)
    if n < 0:
        raise HelmError(3, "helm_trace_timeline")
    return [(lib.helm_trace_kernel_name(buf[i].kernel).decode(), buf[i].stream, buf[i].start_ms, buf[i].end_ms)
            for i in range(n)]


def helm_launch_count():
    return int(load().helm_launch_count())


class Server:
    """Solve server of include/helm_server.h: factor cache, HBM admission, batching, workers.

    submit() takes host complex128 tensors B [nrhs][N] (pinned memory makes the copies
    asynchronous) and returns a ticket; the server writes X, and the tensors are kept alive
    here until wait() returns for the ticket."""

    def __init__(self, hbm_budget_bytes=0, max_batch_rhs=0, workers=0, max_iter=0):
        lib = load()
        o = helm_server_opts(int(hbm_budget_bytes), int(max_batch_rhs), int(workers), int(max_iter))
        h = C.c_void_p()
        _check(lib.helm_server_create(C.byref(o), C.byref(h)), "helm_server_create")
        self._lib, self.handle = lib, h
        self._keep = {}
        self._grids = {}

    def add_model(self, nx, nz, lx, lz, m) -> int:
        m = np.ascontiguousarray(np.asarray(m, dtype=np.float64).reshape(-1))
        if m.size != nx * nz:
            raise ValueError("m must have nx*nz entries")
        g = helm_grid(nx, nz, lx, lz)
        mid = C.c_int32()
        _check(self._lib.helm_server_add_model(self.handle, C.byref(g), m.ctypes.data_as(C.POINTER(C.c_double)),
                                               C.byref(mid)), "helm_server_add_model")
        self._grids[mid.value] = (nx, nz)
        return mid.value

    def footprint(self, model, prec, nrhs) -> int:
        return int(self._lib.helm_server_footprint(self.handle, model, prec, nrhs))

    def submit(self, model, omega, B: torch.Tensor, X: torch.Tensor | None = None, prec=HELM_MIXED, rtol=1e-10,
               adjoint=False):
        grid = self._grids.get(model)   # an unknown id is left to the library (HELM_EINVAL)
        if B.device.type != "cpu" or B.dtype != torch.complex128 or not B.is_contiguous() or B.dim() != 2 \
                or (grid is not None and B.shape[1] != grid[0] * grid[1]):
            raise ValueError("B must be a contiguous host complex128 tensor [nrhs][N]")
        if X is None:
            X = torch.empty_like(B, pin_memory=B.is_pinned())
        req = helm_request(model, float(omega), int(prec), 1 if adjoint else 0, B.shape[0], C.c_void_p(B.data_ptr()),
                           C.c_void_p(X.data_ptr()), float(rtol))
        t = C.c_int64()
        _check(self._lib.helm_server_submit(self.handle, C.byref(req), C.byref(t)), "helm_server_submit")
        self._keep[t.value] = (B, X)
        return t.value

    def wait(self, ticket):
        info = helm_request_info()
        st = self._lib.helm_server_wait(self.handle, ticket, C.byref(info))
        B, X = self._keep.pop(ticket, (None, None))
        out = {k: getattr(info, k) for k, _ in helm_request_info._fields_}
        out["X"] = X
        if st != 0:
            out["error"] = HelmError(st, "helm_server_wait")
        return out

    def stats(self):
        c = helm_server_counters()
        _check(self._lib.helm_server_stats(self.handle, C.byref(c)), "helm_server_stats")
        return {k: getattr(c, k) for k, _ in helm_server_counters._fields_}

    def close(self):
        if self.handle:
            self._lib.helm_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
