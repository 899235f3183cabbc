"""Thin Python binding of libbicgk (argument marshalling only).

Every step of a solve runs in the library's CUDA kernels; this module only
converts arrays to pointers, picks the memory space and the stream, and turns
return codes into exceptions.  Device arrays are torch CUDA tensors (torch is
used for device memory and streams only); host arrays are numpy arrays.  The
function names mirror the C-ABI in include/bicgk.h.
"""
from __future__ import annotations

import ctypes
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

MEM_HOST, MEM_DEVICE = 0, 1
VARIANTS = {
    "classical_plain": 0,
    "classical_merged": 1,
    "reordered_plain": 2,
    "reordered_merged": 3,
    "pipelined_plain": 4,
    "pipelined_merged": 5,
    "precond_plain": 6,
    "precond_merged": 7,
    "ppipe_plain": 8,
    "ppipe_merged": 9,
    "improved_plain": 10,
    "improved_merged": 11,
}
STATUS = {0: "converged", 1: "maxit", 2: "breakdown", 3: "nonfinite"}
FLAG_NO_STOP_TEST = 1
FLAG_JACOBI = 2
MAX_K = 64

_lock = threading.Lock()
_lib = None


class BicgkError(RuntimeError):
    def __init__(self, rc: int, where: str):
        lib = _load()
        detail = lib.bicgk_last_cuda_error().decode()
        super().__init__(f"{where}: {lib.bicgk_strerror(rc).decode()} (rc={rc}){': ' + detail if detail else ''}")
        self.rc = rc


def _load():
    """Load libbicgk.so (building it first if its sources are newer); fail loudly otherwise."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            lib = ctypes.CDLL(path)
            vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            lib.bicgk_csr_create.argtypes = [ctypes.POINTER(vp), i64, i64, vp, vp, vp, ctypes.c_int, vp]
            lib.bicgk_spmm.argtypes = [vp, i32, vp, vp, vp]
            lib.bicgk_spmm_f32.argtypes = [vp, i32, vp, vp, vp]
            lib.bicgk_solve.argtypes = [vp, i32, vp, vp, dbl, i32, ctypes.c_int, i32, ctypes.c_int, vp, vp, vp, vp,
                                        vp, vp]
            lib.bicgk_op_destroy.argtypes = [vp]
            lib.bicgk_strerror.argtypes = [ctypes.c_int]
            lib.bicgk_strerror.restype = ctypes.c_char_p
            lib.bicgk_last_cuda_error.restype = ctypes.c_char_p
            lib.bicgk_version.restype = ctypes.c_char_p
            lib.bicgk_solve_mixed.argtypes = [vp, i32, vp, vp, dbl, i32, dbl, i32, ctypes.c_int, vp, vp, vp, vp,
                                              vp, vp, vp]
            pp = ctypes.POINTER(ctypes.c_void_p)
            lib.bicgk_batch_create.argtypes = [ctypes.POINTER(vp), i32, vp, vp, pp, pp, pp, vp, ctypes.c_int, vp]
            lib.bicgk_batch_tune.argtypes = [vp, i32, vp, vp, vp, vp]
            lib.bicgk_batch_solve.argtypes = [vp, pp, pp, pp, dbl, i32, ctypes.c_int, i32, ctypes.c_int, vp, vp,
                                              vp, vp]
            lib.bicgk_batch_last_launches.argtypes = [vp, ctypes.POINTER(i64)]
            lib.bicgk_batch_last_loop_iters.argtypes = [vp, ctypes.POINTER(i64)]
            lib.bicgk_batch_tune_persistent.argtypes = [vp, i32, vp, vp]
            lib.bicgk_batch_set_deadline.argtypes = [vp, i64]
            lib.bicgk_batch_persistent_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                                        ctypes.POINTER(i32)]
            lib.bicgk_batch_destroy.argtypes = [vp]
            for f in ("bicgk_batch_create", "bicgk_batch_tune", "bicgk_batch_solve", "bicgk_batch_last_launches",
                      "bicgk_batch_last_loop_iters", "bicgk_batch_tune_persistent", "bicgk_batch_set_deadline",
                      "bicgk_batch_persistent_info",
                      "bicgk_batch_destroy"):
                getattr(lib, f).restype = ctypes.c_int
            lib.bicgk_op_transpose.argtypes = [vp, ctypes.POINTER(vp), vp]
            lib.bicgk_op_set_values.argtypes = [vp, vp, ctypes.c_int, vp]
            lib.bicgk_op_transpose_refresh.argtypes = [vp, vp, vp]
            lib.bicgk_op_get_csr.argtypes = [vp, vp, vp, vp, vp]
            lib.bicgk_spmm_t.argtypes = [vp, i32, vp, vp, ctypes.c_int, vp]
            lib.bicgk_sddmm.argtypes = [vp, i32, vp, vp, dbl, vp, vp]
            for f in ("bicgk_op_transpose", "bicgk_spmm_t", "bicgk_sddmm", "bicgk_op_set_values",
                      "bicgk_op_transpose_refresh", "bicgk_op_get_csr"):
                getattr(lib, f).restype = ctypes.c_int
            lib.bicgk_set_profiling.argtypes = [vp, ctypes.c_int]
            lib.bicgk_set_option.argtypes = [vp, ctypes.c_int, i64]
            lib.bicgk_kernel_times.argtypes = [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_char_p),
                                               ctypes.POINTER(i64), ctypes.POINTER(dbl)]
            lib.bicgk_last_stats.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i32)]
            lib.bicgk_last_groups.argtypes = [vp, ctypes.POINTER(i32)]
            for f in ("bicgk_csr_create", "bicgk_spmm", "bicgk_spmm_f32", "bicgk_solve", "bicgk_solve_mixed", "bicgk_op_destroy",
                      "bicgk_set_profiling",
                      "bicgk_set_option",
                      "bicgk_kernel_times", "bicgk_last_stats", "bicgk_last_groups"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def library_path() -> str:
    return _build.LIB


def version() -> str:
    return _load().bicgk_version().decode()


def strerror(rc: int) -> str:
    return _load().bicgk_strerror(rc).decode()


def _check(rc: int, where: str):
    if rc != 0:
        raise BicgkError(rc, where)


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a):
    if a is None:
        return None
    if _is_torch(a):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def csr_create(rowptr, colidx, vals, stream=None) -> int:
    """Create an operator handle from CSR arrays (numpy on the host or torch CUDA tensors)."""
    lib = _load()
    dev = _is_torch(rowptr)
    if dev:
        for t, dt in ((rowptr, "int32"), (colidx, "int32"), (vals, "float64")):
            if not (t.is_cuda and t.is_contiguous() and str(t.dtype).endswith(dt)):
                raise TypeError("device CSR arrays must be contiguous CUDA tensors of int32/int32/float64")
    else:
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        colidx = np.ascontiguousarray(colidx, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.float64)
    h = ctypes.c_void_p()
    n = rowptr.shape[0] - 1
    nnz = colidx.shape[0]
    rc = lib.bicgk_csr_create(ctypes.byref(h), n, nnz, _ptr(rowptr), _ptr(colidx), _ptr(vals),
                              MEM_DEVICE if dev else MEM_HOST, _stream(stream))
    _check(rc, "bicgk_csr_create")
    return h.value


def op_destroy(handle: int) -> None:
    _check(_load().bicgk_op_destroy(ctypes.c_void_p(handle)), "bicgk_op_destroy")


def spmm(handle: int, X, Y, stream=None) -> None:
    """Y = A X for torch CUDA tensors of shape (N, k), float64, contiguous."""
    k = 1 if X.dim() == 1 else X.shape[1]
    _check(_load().bicgk_spmm(ctypes.c_void_p(handle), k, _ptr(X), _ptr(Y), _stream(stream)), "bicgk_spmm")


def spmm_f32(handle: int, X, Y, stream=None) -> None:
    """Y = A X in FP32 (values rounded once to FP32) for torch CUDA tensors of shape (N, k), float32."""
    if X.dtype != Y.dtype or str(X.dtype) != "torch.float32":
        raise TypeError("spmm_f32 takes float32 tensors")
    k = 1 if X.dim() == 1 else X.shape[1]
    _check(_load().bicgk_spmm_f32(ctypes.c_void_p(handle), k, _ptr(X), _ptr(Y), _stream(stream)),
           "bicgk_spmm_f32")


@dataclass
class SolveResult:
    X: object
    iters: np.ndarray
    status: np.ndarray
    hist: np.ndarray | None
    true_relres: np.ndarray | None


def _is_device(a) -> bool:
    return _is_torch(a) and a.is_cuda


def solve(handle: int, B, X0=None, tol: float = 1e-8, maxit: int = 1000, variant="classical_merged",
          flags: int = 0, X=None, want_hist: bool = True, want_true: bool = True, stream=None) -> SolveResult:
    """Solve A X = B, B of shape (N, k), RHS-interleaved, float64, contiguous.

    A CUDA tensor B makes a device call (X0, X on the device too); a numpy array
    or a CPU tensor (pinned for asynchronous copies) makes a host call, in which
    the library copies B/X0 to the GPU and X back inside the call.
    """
    lib = _load()
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    dev = _is_device(B)
    if _is_torch(B):
        if not (B.is_contiguous() and str(B.dtype).endswith("float64")):
            raise TypeError("B must be a contiguous float64 tensor")
        if X0 is not None and (_is_device(X0) != dev or not X0.is_contiguous()):
            raise TypeError("X0 must be a contiguous tensor on the same device as B")
        if X is None:
            import torch
            X = torch.empty_like(B, pin_memory=not dev) if not dev else torch.empty_like(B)
    else:
        B = np.ascontiguousarray(B, dtype=np.float64)
        if X0 is not None:
            X0 = np.ascontiguousarray(X0, dtype=np.float64)
        if X is None:
            X = np.empty_like(B)
    k = 1 if B.ndim == 1 else B.shape[1]
    iters = np.zeros(k, dtype=np.int32)
    status = np.zeros(k, dtype=np.int32)
    hist = np.empty((maxit + 1, k)) if want_hist else None
    trr = np.empty(k) if want_true else None
    rc = lib.bicgk_solve(ctypes.c_void_p(handle), k, _ptr(B), _ptr(X0), float(tol), int(maxit), v, int(flags),
                         MEM_DEVICE if dev else MEM_HOST, _ptr(X), _ptr(iters), _ptr(status), _ptr(hist),
                         _ptr(trr), _stream(stream))
    _check(rc, "bicgk_solve")
    return SolveResult(X, iters, status, hist, trr)


(OPT_VEC_BLOCKS_PER_SM, OPT_SPMM_BLOCKS_PER_SM, OPT_RHS_GROUPS, OPT_FUSED_DOTS, OPT_THETA_IN_S,
 OPT_HOST_ZERO_COPY, OPT_COMPACT, OPT_PERSISTENT, OPT_SPMM32, OPT_SPMM_ROWS) = 1, 2, 3, 4, 5, 6, 7, 8, 9, 10


def set_option(handle: int, option: int, value: int) -> None:
    """Launch-shape option of an operator (see bicgk_set_option in include/bicgk.h)."""
    _check(_load().bicgk_set_option(ctypes.c_void_p(handle), int(option), int(value)), "bicgk_set_option")


@dataclass
class MixedResult:
    X: object
    outer_iters: np.ndarray
    inner_iters: np.ndarray
    status: np.ndarray
    hist: np.ndarray | None
    true_relres: np.ndarray | None


def solve_mixed(handle: int, B, X0=None, tol: float = 1e-10, max_outer: int = 20, inner_tol: float = 1e-5,
                max_inner: int = 2000, X=None, want_hist: bool = True, stream=None) -> MixedResult:
    """FP64 iterative refinement around FP32 BiCGStab inner solves (bicgk_solve_mixed)."""
    lib = _load()
    dev = _is_device(B)
    if _is_torch(B):
        if not (B.is_contiguous() and str(B.dtype).endswith("float64")):
            raise TypeError("B must be a contiguous float64 tensor")
        if X is None:
            import torch
            X = torch.empty_like(B) if dev else torch.empty_like(B, pin_memory=True)
    else:
        B = np.ascontiguousarray(B, dtype=np.float64)
        if X0 is not None:
            X0 = np.ascontiguousarray(X0, dtype=np.float64)
        if X is None:
            X = np.empty_like(B)
    k = 1 if B.ndim == 1 else B.shape[1]
    outer = np.zeros(k, dtype=np.int32)
    inner = np.zeros(k, dtype=np.int32)
    status = np.zeros(k, dtype=np.int32)
    hist = np.empty((max_outer + 1, k)) if want_hist else None
    trr = np.empty(k)
    rc = lib.bicgk_solve_mixed(ctypes.c_void_p(handle), k, _ptr(B), _ptr(X0), float(tol), int(max_outer),
                               float(inner_tol), int(max_inner), MEM_DEVICE if dev else MEM_HOST, _ptr(X),
                               _ptr(outer), _ptr(inner), _ptr(status), _ptr(hist), _ptr(trr), _stream(stream))
    _check(rc, "bicgk_solve_mixed")
    return MixedResult(X, outer, inner, status, hist, trr)


def set_profiling(handle: int, on: bool) -> None:
    _check(_load().bicgk_set_profiling(ctypes.c_void_p(handle), int(bool(on))), "bicgk_set_profiling")


def kernel_times(handle: int) -> dict:
    """{kernel name: (launches, total ms)} recorded while profiling was on."""
    lib = _load()
    n = ctypes.c_int32(0)
    _check(lib.bicgk_kernel_times(ctypes.c_void_p(handle), 0, ctypes.byref(n), None, None, None), "kernel_times")
    m = n.value
    names = (ctypes.c_char_p * max(m, 1))()
    launches = (ctypes.c_int64 * max(m, 1))()
    ms = (ctypes.c_double * max(m, 1))()
    _check(lib.bicgk_kernel_times(ctypes.c_void_p(handle), m, ctypes.byref(n), names, launches, ms), "kernel_times")
    return {names[i].decode(): (int(launches[i]), float(ms[i])) for i in range(m)}


def last_stats(handle: int) -> dict:
    it, ln, kpi = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32()
    _check(_load().bicgk_last_stats(ctypes.c_void_p(handle), ctypes.byref(it), ctypes.byref(ln), ctypes.byref(kpi)),
           "bicgk_last_stats")
    ng = ctypes.c_int32()
    _check(_load().bicgk_last_groups(ctypes.c_void_p(handle), ctypes.byref(ng)), "bicgk_last_groups")
    return {"loop_iters": it.value, "kernel_launches": ln.value, "kernels_per_iter": kpi.value, "groups": ng.value}


class Operator:
    """Owning wrapper of a bicgk operator (CSR matrix on the GPU plus solver workspace)."""

    def __init__(self, csr=None, rowptr=None, colidx=None, vals=None, stream=None):
        if csr is not None:
            rowptr, colidx, vals = csr.rowptr, csr.colidx, csr.vals
        self.n = int(rowptr.shape[0] - 1)
        self.nnz = int(colidx.shape[0])
        self.handle = csr_create(rowptr, colidx, vals, stream)

    def solve(self, B, **kw) -> SolveResult:
        return solve(self.handle, B, **kw)

    def solve_mixed(self, B, **kw) -> MixedResult:
        return solve_mixed(self.handle, B, **kw)

    def transpose(self, stream=None) -> "Operator":
        """A new Operator for A^T (see bicgk_op_transpose)."""
        h = ctypes.c_void_p()
        _check(_load().bicgk_op_transpose(ctypes.c_void_p(self.handle), ctypes.byref(h), _stream(stream)),
               "bicgk_op_transpose")
        t = Operator.__new__(Operator)
        t.n, t.nnz, t.handle = self.n, self.nnz, h.value
        return t

    def set_values(self, vals, stream=None) -> None:
        """New values for the same sparsity pattern (bicgk_op_set_values): host (numpy) or CUDA
        float64 array of nnz entries.  Captured graphs stay valid; the internal transposed copy
        and the FP32/Jacobi arrays follow."""
        mem = MEM_DEVICE if _is_device(vals) else MEM_HOST
        if not _is_torch(vals):
            vals = np.ascontiguousarray(vals, dtype=np.float64)
        _check(_load().bicgk_op_set_values(ctypes.c_void_p(self.handle), _ptr(vals), mem, _stream(stream)),
               "bicgk_op_set_values")

    def transpose_refresh(self, opT: "Operator", stream=None) -> None:
        """Carry this operator's current values to opT, made from it by transpose()."""
        _check(_load().bicgk_op_transpose_refresh(ctypes.c_void_p(self.handle), ctypes.c_void_p(opT.handle),
                                                  _stream(stream)), "bicgk_op_transpose_refresh")

    def get_csr(self, stream=None):
        """(rowptr, colidx, vals) of the operator's device copy, as numpy arrays."""
        rp = np.empty(self.n + 1, np.int32)
        ci = np.empty(self.nnz, np.int32)
        va = np.empty(self.nnz, np.float64)
        _check(_load().bicgk_op_get_csr(ctypes.c_void_p(self.handle), _ptr(rp), _ptr(ci), _ptr(va), _stream(stream)),
               "bicgk_op_get_csr")
        return rp, ci, va

    def spmm_t(self, X, Y=None, method: int = 0, stream=None):
        """Y = A^T X (method 0: explicit transpose, 1: atomic scatter)."""
        if Y is None:
            import torch
            Y = torch.empty_like(X)
        k = 1 if X.dim() == 1 else X.shape[1]
        _check(_load().bicgk_spmm_t(ctypes.c_void_p(self.handle), k, _ptr(X), _ptr(Y), int(method), _stream(stream)),
               "bicgk_spmm_t")
        return Y

    def sddmm(self, L, X, alpha: float = 1.0, G=None, stream=None):
        """G[e] = alpha * sum_c L[i, c] X[j, c] over the entries e = (i, j) of A."""
        if G is None:
            import torch
            G = torch.empty(self.nnz, dtype=X.dtype, device=X.device)
        k = 1 if X.dim() == 1 else X.shape[1]
        _check(_load().bicgk_sddmm(ctypes.c_void_p(self.handle), k, _ptr(L), _ptr(X), float(alpha), _ptr(G),
                                   _stream(stream)), "bicgk_sddmm")
        return G

    def spmm(self, X, Y=None, stream=None):
        if Y is None:
            import torch
            Y = torch.empty_like(X)
        spmm(self.handle, X, Y, stream)
        return Y

    def spmm_f32(self, X, Y=None, stream=None):
        if Y is None:
            import torch
            Y = torch.empty_like(X)
        spmm_f32(self.handle, X, Y, stream)
        return Y

    def close(self):
        if getattr(self, "handle", None):
            op_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


BATCH_GRAPH, BATCH_LOOP, BATCH_PERSISTENT = 0, 1, 2
E_TIMEOUT = -6


def _ptr_array(items):
    arr = (ctypes.c_void_p * len(items))()
    for i, t in enumerate(items):
        arr[i] = None if t is None else (t.data_ptr() if _is_torch(t) else t.ctypes.data)
    return arr


class Batch:
    """Many independent CSR systems (uneven sizes, 1..64 RHS each) solved together (bicgk_batch_*).

    csrs: list of objects with rowptr/colidx/vals (numpy, host) and ks: RHS count per system.
    """

    def __init__(self, csrs, ks, stream=None):
        lib = _load()
        self.ks = [int(k) for k in ks]
        self.n = [int(c.rowptr.shape[0] - 1) for c in csrs]
        rowptr = [np.ascontiguousarray(c.rowptr, dtype=np.int32) for c in csrs]
        colidx = [np.ascontiguousarray(c.colidx, dtype=np.int32) for c in csrs]
        vals = [np.ascontiguousarray(c.vals, dtype=np.float64) for c in csrs]
        n = np.array(self.n, dtype=np.int64)
        nnz = np.array([c.shape[0] for c in colidx], dtype=np.int64)
        k = np.array(self.ks, dtype=np.int32)
        h = ctypes.c_void_p()
        rc = lib.bicgk_batch_create(ctypes.byref(h), len(csrs), _ptr(n), _ptr(nnz), _ptr_array(rowptr),
                                    _ptr_array(colidx), _ptr_array(vals), _ptr(k), MEM_HOST, _stream(stream))
        _check(rc, "bicgk_batch_create")
        self.handle = h.value

    def tune(self, reps: int = 5, stream=None) -> dict:
        m = len(self.ks)
        g, sg, cpl = np.zeros(m, np.int32), np.zeros(m, np.int32), np.zeros(m, np.int32)
        _check(_load().bicgk_batch_tune(ctypes.c_void_p(self.handle), int(reps), _ptr(g), _ptr(sg), _ptr(cpl),
                                        _stream(stream)), "bicgk_batch_tune")
        return {"vec_grid": g, "spmm_grid": sg, "spmm_cols_per_lane": cpl}

    def tune_persistent(self, reps: int = 3, stream=None) -> np.ndarray:
        """Rows per CTA tile of the persistent mode (bicgk_batch_tune_persistent); per system."""
        rows = np.zeros(len(self.ks), np.int32)
        _check(_load().bicgk_batch_tune_persistent(ctypes.c_void_p(self.handle), int(reps), _ptr(rows),
                                                   _stream(stream)), "bicgk_batch_tune_persistent")
        return rows

    def set_deadline(self, microseconds: int) -> None:
        """Longest wait of one grid barrier of the persistent kernel (bicgk_batch_set_deadline)."""
        _check(_load().bicgk_batch_set_deadline(ctypes.c_void_p(self.handle), int(microseconds)),
               "bicgk_batch_set_deadline")

    def persistent_info(self) -> dict:
        g, f, e = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(_load().bicgk_batch_persistent_info(ctypes.c_void_p(self.handle), ctypes.byref(g), ctypes.byref(f),
                                                   ctypes.byref(e)), "persistent_info")
        return {"grid_blocks": g.value, "from_graph": bool(f.value), "graph_error": e.value}

    def last_loop_iters(self) -> int:
        n = ctypes.c_int64()
        _check(_load().bicgk_batch_last_loop_iters(ctypes.c_void_p(self.handle), ctypes.byref(n)),
               "last_loop_iters")
        return n.value

    def solve(self, Bs, Xs=None, X0s=None, tol: float = 1e-8, maxit: int = 1000, variant="classical_merged",
              flags: int = 0, mode: int = BATCH_GRAPH, stream=None):
        """Bs: list of CUDA tensors (n_i, k_i).  Returns (Xs, iters, status, true_relres) with the
        per-column arrays concatenated in system order."""
        import torch
        if Xs is None:
            Xs = [torch.empty_like(b) for b in Bs]
        tot = sum(self.ks)
        iters = np.zeros(tot, np.int32)
        status = np.zeros(tot, np.int32)
        trr = np.empty(tot)
        v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        x0 = None if X0s is None else _ptr_array(X0s)
        rc = _load().bicgk_batch_solve(ctypes.c_void_p(self.handle), _ptr_array(Bs), x0, _ptr_array(Xs),
                                       float(tol), int(maxit), v, int(flags), int(mode), _ptr(iters),
                                       _ptr(status), _ptr(trr), _stream(stream))
        _check(rc, "bicgk_batch_solve")
        return Xs, iters, status, trr

    def last_launches(self) -> int:
        n = ctypes.c_int64()
        _check(_load().bicgk_batch_last_launches(ctypes.c_void_p(self.handle), ctypes.byref(n)), "last_launches")
        return n.value

    def close(self):
        if getattr(self, "handle", None):
            _check(_load().bicgk_batch_destroy(ctypes.c_void_p(self.handle)), "bicgk_batch_destroy")
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
