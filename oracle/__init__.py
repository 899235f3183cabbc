"""FP64 CPU oracle for multi-RHS BiCGStab (test infrastructure only).

The oracle is the correctness reference for the CUDA library: a plain C
implementation of Algorithms 1, 2, 4 and 6 of Krasnopolsky (arXiv:1907.12874),
in the listings' order and notation, with compensated dot products and no
fused multiply-add.  It shares no code with the CUDA path.  Only the tests,
the smoke check and the benchmark's CPU-baseline leg use it.

``build()`` compiles ``bicgstab_ref.c`` with gcc (OpenMP over rows for the
SpMV and the elementwise loops; dot products stay serial, in row order).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bicgstab_ref.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

# variant ids (same order as the library's enum)
CLASSICAL_BASIC, CLASSICAL_MERGED, REORDERED_BASIC, REORDERED_MERGED, PIPELINED_BASIC, PIPELINED_MERGED = range(6)
VARIANTS = {
    "classical_plain": CLASSICAL_BASIC,
    "classical_merged": CLASSICAL_MERGED,
    "reordered_plain": REORDERED_BASIC,
    "reordered_merged": REORDERED_MERGED,
    "pipelined_plain": PIPELINED_BASIC,
    "pipelined_merged": PIPELINED_MERGED,
    "precond_plain": 6,
    "precond_merged": 7,
    "ppipe_plain": 8,
    "ppipe_merged": 9,
    "improved_plain": 10,
    "improved_merged": 11,
}
JACOBI = 2
CONVERGED, MAXIT, BREAKDOWN, NONFINITE = range(4)
NO_STOP_TEST = 1


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, no FMA contraction, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
            lib.oracle_solve.argtypes = [ctypes.c_int, i64, vp, vp, vp, i32, vp, vp, dbl, i32, i32,
                                         vp, vp, vp, vp, vp, vp, vp]
            lib.oracle_solve.restype = ctypes.c_int
            lib.oracle_spmm.argtypes = [i64, vp, vp, vp, i32, vp, vp]
            lib.oracle_spmm.restype = ctypes.c_int
            lib.oracle_threads.restype = ctypes.c_int
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            lib.oracle_set_threads.restype = None
            lib.oracle_solve_mixed.argtypes = [i64, vp, vp, vp, i32, vp, vp, dbl, i32, dbl, i32, vp, vp, vp, vp, vp,
                                               vp]
            lib.oracle_solve_mixed.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def threads() -> int:
    return int(_load().oracle_threads())


def set_threads(n: int) -> None:
    """Run the following oracle calls on n OpenMP threads (timing on one core and on all)."""
    _load().oracle_set_threads(int(n))


def spmm(A, X: np.ndarray) -> np.ndarray:
    """Y = A X for an interleaved (N, k) block."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X.reshape(-1, 1)
    Y = np.empty_like(X)
    rc = _load().oracle_spmm(A.n, _ptr(A.rowptr), _ptr(A.colidx), _ptr(A.vals), X.shape[1], _ptr(X), _ptr(Y))
    if rc != 0:
        raise ValueError("oracle_spmm: bad argument")
    return Y


class Result:
    def __init__(self, X, R, iters, status, hist, true_relres, traffic):
        self.X, self.R, self.iters, self.status = X, R, iters, status
        self.hist, self.true_relres, self.traffic = hist, true_relres, traffic


def solve(A, B: np.ndarray, X0=None, tol: float = 1e-8, maxit: int = 1000,
          variant="classical_merged", flags: int = 0) -> Result:
    """Solve A X = B (B of shape (N, k), RHS-interleaved) with one of the six forms."""
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    B = np.ascontiguousarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B.reshape(-1, 1)
    n, k = B.shape
    if n != A.n:
        raise ValueError("B rows != A rows")
    X0c = None if X0 is None else np.ascontiguousarray(np.asarray(X0, dtype=np.float64).reshape(n, k))
    X = np.empty((n, k))
    R = np.empty((n, k))
    iters = np.zeros(k, dtype=np.int32)
    status = np.zeros(k, dtype=np.int32)
    hist = np.empty((maxit + 1, k))
    trr = np.empty(k)
    traffic = np.zeros(4, dtype=np.int64)
    rc = _load().oracle_solve(v, n, _ptr(A.rowptr), _ptr(A.colidx), _ptr(A.vals), k, _ptr(B), _ptr(X0c),
                              float(tol), int(maxit), int(flags), _ptr(X), _ptr(R), _ptr(iters),
                              _ptr(status), _ptr(hist), _ptr(trr), _ptr(traffic))
    if rc != 0:
        raise ValueError(f"oracle_solve: bad argument (rc={rc})")
    return Result(X, R, iters, status, hist, trr, traffic)


class MixedResult:
    def __init__(self, X, outer_iters, inner_iters, status, hist, true_relres):
        self.X, self.outer_iters, self.inner_iters = X, outer_iters, inner_iters
        self.status, self.hist, self.true_relres = status, hist, true_relres


def solve_mixed(A, B: np.ndarray, X0=None, tol: float = 1e-10, max_outer: int = 20, inner_tol: float = 1e-5,
                max_inner: int = 2000) -> MixedResult:
    """FP64 iterative refinement around FP32 inner solves (Algorithm 2 in FP32 storage)."""
    B = np.ascontiguousarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B.reshape(-1, 1)
    n, k = B.shape
    X0c = None if X0 is None else np.ascontiguousarray(np.asarray(X0, dtype=np.float64).reshape(n, k))
    X = np.empty((n, k))
    outer = np.zeros(k, dtype=np.int32)
    inner = np.zeros(k, dtype=np.int32)
    status = np.zeros(k, dtype=np.int32)
    hist = np.empty((max_outer + 1, k))
    trr = np.empty(k)
    rc = _load().oracle_solve_mixed(n, _ptr(A.rowptr), _ptr(A.colidx), _ptr(A.vals), k, _ptr(B), _ptr(X0c),
                                    float(tol), int(max_outer), float(inner_tol), int(max_inner), _ptr(X),
                                    _ptr(outer), _ptr(inner), _ptr(status), _ptr(hist), _ptr(trr))
    if rc != 0:
        raise ValueError(f"oracle_solve_mixed: bad argument (rc={rc})")
    return MixedResult(X, outer, inner, status, hist, trr)


def adjoint_dense(A, B: np.ndarray, W: np.ndarray):
    """Gradients of L = sum(W * X), X = A^-1 B, by dense LAPACK solves (reference for the adjoint path).

    Lambda = A^-T W;  dL/dB = Lambda;  dL/dA_ij = -sum_c Lambda_ic X_jc on the nonzero pattern
    (from dX = -A^-1 dA X + A^-1 dB).  Returns (X, dB, dvals) with dvals in CSR entry order.
    """
    D = A.to_dense()
    X = np.linalg.solve(D, B)
    lam = np.linalg.solve(D.T, W)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    dvals = -np.einsum("ec,ec->e", lam[rows], X[A.colidx])
    return X, lam, dvals
