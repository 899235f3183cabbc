"""The oracle's pins catch plausible mistakes.

Each case plants one mistake (a dropped term, a wrong sign, a wrong operand
or index) in a copy of the oracle's C source, compiles the copy and runs a
compact set of the pins (LAPACK dense solve, r_j = b - A x_j, equivalence of
the first iterates with Algorithm 1, stop at the first crossing, Table 2
traffic).  The unmodified source must pass the same checks.
"""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from paper_1907_12874_gb300 import inputs as I

SRC = open(os.path.join(os.path.dirname(oracle.__file__), "bicgstab_ref.c")).read()

MUTANTS = {
    "merged r update sign": ("AT(r, i) = si - omega * AT(t, i);", "AT(r, i) = si + omega * AT(t, i);"),
    "p update drops -omega v": ("beta * (AT(p, i) - omega * AT(v, i))", "beta * (AT(p, i))"),
    "beta uses omega/alpha": ("(rho1 / rho) * (alpha / omega)", "(rho1 / rho) * (omega / alpha)"),
    "merged estimate uses psi": ("theta - omega * phi", "theta - omega * psi"),
    "delta against r instead of r0": ("double delta = dot(A, v, r0); rw(2, 0); /* delta_j = (v_j, r_0) */",
                                      "double delta = dot(A, v, r); rw(2, 0); /* delta_j = (v_j, r_0) */"),
    "x update takes t for s": ("AT(x, i) = AT(x, i) + alpha * AT(p, i) + omega * AT(s, i);",
                               "AT(x, i) = AT(x, i) + alpha * AT(p, i) + omega * AT(t, i);"),
    "pipelined q from old s": ("double qn = ri - alpha * sn;", "double qn = ri - alpha * si;"),
    "pipelined alpha denominator sign": ("sigma + beta * delta - beta * omega * psi",
                                         "sigma + beta * delta + beta * omega * psi"),
    "reordered rho sign": ("rho1 = -omega * psi;", "rho1 = omega * psi;"),
    "reordered z uses s for q": ("double zi = thi - omega * AT(q, i);", "double zi = thi - omega * AT(s, i);"),
    "pipelined w drops alpha v": ("double wn = AT(y, i) - omega * (AT(t, i) - alpha * AT(v, i));",
                                  "double wn = AT(y, i) - omega * AT(t, i);"),
    "spmv skips the last entry": ("e < A->rowptr[i + 1]; ++e) acc +=", "e < A->rowptr[i + 1] - 1; ++e) acc +="),
    "stop test 10x too loose": ("est < eps2)", "est < 100.0 * eps2)"),
    "refinement subtracts d": ("AT(x, i) = AT(x, i) + (double)AT(d32, i);", "AT(x, i) = AT(x, i) - (double)AT(d32, i);"),
    "fp32 inner r update sign": ("AT(r, i) = si - of * AT(t, i);", "AT(r, i) = si + of * AT(t, i);"),
    "improved sigma sign": ("double sigma1 = gam - omega1 * eta;", "double sigma1 = gam + omega1 * eta;"),
    "improved tau drops beta tau": ("double tau1 = sigma + beta1 * tau - delta1 * pi;",
                                    "double tau1 = sigma - delta1 * pi;"),
    "improved t uses u_{j+1}": ("double ti = AT(u, i) - alpha1 * qi;", "double ti = AT(s, i) - alpha1 * qi;"),
    "ppipe r^ drops alpha z^": ("AT(rh, i) = qhi - omega * (AT(wh, i) - alpha * AT(zh, i));",
                                "AT(rh, i) = qhi - omega * AT(wh, i);"),
    "ppipe q^ from old s^": ("AT(qh, i) = rhi - alpha * sn;", "AT(qh, i) = rhi - alpha * shi;"),
    "precond x uses p for p^": ("      for (int64_t i = 0; i < n; ++i) AT(x, i) = AT(x, i) + alpha * AT(ph, i) + omega * AT(sh, i);\n      rw(3, 1);\n      out->iters = j + 1;",
                                "      for (int64_t i = 0; i < n; ++i) AT(x, i) = AT(x, i) + alpha * AT(p, i) + omega * AT(sh, i);\n      rw(3, 1);\n      out->iters = j + 1;"),
}


def _compile(src: str, tag: str):
    d = tempfile.mkdtemp(prefix="oracle_mut_")
    c, so = os.path.join(d, "m.c"), os.path.join(d, f"m_{tag}.so")
    open(c, "w").write(src)
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", "-o", so, c, "-lm"],
                   check=True)
    lib = ctypes.CDLL(so)
    i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
    lib.oracle_solve.argtypes = [ctypes.c_int, i64, vp, vp, vp, i32, vp, vp, dbl, i32, i32, vp, vp, vp, vp, vp, vp, vp]
    lib.oracle_solve_mixed.argtypes = [i64, vp, vp, vp, i32, vp, vp, dbl, i32, dbl, i32, vp, vp, vp, vp, vp, vp]
    return lib


def _solve(lib, A, B, variant, tol, maxit, flags=0):
    p = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    n, k = B.shape
    X, R = np.empty((n, k)), np.empty((n, k))
    it, st = np.zeros(k, np.int32), np.zeros(k, np.int32)
    hist, trr, tr = np.empty((maxit + 1, k)), np.empty(k), np.zeros(4, np.int64)
    rc = lib.oracle_solve(oracle.VARIANTS[variant], n, p(A.rowptr), p(A.colidx), p(A.vals), k, p(B), None,
                          tol, maxit, flags, p(X), p(R), p(it), p(st), p(hist), p(trr), p(tr))
    assert rc == 0
    return X, R, it, st, hist, tr


TABLE2 = {"classical_plain": (18, 4), "classical_merged": (14, 4), "pipelined_plain": (34, 9),
          "pipelined_merged": (18, 8), "reordered_plain": (22, 6), "reordered_merged": (15, 6),
          "precond_plain": (18, 4), "precond_merged": (15, 4), "ppipe_plain": (43, 13), "ppipe_merged": (23, 11),
          "improved_plain": (27, 6), "improved_merged": (14, 6)}


def _pins_pass(lib) -> bool:
    A = I.convdiff7(4, peclet=True)
    B = I.rhs(A.n, 2, 5)
    D = A.to_dense()
    Xd = np.linalg.solve(D, B)
    ref1 = None
    for v in oracle.VARIANTS:
        X, R, it, st, hist, tr = _solve(lib, A, B, v, 1e-12, 300)
        if not np.all(st == 0):
            return False
        gap = np.linalg.norm(R - (B - D @ X), axis=0)     # r at the break = b - A x, far below tol*||b||
        if np.any(gap > 0.1 * 1e-12 * np.linalg.norm(B, axis=0)):
            return False
        if np.max(np.linalg.norm(X - Xd, axis=0) / np.linalg.norm(Xd, axis=0)) > 1e-9:
            return False
        eps = 1e-12 * np.linalg.norm(B, axis=0)
        for c in range(2):
            h = hist[: it[c] + 1, c]
            if not (h[-1] < eps[c] and np.all(h[:-1] >= eps[c])):
                return False
        X, R, it, st, hist, tr = _solve(lib, A, B, v, 0.0, 3, 1)
        if np.max(np.abs(R - (B - D @ X))) > 1e-12 * (1 + np.abs(X).max()):
            return False
        if ref1 is None:
            ref1 = X
        elif np.max(np.abs(X - ref1)) > 1e-10 * np.abs(ref1).max():
            return False
        if (tr[0], tr[1]) != (3 * 2 * TABLE2[v][0], 3 * 2 * TABLE2[v][1]):
            return False
    # Jacobi preconditioner (M = diag(A), not a multiple of I here): Algorithms 5, 6 and 7
    A2 = I.perturbed27(4, seed=6)
    Xd2 = np.linalg.solve(A2.to_dense(), B[: A2.n] if A2.n <= B.shape[0] else I.rhs(A2.n, 2, 5))
    B2 = A2.to_dense() @ Xd2
    for v in ("precond_plain", "precond_merged", "ppipe_plain", "ppipe_merged", "reordered_plain", "reordered_merged"):
        X, R, it, st, hist, tr = _solve(lib, A2, B2, v, 1e-12, 300, 2)
        if not np.all(st == 0) or np.max(np.linalg.norm(X - Xd2, axis=0) / np.linalg.norm(Xd2, axis=0)) > 1e-9:
            return False
    # mixed-precision refinement: FP64 accuracy from FP32 inner solves
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    X = np.empty_like(B)
    oi, ii, st = np.zeros(2, np.int32), np.zeros(2, np.int32), np.zeros(2, np.int32)
    hist, trr = np.empty((31, 2)), np.empty(2)
    lib.oracle_solve_mixed(A.n, p(A.rowptr), p(A.colidx), p(A.vals), 2, p(B), None, 1e-13, 30, 1e-5, 500, p(X),
                           p(oi), p(ii), p(st), p(hist), p(trr))
    if not np.all(st == 0) or np.max(np.linalg.norm(X - Xd, axis=0) / np.linalg.norm(Xd, axis=0)) > 1e-9:
        return False
    return True


def test_unmodified_oracle_passes_the_compact_pins():
    assert _pins_pass(_compile(SRC, "orig"))


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistake_is_caught(name):
    old, new = MUTANTS[name]
    assert SRC.count(old) >= 1, f"mutation site not found: {old}"
    lib = _compile(SRC.replace(old, new), name.replace(" ", "_").replace("/", "_"))
    assert not _pins_pass(lib), f"planted mistake not caught: {name}"
