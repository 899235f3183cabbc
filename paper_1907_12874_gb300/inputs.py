"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module only *produces data*: the CSR operators of the workloads and the
right-hand sides.  It holds none of the solver's arithmetic (no products with
A, no dot products, no Krylov recurrences), so the oracle and the CUDA path can
both consume what it makes without sharing any of the method.

Operators
---------
* ``convdiff7(n, beta)`` -- 3-D convection-diffusion ``-lap(u) + beta.grad(u)``
  on the unit cube, n^3 interior unknowns, h = 1/(n+1), homogeneous Dirichlet
  boundary eliminated, first-order upwind convection (beta > 0), every equation
  multiplied by h^2.  Row of unknown (i, j, l), index ``i + n*j + n*n*l``:
  diagonal ``6 + c*(b1+b2+b3)``, "minus" neighbour in dimension d
  ``-1 - c*b_d``, "plus" neighbour ``-1``, columns ascending; ``c = h`` by
  default (convection velocity beta), ``c = 1`` with ``peclet=True`` (mesh
  Peclet number beta).  ``beta = (0, 0, 0)`` gives the 7-point Poisson matrix
  of the paper's single-node tests (Sec. 2.3, 200^3 cells).
* ``perturbed27(n, seed)`` -- 27-point stencil, every off-diagonal
  ``-U[0.5, 1.5]`` drawn independently, diagonal = sum of |off-diagonals| + 1
  (strictly diagonally dominant, nonsymmetric).

Random numbers
--------------
``uniform(seed, count)`` is a counter-based splitmix64 stream: value ``m`` is
``mix(seed + (m+1)*0x9E3779B97F4A7C15)`` (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), turned into a double in [0, 1)
from its top 53 bits and mapped to [-1, 1).  Right-hand sides are drawn in the
RHS-interleaved index order ``i*k + c`` (the paper stores the k vectors
row-wise in one vector, Sec. 3.1).
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

DEFAULT_BETA = (1.0, 0.5, 0.25)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` doubles in [0, 1) from the splitmix64 stream, starting at draw ``offset``."""
    with np.errstate(over="ignore"):
        ctr = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + ctr * _GAMMA
        bits = _mix(z) >> np.uint64(11)
    return bits.astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` doubles in [-1, 1): ``2*u - 1`` of :func:`uniform01` (exact in FP64)."""
    return 2.0 * uniform01(seed, count, offset) - 1.0


def rhs(n_rows: int, k: int, seed: int) -> np.ndarray:
    """RHS block, shape (n_rows, k), C-contiguous, so element (i, c) sits at i*k + c."""
    return uniform(seed, n_rows * k).reshape(n_rows, k)


class CSR:
    """Plain CSR container: int32 row pointers and column indices, FP64 values."""

    def __init__(self, rowptr: np.ndarray, colidx: np.ndarray, vals: np.ndarray, name: str = ""):
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        self.colidx = np.ascontiguousarray(colidx, dtype=np.int32)
        self.vals = np.ascontiguousarray(vals, dtype=np.float64)
        self.name = name

    @property
    def n(self) -> int:
        return int(self.rowptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.colidx.shape[0])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        d[rows, self.colidx] = self.vals
        return d

    def to_scipy(self):
        """scipy CSR of copies of the arrays: scipy may sort or merge the entries of its own arrays in
        place (repeated column indices), which must not change this matrix."""
        import scipy.sparse as sp
        return sp.csr_matrix((self.vals.copy(), self.colidx.copy(), self.rowptr.copy()), shape=(self.n, self.n))


def _assemble(n_rows: int, cols: list, vals: list, valid: list, name: str) -> CSR:
    """Build CSR from per-slot column/value/validity arrays (slots in ascending column order)."""
    cols_a = np.stack(cols, axis=1)
    vals_a = np.stack(vals, axis=1)
    valid_a = np.stack(valid, axis=1)
    counts = valid_a.sum(axis=1)
    rowptr = np.zeros(n_rows + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("nnz exceeds int32 range")
    return CSR(rowptr.astype(np.int32), cols_a[valid_a].astype(np.int32), vals_a[valid_a], name)


def convdiff7(n: int, beta=DEFAULT_BETA, peclet: bool = False) -> CSR:
    """7-point upwind convection-diffusion (or Poisson for beta = 0) on an n^3 grid."""
    if n < 1:
        raise ValueError("n must be >= 1")
    h = 1.0 / (n + 1)
    c = 1.0 if peclet else h
    b = [float(x) for x in beta]
    N = n ** 3
    idx = np.arange(N, dtype=np.int64)
    i, j, l = idx % n, (idx // n) % n, idx // (n * n)
    ones = np.ones(N)
    strides = (1, n, n * n)
    coords = (i, j, l)
    cols, vals, valid = [], [], []
    # ascending column order: -z, -y, -x, diag, +x, +y, +z
    for d in (2, 1, 0):
        cols.append(idx - strides[d])
        vals.append(ones * (-1.0 - c * b[d]))
        valid.append(coords[d] > 0)
    cols.append(idx)
    vals.append(ones * (6.0 + c * (b[0] + b[1] + b[2])))
    valid.append(np.ones(N, dtype=bool))
    for d in (0, 1, 2):
        cols.append(idx + strides[d])
        vals.append(-ones)
        valid.append(coords[d] < n - 1)
    tag = "poisson7" if not any(b) else "convdiff7"
    return _assemble(N, cols, vals, valid, f"{tag}_{n}^3")


def perturbed27(n: int, seed: int, margin: float = 1.0) -> CSR:
    """27-point stencil with off-diagonals -U[0.5,1.5], diagonal = sum|off| + margin."""
    N = n ** 3
    idx = np.arange(N, dtype=np.int64)
    i, j, l = idx % n, (idx // n) % n, idx // (n * n)
    cols, valid, offs = [], [], []
    for dl in (-1, 0, 1):
        for dj in (-1, 0, 1):
            for di in (-1, 0, 1):
                cols.append(idx + di + n * dj + n * n * dl)
                valid.append((i + di >= 0) & (i + di < n) & (j + dj >= 0) & (j + dj < n)
                             & (l + dl >= 0) & (l + dl < n))
                offs.append((di, dj, dl) == (0, 0, 0))
    valid_a = np.stack(valid, axis=1)
    n_off = int(valid_a.sum()) - N
    draws = -(0.5 + uniform01(seed, n_off))  # -U[0.5, 1.5], drawn in row-major nnz order
    vals_a = np.zeros(valid_a.shape)
    off_mask = valid_a.copy()
    off_mask[:, 13] = False
    vals_a[off_mask] = draws
    vals_a[:, 13] = -vals_a.sum(axis=1) + margin  # sum |off| + margin (all off-diagonals negative)
    vals = [vals_a[:, s] for s in range(27)]
    return _assemble(N, cols, vals, valid, f"perturbed27_{n}^3")


def batch_draws(nsys: int = 64, seed: int = 11, lo: int = 16, hi: int = 64, kmax: int = 8):
    """Grid edges and RHS counts of a batch of independent systems: system i has an n_i^3 grid,
    n_i uniform on {lo..hi}, and k_i right-hand sides uniform on {1..kmax}, drawn from one
    splitmix64 stream (the first nsys draws give the grids, the next nsys the RHS counts).  The
    right-hand sides of system i are ``rhs(n_i^3, k_i, 200 + i)``.  The defaults are the batched
    workload: 64 systems, grids 16^3..64^3, 1..8 right-hand sides."""
    u = uniform01(seed, 2 * nsys)
    grids = [int(lo + np.floor(x * (hi - lo + 1))) for x in u[:nsys]]
    ks = [int(1 + np.floor(x * kmax)) for x in u[nsys:]]
    return grids, ks
