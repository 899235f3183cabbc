"""Parity bars measured on the oracle itself, and column-parallel oracle runs.

Test infrastructure: imports the oracle and the input generators only.

Where BiCGStab amplifies rounding differences (nearly symmetric operators: the
h-scaled convection-diffusion of the benchmark configurations, Poisson) the
stopping iterate of any two correct FP64 implementations that sum in different
orders differs by far more than one rounding unit, and so do their iteration
counts.  The bars for comparing the CUDA path with the oracle there are taken
from the oracle's own response to one rounding unit: the oracle solves the same
system again with every entry of b moved by about 2^-52 relative (a fresh draw
each time), and

  * the solution bar is ten times the largest relative change of the
    oracle's solution over the draws and over the case's columns (never below
    the fixed bar the caller gives, 1e-10 for the spec comparison);
  * the iteration bar is twice the largest change of an iteration count over
    the draws and columns, at least one.

The columns of a case share the operator and draw their right-hand sides from
one distribution, so their responses are pooled: on the h-scaled operator the
iteration count of a column is, past the first few dozen iterations, a random
variable under rounding (sixty draws of one 16^3 column spread it over 46..59
around the oracle's 48), and a few draws per column would not see its tails.
The CUDA path injects rounding differences at every iteration (summation order
of the dot products, fused multiply-adds), not only in b, so a factor above one
is needed; ten and two keep the bars within an order of magnitude of what the
oracle itself shows.  Every bar is printed so that a run's log shows it.

Columns never interact (the oracle's column c of a k-column solve is bitwise its
one-column solve of column c; pinned in the oracle tests), so large cases run
the oracle on single columns concurrently: ctypes releases the GIL and each
worker thread runs its column on one OpenMP thread.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle

ULP = 2.0 ** -52

# one line per measured bar, printed by tests/conftest.py in the run's terminal summary
RECORD: list = []


def colerr(X, Xo):
    """Relative 2-norm difference per column (absolute where the reference column is zero)."""
    num = np.linalg.norm(X - Xo, axis=0)
    den = np.linalg.norm(Xo, axis=0)
    return num / np.where(den == 0, 1.0, den)


def _workers(n_jobs: int) -> int:
    return max(1, min(n_jobs, os.cpu_count() or 1))


class Cols:
    """Per-column oracle results stacked as a k-column result (X, iters, status, hist, true_relres)."""

    def __init__(self, results):
        self.X = np.concatenate([r.X for r in results], axis=1)
        self.status = np.concatenate([r.status for r in results])
        self.hist = np.concatenate([r.hist for r in results], axis=1)
        self.true_relres = np.concatenate([r.true_relres for r in results])
        if hasattr(results[0], "iters"):
            self.iters = np.concatenate([r.iters for r in results])
        if hasattr(results[0], "outer_iters"):
            self.outer_iters = np.concatenate([r.outer_iters for r in results])
            self.inner_iters = np.concatenate([r.inner_iters for r in results])


def solve_columns(A, B, cols=None, X0=None, mixed=False, **kw):
    """The oracle on each listed column of B alone (all columns if None), concurrently."""
    cols = list(range(B.shape[1])) if cols is None else list(cols)

    def one(c):
        oracle.set_threads(1)        # this worker thread's OpenMP team only
        b = np.ascontiguousarray(B[:, [c]])
        x0 = None if X0 is None else np.ascontiguousarray(X0[:, [c]])
        return (oracle.solve_mixed if mixed else oracle.solve)(A, b, X0=x0, **kw)

    with ThreadPoolExecutor(_workers(len(cols))) as ex:
        return Cols(list(ex.map(one, cols)))


def rounding_response(A, B, ro, draws=6, seed=11, cols=None, X0=None, with_hist=False, **kw):
    """The oracle's own response to one rounding unit in b, per column of `ro` (an oracle result for
    the columns `cols` of B): (largest relative solution change, largest |change of the iteration
    count|, the iteration counts of every draw as an array (draws, columns)); with `with_hist`, also
    the largest relative change of a residual-history entry that both runs recorded."""
    cols = list(range(B.shape[1])) if cols is None else list(cols)
    rng = np.random.default_rng(seed)
    pert = [B[:, cols] * (1.0 + ULP * rng.standard_normal((B.shape[0], len(cols)))) for _ in range(draws)]
    jobs = [(d, j) for d in range(draws) for j in range(len(cols))]

    def one(job):
        d, j = job
        oracle.set_threads(1)
        b = np.ascontiguousarray(pert[d][:, [j]])
        x0 = None if X0 is None else np.ascontiguousarray(X0[:, [cols[j]]])
        return oracle.solve(A, b, X0=x0, **kw)

    with ThreadPoolExecutor(_workers(len(jobs))) as ex:
        res = list(ex.map(one, jobs))
    sol = np.zeros(len(cols))
    hst = np.zeros(len(cols))
    its = np.zeros((draws, len(cols)), dtype=np.int64)
    for (d, j), r in zip(jobs, res):
        sol[j] = max(sol[j], float(colerr(r.X, ro.X[:, [j]])[0]))
        its[d, j] = int(r.iters[0])
        if with_hist:
            a, b = r.hist[:, 0], ro.hist[:, j]
            both = np.isfinite(a) & np.isfinite(b) & (b != 0)
            if both.any():
                hst[j] = max(hst[j], float(np.max(np.abs(a[both] - b[both]) / np.abs(b[both]))))
    spread = np.abs(its - ro.iters[None, :].astype(np.int64)).max(axis=0)
    if with_hist:
        return sol, spread, its, hst
    return sol, spread, its


def derived_bars(A, B, ro, floor=1e-10, draws=None, seed=11, cols=None, X0=None, label="", **kw):
    """(solution bar, iteration bar) per column from the oracle's rounding response, pooled over
    the case's columns (module doc).  Draws: at least 6 per column and 24 in all by default."""
    ncols = B.shape[1] if cols is None else len(cols)
    if draws is None:
        draws = max(6, -(-24 // ncols))
    sol, spread, _ = rounding_response(A, B, ro, draws=draws, seed=seed, cols=cols, X0=X0, **kw)
    n = sol.shape[0]
    sol_bar = np.full(n, max(floor, 10.0 * float(sol.max())))
    it_bar = np.full(n, max(1, 2 * int(spread.max())))
    line = (f"{label or A.name}: oracle one-unit response over {draws} draws x {n} columns: solution max "
            f"{sol.max():.2e}, iterations +-{int(spread.max())} -> solution bar {sol_bar[0]:.2e}, iteration bar "
            f"+-{it_bar[0]}")
    RECORD.append(line)
    print(f"[bars] {line}")
    return sol_bar, it_bar


def trajectory_bars(A, B, m, floor=1e-12, hist_floor=1e-10, draws=3, seed=17, cols=None,
                    variant="classical_merged", flags=0, ro=None):
    """Bars for x_m after m fixed iterations and for the residual history up to m: max(floor, 10 x
    the oracle's largest relative change of x_m when b moves by one rounding unit), and the same
    for the history entries (at least hist_floor), per column.  Returns (x bar, oracle result,
    oracle x response, history bar)."""
    cols = list(range(B.shape[1])) if cols is None else list(cols)
    kw = dict(tol=0.0, maxit=m, variant=variant, flags=oracle.NO_STOP_TEST | flags)
    if ro is None:
        ro = solve_columns(A, B, cols=cols, **kw)
    sol, _, _, hst = rounding_response(A, B, ro, draws=draws, seed=seed, cols=cols, with_hist=True, **kw)
    return np.maximum(floor, 10.0 * sol), ro, sol, np.maximum(hist_floor, 10.0 * hst)


def column_bars(A, B, ro, floor=1e-10, draws=3, seed=13, X0=None, label="", **kw):
    """Per-column bars for operators where rounding differences do not grow (no pooling): the
    solution bar max(floor, 10 x the column's own largest one-unit response), the iteration bar
    max(1, 2 x the column's largest one-unit change).  A column whose solution is unusually
    sensitive (a near-stagnation phase moves the oracle's own stopping iterate by 1e-10 for one
    rounding unit in b) gets a bar that reflects it; the others keep the floor."""
    sol, spread, _ = rounding_response(A, B, ro, draws=draws, seed=seed, X0=X0, **kw)
    sol_bar = np.maximum(floor, 10.0 * sol)
    it_bar = np.maximum(1, 2 * spread)
    if np.any(sol_bar > floor):
        line = (f"{label or A.name}: per-column one-unit response max {sol.max():.2e} -> solution bars up to "
                f"{sol_bar.max():.2e}")
        RECORD.append(line)
        print(f"[bars] {line}")
    return sol_bar, it_bar
