"""Batched solves: one graph for many uneven systems vs the per-system launch loop and the oracle.

The graph mode runs every system's branch from one launch; the loop mode calls
bicgk_solve per system.  With the same launch shapes both run the same kernels
in the same order per system, so their results are bitwise equal; the autotuner
changes launch shapes (hence summation orders) and is compared at trajectory
level.  Each system is also checked against the oracle (stable operators: the
solution within 1e-10, iterations +-1).
"""
import numpy as np
import pytest

import oracle
from paper_1907_12874_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bk(cuda):
    from paper_1907_12874_gb300 import bicgk
    return bicgk


def _systems(nsys, seed, lo=6, hi=16, kmax=8):
    u = I.uniform01(seed, 2 * nsys)
    grids = (lo + np.floor(u[:nsys] * (hi - lo + 1))).astype(int)
    ks = (1 + np.floor(u[nsys:] * kmax)).astype(int)
    csrs = [I.convdiff7(int(n), peclet=True) if i % 3 else I.perturbed27(int(n), seed=i)
            for i, n in enumerate(grids)]
    Bs = [I.rhs(c.n, int(k), 100 + i) for i, (c, k) in enumerate(zip(csrs, ks))]
    return csrs, [int(k) for k in ks], Bs


def test_graph_mode_equals_loop_and_oracle(bk, cuda):
    torch = cuda
    csrs, ks, Bs = _systems(10, 5)
    Bd = [torch.from_numpy(b).cuda() for b in Bs]
    with bk.Batch(csrs, ks) as bt:
        Xg, itg, stg, trg = bt.solve(Bd, tol=1e-8, maxit=1000, mode=bk.BATCH_GRAPH)
        lg = bt.last_launches()
        Xl, itl, stl, trl = bt.solve(Bd, tol=1e-8, maxit=1000, mode=bk.BATCH_LOOP)
        Xg2, itg2, _, _ = bt.solve(Bd, tol=1e-8, maxit=1000, mode=bk.BATCH_GRAPH)   # graph replay
    assert lg > 0
    assert np.array_equal(itg, itl) and np.array_equal(stg, stl) and np.array_equal(itg, itg2)
    for a, b, c in zip(Xg, Xl, Xg2):
        assert torch.equal(a, b) and torch.equal(a, c)
    off = 0
    for A, k, B, X in zip(csrs, ks, Bs, Xg):
        ro = oracle.solve(A, B, tol=1e-8, maxit=1000)
        it = itg[off:off + k]
        assert np.all(np.abs(it - ro.iters) <= 1), (it, ro.iters)
        Xn = X.cpu().numpy()
        err = np.linalg.norm(Xn - ro.X, axis=0) / np.linalg.norm(ro.X, axis=0)
        assert np.all(err[it == ro.iters] <= 1e-10), err
        assert np.all(stg[off:off + k] == 0) and np.all(trg[off:off + k] < 2e-8)
        off += k


def test_autotuned_shapes(bk, cuda):
    torch = cuda
    csrs, ks, Bs = _systems(6, 9, lo=8, hi=20)
    Bd = [torch.from_numpy(b).cuda() for b in Bs]
    with bk.Batch(csrs, ks) as bt:
        X0, it0, _, _ = bt.solve(Bd, tol=0.0, maxit=8, flags=1)             # default shapes, 8 iterations
        shapes = bt.tune(reps=3)
        assert np.all(shapes["vec_grid"] >= 1) and np.all(shapes["spmm_grid"] >= 1)
        assert set(np.unique(shapes["spmm_cols_per_lane"])) <= {2, 4}
        X1, it1, _, _ = bt.solve(Bd, tol=0.0, maxit=8, flags=1)             # tuned shapes
        Xg, itg, stg, _ = bt.solve(Bd, tol=1e-8, maxit=1000, mode=bk.BATCH_GRAPH)
        Xl, itl, stl, _ = bt.solve(Bd, tol=1e-8, maxit=1000, mode=bk.BATCH_LOOP)
    for a, b in zip(X0, X1):
        a, b = a.cpu().numpy(), b.cpu().numpy()
        assert np.all(np.linalg.norm(a - b, axis=0) <= 1e-12 * np.linalg.norm(a, axis=0))
    assert np.array_equal(itg, itl) and np.array_equal(stg, stl)
    for a, b in zip(Xg, Xl):
        assert torch.equal(a, b)
