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


# systems of the batched workload (64 convection-diffusion systems, grids 16^3..64^3, 1..8 RHS):
# the smallest and largest grids, the largest RHS counts, one-RHS systems
CONFIG4_SAMPLE = [41, 6, 0, 5, 24, 13, 48, 59]


def test_config4_systems_against_oracle(bk, cuda):
    """Eight systems of the batched workload, drawn exactly as the benchmark draws them (h-scaled
    7-point convection-diffusion, grids 16^3 to 64^3, 1 to 8 right-hand sides, rel. tol 1e-8),
    solved as one batch: graph mode bitwise equal to the per-system loop, and every system of the
    graph and the persistent mode against the oracle.  The h-scaled operator is nearly symmetric, where rounding differences grow, so the
    bars are the oracle's own one-rounding-unit response per column (tests/oracle_bars.py)."""
    from oracle_bars import colerr, derived_bars, solve_columns
    torch = cuda
    grids, ks = I.batch_draws()
    sel = [(grids[i], ks[i], i) for i in CONFIG4_SAMPLE]
    assert min(g for g, _, _ in sel) == 16 and max(g for g, _, _ in sel) == 64
    csrs = [I.convdiff7(g) for g, _, _ in sel]
    kk = [k for _, k, _ in sel]
    Bs = [I.rhs(c.n, k, 200 + i) for c, (_, k, i) in zip(csrs, sel)]
    Bd = [torch.from_numpy(b).cuda() for b in Bs]
    with bk.Batch(csrs, kk) as bt:
        Xg, itg, stg, trg = bt.solve(Bd, tol=1e-8, maxit=5000, mode=bk.BATCH_GRAPH)
        Xl, itl, stl, _ = bt.solve(Bd, tol=1e-8, maxit=5000, mode=bk.BATCH_LOOP)
        Xp, itp, stp, trp = bt.solve(Bd, tol=1e-8, maxit=5000, mode=bk.BATCH_PERSISTENT)
    assert np.array_equal(itg, itl) and np.array_equal(stg, stl)
    for a, b in zip(Xg, Xl):
        assert torch.equal(a, b)
    off = 0
    for A, k, B, X, Y, (g, _, i) in zip(csrs, kk, Bs, Xg, Xp, sel):
        ro = solve_columns(A, B, tol=1e-8, maxit=5000)
        sol_bar, it_bar = derived_bars(A, B, ro, tol=1e-8, maxit=5000, label=f"batch system {i} ({g}^3, k={k})")
        for name, its, sts, trs, Z in (("graph", itg, stg, trg, X), ("persistent", itp, stp, trp, Y)):
            it = its[off:off + k]
            err = colerr(Z.cpu().numpy(), ro.X)
            print(f"[batch system {i} {name}] GPU-oracle {np.array2string(err, precision=2)}, iterations GPU "
                  f"{it.tolist()} oracle {ro.iters.tolist()}")
            assert np.all(sts[off:off + k] == 0) and np.all(trs[off:off + k] < 2e-8), name
            assert np.all(np.abs(it - ro.iters) <= it_bar), (name, i, it, ro.iters, it_bar)
            assert np.all(err <= sol_bar), (name, i, err, sol_bar)
        off += k


# ------------------------------------------------------------------ persistent mode

def _oracle_check_stable(csrs, ks, Bs, Xs, its, sts, trs, tol=1e-8, maxit=1000, X0s=None):
    """Every system against the oracle on stable operators: 1e-10 relative and +-1 iteration, or
    ten times a column's own one-rounding-unit response where that is larger (one column of the
    27-point 12^3 system moves by 1.2e-10 in the oracle itself; tests/oracle_bars.py)."""
    from oracle_bars import column_bars
    off = 0
    for i, (A, k, B, X) in enumerate(zip(csrs, ks, Bs, Xs)):
        X0 = None if X0s is None else X0s[i]
        ro = oracle.solve(A, B, X0=X0, tol=tol, maxit=maxit)
        sol_bar, it_bar = column_bars(A, B, ro, X0=X0, tol=tol, maxit=maxit, label=f"system {i} {A.name}")
        it = its[off:off + k]
        assert np.array_equal(sts[off:off + k], ro.status), (i, sts[off:off + k], ro.status)
        assert np.all(np.abs(it - ro.iters) <= it_bar), (i, it, ro.iters)
        Xn = X.cpu().numpy()
        den = np.linalg.norm(ro.X, axis=0)
        err = np.linalg.norm(Xn - ro.X, axis=0) / np.where(den == 0, 1.0, den)
        assert np.all(err[it == ro.iters] <= sol_bar[it == ro.iters]), (i, err, sol_bar)
        off += k


def test_persistent_matches_oracle_and_is_one_launch(bk, cuda):
    """The persistent mode (one cooperative launch for every system) against the oracle on stable
    operators (1e-10, +-1), against the graph mode at trajectory level (8 fixed iterations, 1e-12:
    the two sum the dot products in different orders), bitwise run to run, one kernel launch."""
    torch = cuda
    csrs, ks, Bs = _systems(10, 5)
    Bd = [torch.from_numpy(b).cuda() for b in Bs]
    with bk.Batch(csrs, ks) as bt:
        Xp, itp, stp, trp = bt.solve(Bd, tol=1e-8, maxit=1000, mode=bk.BATCH_PERSISTENT)
        assert bt.last_launches() == 1
        info = bt.persistent_info()
        print(f"[persistent] grid {info['grid_blocks']} blocks, replayed from a CUDA graph: {info['from_graph']}")
        assert info["grid_blocks"] >= 152
        assert bt.last_loop_iters() == int(itp.max())
        Xp2, itp2, _, trp2 = bt.solve(Bd, tol=1e-8, maxit=1000, mode=bk.BATCH_PERSISTENT)
        X8g, _, _, _ = bt.solve(Bd, tol=0.0, maxit=8, flags=1, mode=bk.BATCH_GRAPH)
        X8p, it8, st8, _ = bt.solve(Bd, tol=0.0, maxit=8, flags=1, mode=bk.BATCH_PERSISTENT)
    assert np.array_equal(itp, itp2) and np.array_equal(trp, trp2)
    for a, b in zip(Xp, Xp2):
        assert torch.equal(a, b)
    assert np.all(it8 == 8) and np.all(st8 == 1)
    for a, b in zip(X8p, X8g):
        a, b = a.cpu().numpy(), b.cpu().numpy()
        assert np.all(np.linalg.norm(a - b, axis=0) <= 1e-12 * np.linalg.norm(b, axis=0))
    assert np.all(stp == 0) and np.all(trp < 2e-8)
    _oracle_check_stable(csrs, ks, Bs, Xp, itp, stp, trp)


@pytest.mark.parametrize("ks", [[1, 2, 3], [4, 5, 8], [9, 16], [17, 33, 64]])
def test_persistent_every_column_width(bk, cuda, ks):
    """Every padded width of the persistent kernel (kp = 1, 2, 4, 8, 16, 32, 64: one scalar column,
    one lane per row, 2..32 lanes per row), odd row counts, zero columns and an initial guess:
    x_m after m = 1, 3 fixed iterations within 1e-12 of the oracle, then the full solve at 1e-10
    and +-1."""
    torch = cuda
    csrs = [I.convdiff7(n, peclet=True) if j % 2 == 0 else I.perturbed27(n, seed=j)
            for j, n in enumerate([9, 11, 7][: len(ks)])]
    Bs = [I.rhs(c.n, k, 30 + j) for j, (c, k) in enumerate(zip(csrs, ks))]
    Bs[0][:, 0] = 0.0                                   # b = 0 column: x = 0, 0 iterations
    X0s = [0.01 * I.rhs(c.n, k, 50 + j) for j, (c, k) in enumerate(zip(csrs, ks))]
    Bd = [torch.from_numpy(b).cuda() for b in Bs]
    X0d = [torch.from_numpy(x).cuda() for x in X0s]
    with bk.Batch(csrs, ks) as bt:
        for m in (1, 3):
            Xm, itm, _, _ = bt.solve(Bd, X0s=X0d, tol=0.0, maxit=m, flags=1, mode=bk.BATCH_PERSISTENT)
            for A, B, X0, X in zip(csrs, Bs, X0s, Xm):
                ro = oracle.solve(A, B, X0=X0, tol=0.0, maxit=m, flags=oracle.NO_STOP_TEST)
                Xn = X.cpu().numpy()
                den = np.linalg.norm(ro.X, axis=0)
                assert np.all(np.linalg.norm(Xn - ro.X, axis=0) <= 1e-12 * np.where(den == 0, 1.0, den))
        Xs, its, sts, trs = bt.solve(Bd, X0s=X0d, tol=1e-10, maxit=1000, mode=bk.BATCH_PERSISTENT)
    assert np.all(Xs[0][:, 0].cpu().numpy() == 0.0) and its[0] == 0
    _oracle_check_stable(csrs, ks, Bs, Xs, its, sts, trs, tol=1e-10, X0s=X0s)


def test_persistent_maxit_and_zero_iterations(bk, cuda):
    """maxit = 0 and maxit = 3: statuses and iteration counts as the oracle's, X as the oracle's."""
    torch = cuda
    csrs, ks, Bs = _systems(4, 7)
    Bd = [torch.from_numpy(b).cuda() for b in Bs]
    with bk.Batch(csrs, ks) as bt:
        for maxit in (0, 3):
            Xs, its, sts, _ = bt.solve(Bd, tol=1e-10, maxit=maxit, mode=bk.BATCH_PERSISTENT)
            off = 0
            for A, k, B, X in zip(csrs, ks, Bs, Xs):
                ro = oracle.solve(A, B, tol=1e-10, maxit=maxit)
                assert np.array_equal(its[off:off + k], ro.iters) and np.array_equal(sts[off:off + k], ro.status)
                Xn = X.cpu().numpy()
                assert np.all(np.linalg.norm(Xn - ro.X, axis=0) <= 1e-12 * np.maximum(np.linalg.norm(ro.X, axis=0), 1e-300))
                off += k


def test_persistent_barrier_deadline(bk, cuda):
    """A grid-barrier wait that passes its deadline ends the kernel with an error status instead of
    waiting on: with a zero deadline the first barrier gives up, the call reports BICGK_E_TIMEOUT
    naming the barrier and block, and the next solve on the same batch (deadline restored) is
    correct -- the GPU context stays usable."""
    torch = cuda
    csrs, ks, Bs = _systems(5, 3)
    Bd = [torch.from_numpy(b).cuda() for b in Bs]
    with bk.Batch(csrs, ks) as bt:
        Xr, itr, str_, _ = bt.solve(Bd, tol=1e-8, maxit=1000, mode=bk.BATCH_PERSISTENT)
        Xr = [x.clone() for x in Xr]
        bt.set_deadline(0)
        with pytest.raises(bk.BicgkError) as ei:
            bt.solve(Bd, tol=1e-8, maxit=1000, mode=bk.BATCH_PERSISTENT)
        assert ei.value.rc == bk.E_TIMEOUT and "grid barrier" in str(ei.value)
        bt.set_deadline(1_000_000)
        Xs, its, sts, _ = bt.solve(Bd, tol=1e-8, maxit=1000, mode=bk.BATCH_PERSISTENT)
        torch.cuda.synchronize()
    assert np.array_equal(its, itr) and np.array_equal(sts, str_)
    for a, b in zip(Xs, Xr):
        assert torch.equal(a, b)


def test_persistent_tuner(bk, cuda):
    """The tuner picks rows per CTA tile for the persistent mode; results agree with the default
    tiles at trajectory level (the tile size changes the dot products' summation order)."""
    torch = cuda
    csrs, ks, Bs = _systems(6, 9, lo=8, hi=20)
    Bd = [torch.from_numpy(b).cuda() for b in Bs]
    with bk.Batch(csrs, ks) as bt:
        X0, _, _, _ = bt.solve(Bd, tol=0.0, maxit=8, flags=1, mode=bk.BATCH_PERSISTENT)
        X0 = [x.clone() for x in X0]
        rows = bt.tune_persistent(reps=2)
        assert len(rows) == len(ks) and np.all(rows >= 64)
        X1, _, _, _ = bt.solve(Bd, tol=0.0, maxit=8, flags=1, mode=bk.BATCH_PERSISTENT)
    for a, b in zip(X0, X1):
        a, b = a.cpu().numpy(), b.cpu().numpy()
        assert np.all(np.linalg.norm(a - b, axis=0) <= 1e-12 * np.linalg.norm(a, axis=0))


@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_solve_in_the_persistent_kernel(bk, cuda, k):
    """bicgk_solve with BICGK_OPT_PERSISTENT = 2 runs the whole solve as one cooperative launch of
    the persistent kernel: x_m and the residual history after 6 fixed iterations within 1e-12 and
    1e-10 of the oracle's (and of the graph path's), the solve to tolerance within the oracle's
    bars (stable operator), one kernel launch per solve."""
    from oracle_bars import colerr, column_bars
    torch = cuda
    A = I.convdiff7(14, peclet=True)
    B = I.rhs(A.n, k, 40)
    Bd = torch.from_numpy(B).cuda()
    with bk.Operator(A) as op:
        bk.set_option(op.handle, bk.OPT_PERSISTENT, 1)
        rg = op.solve(Bd, tol=0.0, maxit=6, flags=bk.FLAG_NO_STOP_TEST)
        Xg = rg.X.cpu().numpy()
        bk.set_option(op.handle, bk.OPT_PERSISTENT, 2)
        rp6 = op.solve(Bd, tol=0.0, maxit=6, flags=bk.FLAG_NO_STOP_TEST)
        assert bk.last_stats(op.handle)["kernel_launches"] == 1
        rp = op.solve(Bd, tol=1e-9, maxit=1000)
        X = rp.X.cpu().numpy()
    ro6 = oracle.solve(A, B, tol=0.0, maxit=6, flags=oracle.NO_STOP_TEST)
    X6 = rp6.X.cpu().numpy()
    assert np.all(colerr(X6, ro6.X) <= 1e-12) and np.all(colerr(X6, Xg) <= 1e-12)
    np.testing.assert_allclose(rp6.hist, ro6.hist, rtol=1e-10)
    ro = oracle.solve(A, B, tol=1e-9, maxit=1000)
    sol_bar, it_bar = column_bars(A, B, ro, tol=1e-9, maxit=1000)
    assert np.array_equal(rp.status, ro.status) and np.all(np.abs(rp.iters - ro.iters) <= it_bar)
    assert np.all(colerr(X, ro.X) <= sol_bar), colerr(X, ro.X)
    # histories at each column's own place; near convergence the merged estimate theta - omega phi
    # is a difference of much larger numbers, so two summation orders agree only to about 1e-2 there
    for c in range(k):
        m = int(min(rp.iters[c], ro.iters[c]))
        np.testing.assert_allclose(rp.hist[: m + 1, c], ro.hist[: m + 1, c], rtol=1e-2)
