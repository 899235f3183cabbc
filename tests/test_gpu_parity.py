"""CUDA path vs the FP64 oracle, through the C-ABI (libbicgk.so).

Three kinds of comparison:
  * trajectory: the iterate x_m after m = 1, 2, 4, 8 iterations (fixed count),
    per column, relative 2-norm difference <= 1e-12.  Both sides perform the
    same operations and differ only in rounding (dot-product summation order,
    fused multiply-adds), which stays at 1e-16..1e-14 over these iterations on
    every operator;
  * full solve, stable operators (strongly nonsymmetric upwind and 27-point
    stencils, where rounding differences do not grow): solution within 1e-10
    relative, iteration count within +-1, same status;
  * full solve, nearly symmetric operators (the h-scaled convection-diffusion
    of the 16^3 configuration, Poisson): there BiCGStab amplifies rounding
    differences by about 10^3 every 8 iterations, so the stopping iterate is
    not unique: one rounding unit in b moves the oracle's own solution by up
    to ~1e-7 and its iteration counts by up to 9.  The bars are measured on
    the oracle per case (tests/oracle_bars.py): solution within ten times the
    oracle's largest one-unit response (at least 1e-10), iterations within
    twice its largest one-unit change (at least +-1), same status; besides,
    both true residuals below the tolerance and the GPU iterate as close to
    the exact solution x* = A^-1 b (sparse LU) as its residual allows.
Inputs are the seeded synthetic stencils of the paper's workloads (Sec. 2.3:
7-point Poisson; the upwind convection-diffusion and 27-point operators of the
benchmark configurations).
"""
import numpy as np
import pytest

import oracle
from paper_1907_12874_gb300 import inputs as I
from oracle_bars import derived_bars

pytestmark = pytest.mark.gpu

SOL_RTOL = 1e-10
VARIANTS = list(oracle.VARIANTS)


@pytest.fixture(scope="module")
def bk(cuda):
    from paper_1907_12874_gb300 import bicgk
    return bicgk


def _colerr(X, Xo):
    num = np.linalg.norm(X - Xo, axis=0)
    den = np.linalg.norm(Xo, axis=0)
    return num / np.where(den == 0, 1.0, den)


def _gpu_solve(bk, torch, A, B, **kw):
    with bk.Operator(A) as op:
        Bd = torch.from_numpy(B).cuda()
        X0 = kw.pop("X0", None)
        X0d = None if X0 is None else torch.from_numpy(np.ascontiguousarray(X0)).cuda()
        r = op.solve(Bd, X0=X0d, **kw)
        torch.cuda.synchronize()
        return r, r.X.cpu().numpy()


def _compare(r, X, ro, tol_sol=SOL_RTOL, iters_slack=1):
    assert np.all(np.abs(r.iters - ro.iters) <= iters_slack), (r.iters, ro.iters)
    assert np.array_equal(r.status, ro.status), (r.status, ro.status)
    same = r.iters == ro.iters
    err = _colerr(X, ro.X)
    bar = np.broadcast_to(np.asarray(tol_sol, dtype=float), err.shape)
    assert np.all(err[same] <= bar[same]), (err, bar)
    # where the counts differ by one, both iterates still solve the system to the tolerance
    assert np.all(err <= 1e-6), err
    return err


# ------------------------------------------------------------------ SpMM

def _random_csr(n, seed, max_len=40):
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, max_len, size=n)
    lens[:3] = 0                      # empty rows
    lens[n // 2] = min(n, 3000)       # one long row: the staged tile overflows
    rowptr = np.zeros(n + 1, dtype=np.int32)
    np.cumsum(lens, out=rowptr[1:])
    cols = np.concatenate([rng.choice(n, size=l, replace=False) for l in lens]).astype(np.int32)
    vals = rng.standard_normal(rowptr[-1])
    return I.CSR(rowptr, cols, vals, "random")


@pytest.mark.parametrize("k", [1, 2, 3, 4, 8, 16, 32, 64])
@pytest.mark.parametrize("kind", ["convdiff7", "random"])
def test_spmm_matches_oracle(bk, cuda, k, kind):
    torch = cuda
    A = I.convdiff7(13) if kind == "convdiff7" else _random_csr(3001, 7)
    X = I.rhs(A.n, k, 11)
    Yo = oracle.spmm(A, X)
    with bk.Operator(A) as op:
        Xd = torch.from_numpy(X).cuda()
        Y = op.spmm(Xd).cpu().numpy()
    # same products, same order, FMA on the GPU: bound by |A||X| * few ulps
    absA = I.CSR(A.rowptr, A.colidx, np.abs(A.vals))
    bound = oracle.spmm(absA, np.abs(X)) * (4 * 2.0 ** -52) * np.maximum(1, np.diff(A.rowptr))[:, None]
    assert np.all(np.abs(Y - Yo) <= bound + 1e-300)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 8, 16, 32, 64])
@pytest.mark.parametrize("kind", ["convdiff7", "random", "perturbed27"])
def test_spmm_f32_matches_oracle(bk, cuda, k, kind):
    """FP32 product of the mixed-precision inner solves: y = fl32(A) x summed in FP32 with FMAs in
    CSR order.  Reference: the FP64 oracle on the FP32-rounded values and inputs (exact to far
    below FP32 rounding); bound: recursive FP32 summation, len * 2^-24 * (|A||x|) per entry.  The
    random matrix has empty rows and a 3000-entry row (many chunks, a ragged last chunk)."""
    torch = cuda
    A = {"convdiff7": lambda: I.convdiff7(13), "random": lambda: _random_csr(3001, 7),
         "perturbed27": lambda: I.perturbed27(9, seed=2)}[kind]()
    A32 = I.CSR(A.rowptr, A.colidx, A.vals.astype(np.float32).astype(np.float64))
    X32 = I.rhs(A.n, k, 11).astype(np.float32)
    Yo = oracle.spmm(A32, X32.astype(np.float64))
    with bk.Operator(A) as op:
        Y = op.spmm_f32(torch.from_numpy(X32).cuda()).cpu().numpy().astype(np.float64)
    absA = I.CSR(A.rowptr, A.colidx, np.abs(A32.vals))
    lens = np.maximum(1, np.diff(A.rowptr))[:, None]
    bound = oracle.spmm(absA, np.abs(X32).astype(np.float64)) * (1.01 * 2.0 ** -24) * lens
    assert np.all(np.abs(Y - Yo) <= bound + 1e-300)


@pytest.mark.parametrize("k", [9, 16, 24, 32, 64])
@pytest.mark.parametrize("kind", ["perturbed27_40", "random", "tiny", "perturbed27_9"])
def test_spmm_f32_sweep_is_bitwise_segment(bk, cuda, k, kind):
    """The two FP32 kernels (BICGK_OPT_SPMM32: the sweep kernel, default, and the segment kernel)
    both sum every row in CSR order with FP32 FMAs, so their products are bitwise equal.  The
    random matrix has empty rows and a 3000-entry row (a warp tile over the staging capacity reads
    its entries from global memory); "tiny" has fewer rows than the sweep grid has blocks (empty
    ranges), 9^3 rows leave partial tiles at the ends of the blocks' ranges; k = 9 and 24 are
    padded to kp = 16 and 32."""
    torch = cuda
    A = {"perturbed27_40": lambda: I.perturbed27(40, seed=4), "random": lambda: _random_csr(3001, 7),
         "tiny": lambda: I.convdiff7(3), "perturbed27_9": lambda: I.perturbed27(9, seed=2)}[kind]()
    X32 = torch.from_numpy(I.rhs(A.n, k, 5).astype(np.float32)).cuda()
    with bk.Operator(A) as op:
        Ys = op.spmm_f32(X32)
        bk.set_option(op.handle, bk.OPT_SPMM32, 1)
        Yg = op.spmm_f32(X32)
        bk.set_option(op.handle, bk.OPT_SPMM32, 0)
        Ys2 = op.spmm_f32(X32)
    assert torch.equal(Ys, Yg)
    assert torch.equal(Ys, Ys2)
    assert bool(torch.isfinite(Ys).all())


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("kind", ["convdiff7_13", "random", "tiny", "perturbed27_9", "convdiff7_40", "one_row",
                                  "empty_rows"])
def test_row_products_warp_tile_is_bitwise_block_tile(bk, cuda, k, kind):
    """The two one-lane-per-row products for kp <= 2 (BICGK_OPT_SPMM_ROWS: the warp-tile kernel,
    default for short rows, and the block-tile kernel) both sum every row in CSR order, so FP64
    and FP32 products and whole solves (which also run y = b - A x) are bitwise equal.  The random
    matrix has empty rows and a 3000-entry row, and 27-point rows overflow the warp tile's staging
    (both read those entries from global memory); "tiny" has fewer rows than the grid has warps,
    "one_row" a single row, "empty_rows" no entries at all."""
    torch = cuda
    A = {"convdiff7_13": lambda: I.convdiff7(13), "random": lambda: _random_csr(3001, 7),
         "tiny": lambda: I.convdiff7(3), "perturbed27_9": lambda: I.perturbed27(9, seed=2),
         "convdiff7_40": lambda: I.convdiff7(40),
         "one_row": lambda: I.CSR(np.array([0, 1], np.int32), np.array([0], np.int32), np.array([3.0]), "one_row"),
         "empty_rows": lambda: I.CSR(np.zeros(101, np.int32), np.zeros(0, np.int32), np.zeros(0), "empty")}[kind]()
    if kind == "empty_rows":   # no entries: both products are zero; no solve (A is singular)
        X = torch.from_numpy(I.rhs(A.n, k, 5)).cuda()
        with bk.Operator(A) as op:
            for rows in (2, 1):
                bk.set_option(op.handle, bk.OPT_SPMM_ROWS, rows)
                assert not bool(op.spmm(X).any()) and not bool(op.spmm_f32(X.float()).any())
        return
    X = torch.from_numpy(I.rhs(A.n, k, 5)).cuda()
    B = torch.from_numpy(I.rhs(A.n, k, 6)).cuda()
    out = {}
    with bk.Operator(A) as op:
        bk.set_option(op.handle, bk.OPT_PERSISTENT, 1)   # the graph path's products
        for rows in (2, 1):
            bk.set_option(op.handle, bk.OPT_SPMM_ROWS, rows)
            Y = op.spmm(X)
            Y32 = op.spmm_f32(X.float())
            r = op.solve(B, tol=1e-8, maxit=60, want_hist=False)
            out[rows] = (Y, Y32, torch.as_tensor(r.X), r.iters.copy())
    for a, b in zip(out[2][:3], out[1][:3]):
        assert torch.equal(a, b)
    assert np.array_equal(out[2][3], out[1][3])


@pytest.mark.parametrize("k", [2, 4, 8, 32])
def test_spmm_unaligned_caller_arrays(bk, cuda, k):
    """Caller blocks that start 8 bytes (FP64) or 4 bytes (FP32) past a 16-byte boundary go
    through the operator's workspace; the result is bitwise the aligned call's."""
    torch = cuda
    A = I.convdiff7(11)
    X = I.rhs(A.n, k, 3)
    with bk.Operator(A) as op:
        Xa = torch.from_numpy(X).cuda()
        Ya = op.spmm(Xa)
        buf_x = torch.zeros(A.n * k + 1, dtype=torch.float64, device="cuda")
        buf_y = torch.zeros(A.n * k + 1, dtype=torch.float64, device="cuda")
        Xu = buf_x[1:].view(A.n, k)
        Xu.copy_(Xa)
        Yu = buf_y[1:].view(A.n, k)
        assert Xu.data_ptr() % 16 == 8 and Yu.data_ptr() % 16 == 8
        op.spmm(Xu, Yu)
        assert torch.equal(Ya, Yu)
        X32 = Xa.float()
        Ya32 = op.spmm_f32(X32)
        b32x = torch.zeros(A.n * k + 1, dtype=torch.float32, device="cuda")
        b32y = torch.zeros(A.n * k + 1, dtype=torch.float32, device="cuda")
        Xu32 = b32x[1:].view(A.n, k)
        Xu32.copy_(X32)
        Yu32 = b32y[1:].view(A.n, k)
        assert Xu32.data_ptr() % 16 == 4
        op.spmm_f32(Xu32, Yu32)
        assert torch.equal(Ya32, Yu32)


def _compare_chaotic(r, X, ro, A, B, tol, variant="classical_merged", maxit=1000):
    """Nearly symmetric operators: bars from the oracle's own rounding response (module doc), and
    the bound that ties the iterate to the unique exact solution x*."""
    import scipy.sparse.linalg as sla
    sol_bar, it_bar = derived_bars(A, B, ro, tol=tol, maxit=maxit, variant=variant, label=f"{A.name} {variant}")
    assert np.array_equal(r.status, ro.status), (r.status, ro.status)
    assert np.all(np.abs(r.iters - ro.iters) <= it_bar), (r.iters, ro.iters, it_bar)
    err = _colerr(X, ro.X)
    assert np.all(err <= sol_bar), (err, sol_bar)
    assert np.all(r.status == 0) and np.all(r.true_relres < 2 * tol) and np.all(ro.true_relres < 2 * tol)
    lu = sla.splu(A.to_scipy().tocsc())
    Xs = lu.solve(B)
    eg = np.linalg.norm(X - Xs, axis=0)
    # ||x - x*|| <= ||A^-1|| ||b - A x||: ||A^-1|| by power iteration with the LU factors (1.5 covers
    # the estimate's shortfall)
    v = I.rhs(A.n, 1, 99)[:, 0]
    for _ in range(30):
        w = lu.solve(v)
        w = lu.solve(w, trans="T")
        v = w / np.linalg.norm(w)
    inv_norm = np.sqrt(np.linalg.norm(lu.solve(lu.solve(v), trans="T")))
    bound = inv_norm * r.true_relres * np.linalg.norm(B, axis=0)
    assert np.all(eg <= 1.5 * bound + 1e-14), (eg, bound)
    return err


def _trajectory(bk, torch, A, B, variant, ms=(1, 2, 4, 8), tol_traj=1e-12):
    with bk.Operator(A) as op:
        Bd = torch.from_numpy(B).cuda()
        for m in ms:
            r = op.solve(Bd, tol=0.0, maxit=m, variant=variant, flags=1)
            ro = oracle.solve(A, B, tol=0.0, maxit=m, variant=variant, flags=oracle.NO_STOP_TEST)
            X = r.X.cpu().numpy()
            err = _colerr(X, ro.X)
            assert np.all(err <= tol_traj), (m, err)
            np.testing.assert_allclose(r.hist[: m + 1], ro.hist[: m + 1], rtol=1e-10)


# ------------------------------------------------------------------ full solves

@pytest.mark.parametrize("variant", VARIANTS)
def test_config1_16cubed_k4(bk, cuda, variant):
    """16^3 upwind convection-diffusion, 4 RHS U[-1,1] (seed 1), x0 = 0, rel tol 1e-8."""
    A = I.convdiff7(16)
    B = I.rhs(A.n, 4, 1)
    _trajectory(bk, cuda, A, B, variant)
    ro = oracle.solve(A, B, tol=1e-8, maxit=1000, variant=variant)
    r, X = _gpu_solve(bk, cuda, A, B, tol=1e-8, maxit=1000, variant=variant)
    _compare_chaotic(r, X, ro, A, B, 1e-8, variant=variant)


def _oracle_rounding_sensitivity(A, B, variant, ro, reps=3, seed=11):
    """Per column, the largest relative change of the oracle's own solution when every entry of b
    moves by about one rounding unit (2^-52 relative), over `reps` draws.  This is how far the
    form's recurrences carry a single rounding difference to the stopping iterate."""
    rng = np.random.default_rng(seed)
    worst = np.zeros(B.shape[1])
    for _ in range(reps):
        Bp = B * (1.0 + 2.0 ** -52 * rng.standard_normal(B.shape))
        rp = oracle.solve(A, Bp, tol=1e-8, maxit=1000, variant=variant)
        e = _colerr(rp.X, ro.X)
        worst = np.maximum(worst, np.where(rp.iters == ro.iters, e, 0.0))
    return worst


@pytest.mark.parametrize("variant", VARIANTS)
def test_stable_operator_16cubed(bk, cuda, variant):
    """Strongly nonsymmetric upwind operator (mesh Peclet beta): 1e-10 and +-1 for every form but
    Algorithm 3.  Algorithm 3 forms rho and the alpha denominator tau by scalar recurrences from
    older dots instead of as dots of the current vectors, and on this operator one rounding unit
    in b already moves its stopping iterate by
    about 4e-11 on one column (about 30 times the classical form).  The GPU injects rounding
    differences at every iteration (summation order of the dots), so for Algorithm 3 the bar per
    column is max(1e-10, 10 x the oracle's own one-unit sensitivity), measured here."""
    A = I.convdiff7(16, peclet=True)
    B = I.rhs(A.n, 4, 1)
    _trajectory(bk, cuda, A, B, variant)
    ro = oracle.solve(A, B, tol=1e-8, maxit=1000, variant=variant)
    r, X = _gpu_solve(bk, cuda, A, B, tol=1e-8, maxit=1000, variant=variant)
    tol_sol = SOL_RTOL
    if variant.startswith("improved"):
        tol_sol = np.maximum(SOL_RTOL, 10.0 * _oracle_rounding_sensitivity(A, B, variant, ro))
    _compare(r, X, ro, tol_sol=tol_sol)
    assert np.all(r.status == 0) and np.all(r.true_relres < 2e-8)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("k", [1, 3, 8])
def test_ragged_k_24cubed(bk, cuda, variant, k):
    """Several tiles, padded RHS counts (k = 3 -> 4 columns), odd row count (24^3 is even; 23^3 odd)."""
    A = I.convdiff7(23, peclet=True)
    B = I.rhs(A.n, k, 5)
    ro = oracle.solve(A, B, tol=1e-8, maxit=2000, variant=variant)
    r, X = _gpu_solve(bk, cuda, A, B, tol=1e-8, maxit=2000, variant=variant)
    _compare(r, X, ro)


def test_k64_and_poisson(bk, cuda):
    A = I.convdiff7(12, beta=(0, 0, 0))
    B = I.rhs(A.n, 64, 9)
    _trajectory(bk, cuda, A, B, "classical_merged", ms=(1, 4, 8))
    ro = oracle.solve(A, B, tol=1e-9, maxit=1000, variant="classical_merged")
    r, X = _gpu_solve(bk, cuda, A, B, tol=1e-9, maxit=1000, variant="classical_merged")
    _compare_chaotic(r, X, ro, A, B, 1e-9, variant="classical_merged")


@pytest.mark.parametrize("variant", VARIANTS)
def test_perturbed27(bk, cuda, variant):
    A = I.perturbed27(10, seed=3)
    B = I.rhs(A.n, 2, 4)
    ro = oracle.solve(A, B, tol=1e-10, maxit=500, variant=variant)
    r, X = _gpu_solve(bk, cuda, A, B, tol=1e-10, maxit=500, variant=variant)
    _compare(r, X, ro)


# ------------------------------------------------------------------ edge cases

@pytest.mark.parametrize("variant", VARIANTS)
def test_edge_columns(bk, cuda, variant):
    """b_c = 0 -> x_c = 0 with 0 iterations; x0 = exact -> 0 iterations; maxit status."""
    A = I.convdiff7(8)
    B = I.rhs(A.n, 4, 3)
    B[:, 1] = 0.0
    Xs = I.rhs(A.n, 4, 8)
    X0 = np.zeros_like(B)
    X0[:, 1] = 1.0                      # b = 0 but x0 != 0: result must be 0
    B[:, 2] = oracle.spmm(A, Xs[:, 2:3])[:, 0]
    X0[:, 2] = Xs[:, 2]                 # exact initial guess
    ro = oracle.solve(A, B, X0=X0, tol=1e-8, maxit=1000, variant=variant)
    r, X = _gpu_solve(bk, cuda, A, B, X0=X0, tol=1e-8, maxit=1000, variant=variant)
    _compare(r, X, ro)
    assert r.iters[1] == 0 and r.status[1] == 0 and np.all(X[:, 1] == 0.0)
    assert r.iters[2] == 0 and np.array_equal(X[:, 2], X0[:, 2])
    # maxit = 3: every column that needs more reports MAXIT after exactly 3 iterates
    ro = oracle.solve(A, B, X0=X0, tol=1e-8, maxit=3, variant=variant)
    r, X = _gpu_solve(bk, cuda, A, B, X0=X0, tol=1e-8, maxit=3, variant=variant)
    assert np.array_equal(r.status, ro.status) and np.array_equal(r.iters, ro.iters)
    assert np.all(_colerr(X, ro.X) <= 1e-12)
    # maxit = 0
    r, X = _gpu_solve(bk, cuda, A, B, X0=X0, tol=1e-8, maxit=0, variant=variant)
    ro = oracle.solve(A, B, X0=X0, tol=1e-8, maxit=0, variant=variant)
    assert np.array_equal(r.status, ro.status) and np.array_equal(r.iters, ro.iters)
    assert np.array_equal(X, ro.X)


@pytest.mark.parametrize("variant", VARIANTS)
def test_scaled_identity_one_step(bk, cuda, variant):
    """A = 2I: alpha = 1/2 exactly, s = 0, omega = 0 by the psi = 0 rule: x = b/2 after one iterate."""
    n = 1000
    A = I.CSR(np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.full(n, 2.0))
    B = I.rhs(n, 3, 2)
    r, X = _gpu_solve(bk, cuda, A, B, tol=1e-12, maxit=10, variant=variant)
    ro = oracle.solve(A, B, tol=1e-12, maxit=10, variant=variant)
    assert np.array_equal(r.iters, ro.iters) and np.array_equal(r.status, ro.status)
    np.testing.assert_array_equal(X, B / 2)


@pytest.mark.parametrize("variant", VARIANTS)
def test_fixed_iteration_mode(bk, cuda, variant):
    """NO_STOP_TEST: exactly maxit iterations (the paper's N_it benchmark mode)."""
    A = I.convdiff7(10)
    B = I.rhs(A.n, 2, 6)
    r, X = _gpu_solve(bk, cuda, A, B, tol=0.0, maxit=12, variant=variant, flags=1)
    ro = oracle.solve(A, B, tol=0.0, maxit=12, variant=variant, flags=oracle.NO_STOP_TEST)
    assert np.all(r.iters == 12) and np.all(r.status == 1)
    assert np.all(_colerr(X, ro.X) <= 1e-11)


@pytest.mark.parametrize("persistent", [1, 0])
def test_host_memory_path_is_bitwise_device_path(bk, cuda, persistent):
    """Host blocks give bitwise the device call's results, on the graph path and (automatic at this
    size) in the persistent kernel; repeated device calls are bitwise equal."""
    torch = cuda
    A = I.convdiff7(14)
    B = I.rhs(A.n, 5, 12)
    with bk.Operator(A) as op:
        bk.set_option(op.handle, bk.OPT_PERSISTENT, persistent)
        rh = op.solve(B, tol=1e-8, maxit=500)
        rd = op.solve(torch.from_numpy(B).cuda(), tol=1e-8, maxit=500)
        rd2 = op.solve(torch.from_numpy(B).cuda(), tol=1e-8, maxit=500)
        Xd = rd.X.cpu().numpy()
    assert np.array_equal(rh.X, Xd)                     # same kernels, same order
    assert np.array_equal(Xd, rd2.X.cpu().numpy())      # deterministic reductions
    assert np.array_equal(rh.iters, rd.iters)


def test_profiling_mode_matches_graph_mode(bk, cuda):
    torch = cuda
    A = I.convdiff7(12)
    B = torch.from_numpy(I.rhs(A.n, 4, 13)).cuda()
    with bk.Operator(A) as op:
        rg = op.solve(B, tol=1e-8, maxit=500, variant="pipelined_merged")
        bk.set_profiling(op.handle, True)
        rp = op.solve(B, tol=1e-8, maxit=500, variant="pipelined_merged")
        times = bk.kernel_times(op.handle)
        bk.set_profiling(op.handle, False)
    assert torch.equal(rg.X, rp.X)
    assert "merged_pszqy_3dots" in times and times["merged_pszqy_3dots"][0] == int(rp.iters.max())


@pytest.mark.parametrize("k", [8, 20, 32])
def test_profiling_mode_keeps_the_column_groups(bk, cuda, k):
    """The profiling mode runs the graph mode's column groups one after another: the same kernels
    (names carry the group's column count), bitwise the graph mode's results without compaction."""
    torch = cuda
    A = I.convdiff7(12, peclet=True)
    B = torch.from_numpy(I.rhs(A.n, k, 13)).cuda()
    with bk.Operator(A) as op:
        bk.set_option(op.handle, bk.OPT_COMPACT, 1)
        bk.set_option(op.handle, bk.OPT_PERSISTENT, 1)   # the graph path (k = 8 would run persistent)
        rg = op.solve(B, tol=1e-8, maxit=500)
        groups = bk.last_stats(op.handle)["groups"]
        bk.set_profiling(op.handle, True)
        rp = op.solve(B, tol=1e-8, maxit=500)
        assert bk.last_stats(op.handle)["groups"] == groups
        times = bk.kernel_times(op.handle)
        bk.set_profiling(op.handle, False)
    assert groups == (4 if k >= 32 else 2)
    assert torch.equal(rg.X, rp.X) and np.array_equal(rg.iters, rp.iters)
    kg = 1 << (k // groups - 1).bit_length()
    assert any(name.endswith(f"_k{kg}") for name in times), times.keys()


def test_bad_csr_rejected(bk, cuda):
    rowptr = np.array([0, 2, 1], dtype=np.int32)
    with pytest.raises(bk.BicgkError):
        bk.csr_create(rowptr, np.array([0, 1], dtype=np.int32), np.ones(2))
    with pytest.raises(bk.BicgkError):
        bk.csr_create(np.array([0, 1, 2], dtype=np.int32), np.array([0, 5], dtype=np.int32), np.ones(2))


@pytest.mark.parametrize("groups", [0, 3, 4])
def test_rhs_groups_match_single_group(bk, cuda, groups):
    """k >= 8 runs as concurrent column groups (two by default at k = 20; three and four forced);
    it must agree with one group (and the oracle), device and host buffers alike."""
    torch = cuda
    A = I.convdiff7(12, peclet=True)
    B = I.rhs(A.n, 20, 4)                       # e.g. groups of 10 + 10 columns (kp 16) vs one group (kp 32)
    Bd = torch.from_numpy(B).cuda()
    with bk.Operator(A) as one, bk.Operator(A) as many:
        bk.set_option(one.handle, bk.OPT_RHS_GROUPS, 1)
        bk.set_option(many.handle, bk.OPT_RHS_GROUPS, groups)
        for flags, maxit, tol in ((1, 8, 0.0), (0, 500, 1e-8)):
            r1 = one.solve(Bd, tol=tol, maxit=maxit, flags=flags)
            r2 = many.solve(Bd, tol=tol, maxit=maxit, flags=flags)
            assert bk.last_stats(one.handle)["groups"] == 1
            assert bk.last_stats(many.handle)["groups"] == (groups or 2)
            assert bk.last_stats(many.handle)["kernel_launches"] > bk.last_stats(one.handle)["kernel_launches"]
            X1, X2 = r1.X.cpu().numpy(), r2.X.cpu().numpy()
            assert np.all(np.abs(r1.iters - r2.iters) <= 1) and np.array_equal(r1.status, r2.status)
            assert np.all(_colerr(X2, X1) <= (1e-12 if flags else 1e-10))
        rh = many.solve(B, tol=1e-8, maxit=500)  # host buffers, same groups: same as the device call
        assert np.array_equal(rh.X, r2.X.cpu().numpy()) and np.array_equal(rh.iters, r2.iters)
        # page-locked host buffers: read and written in place by the kernels, or staged
        Bp = torch.from_numpy(B).pin_memory()
        X0 = 0.1 * I.rhs(A.n, 20, 5)
        X0p = torch.from_numpy(X0).pin_memory()
        rd0 = many.solve(Bd, X0=torch.from_numpy(X0).cuda(), tol=1e-8, maxit=500)
        for zc in (0, 1):
            bk.set_option(many.handle, bk.OPT_HOST_ZERO_COPY, zc)
            rp = many.solve(Bp, tol=1e-8, maxit=500)
            assert np.array_equal(rp.X.numpy(), r2.X.cpu().numpy()) and np.array_equal(rp.iters, r2.iters)
            rp0 = many.solve(Bp, X0=X0p, tol=1e-8, maxit=500)
            assert np.array_equal(rp0.X.numpy(), rd0.X.cpu().numpy()) and np.array_equal(rp0.iters, rd0.iters)
    ro = oracle.solve(A, B, tol=1e-8, maxit=500)
    _compare(r2, X2, ro)


@pytest.mark.parametrize("variant", ["precond_plain", "precond_merged", "ppipe_plain", "ppipe_merged",
                                     "reordered_plain", "reordered_merged"])
def test_jacobi_preconditioner(bk, cuda, variant):
    """M = diag(A) on the 27-point operator (its diagonal varies row to row)."""
    A = I.perturbed27(12, seed=8)
    B = I.rhs(A.n, 3, 14)
    _ro = oracle.solve(A, B, tol=1e-10, maxit=500, variant=variant, flags=oracle.JACOBI)
    r, X = _gpu_solve(bk, cuda, A, B, tol=1e-10, maxit=500, variant=variant, flags=2)
    _compare(r, X, _ro)
    # trajectory at rounding level
    rf, Xf = _gpu_solve(bk, cuda, A, B, tol=0.0, maxit=6, variant=variant, flags=3)
    rof = oracle.solve(A, B, tol=0.0, maxit=6, variant=variant, flags=oracle.JACOBI | oracle.NO_STOP_TEST)
    assert np.all(_colerr(Xf, rof.X) <= 1e-12)


def test_jacobi_diagonal_matrix_one_iterate(bk, cuda):
    n = 999
    d = 1.0 + (np.arange(n) % 5)
    A = I.CSR(np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d)
    B = I.rhs(n, 4, 1)
    for v in ("precond_merged", "ppipe_merged", "reordered_merged"):
        r, X = _gpu_solve(bk, cuda, A, B, tol=1e-12, maxit=10, variant=v, flags=2)
        assert np.all(r.iters == 1) and np.all(r.status == 0)
        np.testing.assert_allclose(X, B / d[:, None], rtol=1e-15)


@pytest.mark.parametrize("variant", ["classical_merged", "precond_merged", "reordered_merged"])
@pytest.mark.parametrize("k", [1, 2, 3, 8, 20])
@pytest.mark.parametrize("kind", ["convdiff7_peclet", "perturbed27"])
def test_fused_dots_match_separate_kernels(bk, cuda, variant, k, kind):
    """The dot kernel that follows an SpMM taken into the SpMM's epilogue (BICGK_OPT_FUSED_DOTS),
    and theta = (s, s) taken in the s update (BICGK_OPT_THETA_IN_S), give the iterates of the
    separate kernels up to the summation order of those dots, and the oracle's.  Each forced on
    and off at every kp, so the fused one-lane-per-row kernels (kp <= 2) run with staged tiles
    (7-point stencil: the warp-tile kernel, and the block-tile kernel by BICGK_OPT_SPMM_ROWS = 1)
    and with tiles larger than the stage buffer (27-point stencil, 256-row tiles of 6,912
    entries)."""
    torch = cuda
    A = I.convdiff7(12, peclet=True) if kind == "convdiff7_peclet" else I.perturbed27(11, seed=5)
    B = I.rhs(A.n, k, 4)
    Bd = torch.from_numpy(B).cuda()
    ro = oracle.solve(A, B, tol=0.0, maxit=6, variant=variant, flags=oracle.NO_STOP_TEST)
    X = {}
    with bk.Operator(A) as op:
        bk.set_option(op.handle, bk.OPT_PERSISTENT, 1)   # these options belong to the graph path
        for fz, th in ((1, 1), (2, 1), (1, 2), (2, 2)):
            bk.set_option(op.handle, bk.OPT_FUSED_DOTS, fz)
            bk.set_option(op.handle, bk.OPT_THETA_IN_S, th)
            r = op.solve(Bd, tol=0.0, maxit=6, variant=variant, flags=bk.FLAG_NO_STOP_TEST)
            X[fz, th] = r.X.cpu().numpy()
            assert np.all(_colerr(X[fz, th], ro.X) <= 1e-12), (fz, th)
            np.testing.assert_allclose(r.hist[:7], ro.hist[:7], rtol=1e-10)
            assert np.all(_colerr(X[fz, th], X[1, 1]) <= 1e-13), (fz, th)
        if k <= 2 and kind == "convdiff7_peclet":   # the fused block-tile kernel on short rows too
            bk.set_option(op.handle, bk.OPT_SPMM_ROWS, 1)
            bk.set_option(op.handle, bk.OPT_FUSED_DOTS, 2)
            r = op.solve(Bd, tol=0.0, maxit=6, variant=variant, flags=bk.FLAG_NO_STOP_TEST)
            assert np.all(_colerr(r.X.cpu().numpy(), ro.X) <= 1e-12)
            assert np.all(_colerr(r.X.cpu().numpy(), X[1, 1]) <= 1e-13)
            bk.set_option(op.handle, bk.OPT_SPMM_ROWS, 0)
        r = op.solve(Bd, tol=1e-8, maxit=1000, variant=variant)  # both forced on
        Xf = r.X.cpu().numpy()
    rof = oracle.solve(A, B, tol=1e-8, maxit=1000, variant=variant)
    _compare(r, Xf, rof)


def _compaction_bars(A, B, X0, tol, maxit, variant, flags, ro):
    """Bars for comparing two layouts of the same solve: the form's own sensitivity to one
    rounding unit in b (three draws; Algorithm 3 on the Peclet operator carries it far, the
    others hardly at all) -- ten times the largest change of the solution (at least 1e-9) and
    twice the largest change of an iteration count (at least 1)."""
    sens, spread = 0.0, 0
    g = np.random.default_rng(31)
    for _ in range(3):
        rp = oracle.solve(A, B * (1.0 + 2.0 ** -52 * g.standard_normal(B.shape)), X0=X0, tol=tol,
                          maxit=maxit, variant=variant, flags=oracle.JACOBI if flags else 0)
        sens = max(sens, float(_colerr(rp.X, ro.X).max()))
        spread = max(spread, int(np.abs(rp.iters - ro.iters).max()))
    return max(1e-9, 10.0 * sens), max(1, 2 * spread)


COMPACT_VARIANTS = ["classical_merged", "classical_plain", "precond_merged", "precond_plain",
                    "reordered_merged", "reordered_plain", "pipelined_merged", "pipelined_plain",
                    "ppipe_merged", "ppipe_plain", "improved_merged", "improved_plain"]


@pytest.mark.parametrize("variant", COMPACT_VARIANTS)
@pytest.mark.parametrize("k", [2, 5, 8, 20])
def test_column_compaction_matches_full_layout(bk, cuda, variant, k):
    """A column group narrows its layout whenever at most half of its columns still iterate
    (BICGK_OPT_COMPACT).  Columns of very different difficulty make the groups pass through
    several layouts: initial guesses whose error is the exact solution's times 10^-d, d from 0
    to 8, so the columns meet the relative tolerance after very different iteration counts,
    plus zero columns that stop at the set-up.  The solve must agree with the full layout and
    with the oracle: same status, iterations within one, solutions within the solution
    tolerance, residual histories at the solve's own columns."""
    import scipy.sparse.linalg as sla
    torch = cuda
    A = I.convdiff7(12, peclet=True)
    B = I.rhs(A.n, k, 21)
    rng = np.random.default_rng(k)
    B[:, rng.permutation(k)[: k // 3]] = 0.0          # zero columns: stopped before the loop
    Xs = sla.splu(A.to_scipy().tocsc()).solve(B)
    G0 = Xs + 10.0 ** -rng.integers(0, 9, size=k) * rng.standard_normal(B.shape) * np.abs(Xs).max(axis=0)
    G0[:, np.all(B == 0, axis=0)] = 0.0
    flags = 2 if variant.startswith(("precond", "reordered", "ppipe")) and k % 2 else 0   # Jacobi for some
    Bd = torch.from_numpy(B).cuda()
    G0d = torch.from_numpy(G0).cuda()
    res = {}
    with bk.Operator(A) as op:
        bk.set_option(op.handle, bk.OPT_PERSISTENT, 1)   # compaction belongs to the graph path
        for compact in (1, 0):
            bk.set_option(op.handle, bk.OPT_COMPACT, compact)
            r = op.solve(Bd, X0=G0d, tol=1e-9, maxit=600, variant=variant, flags=flags)
            res[compact] = (r, r.X.cpu().numpy())
    (r1, X1), (r0, X0) = res[1], res[0]
    ro = oracle.solve(A, B, X0=G0, tol=1e-9, maxit=600, variant=variant,
                      flags=oracle.JACOBI if flags else 0)
    bar, islack = _compaction_bars(A, B, G0, 1e-9, 600, variant, flags, ro)
    assert np.array_equal(r0.status, r1.status)
    assert np.all(np.abs(r0.iters - r1.iters) <= islack), (r0.iters, r1.iters)
    assert np.all(_colerr(X0, X1) <= bar), _colerr(X0, X1)
    assert np.all(X0[:, np.all(B == 0, axis=0)] == 0.0)
    # histories: every column's entries sit at its own column, NaN after it stopped.  The two
    # layouts sum the dots in different orders, and the difference grows as the residual falls
    # (2e-6 relative at 1e-8 of the initial residual in the classical form, 8e-4 in the
    # recurrence-based estimates of the Pipelined forms), so the entries agree to 1e-2; the
    # columns' histories differ by orders of magnitude (initial errors 1 to 1e-8), so an entry
    # written at another column's place would not.
    for c in range(k):
        m = int(min(r0.iters[c], r1.iters[c]))
        np.testing.assert_allclose(r0.hist[: m + 1, c], r1.hist[: m + 1, c], rtol=1e-2)
        assert np.all(np.isfinite(r0.hist[: r0.iters[c] + 1, c]))
        assert np.all(np.isnan(r0.hist[r0.iters[c] + 1:, c]))
    if k >= 5:
        assert len(set(ro.iters.tolist())) >= 3       # the columns stop at different iterations
    _compare(r0, X0, ro, tol_sol=max(SOL_RTOL, bar), iters_slack=islack)


@pytest.mark.parametrize("variant", COMPACT_VARIANTS)
def test_column_compaction_down_to_one_column(bk, cuda, variant):
    """Seven of eight columns zero: the group narrows 8 -> 4 -> 2 -> 1 after its first iterations
    and the last column finishes alone in the one-column layout (odd row count, so the padding
    element of every vector is in play).  Host and device buffers, against the oracle."""
    torch = cuda
    A = I.convdiff7(11, peclet=True)                  # 1331 rows
    B = np.zeros((A.n, 8))
    B[:, 5] = I.rhs(A.n, 1, 3)[:, 0]
    ro = oracle.solve(A, B, tol=1e-10, maxit=500, variant=variant)
    with bk.Operator(A) as op:
        bk.set_option(op.handle, bk.OPT_PERSISTENT, 1)   # compaction belongs to the graph path
        r = op.solve(torch.from_numpy(B).cuda(), tol=1e-10, maxit=500, variant=variant)
        X = r.X.cpu().numpy()
        rh = op.solve(torch.from_numpy(B).pin_memory(), tol=1e-10, maxit=500, variant=variant)
        bk.set_option(op.handle, bk.OPT_COMPACT, 1)
        rf = op.solve(torch.from_numpy(B).cuda(), tol=1e-10, maxit=500, variant=variant)
    bar, islack = _compaction_bars(A, B, None, 1e-10, 500, variant, 0, ro)
    _compare(r, X, ro, tol_sol=max(SOL_RTOL, bar), iters_slack=islack)
    assert np.array_equal(rh.X.numpy(), X) and np.array_equal(rh.iters, r.iters)
    assert np.all(np.abs(rf.iters - r.iters) <= islack)
    assert np.all(_colerr(rf.X.cpu().numpy(), X) <= bar)
    assert np.all(r.iters[[0, 1, 2, 3, 4, 6, 7]] == 0) and r.iters[5] > 10


@pytest.mark.parametrize("variant", COMPACT_VARIANTS)
def test_column_compaction_idle_without_stops(bk, cuda, variant):
    """With the stop test off no column stops, the layout never narrows, and the compacted graph
    (its boundaries write the final values only) gives bitwise the full layout's iterates."""
    torch = cuda
    A = I.perturbed27(10, seed=4)
    B = torch.from_numpy(I.rhs(A.n, 6, 8)).cuda()
    out = []
    with bk.Operator(A) as op:
        bk.set_option(op.handle, bk.OPT_PERSISTENT, 1)   # compaction belongs to the graph path
        for compact in (1, 0):
            bk.set_option(op.handle, bk.OPT_COMPACT, compact)
            r = op.solve(B, tol=0.0, maxit=7, variant=variant, flags=bk.FLAG_NO_STOP_TEST)
            out.append((r.X.cpu().numpy(), r.hist.copy(), r.iters.copy(), r.true_relres.copy()))
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b, equal_nan=True)


def test_options_validate_their_values(bk, cuda):
    """Every execution option takes only its documented values (BICGK_E_INVALID otherwise)."""
    A = I.convdiff7(6)
    with bk.Operator(A) as op:
        for opt, good, bad in ((bk.OPT_RHS_GROUPS, (0, 1, 2, 3, 4), (-1, 5)),
                               (bk.OPT_FUSED_DOTS, (0, 1, 2), (-1, 3)),
                               (bk.OPT_THETA_IN_S, (0, 1, 2), (-1, 3)),
                               (bk.OPT_HOST_ZERO_COPY, (0, 1), (-1, 2)),
                               (bk.OPT_COMPACT, (0, 1), (-1, 2)),
                               (bk.OPT_PERSISTENT, (0, 1, 2), (-1, 3)),
                               (bk.OPT_SPMM32, (0, 1), (-1, 2)),
                               (bk.OPT_SPMM_ROWS, (0, 1, 2), (-1, 3))):
            for v in good:
                bk.set_option(op.handle, opt, v)
            for v in bad:
                with pytest.raises(bk.BicgkError):
                    bk.set_option(op.handle, opt, v)
        with pytest.raises(bk.BicgkError):
            bk.set_option(op.handle, 99, 0)


def test_automatic_persistent_route(bk, cuda):
    """BICGK_OPT_PERSISTENT = 0 runs small merged classical solves with three or more right-hand
    sides in one launch of the persistent kernel and everything else on the graph path: 16^3 with
    k = 4 in one launch; k = 1 and 2, 33^3 (35,937 rows), the basic form and the profiling mode on
    the graph path.
    The one-launch solve agrees with the graph path's at trajectory level and with the oracle."""
    torch = cuda
    A = I.convdiff7(16, peclet=True)
    B = torch.from_numpy(I.rhs(A.n, 4, 3)).cuda()
    with bk.Operator(A) as op:
        r = op.solve(B, tol=0.0, maxit=6, flags=bk.FLAG_NO_STOP_TEST)
        assert bk.last_stats(op.handle)["kernel_launches"] == 1
        Xp = r.X.cpu().numpy()
        op.solve(B[:, :1].contiguous(), tol=1e-8, maxit=500)
        assert bk.last_stats(op.handle)["kernel_launches"] > 1
        op.solve(B[:, :2].contiguous(), tol=1e-8, maxit=500)
        assert bk.last_stats(op.handle)["kernel_launches"] > 1
        op.solve(B, tol=1e-8, maxit=500, variant="classical_plain")
        assert bk.last_stats(op.handle)["kernel_launches"] > 1
        bk.set_option(op.handle, bk.OPT_PERSISTENT, 1)
        Xg = op.solve(B, tol=0.0, maxit=6, flags=bk.FLAG_NO_STOP_TEST).X.cpu().numpy()
        assert bk.last_stats(op.handle)["kernel_launches"] > 1
    assert np.all(_colerr(Xp, Xg) <= 1e-12)
    ro = oracle.solve(A, B.cpu().numpy(), tol=0.0, maxit=6, flags=oracle.NO_STOP_TEST)
    assert np.all(_colerr(Xp, ro.X) <= 1e-12)
    A33 = I.convdiff7(33, peclet=True)
    with bk.Operator(A33) as op:
        op.solve(torch.from_numpy(I.rhs(A33.n, 2, 3)).cuda(), tol=0.0, maxit=3, flags=bk.FLAG_NO_STOP_TEST)
        assert bk.last_stats(op.handle)["kernel_launches"] > 1
