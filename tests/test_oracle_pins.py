"""Pins of the FP64 oracle against facts fixed by the paper or by mathematics.

Nothing here compares the oracle with itself: every check is against a
printed value of the paper (Table 2 traffic counts), a library routine
(LAPACK dense solve, scipy sparse products), a closed form (A = cI), a
theorem (finite termination of the BiCG process, r_j = b - A x_j in exact
arithmetic, breakdown of a skew-symmetric operator), or structural facts of
the listings (column independence, equal iterates of equivalent forms).
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1907_12874_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
VARIANTS = list(oracle.VARIANTS)
U = 2.0 ** -53


def _sp(A):
    return A.to_scipy()


# ------------------------------------------------------------------ generators

def test_splitmix64_published_outputs():
    g = json.load(open(os.path.join(GOLDEN, "splitmix64_seed1234567.json")))
    with np.errstate(over="ignore"):
        z = np.uint64(g["seed"]) + np.arange(1, 6, dtype=np.uint64) * I._GAMMA
        out = [int(v) for v in I._mix(z)]
    assert out == g["outputs"]
    u = I.uniform(3, 100000)
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.01


@pytest.mark.parametrize("peclet", [False, True])
def test_convdiff7_equals_kronecker_form(peclet):
    """-lap + upwind beta.grad on n^3, scaled by h^2 == sum of 1-D operators in Kronecker form."""
    import scipy.sparse as sp
    n, beta = 5, (1.0, 0.5, 0.25)
    h = 1.0 / (n + 1)
    c = 1.0 if peclet else h
    Id = sp.identity(n)

    def t1(b):  # 1-D: -u_{i-1} + 2u_i - u_{i+1} plus upwind c*b*(u_i - u_{i-1})
        return sp.diags([-1.0 - c * b, 2.0 + c * b, -1.0], [-1, 0, 1], shape=(n, n))
    # index i + n*j + n^2*l: x (i) is the fastest index
    K = sp.kron(Id, sp.kron(Id, t1(beta[0]))) + sp.kron(Id, sp.kron(t1(beta[1]), Id)) + sp.kron(t1(beta[2]), sp.kron(Id, Id))
    A = I.convdiff7(n, beta, peclet=peclet)
    np.testing.assert_allclose(A.to_dense(), K.toarray(), rtol=0, atol=1e-14)
    assert np.all(np.diff(A.colidx[A.rowptr[0]:A.rowptr[1]]) > 0)
    assert A.nnz == 7 * n ** 3 - 6 * n ** 2


def test_convdiff7_sizes_of_the_workloads():
    A = I.convdiff7(16)
    assert (A.n, A.nnz) == (4096, 27136)
    # 128^3: 7N - 6*128^2 nonzeros
    assert 7 * 128 ** 3 - 6 * 128 ** 2 == 14581760


def test_perturbed27_structure():
    A = I.perturbed27(6, seed=5)
    D = A.to_dense()
    off = D - np.diag(np.diag(D))
    nz = off[off != 0]
    assert nz.min() >= -1.5 and nz.max() <= -0.5
    np.testing.assert_allclose(D.sum(axis=1), 1.0, rtol=0, atol=1e-12)   # diag = sum|off| + 1
    assert not np.allclose(D, D.T)
    assert A.nnz == (3 * 6 - 2) ** 3  # (3n-2)^3 entries of a 27-point stencil


# ------------------------------------------------------------------ dense solves

def _dense_cases():
    return [I.convdiff7(3), I.convdiff7(4), I.convdiff7(6, peclet=True), I.convdiff7(5, beta=(0, 0, 0)),
            I.perturbed27(4, seed=2)]


@pytest.mark.parametrize("variant", VARIANTS)
def test_matches_dense_lapack_solve(variant):
    for A in _dense_cases():
        B = I.rhs(A.n, 3, 17)
        D = A.to_dense()
        Xd = np.linalg.solve(D, B)
        r = oracle.solve(A, B, tol=1e-13, maxit=2000, variant=variant)
        assert np.all(r.status == oracle.CONVERGED), (A.name, r.status)
        cond = np.linalg.cond(D)
        err = np.linalg.norm(r.X - Xd, axis=0) / np.linalg.norm(Xd, axis=0)
        assert np.all(err <= 10 * cond * 1e-13), (A.name, err, cond)


@pytest.mark.parametrize("variant", VARIANTS)
def test_manufactured_solution(variant):
    A = I.convdiff7(12)
    Xs = I.rhs(A.n, 2, 23)
    B = _sp(A) @ Xs                     # scipy product, independent of the oracle's SpMV
    r = oracle.solve(A, B, tol=1e-12, maxit=3000, variant=variant)
    assert np.all(r.status == oracle.CONVERGED)
    err = np.linalg.norm(r.X - Xs, axis=0) / np.linalg.norm(Xs, axis=0)
    assert np.all(err < 1e-8), err
    assert np.all(r.true_relres < 2e-12)


def test_spmm_matches_scipy():
    A = I.perturbed27(5, seed=1)
    X = I.rhs(A.n, 3, 4)
    np.testing.assert_allclose(oracle.spmm(A, X), _sp(A) @ X, rtol=1e-14, atol=1e-14)


# ------------------------------------------------------------------ closed forms and theorems

@pytest.mark.parametrize("variant", VARIANTS)
def test_scaled_identity(variant):
    n = 50
    A2 = I.CSR(np.arange(n + 1), np.arange(n), np.full(n, 2.0))
    B = I.rhs(n, 3, 1)
    r = oracle.solve(A2, B, tol=1e-14, maxit=5, variant=variant)
    assert np.all(r.iters == 1) and np.all(r.status == oracle.CONVERGED)
    np.testing.assert_array_equal(r.X, B / 2)            # alpha = 1/2 exactly, s = 0, omega = 0
    A3 = I.CSR(np.arange(n + 1), np.arange(n), np.full(n, 3.0))
    r = oracle.solve(A3, B, tol=1e-14, maxit=5, variant=variant)
    assert np.all(r.iters == 1)
    np.testing.assert_allclose(r.X, B / 3, rtol=4 * U)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("nvals", [2, 3])
def test_finite_termination_few_eigenvalues(variant, nvals):
    """A with d distinct eigenvalues: the BiCG polynomial vanishes after d steps, so r_d = 0."""
    n = 60
    d = np.array([1.0, 3.0, 7.0][:nvals])[np.arange(n) % nvals]
    A = I.CSR(np.arange(n + 1), np.arange(n), d)
    B = I.rhs(n, 2, 3)
    r = oracle.solve(A, B, tol=1e-11, maxit=50, variant=variant)
    assert np.all(r.status == oracle.CONVERGED)
    assert np.all(r.iters <= nvals), r.iters
    np.testing.assert_allclose(r.X, B / d[:, None], rtol=1e-9)


@pytest.mark.parametrize("variant", VARIANTS)
def test_skew_operator_breaks_down(variant):
    """(A r, r) = 0 for skew-symmetric A: delta_0 = (v_0, r_0) = 0 (for Algorithm 4 (r_0, w_0) = 0)."""
    A = I.CSR(np.array([0, 1, 2]), np.array([1, 0]), np.array([1.0, -1.0]))
    B = np.array([[1.0], [2.0]])
    r = oracle.solve(A, B, tol=1e-12, maxit=10, variant=variant)
    assert r.status[0] == oracle.BREAKDOWN and r.iters[0] == 0
    np.testing.assert_array_equal(r.X, 0.0)


def test_nonfinite_rhs():
    A = I.convdiff7(3)
    B = I.rhs(A.n, 2, 1)
    B[4, 1] = np.nan
    r = oracle.solve(A, B, tol=1e-8, maxit=100)
    assert r.status[1] == oracle.NONFINITE and r.iters[1] == 0
    assert r.status[0] == oracle.CONVERGED


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("m", [1, 4, 15])
def test_recurrence_residual_is_true_residual(variant, m):
    """r_j from the recurrences equals b - A x_j up to rounding (exact in exact arithmetic)."""
    A = I.convdiff7(9)
    B = I.rhs(A.n, 2, 31)
    r = oracle.solve(A, B, tol=0.0, maxit=m, variant=variant, flags=oracle.NO_STOP_TEST)
    true = B - _sp(A) @ r.X
    gap = np.linalg.norm(r.R - true, axis=0)
    normA = np.abs(A.to_dense()).sum(axis=1).max()
    scale = np.linalg.norm(B, axis=0) + normA * np.linalg.norm(r.X, axis=0)
    assert np.all(gap <= 200 * m * U * scale), (gap, scale)


@pytest.mark.parametrize("variant", VARIANTS)
def test_recurrence_residual_at_convergence(variant):
    """The residual returned with a converged column is b - A x of the returned iterate."""
    A = I.convdiff7(9, peclet=True)
    B = I.rhs(A.n, 2, 32)
    r = oracle.solve(A, B, tol=1e-10, maxit=500, variant=variant)
    assert np.all(r.status == oracle.CONVERGED)
    gap = np.linalg.norm(r.R - (B - _sp(A) @ r.X), axis=0) / np.linalg.norm(B, axis=0)
    assert np.all(gap < 0.1 * 1e-10), gap   # rounding drift only, below the tolerance


def test_columns_are_independent_bitwise():
    A = I.convdiff7(8, peclet=True)
    B = I.rhs(A.n, 4, 2)
    for v in VARIANTS:
        rk = oracle.solve(A, B, tol=1e-9, maxit=400, variant=v)
        for c in range(4):
            r1 = oracle.solve(A, B[:, c:c + 1], tol=1e-9, maxit=400, variant=v)
            assert np.array_equal(rk.X[:, c], r1.X[:, 0])
            assert rk.iters[c] == r1.iters[0]
            assert np.array_equal(rk.hist[:, c], r1.hist[:, 0], equal_nan=True)


def test_thread_count_does_not_change_results():
    """Only row-parallel loops are threaded (every row's result is computed by one thread in a
    fixed order) and the dot products are serial, so one thread and all threads agree bitwise."""
    A = I.perturbed27(9, seed=4)
    B = I.rhs(A.n, 3, 6)
    n_all = oracle.threads()
    try:
        oracle.set_threads(1)
        assert oracle.threads() == 1
        r1 = {v: oracle.solve(A, B, tol=1e-10, maxit=300, variant=v) for v in ("classical_merged", "ppipe_plain")}
        y1 = oracle.spmm(A, B)
    finally:
        oracle.set_threads(n_all)
    for v, r in r1.items():
        rn = oracle.solve(A, B, tol=1e-10, maxit=300, variant=v)
        assert np.array_equal(r.X, rn.X) and np.array_equal(r.iters, rn.iters)
    assert np.array_equal(y1, oracle.spmm(A, B))


def test_stop_is_first_crossing():
    """iters is the first j with (estimate of ||r_j||) < tol * ||b||."""
    A = I.convdiff7(10)
    B = I.rhs(A.n, 3, 7)
    for v in VARIANTS:
        r = oracle.solve(A, B, tol=1e-7, maxit=500, variant=v)
        eps = 1e-7 * np.linalg.norm(B, axis=0)
        for c in range(3):
            h = r.hist[: r.iters[c] + 1, c]
            assert h[-1] < eps[c] and np.all(h[:-1] >= eps[c])
            assert np.all(np.isnan(r.hist[r.iters[c] + 1:, c]))


# ------------------------------------------------------------------ equal iterates of equivalent forms

@pytest.mark.parametrize("pair", [("classical_plain", "classical_merged"), ("reordered_plain", "reordered_merged"),
                                  ("pipelined_plain", "pipelined_merged"), ("precond_plain", "precond_merged"),
                                  ("ppipe_plain", "ppipe_merged"), ("improved_plain", "improved_merged")])
def test_basic_and_merged_forms_same_iterates(pair):
    """Merging changes loop structure only: the vectors are bitwise equal (Sec. 2.2)."""
    A = I.convdiff7(9)
    B = I.rhs(A.n, 2, 8)
    a = oracle.solve(A, B, tol=0.0, maxit=20, variant=pair[0], flags=oracle.NO_STOP_TEST)
    b = oracle.solve(A, B, tol=0.0, maxit=20, variant=pair[1], flags=oracle.NO_STOP_TEST)
    assert np.array_equal(a.X, b.X) and np.array_equal(a.R, b.R)


def test_merged_norm_identity():
    """(r_{j+1}, r_{j+1}) = theta - omega*phi (Sec. 1 footnote): merged estimate vs direct dot."""
    A = I.convdiff7(12)
    B = I.rhs(A.n, 2, 9)
    p = oracle.solve(A, B, tol=0.0, maxit=25, variant="classical_plain", flags=oracle.NO_STOP_TEST)
    m = oracle.solve(A, B, tol=0.0, maxit=25, variant="classical_merged", flags=oracle.NO_STOP_TEST)
    # relative error of the estimate is ~u * ||s||^2 / ||r||^2: keep to the range where that is small
    ok = p.hist[1:] > 1e-5 * p.hist[0]
    np.testing.assert_allclose(m.hist[1:][ok], p.hist[1:][ok], rtol=1e-8)


@pytest.mark.parametrize("pair", [("precond_merged", "classical_merged"), ("ppipe_merged", "pipelined_merged"),
                                  ("precond_plain", "classical_plain"), ("ppipe_plain", "pipelined_plain")])
def test_identity_preconditioner_reproduces_unpreconditioned_bitwise(pair):
    """With M = I applied as a copy, Algorithm 5 performs Algorithm 2's arithmetic and Algorithm 7
    Algorithm 4's (the hatted vectors equal the plain ones): the iterates are bitwise equal."""
    A = I.convdiff7(8, peclet=True)
    B = I.rhs(A.n, 2, 13)
    a = oracle.solve(A, B, tol=0.0, maxit=15, variant=pair[0], flags=oracle.NO_STOP_TEST)
    b = oracle.solve(A, B, tol=0.0, maxit=15, variant=pair[1], flags=oracle.NO_STOP_TEST)
    assert np.array_equal(a.X, b.X)


@pytest.mark.parametrize("variant", ["precond_merged", "ppipe_merged", "reordered_merged", "precond_plain"])
def test_jacobi_on_a_diagonal_matrix_is_exact_in_one_iterate(variant):
    """M = diag(A) = A: the preconditioned operator is I, so one iterate solves the system."""
    n = 64
    d = 1.0 + (np.arange(n) % 7)
    A = I.CSR(np.arange(n + 1), np.arange(n), d)
    B = I.rhs(n, 3, 2)
    r = oracle.solve(A, B, tol=1e-12, maxit=10, variant=variant, flags=oracle.JACOBI)
    assert np.all(r.iters == 1) and np.all(r.status == oracle.CONVERGED)
    np.testing.assert_allclose(r.X, B / d[:, None], rtol=4 * U)


@pytest.mark.parametrize("variant", ["precond_merged", "ppipe_merged", "reordered_merged", "precond_plain",
                                     "ppipe_plain", "reordered_plain"])
def test_jacobi_matches_lapack(variant):
    A = I.perturbed27(4, seed=6)
    B = I.rhs(A.n, 2, 3)
    Xd = np.linalg.solve(A.to_dense(), B)
    r = oracle.solve(A, B, tol=1e-13, maxit=500, variant=variant, flags=oracle.JACOBI)
    assert np.all(r.status == oracle.CONVERGED)
    err = np.linalg.norm(r.X - Xd, axis=0) / np.linalg.norm(Xd, axis=0)
    assert np.all(err < 1e-11)


def test_variants_agree_on_first_iterates():
    """Algorithms 1, 3, 4 and 6 generate the same iterates in exact arithmetic."""
    A = I.convdiff7(10, peclet=True)
    B = I.rhs(A.n, 2, 12)
    ref = oracle.solve(A, B, tol=0.0, maxit=4, variant="classical_plain", flags=oracle.NO_STOP_TEST)
    for v in ("reordered_merged", "pipelined_merged", "improved_merged", "improved_plain"):
        r = oracle.solve(A, B, tol=0.0, maxit=4, variant=v, flags=oracle.NO_STOP_TEST)
        err = np.linalg.norm(r.X - ref.X) / np.linalg.norm(ref.X)
        assert err < 1e-10, (v, err)


def test_variants_converge_alike():
    A = I.convdiff7(16)
    B = I.rhs(A.n, 4, 1)
    its = {}
    for v in VARIANTS:
        r = oracle.solve(A, B, tol=1e-8, maxit=1000, variant=v)
        assert np.all(r.status == oracle.CONVERGED)
        assert np.all(r.true_relres < 2e-8)
        its[v] = r.iters
    allits = np.array(list(its.values()))
    # the 16^3 h-scaled operator is rounding-chaotic: equivalent forms spread by up to ~20 %
    assert np.all(allits.max(axis=0) - allits.min(axis=0) <= 0.2 * allits.min(axis=0))


# ------------------------------------------------------------------ Table 2

def test_vector_traffic_matches_table2():
    g = json.load(open(os.path.join(GOLDEN, "table2_vector_traffic.json")))
    A = I.convdiff7(4)
    B = I.rhs(A.n, 1, 3)
    m = 7
    for v in VARIANTS:
        r = oracle.solve(A, B, tol=0.0, maxit=m, variant=v, flags=oracle.NO_STOP_TEST)
        reads, writes, copies, spmv = (int(t) for t in r.traffic)
        exp = g["per_iteration"][v]
        assert (reads, writes) == (m * exp["reads"], m * exp["writes"]), (v, reads, writes)
        # set-up: z_0 = M^-1 r_0 (Alg. 6); r^_0 and w^_0 (Alg. 7)
        setup_copies = {"reordered": 1, "ppipe": 2}.get(v.split("_")[0], 0)
        assert copies == m * g["preconditioner_copies_per_iteration"][v] + setup_copies
        # set-up SpMVs: r_0 and the true residual; w_0, t_0 (Alg. 4, 7); u_0 and A^T r_0 (Alg. 3)
        setup_spmv = 2 + {"pipelined": 2, "ppipe": 2, "improved": 2}.get(v.split("_")[0], 0)
        assert spmv == m * g["spmv_per_iteration"] + setup_spmv


# ------------------------------------------------------------------ mixed-precision refinement

def test_mixed_reaches_fp64_accuracy_lapack():
    """FP32 inner solves inside FP64 refinement still reach the FP64 solution (LAPACK)."""
    for A in (I.perturbed27(4, seed=2), I.convdiff7(5, peclet=True)):
        B = I.rhs(A.n, 2, 7)
        D = A.to_dense()
        Xd = np.linalg.solve(D, B)
        r = oracle.solve_mixed(A, B, tol=1e-13, max_outer=30, inner_tol=1e-5)
        assert np.all(r.status == oracle.CONVERGED)
        assert np.all(r.outer_iters >= 2)              # one FP32 solve cannot reach 1e-13
        err = np.linalg.norm(r.X - Xd, axis=0) / np.linalg.norm(Xd, axis=0)
        assert np.all(err <= 10 * np.linalg.cond(D) * 1e-13), err


def test_mixed_each_pass_contracts_by_the_inner_tolerance():
    """||r_{j+1}|| <= ~inner_tol ||r_j||: x += d with d solving A d = r to inner_tol."""
    A = I.perturbed27(8, seed=4)
    B = I.rhs(A.n, 3, 5)
    r = oracle.solve_mixed(A, B, tol=1e-12, max_outer=20, inner_tol=1e-4)
    assert np.all(r.status == oracle.CONVERGED)
    for c in range(3):
        h = r.hist[: r.outer_iters[c] + 1, c]
        assert np.all(h[1:] / h[:-1] < 1e-3), h
    gap = np.linalg.norm(B - A.to_scipy() @ r.X, axis=0) / np.linalg.norm(B, axis=0)
    np.testing.assert_allclose(gap, r.true_relres, rtol=1e-6)
    assert np.all(gap < 1e-12)


def test_mixed_edge_columns():
    A = I.convdiff7(5)
    B = I.rhs(A.n, 3, 1)
    B[:, 1] = 0.0
    X0 = np.ones_like(B)
    r = oracle.solve_mixed(A, B, X0=X0, tol=1e-10, max_outer=10)
    assert r.status[1] == oracle.CONVERGED and r.outer_iters[1] == 0 and np.all(r.X[:, 1] == 0)
    r0 = oracle.solve_mixed(A, B, X0=X0, tol=1e-10, max_outer=0)
    assert r0.status[0] == oracle.MAXIT and r0.outer_iters[0] == 0
    np.testing.assert_array_equal(r0.X[:, 0], 1.0)
    n = 40
    A2 = I.CSR(np.arange(n + 1), np.arange(n), np.full(n, 2.0))
    B2 = I.rhs(n, 2, 3)
    r2 = oracle.solve_mixed(A2, B2, tol=1e-15, max_outer=10)
    assert np.all(r2.status == oracle.CONVERGED) and np.all(r2.outer_iters <= 3)
    assert np.all(np.linalg.norm(r2.X - B2 / 2, axis=0) <= 2e-15 * np.linalg.norm(B2 / 2, axis=0))


# ------------------------------------------------------------------ adjoint reference

def test_adjoint_dense_matches_central_differences():
    """dL/dB and dL/dA of L = sum(W * A^-1 B) against central differences of the dense solve."""
    A = I.convdiff7(3, peclet=True)
    B = I.rhs(A.n, 2, 4)
    W = I.rhs(A.n, 2, 5)
    X, dB, dvals = oracle.adjoint_dense(A, B, W)
    h = 1e-6

    def loss(vals, Bm):
        M = I.CSR(A.rowptr, A.colidx, vals)
        return float(np.sum(W * np.linalg.solve(M.to_dense(), Bm)))
    for e in (0, 5, A.nnz // 2, A.nnz - 1):
        vp, vm = A.vals.copy(), A.vals.copy()
        vp[e] += h
        vm[e] -= h
        fd = (loss(vp, B) - loss(vm, B)) / (2 * h)
        assert abs(fd - dvals[e]) <= 1e-7 * (1 + abs(fd)), (e, fd, dvals[e])
    for (i, c) in ((0, 0), (7, 1), (A.n - 1, 0)):
        Bp, Bm = B.copy(), B.copy()
        Bp[i, c] += h
        Bm[i, c] -= h
        fd = (loss(A.vals, Bp) - loss(A.vals, Bm)) / (2 * h)
        assert abs(fd - dB[i, c]) <= 1e-7 * (1 + abs(fd))
