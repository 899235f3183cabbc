"""Differentiation path on the GPU: transpose products, SDDMM, adjoint solves and autograd.

References: scipy sparse products for A^T x; numpy for the sampled product; the
dense LAPACK adjoint (oracle.adjoint_dense, itself pinned against central
differences) for the gradients on the 12^3 instance; central differences of
GPU solves for a few entries.
"""
import numpy as np
import pytest

import oracle
from paper_1907_12874_gb300 import inputs as I

pytestmark = pytest.mark.gpu
U = 2.0 ** -52


@pytest.fixture(scope="module")
def bk(cuda):
    from paper_1907_12874_gb300 import bicgk
    return bicgk


def _rand_csr(n, seed):
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, 12, size=n)
    rowptr = np.zeros(n + 1, dtype=np.int32)
    np.cumsum(lens, out=rowptr[1:])
    cols = np.concatenate([rng.choice(n, size=l, replace=False) for l in lens]).astype(np.int32)
    return I.CSR(rowptr, cols, rng.standard_normal(rowptr[-1]))


@pytest.mark.parametrize("k", [1, 3, 8, 32])
@pytest.mark.parametrize("method", [0, 1])
def test_transpose_spmm(bk, cuda, k, method):
    torch = cuda
    for A in (I.convdiff7(9, peclet=True), _rand_csr(700, 3)):
        X = I.rhs(A.n, k, 2)
        ref = A.to_scipy().T @ X
        absT = abs(A.to_scipy()).T
        bound = 8 * U * (absT @ np.abs(X)) * max(1, int(np.diff(A.rowptr).max()) + 8) + 1e-300
        with bk.Operator(A) as op:
            Y = op.spmm_t(torch.from_numpy(X).cuda(), method=method).cpu().numpy()
        assert np.all(np.abs(Y - ref) <= bound)


def test_transpose_operator_solves_adjoint(bk, cuda):
    torch = cuda
    A = I.convdiff7(11, peclet=True)
    B = I.rhs(A.n, 3, 7)
    AT = A.to_scipy().T.tocsr()
    AT.sort_indices()
    At = I.CSR(AT.indptr, AT.indices, AT.data)
    ro = oracle.solve(At, B, tol=1e-10, maxit=500)
    with bk.Operator(A) as op:
        with op.transpose() as opT:
            r = opT.solve(torch.from_numpy(B).cuda(), tol=1e-10, maxit=500)
    X = r.X.cpu().numpy()
    assert np.all(np.abs(r.iters - ro.iters) <= 1)
    err = np.linalg.norm(X - ro.X, axis=0) / np.linalg.norm(ro.X, axis=0)
    assert np.all(err[r.iters == ro.iters] <= 1e-10)


def test_sddmm(bk, cuda):
    torch = cuda
    A = _rand_csr(500, 5)
    for k in (1, 5, 16):
        L, X = I.rhs(A.n, k, 1), I.rhs(A.n, k, 2)
        rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
        ref = -0.5 * np.einsum("ec,ec->e", L[rows], X[A.colidx])
        with bk.Operator(A) as op:
            G = op.sddmm(torch.from_numpy(L).cuda(), torch.from_numpy(X).cuda(), alpha=-0.5).cpu().numpy()
        mag = 0.5 * np.einsum("ec,ec->e", np.abs(L[rows]), np.abs(X[A.colidx]))
        assert np.all(np.abs(G - ref) <= 4 * k * U * mag + 1e-300)


def _grads(torch, A, B, W, tol=1e-12):
    from paper_1907_12874_gb300 import autograd
    dev = torch.device("cuda")
    rp = torch.from_numpy(A.rowptr).to(dev)
    ci = torch.from_numpy(A.colidx).to(dev)
    vals = torch.from_numpy(A.vals.copy()).to(dev).requires_grad_(True)
    Bt = torch.from_numpy(B.copy()).to(dev).requires_grad_(True)
    X = autograd.solve(vals, Bt, rp, ci, tol=tol, maxit=5000)
    loss = (torch.from_numpy(W).to(dev) * X).sum()
    loss.backward()
    return X.detach().cpu().numpy(), Bt.grad.cpu().numpy(), vals.grad.cpu().numpy()


def test_autograd_matches_dense_reference_12cubed(bk, cuda):
    """The 12^3 check instance of the differentiable configuration (1728 rows, 11,232 nonzeros)."""
    torch = cuda
    A = I.convdiff7(12)
    assert (A.n, A.nnz) == (1728, 11232)
    B = I.rhs(A.n, 8, 3)
    W = I.rhs(A.n, 8, 4)
    X, dB, dvals = _grads(torch, A, B, W)
    Xr, dBr, dvr = oracle.adjoint_dense(A, B, W)
    # entry by entry: the solves stop at relative residual 1e-12, so every entry of X, dL/dB and
    # dL/dA is within ||A^-1|| ||A|| 1e-12 (~1e-10 here) of the largest entry of its dense value
    for got, ref in ((X, Xr), (dB, dBr), (dvals, dvr)):
        assert np.all(np.abs(got - ref) <= 1e-9 * np.abs(ref).max()), np.abs(got - ref).max() / np.abs(ref).max()
    assert np.linalg.norm(dvals - dvr) <= 1e-9 * np.linalg.norm(dvr)


def test_autograd_reuses_the_operator_of_a_pattern(bk, cuda):
    """A second call with the same pattern tensors and new values reuses the cached operator (values
    copied in place, the transposed operator refreshed), and both calls' gradients match the dense
    reference entry by entry; a backward after another forward uses its own forward's values."""
    torch = cuda
    from paper_1907_12874_gb300 import autograd
    autograd.clear_cache()
    A = I.convdiff7(10, peclet=True)
    A2 = I.CSR(A.rowptr, A.colidx, A.vals * (1.0 + 0.1 * I.uniform(7, A.nnz)))
    B, W = I.rhs(A.n, 3, 5), I.rhs(A.n, 3, 6)
    dev = torch.device("cuda")
    rp, ci = torch.from_numpy(A.rowptr).to(dev), torch.from_numpy(A.colidx).to(dev)
    outs = []
    for M in (A, A2):
        vals = torch.from_numpy(M.vals.copy()).to(dev).requires_grad_(True)
        Bt = torch.from_numpy(B.copy()).to(dev).requires_grad_(True)
        X = autograd.solve(vals, Bt, rp, ci, tol=1e-12)
        outs.append((M, vals, Bt, X))
    assert len(autograd._cache) == 1
    for M, vals, Bt, X in reversed(outs):     # the first forward's backward runs after the second's forward
        (torch.from_numpy(W).to(dev) * X).sum().backward()
        Xr, dBr, dvr = oracle.adjoint_dense(M, B, W)
        for got, ref in ((X.detach().cpu().numpy(), Xr), (Bt.grad.cpu().numpy(), dBr), (vals.grad.cpu().numpy(), dvr)):
            assert np.all(np.abs(got - ref) <= 1e-9 * np.abs(ref).max())
    autograd.clear_cache()


def _stable_transpose(A):
    """A^T by a stable sort of A's entries by column (numpy), the reference for the device transpose."""
    perm = np.argsort(A.colidx, kind="stable")
    rows = np.repeat(np.arange(A.n, dtype=np.int32), np.diff(A.rowptr))
    rpt = np.zeros(A.n + 1, dtype=np.int32)
    np.cumsum(np.bincount(A.colidx, minlength=A.n), out=rpt[1:])
    return rpt, rows[perm], A.vals[perm]


def _csr_dups(n, seed, max_len=12):
    """Random CSR with empty rows, a long row and repeated column indices within rows."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, max_len, size=n)
    lens[: min(3, n)] = 0
    lens[n // 2] = min(3000, 4 * n)
    rowptr = np.zeros(n + 1, dtype=np.int32)
    np.cumsum(lens, out=rowptr[1:])
    cols = rng.integers(0, n, size=int(rowptr[-1])).astype(np.int32)
    return I.CSR(rowptr, cols, rng.standard_normal(rowptr[-1]))


@pytest.mark.parametrize("case", ["stencil", "dups_small", "dups_3_passes", "no_entries", "one_row"])
def test_device_transpose_is_the_stable_counting_sort(bk, cuda, case):
    """bicgk_op_transpose builds A^T on the GPU; its CSR is bitwise the stable counting sort's
    (row pointers, column indices and values), for a stencil, random patterns with repeated
    columns in a row and empty rows, n above 65,536 (three 8-bit radix passes), no entries, one row."""
    A = {"stencil": lambda: I.perturbed27(9, seed=1),
         "dups_small": lambda: _csr_dups(700, 3),
         "dups_3_passes": lambda: _csr_dups(70001, 4, max_len=6),
         "no_entries": lambda: I.CSR(np.zeros(6, np.int32), np.zeros(0, np.int32), np.zeros(0)),
         "one_row": lambda: I.CSR(np.array([0, 3], np.int32), np.zeros(3, np.int32), np.array([1.0, 2.0, 3.0]))}[case]()
    with bk.Operator(A) as op:
        with op.transpose() as opT:
            rp, ci, va = opT.get_csr()
    rpt, cit, vat = _stable_transpose(A)
    assert np.array_equal(rp, rpt) and np.array_equal(ci, cit) and np.array_equal(va, vat)


def test_new_values_follow_into_products_and_transposes(bk, cuda):
    """bicgk_op_set_values: products, the internal transposed copy (bicgk_spmm_t explicit) and a
    transposed operator refreshed with bicgk_op_transpose_refresh all use the new values."""
    torch = cuda
    A = _csr_dups(900, 8)
    A2 = I.CSR(A.rowptr, A.colidx, I.uniform(5, A.nnz))
    X = I.rhs(A.n, 4, 2)
    Xd = torch.from_numpy(X).cuda()
    with bk.Operator(A) as op:
        op.spmm_t(Xd)                                   # builds the internal transposed copy
        opT = op.transpose()
        op.set_values(torch.from_numpy(A2.vals).cuda())
        op.transpose_refresh(opT)
        Y = op.spmm(Xd).cpu().numpy()
        Yt = op.spmm_t(Xd).cpu().numpy()
        Yt2 = opT.spmm(Xd).cpu().numpy()
        rp, ci, va = opT.get_csr()
        opT.close()
        op.set_values(A.vals)                           # host values
        Y1 = op.spmm(Xd).cpu().numpy()
    S2 = A2.to_scipy()
    bound = 8 * U * (abs(S2) @ np.abs(X)) * 4000 + 1e-300
    assert np.all(np.abs(Y - S2 @ X) <= bound)
    boundT = 8 * U * (abs(S2).T @ np.abs(X)) * 4000 + 1e-300
    assert np.all(np.abs(Yt - S2.T @ X) <= boundT) and np.array_equal(Yt, Yt2)
    assert np.array_equal(va, _stable_transpose(A2)[2])
    assert np.all(np.abs(Y1 - A.to_scipy() @ X) <= 8 * U * (abs(A.to_scipy()) @ np.abs(X)) * 4000 + 1e-300)


def test_autograd_central_differences(bk, cuda):
    """Entries of dL/dA and dL/dB against central differences (h = 1e-6) of GPU solves."""
    torch = cuda
    from paper_1907_12874_gb300 import bicgk
    A = I.convdiff7(8, peclet=True)
    B = I.rhs(A.n, 2, 9)
    W = I.rhs(A.n, 2, 10)
    _, dB, dvals = _grads(torch, A, B, W, tol=1e-13)
    h = 1e-6

    def loss(vals, Bm):
        with bicgk.Operator(rowptr=A.rowptr, colidx=A.colidx, vals=vals) as op:
            r = op.solve(torch.from_numpy(Bm).cuda(), tol=1e-14, maxit=5000)
            return float(np.sum(W * r.X.cpu().numpy()))
    for e in (0, 17, A.nnz // 3, A.nnz - 2):
        vp, vm = A.vals.copy(), A.vals.copy()
        vp[e] += h
        vm[e] -= h
        fd = (loss(vp, B) - loss(vm, B)) / (2 * h)
        assert abs(fd - dvals[e]) <= 1e-5 * (1 + abs(fd)), (e, fd, dvals[e])
    for (i, c) in ((3, 0), (A.n // 2, 1)):
        Bp, Bm = B.copy(), B.copy()
        Bp[i, c] += h
        Bm[i, c] -= h
        fd = (loss(A.vals, Bp) - loss(A.vals, Bm)) / (2 * h)
        assert abs(fd - dB[i, c]) <= 1e-5 * (1 + abs(fd))


def test_autograd_64cubed_k8_runs(bk, cuda):
    """The 64^3, 8-RHS differentiable configuration: gradients satisfy the adjoint equations."""
    torch = cuda
    A = I.convdiff7(64)
    B = I.rhs(A.n, 8, 5)
    W = I.rhs(A.n, 8, 6)
    X, dB, dvals = _grads(torch, A, B, W, tol=1e-10)
    S = A.to_scipy()
    assert np.linalg.norm(S @ X - B) <= 2e-10 * np.linalg.norm(B)
    assert np.linalg.norm(S.T @ dB - W) <= 2e-10 * np.linalg.norm(W)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    ref = -np.einsum("ec,ec->e", dB[rows], X[A.colidx])
    assert np.linalg.norm(dvals - ref) <= 1e-12 * np.linalg.norm(ref)
