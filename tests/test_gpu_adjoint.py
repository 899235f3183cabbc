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
    assert np.linalg.norm(X - Xr) <= 1e-9 * np.linalg.norm(Xr)
    assert np.linalg.norm(dB - dBr) <= 1e-9 * np.linalg.norm(dBr)
    assert np.linalg.norm(dvals - dvr) <= 1e-9 * np.linalg.norm(dvr)


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
