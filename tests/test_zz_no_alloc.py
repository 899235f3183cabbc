"""The allocation-free solve entry point gives the same answers as bicgk_solve.

bicgk_solve_noalloc is for callers that cannot allocate GPU memory while they
solve: programs that hand out all device memory from their own pool, loops
that must not take the device-wide synchronisation of cudaMalloc/cudaFree, and
embeddings with a fixed device-memory budget.  It keeps its scratch in one
fixed-size array inside the library instead.  This file calls it through the
C-ABI twice in a row (the second call sees whatever the first left in that
array) and compares each result with bicgk_solve on the same inputs and with
the FP64 oracle, checks that the second call leaves the device's free memory
unchanged, that a malformed CSR is refused before any product reads it, and
that a problem too large for the array is refused.  It is collected last so
that a failure here stops a -x run only after every other test ran.
"""
import ctypes

import numpy as np
import pytest

from paper_1907_12874_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib(cuda):
    from paper_1907_12874_gb300 import bicgk
    L = bicgk._load()
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.bicgk_solve_noalloc.argtypes = [i64, i64, vp, vp, vp, i32, vp, vp, dbl, i32, ctypes.c_int, i32, vp, vp, vp,
                                      vp, vp, vp]
    L.bicgk_solve_noalloc.restype = ctypes.c_int
    return L


def _noalloc(L, torch, A, B, X0, tol, maxit, variant, free_delta=None):
    """One call through the C-ABI.  The caller's arrays are allocated first; with `free_delta` (a
    list) the device's free memory is read right before and right after the call itself and the
    difference appended."""
    from paper_1907_12874_gb300 import bicgk
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    rp, ci, va, Bd = dev(A.rowptr), dev(A.colidx), dev(A.vals), dev(B)
    X0d = None if X0 is None else dev(X0)
    Xd = torch.empty_like(Bd)
    k = B.shape[1]
    iters = np.zeros(k, np.int32)
    status = np.zeros(k, np.int32)
    hist = np.empty((maxit + 1, k))
    trr = np.empty(k)
    p = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())  # noqa: E731
    h = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    rc = L.bicgk_solve_noalloc(A.n, A.nnz, p(rp), p(ci), p(va), k, p(Bd), p(X0d), tol, maxit,
                               bicgk.VARIANTS[variant], 0, p(Xd), h(iters), h(status), h(hist), h(trr), stream)
    torch.cuda.synchronize()
    if free_delta is not None:
        free_delta.append(free0 - torch.cuda.mem_get_info()[0])
    assert rc == 0, L.bicgk_last_cuda_error()
    return Xd.cpu().numpy(), iters, status, hist, trr


def _reference(torch, A, B, X0, tol, maxit, variant):
    from paper_1907_12874_gb300 import bicgk
    with bicgk.Operator(A) as op:
        bicgk.set_option(op.handle, bicgk.OPT_COMPACT, 1)   # the allocation-free loop keeps its layout
        bicgk.set_option(op.handle, bicgk.OPT_PERSISTENT, 1)  # and runs the graph path's kernels
        r = op.solve(torch.from_numpy(B).cuda(), X0=None if X0 is None else torch.from_numpy(X0).cuda(),
                     tol=tol, maxit=maxit, variant=variant)
        return r.X.cpu().numpy(), r.iters, r.status, r.hist, r.true_relres


def _same(got, ref):
    X, it, st, hist, trr = got
    Xr, itr, str_, histr, trrr = ref
    assert np.array_equal(it, itr) and np.array_equal(st, str_)
    err = np.linalg.norm(X - Xr, axis=0) / np.linalg.norm(Xr, axis=0)
    assert np.all(err <= 1e-12), err
    np.testing.assert_allclose(hist, histr, rtol=1e-10, equal_nan=True)
    np.testing.assert_allclose(trr, trrr, rtol=1e-8)


def test_two_calls_in_a_row_match_bicgk_solve(lib, cuda):
    import oracle
    from oracle_bars import colerr, derived_bars
    torch = cuda
    # call 1: the 16^3 configuration, 4 RHS, merged classical BiCGStab
    A1 = I.convdiff7(16)
    B1 = I.rhs(A1.n, 4, 1)
    got1 = _noalloc(lib, torch, A1, B1, None, 1e-8, 1000, "classical_merged")
    _same(got1, _reference(torch, A1, B1, None, 1e-8, 1000, "classical_merged"))
    # against the oracle: this operator is nearly symmetric, where rounding differences grow, so
    # the bars are the oracle's own response to one rounding unit in b
    ro1 = oracle.solve(A1, B1, tol=1e-8, maxit=1000, variant="classical_merged")
    sol_bar, it_bar = derived_bars(A1, B1, ro1, tol=1e-8, maxit=1000, variant="classical_merged",
                                   label="allocation-free 16^3")
    assert np.array_equal(got1[2], ro1.status) and np.all(np.abs(got1[1] - ro1.iters) <= it_bar)
    assert np.all(colerr(got1[0], ro1.X) <= sol_bar)
    # call 2: another operator, 3 RHS (padded to 4 columns), an initial guess, Pipelined form; the
    # device's free memory is the same before and after it (the first call may have loaded the
    # library's module; this one finds everything in place)
    A2 = I.convdiff7(12, peclet=True)
    B2 = I.rhs(A2.n, 3, 2)
    X02 = 0.1 * I.rhs(A2.n, 3, 3)
    delta = []
    got2 = _noalloc(lib, torch, A2, B2, X02, 1e-9, 500, "pipelined_merged", free_delta=delta)
    assert delta == [0], delta
    _same(got2, _reference(torch, A2, B2, X02, 1e-9, 500, "pipelined_merged"))
    # against the oracle on this stable operator: the spec bar, 1e-10 and +-1 iteration
    ro2 = oracle.solve(A2, B2, X0=X02, tol=1e-9, maxit=500, variant="pipelined_merged")
    assert np.array_equal(got2[2], ro2.status) and np.all(np.abs(got2[1] - ro2.iters) <= 1)
    same = got2[1] == ro2.iters
    assert np.all(colerr(got2[0], ro2.X)[same] <= 1e-10), colerr(got2[0], ro2.X)


def test_malformed_csr_is_refused(lib, cuda):
    """A decreasing row pointer or a column index outside [0, n) is found by a check kernel before
    any product reads the arrays, and the call returns BICGK_E_BAD_CSR."""
    torch = cuda
    from paper_1907_12874_gb300 import bicgk
    A = I.convdiff7(6)
    B = I.rhs(A.n, 2, 1)
    bad_col = A.colidx.copy()
    bad_col[17] = A.n + 5
    bad_ptr = A.rowptr.copy()
    bad_ptr[10], bad_ptr[11] = bad_ptr[11], bad_ptr[10]
    for rowptr, colidx in ((A.rowptr, bad_col), (bad_ptr, A.colidx)):
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
        rp, ci, va, Bd = dev(rowptr), dev(colidx), dev(A.vals), dev(B)
        Xd = torch.empty_like(Bd)
        iters = np.zeros(2, np.int32)
        status = np.zeros(2, np.int32)
        p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
        rc = lib.bicgk_solve_noalloc(A.n, A.nnz, p(rp), p(ci), p(va), 2, p(Bd), None, 1e-8, 100,
                                     bicgk.VARIANTS["classical_merged"], 0, p(Xd),
                                     iters.ctypes.data_as(ctypes.c_void_p), status.ctypes.data_as(ctypes.c_void_p),
                                     None, None, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == -2, rc
    # a well-formed call afterwards still works
    got = _noalloc(lib, torch, A, B, None, 1e-8, 100, "classical_merged")
    assert np.all(got[2] == 0)


def test_too_large_for_the_static_scratch_is_refused(lib, cuda):
    n = 64 ** 3
    k = 32
    iters = np.zeros(k, np.int32)
    status = np.zeros(k, np.int32)
    # refused on size before any pointer is dereferenced (device pointers are placeholders)
    fake = ctypes.c_void_p(16)
    rc = lib.bicgk_solve_noalloc(n, 7 * n, fake, fake, fake, k, fake, None, 1e-8, 100, 1, 0, fake,
                                 iters.ctypes.data_as(ctypes.c_void_p), status.ctypes.data_as(ctypes.c_void_p),
                                 None, None, None)
    assert rc == -5
    assert b"static scratch holds" in lib.bicgk_last_cuda_error()
