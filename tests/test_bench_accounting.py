"""The byte and flop accounting of bench.py (CPU): the per-kernel algorithmic figures behind
`roofline`, the whole-solve HBM figure behind `hbm`, and the traffic table reader.

The vector-pass counts are the paper's Table 2 (reads plus writes of N-vectors per iteration,
basic and merged form); the per-kernel figures follow from what each kernel reads and writes.
"""
import os

import pytest

import bench
from paper_1907_12874_gb300 import inputs as I

N, NNZ, K = 1000, 6950, 32
VEC = 8.0 * N * K


def test_table2_vector_passes():
    # Table 2: basic -> merged vector reads+writes per iteration
    assert bench.TABLE2_VECTORS["classical"] == (22, 18)
    assert bench.TABLE2_VECTORS["reordered"] == (28, 21)
    assert bench.TABLE2_VECTORS["pipelined"] == (43, 26)
    # the M^-1 copies of the preconditioned forms count as one read and one write each
    assert bench.TABLE2_COPIES["precond"] == bench.TABLE2_COPIES["reordered"] == 2
    assert bench.TABLE2_COPIES["classical"] == bench.TABLE2_COPIES["pipelined"] == 0


def test_spmm_and_epilogue_kernels():
    spmm = 12.0 * NNZ + 4.0 * (N + 1) + 2 * VEC        # CSR once, x once, y once
    b, f = bench.kernel_algorithmic("spmm_k32", N, NNZ, K)
    assert b == spmm and f == 2.0 * NNZ * K
    b, f = bench.kernel_algorithmic("spmm_resid_k32", N, NNZ, K)
    assert b == spmm + VEC and f == 2.0 * NNZ * K + N * K        # reads b too; one subtraction
    b, f = bench.kernel_algorithmic("spmm_delta_k32", N, NNZ, K)
    assert b == spmm + VEC and f == 2.0 * NNZ * K + 2.0 * N * K  # r0 read; one FMA per element
    # phi, psi (and theta) read s, which is the product's own x in Algorithm 2
    b, f = bench.kernel_algorithmic("spmm_phi_psi_k32", N, NNZ, K, "classical_merged")
    assert b == spmm and f == 2.0 * NNZ * K + 4.0 * N * K
    b, f = bench.kernel_algorithmic("spmm_g1_k32", N, NNZ, K, "classical_merged")
    assert b == spmm and f == 2.0 * NNZ * K + 6.0 * N * K
    # Algorithm 5 multiplies s^ = M^-1 s, so the epilogue reads s as well
    b, f = bench.kernel_algorithmic("spmm_phi_psi_k32", N, NNZ, K, "precond_merged")
    assert b == spmm + VEC and f == 2.0 * NNZ * K + 4.0 * N * K


@pytest.mark.parametrize("name, reads, writes, fma", [
    ("upd_s", 2, 1, 1), ("upd_s_theta", 2, 1, 2), ("merged_phi_psi_theta", 2, 0, 3),
    ("merged_phi_psi", 2, 0, 2), ("merged_x_r_rho", 5, 2, 4), ("upd_p", 3, 1, 2),
    ("dot_delta", 2, 0, 1),
])
def test_streaming_kernels(name, reads, writes, fma):
    b, f = bench.kernel_algorithmic(name, N, NNZ, K)
    assert b == (reads + writes) * VEC and f == 2.0 * fma * N * K


def test_source_kinds():
    assert bench.kernel_source_kind("spmm_k32") == "spmm"
    assert bench.kernel_source_kind("spmm_resid_k32") == "spmm"
    for fused in ("spmm_delta_k32", "spmm_g1_k32", "spmm_phi_psi_k32", "upd_p", "merged_x_r_rho"):
        assert bench.kernel_source_kind(fused) == "vec"


def test_fused_passes_saved():
    for k in (1, 4, 7):
        assert bench.fused_passes_saved("classical_merged", k) == 0      # one group: no epilogues
    assert bench.fused_passes_saved("classical_merged", 8) == 3          # v re-read; t and s
    assert bench.fused_passes_saved("precond_merged", 32) == 2           # v and t re-read
    assert bench.fused_passes_saved("reordered_merged", 32) == 1         # v re-read
    assert bench.fused_passes_saved("pipelined_merged", 32) == 0
    assert bench.fused_passes_saved("classical_plain", 32) == 0


def test_solve_gbs_by_hand():
    A = I.convdiff7(6)
    n, nnz = A.n, A.nnz
    # merged classical, k = 32 in four groups of 8: per column-iteration two products (x and y
    # once, an eighth of the CSR each) and 18 - 3 vector passes
    per = 2 * (16 * n + (12 * nnz + 4 * (n + 1)) / 8) + 15 * 8 * n
    got = bench.solve_gbs(A, 32, "classical_merged", column_iterations=1000, ms=2.0, groups=4)
    assert got == pytest.approx(1000 * per / 2e-3 / 1e9, rel=1e-12)
    # the basic form of Algorithm 5: 22 passes plus its two M^-1 copies (read and write each)
    per = 2 * (16 * n + (12 * nnz + 4 * (n + 1)) / 4) + 26 * 8 * n
    got = bench.solve_gbs(A, 4, "precond_plain", column_iterations=10, ms=1.0, groups=1)
    assert got == pytest.approx(10 * per / 1e-3 / 1e9, rel=1e-12)


def test_recorded_traffic_follows_the_source_hash(monkeypatch):
    rows = bench.recorded_traffic()
    path = os.path.join(bench.ROOT, "profiles", "ncu_dram_traffic.md")
    assert os.path.exists(path)
    for (name, k), v in rows.items():
        assert k > 0 and v > 0
    # a changed kernel source makes every row of its kind stale
    monkeypatch.setattr(bench, "source_hash", lambda kind: "000000000000")
    assert bench.recorded_traffic() == {}
