"""Benchmark: RHS-iterations/s of multi-RHS BiCGStab on GB300, merged vs plain forms.

Workload (default): 3-D 7-point upwind convection-diffusion on a 128^3 grid
(2,097,152 rows, 14,581,760 nonzeros, FP64 CSR), k = 32 right-hand sides
U[-1,1], x0 = 0, relative tolerance 1e-8, merged classical BiCGStab
(Algorithm 2 of Krasnopolsky, arXiv:1907.12874).  One step = one complete
solve (set-up, iterations until every column stops, true residual).

value    = sum over columns of iterations / solve time (device-resident inputs,
           CUDA events on the solving stream, max over ranks);
e2e      = the same through the C-ABI with pinned host buffers, the copies of
           B in and X out inside the timed region;
roofline = the dominant kernel (largest share of the per-kernel event times of
           one profiled solve): algorithmic bytes or FP64 flops per launch over
           its mean launch time, against the measured HBM copy bandwidth or the
           FP64 peak (152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz);
cpu_baseline = the FP64 oracle on a bounded sample on the host cores.

Multi-GPU (torchrun): every rank solves its own k right-hand sides (different
seeds) on its own GPU; there is no data-path collective (weak scaling).
--impl reference times the oracle instead (the CPU reference arm).
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

HBM_FALLBACK_GBS = 6800.0
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # SMs x FP64 FMA/clk x flop/FMA x max clock
L1_PEAK_BPS = 152 * 128 * 2.070e9                   # SMs x L1 data-path bytes/clk x max clock (nominal)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--grid", type=int, default=128, help="grid edge n (n^3 unknowns)")
    p.add_argument("--k", type=int, default=32, help="right-hand sides per GPU")
    p.add_argument("--variant", default="classical_merged")
    p.add_argument("--tol", type=float, default=1e-8)
    p.add_argument("--maxit", type=int, default=5000)
    p.add_argument("--no-plain", action="store_true", help="skip the plain-form comparison")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--sweep", action="store_true", help="also time every variant at k = 1..32")
    p.add_argument("--replica", action="store_true",
                   help="also run the paper's iteration benchmark: Poisson 200^3, m = 1, 4, 16, every form")
    p.add_argument("--replica-iters", type=int, default=100)
    p.add_argument("--no-mixed", action="store_true",
                   help="skip the mixed-precision comparison (27-point 128^3, k = 32, rel tol 1e-10)")
    p.add_argument("--mixed-grid", type=int, default=128)
    p.add_argument("--no-adjoint", action="store_true",
                   help="skip the differentiable solve (64^3, k = 8: forward + adjoint backward)")
    p.add_argument("--profile-mixed", action="store_true",
                   help="only the mixed-precision solve at --mixed-grid, in the host-loop mode (profiler captures)")
    p.add_argument("--profile-batch", action="store_true",
                   help="only the batched workload in the persistent mode, 10 fixed iterations, twice "
                        "(profiler captures of the persistent kernel)")
    p.add_argument("--no-small-k", action="store_true",
                   help="skip the small-problem comparison of the graph path and the persistent kernel")
    p.add_argument("--no-batch", action="store_true",
                   help="skip the batching comparison (64 systems, grids 16^3..64^3, 1..8 RHS)")
    p.add_argument("--eager", action="store_true",
                   help="run every solve in the library's host-loop mode (same kernels, one launch at a time, "
                        "CUDA events around each) instead of the CUDA graph; profilers cannot see kernels inside "
                        "graphs with conditional nodes")
    p.add_argument("--minimal", action="store_true",
                   help="only the warm-up and timed solves (for profiler captures): no e2e, plain, kernel "
                        "times or CPU baseline")
    return p.parse_args()


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"bicgk_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "sm_min_mhz": min(r[0] for r in rows), "reasons": reasons, "samples": len(rows)}


def kernel_algorithmic(name: str, n: int, nnz: int, k: int, variant: str = "classical_merged"):
    """Algorithmic bytes and FP64 flops of one launch of a kernel class (ideal x reuse)."""
    from paper_1907_12874_gb300 import bicgk as bk  # noqa: F401
    vec = 8.0 * n * k
    if name.startswith("spmm"):
        resid = name.startswith("spmm_resid")
        b = 12.0 * nnz + 4.0 * (n + 1) + 2 * vec + (vec if resid else 0.0)
        f = 2.0 * nnz * k + (n * k if resid else 0.0)
        if name.startswith("spmm_delta"):   # epilogue dot (v, r^0): reads r^0
            b, f = b + vec, f + 2.0 * n * k
        if name.startswith(("spmm_g1", "spmm_phi_psi")):  # epilogue dots (t,s), (t,t)[, (s,s)]
            # s is the product's own x in Algorithm 2 (read once); Algorithm 5 multiplies s^ = M^-1 s
            nd = 3 if name.startswith("spmm_g1") else 2
            b, f = b + (vec if variant.startswith("precond") else 0.0), f + 2.0 * nd * n * k
        return b, f
    table = {  # reads, writes, FP64 flops per element (FMA = 2)
        "dot_delta": (2, 0, 2), "upd_s": (2, 1, 2), "merged_phi_psi_theta": (2, 0, 6),
        "upd_s_theta": (2, 1, 4), "merged_phi_psi": (2, 0, 4),
        "merged_x_r_rho": (5, 2, 8), "upd_p": (3, 1, 4), "dot_phi": (2, 0, 2), "dot_psi": (1, 0, 2),
        "upd_x": (3, 1, 4), "upd_r": (2, 1, 2), "dot_rr": (1, 0, 2), "dot_rho": (2, 0, 2),
        "precond_copy_s": (1, 1, 0), "precond_copy_q": (1, 1, 0), "upd_that": (2, 1, 2),
        "merged_rtilde_4dots": (4, 1, 10), "merged_x_z_vhat": (5, 3, 10), "upd_rtilde": (2, 1, 2),
        "dot_theta": (2, 0, 2), "dot_eta": (1, 0, 2), "upd_z": (2, 1, 2), "upd_vhat": (3, 1, 4),
        "merged_pszqy_3dots": (7, 5, 22), "merged_x_r": (4, 2, 6), "merged_w_4dots": (7, 1, 12),
        "upd_q": (2, 1, 2), "upd_y": (2, 1, 2), "dot_pi": (1, 0, 2), "upd_w_part1": (2, 1, 2),
        "upd_w_part2": (2, 1, 2), "dot_sigma": (2, 0, 2), "setup_classical": (2, 2, 4),
        "setup_reordered": (2, 3, 4), "setup_pipelined": (2, 5, 4), "dot_r0_w0": (2, 0, 2),
        "dot_true_residual": (1, 0, 2),
    }
    r, w, fl = table.get(name, (0, 0, 0))
    return (r + w) * vec, fl * n * k


def launch_columns(name: str, k: int, groups: int) -> int:
    """Columns one launch of a kernel processes: the _k<kp> suffix of a product's name, else the
    padded width of the solve's column groups (the streaming kernels run per group)."""
    m = re.search(r"_k(\d+)$", name)
    if m:
        return int(m.group(1))
    kg = -(-k // max(1, groups))
    return 1 << (kg - 1).bit_length()


# FP64 FMAs per element and column-iteration of the vector operations of a form (the products add
# 2 nnz/N): classical, basic and merged: delta 1, s 1, phi/psi/theta 3 (or theta with s), x 2, r 1,
# rho 1, p 2 (the basic form's (r, r) replaces theta)
VECTOR_FMA = {"classical_merged": 11, "classical_plain": 11}


def solve_fma_per_element(variant: str, A):
    v = VECTOR_FMA.get(variant)
    return None if v is None else v + 2.0 * A.nnz / A.n


KERNEL_SOURCES = {"spmm": ("bicgk_dev.cuh", "bicgk_spmm.cu"),
                  "vec": ("bicgk_dev.cuh", "bicgk_rules.cuh", "bicgk_vec.cu")}


def kernel_source_kind(name: str) -> str:
    """Which sources a kernel class is compiled from: the SpMM kernels, or the streaming kernels
    (which also hold the SpMM with a dot epilogue)."""
    plain_spmm = name.startswith("spmm") and not name.startswith(("spmm_delta", "spmm_g1", "spmm_phi_psi"))
    return "spmm" if plain_spmm else "vec"


def source_hash(kind: str) -> str:
    """Hash of the CUDA sources a kernel class is compiled from (its ncu figures go stale with them)."""
    hsh = hashlib.sha256()
    for f in KERNEL_SOURCES[kind]:
        hsh.update(open(os.path.join(ROOT, "paper_1907_12874_gb300", "csrc", f), "rb").read())
    return hsh.hexdigest()[:12]


def recorded_traffic():
    """Per-launch DRAM bytes from the committed ncu summary, for kernels whose source is unchanged.

    Rows of profiles/ncu_dram_traffic.md: | kernel | k | bytes per launch at the bench size | source hash |.
    """
    path = os.path.join(ROOT, "profiles", "ncu_dram_traffic.md")
    if not os.path.exists(path):
        return {}
    out = {}
    for line in open(path):
        m = re.match(r"\|\s*([a-z0-9_]+)\s*\|\s*(\d+)\s*\|\s*([0-9.e+]+)\s*\|\s*([0-9a-f]{12})\s*\|", line)
        if not m:
            continue
        kind = kernel_source_kind(m.group(1))
        if m.group(4) == source_hash(kind):
            out[(m.group(1), int(m.group(2)))] = float(m.group(3))
    return out


def cpu_oracle_rate(A, B, variant, cols: int, iters: int, want=False):
    """Oracle RHS-iterations/s on `cols` columns x `iters` fixed iterations of the workload (and,
    with `want`, the oracle's result)."""
    import oracle
    t0 = time.perf_counter()
    r = oracle.solve(A, B[:, :cols], tol=0.0, maxit=iters, variant=variant, flags=oracle.NO_STOP_TEST)
    dt = time.perf_counter() - t0
    return (cols * iters / dt, dt, r) if want else (cols * iters / dt, dt)


def oracle_columns(A, B, jobs, workers=None):
    """The oracle on single columns concurrently (columns never interact, so a column solved alone
    is the column of a k-column solve).  jobs: list of (column, kwargs for oracle.solve or, with
    kwargs["mixed"], oracle.solve_mixed); returns the results in order."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor

    def one(job):
        c, kw = job
        kw = dict(kw)
        mixed = kw.pop("mixed", False)
        x0 = kw.pop("X0", None)
        oracle.set_threads(1)
        b = np.ascontiguousarray(B[:, [c]])
        return (oracle.solve_mixed if mixed else oracle.solve)(A, b, X0=x0, **kw)

    with ThreadPoolExecutor(max(1, min(len(jobs), workers or os.cpu_count() or 1))) as ex:
        return list(ex.map(one, jobs))


def colerr(X, Xo):
    """Relative 2-norm difference per column."""
    den = np.linalg.norm(Xo, axis=0)
    return np.linalg.norm(X - Xo, axis=0) / np.where(den == 0, 1.0, den)


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(v: float, pg, device=None) -> float:
    """Largest value over all ranks (the timing rule: the slowest rank sets the step time)."""
    if pg is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_local: float, ms_local: float, pg, device=None) -> float:
    """Whole-job throughput: units of all ranks over the slowest rank's time."""
    if pg is None:
        return units_local / (ms_local / 1e3)
    import torch
    t = torch.tensor([units_local], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item()) / (max_over_ranks(ms_local, pg, device) / 1e3)


def run_reference(args):
    """CPU reference arm: the FP64 oracle as it stands, on the host cores, rank 0 only."""
    world, rank, local, pg = dist_setup(args)
    if rank != 0:
        return
    import oracle
    from paper_1907_12874_gb300 import inputs
    A = inputs.convdiff7(args.grid)
    B = inputs.rhs(A.n, args.k, 2)
    cols, iters = 2, 40        # about 1.6 s of CPU time per step on 16 cores
    for _ in range(args.warmup):
        cpu_oracle_rate(A, B, args.variant, cols, iters)
    rates, secs = [], 0.0
    for _ in range(args.steps):
        r, dt = cpu_oracle_rate(A, B, args.variant, cols, iters)
        rates.append(r)
        secs += dt
    value = args.steps * cols * iters / secs
    sample = f"{cols} columns x {iters} fixed iterations of the {args.grid}^3 k={args.k} workload per step"
    line = {
        "impl": "reference", "metric": "RHS-iterations/s", "value": value, "unit": "RHS-iterations/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, A),
        "cpu_baseline": {"value": value, "unit": "RHS-iterations/s", "cores": oracle.threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "RHS-iterations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(args, A):
    return {"workload": f"convdiff7 upwind {args.grid}^3 (beta=(1,0.5,0.25), h-scaled), k={args.k} RHS U[-1,1], "
                        f"x0=0, rel tol {args.tol:g}, {args.variant}",
            "n_rows": A.n, "nnz": A.nnz, "k": args.k, "variant": args.variant, "rel_tol": args.tol,
            "l2": f"inputs larger than L2: each N x k vector is {8 * A.n * args.k / 1e6:.0f} MB",
            "parallelism": "one independent k-RHS system per GPU"}


def mixed_section(args, bicgk, inputs, torch, dev):
    """27-point perturbed stencil, k = 32: mixed-precision refinement vs FP64 at relative tolerance
    1e-10 (the configuration's target) and again at 1e-8 (the benchmark's tolerance).

    Both solves run to the same FP64 true-residual tolerance on the same GPU; the time is the
    whole solve (CUDA events), the figure of merit the time to solution.
    """
    n = args.mixed_grid
    k = 32
    A = inputs.perturbed27(n, seed=7)
    Bh = inputs.rhs(A.n, k, 3)
    B = torch.from_numpy(Bh).to(dev)
    res = {"workload": f"perturbed27 {n}^3 (off-diagonals -U[0.5,1.5], diag = sum|off| + 1), k={k}, "
                       f"rel tol 1e-10", "n_rows": A.n, "nnz": A.nnz}

    def timed_solve(fn, steps=3):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            r = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, r

    with bicgk.Operator(A) as op64, bicgk.Operator(A) as opm:
        X = torch.empty_like(B)
        ms64, r64 = timed_solve(lambda: op64.solve(B, X=X, tol=1e-10, maxit=5000, want_hist=False))
        msm, rm = timed_solve(lambda: opm.solve_mixed(B, X=X, tol=1e-10, max_outer=20, inner_tol=1e-5,
                                                      max_inner=5000, want_hist=False))
        cols = [0, 31]       # one in each of the two column groups
        Xm = X[:, cols].cpu().numpy()
        # the same comparison at relative residual 1e-8
        ms64b, r64b = timed_solve(lambda: op64.solve(B, X=X, tol=1e-8, maxit=5000, want_hist=False))
        msmb, rmb = timed_solve(lambda: opm.solve_mixed(B, X=X, tol=1e-8, max_outer=20, inner_tol=1e-5,
                                                        max_inner=5000, want_hist=False))
    res["at_rel_tol_1e-8"] = {
        "fp64_ms": ms64b, "fp64_iters_per_rhs": float(r64b.iters.mean()),
        "fp64_converged": bool((r64b.status == 0).all()), "mixed_ms": msmb,
        "mixed_outer_passes": int(rmb.outer_iters.max()), "mixed_fp32_iters_per_rhs": float(rmb.inner_iters.mean()),
        "mixed_max_true_relres": float(rmb.true_relres.max()), "mixed_converged": bool((rmb.status == 0).all()),
        "speedup_vs_fp64": ms64b / msmb}
    res.update({
        "fp64_ms": ms64, "fp64_iters_per_rhs": float(r64.iters.mean()),
        "fp64_max_true_relres": float(r64.true_relres.max()), "fp64_converged": bool((r64.status == 0).all()),
        "mixed_ms": msm, "mixed_outer_passes": int(rm.outer_iters.max()),
        "mixed_fp32_iters_per_rhs": float(rm.inner_iters.mean()),
        "mixed_max_true_relres": float(rm.true_relres.max()), "mixed_converged": bool((rm.status == 0).all()),
        "speedup_vs_fp64": ms64 / msm,
    })
    # the inner solves' dominant kernel, the FP32 product: per-launch event times of one profiled
    # solve (its column groups one after another), against HBM and against the L1 data path that
    # carries one x row of kp floats per nonzero
    with bicgk.Operator(A) as opp:
        bicgk.set_profiling(opp.handle, True)
        opp.solve_mixed(B, tol=1e-10, max_outer=20, inner_tol=1e-5, max_inner=5000, want_hist=False)
        torch.cuda.synchronize()
        times = bicgk.kernel_times(opp.handle)
    inner = {k: v for k, v in times.items() if k.startswith(("fp32_", "spmm32_"))}
    name, (launches, kms) = max(((k, v) for k, v in inner.items() if k.startswith("spmm32_")),
                                key=lambda kv: kv[1][1])
    kp = int(name.rsplit("_k", 1)[1])
    mean_s = kms / launches / 1e3
    alg = 8.0 * A.nnz + 4.0 * (A.n + 1) + 2 * 4.0 * A.n * kp
    x_l1 = 4.0 * A.nnz * kp
    hbm, hbm_kind = hbm_peak()
    res["fp32_product"] = {
        "kernel": name, "launches": launches, "mean_launch_us": mean_s * 1e6,
        "share_of_inner_kernel_time": kms / sum(t for _, t in inner.values()),
        "algorithmic_bytes_per_launch": alg, "hbm_gbs": alg / mean_s / 1e9, "hbm_frac": alg / mean_s / 1e9 / hbm,
        "hbm_peak_kind": f"{hbm_kind} copy bandwidth",
        "l1_x_bytes_per_launch": x_l1, "l1_floor_frac": x_l1 / L1_PEAK_BPS / mean_s,
        "l1_peak_kind": "nominal L1 data path: 152 SMs x 128 B/clk x 2070 MHz"}
    # error against the oracle's refinement (oracle.solve_mixed) on the sampled columns
    kw = dict(mixed=True, tol=1e-10, max_outer=20, inner_tol=1e-5, max_inner=5000)
    ro = oracle_columns(A, Bh, [(c, kw) for c in cols])
    Xo = np.concatenate([r.X for r in ro], axis=1)
    res["oracle_err"] = {"value": float(colerr(Xm, Xo).max()),
                         "max_abs_over_max_abs_x": float(np.abs(Xm - Xo).max() / np.abs(Xo).max()),
                         "what": f"columns {cols} of the rel. tol 1e-10 mixed solve against oracle.solve_mixed: "
                                 "max relative 2-norm difference, and the largest elementwise difference "
                                 "over max |x|"}
    return res


def batch_section(args, bicgk, inputs, torch, dev, nsys=64):
    """64 independent 7-point convection-diffusion systems, grids U{16..64}^3, k U{1..8}, rel tol 1e-8.

    Three ways to run the same batch, CUDA events around each: the persistent mode (one cooperative
    kernel launch for every system, its rows per CTA tile autotuned), the batched graph (one graph
    launch, a branch per system) and the per-system launch loop (bicgk_solve per system), the last
    two with the autotuned per-system launch shapes.
    """
    import oracle
    grids, ks = inputs.batch_draws(nsys)
    csrs = [inputs.convdiff7(n) for n in grids]
    Bs = [torch.from_numpy(inputs.rhs(c.n, k, 200 + i)).to(dev) for i, (c, k) in enumerate(zip(csrs, ks))]
    Xs = [torch.empty_like(b) for b in Bs]
    res = {"workload": f"{nsys} convdiff7 systems, grids U{{16..64}}^3, k U{{1..8}}, rel tol 1e-8, classical_merged",
           "rows_total": int(sum(c.n for c in csrs)), "rhs_total": int(sum(ks))}
    sample = sorted({int(np.argmin(grids)), int(np.argmax(grids)), int(np.argmax(ks))})
    got = {}
    with bicgk.Batch(csrs, ks) as bt:
        t0 = time.perf_counter()
        bt.tune(reps=5)
        torch.cuda.synchronize()
        res["tune_s"] = time.perf_counter() - t0
        t0 = time.perf_counter()
        rows = bt.tune_persistent(reps=3)
        torch.cuda.synchronize()
        res["tune_persistent_s"] = time.perf_counter() - t0
        res["persistent_rows_per_tile"] = sorted({int(r) for r in rows})
        out = {}
        for name, mode in (("persistent", bicgk.BATCH_PERSISTENT), ("graph", bicgk.BATCH_GRAPH),
                           ("loop", bicgk.BATCH_LOOP)):
            bt.solve(Bs, Xs, tol=1e-8, maxit=5000, mode=mode)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            reps = 3
            for _ in range(reps):
                _, iters, status, trr = bt.solve(Bs, Xs, tol=1e-8, maxit=5000, mode=mode)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            out[name] = {"ms": ms, "rhs_iterations_per_s": float(iters.sum()) / (ms / 1e3),
                         "kernel_launches": bt.last_launches(), "converged": bool((status == 0).all()),
                         "max_true_relres": float(trr.max())}
            if mode == bicgk.BATCH_PERSISTENT:
                out[name]["loop_iterations"] = bt.last_loop_iters()
                out[name]["launch"] = bt.persistent_info()
            got[name] = {i: Xs[i].cpu().numpy() for i in sample}
        res.update(out)
        res["graph_speedup_vs_loop"] = out["loop"]["ms"] / out["graph"]["ms"]
        res["persistent_speedup_vs_loop"] = out["loop"]["ms"] / out["persistent"]["ms"]
        res["persistent_speedup_vs_graph"] = out["graph"]["ms"] / out["persistent"]["ms"]
    # error against the oracle's to-tolerance solves of sampled systems: the smallest and the largest
    # grids, a system with the most right-hand sides
    errs = {}
    for i in sample:
        Bh = Bs[i].cpu().numpy()
        ro = oracle_columns(csrs[i], Bh, [(c, dict(tol=1e-8, maxit=5000)) for c in range(ks[i])])
        Xo = np.concatenate([r.X for r in ro], axis=1)
        for name in got:
            errs[f"{name}: system {i} ({grids[i]}^3, k={ks[i]})"] = float(colerr(got[name][i], Xo).max())
    res["oracle_err"] = {"value": max(errs.values()), "systems": errs,
                         "what": "max relative 2-norm difference per column against the oracle's solve to the "
                                 "same tolerance (this nearly symmetric operator amplifies rounding: both "
                                 "stopping iterates sit within the tolerance of the exact solution)"}
    return res


# Table 4 of the paper (Lomonosov-2, one node of 14 Xeon cores, FP64): seconds per iteration of the
# 7-point Poisson problem on a 200^3 grid, basic and merged forms, m = 1, 4, 16 right-hand sides.
PAPER_TABLE4 = {
    "classical": {1: (0.062, 0.058), 4: (0.181, 0.164), 16: (0.65, 0.59)},
    "improved": {1: (0.074, 0.061), 4: (0.236, 0.182), 16: (0.87, 0.66)},
    "pipelined": {1: (0.087, 0.069), 4: (0.282, 0.212), 16: (1.06, 0.78)},
    "precond": {1: (0.066, 0.064), 4: (0.201, 0.189), 16: (0.72, 0.68)},
    "reordered": {1: (0.072, 0.065), 4: (0.224, 0.196), 16: (0.81, 0.70)},
    "ppipe": {1: (0.107, 0.085), 4: (0.368, 0.279), 16: (1.39, 1.03)},
}
# vector reads + writes per iteration (Table 2) and M^-1 copies (one read + one write each)
TABLE2_VECTORS = {"classical": (22, 18), "improved": (33, 20), "pipelined": (43, 26), "precond": (22, 19),
                  "reordered": (28, 21), "ppipe": (56, 34)}
TABLE2_COPIES = {"classical": 0, "improved": 0, "pipelined": 0, "precond": 2, "reordered": 2, "ppipe": 2}


def fused_passes_saved(variant: str, k: int) -> int:
    """Vector passes per iteration that the dot epilogues of the SpMM save (the library fuses when
    a solve runs as concurrent column groups, k >= 8): the dot kernel after v = A p re-reads v; the one
    after t = A s re-reads t and s, and s is the product's own x in Algorithm 2 (in Algorithm 5 the
    product reads s^ = M^-1 s, so the epilogue still reads s)."""
    if k < 8:
        return 0
    return {"classical_merged": 3, "precond_merged": 2, "reordered_merged": 1}.get(variant, 0)


def solve_gbs(A, k: int, variant: str, column_iterations: int, ms: float, groups: int) -> float:
    """Algorithmic HBM GB/s of the useful work of a solve: every column-iteration reads x and
    writes y in the form's two products, pays its share of the CSR reads of its group's products
    (12 nnz + 4 (N + 1) bytes per product, shared by the group's columns), and makes the form's
    vector passes of Table 2 (8 N bytes each, M^-1 copies as one read and one write).  Iterations
    of columns that have already stopped count as time, not as bytes."""
    base, form = variant.rsplit("_", 1)
    N, nnz = A.n, A.nnz
    kg = k / groups
    vecs = TABLE2_VECTORS[base][0 if form == "plain" else 1] + 2 * TABLE2_COPIES[base]
    vecs -= fused_passes_saved(variant, k)
    per_col_iter = 2 * (16 * N + (12 * nnz + 4 * (N + 1)) / kg) + vecs * 8 * N
    return column_iterations * per_col_iter / (ms / 1e3) / 1e9


def sweep_section(args, bicgk, inputs, torch, dev, A, hbm_gbs, nit=40):
    """Every form at k = 1, 2, 4, 8, 16, 32 on the benchmark operator: fixed-iteration timing (graph
    mode, CUDA events), RHS-iterations/s = k / time per iteration of a nit-iteration solve (its
    set-up and finish included), the marginal time of an iteration (a 4 nit-iteration solve minus
    the nit-iteration one, over 3 nit) with the fixed cost per solve it leaves, and the achieved fraction of the
    HBM copy bandwidth for the algorithmic bytes of one iteration: two products of
    12 nnz + 4 (N + 1) + 16 N k bytes (x read once) and 8 N k bytes per vector pass of Table 2
    (M^-1 copies as one read and one write each).  paper_model_ms is the paper's data-transfer
    model T = Sigma / B (Eq. SpMV_mem, x read C + 1 times) with B the measured HBM bandwidth."""
    import oracle
    N, nnz = A.n, A.nnz
    res = {"workload": f"{args.grid}^3 benchmark operator, {nit} fixed iterations per form and k; "
                       f"oracle_err_8_iterations: column 0 after 8 fixed iterations against the oracle's",
           "hbm_gbs": hbm_gbs, "rows": {}}
    with bicgk.Operator(A) as opw:
        for k in (1, 2, 4, 8, 16, 32):
            Bh = inputs.rhs(N, k, 2)
            Bk = torch.from_numpy(Bh).to(dev)
            Xk = torch.empty_like(Bk)
            col0 = {}
            for v in bicgk.VARIANTS:
                base, form = v.rsplit("_", 1)
                opw.solve(Bk, X=Xk, tol=0.0, maxit=3, variant=v, flags=bicgk.FLAG_NO_STOP_TEST, want_hist=False)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                t_solve = {}
                for m in (nit, 4 * nit):
                    e0.record()
                    opw.solve(Bk, X=Xk, tol=0.0, maxit=m, variant=v, flags=bicgk.FLAG_NO_STOP_TEST,
                              want_hist=False, want_true=False)
                    e1.record()
                    torch.cuda.synchronize()
                    t_solve[m] = e0.elapsed_time(e1) / 1e3
                s_it = t_solve[nit] / nit
                # the iteration alone: the difference of the two solves (their set-up, finish and
                # transfers are the same) over the 3 nit iterations between them
                s_marg = (t_solve[4 * nit] - t_solve[nit]) / (3 * nit)
                vecs = TABLE2_VECTORS[base][0 if form == "plain" else 1] + 2 * TABLE2_COPIES[base]
                # the passes this implementation makes (the SpMM dot epilogues save some at k >= 8)
                byts = 2 * (12 * nnz + 4 * (N + 1) + 16 * N * k) + (vecs - fused_passes_saved(v, k)) * 8 * N * k
                C = nnz / N
                model = (2 * N * (8 * k * (C + 1) + 4 * (3 * C + 1)) + vecs * 8 * N * k) / (hbm_gbs * 1e9)
                res["rows"][f"{v}/k{k}"] = {"rhs_iterations_per_s": k / s_it, "ms_per_iter": s_it * 1e3,
                                            "marginal_ms_per_iter": s_marg * 1e3,
                                            "fixed_ms_per_solve": (t_solve[nit] - nit * s_marg) * 1e3,
                                            "algorithmic_gb_per_iter": byts / 1e9,
                                            "hbm_frac": byts / s_it / (hbm_gbs * 1e9),
                                            "hbm_frac_marginal": byts / s_marg / (hbm_gbs * 1e9),
                                            "paper_model_ms": model * 1e3}
                # error against the oracle: column 0 after 8 fixed iterations of the same solve (past
                # a few dozen iterations this operator amplifies rounding differences to the percent
                # level in any two implementations, the oracle's own one-unit response included)
                opw.solve(Bk, X=Xk, tol=0.0, maxit=8, variant=v, flags=bicgk.FLAG_NO_STOP_TEST, want_hist=False)
                col0[v] = Xk[:, :1].cpu().numpy()
            jobs = [(0, dict(tol=0.0, maxit=8, variant=v, flags=oracle.NO_STOP_TEST)) for v in col0]
            for v, ro in zip(col0, oracle_columns(A, Bh, jobs)):
                res["rows"][f"{v}/k{k}"]["oracle_err_8_iterations"] = float(colerr(col0[v], ro.X)[0])
    return res


def small_k_section(args, bicgk, inputs, torch, dev, A128):
    """Small problems, where a kernel's data phase lasts a few microseconds and launch, ramp and
    reduction tails set the pace: the graph path against the persistent kernel (bicgk_solve with
    BICGK_OPT_PERSISTENT = 2, one cooperative launch per solve).
      * the 16^3 configuration (4,096 rows, k = 4, h-scaled convection-diffusion, rel. tol 1e-8):
        time per solve (CUDA events, mean of 20), against the oracle's solve;
      * the 128^3 benchmark operator at k = 1, 2, 4: time per iteration over 40 fixed iterations,
        x after 12 fixed iterations against the oracle's."""
    import oracle
    res = {}
    A16 = inputs.convdiff7(16)
    B16h = inputs.rhs(A16.n, 4, 1)
    B16 = torch.from_numpy(B16h).to(dev)
    X16 = torch.empty_like(B16)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ro = oracle.solve(A16, B16h, tol=1e-8, maxit=1000)
    row = {"workload": "convdiff7 16^3 (4,096 rows), k=4, rel tol 1e-8, classical_merged"}
    with bicgk.Operator(A16) as op:
        for name, opt in (("graph", 1), ("persistent", 2)):
            bicgk.set_option(op.handle, bicgk.OPT_PERSISTENT, opt)
            r = op.solve(B16, X=X16, tol=1e-8, maxit=1000, want_hist=False)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(20):
                r = op.solve(B16, X=X16, tol=1e-8, maxit=1000, want_hist=False)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 20
            row[name] = {"ms_per_solve": ms, "rhs_iterations_per_s": float(r.iters.sum()) / (ms / 1e3),
                         "iters": r.iters.tolist(), "kernel_launches": bicgk.last_stats(op.handle)["kernel_launches"],
                         "oracle_err": float(colerr(X16.cpu().numpy(), ro.X).max()),
                         "max_true_relres": float(r.true_relres.max())}
    row["oracle_iters"] = ro.iters.tolist()
    row["persistent_speedup"] = row["graph"]["ms_per_solve"] / row["persistent"]["ms_per_solve"]
    res["config_16cubed_k4"] = row
    nit = 40
    rows128 = {}
    with bicgk.Operator(A128) as op:
        for k in (1, 2, 4):
            Bh = inputs.rhs(A128.n, k, 2)
            Bk = torch.from_numpy(Bh).to(dev)
            Xk = torch.empty_like(Bk)
            ro12 = oracle_columns(A128, Bh, [(0, dict(tol=0.0, maxit=12, flags=oracle.NO_STOP_TEST))])[0]
            row = {}
            for name, opt in (("graph", 1), ("persistent", 2)):
                bicgk.set_option(op.handle, bicgk.OPT_PERSISTENT, opt)
                op.solve(Bk, X=Xk, tol=0.0, maxit=3, flags=bicgk.FLAG_NO_STOP_TEST, want_hist=False)
                torch.cuda.synchronize()
                e0.record()
                op.solve(Bk, X=Xk, tol=0.0, maxit=nit, flags=bicgk.FLAG_NO_STOP_TEST, want_hist=False, want_true=False)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / nit
                op.solve(Bk, X=Xk, tol=0.0, maxit=12, flags=bicgk.FLAG_NO_STOP_TEST, want_hist=False)
                row[name] = {"us_per_iter": ms * 1e3, "rhs_iterations_per_s": k / (ms / 1e3),
                             "oracle_err_12_iterations": float(colerr(Xk[:, :1].cpu().numpy(), ro12.X)[0])}
            row["persistent_speedup"] = row["graph"]["us_per_iter"] / row["persistent"]["us_per_iter"]
            rows128[f"k{k}"] = row
    res["benchmark_operator_128cubed"] = {"workload": f"{A128.name}, {nit} fixed iterations, classical_merged",
                                          "rows": rows128}
    return res


def replica_section(args, bicgk, inputs, torch, dev, hbm_gbs):
    """The paper's iteration benchmark on the GPU (Sec. 2.3, Tables 3-4): 7-point Poisson on a
    200^3 grid (8,000,000 rows), m = 1, 4, 16 right-hand sides U[-1,1], fixed iteration count, every
    form basic and merged.  Per iteration: measured time (graph mode, CUDA events), the paper's
    data-transfer model T = Sigma / B (Eq. SpMV_mem for the two products, 8 N m bytes per vector
    pass, B = the measured HBM copy bandwidth), and the paper's own Lomonosov-2 times."""
    n = 200
    A = inputs.convdiff7(n, beta=(0.0, 0.0, 0.0))
    N, C = A.n, A.nnz / A.n
    nit = args.replica_iters
    res = {"workload": f"7-point Poisson {n}^3 ({N} rows, {A.nnz} nnz), x0 = 0, B U[-1,1] seed 5, "
                       f"{nit} fixed iterations per timing (the paper uses 1000; the time per iteration "
                       f"is steady)", "hbm_gbs": hbm_gbs, "rows": {}}
    import oracle
    with bicgk.Operator(A) as op:
        for m in (1, 4, 16):
            Bh = inputs.rhs(N, m, 5)
            B = torch.from_numpy(Bh).to(dev)
            X = torch.empty_like(B)
            chk = []
            sig_mul = N * (8 * m * (C + 1) + 4 * (3 * C + 1))
            for base in PAPER_TABLE4:
                row = {}
                for form in ("plain", "merged"):
                    v = f"{base}_{form}"
                    op.solve(B, X=X, tol=0.0, maxit=3, variant=v, flags=bicgk.FLAG_NO_STOP_TEST, want_hist=False)
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    r = op.solve(B, X=X, tol=0.0, maxit=nit, variant=v, flags=bicgk.FLAG_NO_STOP_TEST,
                                 want_hist=False, want_true=False)
                    e1.record()
                    torch.cuda.synchronize()
                    ms = e0.elapsed_time(e1) / nit
                    vecs = TABLE2_VECTORS[base][0 if form == "plain" else 1] + 2 * TABLE2_COPIES[base]
                    model_ms = (2 * sig_mul + vecs * 8 * N * m) / (hbm_gbs * 1e9) * 1e3
                    row[form] = {"ms_per_iter": ms, "model_ms": model_ms,
                                 "all_columns_ran": bool((r.status == 1).all() and (r.iters == nit).all())}
                # error against the oracle: column 0 after 5 fixed iterations of each form
                for form in ("plain", "merged"):
                    v = f"{base}_{form}"
                    op.solve(B, X=X, tol=0.0, maxit=5, variant=v, flags=bicgk.FLAG_NO_STOP_TEST, want_hist=False)
                    chk.append((f"{base}/m{m}", form, v, X[:, :1].cpu().numpy()))
                p_basic, p_merged = PAPER_TABLE4[base][m]
                row["merged_gain"] = row["plain"]["ms_per_iter"] / row["merged"]["ms_per_iter"] - 1
                row["paper_lomonosov2_s"] = {"basic": p_basic, "merged": p_merged, "gain": p_basic / p_merged - 1}
                res["rows"][f"{base}/m{m}"] = row
            jobs = [(0, dict(tol=0.0, maxit=5, variant=v, flags=oracle.NO_STOP_TEST)) for _, _, v, _ in chk]
            for (key, form, _, x), ro in zip(chk, oracle_columns(A, Bh, jobs)):
                res["rows"][key][form]["oracle_err_5_iterations"] = float(colerr(x, ro.X)[0])
    return res


def adjoint_section(args, bicgk, inputs, torch, dev):
    """64^3 convection-diffusion, 8 RHS, loss = sum(w * X): forward + backward wall time (CUDA events).

    The backward solves A^T Lambda = w with BiCGStab on the transposed operator and forms
    dL/dA on the pattern; compared with the forward solve alone (plain FP64 BiCGStab).
    """
    from paper_1907_12874_gb300 import autograd
    A = inputs.convdiff7(64)
    rp = torch.from_numpy(A.rowptr).to(dev)
    ci = torch.from_numpy(A.colidx).to(dev)
    B = torch.from_numpy(inputs.rhs(A.n, 8, 5)).to(dev)
    W = torch.from_numpy(inputs.rhs(A.n, 8, 6)).to(dev)

    def step():
        vals = torch.from_numpy(A.vals.copy()).to(dev).requires_grad_(True)
        Bt = B.clone().requires_grad_(True)
        X = autograd.solve(vals, Bt, rp, ci, tol=1e-8, maxit=5000)
        (W * X).sum().backward()
        return X, vals.grad, Bt.grad

    step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    reps = 3
    for _ in range(reps):
        X, gv, gB = step()
    e1.record()
    torch.cuda.synchronize()
    ms_fb = e0.elapsed_time(e1) / reps
    with bicgk.Operator(A) as op:
        op.solve(B, tol=1e-8, maxit=5000, want_hist=False)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            op.solve(B, tol=1e-8, maxit=5000, want_hist=False)
        e1.record()
        torch.cuda.synchronize()
        ms_f = e0.elapsed_time(e1) / reps
    S = A.to_scipy()
    adj_res = float(np.linalg.norm(S.T @ gB.cpu().numpy() - W.cpu().numpy()) / np.linalg.norm(W.cpu().numpy()))
    # error against the dense reference gradients (oracle.adjoint_dense) on the 12^3 instance
    import oracle
    A12 = inputs.convdiff7(12)
    B12 = inputs.rhs(A12.n, 8, 5)
    W12 = inputs.rhs(A12.n, 8, 6)
    vals12 = torch.from_numpy(A12.vals.copy()).to(dev).requires_grad_(True)
    B12t = torch.from_numpy(B12).to(dev).requires_grad_(True)
    X12 = autograd.solve(vals12, B12t, torch.from_numpy(A12.rowptr).to(dev), torch.from_numpy(A12.colidx).to(dev),
                         tol=1e-12, maxit=5000)
    (torch.from_numpy(W12).to(dev) * X12).sum().backward()
    Xr, dBr, dvr = oracle.adjoint_dense(A12, B12, W12)
    gb_err = float(np.abs(B12t.grad.cpu().numpy() - dBr).max() / np.abs(dBr).max())
    gv_err = float(np.abs(vals12.grad.cpu().numpy() - dvr).max() / np.abs(dvr).max())
    return {"workload": "convdiff7 64^3 (262,144 rows, 1,810,432 nnz), k=8, loss = sum(w*X), rel tol 1e-8",
            "forward_backward_ms": ms_fb, "forward_solve_ms": ms_f, "backward_over_forward": ms_fb / ms_f - 1.0,
            "adjoint_relres": adj_res, "grad_vals_finite": bool(torch.isfinite(gv).all()),
            "oracle_err": {"value": max(gb_err, gv_err), "dL_dB": gb_err, "dL_dA": gv_err,
                           "what": "12^3 instance (1,728 rows), k = 8, solves to rel. tol 1e-12: largest "
                                   "elementwise difference of the gradients from oracle.adjoint_dense (dense "
                                   "LAPACK solves) over the largest gradient entry"}}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    from paper_1907_12874_gb300 import bicgk, inputs

    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    if args.profile_mixed:
        A = inputs.perturbed27(args.mixed_grid, seed=7)
        B = torch.from_numpy(inputs.rhs(A.n, 32, 3)).to(dev)
        with bicgk.Operator(A) as opm:
            bicgk.set_profiling(opm.handle, True)
            for _ in range(1 + args.steps):
                r = opm.solve_mixed(B, tol=1e-10, max_outer=20, inner_tol=1e-5, max_inner=5000, want_hist=False)
            torch.cuda.synchronize()
            times = bicgk.kernel_times(opm.handle)
        print(json.dumps({"profile_mixed": True, "grid": args.mixed_grid, "outer": int(r.outer_iters.max()),
                          "inner": float(r.inner_iters.mean()), "kernel_ms": times}), flush=True)
        return

    if args.profile_batch:
        grids, ks = inputs.batch_draws()
        csrs = [inputs.convdiff7(n) for n in grids]
        Bs = [torch.from_numpy(inputs.rhs(c.n, k, 200 + i)).to(dev) for i, (c, k) in enumerate(zip(csrs, ks))]
        with bicgk.Batch(csrs, ks) as bt:
            for _ in range(2):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                _, iters, _, _ = bt.solve(Bs, tol=0.0, maxit=10, flags=bicgk.FLAG_NO_STOP_TEST,
                                          mode=bicgk.BATCH_PERSISTENT)
                e1.record()
                torch.cuda.synchronize()
            print(json.dumps({"profile_batch": True, "ms_10_iterations": e0.elapsed_time(e1),
                              "persistent": bt.persistent_info(), "column_iterations": int(iters.sum())}), flush=True)
        return

    A = inputs.convdiff7(args.grid)
    B_host = inputs.rhs(A.n, args.k, 2 + rank)
    op = bicgk.Operator(A)
    if args.eager:
        bicgk.set_profiling(op.handle, True)
    Bd = torch.from_numpy(B_host).to(dev)
    Xd = torch.empty_like(Bd)

    def one(variant, B=Bd, X=Xd):
        return op.solve(B, X=X, tol=args.tol, maxit=args.maxit, variant=variant, want_hist=False)

    def timed(variant, steps, warmup, B=Bd, X=Xd, clocks=False):
        for _ in range(warmup):
            one(variant, B, X)
        iters_total = 0
        launches = 0
        barrier(pg)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sampler = ClockSampler(local) if clocks else None
        if sampler:
            sampler.__enter__()
        e0.record(stream)
        results = []
        for _ in range(steps):
            r = one(variant, B, X)
            results.append(r)
            launches += bicgk.last_stats(op.handle)["kernel_launches"]
        e1.record(stream)
        torch.cuda.synchronize()
        if sampler:
            sampler.__exit__()
        barrier(pg)
        ms = e0.elapsed_time(e1)
        iters_total = sum(int(r.iters.sum()) for r in results)
        return ms, iters_total, launches, results, (sampler.summary() if sampler else None)

    # headline: device-resident inputs
    ms, its, launches, results, clocks = timed(args.variant, args.steps, args.warmup, clocks=not args.minimal)
    groups = bicgk.last_stats(op.handle)["groups"]
    # sampled columns of the timed solve, for the oracle's to-tolerance solves below
    tol_cols = [c for c in (0, 9, 18, 27) if c < args.k]
    X_head = Xd[:, tol_cols].cpu().numpy()
    it_head = results[-1].iters[tol_cols].copy()
    bg_pool, bg = None, {}
    value = aggregate_rate(float(its), ms, pg, dev)
    ms = max_over_ranks(ms, pg, dev)
    last = results[-1]
    conv_ok = bool(np.all(last.status == 0))
    relres = float(np.max(last.true_relres))

    if args.minimal:
        op.close()
        if rank == 0:
            print(json.dumps({"metric": "RHS-iterations/s", "value": value, "unit": "RHS-iterations/s",
                              "ms_per_step": ms / args.steps, "eager": args.eager, "iters_per_rhs": float(its) / (args.steps * args.k),
                              "config": workload_config(args, A), "minimal": True}), flush=True)
        return

    # end to end through the C-ABI with pinned host buffers
    Bh = torch.from_numpy(B_host).pin_memory()
    Xh = torch.empty_like(Bh).pin_memory()
    ms_e2e, its_e2e, _, _, clocks_e2e = timed(args.variant, args.steps, 1, B=Bh, X=Xh, clocks=True)
    e2e_value = aggregate_rate(float(its_e2e), ms_e2e, pg, dev)
    nbytes = 8 * A.n * args.k
    # the host link as this process sees it: one plain pinned copy each way (CUDA events)
    link = {}
    for name, dst, src in (("h2d_gbs", Xd, Bh), ("d2h_gbs", Xh, Bd)):
        dst.copy_(src, non_blocking=True)
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(3):
            dst.copy_(src, non_blocking=True)
        c1.record(stream)
        torch.cuda.synchronize()
        link[name] = 3 * nbytes / (c0.elapsed_time(c1) / 1e3) / 1e9

    out = {
        "metric": "RHS-iterations/s", "value": value, "unit": "RHS-iterations/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, A),
        "iters_per_rhs": float(its) / (args.steps * args.k), "rhs_groups": groups,
        "converged": conv_ok, "max_true_relres": relres,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": "RHS-iterations/s", "ms_per_step": ms_e2e / args.steps,
                "iters_per_rhs": float(its_e2e) / (args.steps * args.k), "clocks": clocks_e2e,
                "pinned_copy_gbs": link,
                "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes + 8 * args.k + 8 * args.k},
    }

    # merged vs plain on the same GPU (the paper's comparison, Tab. 4)
    if not args.no_plain:
        plain = args.variant.replace("merged", "plain")
        if plain != args.variant:
            msp, itsp, _, _, _ = timed(plain, args.steps, 1)
            groups_p = bicgk.last_stats(op.handle)["groups"]
            vp = aggregate_rate(float(itsp), msp, pg, dev)
            msp = max_over_ranks(msp, pg, dev)
            hbm, _ = hbm_peak()
            gm = solve_gbs(A, args.k, args.variant, its, ms, groups)
            gp = solve_gbs(A, args.k, plain, itsp, msp, groups_p)
            out["hbm"] = {"unit": "GB/s", "peak_gbs": hbm, "merged_gbs": gm, "merged_frac": gm / hbm,
                          "plain_gbs": gp, "plain_frac": gp / hbm,
                          "bytes": "algorithmic bytes of the useful column-iterations (products: x, y and the "
                                   "group's CSR share; Table 2 vector passes) over the solve time"}
            out["plain"] = {"variant": plain, "value": vp, "ms_per_step": msp / args.steps,
                            "merged_speedup": value / vp}

    # the oracle's to-tolerance solves of the sampled columns, on four host threads while the GPU
    # sections below run (columns never interact, so a column solved alone is that column of the solve)
    if not args.no_cpu and rank == 0 and world == 1:
        import oracle
        from concurrent.futures import ThreadPoolExecutor

        def oracle_tol(c):
            oracle.set_threads(1)
            return oracle.solve(A, np.ascontiguousarray(B_host[:, [c]]), tol=args.tol, maxit=args.maxit,
                                variant=args.variant)
        bg_pool = ThreadPoolExecutor(len(tol_cols))
        bg = {c: bg_pool.submit(oracle_tol, c) for c in tol_cols}

    # per-kernel event times of one solve (profiling mode: the solve's own column groups and
    # kernels, the groups one after another on the same stream) -> roofline of the dominant kernel
    bicgk.set_profiling(op.handle, True)
    one(args.variant)
    torch.cuda.synchronize()
    times = bicgk.kernel_times(op.handle)
    prof_groups = bicgk.last_stats(op.handle)["groups"]
    bicgk.set_profiling(op.handle, args.eager)
    total = sum(t for _, t in times.values())
    dom, (dl, dt) = max(times.items(), key=lambda kv: kv[1][1])
    kl = launch_columns(dom, args.k, prof_groups)
    byts, flops = kernel_algorithmic(dom, A.n, A.nnz, kl, args.variant)
    avg_s = dt / dl / 1e3
    hbm, hbm_kind = hbm_peak()
    t_mem, t_alu = byts / (hbm * 1e9), flops / (FP64_PEAK_TFLOPS * 1e12)
    traffic = recorded_traffic().get((dom, args.k))
    if t_alu > t_mem:
        ach = flops / avg_s / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_TFLOPS, "traffic": traffic, "kernel": dom,
                "peak_kind": "FP64: 152 SMs x 2 FMA/clk x 2 flop x 2070 MHz",
                "hbm_achieved_gbs": byts / avg_s / 1e9, "hbm_peak_gbs": hbm, "hbm_peak_kind": hbm_kind}
    else:
        ach = byts / avg_s / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": traffic, "kernel": dom, "peak_kind": f"{hbm_kind} copy bandwidth",
                "fp64_achieved_tflops": flops / avg_s / 1e12, "fp64_peak_tflops": FP64_PEAK_TFLOPS}
    roof.update({"algorithmic_bytes_per_launch": byts, "flops_per_launch": flops, "launches": dl,
                 "mean_launch_ms": dt / dl, "share": dt / total if total else None,
                 "columns_per_launch": kl, "profiled_groups": prof_groups})
    # the whole solve against the FP64 roof: the form's FP64 FMAs per element and column-iteration
    # (two products of nnz/N FMAs each, the vector operations' FMAs) over the timed solves
    fma = solve_fma_per_element(args.variant, A)
    if fma is not None:
        roof["whole_solve_fp64_tflops"] = 2.0 * fma * A.n * its / (ms / 1e3) / 1e12
        roof["whole_solve_fp64_frac"] = roof["whole_solve_fp64_tflops"] / FP64_PEAK_TFLOPS
        roof["whole_solve_fma_per_element"] = fma
    out["roofline"] = roof
    out["kernel_shares"] = {k: {"launches": v[0], "ms": v[1], "share": v[1] / total} for k, v in
                            sorted(times.items(), key=lambda kv: -kv[1][1])}

    if args.sweep and rank == 0:
        out["sweep"] = sweep_section(args, bicgk, inputs, torch, dev, A, hbm_peak()[0])

    # small problems: the graph path against the persistent kernel
    if not args.no_small_k and rank == 0:
        out["small_k"] = small_k_section(args, bicgk, inputs, torch, dev, A)

    # the paper's own iteration benchmark (Poisson 200^3, every form, m = 1, 4, 16)
    if args.replica and rank == 0:
        out["paper_replica"] = replica_section(args, bicgk, inputs, torch, dev, hbm_peak()[0])

    # mixed precision (FP32 inner solves in FP64 refinement) vs FP64 on the same GPU
    if not args.no_mixed and rank == 0:
        out["mixed_precision"] = mixed_section(args, bicgk, inputs, torch, dev)

    # batch of 64 uneven systems: one graph launch vs the per-system launch loop
    if not args.no_batch and rank == 0:
        out["batching"] = batch_section(args, bicgk, inputs, torch, dev)

    # differentiable solve: forward BiCGStab + adjoint BiCGStab on A^T + gradient on the pattern
    if not args.no_adjoint and rank == 0:
        out["differentiation"] = adjoint_section(args, bicgk, inputs, torch, dev)

    # CPU oracle on the host cores (rank 0, N = 1 only)
    if not args.no_cpu and rank == 0 and world == 1:
        import oracle
        cols, iters = 8, 60    # about 10 s of CPU time on 16 cores
        rate, secs = cpu_oracle_rate(A, B_host, args.variant, cols, iters)
        out["cpu_baseline"] = {"value": rate, "unit": "RHS-iterations/s", "cores": oracle.threads(),
                               "kind": "oracle",
                               "sample": f"{cols} of the {args.k} columns x {iters} fixed iterations "
                                         f"({secs:.1f} s of CPU time)"}
        # error against the oracle in the benchmark's own launch configuration (all k columns, the
        # same column groups and kernels): (1) 12 fixed iterations on the 8 columns, beside the
        # oracle's own change under one rounding unit in b (this operator amplifies rounding
        # differences: by 60 iterations both are at the percent level); (2) the solve to tolerance
        # on sampled columns, against the oracle's solves started above
        m = 12
        op.solve(Bd, X=Xd, tol=0.0, maxit=m, variant=args.variant, flags=bicgk.FLAG_NO_STOP_TEST, want_hist=False)
        Xg = Xd[:, :cols].cpu().numpy()
        kw = dict(tol=0.0, maxit=m, variant=args.variant, flags=oracle.NO_STOP_TEST)
        ro = oracle_columns(A, B_host, [(c, kw) for c in range(cols)])
        g = np.random.default_rng(5)
        Bp = B_host[:, :cols] * (1.0 + 2.0 ** -52 * g.standard_normal((A.n, cols)))
        rp = oracle_columns(A, Bp, [(c, kw) for c in range(cols)])
        Xo = np.concatenate([r.X for r in ro], axis=1)
        err = colerr(Xg, Xo)
        resp = colerr(np.concatenate([r.X for r in rp], axis=1), Xo)
        rt = {c: bg[c].result() for c in tol_cols}
        bg_pool.shutdown()
        Xt = np.concatenate([rt[c].X for c in tol_cols], axis=1)
        err_t = colerr(X_head, Xt)
        out["oracle_err"] = {
            "value": float(err.max()), "per_column": err.tolist(),
            "oracle_one_unit_response": float(resp.max()),
            "what": f"max over columns 0..{cols - 1} of ||x_gpu - x_oracle|| / ||x_oracle|| after {m} fixed "
                    f"iterations of the k = {args.k} solve in the benchmark's launch configuration; "
                    "oracle_one_unit_response: the oracle's own change when b moves by one rounding unit",
            "to_tolerance": {"columns": tol_cols, "max_rel_err": float(err_t.max()), "per_column": err_t.tolist(),
                             "gpu_iters": it_head.tolist(), "oracle_iters": [int(rt[c].iters[0]) for c in tol_cols],
                             "what": "the timed solve's solution on these columns against the oracle's solve to "
                                     "the same tolerance (both stopping iterates lie within the tolerance of the "
                                     "exact solution; rounding differences decide which iterate stops)"}}
        # the oracle's basic form of the same method (one loop per vector operation), all cores
        plain_v = args.variant.replace("_merged", "_plain")
        if plain_v != args.variant:
            colsp, itersp = 2, 30
            ratep, secsp = cpu_oracle_rate(A, B_host, plain_v, colsp, itersp)
            out["cpu_baseline"]["basic_form"] = {"variant": plain_v, "value": ratep, "cores": oracle.threads(),
                                                 "sample": f"{colsp} columns x {itersp} fixed iterations ({secsp:.1f} s)"}
        # the same oracle on one core (the paper's runs use one MPI rank per core)
        all_threads = oracle.threads()
        oracle.set_threads(1)
        rate1, secs1 = cpu_oracle_rate(A, B_host, args.variant, 1, 12)
        oracle.set_threads(all_threads)
        out["cpu_baseline"]["one_core"] = {"value": rate1, "cores": 1,
                                           "sample": f"1 column x 12 fixed iterations ({secs1:.1f} s)"}
    op.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
