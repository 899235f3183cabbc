// Persistent batched solve: merged BiCGStab (Algorithm 2 of Krasnopolsky, arXiv:1907.12874) for
// many independent systems of uneven size and RHS count in ONE cooperative kernel launch.
//
// Why: the per-kernel path launches 5 kernels per iteration per system (plus set-up and final
// kernels).  For small systems (16^3..64^3, 1..8 right-hand sides) every kernel's data phase is
// a few microseconds, so launch, block ramp and the last-block reduction tail set the pace.  Here
// one grid that fits on the GPU at once (cooperative launch: co-residency guaranteed) walks all
// systems' row tiles phase by phase, with a grid-wide barrier between the listing's merged groups.
//
// Work decomposition.  System i is cut into row tiles of R_i = (256 / L) * sub_i rows, L = max(1,
// kp/2) lanes per row (each lane owns columns 2q, 2q+1 of its row, double2 moves; kp = 1 one
// scalar column).  All tiles of all systems form one index space; block b takes tiles b, b + G,
// b + 2G, ...  A tile of a system that no longer iterates is skipped.
//
// One iteration (j), per live system, Algorithm 2's groups as phases:
//   P1  v = A p, delta = (v, r0)          -> alpha = rho / delta            barrier
//   P2  s = r - alpha v                                                     barrier
//   P3  t = A s, phi = (t, s), psi = (t, t), theta = (s, s)
//                                          -> omega, stop test (R1, R6)      barrier
//   P4  x += alpha p + omega s (columns that formed x_{j+1}), r = s - omega t,
//       rho' = (r, r0)                     -> beta, next rho; end of iteration barrier
//   P5  p = r + beta (p - omega v)                                          barrier
// Set-up: pack B, X0 (barrier); r = b - A x, r0 = p = r, (b, b), (r, r) -> eps, rho (barrier).
// Final: true residual ||b - A x|| and X out.
//
// Dot products: a lane's row products, summed over the block's tiles of the system in tile order
// (a system's tiles are contiguous, so a block meets its tiles of one system one after another)
// -> warp butterfly over the lanes of a column -> warps in order -> one partial per block and
// system -> the last of the system's min(G, tiles) blocks to arrive (atomic ticket, no wait) sums
// the partials in block-slot order and runs the listing's scalar rule for every column
// (bicgk_rules.cuh).  The order is fixed by the tiling and the grid, so results are bitwise
// reproducible.
//
// Grid barrier: arrival counter (64-bit, monotone within a launch, cleared by the host before
// every launch) and a spin of thread 0 of each block on an acquire load.  Every wait is bounded:
// after `deadline_ns` of %globaltimer (or an equivalent spin count) the block records the barrier
// and itself in the control block, raises the error flag and returns; blocks that see the flag
// return at their next barrier.  The host reads the flag and reports BICGK_E_TIMEOUT.
//
// Memory ordering: vectors written in one phase are read by other blocks only after a barrier
// (fence + release/acquire on the counter); the CSR is read-only and goes through the read-only
// path; data other blocks write during the launch (partials, scalars, flags, liveness) is read
// with L2-coherent loads.
#include "bicgk_persist.cuh"
#include "bicgk_rules.cuh"

namespace bicgk {

namespace {

constexpr int kPT = kPersistThreads;  // threads per block

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_i32(const int *p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier with a deadline.  Returns false if this launch was aborted (by this block's
// own timeout or another's).  Only thread 0 of a block waits; its arrival target and barrier
// count live in shared memory (no registers held across the phases).
__device__ bool grid_sync(const PersistArgs &pa, unsigned long long *s_target, int *s_index, int *s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long target = *s_target + gridDim.x;
    const int index = *s_index + 1;
    *s_target = target;
    *s_index = index;
    PersistCtl *pc = pa.pc;
    const unsigned long long max_spins = pa.deadline_ns / 16 + 1000000ull;
    __threadfence();
    atomicAdd(&pc->bar, 1ULL);
    int ok = 1;
    const unsigned long long t0 = gtimer();
    for (unsigned long long spin = 0;; ++spin) {
      if (ld_acquire_u64(&pc->bar) >= target) break;
      if (ld_relaxed_i32(&pc->err)) {
        ok = 0;
        break;
      }
      if (gtimer() - t0 > pa.deadline_ns || spin >= max_spins) {
        if (atomicCAS(&pc->err, 0, 1) == 0) {
          pc->err_barrier = index;
          pc->err_block = blockIdx.x;
        }
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// Lanes per row, rows per 256-thread pass, columns per lane.
template <int KP>
struct Geo {
  static constexpr int L = KP >= 4 ? KP / 2 : 1;
  static constexpr int RPP = kPT / L;
};

template <int KP>
__device__ __forceinline__ double2 vld(const double *v, int64_t i, int q) {
  if constexpr (KP == 1) {
    return make_double2(v[i], 0.0);
  } else {
    return reinterpret_cast<const double2 *>(v)[i * (KP / 2) + q];
  }
}
template <int KP>
__device__ __forceinline__ void vst(double *v, int64_t i, int q, double2 x) {
  if constexpr (KP == 1) {
    v[i] = x.x;
  } else {
    reinterpret_cast<double2 *>(v)[i * (KP / 2) + q] = x;
  }
}
__device__ __forceinline__ double2 fma2(double2 s, double2 x, double2 y) {
  return make_double2(fma(s.x, x.x, y.x), fma(s.y, x.y, y.y));
}
__device__ __forceinline__ double2 neg2(double2 s) { return make_double2(-s.x, -s.y); }
__device__ __forceinline__ void dacc(double2 &acc, double2 u, double2 w) {
  acc.x = fma(u.x, w.x, acc.x);
  acc.y = fma(u.y, w.y, acc.y);
}
// Per-column scalar of the lane's two columns (written by other blocks during the launch).
template <int KP>
__device__ __forceinline__ double2 sc2(const PersistSys &S, int slot, int q) {
  const double *p = S.sc + slot * kMaxKp + 2 * q;
  if constexpr (KP == 1) {
    return make_double2(__ldcg(p), 0.0);
  } else {
    return make_double2(__ldcg(p), __ldcg(p + 1));
  }
}

// Shared memory of a block.  The dot-product scratch and the CSR staging buffer share storage:
// a block stages entries only inside a tile's row passes and reduces only between tiles.
struct Smem {
  union {
    struct {
      double red[kPT / 32][3][kMaxKp];  // per-warp dot sums of the block's tiles of a system
      double tmp[kPT];                  // system reduction: per-thread sums
      double res[3 * kMaxKp];           // system reduction: the dots, [d * kp + c]
    } r;
    struct {
      double sval[kPersistStage];       // staged CSR entries of a 256-row pass (kp <= 2)
      int32_t scol[kPersistStage];
    } st;
  } u;
  unsigned long long bar_target;  // grid barrier: arrivals that complete the next barrier
  int bar_index;                  // grid barrier: barriers passed
  int ok;
  int last;
  int pref[kPersistMaxSys + 1];   // tiles of the systems a phase runs, exclusive prefix
  int scan_warp[kPT / 32];
};

// y = A x (or b - A x) for the lane's row i and column pair q.  KP <= 2 may read the tile's
// entries from shared memory (staged: entries [te0, te0 + staged)).
template <int KP>
__device__ __forceinline__ double2 row_product(const PersistSys &S, const double *x, int64_t i, int q,
                                               const Smem &sm, int te0, bool staged) {
  const int e0 = __ldg(S.rowptr + i), e1 = __ldg(S.rowptr + i + 1);
  double2 acc = make_double2(0.0, 0.0);
  if constexpr (KP <= 2) {
    if (staged) {
      for (int e = e0; e < e1; ++e) {
        const double av = sm.u.st.sval[e - te0];
        const double2 u = vld<KP>(x, sm.u.st.scol[e - te0], 0);
        acc.x = fma(av, u.x, acc.x);
        acc.y = fma(av, u.y, acc.y);
      }
      return acc;
    }
  }
  int e = e0;
  for (; e + 1 < e1; e += 2) {
    const int j0 = __ldg(S.colidx + e), j1 = __ldg(S.colidx + e + 1);
    const double a0 = __ldg(S.vals + e), a1 = __ldg(S.vals + e + 1);
    const double2 u0 = vld<KP>(x, j0, q), u1 = vld<KP>(x, j1, q);
    acc.x = fma(a0, u0.x, acc.x);
    acc.y = fma(a0, u0.y, acc.y);
    acc.x = fma(a1, u1.x, acc.x);
    acc.y = fma(a1, u1.y, acc.y);
  }
  if (e < e1) {
    const int j0 = __ldg(S.colidx + e);
    const double a0 = __ldg(S.vals + e);
    const double2 u0 = vld<KP>(x, j0, q);
    acc.x = fma(a0, u0.x, acc.x);
    acc.y = fma(a0, u0.y, acc.y);
  }
  return acc;
}

// Sum the lanes' dot accumulators over the block and store the block's partial [slot][d][c].
template <int KP, int ND>
__device__ void tile_partials(const PersistSys &S, int tl, double2 (&acc)[3], Smem &sm) {
  constexpr int L = Geo<KP>::L;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();  // the reduction scratch shares storage with the staged CSR entries of the last pass
#pragma unroll
  for (int d = 0; d < ND; ++d) {
#pragma unroll
    for (int m = L; m < 32; m <<= 1) {
      acc[d].x += __shfl_xor_sync(0xffffffffu, acc[d].x, m);
      acc[d].y += __shfl_xor_sync(0xffffffffu, acc[d].y, m);
    }
    if (lane < L) {
      if constexpr (KP == 1) {
        sm.u.r.red[w][d][0] = acc[d].x;
      } else {
        sm.u.r.red[w][d][2 * lane] = acc[d].x;
        sm.u.r.red[w][d][2 * lane + 1] = acc[d].y;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < ND * KP) {
    const int d = threadIdx.x / KP, c = threadIdx.x % KP;
    double s = 0.0;
#pragma unroll
    for (int ww = 0; ww < kPT / 32; ++ww) s += sm.u.r.red[ww][d][c];
    S.part[((int64_t)tl * 3 + d) * KP + c] = s;
    __threadfence();
  }
}

// Whether this block is the last of the `parts` blocks that contribute to a system in a phase.
__device__ bool arrive(unsigned *ticket, int parts, Smem &sm) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(ticket, 1u);
    sm.last = prev == (unsigned)(parts - 1);
  }
  __syncthreads();
  if (sm.last) __threadfence();
  return sm.last != 0;
}

// Sum of the system's `parts` block partials in slot order (fixed split over threads), into sm.res.
template <int KP, int ND>
__device__ void sys_sum(const PersistSys &S, int parts, Smem &sm) {
  constexpr int P = ND * KP;
  constexpr int T = kPT / P;  // threads per (dot, column)
  const int t = threadIdx.x;
  if (t < P * T) {
    const int p = t / T, u = t % T;
    const int d = p / KP, c = p % KP;
    double s = 0.0;
    for (int tl = u; tl < parts; tl += T) s += __ldcg(S.part + ((int64_t)tl * 3 + d) * KP + c);
    sm.u.r.tmp[t] = s;
  }
  __syncthreads();
  if (t < P) {
    double s = 0.0;
    for (int u = 0; u < T; ++u) s += sm.u.r.tmp[t * T + u];
    sm.u.r.res[t] = s;  // t = d * KP + c
  }
  __syncthreads();
}

__device__ KArgs rule_args(const PersistSys &S, int kp) {
  KArgs a = {};
  a.sc = S.sc;
  a.fl = S.fl;
  a.ctl = S.ctl;
  a.n = S.n;
  a.kp = kp;
  a.kp_out = kp;
  a.cmap = nullptr;
  a.ext_act = nullptr;
  return a;
}

enum Phase : int { PH_PACK = 0, PH_SETUP, PH_P1, PH_P2, PH_P3, PH_P4, PH_P5, PH_FINAL };

// Dot products a phase takes, and whether it multiplies by A.
template <int PH>
struct PhaseInfo {
  static constexpr int ND = PH == PH_SETUP ? 2 : PH == PH_P1 ? 1 : PH == PH_P3 ? 3 : PH == PH_P4 ? 1 : PH == PH_FINAL ? 1 : 0;
  static constexpr bool SPMM = PH == PH_SETUP || PH == PH_P1 || PH == PH_P3 || PH == PH_FINAL;
};

// The lane's per-column scalars a phase uses (alpha, omega, beta, the x-update flags), loaded once
// per block and system when the block reaches its first tile of the system.
struct LaneSc {
  double2 al, om, be;
  bool u0, u1;
};
template <int KP, int PH>
__device__ LaneSc lane_scalars(const PersistSys &S) {
  const int q = threadIdx.x % Geo<KP>::L;
  LaneSc ls;
  ls.al = ls.om = ls.be = make_double2(0.0, 0.0);
  ls.u0 = ls.u1 = false;
  if constexpr (PH == PH_P2 || PH == PH_P4) ls.al = sc2<KP>(S, S_ALPHA, q);
  if constexpr (PH == PH_P4 || PH == PH_P5) ls.om = sc2<KP>(S, S_OMEGA, q);
  if constexpr (PH == PH_P5) ls.be = sc2<KP>(S, S_BETA, q);
  if constexpr (PH == PH_P4) {
    ls.u0 = __ldcg(S.fl + F_XUPD * kMaxKp + 2 * q) != 0;
    ls.u1 = KP > 1 && __ldcg(S.fl + F_XUPD * kMaxKp + 2 * q + 1) != 0;
  }
  return ls;
}

// One tile of one phase for a system with kp = KP; the lane's dot products are added to acc.
// Not inlined: each (KP, phase) routine gets the block's whole register budget (inlined into the
// one kernel, the union of their live values spilled inside the row loops); the call costs a few
// local-memory moves per tile.
template <int KP, int PH>
__device__ __noinline__ void run_tile(const PersistSys &S, int tl, Smem &sm, double2 (&acc)[3], const LaneSc &ls) {
  constexpr int L = Geo<KP>::L, RPP = Geo<KP>::RPP;
  constexpr bool SPMM = PhaseInfo<PH>::SPMM;
  const int q = threadIdx.x % L;
  const int rr = threadIdx.x / L;
  const int64_t rows = (int64_t)RPP * S.sub;
  const int64_t r0 = (int64_t)tl * rows;
  const int64_t r1 = r0 + rows < S.n ? r0 + rows : S.n;
  double *const *V = S.vec;
  const double2 al = ls.al, om = ls.om, be = ls.be;
  const bool u0 = ls.u0, u1 = ls.u1;
  if constexpr (PH == PH_P2 || PH == PH_P4 || PH == PH_P5) {
    // streaming phases; s and p updates keep two rows per thread in flight (both rows' loads before
    // either's store), the five-vector x/r update one row
    if constexpr (PH == PH_P2) {  // s = r - alpha v
      for (int64_t p0 = r0; p0 < r1; p0 += 2 * RPP) {
        const int64_t i0 = p0 + rr, i1 = p0 + RPP + rr;
        double2 ra = make_double2(0.0, 0.0), va = ra, rb = ra, vb = ra;
        if (i0 < r1) {
          ra = vld<KP>(V[P_R], i0, q);
          va = vld<KP>(V[P_V], i0, q);
        }
        if (i1 < r1) {
          rb = vld<KP>(V[P_R], i1, q);
          vb = vld<KP>(V[P_V], i1, q);
        }
        if (i0 < r1) vst<KP>(V[P_S], i0, q, fma2(neg2(al), va, ra));
        if (i1 < r1) vst<KP>(V[P_S], i1, q, fma2(neg2(al), vb, rb));
      }
    } else if constexpr (PH == PH_P5) {  // p = r + beta (p - omega v)
      for (int64_t p0 = r0; p0 < r1; p0 += 2 * RPP) {
        const int64_t i0 = p0 + rr, i1 = p0 + RPP + rr;
        double2 ra = make_double2(0.0, 0.0), pa_ = ra, va = ra, rb = ra, pb = ra, vb = ra;
        if (i0 < r1) {
          ra = vld<KP>(V[P_R], i0, q);
          pa_ = vld<KP>(V[P_P], i0, q);
          va = vld<KP>(V[P_V], i0, q);
        }
        if (i1 < r1) {
          rb = vld<KP>(V[P_R], i1, q);
          pb = vld<KP>(V[P_P], i1, q);
          vb = vld<KP>(V[P_V], i1, q);
        }
        if (i0 < r1) vst<KP>(V[P_P], i0, q, fma2(be, fma2(neg2(om), va, pa_), ra));
        if (i1 < r1) vst<KP>(V[P_P], i1, q, fma2(be, fma2(neg2(om), vb, pb), rb));
      }
    } else {  // x += alpha p + omega s (columns that formed x_{j+1}); r = s - omega t; rho = (r, r0)
      for (int64_t i = r0 + rr; i < r1; i += RPP) {
        const double2 x = vld<KP>(V[P_X], i, q), p = vld<KP>(V[P_P], i, q), sv = vld<KP>(V[P_S], i, q);
        const double2 t = vld<KP>(V[P_T], i, q);
        if (u0 | u1) {
          const double2 xn = fma2(om, sv, fma2(al, p, x));
          vst<KP>(V[P_X], i, q, make_double2(u0 ? xn.x : x.x, u1 ? xn.y : x.y));
        }
        const double2 r = fma2(neg2(om), t, sv);
        vst<KP>(V[P_R], i, q, r);
        dacc(acc[0], r, vld<KP>(V[P_R0], i, q));
      }
    }
    return;
  }
  for (int64_t p0 = r0; p0 < r1; p0 += RPP) {
    const int64_t pe = p0 + RPP < r1 ? p0 + RPP : r1;
    int te0 = 0;
    bool staged = false;
    if constexpr (SPMM && KP <= 2) {
      // stage this pass's CSR entries (coalesced) when they fit
      te0 = __ldg(S.rowptr + p0);
      const int te1 = __ldg(S.rowptr + pe);
      staged = te1 - te0 <= kPersistStage;
      __syncthreads();
      if (staged)
        for (int e = te0 + threadIdx.x; e < te1; e += kPT) {
          sm.u.st.sval[e - te0] = __ldg(S.vals + e);
          sm.u.st.scol[e - te0] = __ldg(S.colidx + e);
        }
      __syncthreads();
    }
    const int64_t i = p0 + rr;
    if (i < pe) {
      if constexpr (PH == PH_PACK) {
        // B and X0 (leading dimension k) into the kp layout, padding columns zero
        const int c0 = 2 * q, k = S.k;
        double bx = 0.0, by = 0.0, xx = 0.0, xy = 0.0;
        if (c0 < k) {
          bx = S.B[i * k + c0];
          if (S.X0) xx = S.X0[i * k + c0];
        }
        if (KP > 1 && c0 + 1 < k) {
          by = S.B[i * k + c0 + 1];
          if (S.X0) xy = S.X0[i * k + c0 + 1];
        }
        vst<KP>(V[P_B], i, q, make_double2(bx, by));
        vst<KP>(V[P_X], i, q, make_double2(xx, xy));
      } else if constexpr (PH == PH_SETUP) {
        // r0 = b - A x0; r^0 = p0 = r0; (b, b), (r0, r0)
        const double2 ax = row_product<KP>(S, V[P_X], i, q, sm, te0, staged);
        const double2 b = vld<KP>(V[P_B], i, q);
        const double2 r = make_double2(b.x - ax.x, b.y - ax.y);
        vst<KP>(V[P_R], i, q, r);
        vst<KP>(V[P_R0], i, q, r);
        vst<KP>(V[P_P], i, q, r);
        dacc(acc[0], b, b);
        dacc(acc[1], r, r);
      } else if constexpr (PH == PH_P1) {
        const double2 v = row_product<KP>(S, V[P_P], i, q, sm, te0, staged);
        vst<KP>(V[P_V], i, q, v);
        dacc(acc[0], v, vld<KP>(V[P_R0], i, q));
      } else if constexpr (PH == PH_P3) {
        const double2 t = row_product<KP>(S, V[P_S], i, q, sm, te0, staged);
        vst<KP>(V[P_T], i, q, t);
        const double2 s = vld<KP>(V[P_S], i, q);
        dacc(acc[0], t, s);
        dacc(acc[1], t, t);
        dacc(acc[2], s, s);
      } else if constexpr (PH == PH_FINAL) {
        // ||b - A x||^2 of the final iterate; X out (ld = k; b = 0 columns give x = 0)
        const double2 ax = row_product<KP>(S, V[P_X], i, q, sm, te0, staged);
        const double2 b = vld<KP>(V[P_B], i, q);
        const double2 r = make_double2(b.x - ax.x, b.y - ax.y);
        dacc(acc[0], r, r);
        const double2 x = vld<KP>(V[P_X], i, q);
        const int c0 = 2 * q, k = S.k;
        if (c0 < k) S.X[i * k + c0] = __ldcg(S.fl + F_XZERO * kMaxKp + c0) ? 0.0 : x.x;
        if (KP > 1 && c0 + 1 < k) S.X[i * k + c0 + 1] = __ldcg(S.fl + F_XZERO * kMaxKp + c0 + 1) ? 0.0 : x.y;
      }
    }
  }
  if constexpr (PH == PH_PACK) {
    // history = NaN (strided over the system's tiles); per-column scalars and flags cleared
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    for (int64_t e = (int64_t)tl * kPT + threadIdx.x; e < S.hist_len; e += (int64_t)S.ntiles * kPT) S.ctl->hist[e] = nan;
    if (tl == 0) {
      for (int t = threadIdx.x; t < S_NSLOT * kMaxKp; t += kPT) S.sc[t] = 0.0;
      for (int t = threadIdx.x; t < F_NFLAG * kMaxKp; t += kPT) S.fl[t] = 0;
    }
  }
}

// The block's dot sums for system si in this phase: one partial per block at `slot` (0 <= slot <
// parts, the blocks that run tiles of si), then the system's last arriving block sums the parts
// partials in slot order and runs the listing's scalar rule.
template <int KP, int PH>
__device__ void flush(const PersistArgs &pa, int si, int slot, int parts, double2 (&acc)[3], Smem &sm) {
  constexpr int ND = PhaseInfo<PH>::ND;
  const PersistSys &S = pa.sys[si];
  tile_partials<KP, ND>(S, slot, acc, sm);
  if (!arrive(pa.tickets + si, parts, sm)) return;
  sys_sum<KP, ND>(S, parts, sm);
  const KArgs a = rule_args(S, KP);
  const int c = threadIdx.x;
  if constexpr (PH == PH_SETUP) {
    if (c < KP) fin_col<FIN_SETUP>(a, c, sm.u.r.res, KP);
  } else if constexpr (PH == PH_P1) {
    if (c < KP) fin_col<FIN_DELTA>(a, c, sm.u.r.res, KP);
  } else if constexpr (PH == PH_P3) {
    if (c < KP) fin_col<FIN_G1>(a, c, sm.u.r.res, KP);
  } else if constexpr (PH == PH_P4) {
    if (c < KP) fin_col<FIN_RHO>(a, c, sm.u.r.res, KP);
  } else if constexpr (PH == PH_FINAL) {
    if (c < KP) fin_col<FIN_TRUE>(a, c, sm.u.r.res, KP);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    pa.tickets[si] = 0u;  // the next phase's arrivals come after a grid barrier
    if constexpr (PH == PH_SETUP || PH == PH_P4) {
      // loop control of this system (the last reducing step of the set-up / of an iteration)
      Ctl *ctl = S.ctl;
      int any = 0;
      for (int cc = 0; cc < KP; ++cc) any |= S.fl[F_ACT * kMaxKp + cc];
      ctl->any_active = any;
      int go;
      if constexpr (PH == PH_SETUP) {
        go = any && ctl->maxit > 0;
        if (go) atomicAdd(&pa.pc->running, 1);
      } else {
        const int j = ctl->iter + 1;
        ctl->iter = j;
        ctl->loop_iters = j;
        go = any && j < ctl->maxit;
        if (!go) atomicSub(&pa.pc->running, 1);
      }
      pa.live[si] = go;
    }
    __threadfence();
  }
}

// Exclusive prefix over the systems of the tiles this phase runs (a system's tiles if it is live,
// or every system's), in shared memory; returns the total.  Every block computes the same.
__device__ int64_t phase_prefix(const PersistArgs &pa, Smem &sm, bool live_only) {
  int carry = 0;
  for (int base = 0; base < pa.nsys; base += kPT) {
    const int si = base + threadIdx.x;
    int v = 0;
    if (si < pa.nsys) v = (!live_only || __ldcg(pa.live + si)) ? pa.sys[si].ntiles : 0;
    // block-wide exclusive scan of v
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) sm.scan_warp[w] = x;
    __syncthreads();
    int before = 0, total = 0;
    for (int ww = 0; ww < kPT / 32; ++ww) {
      const int t = sm.scan_warp[ww];
      if (ww < w) before += t;
      total += t;
    }
    if (si < pa.nsys) sm.pref[si] = carry + before + x - v;
    carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) sm.pref[pa.nsys] = carry;
  __syncthreads();
  return carry;
}

// The system of phase tile t: the last system whose prefix is <= t (systems without tiles in the
// phase have equal consecutive prefixes and are passed over).
__device__ int find_sys(const Smem &sm, int nsys, int64_t t) {
  int lo = 0, hi = nsys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (sm.pref[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int PH>
__device__ void flush_kp(const PersistArgs &pa, int si, int slot, int parts, double2 (&acc)[3], Smem &sm) {
  switch (pa.sys[si].kp) {
    case 1: flush<1, PH>(pa, si, slot, parts, acc, sm); break;
    case 2: flush<2, PH>(pa, si, slot, parts, acc, sm); break;
    case 4: flush<4, PH>(pa, si, slot, parts, acc, sm); break;
    case 8: flush<8, PH>(pa, si, slot, parts, acc, sm); break;
    case 16: flush<16, PH>(pa, si, slot, parts, acc, sm); break;
    case 32: flush<32, PH>(pa, si, slot, parts, acc, sm); break;
    default: flush<64, PH>(pa, si, slot, parts, acc, sm); break;
  }
}

// Block b runs the contiguous chunk [b T / G, (b + 1) T / G) of the phase's T tiles (the live
// systems' tiles in system order), so it meets one or two systems and the chunks stay balanced as
// systems stop.  The blocks that run tiles of a system are consecutive; the block's slot among them
// and their number follow from the chunk bounds (with T < G every tile is its own block).
//
// The prefix is recomputed where the set of systems may have changed since it was last taken: at
// P1 and P5 (the P4 reducers mark stopped systems), and at the set-up and final phases (every
// system).  P2, P3 and P4 reuse P1's: a P4 reducer changes a system's liveness while other blocks
// may still be in P4, and every block must split the same tile list.
template <int PH>
__device__ void run_phase(const PersistArgs &pa, Smem &sm, bool live_only) {
  constexpr int ND = PhaseInfo<PH>::ND;
  constexpr bool RETAKE = !(PH == PH_P2 || PH == PH_P3 || PH == PH_P4);
  const int64_t T = RETAKE ? phase_prefix(pa, sm, live_only) : sm.pref[pa.nsys];
  const int64_t G = gridDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * T / G, t1 = ((int64_t)blockIdx.x + 1) * T / G;
  int cur = -1, slot = 0, parts = 0;
  double2 acc[3] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
  LaneSc ls;
  for (int64_t t = t0; t < t1; ++t) {
    const int si = find_sys(sm, pa.nsys, t);
    const PersistSys &S = pa.sys[si];
    const int64_t L0 = sm.pref[si], L1 = sm.pref[si + 1];
    const int tl = (int)(t - L0);
    if (si != cur) {
      if constexpr (ND > 0) {
        if (cur >= 0) flush_kp<PH>(pa, cur, slot, parts, acc, sm);
#pragma unroll
        for (int d = 0; d < 3; ++d) acc[d] = make_double2(0.0, 0.0);
      }
      cur = si;
      if (T < G) {  // one tile per block
        slot = tl;
        parts = (int)(L1 - L0);
      } else {      // blocks b_first..b_last, b_first = the last block whose chunk starts at or before L0
        const int64_t bf = ((L0 + 1) * G - 1) / T, bl = (L1 * G - 1) / T;
        slot = (int)(blockIdx.x - bf);
        parts = (int)(bl - bf + 1);
      }
      switch (S.kp) {
        case 1: ls = lane_scalars<1, PH>(S); break;
        case 2: ls = lane_scalars<2, PH>(S); break;
        case 4: ls = lane_scalars<4, PH>(S); break;
        case 8: ls = lane_scalars<8, PH>(S); break;
        case 16: ls = lane_scalars<16, PH>(S); break;
        case 32: ls = lane_scalars<32, PH>(S); break;
        default: ls = lane_scalars<64, PH>(S); break;
      }
    }
    switch (S.kp) {
      case 1: run_tile<1, PH>(S, tl, sm, acc, ls); break;
      case 2: run_tile<2, PH>(S, tl, sm, acc, ls); break;
      case 4: run_tile<4, PH>(S, tl, sm, acc, ls); break;
      case 8: run_tile<8, PH>(S, tl, sm, acc, ls); break;
      case 16: run_tile<16, PH>(S, tl, sm, acc, ls); break;
      case 32: run_tile<32, PH>(S, tl, sm, acc, ls); break;
      default: run_tile<64, PH>(S, tl, sm, acc, ls); break;
    }
  }
  if constexpr (ND > 0) {
    if (cur >= 0) flush_kp<PH>(pa, cur, slot, parts, acc, sm);
  }
}

template <int MINB>
__global__ void __launch_bounds__(kPT, MINB) persist_kernel(const PersistArgs pa) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
  if (threadIdx.x == 0) {
    sm.bar_target = 0ull;
    sm.bar_index = 0;
  }
  run_phase<PH_PACK>(pa, sm, false);
  if (!grid_sync(pa, &sm.bar_target, &sm.bar_index, &sm.ok)) return;
  run_phase<PH_SETUP>(pa, sm, false);
  if (!grid_sync(pa, &sm.bar_target, &sm.bar_index, &sm.ok)) return;
  for (int j = 0;; ++j) {
    if (ld_relaxed_i32(&pa.pc->running) == 0) break;
    run_phase<PH_P1>(pa, sm, true);
    if (!grid_sync(pa, &sm.bar_target, &sm.bar_index, &sm.ok)) return;
    run_phase<PH_P2>(pa, sm, true);
    if (!grid_sync(pa, &sm.bar_target, &sm.bar_index, &sm.ok)) return;
    run_phase<PH_P3>(pa, sm, true);
    if (!grid_sync(pa, &sm.bar_target, &sm.bar_index, &sm.ok)) return;
    run_phase<PH_P4>(pa, sm, true);
    if (!grid_sync(pa, &sm.bar_target, &sm.bar_index, &sm.ok)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) pa.pc->iters = j + 1;
    if (ld_relaxed_i32(&pa.pc->running) == 0) break;
    run_phase<PH_P5>(pa, sm, true);
    if (!grid_sync(pa, &sm.bar_target, &sm.bar_index, &sm.ok)) return;
  }
  run_phase<PH_FINAL>(pa, sm, false);
}

template <int MINB>
void *persist_fn() {
  return reinterpret_cast<void *>(persist_kernel<MINB>);
}
void *persist_variant(int minb) { return minb >= 6 ? persist_fn<6>() : persist_fn<4>(); }

cudaError_t set_smem(int minb) {
  const int smem = (int)sizeof(Smem);
  return minb >= 6 ? cudaFuncSetAttribute(persist_kernel<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)
                   : cudaFuncSetAttribute(persist_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

}  // namespace

cudaError_t add_persist_node(cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps, const PersistArgs &pa,
                             int grid, int minb, cudaGraphNode_t *node) {
  const size_t smem = sizeof(Smem);
  cudaError_t e = set_smem(minb);
  if (e != cudaSuccess) return e;
  PersistArgs arg = pa;
  void *params[1] = {&arg};
  cudaKernelNodeParams kp = {};
  kp.func = persist_variant(minb);
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(kPT);
  kp.sharedMemBytes = (unsigned)smem;
  kp.kernelParams = params;
  kp.extra = nullptr;
  if ((e = cudaGraphAddKernelNode(node, g, deps, ndeps, &kp)) != cudaSuccess) return e;
  cudaLaunchAttributeValue v = {};
  v.cooperative = 1;
  return cudaGraphKernelNodeSetAttribute(*node, cudaLaunchAttributeCooperative, &v);
}

int persist_blocks_per_sm(int minb) {
  int nb = 0;
  if (set_smem(minb) != cudaSuccess) return 0;
  const cudaError_t e = minb >= 6
      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, persist_kernel<6>, kPT, sizeof(Smem))
      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, persist_kernel<4>, kPT, sizeof(Smem));
  if (e != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_persist(const PersistArgs &pa, int grid, int minb, cudaStream_t s) {
  const size_t smem = sizeof(Smem);
  cudaError_t e = set_smem(minb);
  if (e != cudaSuccess) return e;
  PersistArgs arg = pa;
  void *params[1] = {&arg};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kPT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, persist_variant(minb), params);
}

}  // namespace bicgk
