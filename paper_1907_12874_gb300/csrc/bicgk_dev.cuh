// Internal declarations shared by the CUDA translation units of libbicgk.
//
// Layout in HBM (Sec. 3.1 of Krasnopolsky, arXiv:1907.12874: the k vectors
// are stored row-wise in a single vector):
//   every Krylov vector is an N x kp block, element (i, c) at i*kp + c, where
//   kp is k rounded up to a power of two (padding columns hold zeros and are
//   finished before the first iteration), so a double2 never straddles rows
//   and every thread of a streaming kernel owns fixed columns.
//   Per-column scalars are SoA arrays [slot][kMaxKp]; per-column flags likewise.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bicgk {

constexpr int kVecThreads = 512;  // threads per block of the streaming kernels
constexpr int kMaxKp = 64;        // largest padded RHS count
constexpr int kMaxDots = 7;       // largest number of dot products fused in one pass (Algorithm 3)
constexpr int kSpmmThreads = 256; // threads per block of the SpMM kernels
constexpr int kSpmmTileRows = 256;      // rows per staged tile (kp <= 2 path)
constexpr int kSpmmStageMax = 4096;     // largest staged tile (CSR entries)
constexpr int kRedGroup = 16;           // blocks per first-level group of the grid reduction
constexpr int kMaxRedGroups = 128;      // group tickets (grids up to 2048 blocks)
constexpr int kPartBlocksPerSm = 8;     // block partials per SM the reduction buffers hold (SpMM grids)

// Per-column FP64 scalar slots.
enum Slot : int {
  S_RHO = 0, S_ALPHA, S_OMEGA, S_BETA, S_EPS2, S_BN2, S_D0, S_D1, S_D2, S_TRUE,
  // Algorithm 3 (Improved BiCGStab): stored dots of the basic form and the recurrence state
  S_D3, S_D4, S_D5, S_SIGMA, S_SIGP, S_PI, S_TAU, S_PHI, S_AOLD, S_CZ, S_CV, S_DLT,
  S_NSLOT
};
// Per-column int flags.
enum Flag : int { F_ACT = 0, F_XUPD, F_XZERO, F_ITERS, F_STATUS, F_NFLAG };

// Status codes (same values as the public enum).
enum Status : int { ST_CONVERGED = 0, ST_MAXIT = 1, ST_BREAKDOWN = 2, ST_NONFINITE = 3 };

// Device-resident control block.  Written by the host before each solve and
// by the last block of the reducing kernels during it.
struct Ctl {
  double tol;
  double *hist;   // [(maxit+1)][kp] residual-norm history
  int iter;       // current iteration j
  int maxit;
  int k;          // real columns
  int kp;         // padded columns
  int flags;      // bicgk_flags
  int any_active; // some column still iterating
  int loop_iters; // iterations the loop completed
  int compact_req; // the loop stopped to narrow the layout (at most kp/2 columns still active)
  int level;      // layout level of the column compaction (-1 once the final values are out)
  int mode;       // action of the current compaction boundary: 0 none, 1 narrow, 2 final
  unsigned int ticket; // arrival counter of the grid reduction's second level (reset by its last block)
  unsigned int gticket[kMaxRedGroups]; // arrival counters of the first level, one per group of blocks
};

// Vector roles in the workspace.
// Algorithm 5 keeps p^ in V_Q and s^ in V_Y; Algorithm 7 keeps p^ in V_P and q^ in V_RT plus the
// four hatted roles below; Algorithm 3 keeps u in V_W and f_0 = A^T r_0 in V_RT.
enum Vec : int {
  V_X = 0, V_R, V_R0, V_P, V_V, V_S, V_T, V_W, V_Z, V_Q, V_Y, V_TMP, V_RT, V_B, V_SH, V_ZH, V_RH, V_WH, V_NVEC
};

struct KArgs {
  double *v[V_NVEC];
  double *sc;    // [S_NSLOT][kMaxKp]
  int *fl;       // [F_NFLAG][kMaxKp]
  double *part;  // [grid + groups][kMaxDots][kMaxKp]: per-block partial sums, then per-group sums
  Ctl *ctl;
  int64_t n;     // rows
  int kp;
  int use_cond;  // 1 inside the captured graph (the loop is a conditional WHILE node)
  cudaGraphConditionalHandle cond;
  const int *ext_act;  // inner solves of the refinement: columns the outer loop still iterates
  const double *invdiag;  // Jacobi preconditioner 1/a_ii per row (nullptr: M = identity, a copy)
  // column compaction: the solve's column of each layout column (nullptr: the same; -1: padding),
  // the history's row length, and whether the loop may stop to narrow the layout
  const int *cmap;
  int kp_out;
  int compact;
};

// Streaming kernel identifiers (one per fused vector operation of the listings).
enum Op : int {
  // set-up
  OP_SETUP_C = 0, OP_SETUP_R, OP_SETUP_P, OP_DOT_RW0,
  // classical (Algorithms 1 and 2)
  OP_DELTA, OP_UPD_S, OP_G1, OP_G3, OP_UPD_P,
  OP_DOT_TS, OP_DOT_PSI, OP_UPD_X_C, OP_UPD_R_C, OP_DOT_RR, OP_DOT_RHO,
  // reordered (Algorithm 6, M^-1 = copy)
  OP_COPY_SV, OP_UPD_TH, OP_RG4, OP_COPY_QT, OP_UPD_R_R, OP_RFIN,
  OP_UPD_RT, OP_DOT_T_RT, OP_DOT_T_T, OP_DOT_T_R0, OP_DOT_RT_RT, OP_UPD_X_R, OP_UPD_Z_R, OP_UPD_VH,
  // pipelined (Algorithm 4)
  OP_PG1, OP_PG2, OP_PG3,
  OP_PU_P, OP_PU_S, OP_PU_Z, OP_PU_Q, OP_PU_Y, OP_DOT_QY, OP_DOT_YY, OP_DOT_QQ,
  OP_PU_X, OP_PU_R, OP_PU_TMP, OP_PU_W, OP_DOT_R0R, OP_DOT_R0Z, OP_DOT_R0W, OP_DOT_R0S,
  // final true residual norm
  OP_TRUE_RES,
  // mixed-precision refinement: FP32 inner solve (merged classical BiCGStab, Algorithm 2)
  OP32_SETUP, OP32_DELTA, OP32_UPD_S, OP32_G1, OP32_G3, OP32_UPD_P,
  // mixed-precision refinement: FP64 outer steps (V_Q / V_Y point to the FP32 b and d blocks)
  OP_IR_SETUP, OP_IR_RESID, OP_IR_UPDATE,
  // preconditioner applications y = M^-1 x (identity copy or Jacobi)
  OP_PREC_P_Q, OP_PREC_S_Y, OP_PREC_R_RH, OP_PREC_W_WH, OP_PREC_Z_ZH, OP_PREC_R_Z, OP_PREC_V_S, OP_PREC_T_Q,
  // Algorithm 5 (preconditioned BiCGStab)
  OP5_RRHO, OP5_UPD_X,
  // Algorithm 7 (preconditioned Pipelined BiCGStab)
  OP7_SETUP, OP7_L1, OP7_L2, OP7_L4, OP7_L5, OP7_PU_PH, OP7_PU_SH, OP7_PU_QH, OP7_X, OP7_TMPH, OP7_RH,
  // Algorithm 3 (Improved BiCGStab)
  OP3_SETUP, OP3_SIG0, OP3_L1, OP3_L2, OP3_L3, OP3_Z, OP3_V, OP3_S, OP3_T, OP3_D_R0S, OP3_D_R0Q, OP3_D_F0S,
  OP3_D_F0T, OP3_D_ST, OP3_D_TT, OP3_D_SS, OP3_X,
  // Algorithms 2 and 5 with theta = (s, s) taken where s is formed: the s update with that dot,
  // and group 1 reduced to phi = (t, s), psi = (t, t)
  OP_UPD_S_TH, OP_G1_PP,
  OP_COUNT
};

const char *op_name(int op);
// Reads and writes of full N x k vectors one launch of `op` makes (for traffic accounting).
void op_traffic(int op, int *reads, int *writes);
int op_has_dots(int op);

// Launch one streaming kernel.  grid must not exceed the partial-sum capacity.
cudaError_t launch_vec(int op, const KArgs &a, int grid, cudaStream_t s);
// Blocks per SM the streaming kernel of `op` reaches (occupancy query).
int vec_blocks_per_sm(int op);

// Staged-tile helpers of the one-lane-per-row products (kp <= 2).
//
// stage_entries: entries [te0, te1) of a row tile into shared memory.  Each thread issues the
// loads of up to kStageUnroll entries before it stores any of them, so a tile costs one DRAM
// latency per round of blockDim.x * kStageUnroll entries instead of one per blockDim.x entries.
constexpr int kStageUnroll = 4;
template <typename T>
__device__ __forceinline__ void stage_entries(const int32_t *__restrict__ ci, const T *__restrict__ va, int te0,
                                              int te1, T *s_val, int32_t *s_col) {
  const int nt = (int)blockDim.x;
  for (int e = te0 + (int)threadIdx.x; e < te1; e += nt * kStageUnroll) {
    T v[kStageUnroll];
    int32_t c[kStageUnroll];
#pragma unroll
    for (int u = 0; u < kStageUnroll; ++u) {
      const int q = e + u * nt;
      if (q < te1) {
        v[u] = __ldg(va + q);
        c[u] = __ldg(ci + q);
      }
    }
#pragma unroll
    for (int u = 0; u < kStageUnroll; ++u) {
      const int q = e + u * nt;
      if (q < te1) {
        s_val[q - te0] = v[u];
        s_col[q - te0] = c[u];
      }
    }
  }
}

// One row's sum over staged entries [q0, q1) (tile-relative), four x gathers in flight, the FMAs
// in entry order (the sum of the entry-by-entry loop).  X: T (kp = 1) or its two-wide vector
// (kp = 2); the result has X's type.
template <typename T>
__device__ __forceinline__ T staged_row(const T *s_val, const int32_t *s_col, const T *__restrict__ xs, int q0,
                                        int q1) {
  T y = 0;
  int q = q0;
  for (; q + 3 < q1; q += 4) {
    T a[4], u[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      a[j] = s_val[q + j];
      u[j] = __ldg(xs + s_col[q + j]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) y = fma(a[j], u[j], y);
  }
  for (; q < q1; ++q) y = fma(s_val[q], __ldg(xs + s_col[q]), y);
  return y;
}
template <typename T, typename T2>
__device__ __forceinline__ T2 staged_row2(const T *s_val, const int32_t *s_col, const T2 *__restrict__ x2, int q0,
                                          int q1) {
  T2 y;
  y.x = 0;
  y.y = 0;
  for (int q = q0; q < q1; ++q) {
    const T a = s_val[q];
    const T2 u = __ldg(x2 + s_col[q]);
    y.x = fma(a, u.x, y.x);
    y.y = fma(a, u.y, y.y);
  }
  return y;
}

// SpMM: y = A x (mode 0) or y = b - A x (mode 1) for kp in {1,2,4,...,64}.
// vals, x, y, b point to double (launch_spmm) or float (launch_spmm32) arrays.
struct SpmmArgs {
  const int32_t *rowptr;
  const int32_t *colidx;
  const void *vals;
  const void *x;
  void *y;
  const void *b;
  int64_t n;
  int stage_cap;  // staged CSR entries per tile (kp <= 2); 0 = read entries directly
  int cols_per_lane = 2;  // RHS-tile width of a lane (kp >= 8 also accepts 4)
  int fp32_kernel = 0;    // FP32, kp >= 16: 0 the sweep kernel, 1 the segment kernel
  int warp_rows = 0;      // kp <= 2: 1 the warp-tile kernel (short rows), 0 the block-tile kernel
};
cudaError_t launch_spmm(int kp, int mode, const SpmmArgs &a, int grid, cudaStream_t s);

// One lane per row (kp <= 2) in warp tiles, for matrices with short rows (at most 8 entries on
// average, e.g. the 7-point stencils); the row loop of spmm_warp_kernel and of the fused product
// with a dot epilogue.  The block-tile kernel stages a 256-row tile per block between two block
// barriers, so a block waits for the tile's CSR entries (DRAM) and then for its x gathers, one
// after the other.  Here every warp owns tiles of 32 consecutive rows and runs a two-stage
// prefetch: while it multiplies tile t, the CSR entries of tile t+1 (whose row pointers arrived
// during tile t-1) and the row pointers of tile t+2 are in flight in registers; at the start of a
// tile they move to the warp's shared-memory slice (sv, sc: kWarpCap entries), from which each
// lane reads its row's entries.  The entries, read once, are streamed past L1 (evict-first), which
// keeps L1 for the x rows that neighbouring rows share (128^3 7-point, k = 1: 43.0 against 47.5 us
// with read-only loads).  Blocks sweep contiguous row ranges (range b of gridDim.x equal parts),
// warps taking consecutive tiles.  Each row is summed in CSR order (bitwise the block-tile
// kernel's sums); a tile with more than kWarpCap entries reads its entries from global memory.
// fn(row, y) is called for every row of the range, y of type T (kp = 1) or its two-wide vector.
constexpr int kWarpCap = 256;             // staged entries per 32-row warp tile
constexpr int kWarpMW = kWarpCap / 32;    // prefetch registers per lane (entries)

template <typename T>
struct Wide2;
template <>
struct Wide2<double> {
  using type = double2;
};
template <>
struct Wide2<float> {
  using type = float2;
};

template <typename T, int KP, class Fn>
__device__ __forceinline__ void warp_tile_rows(const SpmmArgs &a, T *sv, int32_t *sc, Fn fn) {
  static_assert(KP == 1 || KP == 2, "warp tiles: kp <= 2");
  using T2 = typename Wide2<T>::type;
  constexpr int NW = kSpmmThreads / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int32_t *__restrict__ rp = a.rowptr;
  const int32_t *__restrict__ ci = a.colidx;
  const T *__restrict__ va = static_cast<const T *>(a.vals);
  const int64_t rb0 = a.n * blockIdx.x / gridDim.x, rb1 = a.n * (blockIdx.x + 1) / gridDim.x;
  constexpr int64_t step = (int64_t)32 * NW;
  int64_t r = rb0 + (int64_t)32 * w;
  if (r >= rb1) return;  // no tile for this warp
  // lane l holds the row pointer of row r + l, and of row r + 32 (clipped to the range's end: rows
  // past it are empty), for the current tile and the next
  auto rp_at = [&](int64_t i) { return __ldg(rp + (i < rb1 ? i : rb1)); };
  int lo = rp_at(r + lane), hi = rp_at(r + 32);
  int lo_n = 0, hi_n = 0;
  if (r + step < rb1) {
    lo_n = rp_at(r + step + lane);
    hi_n = rp_at(r + step + 32);
  }
  int cn[kWarpMW];
  T vn[kWarpMW];
  {
    const int e0 = __shfl_sync(0xffffffffu, lo, 0), cnt = hi - e0;
#pragma unroll
    for (int m = 0; m < kWarpMW; ++m) {
      const int q = m * 32 + lane;
      cn[m] = 0;
      vn[m] = 0;
      if (cnt <= kWarpCap && q < cnt) {
        cn[m] = __ldcs(ci + e0 + q);
        vn[m] = __ldcs(va + e0 + q);
      }
    }
  }
  for (;;) {
    const int e0 = __shfl_sync(0xffffffffu, lo, 0);
    const int cnt = hi - e0;
    const bool staged = cnt <= kWarpCap;
    if (staged) {
#pragma unroll
      for (int m = 0; m < kWarpMW; ++m) {
        const int q = m * 32 + lane;
        if (q < cnt) {
          sc[q] = cn[m];
          sv[q] = vn[m];
        }
      }
    }
    __syncwarp();
    // prefetch: the entries of the next tile, the row pointers of the one after
    const int64_t rn = r + step;
    int lo_nn = 0, hi_nn = 0;
    if (rn < rb1) {
      const int f0 = __shfl_sync(0xffffffffu, lo_n, 0), cntn = hi_n - f0;
      if (cntn <= kWarpCap) {
#pragma unroll
        for (int m = 0; m < kWarpMW; ++m) {
          const int q = m * 32 + lane;
          if (q < cntn) {
            cn[m] = __ldcs(ci + f0 + q);
            vn[m] = __ldcs(va + f0 + q);
          }
        }
      }
      if (rn + step < rb1) {
        lo_nn = rp_at(rn + step + lane);
        hi_nn = rp_at(rn + step + 32);
      }
    }
    // this lane's row: entries [lo, next lane's lo) (lane 31: up to hi)
    const int up = __shfl_down_sync(0xffffffffu, lo, 1);
    const int re = lane == 31 ? hi : up;
    const int64_t row = r + lane;
    if (row < rb1) {
      if constexpr (KP == 1) {
        const T *__restrict__ xs = static_cast<const T *>(a.x);
        T y;
        if (staged) {
          y = staged_row<T>(sv, sc, xs, lo - e0, re - e0);
        } else {
          y = 0;
          for (int e = lo; e < re; ++e) y = fma(__ldg(va + e), __ldg(xs + __ldg(ci + e)), y);
        }
        fn(row, y);
      } else {
        const T2 *__restrict__ x2 = static_cast<const T2 *>(a.x);
        T2 y;
        if (staged) {
          y = staged_row2<T, T2>(sv, sc, x2, lo - e0, re - e0);
        } else {
          y.x = 0;
          y.y = 0;
          for (int e = lo; e < re; ++e) {
            const T av = __ldg(va + e);
            const T2 u = __ldg(x2 + __ldg(ci + e));
            y.x = fma(av, u.x, y.x);
            y.y = fma(av, u.y, y.y);
          }
        }
        fn(row, y);
      }
    }
    __syncwarp();
    if (rn >= rb1) break;
    r = rn;
    lo = lo_n;
    hi = hi_n;
    lo_n = lo_nn;
    hi_n = hi_nn;
  }
}
int spmm_blocks_per_sm(int kp, int mode, int stage_cap, int warp_rows = 0);
// y = A x with the dots of the next listing step taken in the product's epilogue (FP64), then
// the grid reduction and that step's scalar rule, as the separate dot kernel would do them.
enum SpmmEpi : int {
  EPI_DELTA = 0,  // delta = (v, r^0) after v = A p: the dot kernel OP_DELTA
  EPI_G1 = 1,     // (t, s), (t, t), (s, s) after t = A s: group 1 of Algorithm 2 (OP_G1)
  EPI_G1_PP = 2,  // (t, s), (t, t) after t = A s, theta from OP_UPD_S_TH (OP_G1_PP)
};
cudaError_t launch_spmm_dot(int kp, int epi, const SpmmArgs &s, const KArgs &a, int grid, cudaStream_t st);
int spmm_dot_blocks_per_sm(int kp, int epi, int stage_cap, int warp_rows = 0);  // occupancy of the fused kernel
const char *spmm_dot_name(int epi);
// y = A^T x (ld = k) by an atomic scatter over the rows of A.
cudaError_t launch_spmm_t_atomic(const int32_t *rowptr, const int32_t *colidx, const double *vals, const double *x,
                                 double *y, int64_t n, int k, cudaStream_t s);
// g_e = alpha * sum_c l_ic x_jc over the entries e = (i, j) of A (ld = k).
cudaError_t launch_sddmm(const int32_t *rowptr, const int32_t *colidx, const double *l, const double *x, double alpha,
                         double *g, int64_t n, int k, cudaStream_t s);
// FP32 y = A x (values, x and y float; one FP32 FMA per nonzero and column).
cudaError_t launch_spmm32(int kp, const SpmmArgs &a, int grid, cudaStream_t s);
int spmm32_blocks_per_sm(int kp, int stage_cap, int fp32_kernel, int warp_rows = 0);

// Pack columns [0, ncols) of a caller block with leading dimension ld into the workspace layout
// (ld = kp, zero padding); X0 may be null.
cudaError_t launch_pack(const double *B, const double *X0, int ld, int ncols, const KArgs &a, cudaStream_t s);
// Unpack workspace role `role` (ld = kp) into columns [0, ncols) of a caller block with leading
// dimension ld; with use_xzero, columns with b_c = 0 are written as zeros.
cudaError_t launch_unpack_role(double *X, int ld, int ncols, const KArgs &a, int role, int use_xzero,
                               cudaStream_t s);
// Caller blocks of one batched system, read by the kernels through a device pointer so a
// captured graph serves every call (the host rewrites the table before each launch).
struct BatchIO {
  const double *B;
  const double *X0;  // nullable
  double *X;
};
// pack / unpack through a BatchIO entry (ld = ncols = the system's k)
cudaError_t launch_pack_io(const BatchIO *io, int k, const KArgs &a, cudaStream_t s);
cudaError_t launch_unpack_io(const BatchIO *io, int k, const KArgs &a, cudaStream_t s);
// dst = (float)src elementwise.
cudaError_t launch_to_float(const double *src, float *dst, int64_t n, cudaStream_t s);
// Jacobi preconditioner: invdiag[i] = 1 / (sum of the row's diagonal entries), 1 where that is 0.
cudaError_t launch_invdiag(const int32_t *rowptr, const int32_t *colidx, const double *vals, double *invdiag,
                           int64_t n, cudaStream_t s);
// Fill the history with NaN and clear the per-column state.
cudaError_t launch_reset(const KArgs &a, int64_t hist_len, cudaStream_t s);
// Column compaction boundary `boundary` (1..L+1) between layout level boundary-1 (src) and
// boundary (dst, half as many columns; unused when `last`).  The plan kernel decides from the
// control block (narrow, write the final values, or nothing), moves the per-column scalars and
// flags of the columns that leave to fin_sc / fin_fl (indexed by the solve's column), compacts
// the rest, writes dst's column map to cmap_out and the kept source columns to act, and sets the
// next level's loop condition.  The move kernel writes the x of the columns that leave to xf
// (kp_out layout) and gathers the roles in live_mask (bit r for role r: the vectors an iteration
// reads before writing them) of the kept ones into dst's slots; at an odd length it zeroes the
// padding element of dst's roles in loop_mask.
cudaError_t launch_compact(const KArgs &src, const KArgs &dst, int boundary, int last,
                           cudaGraphConditionalHandle next, double *fin_sc, int *fin_fl, int *cmap_out,
                           int *act, double *xf, unsigned live_mask, unsigned loop_mask, int grid,
                           cudaStream_t s);
// In-place compaction of `role` at the same boundary (after launch_compact): the kept columns of
// src's layout into dst's narrower one in the same vector, through `scratch` (n_rows*dst.kp
// doubles).  Does nothing unless the boundary narrows.
cudaError_t launch_compact_inplace(const KArgs &src, const KArgs &dst, const int *act, int role, double *scratch,
                                   int grid, cudaStream_t s);

}  // namespace bicgk
