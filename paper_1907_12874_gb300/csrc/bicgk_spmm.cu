// CSR sparse matrix times a block of k RHS-interleaved vectors, FP64 (and FP32 for the inner
// solves of the mixed-precision refinement):
//   y_ic = sum_j a_ij x_jc           (mode 0: the SpMV of Algorithms 1-6)
//   y_ic = b_ic - sum_j a_ij x_jc    (mode 1: r_0 = b - A x_0 and the final
//                                     true residual)
// The operation whose traffic the paper models as Sigma_mul (Sec. 3.1, Eq.
// SpMV_mem): CRS with 4-byte indices and 8-byte values, k vectors stored
// row-wise.
//
// FP64 arithmetic is the scarce resource on this GPU (two FP64 lanes per SM
// per clock), so every lane computes complete row sums for the two columns it
// owns: no partial sums are combined across lanes, and each (nonzero, column)
// pair costs exactly one FMA.
//
//   kp >= 4: a row is owned by kp/2 consecutive lanes, lane l of the group
//            holding columns 2l, 2l+1; the x row and the y row move as one
//            coalesced run of kp doubles (double2 per lane).  The group's CSR
//            entries are broadcast loads through L1.
//   kp <= 2: one lane per row, the row's CSR entries read from shared memory
//            (coalesced staging, so the lanes' strided reads of their own rows
//            do not scatter over L1).  Two kernels: the warp-tile kernel (short
//            rows: each warp prefetches the entries of its next 32-row tile into
//            registers while it multiplies the current one) and the block-tile
//            kernel (a block stages 256-row tiles between two barriers, each
//            thread's loads of a round issued before its stores; each lane then
//            keeps four x gathers in flight).  A tile with more entries than the
//            staging holds reads them from global.
#include <type_traits>

#include "bicgk_dev.cuh"

namespace bicgk {

namespace {

// Element type T (double: the FP64 path; float: the FP32 inner solves of the mixed-precision
// refinement) and its two-wide vector type.
template <typename T>
struct Vec2;
template <>
struct Vec2<double> {
  using type = double2;
  __device__ static type make(double x, double y) { return make_double2(x, y); }
};
template <>
struct Vec2<float> {
  using type = float2;
  __device__ static type make(float x, float y) { return make_float2(x, y); }
};

template <typename T, int KP, int MODE, int CPL>
__global__ void __launch_bounds__(kSpmmThreads) spmm_group_kernel(const SpmmArgs a) {
  static_assert(KP >= 4 && KP >= CPL && (CPL == 2 || CPL == 4), "group kernel: kp >= 4, 2 or 4 columns per lane");
  using T2 = typename Vec2<T>::type;
  constexpr int L = KP / CPL;                 // lanes per row
  constexpr int H = CPL / 2;                  // two-wide vectors per lane
  constexpr int RPP = kSpmmThreads / L;       // rows per pass of a block
  const int g = threadIdx.x / L, cl = threadIdx.x % L;
  const int32_t *__restrict__ rp = a.rowptr;
  const int32_t *__restrict__ ci = a.colidx;
  const T *__restrict__ va = static_cast<const T *>(a.vals);
  const T2 *__restrict__ x2 = static_cast<const T2 *>(a.x);
  T2 *__restrict__ y2 = static_cast<T2 *>(a.y);
  const int64_t stride = (int64_t)gridDim.x * RPP;
  for (int64_t r = (int64_t)blockIdx.x * RPP + g; r < a.n; r += stride) {
    const int e0 = __ldg(rp + r), e1 = __ldg(rp + r + 1);
    T2 acc[H];
#pragma unroll
    for (int h = 0; h < H; ++h) acc[h] = Vec2<T>::make(0, 0);
    // FP32: four nonzeros per step.  Their column indices, values and x rows are all loaded
    // before the first FMA (memory-level parallelism for the gathers); the FMAs then run in entry
    // order, so the sum is the one of a loop over single entries.  The FP64 kernel is bound by its
    // FMA pipe instead, and the extra registers spill there.
    int e = e0;
    if constexpr (sizeof(T) == 4) {
      for (; e + 3 < e1; e += 4) {
        int j[4];
        T av[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          j[q] = __ldg(ci + e + q);
          av[q] = __ldg(va + e + q);
        }
        T2 u[4][H];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int h = 0; h < H; ++h) u[q][h] = __ldg(x2 + (int64_t)j[q] * (KP / 2) + cl * H + h);
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int h = 0; h < H; ++h) {
            acc[h].x = fma(av[q], u[q][h].x, acc[h].x);
            acc[h].y = fma(av[q], u[q][h].y, acc[h].y);
          }
      }
    }
    for (; e + 1 < e1; e += 2) {
      const int j0 = __ldg(ci + e), j1 = __ldg(ci + e + 1);
      const T a0 = __ldg(va + e), a1 = __ldg(va + e + 1);
      T2 u0[H], u1[H];
#pragma unroll
      for (int h = 0; h < H; ++h) {
        u0[h] = __ldg(x2 + (int64_t)j0 * (KP / 2) + cl * H + h);
        u1[h] = __ldg(x2 + (int64_t)j1 * (KP / 2) + cl * H + h);
      }
#pragma unroll
      for (int h = 0; h < H; ++h) {
        acc[h].x = fma(a0, u0[h].x, acc[h].x);
        acc[h].y = fma(a0, u0[h].y, acc[h].y);
        acc[h].x = fma(a1, u1[h].x, acc[h].x);
        acc[h].y = fma(a1, u1[h].y, acc[h].y);
      }
    }
    if (e < e1) {
      const int j0 = __ldg(ci + e);
      const T a0 = __ldg(va + e);
#pragma unroll
      for (int h = 0; h < H; ++h) {
        const T2 u0 = __ldg(x2 + (int64_t)j0 * (KP / 2) + cl * H + h);
        acc[h].x = fma(a0, u0.x, acc[h].x);
        acc[h].y = fma(a0, u0.y, acc[h].y);
      }
    }
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const int64_t o = r * (KP / 2) + cl * H + h;
      if constexpr (MODE == 1) {
        const T2 bv = static_cast<const T2 *>(a.b)[o];
        acc[h] = Vec2<T>::make(bv.x - acc[h].x, bv.y - acc[h].y);
      }
      y2[o] = acc[h];
    }
  }
}

// One lane per row, CSR entries of each 256-row tile staged in shared memory.
template <typename T, int KP, int MODE>
__global__ void __launch_bounds__(kSpmmThreads) spmm_row_kernel(const SpmmArgs a) {
  static_assert(KP == 1 || KP == 2, "row kernel handles kp <= 2");
  using T2 = typename Vec2<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int cap = a.stage_cap;
  T *s_val = reinterpret_cast<T *>(smem_raw);
  int32_t *s_col = reinterpret_cast<int32_t *>(s_val + cap);
  const int32_t *__restrict__ rp = a.rowptr;
  const int32_t *__restrict__ ci = a.colidx;
  const T *__restrict__ va = static_cast<const T *>(a.vals);
  const T *__restrict__ xs = static_cast<const T *>(a.x);
  const int64_t ntiles = (a.n + kSpmmTileRows - 1) / kSpmmTileRows;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t r0 = t * kSpmmTileRows;
    const int64_t r1 = (r0 + kSpmmTileRows < a.n) ? r0 + kSpmmTileRows : a.n;
    const int te0 = __ldg(rp + r0), te1 = __ldg(rp + r1);
    const bool staged = (te1 - te0) <= cap;
    if (staged) stage_entries<T>(ci, va, te0, te1, s_val, s_col);
    __syncthreads();
    const int64_t r = r0 + threadIdx.x;
    if (r < r1) {
      const int e0 = __ldg(rp + r), e1 = __ldg(rp + r + 1);
      if constexpr (KP == 1) {
        T acc = 0;
        if (staged)
          acc = staged_row<T>(s_val, s_col, xs, e0 - te0, e1 - te0);
        else
          for (int e = e0; e < e1; ++e) acc = fma(__ldg(va + e), __ldg(xs + __ldg(ci + e)), acc);
        if constexpr (MODE == 1) acc = static_cast<const T *>(a.b)[r] - acc;
        static_cast<T *>(a.y)[r] = acc;
      } else {
        const T2 *__restrict__ x2 = static_cast<const T2 *>(a.x);
        T2 acc = Vec2<T>::make(0, 0);
        if (staged) {
          acc = staged_row2<T, T2>(s_val, s_col, x2, e0 - te0, e1 - te0);
        } else {
          for (int e = e0; e < e1; ++e) {
            const T av = __ldg(va + e);
            const T2 u = __ldg(x2 + __ldg(ci + e));
            acc.x = fma(av, u.x, acc.x);
            acc.y = fma(av, u.y, acc.y);
          }
        }
        if constexpr (MODE == 1) {
          const T2 bv = static_cast<const T2 *>(a.b)[r];
          acc = Vec2<T>::make(bv.x - acc.x, bv.y - acc.y);
        }
        static_cast<T2 *>(a.y)[r] = acc;
      }
    }
    __syncthreads();
  }
}

// One lane per row (kp <= 2), warp tiles, for matrices with short rows: warp_tile_rows
// (bicgk_dev.cuh) with the product stored (mode 0) or subtracted from b (mode 1).
template <typename T, int KP, int MODE>
__global__ void __launch_bounds__(kSpmmThreads) spmm_warp_kernel(const SpmmArgs a) {
  static_assert(KP == 1 || KP == 2, "warp kernel handles kp <= 2");
  using T2 = typename Vec2<T>::type;
  __shared__ T s_val[kSpmmThreads / 32][kWarpCap];
  __shared__ int32_t s_col[kSpmmThreads / 32][kWarpCap];
  const int w = threadIdx.x >> 5;
  warp_tile_rows<T, KP>(a, s_val[w], s_col[w], [&](int64_t row, auto y) {
    if constexpr (KP == 1) {
      if constexpr (MODE == 1) y = static_cast<const T *>(a.b)[row] - y;
      static_cast<T *>(a.y)[row] = y;
    } else {
      if constexpr (MODE == 1) {
        const T2 bv = static_cast<const T2 *>(a.b)[row];
        y = Vec2<T>::make(bv.x - y.x, bv.y - y.y);
      }
      static_cast<T2 *>(a.y)[row] = y;
    }
  });
}

// FP32, kp >= 8 (the inner solves of the mixed-precision refinement).  The FP32 product is
// bound by the L1 data path, not by FMAs: in the group kernel every lane of a row re-reads the
// row's column index and value for each nonzero as a broadcast load, which costs the L1 about
// as much as the x row itself.  Here a row is owned by L = kp/4 lanes with 4 columns each (one
// 16-byte load of the x row per nonzero); the row's CSR entries are read C at a time with one
// coalesced load per lane and passed to the row's lanes by shuffles, so the L1 carries the x
// rows and one load per lane per chunk.  The gathers of a chunk (up to 8 in flight) are issued
// before its FMAs; the FMAs run in entry order, so every sum is the one of the entry-by-entry
// loop.
template <int KP>
__global__ void __launch_bounds__(kSpmmThreads) spmm32_seg_kernel(const SpmmArgs a) {
  static_assert(KP >= 8 && KP <= 64, "segment kernel: 8 <= kp <= 64");
  constexpr int L = KP / 4;           // lanes per row
  constexpr int C = L > 8 ? L : 8;    // CSR entries per chunk
  constexpr int M = C / L;            // entries each lane loads per chunk
  constexpr int G = 8;                // gathers in flight
  constexpr int RPP = kSpmmThreads / L;
  const int lane = threadIdx.x & 31;
  const int g = threadIdx.x / L, cl = threadIdx.x % L;
  const unsigned segmask = L == 32 ? 0xffffffffu : (((1u << L) - 1u) << (lane & ~(L - 1)));
  const int32_t *__restrict__ rp = a.rowptr;
  const int32_t *__restrict__ ci = a.colidx;
  const float *__restrict__ va = static_cast<const float *>(a.vals);
  const float4 *__restrict__ x4 = static_cast<const float4 *>(a.x);
  float4 *__restrict__ y4 = static_cast<float4 *>(a.y);
  const int64_t stride = (int64_t)gridDim.x * RPP;
  for (int64_t r = (int64_t)blockIdx.x * RPP + g; r < a.n; r += stride) {
    const int e0 = __ldg(rp + r), e1 = __ldg(rp + r + 1);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int base = e0; base < e1; base += C) {
      const int cnt = (e1 - base < C) ? e1 - base : C;
      // entry q of the chunk is held by lane q % L in slot q / L
      int jj[M];
      float aa[M];
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const int q = m * L + cl;
        jj[m] = 0;
        aa[m] = 0.f;
        if (q < cnt) {
          jj[m] = __ldg(ci + base + q);
          aa[m] = __ldg(va + base + q);
        }
      }
#pragma unroll
      for (int h = 0; h < C; h += G) {
        float4 u[G];
        float av[G];
#pragma unroll
        for (int t = 0; t < G; ++t) {
          const int q = h + t;
          const int j = __shfl_sync(segmask, jj[q / L], q % L, L);
          av[t] = __shfl_sync(segmask, aa[q / L], q % L, L);
          u[t] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (q < cnt) u[t] = __ldg(x4 + (int64_t)j * (KP / 4) + cl);
        }
#pragma unroll
        for (int t = 0; t < G; ++t) {
          if (h + t < cnt) {
            acc.x = fmaf(av[t], u[t].x, acc.x);
            acc.y = fmaf(av[t], u[t].y, acc.y);
            acc.z = fmaf(av[t], u[t].z, acc.z);
            acc.w = fmaf(av[t], u[t].w, acc.w);
          }
        }
      }
    }
    y4[r * (KP / 4) + cl] = acc;
  }
}

// FP32, kp = 16, 32, 64: the sweep kernel.  The segment kernel above waits, for every chunk of a
// row, for the chunk's CSR entries to come from DRAM before it can issue the chunk's gathers, and
// its blocks stride over the whole matrix, so the x rows one SM gathers are reused in its L1 only
// within one 32-row tile (hit rate about 60 % on the 27-point operator).  Here
//   * every block sweeps one contiguous range of rows (range b of gridDim.x equal parts), its
//     warps taking consecutive R-row tiles, so the x rows of the neighbouring grid lines stay in
//     the SM's L1 while the sweep passes them (on a 3-D stencil all but the rows of the next line
//     of the three planes are hits);
//   * a warp owns its tiles and runs a two-stage prefetch: while it multiplies tile t, the CSR
//     entries of tile t+1 (whose row pointers arrived during tile t-1) and the row pointers of
//     tile t+2 are in flight, so the DRAM latency of the matrix stream is hidden behind the
//     gathers;
//   * a tile's entries move from the prefetch registers to the warp's shared-memory slice as
//     (column, value) pairs: one 8-byte broadcast read per nonzero serves all L lanes of a row.
// A row is owned by L = kp/4 lanes with 4 columns each (one 16-byte x load per nonzero, the
// warp's load covering R = 32/L rows); G gathers are in flight per lane, then their FMAs run in
// entry order, so every sum is bitwise the one of the entry-by-entry loop (and of the segment
// kernel).  A tile with more than CAP entries reads its entries from global memory instead.
// Measured (ncu, 27-point 96^3, kp = 32): the L1 hit rate rises from 59 to 69 % and the L1 data
// pipe, the limit of both kernels, stays about 70 % busy; 1.1-1.2x faster than the segment kernel
// at kp = 16, 32 and 64.
template <int KP, int THREADS>
struct SweepGeo {
  static constexpr int L = KP / 4;                     // lanes per row
  static constexpr int R = 32 / L;                     // rows per warp tile
  static constexpr int CAP = 32 * R > 128 ? 32 * R : 128;  // staged entries per warp tile
  static constexpr int MW = CAP / 32;                  // prefetch registers per lane (pairs)
  static constexpr int NW = THREADS / 32;              // warps per block
};

template <int KP, int G>
__device__ __forceinline__ void sweep_fma(float4 &acc, const float *av, const float4 *u, int n) {
#pragma unroll
  for (int t = 0; t < G; ++t) {
    if (t < n) {
      acc.x = fmaf(av[t], u[t].x, acc.x);
      acc.y = fmaf(av[t], u[t].y, acc.y);
      acc.z = fmaf(av[t], u[t].z, acc.z);
      acc.w = fmaf(av[t], u[t].w, acc.w);
    }
  }
}

// Row sum from the warp's staged entries sm[q0, q1), G gathers per round.  (Reading two entries
// per 16-byte shared load, from even positions, was measured 5-15 % slower: the masked first
// round and the wider registers cost more than the shared-memory wavefronts saved.)
template <int KP, int G>
__device__ __forceinline__ float4 sweep_row_staged(const int2 *__restrict__ sm, const float4 *__restrict__ x4, int q0,
                                                   int q1, int cl) {
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int q = q0; q < q1; q += G) {
    float4 u[G];
    float av[G];
#pragma unroll
    for (int t = 0; t < G; ++t) {
      av[t] = 0.f;
      u[t] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (q + t < q1) {
        const int2 ja = sm[q + t];
        av[t] = __int_as_float(ja.y);
        u[t] = __ldg(x4 + (int64_t)ja.x * (KP / 4) + cl);
      }
    }
    sweep_fma<KP, G>(acc, av, u, q1 - q);
  }
  return acc;
}

// Row sum with the entries read from global memory (a tile over the staging capacity).
template <int KP, int G>
__device__ __forceinline__ float4 sweep_row_global(const int32_t *__restrict__ ci, const float *__restrict__ va,
                                                   const float4 *__restrict__ x4, int e0, int e1, int cl) {
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int q = e0; q < e1; q += G) {
    float4 u[G];
    float av[G];
#pragma unroll
    for (int t = 0; t < G; ++t) {
      av[t] = 0.f;
      u[t] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (q + t < e1) {
        av[t] = __ldg(va + q + t);
        u[t] = __ldg(x4 + (int64_t)__ldg(ci + q + t) * (KP / 4) + cl);
      }
    }
    sweep_fma<KP, G>(acc, av, u, e1 - q);
  }
  return acc;
}

template <int KP, int G, int THREADS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) spmm32_sweep_kernel(const SpmmArgs a) {
  static_assert(KP >= 16 && KP <= 64, "sweep kernel: 16 <= kp <= 64");
  using Geo = SweepGeo<KP, THREADS>;
  constexpr int L = Geo::L, R = Geo::R, CAP = Geo::CAP, MW = Geo::MW, NW = Geo::NW;
  __shared__ __align__(16) int2 stage[NW][CAP];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int g = lane / L, cl = lane % L;
  const int32_t *__restrict__ rp = a.rowptr;
  const int32_t *__restrict__ ci = a.colidx;
  const float *__restrict__ va = static_cast<const float *>(a.vals);
  const float4 *__restrict__ x4 = static_cast<const float4 *>(a.x);
  float4 *__restrict__ y4 = static_cast<float4 *>(a.y);
  const int64_t rb0 = a.n * blockIdx.x / gridDim.x, rb1 = a.n * (blockIdx.x + 1) / gridDim.x;
  constexpr int64_t step = (int64_t)R * NW;
  int64_t r = rb0 + (int64_t)R * w;
  if (r >= rb1) return;  // no tile for this warp (the kernel has no block-wide barrier)
  int2 *sm = stage[w];
  // lane l <= R holds the row pointer of row r + l (clipped to the range's end: rows past it are
  // empty), for the current tile and the next one
  int rp_cur = lane <= R ? __ldcs(rp + (r + lane < rb1 ? r + lane : rb1)) : 0;
  int rp_nxt = 0;
  if (lane <= R && r + step < rb1) rp_nxt = __ldcs(rp + (r + step + lane < rb1 ? r + step + lane : rb1));
  int cn[MW];
  float vn[MW];
  {
    const int e0 = __shfl_sync(0xffffffffu, rp_cur, 0), cnt = __shfl_sync(0xffffffffu, rp_cur, R) - e0;
#pragma unroll
    for (int m = 0; m < MW; ++m) {
      const int q = m * 32 + lane;
      cn[m] = 0;
      vn[m] = 0.f;
      if (cnt <= CAP && q < cnt) {
        cn[m] = __ldcs(ci + e0 + q);
        vn[m] = __ldcs(va + e0 + q);
      }
    }
  }
  for (;;) {
    const int e0 = __shfl_sync(0xffffffffu, rp_cur, 0);
    const int cnt = __shfl_sync(0xffffffffu, rp_cur, R) - e0;
    const bool staged = cnt <= CAP;
    if (staged) {
#pragma unroll
      for (int m = 0; m < MW; ++m) {
        const int q = m * 32 + lane;
        if (q < cnt) sm[q] = make_int2(cn[m], __float_as_int(vn[m]));
      }
    }
    __syncwarp();
    // prefetch: the entries of the next tile, the row pointers of the one after
    const int64_t rn = r + step;
    int rp_nn = 0;
    if (rn < rb1) {
      const int f0 = __shfl_sync(0xffffffffu, rp_nxt, 0);
      const int cntn = __shfl_sync(0xffffffffu, rp_nxt, R) - f0;
      if (cntn <= CAP) {
#pragma unroll
        for (int m = 0; m < MW; ++m) {
          const int q = m * 32 + lane;
          if (q < cntn) {
            cn[m] = __ldcs(ci + f0 + q);
            vn[m] = __ldcs(va + f0 + q);
          }
        }
      }
      if (lane <= R && rn + step < rb1) rp_nn = __ldcs(rp + (rn + step + lane < rb1 ? rn + step + lane : rb1));
    }
    const int rs = __shfl_sync(0xffffffffu, rp_cur, g), re = __shfl_sync(0xffffffffu, rp_cur, g + 1);
    const float4 acc = staged ? sweep_row_staged<KP, G>(sm, x4, rs - e0, re - e0, cl)
                              : sweep_row_global<KP, G>(ci, va, x4, rs, re, cl);
    const int64_t row = r + g;
    if (row < rb1) y4[row * (KP / 4) + cl] = acc;
    __syncwarp();
    if (rn >= rb1) break;
    r = rn;
    rp_cur = rp_nxt;
    rp_nxt = rp_nn;
  }
}

// Sweep-kernel shape (measured on the 27-point operator at 96^3 and 128^3): 4 gathers in flight
// per lane (8 spill registers at 64 per thread and run 10-50 % slower), 32 warps per SM in
// blocks of sweep_threads(kp).  More warps per SM run slower: three or four sweeps per SM no
// longer keep their neighbouring grid lines in L1 together (at most 40 registers per thread, too).
constexpr int kSweepG = 4;
constexpr int sweep_threads(int kp) { return kp == 32 ? 512 : 1024; }
constexpr int sweep_blocks_per_sm(int kp) { return 1024 / sweep_threads(kp); }

template <typename T, int KP, int MODE>
cudaError_t launch_kp(const SpmmArgs &a, int grid, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value && MODE == 0 && KP >= 16) {
    if (a.fp32_kernel == 1)
      spmm32_seg_kernel<KP><<<grid, kSpmmThreads, 0, s>>>(a);
    else
      spmm32_sweep_kernel<KP, kSweepG, sweep_threads(KP), sweep_blocks_per_sm(KP)><<<grid, sweep_threads(KP), 0, s>>>(a);
  } else if constexpr (std::is_same<T, float>::value && MODE == 0 && KP >= 8) {
    spmm32_seg_kernel<KP><<<grid, kSpmmThreads, 0, s>>>(a);
  } else if constexpr (KP <= 2) {
    if (a.warp_rows) {
      spmm_warp_kernel<T, KP, MODE><<<grid, kSpmmThreads, 0, s>>>(a);
    } else {
      const size_t smem = (size_t)a.stage_cap * (sizeof(T) + sizeof(int32_t));
      spmm_row_kernel<T, KP, MODE><<<grid, kSpmmThreads, smem, s>>>(a);
    }
  } else if constexpr (KP >= 8) {
    if (a.cols_per_lane == 4)
      spmm_group_kernel<T, KP, MODE, 4><<<grid, kSpmmThreads, 0, s>>>(a);
    else
      spmm_group_kernel<T, KP, MODE, 2><<<grid, kSpmmThreads, 0, s>>>(a);
  } else {
    spmm_group_kernel<T, KP, MODE, 2><<<grid, kSpmmThreads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

template <typename T, int KP, int MODE>
int occ_kp(int stage_cap, int fp32_kernel, int warp_rows) {
  int nb = 0;
  cudaError_t e;
  if constexpr (std::is_same<T, float>::value && MODE == 0 && KP >= 16) {
    if (fp32_kernel != 1) {  // the sweep kernel: sweep_blocks_per_sm(kp) if they fit
      constexpr int TH = sweep_threads(KP), MB = sweep_blocks_per_sm(KP);
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, spmm32_sweep_kernel<KP, kSweepG, TH, MB>, TH, 0);
      if (e != cudaSuccess || nb < 1) return 1;
      return nb < MB ? nb : MB;
    }
  }
  if constexpr (std::is_same<T, float>::value && MODE == 0 && KP >= 8)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, spmm32_seg_kernel<KP>, kSpmmThreads, 0);
  else if constexpr (KP <= 2) {
    if (warp_rows)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, spmm_warp_kernel<T, KP, MODE>, kSpmmThreads, 0);
    else
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, spmm_row_kernel<T, KP, MODE>, kSpmmThreads,
                                                        (size_t)stage_cap * (sizeof(T) + sizeof(int32_t)));
  }
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, spmm_group_kernel<T, KP, MODE, 2>, kSpmmThreads, 0);
  if (e != cudaSuccess || nb < 1) return 1;
  return nb;
}

template <typename T, int MODE>
cudaError_t launch_mode(int kp, const SpmmArgs &a, int grid, cudaStream_t s) {
  switch (kp) {
    case 1: return launch_kp<T, 1, MODE>(a, grid, s);
    case 2: return launch_kp<T, 2, MODE>(a, grid, s);
    case 4: return launch_kp<T, 4, MODE>(a, grid, s);
    case 8: return launch_kp<T, 8, MODE>(a, grid, s);
    case 16: return launch_kp<T, 16, MODE>(a, grid, s);
    case 32: return launch_kp<T, 32, MODE>(a, grid, s);
    case 64: return launch_kp<T, 64, MODE>(a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int MODE>
int occ_mode(int kp, int stage_cap, int fp32_kernel = 0, int warp_rows = 0) {
  switch (kp) {
    case 1: return occ_kp<T, 1, MODE>(stage_cap, fp32_kernel, warp_rows);
    case 2: return occ_kp<T, 2, MODE>(stage_cap, fp32_kernel, warp_rows);
    case 4: return occ_kp<T, 4, MODE>(stage_cap, fp32_kernel, warp_rows);
    case 8: return occ_kp<T, 8, MODE>(stage_cap, fp32_kernel, warp_rows);
    case 16: return occ_kp<T, 16, MODE>(stage_cap, fp32_kernel, warp_rows);
    case 32: return occ_kp<T, 32, MODE>(stage_cap, fp32_kernel, warp_rows);
    case 64: return occ_kp<T, 64, MODE>(stage_cap, fp32_kernel, warp_rows);
    default: return 1;
  }
}

// y = A^T x by scattering over the rows of A: y_jc += a_ij x_ic with FP64 atomics (y zeroed
// first).  No transposed copy is needed; the summation order into y_jc is not fixed.
__global__ void spmm_t_atomic_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                     const double *__restrict__ va, const double *__restrict__ x,
                                     double *__restrict__ y, int64_t n, int k) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t total = n * k;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
    const int64_t i = t / k;
    const int c = (int)(t - i * k);
    const double xi = x[t];
    for (int e = __ldg(rp + i); e < __ldg(rp + i + 1); ++e) atomicAdd(y + (int64_t)__ldg(ci + e) * k + c, __ldg(va + e) * xi);
  }
}

// Sampled product on the pattern of A: g_e = alpha * sum_c l_ic x_jc for every entry e = (i, j)
// (the gradient of a loss with respect to the matrix values, with l the adjoint solution).
// One thread per row, k FMAs per entry in column order; ld = k for both blocks.
__global__ void sddmm_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                             const double *__restrict__ l, const double *__restrict__ x, double alpha,
                             double *__restrict__ g, int64_t n, int k) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double *li = l + i * k;
    for (int e = __ldg(rp + i); e < __ldg(rp + i + 1); ++e) {
      const double *xj = x + (int64_t)__ldg(ci + e) * k;
      double acc = 0.0;
      for (int c = 0; c < k; ++c) acc = fma(__ldg(li + c), __ldg(xj + c), acc);
      g[e] = alpha * acc;
    }
  }
}

}  // namespace

cudaError_t launch_spmm_t_atomic(const int32_t *rowptr, const int32_t *colidx, const double *vals, const double *x,
                                 double *y, int64_t n, int k, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(y, 0, sizeof(double) * n * k, s);
  if (e != cudaSuccess) return e;
  const int64_t total = n * k;
  int grid = (int)((total + 255) / 256);
  if (grid > 152 * 16) grid = 152 * 16;
  if (grid < 1) grid = 1;
  spmm_t_atomic_kernel<<<grid, 256, 0, s>>>(rowptr, colidx, vals, x, y, n, k);
  return cudaGetLastError();
}

cudaError_t launch_sddmm(const int32_t *rowptr, const int32_t *colidx, const double *l, const double *x, double alpha,
                         double *g, int64_t n, int k, cudaStream_t s) {
  int grid = (int)((n + 255) / 256);
  if (grid > 152 * 16) grid = 152 * 16;
  if (grid < 1) grid = 1;
  sddmm_kernel<<<grid, 256, 0, s>>>(rowptr, colidx, l, x, alpha, g, n, k);
  return cudaGetLastError();
}

cudaError_t launch_spmm(int kp, int mode, const SpmmArgs &a, int grid, cudaStream_t s) {
  return mode == 0 ? launch_mode<double, 0>(kp, a, grid, s) : launch_mode<double, 1>(kp, a, grid, s);
}

int spmm_blocks_per_sm(int kp, int mode, int stage_cap, int warp_rows) {
  return mode == 0 ? occ_mode<double, 0>(kp, stage_cap, 0, warp_rows) : occ_mode<double, 1>(kp, stage_cap, 0, warp_rows);
}

cudaError_t launch_spmm32(int kp, const SpmmArgs &a, int grid, cudaStream_t s) {
  return launch_mode<float, 0>(kp, a, grid, s);
}

int spmm32_blocks_per_sm(int kp, int stage_cap, int fp32_kernel, int warp_rows) {
  return occ_mode<float, 0>(kp, stage_cap, fp32_kernel, warp_rows);
}

}  // namespace bicgk
