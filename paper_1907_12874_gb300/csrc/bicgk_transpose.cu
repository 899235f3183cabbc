// Device-side CSR transpose: the CSR of A^T built on the GPU, for the Aᵀ products of the adjoint
// solve (dL/dB and dL/dA of the differentiable solve) and f_0 = A^T r_0 of Algorithm 3.
//
// Row j of A^T lists the rows i of A that hold column j, ascending in i (entries of one row of A
// that repeat a column keep their order).  That order is the one of a STABLE sort of A's entries
// by column, since A's entries are stored row by row: the entries are sorted as (column, entry
// index) pairs by a least-significant-digit radix sort, 8 bits a pass, each pass stable:
//   1. per tile of 2048 entries, a histogram of the pass's digit (shared-memory counters);
//   2. an exclusive scan of the histograms in digit-major order gives every (digit, tile) its
//      output offset, so digit d's entries land after every smaller digit's, tiles in order;
//   3. per tile, each entry's rank among the tile's earlier entries with its digit -- rounds of
//      256 entries in order, warps in order, lanes in order (warp match + population counts) --
//      places it at offset + rank.
// Every step is a fixed function of the input (no atomics decide a position), so the result is
// bitwise the host counting sort's.  The row pointers of A^T are the exclusive scan of the
// column counts; the entry permutation is kept so that new values of A (same pattern) can be
// carried to A^T with one gather.
#include "bicgk_dev.cuh"
#include "bicgk_transpose.cuh"

namespace bicgk {

namespace {

constexpr int kTT = 256;                // threads per block
constexpr int kTItems = 8;              // entries per thread and tile
constexpr int kTTile = kTT * kTItems;   // entries per tile
constexpr int kBins = 256;              // radix digit values (8 bits)

// ---- exclusive scan of int32 counts (sums fit in int32: at most nnz)

__device__ int block_exclusive_scan(int v, int *s_warp, int *total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int i = 0; i < kTT / 32; ++i) {
      const int t = s_warp[i];
      s_warp[i] = run;
      run += t;
    }
    *total = run;
  }
  __syncthreads();
  const int r = s_warp[w] + x - v;
  __syncthreads();
  return r;
}

__global__ void scan_tile_sums(const int *__restrict__ in, int64_t m, int *__restrict__ sums) {
  __shared__ int s_warp[kTT / 32];
  __shared__ int s_total;
  const int64_t base = (int64_t)blockIdx.x * kTTile;
  int v = 0;
  for (int q = 0; q < kTItems; ++q) {
    const int64_t e = base + (int64_t)threadIdx.x * kTItems + q;
    if (e < m) v += in[e];
  }
  block_exclusive_scan(v, s_warp, &s_total);
  if (threadIdx.x == 0) sums[blockIdx.x] = s_total;
}

// One block: exclusive scan of the tile sums, in place.
__global__ void scan_sums(int *sums, int64_t nt) {
  __shared__ int s_warp[kTT / 32];
  __shared__ int s_total;
  int carry = 0;
  for (int64_t b = 0; b < nt; b += kTT) {
    const int64_t i = b + threadIdx.x;
    const int v = i < nt ? sums[i] : 0;
    const int r = block_exclusive_scan(v, s_warp, &s_total);
    if (i < nt) sums[i] = carry + r;
    carry += s_total;
    __syncthreads();
  }
}

__global__ void scan_apply(const int *__restrict__ in, int64_t m, const int *__restrict__ sums, int *__restrict__ out) {
  __shared__ int s_warp[kTT / 32];
  __shared__ int s_total;
  const int64_t base = (int64_t)blockIdx.x * kTTile + (int64_t)threadIdx.x * kTItems;
  int v[kTItems];
  int t = 0;
  for (int q = 0; q < kTItems; ++q) {
    v[q] = base + q < m ? in[base + q] : 0;
    t += v[q];
  }
  int run = sums[blockIdx.x] + block_exclusive_scan(t, s_warp, &s_total);
  for (int q = 0; q < kTItems; ++q) {
    if (base + q < m) out[base + q] = run;
    run += v[q];
  }
}

// ---- counts, row of every entry, radix passes, gathers

__global__ void col_count_kernel(const int32_t *__restrict__ colidx, int64_t nnz, int *__restrict__ cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) atomicAdd(cnt + colidx[e], 1);
}

__global__ void row_of_kernel(const int32_t *__restrict__ rowptr, int64_t n, int32_t *__restrict__ row_of) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) row_of[e] = (int32_t)i;
}

__global__ void iota_kernel(int32_t *__restrict__ v, int64_t m) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) v[e] = (int32_t)e;
}

__global__ void radix_hist(const int32_t *__restrict__ keys, int64_t nnz, int shift, int *__restrict__ hist,
                           int64_t ntiles) {
  __shared__ int s_h[kBins];
  s_h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kTTile;
  for (int q = 0; q < kTItems; ++q) {
    const int64_t e = base + (int64_t)q * kTT + threadIdx.x;
    if (e < nnz) atomicAdd(&s_h[(keys[e] >> shift) & (kBins - 1)], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = s_h[threadIdx.x];
}

// Stable scatter of one pass: entry e of the tile goes to off[digit][tile] + its rank among the
// tile's earlier entries with that digit.
__global__ void radix_scatter(const int32_t *__restrict__ keys, const int32_t *__restrict__ vals, int64_t nnz,
                              int shift, const int *__restrict__ off, int64_t ntiles, int32_t *__restrict__ keys_out,
                              int32_t *__restrict__ vals_out) {
  __shared__ int s_cnt[kTT / 32][kBins];   // entries of each digit per warp (this round)
  __shared__ int s_run[kBins];             // entries of each digit in earlier rounds
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < (kTT / 32) * kBins; i += kTT) (&s_cnt[0][0])[i] = 0;
  s_run[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kTTile;
  const unsigned lt = (1u << lane) - 1u;
  for (int q = 0; q < kTItems; ++q) {
    const int64_t e = base + (int64_t)q * kTT + threadIdx.x;
    const bool valid = e < nnz;
    const int32_t key = valid ? keys[e] : 0;
    const int32_t val = valid ? vals[e] : 0;
    const int d = valid ? (key >> shift) & (kBins - 1) : kBins;   // kBins: no entry
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lt);
    if (valid && rank == 0) s_cnt[w][d] = __popc(peers);
    __syncthreads();
    {  // thread b: per-warp offsets of digit b in this round (warps in order)
      const int b = threadIdx.x;
      int run = s_run[b];
      for (int ww = 0; ww < kTT / 32; ++ww) {
        const int c = s_cnt[ww][b];
        s_cnt[ww][b] = run;
        run += c;
      }
      s_run[b] = run;
    }
    __syncthreads();
    if (valid) {
      const int64_t pos = (int64_t)off[(int64_t)d * ntiles + blockIdx.x] + s_cnt[w][d] + rank;
      keys_out[pos] = key;
      vals_out[pos] = val;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < (kTT / 32) * kBins; i += kTT) (&s_cnt[0][0])[i] = 0;
    __syncthreads();
  }
}

// A^T's column indices and values from the sorted permutation of A's entries.
__global__ void transpose_gather(const int32_t *__restrict__ perm, const int32_t *__restrict__ row_of,
                                 const double *__restrict__ vals, int64_t nnz, int32_t *__restrict__ colT,
                                 double *__restrict__ valT) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride) {
    const int32_t e = perm[p];
    colT[p] = row_of[e];
    valT[p] = vals[e];
  }
}

__global__ void permute_values(const int32_t *__restrict__ perm, const double *__restrict__ vals, int64_t nnz,
                               double *__restrict__ valT) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride) valT[p] = vals[perm[p]];
}

__global__ void max_tile_kernel(const int32_t *__restrict__ rowptr, int64_t n, int *__restrict__ maxtile) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int m = 0;
  for (int64_t r0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kSpmmTileRows; r0 < n;
       r0 += stride * kSpmmTileRows) {
    const int64_t r1 = r0 + kSpmmTileRows < n ? r0 + kSpmmTileRows : n;
    const int t = rowptr[r1] - rowptr[r0];
    if (t > m) m = t;
  }
  atomicMax(maxtile, m);
}

int grid_for(int64_t work) {
  int64_t g = (work + kTT - 1) / kTT;
  return (int)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

// Exclusive scan of m ints (in may equal out); tmp holds ceil(m / kTTile) ints.
cudaError_t exclusive_scan(const int *in, int *out, int64_t m, int *tmp, cudaStream_t s) {
  const int64_t nt = (m + kTTile - 1) / kTTile;
  if (nt < 1) return cudaSuccess;
  scan_tile_sums<<<(unsigned)nt, kTT, 0, s>>>(in, m, tmp);
  scan_sums<<<1, kTT, 0, s>>>(tmp, nt);
  scan_apply<<<(unsigned)nt, kTT, 0, s>>>(in, m, tmp, out);
  return cudaGetLastError();
}

}  // namespace

size_t transpose_scratch_bytes(int64_t n, int64_t nnz) {
  const int64_t ntiles = (nnz + kTTile - 1) / kTTile;
  const int64_t hist = (int64_t)kBins * (ntiles > 0 ? ntiles : 1);
  const int64_t sums = (hist > n + 1 ? hist : n + 1) / kTTile + 2;
  // row_of, two key and two value buffers (nnz each), histogram/offsets, scan sums, counts, max
  return sizeof(int32_t) * (5 * (size_t)(nnz > 0 ? nnz : 1) + (size_t)hist + (size_t)sums + (size_t)(n + 2) + 4);
}

cudaError_t launch_transpose(const int32_t *rowptr, const int32_t *colidx, const double *vals, int64_t n, int64_t nnz,
                             int32_t *rowptrT, int32_t *colT, double *valT, int32_t *perm, int *maxtile, void *scratch,
                             cudaStream_t s) {
  const int64_t ntiles = (nnz + kTTile - 1) / kTTile;
  const int64_t hist_len = (int64_t)kBins * (ntiles > 0 ? ntiles : 1);
  int32_t *row_of = static_cast<int32_t *>(scratch);
  int32_t *k0 = row_of + (nnz > 0 ? nnz : 1);
  int32_t *k1 = k0 + (nnz > 0 ? nnz : 1);
  int32_t *v1 = k1 + (nnz > 0 ? nnz : 1);
  int32_t *v0 = v1 + (nnz > 0 ? nnz : 1);
  int *hist = reinterpret_cast<int *>(v0 + (nnz > 0 ? nnz : 1));
  int *sums = hist + hist_len;
  const int64_t sums_len = (hist_len > n + 1 ? hist_len : n + 1) / kTTile + 2;
  int *cnt = sums + sums_len;
  cudaError_t e;
  // row pointers of A^T: column counts, exclusive scan (count[n] = 0 gives rowptrT[n] = nnz)
  if ((e = cudaMemsetAsync(cnt, 0, sizeof(int) * (n + 1), s)) != cudaSuccess) return e;
  if (nnz > 0) col_count_kernel<<<grid_for(nnz), kTT, 0, s>>>(colidx, nnz, cnt);
  if ((e = exclusive_scan(cnt, rowptrT, n + 1, sums, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(maxtile, 0, sizeof(int), s)) != cudaSuccess) return e;
  max_tile_kernel<<<grid_for((n + kSpmmTileRows - 1) / kSpmmTileRows), kTT, 0, s>>>(rowptrT, n, maxtile);
  if (nnz == 0) return cudaGetLastError();
  // stable sort of (column, entry) by column, 8 bits a pass, as many passes as n - 1 needs
  row_of_kernel<<<grid_for(n), kTT, 0, s>>>(rowptr, n, row_of);
  if ((e = cudaMemcpyAsync(k0, colidx, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
  iota_kernel<<<grid_for(nnz), kTT, 0, s>>>(v0, nnz);
  int bits = 0;
  while (bits < 31 && ((int64_t)1 << bits) < n) ++bits;
  const int passes = bits == 0 ? 1 : (bits + 7) / 8;
  int32_t *ki = k0, *vi = v0, *ko = k1, *vo = v1;
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = 8 * pass;
    radix_hist<<<(unsigned)ntiles, kTT, 0, s>>>(ki, nnz, shift, hist, ntiles);
    if ((e = exclusive_scan(hist, hist, hist_len, sums, s)) != cudaSuccess) return e;
    radix_scatter<<<(unsigned)ntiles, kTT, 0, s>>>(ki, vi, nnz, shift, hist, ntiles, ko, vo);
    int32_t *t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
  }
  if ((e = cudaMemcpyAsync(perm, vi, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
  transpose_gather<<<grid_for(nnz), kTT, 0, s>>>(perm, row_of, vals, nnz, colT, valT);
  return cudaGetLastError();
}

cudaError_t launch_permute_values(const int32_t *perm, const double *vals, int64_t nnz, double *valT, cudaStream_t s) {
  if (nnz == 0) return cudaSuccess;
  permute_values<<<grid_for(nnz), kTT, 0, s>>>(perm, vals, nnz, valT);
  return cudaGetLastError();
}

}  // namespace bicgk
