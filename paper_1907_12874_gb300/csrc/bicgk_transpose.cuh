// Device-side CSR transpose (bicgk_transpose.cu), used by the C-ABI in bicgk_api.cu.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace bicgk {

// Device scratch the transpose of an n x n matrix with nnz entries needs (bytes).
size_t transpose_scratch_bytes(int64_t n, int64_t nnz);
// A^T of the CSR (rowptr, colidx, vals): rowptrT[n+1], colT[nnz], valT[nnz], and perm[nnz] = the
// entry of A that each entry of A^T copies; *maxtile = the most entries in a 256-row tile of A^T.
cudaError_t launch_transpose(const int32_t *rowptr, const int32_t *colidx, const double *vals, int64_t n, int64_t nnz,
                             int32_t *rowptrT, int32_t *colT, double *valT, int32_t *perm, int *maxtile, void *scratch,
                             cudaStream_t s);
// valT[p] = vals[perm[p]]: new values of A (same pattern) carried to A^T.
cudaError_t launch_permute_values(const int32_t *perm, const double *vals, int64_t nnz, double *valT, cudaStream_t s);

}  // namespace bicgk
