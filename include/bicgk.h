/*
 * bicgk -- BiCGStab with k right-hand sides on one GB300 GPU (sm_103a).
 *
 * C-ABI of the library libbicgk.so.  Plain pointers and sizes only.
 *
 * Method: B. Krasnopolsky, "Revisiting Performance of BiCGStab Methods for
 * Solving Systems with Multiple Right-Hand Sides", arXiv:1907.12874.
 *   - classical BiCGStab, basic (Algorithm 1) and merged (Algorithm 2) forms;
 *   - preconditioned (Algorithm 5), preconditioned Pipelined (Algorithm 7) and
 *     Improved (Algorithm 3) BiCGStab, basic and merged forms;
 *   - Reordered BiCGStab (Algorithm 6) with the identity preconditioner
 *     applied as a vector copy (Sec. 2.3), basic and merged forms;
 *   - Pipelined BiCGStab (Algorithm 4), basic and merged forms;
 *   "basic" = one kernel per vector operation of the listing (the 4-vector
 *   update of Algorithm 4 as two kernels, Table 2 footnote); "merged" = one
 *   kernel per merged line of the listing (updates fused with their dot
 *   products and the residual-norm estimate, Sec. 2.2).
 *
 * Data layout (Sec. 3.1): the k vectors of a block are stored row-wise in
 * one array, element (i, c) at index i*k + c ("RHS-interleaved", N x k,
 * row-major).  The matrix is CSR with int32 row pointers and column indices
 * and FP64 values (the CRS format of the paper's traffic model, Eq. for
 * Sigma_mul in Sec. 3.1).
 *
 * All entry points return 0 on success or a negative BICGK_E* code; they never
 * abort the process.  bicgk_strerror() names a code.
 * Thread safety: distinct operators may be used from distinct threads; one
 * operator runs one call at a time (its workspace is shared by its calls).
 */
#ifndef BICGK_H
#define BICGK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque operator: device copy of the CSR matrix plus solver workspace. */
typedef struct bicgk_op_s *bicgk_op;

/* Where a caller-owned array lives. */
enum bicgk_mem { BICGK_MEM_HOST = 0, BICGK_MEM_DEVICE = 1 };

/* Method forms (same order as the oracle). */
enum bicgk_variant {
  BICGK_CLASSICAL_PLAIN = 0,  /* Algorithm 1, one kernel per vector op              */
  BICGK_CLASSICAL_MERGED = 1, /* Algorithm 2                                        */
  BICGK_REORDERED_PLAIN = 2,  /* Algorithm 6 with M^-1 = copy, one kernel per op   */
  BICGK_REORDERED_MERGED = 3, /* Algorithm 6 with M^-1 = copy                       */
  BICGK_PIPELINED_PLAIN = 4,  /* Algorithm 4, one kernel per op                     */
  BICGK_PIPELINED_MERGED = 5, /* Algorithm 4                                        */
  BICGK_PRECOND_PLAIN = 6,    /* Algorithm 5 (preconditioned), one kernel per op    */
  BICGK_PRECOND_MERGED = 7,   /* Algorithm 5                                        */
  BICGK_PPIPE_PLAIN = 8,      /* Algorithm 7 (preconditioned Pipelined), per op     */
  BICGK_PPIPE_MERGED = 9,     /* Algorithm 7                                        */
  BICGK_IMPROVED_PLAIN = 10,  /* Algorithm 3 (Improved, needs A^T r_0), per op      */
  BICGK_IMPROVED_MERGED = 11  /* Algorithm 3                                        */
};

/* Per-RHS outcome written to status[c]. */
enum bicgk_rhs_status {
  BICGK_CONVERGED = 0, /* stop test passed (or b_c = 0, or r_0 already small)   */
  BICGK_MAXIT = 1,     /* maxit iterations done without passing the stop test   */
  BICGK_BREAKDOWN = 2, /* a scalar recurrence divided by an exact zero          */
  BICGK_NONFINITE = 3  /* a dot product or scalar became Inf or NaN             */
};

/* Solve flags (bit mask). */
enum bicgk_flags {
  BICGK_FLAG_NO_STOP_TEST = 1, /* run exactly maxit iterations (fixed-count benchmarking,
                                  Sec. 2.3 uses N_it = 1000); breakdown rules still apply */
  BICGK_FLAG_JACOBI = 2        /* M = diag(A) (Jacobi) instead of the identity copy in the forms
                                  that apply M^-1 (Algorithms 5, 6, 7); a zero diagonal counts as 1 */
};

/* Error codes. */
enum bicgk_error {
  BICGK_OK = 0,
  BICGK_E_INVALID = -1,  /* bad argument (null pointer, size out of range, bad enum)   */
  BICGK_E_BAD_CSR = -2,  /* row pointers not monotone, column index out of range, ...   */
  BICGK_E_CUDA = -3,     /* a CUDA runtime call failed (bicgk_last_cuda_error() has it) */
  BICGK_E_NOMEM = -4,    /* device or pinned host allocation failed                     */
  BICGK_E_UNSUPPORTED = -5, /* k above BICGK_MAX_K, or no sm_103 device                 */
  BICGK_E_TIMEOUT = -6     /* a grid-barrier wait of the persistent batch kernel passed
                              its deadline; the solve was abandoned (outputs undefined)  */
};

#define BICGK_MAX_K 64

/*
 * Create an operator from a CSR matrix (n_rows x n_rows, nnz entries).
 *   rowptr[n_rows+1], colidx[nnz] (int32), vals[nnz] (FP64), in memory space
 *   `mem`.  The arrays are copied to the current CUDA device; the caller keeps
 *   ownership of its arrays.  The matrix is validated: rowptr[0] == 0,
 *   rowptr non-decreasing, rowptr[n_rows] == nnz, 0 <= colidx < n_rows
 *   (BICGK_E_BAD_CSR otherwise).  Column indices need not be sorted.
 *   stream: a cudaStream_t (NULL = legacy default stream) used for the copies.
 * On success *out receives the operator; release it with bicgk_op_destroy().
 */
int bicgk_csr_create(bicgk_op *out, int64_t n_rows, int64_t nnz, const int32_t *rowptr,
                     const int32_t *colidx, const double *vals, int mem, void *stream);

/*
 * Y = A X for a block of k vectors (the SpMV of Algorithms 1-7 applied to k
 * row-interleaved vectors; the operation behind Sigma_mul, Sec. 3.1).
 *   X, Y: device arrays of n_rows*k FP64, RHS-interleaved (i*k + c); they must
 *   not overlap.  1 <= k <= BICGK_MAX_K.  Any 8-byte alignment is accepted
 *   (unaligned or non-power-of-two blocks go through the operator's workspace).
 *   Runs on `stream`, returns without synchronising.
 */
int bicgk_spmm(bicgk_op A, int32_t k, const double *X, double *Y, void *stream);

/*
 * Y = A X in FP32: the product of the FP32 inner solves of bicgk_solve_mixed
 * (the SpMV of Sec. 3.1 with the values rounded once to FP32), for callers that
 * keep FP32 blocks.
 *   X, Y: device arrays of n_rows*k FP32, RHS-interleaved (i*k + c); they must
 *   not overlap; 4-byte alignment suffices.  1 <= k <= BICGK_MAX_K.
 *   y_ic = sum over the entries of row i, in CSR order, of fl32(a_ij) x_jc,
 *   accumulated in FP32 with fused multiply-adds.
 * The FP32 copy of the values is made on the first FP32 use and kept with the
 * operator.  Errors: BICGK_E_INVALID (null or equal pointers, k < 1),
 * BICGK_E_UNSUPPORTED (k > BICGK_MAX_K), BICGK_E_NOMEM, BICGK_E_CUDA.  Runs on
 * `stream`, returns without synchronising.
 */
int bicgk_spmm_f32(bicgk_op A, int32_t k, const float *X, float *Y, void *stream);

/*
 * Solve A X = B for k right-hand sides with one of the twelve forms of
 * bicgk_variant (Algorithms 1-7, basic and merged).
 *   B      : n_rows*k FP64, RHS-interleaved, in space `mem`.
 *   X0     : initial guess in the same layout and space, or NULL for zero.
 *   X      : n_rows*k FP64 output in the same layout and space (may alias X0).
 *   rel_tol: column c stops when its squared residual-norm estimate falls
 *            strictly below (rel_tol * ||b_c||_2)^2 (the listings' test with
 *            eps = rel_tol*||b_c||).  rel_tol >= 0.
 *   maxit  : maximum iterations, 0 <= maxit <= 1e7.
 *   flags  : bicgk_flags.
 *   iters  : host int32[k]  -- iterates x_{j+1} formed by column c.
 *   status : host int32[k]  -- bicgk_rhs_status per column.
 *   resid_hist: host FP64[(maxit+1)*k] or NULL; entry (j, c) at j*k + c is
 *            ||r_0|| for j = 0 and the method's estimate of ||r_j|| after
 *            iteration j-1 (sqrt of the quantity of the stop test, 0 when it is
 *            negative); NaN where column c formed no iterate j.
 *   true_relres: host FP64[k] or NULL -- ||b_c - A x_c|| / ||b_c|| recomputed
 *            from the final X (0 when b_c = 0).
 * Everything runs on `stream` (cudaStream_t, NULL = legacy default); the call
 * returns after all outputs are valid.  A non-converged column is not an error.
 * Per-column rules where the paper is silent: b_c = 0 gives x_c = 0 with 0
 * iterations; a column whose ||r_0|| already passes the test keeps x0; a
 * column stops independently of the others and is not written afterwards.
 * Execution (bicgk_set_option): from k = 8 the columns run as concurrent
 * groups on internal streams joined back to `stream`; a group narrows its
 * layout as its columns stop; host
 * blocks that are page-locked are read and written in place.  Columns never
 * interact, so these change summation orders only: iterates agree with a
 * one-group solve to rounding, and a column's iteration count can differ by
 * the few iterations that rounding moves near the tolerance.
 * The first call per (variant, k) builds and caches a CUDA graph; callers must
 * not capture this call into a graph of their own.
 */
int bicgk_solve(bicgk_op A, int32_t k, const double *B, const double *X0, double rel_tol, int32_t maxit,
                int variant, int32_t flags, int mem, double *X, int32_t *iters, int32_t *status,
                double *resid_hist, double *true_relres, void *stream);

/*
 * Transpose products for the adjoint (differentiation) path.  No counterpart in the paper.
 *
 * bicgk_op_transpose: *AT receives a new operator for A^T (same size and nonzeros), built on the
 *   GPU from A's device CSR by a stable radix sort of the entries by column: row j of A^T lists
 *   the rows i of A holding column j in ascending order (repeated columns of a row in their
 *   order), the result of a stable counting sort, bitwise.  AT keeps the entry permutation, so
 *   bicgk_op_transpose_refresh can carry new values of A to it.  Allocates the operator and a
 *   temporary of about 20 bytes per nonzero.  Release AT with bicgk_op_destroy().
 * bicgk_op_set_values: new values vals[nnz] (space `mem`) for A's sparsity pattern, copied in
 *   place: A's captured graphs stay valid, and A's internal transposed copy (bicgk_spmm_t,
 *   Algorithm 3), FP32 copy and Jacobi diagonal follow.  Returns when the copy is done.
 * bicgk_op_transpose_refresh: AT (made from A by bicgk_op_transpose) takes A's current values.
 *   BICGK_E_INVALID if AT was not made that way or the sizes differ.
 * bicgk_op_get_csr: copies the operator's device CSR to the host arrays rowptr[n_rows+1],
 *   colidx[nnz], vals[nnz] (each nullable).
 * bicgk_spmm_t: Y = A^T X for device blocks of n_rows*k FP64 (ld = k).
 *   method BICGK_TRANSPOSE_EXPLICIT: the SpMM kernel on a transposed copy that A builds on the
 *   first call and keeps (atomic-free, deterministic); BICGK_TRANSPOSE_ATOMIC: a scatter over the
 *   rows of A with FP64 atomic adds (no extra memory; the summation order is not fixed).
 * bicgk_sddmm: G[e] = alpha * sum_c L[i*k+c] * X[j*k+c] for every entry e = (i, j) of A, in CSR
 *   order (device arrays; G has nnz entries).  With L the adjoint solution of A^T L = dLoss/dX,
 *   X the solution and alpha = -1 this is dLoss/dA on the sparsity pattern.
 */
enum bicgk_transpose_method { BICGK_TRANSPOSE_EXPLICIT = 0, BICGK_TRANSPOSE_ATOMIC = 1 };
int bicgk_op_transpose(bicgk_op A, bicgk_op *AT, void *stream);
int bicgk_op_set_values(bicgk_op A, const double *vals, int mem, void *stream);
int bicgk_op_transpose_refresh(bicgk_op A, bicgk_op AT, void *stream);
int bicgk_op_get_csr(bicgk_op A, int32_t *rowptr, int32_t *colidx, double *vals, void *stream);
int bicgk_spmm_t(bicgk_op A, int32_t k, const double *X, double *Y, int method, void *stream);
int bicgk_sddmm(bicgk_op A, int32_t k, const double *L, const double *X, double alpha, double *G, void *stream);

/*
 * Mixed-precision solve of A X = B: FP64 iterative refinement around FP32
 * BiCGStab inner solves (no counterpart in the paper, which runs in FP64; the
 * inner solver is the paper's merged BiCGStab, Algorithm 2).
 *   pass j (0 <= j <= max_outer): r = b - A x in FP64 (FP64 matrix); column c
 *   stops when ||r_c|| < rel_tol*||b_c|| (status CONVERGED) or at j = max_outer
 *   (MAXIT); otherwise A d = fl32(r) is solved with FP32 matrix values and FP32
 *   vectors (elementwise updates in FP32; dot products with exact FP32 products
 *   summed in float-float per thread and in FP64 across threads; scalars alpha,
 *   omega, rho, beta in FP64) from d = 0 until its residual estimate falls below
 *   inner_tol*||fl32(r)|| or max_inner iterations, and x += d in FP64.
 *   B, X0 (nullable), X: n_rows*k FP64 in space `mem`, as for bicgk_solve.
 *   outer_iters[k]: refinement passes that updated x_c; inner_iters[k]: FP32
 *   iterations summed over the passes; status[k]: bicgk_rhs_status of the
 *   refinement; resid_hist[(max_outer+1)*k] (nullable): ||b_c - A x_c|| before
 *   pass j (FP64), NaN after column c stopped; true_relres[k] (nullable): the
 *   final ||b_c - A x_c|| / ||b_c||.
 *   0 <= max_outer <= 1000, 1 <= max_inner, 0 < inner_tol < 1.
 * Runs on `stream` and returns when all outputs are valid.
 */
int bicgk_solve_mixed(bicgk_op A, int32_t k, const double *B, const double *X0, double rel_tol, int32_t max_outer,
                      double inner_tol, int32_t max_inner, int mem, double *X, int32_t *outer_iters,
                      int32_t *inner_iters, int32_t *status, double *resid_hist, double *true_relres,
                      void *stream);

/*
 * bicgk_solve without any GPU memory allocation (the paper has no counterpart;
 * this is an interface for callers that cannot allocate).
 *
 * Who needs it: code that owns all device memory through its own pool (a
 * cudaMalloc/cudaFree from inside the solve would bypass the pool and
 * synchronise the whole device), loops that must not take the implicit
 * synchronisation of an allocation, and embeddings that run within a fixed
 * device-memory budget.  The caller passes every input and output; the CSR
 * arrays (rowptr[n_rows+1], colidx[nnz], vals[nnz]; layout and meaning as in
 * bicgk_csr_create) and B, X0 (nullable), X are DEVICE pointers in the layout
 * of bicgk_solve.  A check kernel validates the CSR before any product reads
 * it (row pointers from 0, never decreasing, ending at nnz; column indices in
 * [0, n_rows)) and a malformed one returns BICGK_E_BAD_CSR; iters, status, resid_hist and
 * true_relres are host arrays as there, and every other argument means the
 * same.  Results equal bicgk_solve's with one column group and no column
 * compaction (BICGK_OPT_RHS_GROUPS = 1, BICGK_OPT_COMPACT = 1), within rounding
 * of the same kernels.
 *
 * Scratch: one 16 MiB file-scope device array in this library, which every
 * GPU that loads the library keeps until the process exits.  A problem fits if
 *   8*18*(n_rows*kp + 34) + 8*(maxit+1)*kp + 8*448*(8*SMs + 128) + ~2 KB <= 16 MiB
 * (kp = k rounded up to a power of two; about n_rows*kp <= 80,000 at
 * maxit = 1000); larger problems return BICGK_E_UNSUPPORTED with the sizes in
 * bicgk_last_cuda_error().  variant: 0..9 (the Improved form needs a
 * transposed copy of A and is refused); flags: BICGK_FLAG_NO_STOP_TEST only.  The iteration loop runs from the host (one
 * stream synchronisation per iteration), not from a CUDA graph.
 *
 * Every call, on any stream or thread, uses the same array and leaves its
 * contents behind; what must start at zero (reduction ticket, iteration
 * counter, per-column state, padding) is cleared by each call.  Calls whose GPU
 * work overlaps in time race on the array and give wrong results: serialise
 * them.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, under a lock (first calls
 * from several host threads are safe); make that first call before any stream
 * capture.  Returns when all outputs are valid.
 */
int bicgk_solve_noalloc(int64_t n_rows, int64_t nnz, const int32_t *rowptr, const int32_t *colidx,
                        const double *vals, int32_t k, const double *B, const double *X0, double rel_tol,
                        int32_t maxit, int variant, int32_t flags, double *X, int32_t *iters, int32_t *status,
                        double *resid_hist, double *true_relres, void *stream);

/* Launch-shape options of an operator (bicgk_set_option); 0 restores the default. */
enum bicgk_option {
  BICGK_OPT_VEC_BLOCKS_PER_SM = 1, /* blocks of 512 threads per SM for the streaming kernels (0..4;
                                      default: the occupancy maximum, 2; one for the kernels
                                      that only reduce when kp <= 2, and one for every
                                      streaming kernel of a solve that runs four concurrent
                                      column groups); a value caps the occupancy maximum       */
  BICGK_OPT_SPMM_BLOCKS_PER_SM = 2, /* blocks of 256 threads per SM for the SpMM (0..32; default:
                                      the occupancy maximum, at most 4 in a solve of four
                                      concurrent column groups and in a one-group solve of
                                      kp = 4); a value caps the occupancy maximum              */
  BICGK_OPT_RHS_GROUPS = 3,         /* 0 (default): k >= 8 is solved as two column groups
                                      running concurrently on internal streams, k >= 32 as four
                                      (bicgk_solve_mixed: two from k = 16); 1: one group;
                                      2..4: that many groups (at most k).  Profiling mode runs
                                      the same groups one after another on the caller's stream. */
  BICGK_OPT_FUSED_DOTS = 4,         /* merged forms of Algorithms 2, 5 and 6: take the dot
                                      kernel that follows an SpMM in the listing (delta after
                                      v = A p; group 1 after t = A s, Algorithms 2 and 5) into
                                      the SpMM's epilogue.  0: when the solve runs as two or
                                      more column groups (default); 1: never; 2: always.  The iterates are
                                      the same up to the summation order of those dots.        */
  BICGK_OPT_THETA_IN_S = 5,         /* merged forms of Algorithms 2 and 5: take theta = (s, s)
                                      of group 1 in the kernel that forms s = r - alpha v
                                      (Algorithm 5: before s^ = M^-1 s), leaving phi = (t, s)
                                      and psi = (t, t) to group 1.  0: for k >= 4, except the
                                      merged classical form when its dots are folded into the
                                      SpMM of two column groups (default); 1: never; 2: always.
                                      Same iterates up to the summation order of theta.        */
  BICGK_OPT_HOST_ZERO_COPY = 6,     /* host calls (BICGK_MEM_HOST) whose B, X (and X0) are all
                                      page-locked: 0 (default): the kernels read B and write X
                                      in place through their mapped device addresses, group by
                                      group, overlapping the transfer with the solve; 1: copy
                                      through a device staging block as for pageable memory.   */
  BICGK_OPT_COMPACT = 7,            /* every form.  0 (default): when at most half of a
                                      column group's columns are still iterating, the group
                                      continues in a layout of half the width (down to one
                                      column), so stopped columns stop costing arithmetic;
                                      1: never.  The iterates are those of the full layout up
                                      to summation order.                                      */
  BICGK_OPT_PERSISTENT = 8,         /* merged classical BiCGStab (Algorithm 2) without
                                      preconditioner: run the solve as ONE cooperative launch of
                                      the persistent batch kernel (a one-system batch over this
                                      operator, kept for the next solve of the same k, whose
                                      first solve tunes its launch shape with
                                      bicgk_batch_tune_persistent; see BICGK_BATCH_PERSISTENT;
                                      host blocks are staged), with its scalar rules and a
                                      residual history.  0 (default): for small systems with at
                                      least three right-hand sides (n_rows <= 32,768,
                                      4 <= kp <= 16, n_rows*kp <= 2^19), where one launch is
                                      faster than the
                                      graph path's many; 1: never; 2: always.  Never in
                                      profiling mode.                                          */
  BICGK_OPT_SPMM32 = 9,             /* the FP32 product of bicgk_solve_mixed and bicgk_spmm_f32
                                      for kp >= 16 (kp: k rounded up to a power of two):
                                      0 (default): the sweep kernel (each block sweeps one
                                      contiguous range of rows, CSR entries prefetched a tile
                                      ahead); 1: the segment kernel (blocks stride over the
                                      rows).  Both sum every row in CSR order with FP32 FMAs:
                                      their results are bitwise equal.                         */
  BICGK_OPT_SPMM_ROWS = 10          /* the one-lane-per-row product for kp <= 2 (FP64 and FP32):
                                      0 (default): the warp-tile kernel where the rows hold at
                                      most 8 entries on average (nnz <= 8 n_rows), else the
                                      block-tile kernel; 1: always the block-tile kernel (a
                                      block stages 256-row tiles of CSR entries in shared
                                      memory between barriers); 2: always the warp-tile kernel
                                      (each warp prefetches the entries of its next 32-row tile
                                      while it multiplies the current one).  Both sum every row
                                      in CSR order: their results are bitwise equal.           */
};

/*
 * Set a launch-shape option of operator A (no counterpart in the paper: GPU
 * launch configuration).  Fewer blocks per SM leave room for kernels of other
 * streams to run alongside; two RHS groups let the FP64-bound SpMM of one group
 * overlap the bandwidth-bound vector kernels of the other (the columns never
 * interact, so every column's iterates are those of a solve of its group).
 * Cached graphs are dropped and re-captured on the next solve.  Returns
 * BICGK_E_INVALID for an unknown option or value.
 */
int bicgk_set_option(bicgk_op A, int option, int64_t value);

/*
 * Batches: many independent systems of uneven size and RHS count, solved together (no
 * counterpart in the paper; a GPU systems extension that does not change the method).
 *
 * bicgk_batch_create: system i is the CSR matrix (n_rows[i], nnz[i], rowptr[i], colidx[i],
 *   vals[i]) in space `mem` (validated and copied as by bicgk_csr_create) with k[i] right-hand
 *   sides (1..BICGK_MAX_K).  1 <= nsys <= 4096.
 * bicgk_batch_tune: autotuner.  For every system, times its streaming kernel (group 3 of
 *   Algorithm 2) over grid sizes of 1..64 double2 chunks per thread, and its SpMM over
 *   1..64 passes of rows per block (rows per CTA) and 2 or 4 columns per lane (RHS-tile width,
 *   kp >= 8), `reps` launches each, and keeps the fastest, within at most 4 SpMM blocks of 256
 *   and 1 streaming block of 512 threads per SM (the systems share the GPU in the graph mode;
 *   without tuning those are the shapes).  Writes the chosen grid sizes and tile widths to the
 *   nullable arrays [nsys].  The shapes apply to both solve modes.
 * bicgk_batch_solve: B[i], X0[i] (X0 nullable, or entries nullable), X[i] are DEVICE arrays of
 *   n_rows[i]*k[i] FP64 in the layout of bicgk_solve; every other argument as there.  iters,
 *   status, true_relres (nullable) are host arrays of sum(k) entries, systems in order.
 *   mode BICGK_BATCH_GRAPH: one CUDA-graph launch with an independent branch (set-up,
 *   conditional WHILE loop, true residual) per system; BICGK_BATCH_LOOP: bicgk_solve on each
 *   system in turn (the per-system launch loop).  Both modes run every system as one column
 *   group without dot epilogues or column compaction (BICGK_OPT_RHS_GROUPS = 1,
 *   BICGK_OPT_FUSED_DOTS = 1, BICGK_OPT_COMPACT = 1) and the same kernel sequence, so their
 *   results are bitwise equal.  Residual histories are not returned.
 *   mode BICGK_BATCH_PERSISTENT: the whole batch -- pack, set-up, every iteration of every
 *   system, true residual, unpack -- in ONE cooperative kernel launch (replayed from a CUDA
 *   graph), merged classical BiCGStab (Algorithm 2) only, M = identity, at most 1024 systems
 *   (other variants, BICGK_FLAG_JACOBI, more systems: BICGK_E_UNSUPPORTED).  A grid sized to be
 *   co-resident walks the row tiles of the systems still iterating phase by phase (Algorithm
 *   2's merged groups), each block a contiguous share of them, with a grid-wide barrier between
 *   phases; a system stops costing work once all its columns stopped.  Same scalar rules as the
 *   other modes; dot products are summed per row tile, so results differ from theirs by
 *   summation order only (and are bitwise reproducible run to run).  Every barrier wait is
 *   bounded by the batch's deadline (bicgk_batch_set_deadline; default 1 s): past it the kernel
 *   returns, the call returns BICGK_E_TIMEOUT, bicgk_last_cuda_error() names the barrier and
 *   the block, and the next solve starts from a clean state.
 * bicgk_batch_tune_persistent: autotuner of the persistent mode: rows per CTA tile (1, 2, 4 or
 *   8 passes of 256 threads: 256..2048 rows at kp <= 2, 64..512 at kp = 8) x blocks per SM (the
 *   kernel compiled for 4 blocks of up to 64 registers a thread, or 6 of up to 40) on the full
 *   co-resident grid, then the best of those on 1/2, 1/4, 1/8, 1/16 of the grid (small
 *   problems: fewer blocks in every barrier and reduction); times `reps` persistent solves of 4
 *   fixed iterations with right-hand sides of ones for each of the 12 shapes and keeps the
 *   fastest (allocates two temporary blocks).  Writes each system's rows per tile to the
 *   nullable array [nsys]; bicgk_batch_persistent_info gives the grid.
 * bicgk_batch_set_deadline: longest wait of one grid barrier of the persistent kernel, in
 *   microseconds (0..3.6e9; 0 makes every wait that does not find all blocks arrived fail).
 * bicgk_batch_last_launches: kernels the last bicgk_batch_solve launched (persistent: 1).
 * bicgk_batch_last_loop_iters: iterations the persistent kernel's loop ran in the last
 *   persistent solve (the slowest system's).
 * bicgk_batch_persistent_info: blocks of the persistent grid (co-resident: SMs x blocks per
 *   SM) and whether its launch is replayed from a CUDA graph (1: a graph of three memset nodes
 *   and one cooperative kernel node) or launched directly (0: the runtime refused the graph;
 *   graph_error is the cudaError_t it gave); nullable outputs.
 */
typedef struct bicgk_batch_s *bicgk_batch;
enum bicgk_batch_mode { BICGK_BATCH_GRAPH = 0, BICGK_BATCH_LOOP = 1, BICGK_BATCH_PERSISTENT = 2 };
int bicgk_batch_create(bicgk_batch *out, int32_t nsys, const int64_t *n_rows, const int64_t *nnz,
                       const int32_t *const *rowptr, const int32_t *const *colidx, const double *const *vals,
                       const int32_t *k, int mem, void *stream);
int bicgk_batch_tune(bicgk_batch b, int32_t reps, int32_t *vec_grid_out, int32_t *spmm_grid_out,
                     int32_t *spmm_cpl_out, void *stream);
int bicgk_batch_solve(bicgk_batch b, const double *const *B, const double *const *X0, double *const *X,
                      double rel_tol, int32_t maxit, int variant, int32_t flags, int mode, int32_t *iters,
                      int32_t *status, double *true_relres, void *stream);
int bicgk_batch_tune_persistent(bicgk_batch b, int32_t reps, int32_t *rows_per_tile_out, void *stream);
int bicgk_batch_set_deadline(bicgk_batch b, int64_t microseconds);
int bicgk_batch_last_launches(bicgk_batch b, int64_t *kernel_launches);
int bicgk_batch_last_loop_iters(bicgk_batch b, int64_t *iters);
int bicgk_batch_persistent_info(bicgk_batch b, int32_t *grid_blocks, int32_t *from_graph, int32_t *graph_error);
int bicgk_batch_destroy(bicgk_batch b);

/* Release the operator and all device memory it holds.  NULL is accepted. */
int bicgk_op_destroy(bicgk_op A);

/* Static description of an error code. */
const char *bicgk_strerror(int rc);

/* Text of the last CUDA error seen by this thread ("" if none). */
const char *bicgk_last_cuda_error(void);

/*
 * Per-kernel timing (profiling aid).  With bicgk_set_profiling(A, 1) the next
 * solves run their iteration loop without the CUDA graph, one launch at a time
 * on the caller's stream, with a CUDA event pair around every launch; the
 * column groups of a solve are the graph mode's, run one after another, so the
 * kernels timed are the ones the graph mode runs;
 * bicgk_kernel_times() then reports, for kernel class i (0 <= i < *n_out),
 * its name (with the group's column count, e.g. "spmm_phi_psi_k8"), launch
 * count and summed event time in milliseconds since the last
 * bicgk_set_profiling() call.  Results are identical to the graph mode without
 * column compaction (BICGK_OPT_COMPACT = 1; the profiling mode does not compact).
 *   names: array of *n_out C strings owned by the library (may be NULL).
 */
int bicgk_set_profiling(bicgk_op A, int on);
int bicgk_kernel_times(bicgk_op A, int32_t max_n, int32_t *n_out, const char **names, int64_t *launches,
                       double *total_ms);

/*
 * Launch statistics of the last bicgk_solve(): iterations the loop ran
 * (max over columns), kernels launched by the library in that call, and the
 * number of kernels one iteration of the loop launches.
 */
int bicgk_last_stats(bicgk_op A, int32_t *loop_iters, int64_t *kernel_launches, int32_t *kernels_per_iter);

/*
 * Column groups the last bicgk_solve() ran concurrently (1..4; BICGK_OPT_RHS_GROUPS).  Returns
 * BICGK_E_INVALID for a null argument.
 */
int bicgk_last_groups(bicgk_op A, int32_t *groups);

/* Library build identification ("bicgk <version> sm_103a"). */
const char *bicgk_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BICGK_H */
