// Persistent batched solve (one cooperative launch for many systems): shared declarations of
// bicgk_persist.cu and the C-ABI in bicgk_api.cu.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "bicgk_dev.cuh"

namespace bicgk {

constexpr int kPersistThreads = 256;  // threads per block of the persistent kernel
constexpr int kPersistStage = 2048;   // staged CSR entries per 256-row pass (kp <= 2)
constexpr int kPersistMaxSys = 1024;  // systems of one persistent batch (tile prefix in shared memory)

// Vector roles of a system in the persistent solve (pointers into its batch workspace).
enum PersistRole : int { P_X = 0, P_R, P_R0, P_P, P_V, P_S, P_T, P_B, P_NROLE };

// One system: its CSR, workspace, per-column state and caller blocks, and its place in the
// grid's tile space (tiles of (256 / max(1, kp/2)) * sub rows).
struct PersistSys {
  const int32_t *rowptr;
  const int32_t *colidx;
  const double *vals;
  double *vec[P_NROLE];  // N x kp blocks, element (i, c) at i*kp + c
  double *sc;            // [S_NSLOT][kMaxKp]
  int *fl;               // [F_NFLAG][kMaxKp]
  Ctl *ctl;              // tol, maxit, k, kp, flags, history pointer, iteration counter
  double *part;          // per-tile dot partials [ntiles][3][kp]
  const double *B;       // caller blocks, leading dimension k (X0 nullable)
  const double *X0;
  double *X;
  int64_t n;
  int64_t tile0;         // first tile of this system in the grid's tile space
  int64_t hist_len;      // history entries to reset, (maxit + 1) * kp
  int ntiles;
  int k;
  int kp;
  int sub;               // 256-thread passes per tile (rows per CTA tile, tuned)
};

// Control block of one launch (cleared by the host before each launch).
struct PersistCtl {
  unsigned long long bar;  // grid-barrier arrivals
  int err;                 // 1: a barrier wait passed its deadline
  int err_barrier;         // which barrier (1-based count within the launch)
  int err_block;           // the block that gave up first
  int running;             // systems still iterating
  int iters;               // loop iterations completed
  int pad[3];
};

struct PersistArgs {
  const PersistSys *sys;
  unsigned *tickets;  // per system: tile arrivals of the current phase
  int *live;          // per system: still iterating
  PersistCtl *pc;
  int64_t ntiles;     // tiles of all systems
  int nsys;
  int pad;
  unsigned long long deadline_ns;  // longest wait at one grid barrier
};

// Rows of one 256-thread pass for padded width kp.
inline int persist_rows_per_pass(int kp) { return kPersistThreads / (kp >= 4 ? kp / 2 : 1); }
// Co-resident blocks per SM of the persistent kernel compiled for `minb` blocks per SM (4: up to
// 64 registers a thread; 6: up to 40); 0 on error.
int persist_blocks_per_sm(int minb);
// Cooperative launch of `grid` blocks (grid must not exceed the co-resident count).
cudaError_t launch_persist(const PersistArgs &pa, int grid, int minb, cudaStream_t s);
// The same launch as a cooperative kernel node of graph g after `deps`.
cudaError_t add_persist_node(cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps, const PersistArgs &pa,
                             int grid, int minb, cudaGraphNode_t *node);

}  // namespace bicgk
