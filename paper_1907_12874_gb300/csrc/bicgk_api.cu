// Host side of libbicgk: the C-ABI declared in include/bicgk.h.
//
// A solve is three parts on the caller's stream:
//   1. pack: B (and X0) from the caller's N x k layout into the N x kp
//      workspace, control block upload, history reset;
//   2. one CUDA-graph launch: set-up kernels (r_0 = b - A x_0, norms, the
//      variant's initial vectors), a conditional WHILE node whose body is one
//      iteration of the chosen listing, and the true-residual kernels.  The
//      last reducing kernel of the body clears the loop condition when every
//      column has stopped or maxit is reached, so the iteration loop never
//      returns to the host;
//   3. unpack X and copy the per-column results to the host.
// The graph of each (variant, kp) is captured once per operator and reused.
#include <condition_variable>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <initializer_list>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "../../include/bicgk.h"
#include "bicgk_dev.cuh"
#include "bicgk_persist.cuh"
#include "bicgk_transpose.cuh"

using namespace bicgk;

namespace {

thread_local std::string g_cuda_err;

int cuda_fail(cudaError_t e, const char *what) {
  g_cuda_err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? BICGK_E_NOMEM : BICGK_E_CUDA;
}

#define CK(call)                                         \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

// One step of a kernel sequence: a streaming op, or an SpMM between workspace roles.
struct Step {
  int spmm;  // 0: streaming op `op`; 1: y = A x; 2: y = b - A x; 3: y = A x in FP32; 4: y = A^T x;
             // 5: y = A x with the dots of epilogue `op` (SpmmEpi)
  int op;
  int x, y, b;
};
Step vec(int op) { return Step{0, op, 0, 0, 0}; }
Step spmm(int x, int y) { return Step{1, -1, x, y, 0}; }
Step resid(int x, int y, int b) { return Step{2, -1, x, y, b}; }
Step spmm32(int x, int y) { return Step{3, -1, x, y, 0}; }
Step spmm_t(int x, int y) { return Step{4, -1, x, y, 0}; }
Step spmm_dot(int x, int y, int epi) { return Step{5, epi, x, y, 0}; }



struct Seq {
  std::vector<Step> setup, body, fin;
};

// FP32 inner solve of the mixed-precision refinement: merged classical BiCGStab (Algorithm 2)
// from d_0 = 0, so r_0 = b and the set-up needs no SpMM.
Seq make_inner32_seq() {
  Seq q;
  q.setup = {vec(OP32_SETUP)};
  q.body = {spmm32(V_P, V_V), vec(OP32_DELTA), vec(OP32_UPD_S), spmm32(V_S, V_T), vec(OP32_G1), vec(OP32_G3),
            vec(OP32_UPD_P)};
  return q;
}

// Kernel sequences of the twelve forms (one Step = one kernel launch).  `jacobi`: M = diag(A)
// instead of the identity copy for the forms that apply M^-1 (Algorithms 5, 6, 7).
// `opts` (SEQ_* bits): SEQ_FUSE, the merged forms take the dot kernel that follows an SpMM into
// the SpMM's epilogue (delta after v = A p, group 1 after t = A s); SEQ_THETA_S, the merged
// forms of Algorithms 2 and 5 take theta = (s, s) in the s update instead of in group 1.
enum SeqOpt : int { SEQ_FUSE = 1, SEQ_THETA_S = 2 };
Seq make_seq(int variant, bool jacobi = false, int opts = 0) {
  const bool fuse = opts & SEQ_FUSE, theta_s = opts & SEQ_THETA_S;
  const int op_s = theta_s ? OP_UPD_S_TH : OP_UPD_S, op_g1 = theta_s ? OP_G1_PP : OP_G1;
  const int epi_g1 = theta_s ? EPI_G1_PP : EPI_G1;
  Seq q;
  // y = A x followed by the dot kernel `op` of the listing, fused when `fuse`
  auto spmm_then = [](int x, int y, int op, int epi, bool fuse, std::vector<Step> &body) {
    if (fuse) {
      body.push_back(spmm_dot(x, y, epi));
    } else {
      body.push_back(spmm(x, y));
      body.push_back(vec(op));
    }
  };
  const bool fuse_delta = fuse, fuse_g1 = fuse;
  q.fin = {resid(V_X, V_TMP, V_B), vec(OP_TRUE_RES)};
  switch (variant) {
    case BICGK_CLASSICAL_MERGED:  // Algorithm 2
      q.setup = {resid(V_X, V_R, V_B), vec(OP_SETUP_C)};
      spmm_then(V_P, V_V, OP_DELTA, EPI_DELTA, fuse_delta, q.body);
      q.body.push_back(vec(op_s));
      spmm_then(V_S, V_T, op_g1, epi_g1, fuse_g1, q.body);
      q.body.push_back(vec(OP_G3));
      q.body.push_back(vec(OP_UPD_P));
      break;
    case BICGK_CLASSICAL_PLAIN:  // Algorithm 1, one kernel per line
      q.setup = {resid(V_X, V_R, V_B), vec(OP_SETUP_C)};
      q.body = {spmm(V_P, V_V), vec(OP_DELTA), vec(OP_UPD_S), spmm(V_S, V_T), vec(OP_DOT_TS),
                vec(OP_DOT_PSI), vec(OP_UPD_X_C), vec(OP_UPD_R_C), vec(OP_DOT_RR), vec(OP_DOT_RHO),
                vec(OP_UPD_P)};
      break;
    case BICGK_REORDERED_MERGED:  // Algorithm 6; v^ in V_P, t^ in V_TMP
      q.setup = {resid(V_X, V_R, V_B), vec(OP_SETUP_R)};
      if (jacobi) q.setup.push_back(vec(OP_PREC_R_Z));
      spmm_then(V_P, V_V, OP_DELTA, EPI_DELTA, fuse_delta, q.body);
      for (int op : {OP_PREC_V_S, OP_UPD_TH}) q.body.push_back(vec(op));
      q.body.push_back(spmm(V_TMP, V_T));
      for (int op : {OP_RG4, OP_PREC_T_Q, OP_UPD_R_R, OP_RFIN}) q.body.push_back(vec(op));
      break;
    case BICGK_REORDERED_PLAIN:
      q.setup = {resid(V_X, V_R, V_B), vec(OP_SETUP_R)};
      if (jacobi) q.setup.push_back(vec(OP_PREC_R_Z));
      q.body = {spmm(V_P, V_V), vec(OP_DELTA), vec(OP_PREC_V_S), vec(OP_UPD_TH), spmm(V_TMP, V_T),
                vec(OP_UPD_RT), vec(OP_DOT_T_RT), vec(OP_DOT_T_T), vec(OP_DOT_T_R0), vec(OP_DOT_RT_RT),
                vec(OP_PREC_T_Q), vec(OP_UPD_R_R), vec(OP_UPD_X_R), vec(OP_UPD_Z_R), vec(OP_UPD_VH)};
      break;
    case BICGK_PIPELINED_MERGED:  // Algorithm 4
      q.setup = {resid(V_X, V_R, V_B), vec(OP_SETUP_P), spmm(V_R, V_W), spmm(V_W, V_T), vec(OP_DOT_RW0)};
      q.body = {vec(OP_PG1), spmm(V_Z, V_V), vec(OP_PG2), vec(OP_PG3), spmm(V_W, V_T)};
      break;
    case BICGK_PIPELINED_PLAIN:
      q.setup = {resid(V_X, V_R, V_B), vec(OP_SETUP_P), spmm(V_R, V_W), spmm(V_W, V_T), vec(OP_DOT_RW0)};
      q.body = {vec(OP_PU_P), vec(OP_PU_S), vec(OP_PU_Z), vec(OP_PU_Q), vec(OP_PU_Y), vec(OP_DOT_QY),
                vec(OP_DOT_YY), vec(OP_DOT_QQ), spmm(V_Z, V_V), vec(OP_PU_X), vec(OP_PU_R), vec(OP_PU_TMP),
                vec(OP_PU_W), vec(OP_DOT_R0R), vec(OP_DOT_R0Z), vec(OP_DOT_R0W), vec(OP_DOT_R0S),
                spmm(V_W, V_T)};
      break;
    case BICGK_PRECOND_MERGED:  // Algorithm 5; p^ in V_Q, s^ in V_Y
      q.setup = {resid(V_X, V_R, V_B), vec(OP_SETUP_C)};
      q.body.push_back(vec(OP_PREC_P_Q));
      spmm_then(V_Q, V_V, OP_DELTA, EPI_DELTA, fuse_delta, q.body);
      q.body.push_back(vec(op_s));
      q.body.push_back(vec(OP_PREC_S_Y));
      spmm_then(V_Y, V_T, op_g1, epi_g1, fuse_g1, q.body);
      for (int op : {OP5_RRHO, OP5_UPD_X, OP_UPD_P}) q.body.push_back(vec(op));
      break;
    case BICGK_PRECOND_PLAIN:
      q.setup = {resid(V_X, V_R, V_B), vec(OP_SETUP_C)};
      q.body = {vec(OP_PREC_P_Q), spmm(V_Q, V_V), vec(OP_DELTA), vec(OP_UPD_S), vec(OP_PREC_S_Y), spmm(V_Y, V_T),
                vec(OP_DOT_TS), vec(OP_DOT_PSI), vec(OP5_UPD_X), vec(OP_UPD_R_C), vec(OP_DOT_RR),
                vec(OP_DOT_RHO), vec(OP_UPD_P)};
      break;
    case BICGK_PPIPE_MERGED:  // Algorithm 7; p^ in V_P, q^ in V_RT
      q.setup = {resid(V_X, V_R, V_B), vec(OP7_SETUP), vec(OP_PREC_R_RH), spmm(V_RH, V_W), vec(OP_PREC_W_WH),
                 spmm(V_WH, V_T), vec(OP_DOT_RW0)};
      q.body = {vec(OP7_L1), vec(OP7_L2), vec(OP_PREC_Z_ZH), spmm(V_ZH, V_V), vec(OP7_L4), vec(OP7_L5),
                vec(OP_PREC_W_WH), spmm(V_WH, V_T)};
      break;
    case BICGK_PPIPE_PLAIN:
      q.setup = {resid(V_X, V_R, V_B), vec(OP7_SETUP), vec(OP_PREC_R_RH), spmm(V_RH, V_W), vec(OP_PREC_W_WH),
                 spmm(V_WH, V_T), vec(OP_DOT_RW0)};
      q.body = {vec(OP7_PU_PH), vec(OP7_PU_SH), vec(OP7_PU_QH), vec(OP_PU_S), vec(OP_PU_Z), vec(OP_PU_Q),
                vec(OP_PU_Y), vec(OP_DOT_QY), vec(OP_DOT_YY), vec(OP_DOT_QQ), vec(OP_PREC_Z_ZH), spmm(V_ZH, V_V),
                vec(OP7_X), vec(OP7_TMPH), vec(OP7_RH), vec(OP_PU_R), vec(OP_PU_TMP), vec(OP_PU_W),
                vec(OP_DOT_R0R), vec(OP_DOT_R0Z), vec(OP_DOT_R0W), vec(OP_DOT_R0S), vec(OP_PREC_W_WH),
                spmm(V_WH, V_T)};
      break;
    case BICGK_IMPROVED_MERGED:  // Algorithm 3; u in V_W, f_0 = A^T r_0 in V_RT
      q.setup = {resid(V_X, V_R, V_B), vec(OP3_SETUP), spmm(V_R, V_W), spmm_t(V_R, V_RT), vec(OP3_SIG0)};
      q.body = {vec(OP3_L1), spmm(V_V, V_Q), vec(OP3_L2), vec(OP3_L3), spmm(V_R, V_W)};
      break;
    case BICGK_IMPROVED_PLAIN:
      q.setup = {resid(V_X, V_R, V_B), vec(OP3_SETUP), spmm(V_R, V_W), spmm_t(V_R, V_RT), vec(OP3_SIG0)};
      q.body = {vec(OP3_Z), vec(OP3_V), vec(OP3_S), spmm(V_V, V_Q), vec(OP3_T), vec(OP3_D_R0S), vec(OP3_D_R0Q),
                vec(OP3_D_F0S), vec(OP3_D_F0T), vec(OP3_D_ST), vec(OP3_D_TT), vec(OP3_D_SS), vec(OP_UPD_R_C),
                vec(OP3_X), spmm(V_R, V_W)};
      break;
  }
  return q;
}

int pow2_at_least(int k) {
  int p = 1;
  while (p < k) p <<= 1;
  return p;
}

struct GraphEntry {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

struct ProfEntry {
  int64_t launches = 0;
  double ms = 0.0;
};

constexpr int kMaxGroups = 4;     // column groups solved concurrently (at most)
constexpr int kSplitMinK = 8;     // smallest k that is split into two groups
constexpr int kSplit4MinK = 32;   // smallest k that is split into four groups
constexpr int kMixedSplitMinK = 16;  // the same for the mixed-precision refinement (two groups)
constexpr int kMaxLevels = 6;     // column compaction: layouts of kp, kp/2, ..., 1 columns (kp <= 64)

// Solver state of one group of columns: N x kp vectors, per-column scalars and flags, block
// partials, control block, history, the group's stream and its captured graphs.
struct Workspace {
  bool shared_state = false; // d_sc, d_fl, d_ctl point into a batch's arrays (not owned)
  int ebytes = 8;            // bytes per vector element (8: FP64, 4: FP32)
  int kp = 0;
  int64_t vstride = 0;       // doubles between consecutive workspace vectors
  double *d_vec = nullptr;
  double *d_sc = nullptr;
  int *d_fl = nullptr;
  double *d_part = nullptr;
  Ctl *d_ctl = nullptr;
  Ctl *h_ctl = nullptr;      // pinned
  double *d_hist = nullptr;
  int64_t hist_cap = 0;      // doubles
  double *h_hist = nullptr;  // pinned, hist_cap doubles
  int *h_fl = nullptr;       // pinned, F_NFLAG * kMaxKp
  double *h_sc = nullptr;    // pinned, S_NSLOT * kMaxKp
  cudaStream_t stream = nullptr;  // the group's own stream (split solves)
  cudaEvent_t done = nullptr;
  cudaEvent_t packed = nullptr;  // this group has read its columns of a host B (zero-copy path)
  // column compaction: per layout level the solve's column of each layout column, the kept source
  // columns of the current boundary, and the final per-column scalars and flags (solve's columns)
  int *d_cmap = nullptr;     // [kMaxLevels + 1][kMaxKp]
  int *d_act = nullptr;      // [kMaxKp]
  double *d_fin_sc = nullptr;  // [S_NSLOT][kMaxKp]
  int *d_fin_fl = nullptr;     // [F_NFLAG][kMaxKp]
  double *d_xf = nullptr;      // final x of a compacted solve (n_rows*kp + 2; made on first use)
  double *d_cscratch = nullptr;  // in-place compaction scratch (n_rows*kp/2 + 2)
  int64_t cbuf_elems = 0;      // n_rows*kp the two blocks above were made for
  std::map<int, GraphEntry> graphs;  // per variant, for this kp
};

}  // namespace

class CopyPool;

struct bicgk_op_s {
  int device = 0;
  int nsm = 0;
  int64_t n = 0, nnz = 0;
  int32_t *d_rowptr = nullptr, *d_col = nullptr;
  double *d_val = nullptr;
  float *d_val32 = nullptr;  // FP32 copy of the values (mixed-precision solves; made on first use)
  int stage_cap = 0;
  Workspace ws[kMaxGroups];
  Workspace ws32[kMaxGroups];  // FP32 inner-solve workspaces of the mixed-precision refinement
  bicgk_op trans = nullptr;  // operator of A^T (atomic-free transpose products; made on first use)
  int32_t *d_perm = nullptr;  // an operator made by bicgk_op_transpose: the entry of its source
                              // that each of its entries copies (to carry new values over)
  double *d_invdiag = nullptr;  // Jacobi preconditioner 1/a_ii (made on first use)
  double *d_stage[2] = {nullptr, nullptr};  // caller-layout staging for host-memory calls
  int64_t stage_elems = 0;
  void *h_bounce = nullptr;  // two page-locked chunks for copies of pageable host blocks
  CopyPool *copy_pool = nullptr;  // host threads for those copies (made with the chunks)
  cudaEvent_t bounce_ev[2] = {nullptr, nullptr};
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t fork = nullptr;
  // profiling
  bool profiling = false;
  std::map<std::string, ProfEntry> prof;
  std::vector<std::string> prof_names;
  std::vector<cudaEvent_t> ev;
  // options (0 = default)
  int opt_vec_blocks = 0;
  int opt_spmm_blocks = 0;
  int opt_groups = 0;
  int opt_fused = 0;  // BICGK_OPT_FUSED_DOTS
  int opt_theta = 0;  // BICGK_OPT_THETA_IN_S
  int opt_zero_copy = 0;  // BICGK_OPT_HOST_ZERO_COPY
  int opt_compact = 0;    // BICGK_OPT_COMPACT
  int opt_persistent = 0; // BICGK_OPT_PERSISTENT
  int opt_spmm32 = 0;     // BICGK_OPT_SPMM32
  int opt_spmm_rows = 0;  // BICGK_OPT_SPMM_ROWS
  int cur_groups = 1;     // column groups of the solve being captured or run (launch shapes)
  bicgk_batch pbatch = nullptr;  // one-system batch over this operator for the persistent kernel
  int pbatch_k = 0;
  // launch shapes chosen by the batch autotuner (0 = the per-SM rule above)
  int grid_vec_abs = 0;
  int grid_spmm_abs = 0;
  int spmm_cpl = 2;
  // last solve statistics
  int32_t last_loop_iters = 0;
  int64_t last_launches = 0;
  int32_t last_kernels_per_iter = 0;
  int32_t last_groups = 0;
};

namespace {

KArgs make_args(bicgk_op A, const Workspace &W, int use_cond, cudaGraphConditionalHandle h,
                const int *ext_act = nullptr, const double *invdiag = nullptr) {
  KArgs a;
  a.ext_act = ext_act;
  a.invdiag = invdiag;
  for (int r = 0; r < V_NVEC; ++r) a.v[r] = W.d_vec + (int64_t)r * W.vstride;
  a.sc = W.d_sc;
  a.fl = W.d_fl;
  a.part = W.d_part;
  a.ctl = W.d_ctl;
  a.n = A->n;
  a.kp = W.kp;
  a.use_cond = use_cond;
  a.cond = h;
  a.cmap = nullptr;
  a.kp_out = W.kp;
  a.compact = 0;
  return a;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Blocks of the streaming kernel of `op`: the occupancy (at most 4 per SM), or fewer by option.
// A kernel that only reduces (no vector written) runs one block per SM at kp <= 2: there each
// thread has few chunks, and the per-thread share of the block reduction (FP64 additions on the
// FP64 pipe) and the reduction tail of a larger grid cost more than the latency hiding they buy
// (128^3, k = 1: delta 18.8 -> 17.4 us, group 1 30.3 -> 25.8 us).
int vec_grid(bicgk_op A, int op, int kp = 0) {
  if (A->grid_vec_abs > 0) return A->grid_vec_abs;
  int nb = vec_blocks_per_sm(op);
  if (nb > 4) nb = 4;
  if (kp >= 1 && kp <= 2 && op_has_dots(op)) {
    int r = 0, w = 0;
    op_traffic(op, &r, &w);
    if (w == 0) nb = 1;
  }
  if (A->opt_vec_blocks > 0) {
    if (A->opt_vec_blocks < nb) nb = A->opt_vec_blocks;
  } else if (A->cur_groups >= 4) {
    nb = 1;  // four concurrent groups: the other groups' kernels fill the SMs (see auto_spmm_cap)
  }
  return A->nsm * nb;
}

// Automatic cap on the SpMM blocks per SM (0: none), by the solve's concurrency.  Measured at 128^3
// (7-point, merged classical, fixed 300 iterations, ms per iteration): with four concurrent groups
// 4 product blocks per SM and 1 streaming block per SM (vec_grid) gave 2.884 against 2.961 (k = 32)
// and 5.737 against 5.845 (k = 64): fewer blocks of each kernel let the four groups' FP64-bound
// products and bandwidth-bound updates share every SM; over the twelve forms at k = 32 (bench
// sweep) nine gained 2-5 %, the merged Pipelined and Improved forms lost 0.5-1.4 %.  With two
// groups 4 product blocks were 10 % slower, and the streaming cap helped merged classical
// (0.5-2 %) but cost other forms up to 5 %: neither is taken.  One group of kp = 4 took 0.449
// against 0.462 with 4 product blocks (every form 2-3 % faster; the streaming cap was slower).
int auto_spmm_cap(bicgk_op A, int kp) {
  if (A->cur_groups >= 4 || (A->cur_groups == 1 && kp == 4)) return 4;
  return 0;
}

// The kp <= 2 product: the warp-tile kernel for short rows (BICGK_OPT_SPMM_ROWS).
int use_warp_rows(bicgk_op A) {
  return A->opt_spmm_rows == 2 || (A->opt_spmm_rows == 0 && A->nnz <= 8 * A->n);
}

int spmm_grid(bicgk_op A, int kp, int mode) {
  if (A->grid_spmm_abs > 0) return A->grid_spmm_abs;
  int nb = spmm_blocks_per_sm(kp, mode, A->stage_cap, kp <= 2 ? use_warp_rows(A) : 0);
  const int cap = A->opt_spmm_blocks > 0 ? A->opt_spmm_blocks : auto_spmm_cap(A, kp);
  if (cap > 0 && cap < nb) nb = cap;
  return A->nsm * nb;
}

cudaError_t launch_step(bicgk_op A, const Step &st, const KArgs &a, cudaStream_t s) {
  if (st.spmm == 0) return launch_vec(st.op, a, vec_grid(A, st.op, a.kp), s);
  SpmmArgs sa;
  sa.rowptr = A->d_rowptr;
  sa.colidx = A->d_col;
  sa.vals = A->d_val;
  sa.x = a.v[st.x];
  sa.y = a.v[st.y];
  sa.b = st.spmm == 2 ? a.v[st.b] : nullptr;
  sa.n = A->n;
  sa.stage_cap = a.kp <= 2 ? A->stage_cap : 0;
  sa.warp_rows = a.kp <= 2 ? use_warp_rows(A) : 0;
  sa.cols_per_lane = a.kp >= 8 ? A->spmm_cpl : 2;
  if (st.spmm == 4) {  // y = A^T x: the SpMM kernel over the transposed copy
    bicgk_op T = A->trans;
    sa.rowptr = T->d_rowptr;
    sa.colidx = T->d_col;
    sa.vals = T->d_val;
    sa.stage_cap = a.kp <= 2 ? T->stage_cap : 0;
    sa.warp_rows = a.kp <= 2 ? use_warp_rows(T) : 0;
    return launch_spmm(a.kp, 0, sa, spmm_grid(T, a.kp, 0), s);
  }
  if (st.spmm == 3) {
    sa.vals = A->d_val32;
    sa.fp32_kernel = A->opt_spmm32;
    return launch_spmm32(a.kp, sa, A->nsm * spmm32_blocks_per_sm(a.kp, sa.stage_cap, sa.fp32_kernel, sa.warp_rows), s);
  }
  if (st.spmm == 5) {  // the fused kernel's grid: its occupancy, at most the reduction buffers' capacity
    int nb = spmm_dot_blocks_per_sm(a.kp, st.op, sa.stage_cap, sa.warp_rows);
    if (nb > kPartBlocksPerSm) nb = kPartBlocksPerSm;
    const int cap = A->opt_spmm_blocks > 0 ? A->opt_spmm_blocks : auto_spmm_cap(A, a.kp);
    if (cap > 0 && cap < nb) nb = cap;
    return launch_spmm_dot(a.kp, st.op, sa, a, A->nsm * nb, s);
  }
  const int mode = st.spmm == 2 ? 1 : 0;
  return launch_spmm(a.kp, mode, sa, spmm_grid(A, a.kp, mode), s);
}

std::string step_name(const Step &st, int kp) {
  if (st.spmm == 0) return op_name(st.op);
  if (st.spmm == 5) return std::string(spmm_dot_name(st.op)) + "_k" + std::to_string(kp);
  if (st.spmm == 3) return "spmm32_k" + std::to_string(kp);
  return std::string(st.spmm == 2 ? "spmm_resid_k" : "spmm_k") + std::to_string(kp);
}

void drop_graphs(Workspace &W) {
  for (auto &kv : W.graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  W.graphs.clear();
}

void drop_all_graphs(bicgk_op A) {
  for (Workspace &W : A->ws) drop_graphs(W);
}

void free_vectors(Workspace &W) {
  drop_graphs(W);
  cudaFree(W.d_vec);
  if (!W.shared_state) {
    cudaFree(W.d_sc);
    cudaFree(W.d_fl);
  }
  cudaFree(W.d_part);
  W.d_vec = nullptr;
  W.d_sc = nullptr;
  W.d_fl = nullptr;
  W.d_part = nullptr;
  W.kp = 0;
}

void free_workspace(Workspace &W) {
  free_vectors(W);
  if (!W.shared_state) cudaFree(W.d_ctl);
  cudaFree(W.d_hist);
  cudaFreeHost(W.h_ctl);
  cudaFreeHost(W.h_hist);
  cudaFreeHost(W.h_fl);
  cudaFreeHost(W.h_sc);
  cudaFree(W.d_cmap);
  cudaFree(W.d_act);
  cudaFree(W.d_fin_sc);
  cudaFree(W.d_fin_fl);
  cudaFree(W.d_xf);
  cudaFree(W.d_cscratch);
  if (W.done) cudaEventDestroy(W.done);
  if (W.packed) cudaEventDestroy(W.packed);
  if (W.stream) cudaStreamDestroy(W.stream);
  W = Workspace();
}

// Allocate (once) the control block, host staging and stream of a workspace, and its
// vectors for kp columns (reallocated when kp changes).
int ensure_workspace(bicgk_op A, Workspace &W, int kp) {
  if (!W.d_ctl) {
    CK(cudaMalloc(&W.d_ctl, sizeof(Ctl)));
    CK(cudaMemset(W.d_ctl, 0, sizeof(Ctl)));
    CK(cudaMallocHost(&W.h_ctl, sizeof(Ctl)));
    CK(cudaMallocHost(&W.h_fl, sizeof(int) * F_NFLAG * kMaxKp));
    CK(cudaMallocHost(&W.h_sc, sizeof(double) * S_NSLOT * kMaxKp));
    CK(cudaStreamCreateWithFlags(&W.stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&W.done, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&W.packed, cudaEventDisableTiming));
    CK(cudaMalloc(&W.d_cmap, sizeof(int) * (kMaxLevels + 1) * kMaxKp));
    CK(cudaMalloc(&W.d_act, sizeof(int) * kMaxKp));
    CK(cudaMalloc(&W.d_fin_sc, sizeof(double) * S_NSLOT * kMaxKp));
    CK(cudaMalloc(&W.d_fin_fl, sizeof(int) * F_NFLAG * kMaxKp));
  }
  if (W.kp == kp) return BICGK_OK;
  free_vectors(W);
  const int64_t elems = A->n * kp + 2;
  // vectors start on 256-byte boundaries; vstride counts doubles whatever the element type
  W.vstride = W.ebytes == 8 ? (elems + 31) / 32 * 32 : (elems + 63) / 64 * 32;
  const size_t bytes = (size_t)W.vstride * V_NVEC * sizeof(double);
  CK(cudaMalloc(&W.d_vec, bytes));
  CK(cudaMemset(W.d_vec, 0, bytes));
  CK(cudaMalloc(&W.d_sc, sizeof(double) * S_NSLOT * kMaxKp));
  CK(cudaMalloc(&W.d_fl, sizeof(int) * F_NFLAG * kMaxKp));
  CK(cudaMalloc(&W.d_part, sizeof(double) * ((size_t)A->nsm * kPartBlocksPerSm + kMaxRedGroups) * kMaxDots * kMaxKp));
  CK(cudaMemset(W.d_sc, 0, sizeof(double) * S_NSLOT * kMaxKp));
  CK(cudaMemset(W.d_fl, 0, sizeof(int) * F_NFLAG * kMaxKp));
  W.kp = kp;
  return BICGK_OK;
}

int ensure_hist(Workspace &W, int64_t elems) {
  if (elems <= W.hist_cap) return BICGK_OK;
  cudaFree(W.d_hist);
  cudaFreeHost(W.h_hist);
  W.d_hist = nullptr;
  W.h_hist = nullptr;
  W.hist_cap = 0;
  CK(cudaMalloc(&W.d_hist, sizeof(double) * elems));
  CK(cudaMallocHost(&W.h_hist, sizeof(double) * elems));
  W.hist_cap = elems;
  return BICGK_OK;
}

// Device address of a page-locked host block (cudaHostAlloc, cudaHostRegister), or nullptr for
// any other pointer: pageable host memory goes through the staged copy.
const void *mapped_host_ptr(const void *p) {
  if (!p) return nullptr;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// Copies between the device and pageable host blocks.  A cudaMemcpyAsync from or to pageable
// memory measured about 3 GB/s on these hosts (the driver stages it); instead the block moves
// through two page-locked chunks of the operator, host threads filling (or draining) one chunk
// while the DMA engine moves the other.
constexpr size_t kBounceBytes = size_t(32) << 20;

}  // namespace

// Host threads kept by an operator for its copies of pageable blocks through the bounce chunks:
// every chunk is split between the calling thread and the workers (starting threads per 32 MB
// chunk would cost about as much as the copy).  Workers that cannot start are simply absent.
class CopyPool {
 public:
  explicit CopyPool(unsigned workers) {
    try {
      for (unsigned i = 0; i < workers; ++i) th_.emplace_back([this, i] { loop(i); });
    } catch (...) {
    }
  }
  ~CopyPool() {
    {
      std::lock_guard<std::mutex> l(mu_);
      stop_ = true;
    }
    go_.notify_all();
    for (std::thread &t : th_) t.join();
  }
  // dst <- src (bytes); returns when every share is copied.
  void copy(void *dst, const void *src, size_t bytes) {
    const unsigned nw = (unsigned)th_.size();
    if (nw == 0 || bytes < (size_t(1) << 20)) {
      std::memcpy(dst, src, bytes);
      return;
    }
    const size_t part = (bytes + nw) / (nw + 1);
    {
      std::lock_guard<std::mutex> l(mu_);
      dst_ = static_cast<char *>(dst);
      src_ = static_cast<const char *>(src);
      bytes_ = bytes;
      part_ = part;
      pending_ = nw;
      ++gen_;
    }
    go_.notify_all();
    const size_t off = (size_t)nw * part;  // the caller's share: the last one
    if (off < bytes) std::memcpy(static_cast<char *>(dst) + off, static_cast<const char *>(src) + off, bytes - off);
    std::unique_lock<std::mutex> l(mu_);
    done_.wait(l, [&] { return pending_ == 0; });
  }

 private:
  void loop(unsigned i) {
    uint64_t seen = 0;
    std::unique_lock<std::mutex> l(mu_);
    for (;;) {
      go_.wait(l, [&] { return stop_ || gen_ != seen; });
      if (stop_) return;
      seen = gen_;
      char *d = dst_;
      const char *sp = src_;
      const size_t off = (size_t)i * part_, bytes = bytes_;
      const size_t len = off < bytes ? (part_ < bytes - off ? part_ : bytes - off) : 0;
      l.unlock();
      if (len) std::memcpy(d + off, sp + off, len);
      l.lock();
      if (--pending_ == 0) done_.notify_one();
    }
  }
  std::vector<std::thread> th_;
  std::mutex mu_;
  std::condition_variable go_, done_;
  char *dst_ = nullptr;
  const char *src_ = nullptr;
  size_t bytes_ = 0, part_ = 0;
  unsigned pending_ = 0;
  uint64_t gen_ = 0;
  bool stop_ = false;
};

namespace {

void parallel_memcpy(bicgk_op A, void *dst, const void *src, size_t bytes) {
  if (A->copy_pool) A->copy_pool->copy(dst, src, bytes);
  else std::memcpy(dst, src, bytes);
}

int ensure_bounce(bicgk_op A) {
  if (!A->copy_pool) {  // up to 7 workers beside the calling thread
    const unsigned hw = std::thread::hardware_concurrency();
    const unsigned nt = hw < 8 ? (hw ? hw : 1) : 8;
    try {
      A->copy_pool = new CopyPool(nt - 1);
    } catch (...) {
      A->copy_pool = nullptr;  // plain copies
    }
  }
  if (A->h_bounce) return BICGK_OK;
  for (int i = 0; i < 2; ++i)
    if (!A->bounce_ev[i]) CK(cudaEventCreateWithFlags(&A->bounce_ev[i], cudaEventDisableTiming));
  CK(cudaMallocHost(&A->h_bounce, 2 * kBounceBytes));
  return BICGK_OK;
}

// dst (device) <- src (pageable host), queued on s; src may be reused when this returns.
int copy_in_pageable(bicgk_op A, void *dst, const void *src, size_t bytes, cudaStream_t s) {
  int rc = ensure_bounce(A);
  if (rc) return rc;
  for (size_t off = 0, i = 0; off < bytes; off += kBounceBytes, ++i) {
    const int slot = (int)(i & 1);
    const size_t len = kBounceBytes < bytes - off ? kBounceBytes : bytes - off;
    char *b = static_cast<char *>(A->h_bounce) + slot * kBounceBytes;
    CK(cudaEventSynchronize(A->bounce_ev[slot]));  // the chunk's previous copy has finished
    parallel_memcpy(A, b, static_cast<const char *>(src) + off, len);
    CK(cudaMemcpyAsync(static_cast<char *>(dst) + off, b, len, cudaMemcpyHostToDevice, s));
    CK(cudaEventRecord(A->bounce_ev[slot], s));
  }
  return BICGK_OK;
}

// dst (pageable host) <- src (device) after the work queued on s; returns when dst is written.
int copy_out_pageable(bicgk_op A, void *dst, const void *src, size_t bytes, cudaStream_t s) {
  int rc = ensure_bounce(A);
  if (rc) return rc;
  const size_t n = (bytes + kBounceBytes - 1) / kBounceBytes;
  for (size_t i = 0; i < n && i < 2; ++i) {  // two chunks in flight
    const size_t off = i * kBounceBytes, len = kBounceBytes < bytes - off ? kBounceBytes : bytes - off;
    CK(cudaMemcpyAsync(static_cast<char *>(A->h_bounce) + (i & 1) * kBounceBytes,
                       static_cast<const char *>(src) + off, len, cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(A->bounce_ev[i & 1], s));
  }
  for (size_t i = 0; i < n; ++i) {
    const int slot = (int)(i & 1);
    const size_t off = i * kBounceBytes, len = kBounceBytes < bytes - off ? kBounceBytes : bytes - off;
    CK(cudaEventSynchronize(A->bounce_ev[slot]));
    parallel_memcpy(A, static_cast<char *>(dst) + off, static_cast<char *>(A->h_bounce) + slot * kBounceBytes, len);
    if (i + 2 < n) {  // the drained chunk takes the one after next
      const size_t o2 = (i + 2) * kBounceBytes, l2 = kBounceBytes < bytes - o2 ? kBounceBytes : bytes - o2;
      CK(cudaMemcpyAsync(static_cast<char *>(A->h_bounce) + slot * kBounceBytes, static_cast<const char *>(src) + o2,
                         l2, cudaMemcpyDeviceToHost, s));
      CK(cudaEventRecord(A->bounce_ev[slot], s));
    }
  }
  return BICGK_OK;
}

// Host block -> device: a plain copy from page-locked memory, the chunked one from pageable.
int copy_in_host(bicgk_op A, void *dst, const void *src, size_t bytes, cudaStream_t s) {
  if (mapped_host_ptr(src)) {
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
    return BICGK_OK;
  }
  return copy_in_pageable(A, dst, src, bytes, s);
}
int copy_out_host(bicgk_op A, void *dst, const void *src, size_t bytes, cudaStream_t s) {
  if (mapped_host_ptr(dst)) {
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s));
    return BICGK_OK;
  }
  return copy_out_pageable(A, dst, src, bytes, s);
}

int ensure_stage(bicgk_op A, int64_t elems) {
  if (elems <= A->stage_elems) return BICGK_OK;
  cudaFree(A->d_stage[0]);
  cudaFree(A->d_stage[1]);
  A->d_stage[0] = A->d_stage[1] = nullptr;
  A->stage_elems = 0;
  CK(cudaMalloc(&A->d_stage[0], sizeof(double) * elems));
  CK(cudaMalloc(&A->d_stage[1], sizeof(double) * elems));
  A->stage_elems = elems;
  return BICGK_OK;
}

// Capture q.setup + WHILE(q.body) + q.fin for workspace W into one graph.
int build_graph_seq(bicgk_op A, Workspace &W, const Seq &q, const int *ext_act, GraphEntry *ge,
                    const double *invdiag = nullptr) {
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  ge->graph = g;
  cudaGraphConditionalHandle h;
  CK(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
  const KArgs a = make_args(A, W, 1, h, ext_act, invdiag);
  cudaStream_t cs = A->cap_stream;
  // set-up
  CK(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  for (const Step &st : q.setup) {
    cudaError_t e = launch_step(A, st, a, cs);
    if (e != cudaSuccess) {
      cudaGraph_t dummy;
      cudaStreamEndCapture(cs, &dummy);
      return cuda_fail(e, "capture set-up");
    }
  }
  cudaStreamCaptureStatus cst;
  const cudaGraphNode_t *deps = nullptr;
  size_t ndeps = 0;
  CK(cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps));
  std::vector<cudaGraphNode_t> leaves(deps, deps + ndeps);
  cudaGraph_t tmp;
  CK(cudaStreamEndCapture(cs, &tmp));
  // WHILE node: one iteration of the listing per pass
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t wnode;
  CK(cudaGraphAddNode(&wnode, g, leaves.data(), nullptr, leaves.size(), &p));
  cudaGraph_t body = p.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  for (const Step &st : q.body) {
    cudaError_t e = launch_step(A, st, a, cs);
    if (e != cudaSuccess) {
      cudaGraph_t dummy;
      cudaStreamEndCapture(cs, &dummy);
      return cuda_fail(e, "capture body");
    }
  }
  CK(cudaStreamEndCapture(cs, &tmp));
  if (!q.fin.empty()) {
    CK(cudaStreamBeginCaptureToGraph(cs, g, &wnode, nullptr, 1, cudaStreamCaptureModeThreadLocal));
    for (const Step &st : q.fin) {
      cudaError_t e = launch_step(A, st, a, cs);
      if (e != cudaSuccess) {
        cudaGraph_t dummy;
        cudaStreamEndCapture(cs, &dummy);
        return cuda_fail(e, "capture final");
      }
    }
    CK(cudaStreamEndCapture(cs, &tmp));
  }
  CK(cudaGraphInstantiate(&ge->exec, g, 0));
  return BICGK_OK;
}

// Roles of a compacted form: the live vectors at the top of an iteration (read before written in
// the loop body; gathered at a boundary), a slot the form never uses for each of them (the odd
// levels' copy), and every role the loop uses.
struct CompactRoles {
  int nlive = 0;
  int live[6] = {0, 0, 0, 0, 0, 0};
  int alt[6] = {0, 0, 0, 0, 0, 0};
  unsigned loop_mask = 0;
  unsigned inplace_mask = 0;  // roles compacted in place through a scratch block (no second copy)
  unsigned live_mask() const {
    unsigned m = 0;
    for (int i = 0; i < nlive; ++i) m |= 1u << live[i];
    return m;
  }
};

CompactRoles compact_roles(int variant) {
  CompactRoles c;
  auto mask = [](std::initializer_list<int> roles) {
    unsigned m = 0;
    for (int r : roles) m |= 1u << r;
    return m;
  };
  if (variant == BICGK_PIPELINED_MERGED || variant == BICGK_PIPELINED_PLAIN || variant == BICGK_PPIPE_MERGED ||
      variant == BICGK_PPIPE_PLAIN || variant == BICGK_IMPROVED_MERGED || variant == BICGK_IMPROVED_PLAIN) {
    // Algorithms 3, 4, 7 carry many vectors from one iteration to the next and use nearly every
    // slot: every role but b is compacted in place (the ones the loop does not carry cost a
    // copy of dead data at the few boundaries a solve reaches)
    for (int r = 0; r < V_NVEC; ++r)
      if (r != V_B) c.inplace_mask |= 1u << r;
    return c;
  }
  if (variant == BICGK_REORDERED_MERGED || variant == BICGK_REORDERED_PLAIN) {
    // Algorithm 6: x, r, r^0, v^ (in V_P) and z; the loop also uses v, s, t, q, t^, r~
    const int live[5] = {V_X, V_R, V_R0, V_P, V_Z}, alt[5] = {V_W, V_Y, V_SH, V_ZH, V_RH};
    c.nlive = 5;
    for (int i = 0; i < 5; ++i) c.live[i] = live[i], c.alt[i] = alt[i];
    c.loop_mask = mask({V_X, V_R, V_R0, V_P, V_V, V_S, V_T, V_Z, V_Q, V_TMP, V_RT});
  } else {
    // Algorithms 1, 2, 5: x, r, r^0, p; the loop also uses v, s, t and p^, s^ (in V_Q, V_Y)
    const int live[4] = {V_X, V_R, V_R0, V_P}, alt[4] = {V_W, V_Z, V_RT, V_SH};
    c.nlive = 4;
    for (int i = 0; i < 4; ++i) c.live[i] = live[i], c.alt[i] = alt[i];
    c.loop_mask = mask({V_X, V_R, V_R0, V_P, V_V, V_S, V_T, V_Q, V_Y});
  }
  return c;
}

// Arguments of compaction level l (kp0 >> l columns): the live vectors alternate between two slot
// sets so that each boundary gathers into vectors the previous level does not read; the other
// roles of the loop are rewritten every iteration before they are read.
KArgs level_args(bicgk_op A, const Workspace &W, int l, cudaGraphConditionalHandle h, const double *invdiag,
                 const CompactRoles &cr) {
  KArgs a = make_args(A, W, 1, h, nullptr, invdiag);
  a.kp = W.kp >> l;
  a.kp_out = W.kp;
  a.cmap = l > 0 ? W.d_cmap + l * kMaxKp : nullptr;
  a.compact = a.kp > 1;
  if (l & 1)
    for (int i = 0; i < cr.nlive; ++i) a.v[cr.live[i]] = W.d_vec + (int64_t)cr.alt[i] * W.vstride;
  return a;
}

// Arguments of the final kernels and the unpack of a compacted solve: the full layout, x from the
// final block, the final per-column scalars and flags.
KArgs final_args(bicgk_op A, const Workspace &W, const double *invdiag) {
  KArgs a = make_args(A, W, 0, cudaGraphConditionalHandle{}, nullptr, invdiag);
  a.v[V_X] = W.d_xf;
  a.sc = W.d_fin_sc;
  a.fl = W.d_fin_fl;
  return a;
}

// Whether a solve's group of kp columns narrows its layout as its columns stop
// (BICGK_OPT_COMPACT): every form, with the roles listed above.
bool compact_columns(bicgk_op A, int variant, int kp) {
  (void)variant;
  return A->opt_compact != 1 && !A->profiling && kp >= 2;
}

// The graph of a compacted solve: set-up; WHILE(level 0); then per level l = 1..L a compaction
// boundary (plan + move kernels) and WHILE(level l); a last boundary that writes the final values
// of the last level; the final kernels on the full layout.  Levels that are not reached cost their
// boundary kernels' launches only (they return at once).
int build_graph_compact(bicgk_op A, Workspace &W, const Seq &q, GraphEntry *ge, const double *invdiag,
                        int variant) {
  const CompactRoles cr = compact_roles(variant);
  const int64_t elems = A->n * W.kp;
  if (W.cbuf_elems != elems) {
    cudaFree(W.d_xf);
    cudaFree(W.d_cscratch);
    W.d_xf = W.d_cscratch = nullptr;
    W.cbuf_elems = 0;
    CK(cudaMalloc(&W.d_xf, sizeof(double) * (elems + 2)));
    CK(cudaMalloc(&W.d_cscratch, sizeof(double) * (elems / 2 + 2)));
    W.cbuf_elems = elems;
  }
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  ge->graph = g;
  int L = 0;
  while ((W.kp >> L) > 1) ++L;
  cudaGraphConditionalHandle h[kMaxLevels + 1];
  for (int l = 0; l <= L; ++l) CK(cudaGraphConditionalHandleCreate(&h[l], g, 0, 0));
  KArgs lv[kMaxLevels + 1];
  for (int l = 0; l <= L; ++l) lv[l] = level_args(A, W, l, h[l], invdiag, cr);
  const KArgs af = final_args(A, W, invdiag);
  double *xf = W.d_xf;
  cudaStream_t cs = A->cap_stream;
  cudaGraph_t tmp;
  auto fail = [&](cudaError_t e, const char *what) {
    cudaGraph_t dummy;
    cudaStreamEndCapture(cs, &dummy);
    return cuda_fail(e, what);
  };
  // set-up, then per level: WHILE(body), boundary
  CK(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  for (const Step &st : q.setup) {
    cudaError_t e = launch_step(A, st, lv[0], cs);
    if (e != cudaSuccess) return fail(e, "capture set-up");
  }
  for (int l = 0; l <= L; ++l) {
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    CK(cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps));
    std::vector<cudaGraphNode_t> leaves(deps, deps + ndeps);
    CK(cudaStreamEndCapture(cs, &tmp));
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h[l];
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t wnode;
    CK(cudaGraphAddNode(&wnode, g, leaves.data(), nullptr, leaves.size(), &p));
    CK(cudaStreamBeginCaptureToGraph(cs, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                     cudaStreamCaptureModeThreadLocal));
    for (const Step &st : q.body) {
      cudaError_t e = launch_step(A, st, lv[l], cs);
      if (e != cudaSuccess) return fail(e, "capture body");
    }
    CK(cudaStreamEndCapture(cs, &tmp));
    CK(cudaStreamBeginCaptureToGraph(cs, g, &wnode, nullptr, 1, cudaStreamCaptureModeThreadLocal));
    const bool last = l == L;
    const KArgs &dst = last ? lv[l] : lv[l + 1];
    cudaError_t e = launch_compact(lv[l], dst, l + 1, last ? 1 : 0, last ? h[l] : h[l + 1], W.d_fin_sc,
                                   W.d_fin_fl, last ? W.d_act : W.d_cmap + (l + 1) * kMaxKp, W.d_act, xf,
                                   cr.live_mask(), cr.loop_mask, A->nsm * 4, cs);
    for (int r = 0; e == cudaSuccess && !last && r < V_NVEC; ++r)
      if ((cr.inplace_mask >> r) & 1u) e = launch_compact_inplace(lv[l], dst, W.d_act, r, W.d_cscratch, A->nsm * 4, cs);
    if (e != cudaSuccess) return fail(e, "capture compaction");
  }
  for (const Step &st : q.fin) {
    cudaError_t e = launch_step(A, st, af, cs);
    if (e != cudaSuccess) return fail(e, "capture final");
  }
  CK(cudaStreamEndCapture(cs, &tmp));
  CK(cudaGraphInstantiate(&ge->exec, g, 0));
  return BICGK_OK;
}

// Column groups of a solve of k columns (BICGK_OPT_RHS_GROUPS; the profiling mode runs the same
// groups one after another).  Automatic: two from k = 8, four
// from k = 32.  Each group's loop runs until its own slowest column stops, and a group that
// finishes early leaves the GPU to the others, so smaller groups waste fewer iterations on
// stopped columns: at 128^3, k = 32 four groups of 8 cost the same per iteration as two of 16
// (3,033 vs 3,047 us) and solved 2.7 % more column-iterations per second over nine right-hand
// sides (k = 64: -1.2 % per iteration, +2.3 % per solve).  At k = 16 four groups of 4 were 2 %
// slower per iteration and even per solve; at k = 8 two groups of 4 beat one of 8 (830 vs
// 872 us per iteration, +4.4 % per solve); at k = 4 two groups of 2 were 17 % slower.
int num_groups(bicgk_op A, int k) {
  if (A->opt_groups == 0) return k >= kSplit4MinK ? 4 : k >= kSplitMinK ? 2 : 1;
  return A->opt_groups < k ? A->opt_groups : k;
}

// Whether a solve of k columns takes the merged forms' dot kernels into the SpMM epilogues
// (BICGK_OPT_FUSED_DOTS).  Automatic: when the columns are split into concurrent groups.  There
// it was measured faster with two groups (fewer kernels per iteration for the groups to share the
// GPU: 3-4 % at k = 16 and 32; two groups of 4 at k = 8 with it beat one group of 8 without it)
// and neutral to 2 % faster with four groups of 8 at k = 32; with one group the fused SpMM's
// grid-wide reduction costs more than the separate dot kernel (2-8 % slower at k = 1..8).
// Profiling mode decides the same way.
bool fuse_dots(bicgk_op A, int k) {
  if (A->opt_fused == 1) return false;
  if (A->opt_fused == 2) return true;
  return num_groups(A, k) >= 2;
}

// Whether theta = (s, s) of Algorithms 2 and 5 is taken in the s update (BICGK_OPT_THETA_IN_S).
// Automatic, from fixed-iteration timings at 128^3 (7-point stencil): from k = 4 on, where the
// s update stays bandwidth-bound with the extra FMA and group 1 sheds a third of its FP64 work
// (0.5-2 % per iteration at k = 4..16, 3 % at k = 32 without the dot epilogues), except for the
// classical form with the epilogues in two groups, where it gained nothing at k = 32 and cost 1 %
// at k = 16 (with four groups of 8 at k = 32 it gains 0.8 %).  At k = 1 the reduction added to
// the s update costs more than it saves.
bool theta_in_s(bicgk_op A, int k, int variant) {
  if (A->opt_theta == 1) return false;
  if (A->opt_theta == 2) return true;
  return k >= 4 && !(variant == BICGK_CLASSICAL_MERGED && fuse_dots(A, k) && num_groups(A, k) == 2);
}

int seq_opts(bicgk_op A, int k, int variant) {
  return (fuse_dots(A, k) ? SEQ_FUSE : 0) | (theta_in_s(A, k, variant) ? SEQ_THETA_S : 0);
}

// Whether bicgk_solve runs this solve in the persistent kernel (BICGK_OPT_PERSISTENT): merged
// classical BiCGStab without preconditioner, not in profiling mode.  Automatic: small systems with
// at least two right-hand sides -- at most 32,768 rows, kp <= 16 and rows x kp <= 2^19 -- where
// one launch beats the graph path's launches (measured on the h-scaled 7-point operator to 1e-8:
// 12^3..32^3 with k = 2..16 1.07-1.80x faster; k = 1 and from 40^3 on the graph path is as fast or
// faster, because each thread of the persistent kernel keeps fewer memory operations in flight).
bool use_persistent(bicgk_op A, int k, int variant, bool jacobi) {
  if (A->opt_persistent == 1 || A->profiling || variant != BICGK_CLASSICAL_MERGED || jacobi) return false;
  if (A->opt_persistent == 2) return true;
  const int kp = pow2_at_least(k);
  return kp >= 4 && kp <= 16 && A->n <= 32768 && A->n * kp <= (int64_t(1) << 19);
}

int build_graph(bicgk_op A, Workspace &W, int variant, bool jacobi, int opts, GraphEntry *ge) {
  return build_graph_seq(A, W, make_seq(variant, jacobi, opts), nullptr, ge, jacobi ? A->d_invdiag : nullptr);
}

// What a form needs beyond the operator: the transposed copy (Algorithm 3), the Jacobi diagonal.
int ensure_variant_data(bicgk_op A, int variant, bool jacobi, cudaStream_t s) {
  if ((variant == BICGK_IMPROVED_PLAIN || variant == BICGK_IMPROVED_MERGED) && !A->trans) {
    int rc = bicgk_op_transpose(A, &A->trans, s);
    if (rc) return rc;
  }
  if (jacobi && !A->d_invdiag) {
    CK(cudaMalloc(&A->d_invdiag, sizeof(double) * A->n));
    CK(launch_invdiag(A->d_rowptr, A->d_col, A->d_val, A->d_invdiag, A->n, s));
  }
  return BICGK_OK;
}

int check_device(int *dev, int *nsm) {
  CK(cudaGetDevice(dev));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, *dev));
  if (prop.major != 10 || prop.minor != 3) {
    g_cuda_err = std::string("device is sm_") + std::to_string(prop.major) + std::to_string(prop.minor) +
                 ", library is built for sm_103a";
    return BICGK_E_UNSUPPORTED;
  }
  *nsm = prop.multiProcessorCount;
  return BICGK_OK;
}

// An operator with device arrays for n rows and nnz entries (contents undefined), its capture
// stream and fork event.
int op_alloc(bicgk_op *out, int dev, int nsm, int64_t n, int64_t nnz) {
  bicgk_op A = new bicgk_op_s();
  A->device = dev;
  A->nsm = nsm;
  A->n = n;
  A->nnz = nnz;
  cudaError_t e;
  // pad by 16 bytes so vectorised reads of the last entries stay inside the allocation
  if ((e = cudaMalloc(&A->d_rowptr, sizeof(int32_t) * (n + 1) + 16)) != cudaSuccess ||
      (e = cudaMalloc(&A->d_col, sizeof(int32_t) * nnz + 16)) != cudaSuccess ||
      (e = cudaMalloc(&A->d_val, sizeof(double) * nnz + 16)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&A->cap_stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&A->fork, cudaEventDisableTiming)) != cudaSuccess) {
    bicgk_op_destroy(A);
    return cuda_fail(e, "operator allocation");
  }
  *out = A;
  return BICGK_OK;
}

// Arrays an operator derives from its values (FP32 copy, Jacobi diagonal), recomputed after the
// values changed.
int refresh_derived(bicgk_op A, cudaStream_t s) {
  if (A->d_val32) CK(launch_to_float(A->d_val, A->d_val32, A->nnz, s));
  if (A->d_invdiag) CK(launch_invdiag(A->d_rowptr, A->d_col, A->d_val, A->d_invdiag, A->n, s));
  return BICGK_OK;
}

void prof_record(bicgk_op A, const std::string &name, float ms) {
  ProfEntry &e = A->prof[name];
  e.launches += 1;
  e.ms += ms;
}

// Profiling mode: the loop runs from the host, one launch at a time, each bracketed by events.
int run_profiled_seq(bicgk_op A, Workspace &W, const Seq &q, const KArgs &a, cudaStream_t s) {
  const size_t nmax = q.body.size() > q.setup.size() ? q.body.size() : q.setup.size();
  while (A->ev.size() < 2 * (nmax + 2)) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    A->ev.push_back(e);
  }
  auto run_list = [&](const std::vector<Step> &steps) -> int {
    for (size_t i = 0; i < steps.size(); ++i) {
      CK(cudaEventRecord(A->ev[2 * i], s));
      CK(launch_step(A, steps[i], a, s));
      CK(cudaEventRecord(A->ev[2 * i + 1], s));
    }
    CK(cudaMemcpyAsync(W.h_ctl, W.d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (size_t i = 0; i < steps.size(); ++i) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, A->ev[2 * i], A->ev[2 * i + 1]));
      prof_record(A, step_name(steps[i], a.kp), ms);
    }
    return BICGK_OK;
  };
  int rc = run_list(q.setup);
  if (rc) return rc;
  bool go = W.h_ctl->any_active && W.h_ctl->maxit > 0;
  while (go) {
    rc = run_list(q.body);
    if (rc) return rc;
    go = W.h_ctl->any_active && W.h_ctl->iter < W.h_ctl->maxit;
  }
  return run_list(q.fin);
}

int run_profiled(bicgk_op A, Workspace &W, int variant, bool jacobi, int opts, const KArgs &a, cudaStream_t s) {
  return run_profiled_seq(A, W, make_seq(variant, jacobi, opts), a, s);
}

}  // namespace

// Defined with the batches below.
int persist_single(bicgk_op A, int32_t k, const double *B, const double *X0, double rel_tol, int32_t maxit,
                   int32_t flags, double *X, int32_t *iters, int32_t *status, double *resid_hist,
                   double *true_relres, cudaStream_t s);

extern "C" {

const char *bicgk_version(void) { return "bicgk 0.2 sm_103a"; }

const char *bicgk_strerror(int rc) {
  switch (rc) {
    case BICGK_OK: return "ok";
    case BICGK_E_INVALID: return "invalid argument";
    case BICGK_E_BAD_CSR: return "malformed CSR matrix";
    case BICGK_E_CUDA: return "CUDA runtime error";
    case BICGK_E_NOMEM: return "out of memory";
    case BICGK_E_UNSUPPORTED: return "unsupported configuration";
    case BICGK_E_TIMEOUT: return "a device-side wait passed its deadline";
    default: return "unknown error";
  }
}

const char *bicgk_last_cuda_error(void) { return g_cuda_err.c_str(); }

int bicgk_csr_create(bicgk_op *out, int64_t n_rows, int64_t nnz, const int32_t *rowptr, const int32_t *colidx,
                     const double *vals, int mem, void *stream) {
  if (!out || n_rows < 1 || nnz < 0 || n_rows > INT32_MAX - 1 || nnz > INT32_MAX || !rowptr ||
      (nnz > 0 && (!colidx || !vals)) || (mem != BICGK_MEM_HOST && mem != BICGK_MEM_DEVICE))
    return BICGK_E_INVALID;
  *out = nullptr;
  int dev = 0, nsm = 0;
  int rc = check_device(&dev, &nsm);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  // validate on the host
  std::vector<int32_t> hrp, hci;
  const int32_t *rp = rowptr, *cix = colidx;
  if (mem == BICGK_MEM_DEVICE) {
    hrp.resize(n_rows + 1);
    hci.resize(nnz);
    CK(cudaMemcpyAsync(hrp.data(), rowptr, sizeof(int32_t) * (n_rows + 1), cudaMemcpyDeviceToHost, s));
    if (nnz) CK(cudaMemcpyAsync(hci.data(), colidx, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    rp = hrp.data();
    cix = hci.data();
  }
  if (rp[0] != 0 || rp[n_rows] != nnz) return BICGK_E_BAD_CSR;
  for (int64_t i = 0; i < n_rows; ++i)
    if (rp[i + 1] < rp[i]) return BICGK_E_BAD_CSR;
  for (int64_t e = 0; e < nnz; ++e)
    if (cix[e] < 0 || cix[e] >= n_rows) return BICGK_E_BAD_CSR;
  // largest tile (kSpmmTileRows rows) for the staged SpMM
  int64_t maxtile = 0;
  for (int64_t r0 = 0; r0 < n_rows; r0 += kSpmmTileRows) {
    const int64_t r1 = r0 + kSpmmTileRows < n_rows ? r0 + kSpmmTileRows : n_rows;
    const int64_t t = rp[r1] - rp[r0];
    if (t > maxtile) maxtile = t;
  }
  bicgk_op A = nullptr;
  if ((rc = op_alloc(&A, dev, nsm, n_rows, nnz))) return rc;
  A->stage_cap = (int)(maxtile < kSpmmStageMax ? maxtile : kSpmmStageMax);
  const cudaMemcpyKind kind = mem == BICGK_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(A->d_rowptr, rowptr, sizeof(int32_t) * (n_rows + 1), kind, s)) != cudaSuccess ||
      (nnz && (e = cudaMemcpyAsync(A->d_col, colidx, sizeof(int32_t) * nnz, kind, s)) != cudaSuccess) ||
      (nnz && (e = cudaMemcpyAsync(A->d_val, vals, sizeof(double) * nnz, kind, s)) != cudaSuccess) ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    bicgk_op_destroy(A);
    return cuda_fail(e, "bicgk_csr_create");
  }
  *out = A;
  return BICGK_OK;
}

int bicgk_op_destroy(bicgk_op A) {
  if (!A) return BICGK_OK;
  cudaDeviceSynchronize();
  if (A->pbatch) bicgk_batch_destroy(A->pbatch);  // borrows A: leaves it alone
  if (A->trans) bicgk_op_destroy(A->trans);
  cudaFree(A->d_invdiag);
  for (Workspace &W : A->ws) free_workspace(W);
  for (Workspace &V : A->ws32) free_workspace(V);
  cudaFree(A->d_val32);
  cudaFree(A->d_perm);
  cudaFree(A->d_rowptr);
  cudaFree(A->d_col);
  cudaFree(A->d_val);
  cudaFree(A->d_stage[0]);
  cudaFree(A->d_stage[1]);
  cudaFreeHost(A->h_bounce);
  delete A->copy_pool;
  for (cudaEvent_t e : A->bounce_ev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : A->ev) cudaEventDestroy(e);
  if (A->fork) cudaEventDestroy(A->fork);
  if (A->cap_stream) cudaStreamDestroy(A->cap_stream);
  delete A;
  return BICGK_OK;
}

int bicgk_spmm(bicgk_op A, int32_t k, const double *X, double *Y, void *stream) {
  if (!A || !X || !Y || k < 1 || X == Y) return BICGK_E_INVALID;
  if (k > BICGK_MAX_K) return BICGK_E_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  const int kp = pow2_at_least(k);
  SpmmArgs sa;
  sa.rowptr = A->d_rowptr;
  sa.colidx = A->d_col;
  sa.vals = A->d_val;
  sa.b = nullptr;
  sa.n = A->n;
  sa.stage_cap = kp <= 2 ? A->stage_cap : 0;
  sa.warp_rows = kp <= 2 ? use_warp_rows(A) : 0;
  // the caller's layout is the kernel layout when k is a power of two; the kernels read and
  // write kp >= 2 blocks as 16-byte vectors, so the caller's arrays must then be 16-byte aligned
  if (kp == k && (kp == 1 || (aligned16(X) && aligned16(Y)))) {
    sa.x = X;
    sa.y = Y;
    CK(launch_spmm(kp, 0, sa, spmm_grid(A, kp, 0), s));
    return BICGK_OK;
  }
  Workspace &W = A->ws[0];
  int rc = ensure_workspace(A, W, kp);
  if (rc) return rc;
  const KArgs a = make_args(A, W, 0, cudaGraphConditionalHandle{});
  CK(launch_pack(X, nullptr, k, k, a, s));
  sa.x = a.v[V_B];
  sa.y = a.v[V_TMP];
  CK(launch_spmm(kp, 0, sa, spmm_grid(A, kp, 0), s));
  CK(launch_unpack_role(Y, k, k, a, V_TMP, 0, s));
  return BICGK_OK;
}

int bicgk_spmm_f32(bicgk_op A, int32_t k, const float *X, float *Y, void *stream) {
  if (!A || !X || !Y || k < 1 || (const void *)X == (const void *)Y) return BICGK_E_INVALID;
  if (k > BICGK_MAX_K) return BICGK_E_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  const int kp = pow2_at_least(k);
  if (!A->d_val32) {
    CK(cudaMalloc(&A->d_val32, sizeof(float) * A->nnz + 16));
    CK(launch_to_float(A->d_val, A->d_val32, A->nnz, s));
  }
  SpmmArgs sa;
  sa.rowptr = A->d_rowptr;
  sa.colidx = A->d_col;
  sa.vals = A->d_val32;
  sa.b = nullptr;
  sa.n = A->n;
  sa.stage_cap = kp <= 2 ? A->stage_cap : 0;
  sa.cols_per_lane = 2;
  sa.fp32_kernel = A->opt_spmm32;
  sa.warp_rows = kp <= 2 ? use_warp_rows(A) : 0;
  const int grid = A->nsm * spmm32_blocks_per_sm(kp, sa.stage_cap, sa.fp32_kernel, sa.warp_rows);
  if (kp == k && (kp == 1 || (aligned16(X) && aligned16(Y)))) {
    sa.x = X;
    sa.y = Y;
    CK(launch_spmm32(kp, sa, grid, s));
    return BICGK_OK;
  }
  // pad to kp columns (zeros) in the FP32 workspace with pitched copies, multiply, copy back
  Workspace &V = A->ws32[0];
  V.ebytes = 4;
  int rc = ensure_workspace(A, V, kp);
  if (rc) return rc;
  float *xb = reinterpret_cast<float *>(V.d_vec + (int64_t)V_B * V.vstride);
  float *yb = reinterpret_cast<float *>(V.d_vec + (int64_t)V_TMP * V.vstride);
  const size_t w = sizeof(float) * (size_t)k, wp = sizeof(float) * (size_t)kp;
  if (kp != k) CK(cudaMemsetAsync(xb, 0, wp * (size_t)A->n, s));
  CK(cudaMemcpy2DAsync(xb, wp, X, w, w, (size_t)A->n, cudaMemcpyDeviceToDevice, s));
  sa.x = xb;
  sa.y = yb;
  CK(launch_spmm32(kp, sa, grid, s));
  CK(cudaMemcpy2DAsync(Y, w, yb, wp, w, (size_t)A->n, cudaMemcpyDeviceToDevice, s));
  return BICGK_OK;
}

int bicgk_solve(bicgk_op A, int32_t k, const double *B, const double *X0, double rel_tol, int32_t maxit,
                int variant, int32_t flags, int mem, double *X, int32_t *iters, int32_t *status,
                double *resid_hist, double *true_relres, void *stream) {
  if (!A || !B || !X || !iters || !status || k < 1 || !(rel_tol >= 0.0) || maxit < 0 || maxit > 10000000 ||
      variant < 0 || variant > 11 || (mem != BICGK_MEM_HOST && mem != BICGK_MEM_DEVICE) || (flags & ~3))
    return BICGK_E_INVALID;
  if (k > BICGK_MAX_K) return BICGK_E_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  const bool jacobi = (flags & BICGK_FLAG_JACOBI) != 0;
  if (use_persistent(A, k, variant, jacobi)) {
    if (mem == BICGK_MEM_DEVICE)
      return persist_single(A, k, B, X0, rel_tol, maxit, flags, X, iters, status, resid_hist, true_relres, s);
    // host blocks: staged through the operator's device blocks
    int rc = ensure_stage(A, A->n * k);
    if (rc) return rc;
    if ((rc = copy_in_host(A, A->d_stage[0], B, sizeof(double) * A->n * k, s))) return rc;
    if (X0 && (rc = copy_in_host(A, A->d_stage[1], X0, sizeof(double) * A->n * k, s))) return rc;
    if ((rc = persist_single(A, k, A->d_stage[0], X0 ? A->d_stage[1] : nullptr, rel_tol, maxit, flags,
                             A->d_stage[0], iters, status, resid_hist, true_relres, s)))
      return rc;
    if ((rc = copy_out_host(A, X, A->d_stage[0], sizeof(double) * A->n * k, s))) return rc;
    CK(cudaStreamSynchronize(s));
    return BICGK_OK;
  }
  const int opts = seq_opts(A, k, variant);
  const int gkey = variant + 100 * (jacobi ? 1 : 0) + 1000 * opts;
  int rc0 = ensure_variant_data(A, variant, jacobi, s);
  if (rc0) return rc0;
  // columns are independent: from k = kSplitMinK they are split into groups solved concurrently,
  // so that one group's FP64-bound SpMM overlaps another group's bandwidth-bound vector kernels.
  // The profiling mode keeps the same groups (so it times the kernels the solve runs) but runs
  // them one after another on the caller's stream.
  const int ngroups = num_groups(A, k);
  const bool concurrent = !A->profiling && ngroups >= 2;
  // the launch shapes follow the solve's groups (auto_spmm_cap, vec_grid), in the profiling mode
  // too, so that it times the kernels the graph runs; other entry points see one group
  struct GroupsScope {
    bicgk_op A;
    ~GroupsScope() { A->cur_groups = 1; }
  } groups_scope{A};
  A->cur_groups = ngroups;
  int c0[kMaxGroups + 1];
  for (int g = 0; g <= ngroups; ++g) c0[g] = (int)((int64_t)g * k / ngroups);
  int rc;
  for (int g = 0; g < ngroups; ++g) {
    const int kg = c0[g + 1] - c0[g];
    const int kpg = pow2_at_least(kg);
    if ((rc = ensure_workspace(A, A->ws[g], kpg))) return rc;
    if ((rc = ensure_hist(A->ws[g], (int64_t)(maxit + 1) * kpg))) return rc;
  }
  const Seq q = make_seq(variant, jacobi, opts);
  // inputs.  Page-locked host blocks are read and written in place by the pack and unpack kernels
  // (mapped over the host link): each group moves only its own columns, the groups' reads one
  // after another so that the first group iterates while the next ones still read B, and each
  // group writes its X as soon as it stops.  Other host blocks go through a staged copy.
  const double *dB = B, *dX0 = X0;
  double *dX = X;
  bool zero_copy = false;
  if (mem == BICGK_MEM_HOST && A->opt_zero_copy != 1) {
    const void *mb = mapped_host_ptr(B), *mx = mapped_host_ptr(X), *m0 = mapped_host_ptr(X0);
    if (mb && mx && (!X0 || m0)) {
      zero_copy = true;
      dB = static_cast<const double *>(mb);
      dX = static_cast<double *>(const_cast<void *>(mx));
      dX0 = static_cast<const double *>(m0);
    }
  }
  const bool staged = mem == BICGK_MEM_HOST && !zero_copy;
  if (staged) {
    if ((rc = ensure_stage(A, A->n * k))) return rc;
    if ((rc = copy_in_host(A, A->d_stage[0], B, sizeof(double) * A->n * k, s))) return rc;
    dB = A->d_stage[0];
    if (X0) {
      if ((rc = copy_in_host(A, A->d_stage[1], X0, sizeof(double) * A->n * k, s))) return rc;
      dX0 = A->d_stage[1];
    }
    dX = A->d_stage[0];  // X overwrites the staged B after both groups have packed it
  }
  if (concurrent) CK(cudaEventRecord(A->fork, s));
  int64_t launches = 0;
  for (int g = 0; g < ngroups; ++g) {
    Workspace &W = A->ws[g];
    cudaStream_t gs = concurrent ? W.stream : s;
    if (concurrent) CK(cudaStreamWaitEvent(gs, A->fork, 0));
    const int kg = c0[g + 1] - c0[g];
    const int64_t hist_len = (int64_t)(maxit + 1) * W.kp;
    Ctl *hc = W.h_ctl;
    memset(hc, 0, sizeof(Ctl));
    hc->tol = rel_tol;
    hc->hist = W.d_hist;
    hc->maxit = maxit;
    hc->k = kg;
    hc->kp = W.kp;
    hc->flags = flags;
    CK(cudaMemcpyAsync(W.d_ctl, hc, sizeof(Ctl), cudaMemcpyHostToDevice, gs));
    const KArgs a0 = make_args(A, W, 0, cudaGraphConditionalHandle{}, nullptr, jacobi ? A->d_invdiag : nullptr);
    CK(launch_reset(a0, hist_len, gs));
    if (zero_copy && g > 0) CK(cudaStreamWaitEvent(gs, A->ws[g - 1].packed, 0));
    CK(launch_pack(dB + c0[g], dX0 ? dX0 + c0[g] : nullptr, k, kg, a0, gs));
    if (zero_copy) CK(cudaEventRecord(W.packed, gs));
    launches += 2;  // reset, pack
    if (A->profiling) {
      if ((rc = run_profiled(A, W, variant, jacobi, opts, a0, gs))) return rc;
    } else {
      const bool cg = compact_columns(A, variant, W.kp);
      const int key = gkey + 10000 * (cg ? 1 : 0) + 100000 * ngroups;  // shapes depend on the groups
      auto it = W.graphs.find(key);
      if (it == W.graphs.end()) {
        GraphEntry ge;
        rc = cg ? build_graph_compact(A, W, q, &ge, jacobi ? A->d_invdiag : nullptr, variant)
                : build_graph(A, W, variant, jacobi, opts, &ge);
        if (rc) {
          if (ge.exec) cudaGraphExecDestroy(ge.exec);
          if (ge.graph) cudaGraphDestroy(ge.graph);
          return rc;
        }
        it = W.graphs.emplace(key, ge).first;
      }
      CK(cudaGraphLaunch(it->second.exec, gs));
    }
    if (concurrent && staged) {
      // the staged B is overwritten by X only after every group has packed its columns
      CK(cudaEventRecord(W.done, gs));
    }
  }
  for (int g = 0; g < ngroups; ++g) {
    Workspace &W = A->ws[g];
    cudaStream_t gs = concurrent ? W.stream : s;
    if (concurrent && staged)
      for (int h = 0; h < ngroups; ++h)
        if (h != g) CK(cudaStreamWaitEvent(gs, A->ws[h].done, 0));
    const int kg = c0[g + 1] - c0[g];
    const int64_t hist_len = (int64_t)(maxit + 1) * W.kp;
    // a compacted solve reports from the final block and arrays
    const bool cg = compact_columns(A, variant, W.kp);
    const KArgs a0 = cg ? final_args(A, W, nullptr) : make_args(A, W, 0, cudaGraphConditionalHandle{});
    CK(launch_unpack_role(dX + c0[g], k, kg, a0, V_X, 1, gs));
    CK(cudaMemcpyAsync(W.h_ctl, W.d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, gs));
    CK(cudaMemcpyAsync(W.h_fl, a0.fl, sizeof(int) * F_NFLAG * kMaxKp, cudaMemcpyDeviceToHost, gs));
    CK(cudaMemcpyAsync(W.h_sc, a0.sc, sizeof(double) * S_NSLOT * kMaxKp, cudaMemcpyDeviceToHost, gs));
    if (cg) {
      int levels = 0;
      while ((W.kp >> levels) > 1) ++levels;
      int inplace = 0;
      for (unsigned m = compact_roles(variant).inplace_mask; m; m &= m - 1) ++inplace;
      // the compaction boundaries' plan and move kernels, and the in-place gathers and copies
      launches += 2 * (levels + 1) + 2 * (int64_t)inplace * levels;
    }
    if (resid_hist)
      CK(cudaMemcpyAsync(W.h_hist, W.d_hist, sizeof(double) * hist_len, cudaMemcpyDeviceToHost, gs));
    if (concurrent) {
      CK(cudaEventRecord(W.done, gs));
      CK(cudaStreamWaitEvent(s, W.done, 0));
    }
    launches += 1;  // unpack
  }
  if (staged && (rc = copy_out_host(A, X, dX, sizeof(double) * A->n * k, s))) return rc;
  CK(cudaStreamSynchronize(s));
  int32_t loop_iters = 0;
  for (int g = 0; g < ngroups; ++g) {
    Workspace &W = A->ws[g];
    const int kg = c0[g + 1] - c0[g];
    for (int c = 0; c < kg; ++c) {
      iters[c0[g] + c] = W.h_fl[F_ITERS * kMaxKp + c];
      status[c0[g] + c] = W.h_fl[F_STATUS * kMaxKp + c];
      if (true_relres) true_relres[c0[g] + c] = W.h_sc[S_TRUE * kMaxKp + c];
    }
    if (resid_hist)
      for (int64_t j = 0; j <= maxit; ++j)
        for (int c = 0; c < kg; ++c) resid_hist[j * k + c0[g] + c] = W.h_hist[j * W.kp + c];
    if (W.h_ctl->loop_iters > loop_iters) loop_iters = W.h_ctl->loop_iters;
    launches += (int64_t)q.setup.size() + (int64_t)W.h_ctl->loop_iters * q.body.size() + q.fin.size();
  }
  A->last_loop_iters = loop_iters;
  A->last_kernels_per_iter = (int32_t)q.body.size();
  A->last_launches = launches;
  A->last_groups = ngroups;
  return BICGK_OK;
}


int bicgk_solve_mixed(bicgk_op A, int32_t k, const double *B, const double *X0, double rel_tol, int32_t max_outer,
                      double inner_tol, int32_t max_inner, int mem, double *X, int32_t *outer_iters,
                      int32_t *inner_iters, int32_t *status, double *resid_hist, double *true_relres,
                      void *stream) {
  if (!A || !B || !X || !outer_iters || !inner_iters || !status || k < 1 || !(rel_tol >= 0.0) ||
      !(inner_tol > 0.0 && inner_tol < 1.0) || max_outer < 0 || max_outer > 1000 || max_inner < 1 ||
      max_inner > 10000000 || (mem != BICGK_MEM_HOST && mem != BICGK_MEM_DEVICE))
    return BICGK_E_INVALID;
  if (k > BICGK_MAX_K) return BICGK_E_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  // columns are independent: they run as concurrent groups, each with its own FP64 outer and
  // FP32 inner workspaces; the refinement passes of the groups advance together.  Automatic: two
  // groups from k = 16 (27-point operator, 128^3, k = 32: 98.9 ms against 101.0 for one group and
  // 110.6 for four of 8, whose FP32 products are less efficient)
  // (the profiling mode runs the same groups one after another on the caller's stream)
  const int ngroups = A->opt_groups == 0 ? (k >= kMixedSplitMinK ? 2 : 1) : num_groups(A, k);
  const bool concurrent = !A->profiling && ngroups >= 2;
  int c0[kMaxGroups + 1];
  for (int g = 0; g <= ngroups; ++g) c0[g] = (int)((int64_t)g * k / ngroups);
  int rc;
  for (int g = 0; g < ngroups; ++g) {
    const int kpg = pow2_at_least(c0[g + 1] - c0[g]);
    Workspace &W = A->ws[g];
    Workspace &V = A->ws32[g];
    V.ebytes = 4;
    if ((rc = ensure_workspace(A, W, kpg)) || (rc = ensure_workspace(A, V, kpg)) ||
        (rc = ensure_hist(W, (int64_t)(max_outer + 1) * kpg)) ||
        (rc = ensure_hist(V, (int64_t)(max_inner + 1) * kpg)))
      return rc;
  }
  if (!A->d_val32) {
    CK(cudaMalloc(&A->d_val32, sizeof(float) * A->nnz + 16));
    CK(launch_to_float(A->d_val, A->d_val32, A->nnz, s));
  }
  const double *dB = B, *dX0 = X0;
  double *dX = X;
  if (mem == BICGK_MEM_HOST) {
    if ((rc = ensure_stage(A, A->n * k))) return rc;
    if ((rc = copy_in_host(A, A->d_stage[0], B, sizeof(double) * A->n * k, s))) return rc;
    dB = A->d_stage[0];
    if (X0) {
      if ((rc = copy_in_host(A, A->d_stage[1], X0, sizeof(double) * A->n * k, s))) return rc;
      dX0 = A->d_stage[1];
    }
    dX = A->d_stage[1];  // X goes to the second staging block: the groups pack B from the first
  }
  if (concurrent) CK(cudaEventRecord(A->fork, s));
  const Seq qi = make_inner32_seq();
  const Step res = resid(V_X, V_R, V_B);
  int64_t launches = 0;
  std::vector<int32_t> inner_total(k, 0);
  bool live[kMaxGroups];
  for (int g = 0; g < ngroups; ++g) {
    Workspace &W = A->ws[g];
    Workspace &V = A->ws32[g];
    cudaStream_t gs = concurrent ? W.stream : s;
    if (concurrent) CK(cudaStreamWaitEvent(gs, A->fork, 0));
    const int kg = c0[g + 1] - c0[g];
    // outer (FP64) state
    Ctl *hc = W.h_ctl;
    memset(hc, 0, sizeof(Ctl));
    hc->tol = rel_tol;
    hc->hist = W.d_hist;
    hc->maxit = max_outer;
    hc->k = kg;
    hc->kp = W.kp;
    CK(cudaMemcpyAsync(W.d_ctl, hc, sizeof(Ctl), cudaMemcpyHostToDevice, gs));
    const KArgs ao = make_args(A, W, 0, cudaGraphConditionalHandle{});
    CK(launch_reset(ao, (int64_t)(max_outer + 1) * W.kp, gs));
    CK(launch_pack(dB + c0[g], dX0 ? dX0 + c0[g] : nullptr, k, kg, ao, gs));
    CK(launch_vec(OP_IR_SETUP, ao, vec_grid(A, OP_IR_SETUP), gs));
    launches += 3;
    // inner FP32 solve graph (columns the outer loop still refines: the outer active flags)
    if (V.graphs.find(-1) == V.graphs.end()) {
      GraphEntry ge;
      if ((rc = build_graph_seq(A, V, qi, W.d_fl + F_ACT * kMaxKp, &ge))) {
        if (ge.exec) cudaGraphExecDestroy(ge.exec);
        if (ge.graph) cudaGraphDestroy(ge.graph);
        return rc;
      }
      V.graphs.emplace(-1, ge);
    }
    live[g] = true;
  }
  for (int pass = 0;; ++pass) {
    // every group still refining: r = b - A x (FP64), (r,r), stop test, b32 = fl32(r)
    for (int g = 0; g < ngroups; ++g) {
      if (!live[g]) continue;
      Workspace &W = A->ws[g];
      Workspace &V = A->ws32[g];
      cudaStream_t gs = concurrent ? W.stream : s;
      const KArgs ao = make_args(A, W, 0, cudaGraphConditionalHandle{});
      KArgs air = ao;  // outer steps that touch the FP32 blocks: b32 in V_Q, d in V_Y
      const KArgs ai0 = make_args(A, V, 0, cudaGraphConditionalHandle{});
      air.v[V_Q] = ai0.v[V_B];
      air.v[V_Y] = ai0.v[V_X];
      CK(launch_step(A, res, ao, gs));
      CK(launch_vec(OP_IR_RESID, air, vec_grid(A, OP_IR_RESID), gs));
      CK(cudaMemcpyAsync(W.h_ctl, W.d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, gs));
      launches += 2;
    }
    bool any = false;
    for (int g = 0; g < ngroups; ++g) {
      if (!live[g]) continue;
      Workspace &W = A->ws[g];
      Workspace &V = A->ws32[g];
      CK(cudaStreamSynchronize(concurrent ? W.stream : s));
      if (pass > 0)
        for (int c = 0; c < c0[g + 1] - c0[g]; ++c) inner_total[c0[g] + c] += V.h_fl[F_ITERS * kMaxKp + c];
      live[g] = W.h_ctl->any_active != 0;
      any = any || live[g];
    }
    if (!any) break;
    // every group still refining: FP32 inner solve of A d = r, then x += d (FP64)
    for (int g = 0; g < ngroups; ++g) {
      if (!live[g]) continue;
      Workspace &W = A->ws[g];
      Workspace &V = A->ws32[g];
      cudaStream_t gs = concurrent ? W.stream : s;
      const KArgs ao = make_args(A, W, 0, cudaGraphConditionalHandle{});
      KArgs air = ao;
      const KArgs ai0 = make_args(A, V, 0, cudaGraphConditionalHandle{});
      air.v[V_Q] = ai0.v[V_B];
      air.v[V_Y] = ai0.v[V_X];
      Ctl *hi = V.h_ctl;
      memset(hi, 0, sizeof(Ctl));
      hi->tol = inner_tol;
      hi->hist = V.d_hist;
      hi->maxit = max_inner;
      hi->k = c0[g + 1] - c0[g];
      hi->kp = V.kp;
      CK(cudaMemcpyAsync(V.d_ctl, hi, sizeof(Ctl), cudaMemcpyHostToDevice, gs));
      CK(launch_reset(ai0, (int64_t)(max_inner + 1) * V.kp, gs));
      if (A->profiling) {  // the same kernels from a host loop, each timed (profilers see them)
        const KArgs ai = make_args(A, V, 0, cudaGraphConditionalHandle{}, W.d_fl + F_ACT * kMaxKp);
        if ((rc = run_profiled_seq(A, V, qi, ai, gs))) return rc;
      } else {
        CK(cudaGraphLaunch(V.graphs.find(-1)->second.exec, gs));
      }
      CK(launch_vec(OP_IR_UPDATE, air, vec_grid(A, OP_IR_UPDATE), gs));
      CK(cudaMemcpyAsync(V.h_fl, V.d_fl, sizeof(int) * F_NFLAG * kMaxKp, cudaMemcpyDeviceToHost, gs));
      CK(cudaMemcpyAsync(V.h_ctl, V.d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, gs));
      launches += 2;
    }
  }
  for (int g = 0; g < ngroups; ++g) {
    Workspace &W = A->ws[g];
    cudaStream_t gs = concurrent ? W.stream : s;
    const KArgs ao = make_args(A, W, 0, cudaGraphConditionalHandle{});
    CK(launch_unpack_role(dX + c0[g], k, c0[g + 1] - c0[g], ao, V_X, 1, gs));
    CK(cudaMemcpyAsync(W.h_fl, W.d_fl, sizeof(int) * F_NFLAG * kMaxKp, cudaMemcpyDeviceToHost, gs));
    CK(cudaMemcpyAsync(W.h_sc, W.d_sc, sizeof(double) * S_NSLOT * kMaxKp, cudaMemcpyDeviceToHost, gs));
    if (resid_hist)
      CK(cudaMemcpyAsync(W.h_hist, W.d_hist, sizeof(double) * (max_outer + 1) * W.kp, cudaMemcpyDeviceToHost,
                         gs));
    if (concurrent) {
      CK(cudaEventRecord(W.done, gs));
      CK(cudaStreamWaitEvent(s, W.done, 0));
    }
    launches += 1;
  }
  if (mem == BICGK_MEM_HOST && (rc = copy_out_host(A, X, dX, sizeof(double) * A->n * k, s))) return rc;
  CK(cudaStreamSynchronize(s));
  int32_t loop_max = 0;
  for (int g = 0; g < ngroups; ++g) {
    Workspace &W = A->ws[g];
    const int kg = c0[g + 1] - c0[g];
    for (int c = 0; c < kg; ++c) {
      status[c0[g] + c] = W.h_fl[F_STATUS * kMaxKp + c];
      outer_iters[c0[g] + c] = W.h_fl[F_ITERS * kMaxKp + c];
      inner_iters[c0[g] + c] = inner_total[c0[g] + c];
      if (true_relres) true_relres[c0[g] + c] = W.h_sc[S_TRUE * kMaxKp + c];
      if (inner_total[c0[g] + c] > loop_max) loop_max = inner_total[c0[g] + c];
    }
    if (resid_hist)
      for (int64_t j = 0; j <= max_outer; ++j)
        for (int c = 0; c < kg; ++c) resid_hist[j * k + c0[g] + c] = W.h_hist[j * W.kp + c];
  }
  A->last_loop_iters = loop_max;
  A->last_kernels_per_iter = (int32_t)qi.body.size();
  A->last_launches = launches;
  A->last_groups = ngroups;
  return BICGK_OK;
}


int bicgk_op_transpose(bicgk_op A, bicgk_op *AT, void *stream) {
  if (!A || !AT) return BICGK_E_INVALID;
  *AT = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = A->n, nnz = A->nnz;
  bicgk_op T = nullptr;
  int rc = op_alloc(&T, A->device, A->nsm, n, nnz);
  if (rc) return rc;
  void *scratch = nullptr;
  int *d_max = nullptr;
  int maxtile = 0;
  cudaError_t e;
  if ((e = cudaMalloc(&T->d_perm, sizeof(int32_t) * nnz + 16)) != cudaSuccess ||
      (e = cudaMalloc(&scratch, transpose_scratch_bytes(n, nnz))) != cudaSuccess ||
      (e = cudaMalloc(&d_max, sizeof(int))) != cudaSuccess ||
      (e = launch_transpose(A->d_rowptr, A->d_col, A->d_val, n, nnz, T->d_rowptr, T->d_col, T->d_val, T->d_perm, d_max,
                            scratch, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&maxtile, d_max, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    cudaFree(scratch);
    cudaFree(d_max);
    bicgk_op_destroy(T);
    return cuda_fail(e, "bicgk_op_transpose");
  }
  cudaFree(scratch);
  cudaFree(d_max);
  T->stage_cap = maxtile < kSpmmStageMax ? maxtile : kSpmmStageMax;
  *AT = T;
  return BICGK_OK;
}

int bicgk_op_set_values(bicgk_op A, const double *vals, int mem, void *stream) {
  if (!A || (A->nnz > 0 && !vals) || (mem != BICGK_MEM_HOST && mem != BICGK_MEM_DEVICE)) return BICGK_E_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  if (A->nnz > 0)
    CK(cudaMemcpyAsync(A->d_val, vals, sizeof(double) * A->nnz,
                       mem == BICGK_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  int rc = refresh_derived(A, s);
  if (rc) return rc;
  if (A->trans) {
    CK(launch_permute_values(A->trans->d_perm, A->d_val, A->nnz, A->trans->d_val, s));
    if ((rc = refresh_derived(A->trans, s))) return rc;
  }
  CK(cudaStreamSynchronize(s));
  return BICGK_OK;
}

int bicgk_op_transpose_refresh(bicgk_op A, bicgk_op AT, void *stream) {
  if (!A || !AT || !AT->d_perm || AT->n != A->n || AT->nnz != A->nnz) return BICGK_E_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  CK(launch_permute_values(AT->d_perm, A->d_val, A->nnz, AT->d_val, s));
  int rc = refresh_derived(AT, s);
  if (rc) return rc;
  CK(cudaStreamSynchronize(s));
  return BICGK_OK;
}

int bicgk_op_get_csr(bicgk_op A, int32_t *rowptr, int32_t *colidx, double *vals, void *stream) {
  if (!A) return BICGK_E_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  if (rowptr) CK(cudaMemcpyAsync(rowptr, A->d_rowptr, sizeof(int32_t) * (A->n + 1), cudaMemcpyDeviceToHost, s));
  if (colidx && A->nnz) CK(cudaMemcpyAsync(colidx, A->d_col, sizeof(int32_t) * A->nnz, cudaMemcpyDeviceToHost, s));
  if (vals && A->nnz) CK(cudaMemcpyAsync(vals, A->d_val, sizeof(double) * A->nnz, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return BICGK_OK;
}

int bicgk_spmm_t(bicgk_op A, int32_t k, const double *X, double *Y, int method, void *stream) {
  if (!A || !X || !Y || k < 1 || X == Y || (method != BICGK_TRANSPOSE_EXPLICIT && method != BICGK_TRANSPOSE_ATOMIC))
    return BICGK_E_INVALID;
  if (k > BICGK_MAX_K) return BICGK_E_UNSUPPORTED;
  if (method == BICGK_TRANSPOSE_ATOMIC) {
    CK(launch_spmm_t_atomic(A->d_rowptr, A->d_col, A->d_val, X, Y, A->n, k, (cudaStream_t)stream));
    return BICGK_OK;
  }
  if (!A->trans) {
    int rc = bicgk_op_transpose(A, &A->trans, stream);
    if (rc) return rc;
  }
  return bicgk_spmm(A->trans, k, X, Y, stream);
}

int bicgk_sddmm(bicgk_op A, int32_t k, const double *L, const double *X, double alpha, double *G, void *stream) {
  if (!A || !L || !X || !G || k < 1) return BICGK_E_INVALID;
  CK(launch_sddmm(A->d_rowptr, A->d_col, L, X, alpha, G, A->n, k, (cudaStream_t)stream));
  return BICGK_OK;
}

int bicgk_set_option(bicgk_op A, int option, int64_t value) {
  if (!A) return BICGK_E_INVALID;
  switch (option) {
    case BICGK_OPT_VEC_BLOCKS_PER_SM:
      if (value < 0 || value > 4) return BICGK_E_INVALID;
      A->opt_vec_blocks = (int)value;
      break;
    case BICGK_OPT_SPMM_BLOCKS_PER_SM:
      if (value < 0 || value > 32) return BICGK_E_INVALID;
      A->opt_spmm_blocks = (int)value;
      break;
    case BICGK_OPT_RHS_GROUPS:
      if (value < 0 || value > kMaxGroups) return BICGK_E_INVALID;
      A->opt_groups = (int)value;
      break;
    case BICGK_OPT_FUSED_DOTS:
      if (value < 0 || value > 2) return BICGK_E_INVALID;
      A->opt_fused = (int)value;
      break;
    case BICGK_OPT_THETA_IN_S:
      if (value < 0 || value > 2) return BICGK_E_INVALID;
      A->opt_theta = (int)value;
      break;
    case BICGK_OPT_HOST_ZERO_COPY:
      if (value < 0 || value > 1) return BICGK_E_INVALID;
      A->opt_zero_copy = (int)value;
      break;
    case BICGK_OPT_COMPACT:
      if (value < 0 || value > 1) return BICGK_E_INVALID;
      A->opt_compact = (int)value;
      break;
    case BICGK_OPT_PERSISTENT:
      if (value < 0 || value > 2) return BICGK_E_INVALID;
      A->opt_persistent = (int)value;
      break;
    case BICGK_OPT_SPMM32:
      if (value < 0 || value > 1) return BICGK_E_INVALID;
      A->opt_spmm32 = (int)value;
      break;
    case BICGK_OPT_SPMM_ROWS:
      if (value < 0 || value > 2) return BICGK_E_INVALID;
      A->opt_spmm_rows = (int)value;
      break;
    default:
      return BICGK_E_INVALID;
  }
  drop_all_graphs(A);  // grid sizes are baked into the captured graphs
  for (Workspace &V : A->ws32) drop_graphs(V);
  return BICGK_OK;
}

int bicgk_set_profiling(bicgk_op A, int on) {
  if (!A) return BICGK_E_INVALID;
  A->profiling = on != 0;
  A->prof.clear();
  return BICGK_OK;
}

int bicgk_kernel_times(bicgk_op A, int32_t max_n, int32_t *n_out, const char **names, int64_t *launches,
                       double *total_ms) {
  if (!A || !n_out || max_n < 0) return BICGK_E_INVALID;
  A->prof_names.clear();
  for (auto &kv : A->prof) A->prof_names.push_back(kv.first);
  int32_t i = 0;
  for (auto &kv : A->prof) {
    if (i >= max_n) break;
    if (names) names[i] = A->prof_names[i].c_str();
    if (launches) launches[i] = kv.second.launches;
    if (total_ms) total_ms[i] = kv.second.ms;
    ++i;
  }
  *n_out = (int32_t)A->prof.size();
  return BICGK_OK;
}

int bicgk_last_stats(bicgk_op A, int32_t *loop_iters, int64_t *kernel_launches, int32_t *kernels_per_iter) {
  if (!A) return BICGK_E_INVALID;
  if (loop_iters) *loop_iters = A->last_loop_iters;
  if (kernel_launches) *kernel_launches = A->last_launches;
  if (kernels_per_iter) *kernels_per_iter = A->last_kernels_per_iter;
  return BICGK_OK;
}

int bicgk_last_groups(bicgk_op A, int32_t *groups) {
  if (!A || !groups) return BICGK_E_INVALID;
  *groups = A->last_groups;
  return BICGK_OK;
}

}  // extern "C"


// ----------------------------------------------------------------------------
// Batches of independent systems (uneven sizes and RHS counts) in one graph.
//
// Every system keeps its own operator (CSR copy, launch shapes) and a batch workspace whose
// control block, flags and scalars live in batch-wide arrays, so one upload and one readback
// serve all systems.  The batched graph holds one independent branch per system: reset, pack
// (caller pointers read from a device table), the form's set-up, a conditional WHILE node over
// one iteration, the true residual and unpack.  One launch runs every branch; the branches have
// no edges between them, so the GPU overlaps the systems' kernels.
struct bicgk_batch_s {
  int nsys = 0;
  bool borrowed = false;      // the operators belong to the caller (a one-system batch of bicgk_solve)
  std::vector<bicgk_op> ops;
  std::vector<int> k;
  std::vector<Workspace> ws;  // batch workspaces (shared state)
  Ctl *d_ctl = nullptr, *h_ctl = nullptr;
  int *d_fl = nullptr, *h_fl = nullptr;
  double *d_sc = nullptr, *h_sc = nullptr;
  BatchIO *d_io = nullptr, *h_io = nullptr;
  int64_t hist_iters = 0;     // history capacity of every system, in iterations + 1
  std::map<int, GraphEntry> graphs;
  int64_t last_launches = 0;
  // persistent mode: one cooperative launch over every system's row tiles
  PersistSys *d_psys = nullptr, *h_psys = nullptr;
  unsigned *d_tickets = nullptr;
  int *d_live = nullptr;
  PersistCtl *d_pc = nullptr, *h_pc = nullptr;
  double *d_ppart = nullptr;
  size_t ppart_cap = 0;       // doubles
  int64_t p_ntiles = 0;
  int p_grid = 0;
  int p_sub = 1;              // 256-thread passes per tile (rows per CTA tile; bicgk_batch_tune_persistent)
  int p_minb = 4;             // blocks per SM of the kernel variant (4 or 6; bicgk_batch_tune_persistent)
  int p_div = 1;              // the grid is the co-resident maximum / p_div blocks (tuned)
  int64_t deadline_us = 1000000;  // longest wait at one grid barrier
  GraphEntry pgraph;          // clear the control block, the cooperative kernel
  bool pgraph_ok = false;
  bool p_direct = false;      // the runtime could not put the cooperative launch in a graph
  int p_capture_err = 0;      // the cudaError_t it gave
  int64_t p_loop_iters = 0;
};

namespace {

void batch_drop_graphs(bicgk_batch b) {
  for (auto &kv : b->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  b->graphs.clear();
}

int batch_ensure(bicgk_batch b, int32_t maxit) {
  const int64_t need = (int64_t)maxit + 1;
  for (int i = 0; i < b->nsys; ++i) {
    Workspace &W = b->ws[i];
    bicgk_op A = b->ops[i];
    const int kp = pow2_at_least(b->k[i]);
    if (W.kp != kp) {
      const int64_t elems = A->n * kp + 2;
      W.vstride = (elems + 31) / 32 * 32;
      const size_t bytes = (size_t)W.vstride * V_NVEC * sizeof(double);
      CK(cudaMalloc(&W.d_vec, bytes));
      CK(cudaMemset(W.d_vec, 0, bytes));
      CK(cudaMalloc(&W.d_part, sizeof(double) * ((size_t)A->nsm * kPartBlocksPerSm + kMaxRedGroups) * kMaxDots * kMaxKp));
      W.kp = kp;
    }
  }
  if (need > b->hist_iters) {
    for (int i = 0; i < b->nsys; ++i) {
      Workspace &W = b->ws[i];
      cudaFree(W.d_hist);
      W.d_hist = nullptr;
      CK(cudaMalloc(&W.d_hist, sizeof(double) * need * W.kp));
      W.hist_cap = need * W.kp;
    }
    b->hist_iters = need;
    batch_drop_graphs(b);  // the history length is baked into the reset nodes
  }
  return BICGK_OK;
}

int batch_build_graph(bicgk_batch b, int variant, bool jacobi, GraphEntry *ge) {
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  ge->graph = g;
  cudaStream_t cs = b->ops[0]->cap_stream;
  cudaGraph_t tmp;
  for (int i = 0; i < b->nsys; ++i) {
    bicgk_op A = b->ops[i];
    Workspace &W = b->ws[i];
    const Seq q = make_seq(variant, jacobi, seq_opts(A, b->k[i], variant));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
    const KArgs a = make_args(A, W, 1, h, nullptr, jacobi ? A->d_invdiag : nullptr);
    CK(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = launch_reset(a, W.hist_cap, cs);
    if (e == cudaSuccess) e = launch_pack_io(b->d_io + i, b->k[i], a, cs);
    for (size_t t = 0; e == cudaSuccess && t < q.setup.size(); ++t) e = launch_step(A, q.setup[t], a, cs);
    if (e != cudaSuccess) {
      cudaStreamEndCapture(cs, &tmp);
      return cuda_fail(e, "batch capture set-up");
    }
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    CK(cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps));
    std::vector<cudaGraphNode_t> leaves(deps, deps + ndeps);
    CK(cudaStreamEndCapture(cs, &tmp));
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t wnode;
    CK(cudaGraphAddNode(&wnode, g, leaves.data(), nullptr, leaves.size(), &p));
    CK(cudaStreamBeginCaptureToGraph(cs, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                     cudaStreamCaptureModeThreadLocal));
    for (size_t t = 0; e == cudaSuccess && t < q.body.size(); ++t) e = launch_step(A, q.body[t], a, cs);
    if (e != cudaSuccess) {
      cudaStreamEndCapture(cs, &tmp);
      return cuda_fail(e, "batch capture body");
    }
    CK(cudaStreamEndCapture(cs, &tmp));
    CK(cudaStreamBeginCaptureToGraph(cs, g, &wnode, nullptr, 1, cudaStreamCaptureModeThreadLocal));
    for (size_t t = 0; e == cudaSuccess && t < q.fin.size(); ++t) e = launch_step(A, q.fin[t], a, cs);
    if (e == cudaSuccess) e = launch_unpack_io(b->d_io + i, b->k[i], a, cs);
    if (e != cudaSuccess) {
      cudaStreamEndCapture(cs, &tmp);
      return cuda_fail(e, "batch capture final");
    }
    CK(cudaStreamEndCapture(cs, &tmp));
  }
  CK(cudaGraphInstantiate(&ge->exec, g, 0));
  return BICGK_OK;
}

void persist_drop_graph(bicgk_batch b) {
  if (b->pgraph.exec) cudaGraphExecDestroy(b->pgraph.exec);
  if (b->pgraph.graph) cudaGraphDestroy(b->pgraph.graph);
  b->pgraph = GraphEntry{};
  b->pgraph_ok = false;
}

// Tiles, descriptors and buffers of the persistent mode for the batch's current workspaces (after
// batch_ensure).  Caller blocks and history length are filled per solve.
int persist_prepare(bicgk_batch b) {
  const int n = b->nsys;
  if (!b->d_psys) {
    CK(cudaMalloc(&b->d_psys, sizeof(PersistSys) * n));
    CK(cudaMallocHost(&b->h_psys, sizeof(PersistSys) * n));
    CK(cudaMalloc(&b->d_tickets, sizeof(unsigned) * n));
    CK(cudaMalloc(&b->d_live, sizeof(int) * n));
    CK(cudaMalloc(&b->d_pc, sizeof(PersistCtl)));
    CK(cudaMallocHost(&b->h_pc, sizeof(PersistCtl)));
    memset(b->h_psys, 0, sizeof(PersistSys) * n);
  }
  int64_t tiles = 0;
  size_t part = 0;
  for (int i = 0; i < n; ++i) {
    bicgk_op A = b->ops[i];
    Workspace &W = b->ws[i];
    const int64_t rows = (int64_t)persist_rows_per_pass(W.kp) * b->p_sub;
    PersistSys &S = b->h_psys[i];
    S.rowptr = A->d_rowptr;
    S.colidx = A->d_col;
    S.vals = A->d_val;
    const int roles[P_NROLE] = {V_X, V_R, V_R0, V_P, V_V, V_S, V_T, V_B};
    for (int r = 0; r < P_NROLE; ++r) S.vec[r] = W.d_vec + (size_t)roles[r] * W.vstride;
    S.sc = W.d_sc;
    S.fl = W.d_fl;
    S.ctl = W.d_ctl;
    S.n = A->n;
    S.k = b->k[i];
    S.kp = W.kp;
    S.sub = b->p_sub;
    S.ntiles = (int)((A->n + rows - 1) / rows);
    S.tile0 = tiles;
    tiles += S.ntiles;
    part += (size_t)S.ntiles * 3 * W.kp;
  }
  if (part > b->ppart_cap) {
    cudaFree(b->d_ppart);
    b->d_ppart = nullptr;
    CK(cudaMalloc(&b->d_ppart, sizeof(double) * part));
    b->ppart_cap = part;
    persist_drop_graph(b);
  }
  size_t off = 0;
  for (int i = 0; i < n; ++i) {
    b->h_psys[i].part = b->d_ppart + off;
    off += (size_t)b->h_psys[i].ntiles * 3 * b->h_psys[i].kp;
  }
  if (tiles != b->p_ntiles) persist_drop_graph(b);
  b->p_ntiles = tiles;
  if (!b->p_grid) {
    const int nb = persist_blocks_per_sm(b->p_minb);
    if (nb < 1) return cuda_fail(cudaGetLastError(), "persistent kernel occupancy");
    const int full = b->ops[0]->nsm * (nb < b->p_minb ? nb : b->p_minb);
    b->p_grid = full / b->p_div > 0 ? full / b->p_div : 1;
  }
  return BICGK_OK;
}

// One persistent solve on stream s (descriptors and control blocks already uploaded): a graph of
// the control-block reset and the cooperative kernel, captured once per shape.
int persist_launch(bicgk_batch b, cudaStream_t s) {
  PersistArgs pa;
  pa.sys = b->d_psys;
  pa.tickets = b->d_tickets;
  pa.live = b->d_live;
  pa.pc = b->d_pc;
  pa.ntiles = b->p_ntiles;
  pa.nsys = b->nsys;
  pa.pad = 0;
  pa.deadline_ns = (unsigned long long)b->deadline_us * 1000ull;
  if (!b->pgraph_ok && !b->p_direct) {
    // graph: clear the control block, tickets and liveness; then the cooperative kernel node
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    cudaGraphNode_t m[3], kn;
    cudaError_t e = cudaGraphCreate(&g, 0);
    const struct {
      void *p;
      size_t bytes;
    } clr[3] = {{b->d_pc, sizeof(PersistCtl)}, {b->d_tickets, sizeof(unsigned) * b->nsys},
                {b->d_live, sizeof(int) * b->nsys}};
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
      cudaMemsetParams mp = {};
      mp.dst = clr[i].p;
      mp.value = 0;
      mp.elementSize = 4;
      mp.width = clr[i].bytes / 4;
      mp.height = 1;
      mp.pitch = clr[i].bytes;
      e = cudaGraphAddMemsetNode(&m[i], g, nullptr, 0, &mp);
    }
    if (e == cudaSuccess) e = add_persist_node(g, m, 3, pa, b->p_grid, b->p_minb, &kn);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
    if (e != cudaSuccess) {
      // a runtime that cannot put a cooperative launch in a graph: launch it directly from now on
      if (g) cudaGraphDestroy(g);
      b->p_capture_err = (int)e;
      cudaGetLastError();
      b->p_direct = true;
    } else {
      b->pgraph.graph = g;
      b->pgraph.exec = ge;
      b->pgraph_ok = true;
    }
  }
  if (b->p_direct) {
    CK(cudaMemsetAsync(b->d_pc, 0, sizeof(PersistCtl), s));
    CK(cudaMemsetAsync(b->d_tickets, 0, sizeof(unsigned) * b->nsys, s));
    CK(cudaMemsetAsync(b->d_live, 0, sizeof(int) * b->nsys, s));
    CK(launch_persist(pa, b->p_grid, b->p_minb, s));
    return BICGK_OK;
  }
  CK(cudaGraphLaunch(b->pgraph.exec, s));
  return BICGK_OK;
}

// Mean time of `reps` launches of one kernel configuration (CUDA events on stream s).
template <class F>
int time_launches(F launch, int reps, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, float *ms) {
  CK(launch());  // warm
  CK(cudaEventRecord(e0, s));
  for (int r = 0; r < reps; ++r) CK(launch());
  CK(cudaEventRecord(e1, s));
  CK(cudaEventSynchronize(e1));
  CK(cudaEventElapsedTime(ms, e0, e1));
  *ms /= reps;
  return BICGK_OK;
}

}  // namespace

namespace {

// Control blocks, flags, scalars and caller-pointer table of a batch, and the workspaces' views
// of them.
int batch_alloc_state(bicgk_batch b) {
  const int nsys = b->nsys;
  cudaError_t e = cudaSuccess;
  {
    if ((e = cudaMalloc(&b->d_ctl, sizeof(Ctl) * nsys)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_fl, sizeof(int) * F_NFLAG * kMaxKp * nsys)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_sc, sizeof(double) * S_NSLOT * kMaxKp * nsys)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_io, sizeof(BatchIO) * nsys)) != cudaSuccess ||
        (e = cudaMallocHost(&b->h_ctl, sizeof(Ctl) * nsys)) != cudaSuccess ||
        (e = cudaMallocHost(&b->h_fl, sizeof(int) * F_NFLAG * kMaxKp * nsys)) != cudaSuccess ||
        (e = cudaMallocHost(&b->h_sc, sizeof(double) * S_NSLOT * kMaxKp * nsys)) != cudaSuccess ||
        (e = cudaMallocHost(&b->h_io, sizeof(BatchIO) * nsys)) != cudaSuccess ||
        (e = cudaMemset(b->d_ctl, 0, sizeof(Ctl) * nsys)) != cudaSuccess ||
        (e = cudaMemset(b->d_fl, 0, sizeof(int) * F_NFLAG * kMaxKp * nsys)) != cudaSuccess ||
        (e = cudaMemset(b->d_sc, 0, sizeof(double) * S_NSLOT * kMaxKp * nsys)) != cudaSuccess)
      return cuda_fail(e, "batch state");
  }
  for (int i = 0; i < nsys; ++i) {
    Workspace &W = b->ws[i];
    W.shared_state = true;
    W.d_ctl = b->d_ctl + i;
    W.d_fl = b->d_fl + (size_t)i * F_NFLAG * kMaxKp;
    W.d_sc = b->d_sc + (size_t)i * S_NSLOT * kMaxKp;
  }
  return BICGK_OK;
}

}  // namespace

// One solve of the operator's own system by the persistent kernel (bicgk_solve with
// BICGK_OPT_PERSISTENT): a one-system batch that borrows the operator, kept for the next solve of
// the same width.  Device blocks only.
int persist_single(bicgk_op A, int32_t k, const double *B, const double *X0, double rel_tol, int32_t maxit,
                   int32_t flags, double *X, int32_t *iters, int32_t *status, double *resid_hist,
                   double *true_relres, cudaStream_t s) {
  if (A->pbatch && A->pbatch_k != k) {
    bicgk_batch_destroy(A->pbatch);
    A->pbatch = nullptr;
  }
  if (!A->pbatch) {
    bicgk_batch b = new bicgk_batch_s();
    b->nsys = 1;
    b->borrowed = true;
    b->k.assign(1, k);
    b->ops.assign(1, A);
    b->ws.resize(1);
    int rc = batch_alloc_state(b);
    if (rc) {
      bicgk_batch_destroy(b);
      return rc;
    }
    A->pbatch = b;
    A->pbatch_k = k;
    // the first solve of this width picks the launch shape (a few short solves, temporaries)
    if ((rc = bicgk_batch_tune_persistent(b, 2, nullptr, s))) return rc;
  }
  bicgk_batch b = A->pbatch;
  const double *Bv[1] = {B};
  const double *X0v[1] = {X0};
  double *Xv[1] = {X};
  int rc = bicgk_batch_solve(b, Bv, X0 ? X0v : nullptr, Xv, rel_tol, maxit, BICGK_CLASSICAL_MERGED, flags,
                             BICGK_BATCH_PERSISTENT, iters, status, true_relres, s);
  if (rc) return rc;
  if (resid_hist) {
    const Workspace &W = b->ws[0];
    CK(cudaMemcpy2DAsync(resid_hist, sizeof(double) * k, W.d_hist, sizeof(double) * W.kp, sizeof(double) * k,
                         (size_t)maxit + 1, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  A->last_loop_iters = (int32_t)b->p_loop_iters;
  A->last_launches = 1;
  A->last_kernels_per_iter = 0;
  A->last_groups = 1;
  return BICGK_OK;
}

extern "C" {

int bicgk_batch_create(bicgk_batch *out, int32_t nsys, const int64_t *n_rows, const int64_t *nnz,
                       const int32_t *const *rowptr, const int32_t *const *colidx, const double *const *vals,
                       const int32_t *k, int mem, void *stream) {
  if (!out || nsys < 1 || nsys > 4096 || !n_rows || !nnz || !rowptr || !colidx || !vals || !k) return BICGK_E_INVALID;
  *out = nullptr;
  for (int i = 0; i < nsys; ++i)
    if (k[i] < 1) return BICGK_E_INVALID;
    else if (k[i] > BICGK_MAX_K) return BICGK_E_UNSUPPORTED;
  bicgk_batch b = new bicgk_batch_s();
  b->nsys = nsys;
  b->k.assign(k, k + nsys);
  b->ops.assign(nsys, nullptr);
  b->ws.resize(nsys);
  int rc = BICGK_OK;
  for (int i = 0; i < nsys && rc == BICGK_OK; ++i)
    rc = bicgk_csr_create(&b->ops[i], n_rows[i], nnz[i], rowptr[i], colidx[i], vals[i], mem, stream);
  // each system runs as one column group without dot epilogues or column compaction, in the
  // graph and in the launch loop alike (the loop calls bicgk_solve with these operators, on the
  // graph path)
  // Launch shapes: the systems' kernels share the GPU (the graph runs them as concurrent
  // branches), so each takes at most 4 SpMM blocks and 1 streaming block per SM, the caps that pay
  // for four concurrent column groups of one solve (auto_spmm_cap).  Measured on the 64-system
  // batch (16^3-64^3, k = 1..8, tuned shapes): graph 313 against 339 ms, launch loop 596 against
  // 627 ms (the streaming cap carries it: 4 SpMM blocks with 2 streaming blocks changed nothing).
  for (int i = 0; i < nsys && rc == BICGK_OK; ++i) {
    b->ops[i]->opt_groups = 1;
    b->ops[i]->opt_fused = 1;
    b->ops[i]->opt_compact = 1;
    b->ops[i]->opt_persistent = 1;
    b->ops[i]->opt_spmm_blocks = 4;
    b->ops[i]->opt_vec_blocks = 1;
  }
  if (rc == BICGK_OK) rc = batch_alloc_state(b);
  if (rc != BICGK_OK) {
    bicgk_batch_destroy(b);
    return rc;
  }
  *out = b;
  return BICGK_OK;
}


int bicgk_batch_destroy(bicgk_batch b) {
  if (!b) return BICGK_OK;
  cudaDeviceSynchronize();
  batch_drop_graphs(b);
  persist_drop_graph(b);
  cudaFree(b->d_psys);
  cudaFreeHost(b->h_psys);
  cudaFree(b->d_tickets);
  cudaFree(b->d_live);
  cudaFree(b->d_pc);
  cudaFreeHost(b->h_pc);
  cudaFree(b->d_ppart);
  for (Workspace &W : b->ws) {
    cudaFree(W.d_vec);
    cudaFree(W.d_part);
    cudaFree(W.d_hist);
  }
  if (!b->borrowed)
    for (bicgk_op A : b->ops) bicgk_op_destroy(A);
  cudaFree(b->d_ctl);
  cudaFree(b->d_fl);
  cudaFree(b->d_sc);
  cudaFree(b->d_io);
  cudaFreeHost(b->h_ctl);
  cudaFreeHost(b->h_fl);
  cudaFreeHost(b->h_sc);
  cudaFreeHost(b->h_io);
  delete b;
  return BICGK_OK;
}

int bicgk_batch_tune(bicgk_batch b, int32_t reps, int32_t *vec_grid_out, int32_t *spmm_grid_out,
                     int32_t *spmm_cpl_out, void *stream) {
  if (!b || reps < 1 || reps > 1000) return BICGK_E_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = batch_ensure(b, 1);
  if (rc) return rc;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  for (int i = 0; i < b->nsys && rc == BICGK_OK; ++i) {
    bicgk_op A = b->ops[i];
    Workspace &W = b->ws[i];
    // a control block with every column inactive: the timed kernels change no solver state
    Ctl *hc = b->h_ctl + i;
    memset(hc, 0, sizeof(Ctl));
    hc->hist = W.d_hist;
    hc->maxit = 1 << 30;
    hc->k = b->k[i];
    hc->kp = W.kp;
    CK(cudaMemcpyAsync(W.d_ctl, hc, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(W.d_fl, 0, sizeof(int) * F_NFLAG * kMaxKp, s));
    const KArgs a = make_args(A, W, 0, cudaGraphConditionalHandle{});
    const int64_t chunks = (A->n * W.kp + 1) / 2;
    // streaming kernels: grid for u double2 chunks per thread (rows per CTA), timed on group 3
    A->grid_vec_abs = 0;
    const int gmax = vec_grid(A, OP_G3);
    int best_vec = gmax;
    float best = 1e30f;
    for (int u = 1; u <= 64; u *= 2) {
      int g = (int)((chunks + (int64_t)kVecThreads * u - 1) / ((int64_t)kVecThreads * u));
      if (g > gmax) g = gmax;
      if (g < 1) g = 1;
      float ms = 0.f;
      rc = time_launches([&] { return launch_vec(OP_G3, a, g, s); }, reps, s, e0, e1, &ms);
      if (rc) break;
      if (ms < best * 0.98f) {
        best = ms;
        best_vec = g;
      }
      if (g == 1) break;
    }
    // SpMM: rows per CTA and RHS-tile width (columns per lane)
    A->grid_spmm_abs = 0;
    A->spmm_cpl = 2;
    const int smax = spmm_grid(A, W.kp, 0);
    int best_spmm = smax, best_cpl = 2;
    best = 1e30f;
    for (int cpl = 2; cpl <= (W.kp >= 8 ? 4 : 2) && rc == BICGK_OK; cpl *= 2) {
      const int rpp = W.kp <= 2 ? kSpmmTileRows : kSpmmThreads / (W.kp / cpl);
      for (int r = 1; r <= 64; r *= 2) {
        int g = (int)((A->n + (int64_t)rpp * r - 1) / ((int64_t)rpp * r));
        if (g > smax) g = smax;
        if (g < 1) g = 1;
        A->spmm_cpl = cpl;
        A->grid_spmm_abs = g;
        float ms = 0.f;
        rc = time_launches([&] { return launch_step(A, spmm(V_P, V_V), a, s); }, reps, s, e0, e1, &ms);
        if (rc) break;
        if (ms < best * 0.98f) {
          best = ms;
          best_spmm = g;
          best_cpl = cpl;
        }
        if (g == 1) break;
      }
    }
    A->grid_vec_abs = best_vec;
    A->grid_spmm_abs = best_spmm;
    A->spmm_cpl = best_cpl;
    drop_all_graphs(A);
    if (vec_grid_out) vec_grid_out[i] = best_vec;
    if (spmm_grid_out) spmm_grid_out[i] = best_spmm;
    if (spmm_cpl_out) spmm_cpl_out[i] = best_cpl;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  batch_drop_graphs(b);
  return rc;
}

int bicgk_batch_solve(bicgk_batch b, const double *const *B, const double *const *X0, double *const *X,
                      double rel_tol, int32_t maxit, int variant, int32_t flags, int mode, int32_t *iters,
                      int32_t *status, double *true_relres, void *stream) {
  if (!b || !B || !X || !iters || !status || !(rel_tol >= 0.0) || maxit < 0 || maxit > 10000000 || variant < 0 ||
      variant > 11 || (flags & ~3) ||
      (mode != BICGK_BATCH_GRAPH && mode != BICGK_BATCH_LOOP && mode != BICGK_BATCH_PERSISTENT))
    return BICGK_E_INVALID;
  const bool jacobi = (flags & BICGK_FLAG_JACOBI) != 0;
  if (mode == BICGK_BATCH_PERSISTENT && (variant != BICGK_CLASSICAL_MERGED || jacobi || b->nsys > kPersistMaxSys)) {
    g_cuda_err = "persistent batch mode runs merged classical BiCGStab (Algorithm 2) without preconditioner, "
                 "for at most " + std::to_string(kPersistMaxSys) + " systems";
    return BICGK_E_UNSUPPORTED;
  }
  const int gkey = variant + 100 * (jacobi ? 1 : 0);
  for (int i = 0; i < b->nsys; ++i)
    if (!B[i] || !X[i]) return BICGK_E_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  int rc;
  int64_t off = 0, launches = 0;
  if (mode == BICGK_BATCH_LOOP) {  // one bicgk_solve per system
    for (int i = 0; i < b->nsys; ++i) {
      if ((rc = bicgk_solve(b->ops[i], b->k[i], B[i], X0 ? X0[i] : nullptr, rel_tol, maxit, variant, flags,
                            BICGK_MEM_DEVICE, X[i], iters + off, status + off, nullptr,
                            true_relres ? true_relres + off : nullptr, stream)))
        return rc;
      launches += b->ops[i]->last_launches;
      off += b->k[i];
    }
    b->last_launches = launches;
    return BICGK_OK;
  }
  if ((rc = batch_ensure(b, maxit))) return rc;
  if (mode == BICGK_BATCH_PERSISTENT) {  // one cooperative launch for every system
    if ((rc = persist_prepare(b))) return rc;
    for (int i = 0; i < b->nsys; ++i) {
      Ctl *hc = b->h_ctl + i;
      memset(hc, 0, sizeof(Ctl));
      hc->tol = rel_tol;
      hc->hist = b->ws[i].d_hist;
      hc->maxit = maxit;
      hc->k = b->k[i];
      hc->kp = b->ws[i].kp;
      hc->flags = flags;
      PersistSys &S = b->h_psys[i];
      S.B = B[i];
      S.X0 = X0 ? X0[i] : nullptr;
      S.X = X[i];
      S.hist_len = (int64_t)(maxit + 1) * b->ws[i].kp;
    }
    CK(cudaMemcpyAsync(b->d_ctl, b->h_ctl, sizeof(Ctl) * b->nsys, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(b->d_psys, b->h_psys, sizeof(PersistSys) * b->nsys, cudaMemcpyHostToDevice, s));
    if ((rc = persist_launch(b, s))) return rc;
    CK(cudaMemcpyAsync(b->h_fl, b->d_fl, sizeof(int) * F_NFLAG * kMaxKp * b->nsys, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(b->h_sc, b->d_sc, sizeof(double) * S_NSLOT * kMaxKp * b->nsys, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(b->h_pc, b->d_pc, sizeof(PersistCtl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (b->h_pc->err) {
      g_cuda_err = "persistent batch solve: grid barrier " + std::to_string(b->h_pc->err_barrier) +
                   " of block " + std::to_string(b->h_pc->err_block) + " waited longer than the deadline (" +
                   std::to_string(b->deadline_us) + " us); the solve was abandoned";
      return BICGK_E_TIMEOUT;
    }
    for (int i = 0; i < b->nsys; ++i) {
      const int *fl = b->h_fl + (size_t)i * F_NFLAG * kMaxKp;
      const double *sc = b->h_sc + (size_t)i * S_NSLOT * kMaxKp;
      for (int c = 0; c < b->k[i]; ++c) {
        iters[off + c] = fl[F_ITERS * kMaxKp + c];
        status[off + c] = fl[F_STATUS * kMaxKp + c];
        if (true_relres) true_relres[off + c] = sc[S_TRUE * kMaxKp + c];
      }
      off += b->k[i];
    }
    b->p_loop_iters = b->h_pc->iters;
    b->last_launches = 1;
    return BICGK_OK;
  }
  for (int i = 0; i < b->nsys; ++i)
    if ((rc = ensure_variant_data(b->ops[i], variant, jacobi, s))) return rc;
  for (int i = 0; i < b->nsys; ++i) {
    Ctl *hc = b->h_ctl + i;
    memset(hc, 0, sizeof(Ctl));
    hc->tol = rel_tol;
    hc->hist = b->ws[i].d_hist;
    hc->maxit = maxit;
    hc->k = b->k[i];
    hc->kp = b->ws[i].kp;
    hc->flags = flags;
    b->h_io[i].B = B[i];
    b->h_io[i].X0 = X0 ? X0[i] : nullptr;
    b->h_io[i].X = X[i];
  }
  CK(cudaMemcpyAsync(b->d_ctl, b->h_ctl, sizeof(Ctl) * b->nsys, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(b->d_io, b->h_io, sizeof(BatchIO) * b->nsys, cudaMemcpyHostToDevice, s));
  auto it = b->graphs.find(gkey);
  if (it == b->graphs.end()) {
    GraphEntry ge;
    if ((rc = batch_build_graph(b, variant, jacobi, &ge))) {
      if (ge.exec) cudaGraphExecDestroy(ge.exec);
      if (ge.graph) cudaGraphDestroy(ge.graph);
      return rc;
    }
    it = b->graphs.emplace(gkey, ge).first;
  }
  CK(cudaGraphLaunch(it->second.exec, s));
  CK(cudaMemcpyAsync(b->h_fl, b->d_fl, sizeof(int) * F_NFLAG * kMaxKp * b->nsys, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(b->h_sc, b->d_sc, sizeof(double) * S_NSLOT * kMaxKp * b->nsys, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(b->h_ctl, b->d_ctl, sizeof(Ctl) * b->nsys, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int i = 0; i < b->nsys; ++i) {
    const Seq q = make_seq(variant, jacobi, seq_opts(b->ops[i], b->k[i], variant));
    const int *fl = b->h_fl + (size_t)i * F_NFLAG * kMaxKp;
    const double *sc = b->h_sc + (size_t)i * S_NSLOT * kMaxKp;
    for (int c = 0; c < b->k[i]; ++c) {
      iters[off + c] = fl[F_ITERS * kMaxKp + c];
      status[off + c] = fl[F_STATUS * kMaxKp + c];
      if (true_relres) true_relres[off + c] = sc[S_TRUE * kMaxKp + c];
    }
    off += b->k[i];
    launches += 2 + (int64_t)q.setup.size() + (int64_t)b->h_ctl[i].loop_iters * q.body.size() + q.fin.size() + 1;
  }
  b->last_launches = launches;
  return BICGK_OK;
}

int bicgk_batch_tune_persistent(bicgk_batch b, int32_t reps, int32_t *rows_per_tile_out, void *stream) {
  if (!b || reps < 1 || reps > 1000) return BICGK_E_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  // right-hand sides of ones and a scratch solution for every system (one buffer each, shared)
  size_t most = 0;
  for (int i = 0; i < b->nsys; ++i) {
    const size_t e = (size_t)b->ops[i]->n * b->k[i];
    if (e > most) most = e;
  }
  double *d_one = nullptr, *d_x = nullptr;
  CK(cudaMalloc(&d_one, sizeof(double) * most));
  cudaError_t e = cudaMalloc(&d_x, sizeof(double) * most);
  if (e != cudaSuccess) {
    cudaFree(d_one);
    return cuda_fail(e, "bicgk_batch_tune_persistent");
  }
  std::vector<double> ones(most, 1.0);
  std::vector<const double *> Bv(b->nsys, d_one);
  std::vector<double *> Xv(b->nsys, d_x);
  std::vector<int32_t> it(1 + std::accumulate(b->k.begin(), b->k.end(), 0)), st(it.size());
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = BICGK_OK;
  if ((e = cudaMemcpy(d_one, ones.data(), sizeof(double) * most, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess)
    rc = cuda_fail(e, "bicgk_batch_tune_persistent");
  // blocks per SM (the kernel variant for 4 or 6) x rows per CTA tile (1, 2, 4, 8 passes of 256
  // threads) at the full co-resident grid, then that shape on 1/2 .. 1/16 of the grid (small
  // problems: fewer blocks take part in every barrier and reduction); 4 fixed iterations of every
  // system
  int best_sub = b->p_sub, best_minb = b->p_minb, best_div = 1;
  float best = 1e30f;
  for (int cfg = 0; cfg < 12 && rc == BICGK_OK; ++cfg) {
    const int sub = cfg < 8 ? 1 << (cfg & 3) : best_sub;
    const int minb = cfg < 8 ? (cfg < 4 ? 4 : 6) : best_minb;
    const int div = cfg < 8 ? 1 : 2 << (cfg - 8);
    if (minb != b->p_minb || div != b->p_div) {
      b->p_minb = minb;
      b->p_div = div;
      b->p_grid = 0;  // re-derived from the variant's occupancy
      persist_drop_graph(b);
    }
    b->p_sub = sub;
    float total = 0.f;
    for (int r = 0; r <= reps && rc == BICGK_OK; ++r) {
      cudaEventRecord(e0, s);
      rc = bicgk_batch_solve(b, Bv.data(), nullptr, Xv.data(), 0.0, 4, BICGK_CLASSICAL_MERGED,
                             BICGK_FLAG_NO_STOP_TEST, BICGK_BATCH_PERSISTENT, it.data(), st.data(), nullptr, stream);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0) total += ms;  // the first solve of a shape captures its graph
    }
    if (rc == BICGK_OK && total < best * 0.98f) {
      best = total;
      best_sub = sub;
      best_minb = minb;
      best_div = div;
    }
  }
  b->p_sub = best_sub;
  if (b->p_minb != best_minb || b->p_div != best_div) b->p_grid = 0;
  b->p_minb = best_minb;
  b->p_div = best_div;
  persist_drop_graph(b);
  if (rc == BICGK_OK) rc = persist_prepare(b);
  if (rc == BICGK_OK && rows_per_tile_out)
    for (int i = 0; i < b->nsys; ++i) rows_per_tile_out[i] = persist_rows_per_pass(b->ws[i].kp) * best_sub;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(d_one);
  cudaFree(d_x);
  return rc;
}

int bicgk_batch_set_deadline(bicgk_batch b, int64_t microseconds) {
  if (!b || microseconds < 0 || microseconds > (int64_t)3600 * 1000000) return BICGK_E_INVALID;
  if (b->deadline_us != microseconds) persist_drop_graph(b);  // the deadline is a kernel argument
  b->deadline_us = microseconds;
  return BICGK_OK;
}

int bicgk_batch_last_loop_iters(bicgk_batch b, int64_t *iters) {
  if (!b || !iters) return BICGK_E_INVALID;
  *iters = b->p_loop_iters;
  return BICGK_OK;
}

int bicgk_batch_persistent_info(bicgk_batch b, int32_t *grid_blocks, int32_t *from_graph, int32_t *graph_error) {
  if (!b) return BICGK_E_INVALID;
  if (grid_blocks) *grid_blocks = b->p_grid;
  if (from_graph) *from_graph = b->pgraph_ok ? 1 : 0;
  if (graph_error) *graph_error = b->p_capture_err;
  return BICGK_OK;
}

int bicgk_batch_last_launches(bicgk_batch b, int64_t *kernel_launches) {
  if (!b || !kernel_launches) return BICGK_E_INVALID;
  *kernel_launches = b->last_launches;
  return BICGK_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------
// Allocation-free solve.
//
// For callers that must not allocate GPU memory during a solve: code that owns
// all device memory through its own pool (a cudaMalloc from inside it would
// bypass the pool and synchronise the device), real-time loops in which an
// allocation's implicit synchronisation is not allowed, and embeddings that
// run with a fixed device-memory budget.  Everything the solve needs beyond
// the caller's arrays lives in one file-scope device array of fixed size,
// held by every GPU that loads this library until the process exits.
namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
void *g_static_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_static_scratch_mu;  // the per-device address is looked up once, by one thread

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// The caller's CSR is checked on the device before any product reads it: row pointers start at 0,
// never decrease and end at nnz; every column index lies in [0, n).  Any violation sets *bad.
__global__ void noalloc_csr_check(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                                  int64_t n, int64_t nnz, int *bad) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool ok = true;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += stride) {
    const int32_t a = rowptr[i];
    if (i == 0 && a != 0) ok = false;
    if (i == n && a != nnz) ok = false;
    if (i < n && rowptr[i + 1] < a) ok = false;
  }
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
    const int32_t c = colidx[e];
    if (c < 0 || c >= n) ok = false;
  }
  if (!ok) atomicOr(bad, 1);
}

}  // namespace

extern "C" int bicgk_solve_noalloc(int64_t n_rows, int64_t nnz, const int32_t *rowptr, const int32_t *colidx,
                                   const double *vals, int32_t k, const double *B, const double *X0,
                                   double rel_tol, int32_t maxit, int variant, int32_t flags, double *X,
                                   int32_t *iters, int32_t *status, double *resid_hist, double *true_relres,
                                   void *stream) {
  if (n_rows < 1 || nnz < 0 || n_rows > INT32_MAX - 1 || nnz > INT32_MAX || !rowptr || (nnz > 0 && (!colidx || !vals)) ||
      !B || !X || !iters || !status || k < 1 || !(rel_tol >= 0.0) || maxit < 0 || maxit > 10000000 ||
      variant < 0 || variant > 9 || (flags & ~1))
    return BICGK_E_INVALID;
  if (k > BICGK_MAX_K) return BICGK_E_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, major = 0, minor = 0, nsm = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
  CK(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  if (major != 10 || minor != 3 || dev >= kMaxDevices) {
    g_cuda_err = "bicgk_solve_noalloc: needs an sm_103 device with index < 64";
    return BICGK_E_UNSUPPORTED;
  }
  // scratch layout: V_NVEC (18) vectors | scalars | flags | block partials | control block | history
  const int kp = pow2_at_least(k);
  const int64_t vstride = (n_rows * kp + 2 + 31) / 32 * 32;
  const int64_t hist_len = (int64_t)(maxit + 1) * kp;
  const size_t b_vec = round256(sizeof(double) * (size_t)vstride * V_NVEC);
  const size_t b_sc = round256(sizeof(double) * S_NSLOT * kMaxKp);
  const size_t b_fl = round256(sizeof(int) * F_NFLAG * kMaxKp);
  const size_t b_part = round256(sizeof(double) * ((size_t)nsm * kPartBlocksPerSm + kMaxRedGroups) * kMaxDots * kMaxKp);
  const size_t b_ctl = round256(sizeof(Ctl));
  const size_t b_hist = round256(sizeof(double) * (size_t)hist_len);
  const size_t b_chk = 256;  // the CSR check's flag
  const size_t need = b_vec + b_sc + b_fl + b_part + b_ctl + b_hist + b_chk;
  if (need > kStaticScratchBytes) {
    g_cuda_err = "bicgk_solve_noalloc: this problem needs " + std::to_string(need) +
                 " bytes of scratch; the static scratch holds " + std::to_string(kStaticScratchBytes);
    return BICGK_E_UNSUPPORTED;
  }
  // first call on this device: host code needs the array's device address (looked up under a
  // lock, so first calls from several host threads at once are safe)
  unsigned char *base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_scratch_mu);
    if (!g_static_scratch_addr[dev]) {
      void *p = nullptr;
      CK(cudaGetSymbolAddress(&p, g_static_scratch));
      g_static_scratch_addr[dev] = p;
    }
    base = static_cast<unsigned char *>(g_static_scratch_addr[dev]);
  }
  // the CSR check, before anything reads the arrays
  int *d_bad = reinterpret_cast<int *>(base + b_vec + b_sc + b_fl + b_part + b_ctl + b_hist);
  int h_bad = 0;
  CK(cudaMemsetAsync(d_bad, 0, sizeof(int), s));
  noalloc_csr_check<<<nsm * 4, 256, 0, s>>>(rowptr, colidx, n_rows, nnz, d_bad);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(&h_bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (h_bad) {
    g_cuda_err = "bicgk_solve_noalloc: malformed CSR (row pointers or column indices)";
    return BICGK_E_BAD_CSR;
  }
  // an operator view of the caller's CSR and the static scratch (owns nothing)
  bicgk_op_s A;
  A.device = dev;
  A.nsm = nsm;
  A.n = n_rows;
  A.nnz = nnz;
  A.d_rowptr = const_cast<int32_t *>(rowptr);
  A.d_col = const_cast<int32_t *>(colidx);
  A.d_val = const_cast<double *>(vals);
  A.stage_cap = 0;  // the k <= 2 SpMM reads CSR entries from global memory (same arithmetic)
  A.opt_spmm_rows = 1;  // ... in the block-tile kernel, whose grid needs no shared memory here
  A.opt_groups = 1;  // one column group, no dot epilogues: bicgk_solve's sequence for k < 8
  A.opt_fused = 1;
  Workspace W;
  W.kp = kp;
  W.vstride = vstride;
  W.d_vec = reinterpret_cast<double *>(base);
  W.d_sc = reinterpret_cast<double *>(base + b_vec);
  W.d_fl = reinterpret_cast<int *>(base + b_vec + b_sc);
  W.d_part = reinterpret_cast<double *>(base + b_vec + b_sc + b_fl);
  W.d_ctl = reinterpret_cast<Ctl *>(base + b_vec + b_sc + b_fl + b_part);
  W.d_hist = reinterpret_cast<double *>(base + b_vec + b_sc + b_fl + b_part + b_ctl);
  // control block: the reduction ticket and the iteration counter start at zero
  Ctl hc;
  memset(&hc, 0, sizeof(hc));
  hc.tol = rel_tol;
  hc.hist = W.d_hist;
  hc.maxit = maxit;
  hc.k = k;
  hc.kp = kp;
  hc.flags = flags;
  CK(cudaMemcpyAsync(W.d_ctl, &hc, sizeof(Ctl), cudaMemcpyHostToDevice, s));
  const KArgs a = make_args(&A, W, 0, cudaGraphConditionalHandle{});
  CK(launch_reset(a, hist_len, s));        // history = NaN, per-column scalars and flags = 0
  CK(launch_pack(B, X0, k, k, a, s));      // B and X0 in, padding columns and pad elements = 0
  const Seq q = make_seq(variant, false, seq_opts(&A, k, variant));
  Ctl poll;
  auto run = [&](const std::vector<Step> &steps) -> int {
    for (const Step &st : steps) CK(launch_step(&A, st, a, s));
    CK(cudaMemcpyAsync(&poll, W.d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return BICGK_OK;
  };
  int rc = run(q.setup);
  if (rc) return rc;
  bool go = poll.any_active && maxit > 0;
  while (go) {
    rc = run(q.body);
    if (rc) return rc;
    go = poll.any_active && poll.iter < maxit;
  }
  for (const Step &st : q.fin) CK(launch_step(&A, st, a, s));
  CK(launch_unpack_role(X, k, k, a, V_X, 1, s));
  CK(cudaMemcpyAsync(iters, W.d_fl + F_ITERS * kMaxKp, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(status, W.d_fl + F_STATUS * kMaxKp, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, s));
  if (true_relres)
    CK(cudaMemcpyAsync(true_relres, W.d_sc + S_TRUE * kMaxKp, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
  if (resid_hist)
    CK(cudaMemcpy2DAsync(resid_hist, sizeof(double) * k, W.d_hist, sizeof(double) * kp, sizeof(double) * k,
                         (size_t)maxit + 1, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return BICGK_OK;
}
