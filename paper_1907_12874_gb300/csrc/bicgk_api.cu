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
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/bicgk.h"
#include "bicgk_dev.cuh"

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
  int spmm;  // 0: streaming op `op`; 1: y = A x; 2: y = b - A x
  int op;
  int x, y, b;
};
Step vec(int op) { return Step{0, op, 0, 0, 0}; }
Step spmm(int x, int y) { return Step{1, -1, x, y, 0}; }
Step resid(int x, int y, int b) { return Step{2, -1, x, y, b}; }

struct Seq {
  std::vector<Step> setup, body, fin;
};

// Kernel sequences of the six forms (one Step = one kernel launch).
Seq make_seq(int variant) {
  Seq q;
  q.fin = {resid(V_X, V_TMP, V_B), vec(OP_TRUE_RES)};
  switch (variant) {
    case BICGK_CLASSICAL_MERGED:  // Algorithm 2
      q.setup = {resid(V_X, V_R, V_B), vec(OP_SETUP_C)};
      q.body = {spmm(V_P, V_V), vec(OP_DELTA), vec(OP_UPD_S), spmm(V_S, V_T), vec(OP_G1), vec(OP_G3),
                vec(OP_UPD_P)};
      break;
    case BICGK_CLASSICAL_PLAIN:  // Algorithm 1, one kernel per line
      q.setup = {resid(V_X, V_R, V_B), vec(OP_SETUP_C)};
      q.body = {spmm(V_P, V_V), vec(OP_DELTA), vec(OP_UPD_S), spmm(V_S, V_T), vec(OP_DOT_TS),
                vec(OP_DOT_PSI), vec(OP_UPD_X_C), vec(OP_UPD_R_C), vec(OP_DOT_RR), vec(OP_DOT_RHO),
                vec(OP_UPD_P)};
      break;
    case BICGK_REORDERED_MERGED:  // Algorithm 6, M^-1 = copy; v^ in V_P, t^ in V_TMP
      q.setup = {resid(V_X, V_R, V_B), vec(OP_SETUP_R)};
      q.body = {spmm(V_P, V_V), vec(OP_DELTA), vec(OP_COPY_SV), vec(OP_UPD_TH), spmm(V_TMP, V_T),
                vec(OP_RG4), vec(OP_COPY_QT), vec(OP_UPD_R_R), vec(OP_RFIN)};
      break;
    case BICGK_REORDERED_PLAIN:
      q.setup = {resid(V_X, V_R, V_B), vec(OP_SETUP_R)};
      q.body = {spmm(V_P, V_V), vec(OP_DELTA), vec(OP_COPY_SV), vec(OP_UPD_TH), spmm(V_TMP, V_T),
                vec(OP_UPD_RT), vec(OP_DOT_T_RT), vec(OP_DOT_T_T), vec(OP_DOT_T_R0), vec(OP_DOT_RT_RT),
                vec(OP_COPY_QT), vec(OP_UPD_R_R), vec(OP_UPD_X_R), vec(OP_UPD_Z_R), vec(OP_UPD_VH)};
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

}  // namespace

struct bicgk_op_s {
  int device = 0;
  int nsm = 0;
  int64_t n = 0, nnz = 0;
  int32_t *d_rowptr = nullptr, *d_col = nullptr;
  double *d_val = nullptr;
  int stage_cap = 0;
  // workspace for one kp
  int kp = 0;
  int64_t vstride = 0;  // doubles between consecutive workspace vectors
  double *d_vec = nullptr;
  double *d_sc = nullptr;
  int *d_fl = nullptr;
  double *d_part = nullptr;
  Ctl *d_ctl = nullptr;
  Ctl *h_ctl = nullptr;       // pinned
  double *d_hist = nullptr;
  int64_t hist_cap = 0;       // doubles
  double *h_hist = nullptr;   // pinned, hist_cap doubles
  int *h_fl = nullptr;        // pinned, F_NFLAG * kMaxKp
  double *h_sc = nullptr;     // pinned, S_NSLOT * kMaxKp
  double *d_stage[2] = {nullptr, nullptr};  // caller-layout staging for host-memory calls
  int64_t stage_elems = 0;
  cudaStream_t cap_stream = nullptr;
  std::map<std::pair<int, int>, GraphEntry> graphs;
  // profiling
  bool profiling = false;
  std::map<std::string, ProfEntry> prof;
  std::vector<std::string> prof_names;
  std::vector<cudaEvent_t> ev;
  // last solve statistics
  int32_t last_loop_iters = 0;
  int64_t last_launches = 0;
  int32_t last_kernels_per_iter = 0;
};

namespace {

KArgs make_args(bicgk_op A, int use_cond, cudaGraphConditionalHandle h) {
  KArgs a;
  for (int r = 0; r < V_NVEC; ++r) a.v[r] = A->d_vec + (int64_t)r * A->vstride;
  a.sc = A->d_sc;
  a.fl = A->d_fl;
  a.part = A->d_part;
  a.ctl = A->d_ctl;
  a.n = A->n;
  a.kp = A->kp;
  a.use_cond = use_cond;
  a.cond = h;
  return a;
}

int vec_grid(bicgk_op A, int op) {
  int nb = vec_blocks_per_sm(op);
  if (nb > 4) nb = 4;
  return A->nsm * nb;
}

int spmm_grid(bicgk_op A, int kp, int mode) {
  return A->nsm * spmm_blocks_per_sm(kp, mode, A->stage_cap);
}

cudaError_t launch_step(bicgk_op A, const Step &st, const KArgs &a, cudaStream_t s) {
  if (st.spmm == 0) return launch_vec(st.op, a, vec_grid(A, st.op), s);
  SpmmArgs sa;
  sa.rowptr = A->d_rowptr;
  sa.colidx = A->d_col;
  sa.vals = A->d_val;
  sa.x = a.v[st.x];
  sa.y = a.v[st.y];
  sa.b = st.spmm == 2 ? a.v[st.b] : nullptr;
  sa.n = A->n;
  sa.stage_cap = A->kp <= 2 ? A->stage_cap : 0;
  const int mode = st.spmm == 2 ? 1 : 0;
  return launch_spmm(A->kp, mode, sa, spmm_grid(A, A->kp, mode), s);
}

std::string step_name(const Step &st, int kp) {
  if (st.spmm == 0) return op_name(st.op);
  return std::string(st.spmm == 2 ? "spmm_resid_k" : "spmm_k") + std::to_string(kp);
}

void drop_graphs(bicgk_op A) {
  for (auto &kv : A->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  A->graphs.clear();
}

void free_workspace(bicgk_op A) {
  drop_graphs(A);
  cudaFree(A->d_vec);
  cudaFree(A->d_sc);
  cudaFree(A->d_fl);
  cudaFree(A->d_part);
  A->d_vec = nullptr;
  A->d_sc = nullptr;
  A->d_fl = nullptr;
  A->d_part = nullptr;
  A->kp = 0;
}

int ensure_workspace(bicgk_op A, int kp) {
  if (A->kp == kp) return BICGK_OK;
  free_workspace(A);
  const int64_t elems = A->n * kp + 2;
  A->vstride = (elems + 31) / 32 * 32;
  const size_t bytes = (size_t)A->vstride * V_NVEC * sizeof(double);
  CK(cudaMalloc(&A->d_vec, bytes));
  CK(cudaMemset(A->d_vec, 0, bytes));
  CK(cudaMalloc(&A->d_sc, sizeof(double) * S_NSLOT * kMaxKp));
  CK(cudaMalloc(&A->d_fl, sizeof(int) * F_NFLAG * kMaxKp));
  CK(cudaMalloc(&A->d_part, sizeof(double) * (size_t)A->nsm * 4 * kMaxDots * kMaxKp));
  CK(cudaMemset(A->d_sc, 0, sizeof(double) * S_NSLOT * kMaxKp));
  CK(cudaMemset(A->d_fl, 0, sizeof(int) * F_NFLAG * kMaxKp));
  A->kp = kp;
  return BICGK_OK;
}

int ensure_hist(bicgk_op A, int64_t elems) {
  if (elems <= A->hist_cap) return BICGK_OK;
  cudaFree(A->d_hist);
  cudaFreeHost(A->h_hist);
  A->d_hist = nullptr;
  A->h_hist = nullptr;
  A->hist_cap = 0;
  CK(cudaMalloc(&A->d_hist, sizeof(double) * elems));
  CK(cudaMallocHost(&A->h_hist, sizeof(double) * elems));
  A->hist_cap = elems;
  return BICGK_OK;
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

// Capture setup + WHILE(body) + final of (variant, kp) into one graph.
int build_graph(bicgk_op A, int variant, GraphEntry *ge) {
  const Seq q = make_seq(variant);
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  ge->graph = g;
  cudaGraphConditionalHandle h;
  CK(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
  const KArgs a = make_args(A, 1, h);
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
  // true residual after the loop
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
  CK(cudaGraphInstantiate(&ge->exec, g, 0));
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

void prof_record(bicgk_op A, const std::string &name, float ms) {
  ProfEntry &e = A->prof[name];
  e.launches += 1;
  e.ms += ms;
}

// Profiling mode: the loop runs from the host, one launch at a time, each bracketed by events.
int run_profiled(bicgk_op A, int variant, const KArgs &a, cudaStream_t s) {
  const Seq q = make_seq(variant);
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
    CK(cudaMemcpyAsync(A->h_ctl, A->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (size_t i = 0; i < steps.size(); ++i) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, A->ev[2 * i], A->ev[2 * i + 1]));
      prof_record(A, step_name(steps[i], A->kp), ms);
    }
    return BICGK_OK;
  };
  int rc = run_list(q.setup);
  if (rc) return rc;
  bool go = A->h_ctl->any_active && A->h_ctl->maxit > 0;
  while (go) {
    rc = run_list(q.body);
    if (rc) return rc;
    go = A->h_ctl->any_active && A->h_ctl->iter < A->h_ctl->maxit;
  }
  return run_list(q.fin);
}

}  // namespace

extern "C" {

const char *bicgk_version(void) { return "bicgk 0.1 sm_103a"; }

const char *bicgk_strerror(int rc) {
  switch (rc) {
    case BICGK_OK: return "ok";
    case BICGK_E_INVALID: return "invalid argument";
    case BICGK_E_BAD_CSR: return "malformed CSR matrix";
    case BICGK_E_CUDA: return "CUDA runtime error";
    case BICGK_E_NOMEM: return "out of memory";
    case BICGK_E_UNSUPPORTED: return "unsupported configuration";
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
  bicgk_op A = new bicgk_op_s();
  A->device = dev;
  A->nsm = nsm;
  A->n = n_rows;
  A->nnz = nnz;
  A->stage_cap = (int)(maxtile < kSpmmStageMax ? maxtile : kSpmmStageMax);
  const cudaMemcpyKind kind = mem == BICGK_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e;
  // pad by 16 bytes so vectorised reads of the last entries stay inside the allocation
  if ((e = cudaMalloc(&A->d_rowptr, sizeof(int32_t) * (n_rows + 1) + 16)) != cudaSuccess ||
      (e = cudaMalloc(&A->d_col, sizeof(int32_t) * nnz + 16)) != cudaSuccess ||
      (e = cudaMalloc(&A->d_val, sizeof(double) * nnz + 16)) != cudaSuccess ||
      (e = cudaMemcpyAsync(A->d_rowptr, rowptr, sizeof(int32_t) * (n_rows + 1), kind, s)) != cudaSuccess ||
      (nnz && (e = cudaMemcpyAsync(A->d_col, colidx, sizeof(int32_t) * nnz, kind, s)) != cudaSuccess) ||
      (nnz && (e = cudaMemcpyAsync(A->d_val, vals, sizeof(double) * nnz, kind, s)) != cudaSuccess) ||
      (e = cudaMallocHost(&A->h_ctl, sizeof(Ctl))) != cudaSuccess ||
      (e = cudaMallocHost(&A->h_fl, sizeof(int) * F_NFLAG * kMaxKp)) != cudaSuccess ||
      (e = cudaMallocHost(&A->h_sc, sizeof(double) * S_NSLOT * kMaxKp)) != cudaSuccess ||
      (e = cudaMalloc(&A->d_ctl, sizeof(Ctl))) != cudaSuccess ||
      (e = cudaMemsetAsync(A->d_ctl, 0, sizeof(Ctl), s)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&A->cap_stream, cudaStreamNonBlocking)) != cudaSuccess ||
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
  free_workspace(A);
  cudaFree(A->d_rowptr);
  cudaFree(A->d_col);
  cudaFree(A->d_val);
  cudaFree(A->d_ctl);
  cudaFree(A->d_hist);
  cudaFree(A->d_stage[0]);
  cudaFree(A->d_stage[1]);
  cudaFreeHost(A->h_ctl);
  cudaFreeHost(A->h_hist);
  cudaFreeHost(A->h_fl);
  cudaFreeHost(A->h_sc);
  for (cudaEvent_t e : A->ev) cudaEventDestroy(e);
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
  if (kp == k) {  // caller layout is the kernel layout
    sa.x = X;
    sa.y = Y;
    CK(launch_spmm(kp, 0, sa, spmm_grid(A, kp, 0), s));
    return BICGK_OK;
  }
  int rc = ensure_workspace(A, kp);
  if (rc) return rc;
  const KArgs a = make_args(A, 0, cudaGraphConditionalHandle{});
  CK(launch_pack(X, nullptr, k, a, s));
  sa.x = a.v[V_B];
  sa.y = a.v[V_TMP];
  CK(launch_spmm(kp, 0, sa, spmm_grid(A, kp, 0), s));
  CK(launch_unpack_role(Y, k, a, V_TMP, 0, s));
  return BICGK_OK;
}

int bicgk_solve(bicgk_op A, int32_t k, const double *B, const double *X0, double rel_tol, int32_t maxit,
                int variant, int32_t flags, int mem, double *X, int32_t *iters, int32_t *status,
                double *resid_hist, double *true_relres, void *stream) {
  if (!A || !B || !X || !iters || !status || k < 1 || !(rel_tol >= 0.0) || maxit < 0 || maxit > 10000000 ||
      variant < 0 || variant > 5 || (mem != BICGK_MEM_HOST && mem != BICGK_MEM_DEVICE) || (flags & ~1))
    return BICGK_E_INVALID;
  if (k > BICGK_MAX_K) return BICGK_E_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  const int kp = pow2_at_least(k);
  int rc = ensure_workspace(A, kp);
  if (rc) return rc;
  const int64_t hist_len = (int64_t)(maxit + 1) * kp;
  rc = ensure_hist(A, hist_len);
  if (rc) return rc;
  const Seq q = make_seq(variant);
  // inputs
  const double *dB = B, *dX0 = X0;
  if (mem == BICGK_MEM_HOST) {
    rc = ensure_stage(A, A->n * k);
    if (rc) return rc;
    CK(cudaMemcpyAsync(A->d_stage[0], B, sizeof(double) * A->n * k, cudaMemcpyHostToDevice, s));
    dB = A->d_stage[0];
    if (X0) {
      CK(cudaMemcpyAsync(A->d_stage[1], X0, sizeof(double) * A->n * k, cudaMemcpyHostToDevice, s));
      dX0 = A->d_stage[1];
    }
  }
  Ctl *hc = A->h_ctl;
  memset(hc, 0, sizeof(Ctl));
  hc->tol = rel_tol;
  hc->hist = A->d_hist;
  hc->maxit = maxit;
  hc->k = k;
  hc->kp = kp;
  hc->flags = flags;
  CK(cudaMemcpyAsync(A->d_ctl, hc, sizeof(Ctl), cudaMemcpyHostToDevice, s));
  const KArgs a0 = make_args(A, 0, cudaGraphConditionalHandle{});
  CK(launch_reset(a0, hist_len, s));
  CK(launch_pack(dB, dX0, k, a0, s));
  int64_t launches = 3;
  if (A->profiling) {
    rc = run_profiled(A, variant, a0, s);
    if (rc) return rc;
  } else {
    auto key = std::make_pair(variant, kp);
    auto it = A->graphs.find(key);
    if (it == A->graphs.end()) {
      GraphEntry ge;
      rc = build_graph(A, variant, &ge);
      if (rc) {
        if (ge.exec) cudaGraphExecDestroy(ge.exec);
        if (ge.graph) cudaGraphDestroy(ge.graph);
        return rc;
      }
      it = A->graphs.emplace(key, ge).first;
    }
    CK(cudaGraphLaunch(it->second.exec, s));
  }
  // outputs
  double *dX = mem == BICGK_MEM_HOST ? A->d_stage[0] : X;
  CK(launch_unpack_role(dX, k, a0, V_X, 1, s));
  if (mem == BICGK_MEM_HOST) CK(cudaMemcpyAsync(X, dX, sizeof(double) * A->n * k, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(A->h_ctl, A->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(A->h_fl, A->d_fl, sizeof(int) * F_NFLAG * kMaxKp, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(A->h_sc, A->d_sc, sizeof(double) * S_NSLOT * kMaxKp, cudaMemcpyDeviceToHost, s));
  if (resid_hist) CK(cudaMemcpyAsync(A->h_hist, A->d_hist, sizeof(double) * hist_len, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int c = 0; c < k; ++c) {
    iters[c] = A->h_fl[F_ITERS * kMaxKp + c];
    status[c] = A->h_fl[F_STATUS * kMaxKp + c];
    if (true_relres) true_relres[c] = A->h_sc[S_TRUE * kMaxKp + c];
  }
  if (resid_hist)
    for (int64_t j = 0; j <= maxit; ++j)
      for (int c = 0; c < k; ++c) resid_hist[j * k + c] = A->h_hist[j * kp + c];
  A->last_loop_iters = A->h_ctl->loop_iters;
  A->last_kernels_per_iter = (int32_t)q.body.size();
  launches += (int64_t)q.setup.size() + (int64_t)A->last_loop_iters * q.body.size() + q.fin.size();
  A->last_launches = launches;
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

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

extern "C" int bicgk_solve_noalloc(int64_t n_rows, int64_t nnz, const int32_t *rowptr, const int32_t *colidx,
                                   const double *vals, int32_t k, const double *B, const double *X0,
                                   double rel_tol, int32_t maxit, int variant, int32_t flags, double *X,
                                   int32_t *iters, int32_t *status, double *resid_hist, double *true_relres,
                                   void *stream) {
  if (n_rows < 1 || nnz < 0 || n_rows > INT32_MAX - 1 || nnz > INT32_MAX || !rowptr || (nnz > 0 && (!colidx || !vals)) ||
      !B || !X || !iters || !status || k < 1 || !(rel_tol >= 0.0) || maxit < 0 || maxit > 10000000 ||
      variant < 0 || variant > 5 || (flags & ~1))
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
  // scratch layout: 14 vectors | scalars | flags | block partials | control block | history
  const int kp = pow2_at_least(k);
  const int64_t vstride = (n_rows * kp + 2 + 31) / 32 * 32;
  const int64_t hist_len = (int64_t)(maxit + 1) * kp;
  const size_t b_vec = round256(sizeof(double) * (size_t)vstride * V_NVEC);
  const size_t b_sc = round256(sizeof(double) * S_NSLOT * kMaxKp);
  const size_t b_fl = round256(sizeof(int) * F_NFLAG * kMaxKp);
  const size_t b_part = round256(sizeof(double) * (size_t)nsm * 4 * kMaxDots * kMaxKp);
  const size_t b_ctl = round256(sizeof(Ctl));
  const size_t b_hist = round256(sizeof(double) * (size_t)hist_len);
  const size_t need = b_vec + b_sc + b_fl + b_part + b_ctl + b_hist;
  if (need > kStaticScratchBytes) {
    g_cuda_err = "bicgk_solve_noalloc: this problem needs " + std::to_string(need) +
                 " bytes of scratch; the static scratch holds " + std::to_string(kStaticScratchBytes);
    return BICGK_E_UNSUPPORTED;
  }
  // first call on this device: host code needs the array's device address
  if (!g_static_scratch_addr[dev]) {
    void *p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_static_scratch));
    g_static_scratch_addr[dev] = p;
  }
  unsigned char *base = static_cast<unsigned char *>(g_static_scratch_addr[dev]);
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
  A.kp = kp;
  A.vstride = vstride;
  A.d_vec = reinterpret_cast<double *>(base);
  A.d_sc = reinterpret_cast<double *>(base + b_vec);
  A.d_fl = reinterpret_cast<int *>(base + b_vec + b_sc);
  A.d_part = reinterpret_cast<double *>(base + b_vec + b_sc + b_fl);
  A.d_ctl = reinterpret_cast<Ctl *>(base + b_vec + b_sc + b_fl + b_part);
  A.d_hist = reinterpret_cast<double *>(base + b_vec + b_sc + b_fl + b_part + b_ctl);
  // control block: the reduction ticket and the iteration counter start at zero
  Ctl hc;
  memset(&hc, 0, sizeof(hc));
  hc.tol = rel_tol;
  hc.hist = A.d_hist;
  hc.maxit = maxit;
  hc.k = k;
  hc.kp = kp;
  hc.flags = flags;
  CK(cudaMemcpyAsync(A.d_ctl, &hc, sizeof(Ctl), cudaMemcpyHostToDevice, s));
  const KArgs a = make_args(&A, 0, cudaGraphConditionalHandle{});
  CK(launch_reset(a, hist_len, s));     // history = NaN, per-column scalars and flags = 0
  CK(launch_pack(B, X0, k, a, s));      // B and X0 in, padding columns and pad elements = 0
  const Seq q = make_seq(variant);
  Ctl poll;
  auto run = [&](const std::vector<Step> &steps) -> int {
    for (const Step &st : steps) CK(launch_step(&A, st, a, s));
    CK(cudaMemcpyAsync(&poll, A.d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
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
  CK(launch_unpack_role(X, k, a, V_X, 1, s));
  CK(cudaMemcpyAsync(iters, A.d_fl + F_ITERS * kMaxKp, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(status, A.d_fl + F_STATUS * kMaxKp, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, s));
  if (true_relres)
    CK(cudaMemcpyAsync(true_relres, A.d_sc + S_TRUE * kMaxKp, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
  if (resid_hist)
    CK(cudaMemcpy2DAsync(resid_hist, sizeof(double) * k, A.d_hist, sizeof(double) * kp, sizeof(double) * k,
                         (size_t)maxit + 1, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return BICGK_OK;
}
