// Streaming kernels of BiCGStab with k right-hand sides: vector updates fused
// with their per-RHS dot products (the merged operations of Sec. 2.2 and the
// listings of Algorithms 2, 4 and 6), the one-operation-per-kernel forms of
// Algorithms 1, 4 and 6 ("basic"), and the per-column scalar recurrences.
//
// One kernel = one pass over the N x kp blocks it touches.  Every thread
// moves double2 chunks in a grid-stride loop; since the stride (in elements)
// is a multiple of kp, a thread always sees the same two columns, so its dot
// partials are per-column registers.  A dot product is reduced in a fixed
// order: warp butterfly over lanes that share columns -> shared memory across
// warps -> one partial per block -> the last block to arrive (atomic ticket,
// no spin-wait) sums the block partials in block order and runs the scalar
// recurrence of the listing for every column.  The same inputs therefore give
// bitwise the same result on every run.
//
// The scalar recurrences (bicgk_rules.cuh) follow the oracle's rules R1-R6
// with explicitly rounded operations.
#include <type_traits>

#include "bicgk_dev.cuh"
#include "bicgk_rules.cuh"

namespace bicgk {

namespace {

__device__ __forceinline__ double2 ld2(const double *p, int64_t i) {
  return reinterpret_cast<const double2 *>(p)[i];
}
__device__ __forceinline__ void st2(double *p, int64_t i, double2 v) { reinterpret_cast<double2 *>(p)[i] = v; }

// y + s*x elementwise (one FMA per element)
__device__ __forceinline__ double2 fma2(double2 s, double2 x, double2 y) {
  return make_double2(fma(s.x, x.x, y.x), fma(s.y, x.y, y.y));
}
__device__ __forceinline__ double2 neg2(double2 s) { return make_double2(-s.x, -s.y); }
__device__ __forceinline__ void dot_acc(double2 &acc, double2 u, double2 w) {
  acc.x = fma(u.x, w.x, acc.x);
  acc.y = fma(u.y, w.y, acc.y);
}
__device__ __forceinline__ double2 sel2(bool u0, bool u1, double2 nv, double2 ov) {
  return make_double2(u0 ? nv.x : ov.x, u1 ? nv.y : ov.y);
}

// Per-thread scalars of its two columns.
struct Sc2 {
  double2 al, om, be;
  double2 cz, cv, dl;    // Algorithm 3: beta (alpha_{j+1}/alpha_j), alpha_{j+1} delta_{j+1}, delta_{j+1}
  float2 alf, omf, bef;  // the same scalars rounded to FP32 (FP32 inner solves)
  bool u0, u1;
};

// Float-float accumulator of one FP32 dot product per column (the FP32 inner solves): the
// products are split exactly (p + e = u*w) and summed with an error-free two-sum, so a thread's
// partial sum carries about 48 bits; it becomes one FP64 value before the FP64 grid reduction.
struct FF2 {
  float2 hi, lo;
};
__device__ __forceinline__ void ff_add(float &hi, float &lo, float u, float w) {
  const float p = __fmul_rn(u, w);
  const float e = fmaf(u, w, -p);
  const float s = __fadd_rn(hi, p);
  const float bb = __fadd_rn(s, -hi);
  const float err = __fadd_rn(__fadd_rn(hi, -__fadd_rn(s, -bb)), __fadd_rn(p, -bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, e));
}
__device__ __forceinline__ void dot_ff(FF2 &acc, float2 u, float2 w) {
  ff_add(acc.hi.x, acc.lo.x, u.x, w.x);
  ff_add(acc.hi.y, acc.lo.y, u.y, w.y);
}
__device__ __forceinline__ double2 to_d2(const double2 &a) { return a; }
__device__ __forceinline__ double2 to_d2(const FF2 &a) {
  return make_double2((double)a.hi.x + (double)a.lo.x, (double)a.hi.y + (double)a.lo.y);
}
__device__ __forceinline__ void acc_zero(double2 &a) { a = make_double2(0.0, 0.0); }
__device__ __forceinline__ void acc_zero(FF2 &a) {
  a.hi = make_float2(0.f, 0.f);
  a.lo = make_float2(0.f, 0.f);
}
__device__ __forceinline__ float2 ld2f(const double *p, int64_t i) {
  return reinterpret_cast<const float2 *>(p)[i];
}
__device__ __forceinline__ void st2f(double *p, int64_t i, float2 v) { reinterpret_cast<float2 *>(p)[i] = v; }
__device__ __forceinline__ float2 fma2f(float2 s, float2 x, float2 y) {
  return make_float2(fmaf(s.x, x.x, y.x), fmaf(s.y, x.y, y.y));
}
__device__ __forceinline__ float2 neg2f(float2 s) { return make_float2(-s.x, -s.y); }
__device__ __forceinline__ float2 sel2f(bool u0, bool u1, float2 nv, float2 ov) {
  return make_float2(u0 ? nv.x : ov.x, u1 ? nv.y : ov.y);
}

// Vector and accumulator types of an op (FP64 ops leave them at the default).
template <class D, class = void>
struct OpTypes {
  using V2 = double2;
  using Acc = double2;
};
template <class D>
struct OpTypes<D, std::void_t<typename D::V2>> {
  using V2 = typename D::V2;
  using Acc = typename D::Acc;
};

// ------------------------------------------------------------------ fused element ops
//
// Each op: ND dots, FIN rule, CTL action, NL loaded double2 per chunk,
// load() then comp() so two chunks can be in flight per thread.

#define V(role) a.v[role]

template <int OP>
struct OpDef;

// ---- set-up
template <>
struct OpDef<OP_SETUP_C> {  // r^_0 = r_0, p_0 = r_0; (b,b), (r_0,r_0)
  static constexpr int ND = 2, FIN = FIN_SETUP, CTL = CTL_START, NL = 2;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_B), i); v[1] = ld2(V(V_R), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &, double2 (&acc)[ND]) {
    st2(V(V_R0), i, v[1]);
    st2(V(V_P), i, v[1]);
    dot_acc(acc[0], v[0], v[0]);
    dot_acc(acc[1], v[1], v[1]);
  }
};
template <>
struct OpDef<OP_SETUP_R> {  // r^_0 = r_0, z_0 = M^-1 r_0, v^_0 = z_0; (b,b), (r_0,r_0)
  static constexpr int ND = 2, FIN = FIN_SETUP, CTL = CTL_START, NL = 2;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_B), i); v[1] = ld2(V(V_R), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &, double2 (&acc)[ND]) {
    st2(V(V_R0), i, v[1]);
    st2(V(V_Z), i, v[1]);
    st2(V(V_P), i, v[1]);
    dot_acc(acc[0], v[0], v[0]);
    dot_acc(acc[1], v[1], v[1]);
  }
};
template <>
struct OpDef<OP_SETUP_P> {  // r^_0 = r_0; p_{-1} = s_{-1} = z_{-1} = v_{-1} = 0; (b,b), (r_0,r_0)
  static constexpr int ND = 2, FIN = FIN_SETUP, CTL = CTL_NONE, NL = 2;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_B), i); v[1] = ld2(V(V_R), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &, double2 (&acc)[ND]) {
    const double2 z = make_double2(0.0, 0.0);
    st2(V(V_R0), i, v[1]);
    st2(V(V_P), i, z);
    st2(V(V_S), i, z);
    st2(V(V_Z), i, z);
    st2(V(V_V), i, z);
    dot_acc(acc[0], v[0], v[0]);
    dot_acc(acc[1], v[1], v[1]);
  }
};

// Dot-only kernel (u, w) with a finalize rule.
template <int VA, int VB, int FIN_, int CTL_>
struct DotOp {
  static constexpr int ND = 1, FIN = FIN_, CTL = CTL_, NL = (VA == VB) ? 1 : 2;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) {
    v[0] = ld2(V(VA), i);
    if constexpr (NL == 2) v[NL - 1] = ld2(V(VB), i);
  }
  __device__ static void comp(const KArgs &, int64_t, const double2 (&v)[NL], const Sc2 &, double2 (&acc)[ND]) {
    dot_acc(acc[0], v[0], v[NL - 1]);
  }
};
template <> struct OpDef<OP_DOT_RW0> : DotOp<V_R0, V_W, FIN_RW0, CTL_START> {};

// ---- classical
template <> struct OpDef<OP_DELTA> : DotOp<V_V, V_R0, FIN_DELTA, CTL_NONE> {};
template <>
struct OpDef<OP_UPD_S> {  // s_j = r_j - alpha_j v_j
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 2;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_R), i); v[1] = ld2(V(V_V), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    st2(V(V_S), i, fma2(neg2(s.al), v[1], v[0]));
  }
};
template <>
struct OpDef<OP_G1> {  // phi = (t,s), psi = (t,t), theta = (s,s)
  static constexpr int ND = 3, FIN = FIN_G1, CTL = CTL_NONE, NL = 2;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_T), i); v[1] = ld2(V(V_S), i); }
  __device__ static void comp(const KArgs &, int64_t, const double2 (&v)[NL], const Sc2 &, double2 (&acc)[ND]) {
    dot_acc(acc[0], v[0], v[1]);
    dot_acc(acc[1], v[0], v[0]);
    dot_acc(acc[2], v[1], v[1]);
  }
};
template <>
struct OpDef<OP_UPD_S_TH> {  // s_j = r_j - alpha_j v_j with theta = (s_j, s_j), stored for group 1
  static constexpr int ND = 1, FIN = FIN_STORE_D0, CTL = CTL_NONE, NL = 2;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_R), i); v[1] = ld2(V(V_V), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&acc)[ND]) {
    const double2 sv = fma2(neg2(s.al), v[1], v[0]);
    st2(V(V_S), i, sv);
    dot_acc(acc[0], sv, sv);
  }
};
template <>
struct OpDef<OP_G1_PP> {  // phi = (t,s), psi = (t,t); theta from OP_UPD_S_TH
  static constexpr int ND = 2, FIN = FIN_G1_TH, CTL = CTL_NONE, NL = 2;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_T), i); v[1] = ld2(V(V_S), i); }
  __device__ static void comp(const KArgs &, int64_t, const double2 (&v)[NL], const Sc2 &, double2 (&acc)[ND]) {
    dot_acc(acc[0], v[0], v[1]);
    dot_acc(acc[1], v[0], v[0]);
  }
};
template <>
struct OpDef<OP_G3> {  // x += alpha p + omega s; r = s - omega t; rho = (r, r_0)
  static constexpr int ND = 1, FIN = FIN_RHO, CTL = CTL_END_ITER, NL = 5;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) {
    v[0] = ld2(V(V_X), i); v[1] = ld2(V(V_P), i); v[2] = ld2(V(V_S), i); v[3] = ld2(V(V_T), i); v[4] = ld2(V(V_R0), i);
  }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&acc)[ND]) {
    const double2 xn = fma2(s.om, v[2], fma2(s.al, v[1], v[0]));
    if (s.u0 | s.u1) st2(V(V_X), i, sel2(s.u0, s.u1, xn, v[0]));
    const double2 r = fma2(neg2(s.om), v[3], v[2]);
    st2(V(V_R), i, r);
    dot_acc(acc[0], r, v[4]);
  }
};
template <>
struct OpDef<OP_UPD_P> {  // p = r + beta (p - omega v)
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 3;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_R), i); v[1] = ld2(V(V_P), i); v[2] = ld2(V(V_V), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    st2(V(V_P), i, fma2(s.be, fma2(neg2(s.om), v[2], v[1]), v[0]));
  }
};
template <> struct OpDef<OP_DOT_TS> : DotOp<V_T, V_S, FIN_STORE_D0, CTL_NONE> {};
template <> struct OpDef<OP_DOT_PSI> : DotOp<V_T, V_T, FIN_PSI, CTL_NONE> {};
template <>
struct OpDef<OP_UPD_X_C> {  // x += alpha p + omega s
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 3;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_X), i); v[1] = ld2(V(V_P), i); v[2] = ld2(V(V_S), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    const double2 xn = fma2(s.om, v[2], fma2(s.al, v[1], v[0]));
    if (s.u0 | s.u1) st2(V(V_X), i, sel2(s.u0, s.u1, xn, v[0]));
  }
};
template <>
struct OpDef<OP_UPD_R_C> {  // r = s - omega t
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 2;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_S), i); v[1] = ld2(V(V_T), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    st2(V(V_R), i, fma2(neg2(s.om), v[1], v[0]));
  }
};
template <> struct OpDef<OP_DOT_RR> : DotOp<V_R, V_R, FIN_RR, CTL_NONE> {};
template <> struct OpDef<OP_DOT_RHO> : DotOp<V_R, V_R0, FIN_RHO, CTL_END_ITER> {};

// ---- reordered (v^ lives in V_P, t^ in V_TMP, r~ in V_RT)
template <>
struct OpDef<OP_COPY_SV> {  // s_j = M^-1 v_j (identity: copy)
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 1;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_V), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &, double2 (&)[1]) { st2(V(V_S), i, v[0]); }
};
template <>
struct OpDef<OP_COPY_QT> {  // q_j = M^-1 t_j (identity: copy)
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 1;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_T), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &, double2 (&)[1]) { st2(V(V_Q), i, v[0]); }
};
template <>
struct OpDef<OP_UPD_TH> {  // t^_j = z_j - alpha_j s_j
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 2;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_Z), i); v[1] = ld2(V(V_S), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    st2(V(V_TMP), i, fma2(neg2(s.al), v[1], v[0]));
  }
};
template <>
struct OpDef<OP_RG4> {  // r~ = r - alpha v; theta = (t,r~), phi = (t,t), psi = (t,r_0), eta = (r~,r~)
  static constexpr int ND = 4, FIN = FIN_R4_MERGED, CTL = CTL_END_ITER, NL = 4;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) {
    v[0] = ld2(V(V_R), i); v[1] = ld2(V(V_V), i); v[2] = ld2(V(V_T), i); v[3] = ld2(V(V_R0), i);
  }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&acc)[ND]) {
    const double2 rt = fma2(neg2(s.al), v[1], v[0]);
    st2(V(V_RT), i, rt);
    dot_acc(acc[0], v[2], rt);
    dot_acc(acc[1], v[2], v[2]);
    dot_acc(acc[2], v[2], v[3]);
    dot_acc(acc[3], rt, rt);
  }
};
template <>
struct OpDef<OP_UPD_R_R> {  // r_{j+1} = r~_j - omega_j t_j
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 2;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_RT), i); v[1] = ld2(V(V_T), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    st2(V(V_R), i, fma2(neg2(s.om), v[1], v[0]));
  }
};
template <>
struct OpDef<OP_RFIN> {  // x += alpha v^ + omega t^; z = t^ - omega q; v^ = z + beta (v^ - omega s)
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 5;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) {
    v[0] = ld2(V(V_X), i); v[1] = ld2(V(V_P), i); v[2] = ld2(V(V_TMP), i); v[3] = ld2(V(V_Q), i); v[4] = ld2(V(V_S), i);
  }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    const double2 xn = fma2(s.om, v[2], fma2(s.al, v[1], v[0]));
    if (s.u0 | s.u1) st2(V(V_X), i, sel2(s.u0, s.u1, xn, v[0]));
    const double2 z = fma2(neg2(s.om), v[3], v[2]);
    st2(V(V_Z), i, z);
    st2(V(V_P), i, fma2(s.be, fma2(neg2(s.om), v[4], v[1]), z));
  }
};
template <>
struct OpDef<OP_UPD_RT> {  // r~ = r - alpha v
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 2;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_R), i); v[1] = ld2(V(V_V), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    st2(V(V_RT), i, fma2(neg2(s.al), v[1], v[0]));
  }
};
template <> struct OpDef<OP_DOT_T_RT> : DotOp<V_T, V_RT, FIN_STORE_D0, CTL_NONE> {};
template <> struct OpDef<OP_DOT_T_T> : DotOp<V_T, V_T, FIN_STORE_D1, CTL_NONE> {};
template <> struct OpDef<OP_DOT_T_R0> : DotOp<V_T, V_R0, FIN_STORE_D2, CTL_NONE> {};
template <> struct OpDef<OP_DOT_RT_RT> : DotOp<V_RT, V_RT, FIN_R4_PLAIN, CTL_END_ITER> {};
template <>
struct OpDef<OP_UPD_X_R> {  // x += alpha v^ + omega t^
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 3;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_X), i); v[1] = ld2(V(V_P), i); v[2] = ld2(V(V_TMP), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    const double2 xn = fma2(s.om, v[2], fma2(s.al, v[1], v[0]));
    if (s.u0 | s.u1) st2(V(V_X), i, sel2(s.u0, s.u1, xn, v[0]));
  }
};
template <>
struct OpDef<OP_UPD_Z_R> {  // z = t^ - omega q
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 2;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_TMP), i); v[1] = ld2(V(V_Q), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    st2(V(V_Z), i, fma2(neg2(s.om), v[1], v[0]));
  }
};
template <>
struct OpDef<OP_UPD_VH> {  // v^ = z + beta (v^ - omega s)
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 3;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_Z), i); v[1] = ld2(V(V_P), i); v[2] = ld2(V(V_S), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    st2(V(V_P), i, fma2(s.be, fma2(neg2(s.om), v[2], v[1]), v[0]));
  }
};

// ---- pipelined
template <>
struct OpDef<OP_PG1> {  // p, s, z recurrences; q = r - alpha s; y = w - alpha z; theta, phi, pi
  static constexpr int ND = 3, FIN = FIN_PG1_MERGED, CTL = CTL_NONE, NL = 7;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) {
    v[0] = ld2(V(V_R), i); v[1] = ld2(V(V_W), i); v[2] = ld2(V(V_T), i); v[3] = ld2(V(V_P), i);
    v[4] = ld2(V(V_S), i); v[5] = ld2(V(V_Z), i); v[6] = ld2(V(V_V), i);
  }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&acc)[ND]) {
    const double2 nom = neg2(s.om), nal = neg2(s.al);
    const double2 p = fma2(s.be, fma2(nom, v[4], v[3]), v[0]);
    const double2 sn = fma2(s.be, fma2(nom, v[5], v[4]), v[1]);
    const double2 zn = fma2(s.be, fma2(nom, v[6], v[5]), v[2]);
    const double2 q = fma2(nal, sn, v[0]);
    const double2 y = fma2(nal, zn, v[1]);
    st2(V(V_P), i, p);
    st2(V(V_S), i, sn);
    st2(V(V_Z), i, zn);
    st2(V(V_Q), i, q);
    st2(V(V_Y), i, y);
    dot_acc(acc[0], q, y);
    dot_acc(acc[1], y, y);
    dot_acc(acc[2], q, q);
  }
};
template <>
struct OpDef<OP_PG2> {  // x += alpha p + omega q; r = q - omega y
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 4;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) {
    v[0] = ld2(V(V_X), i); v[1] = ld2(V(V_P), i); v[2] = ld2(V(V_Q), i); v[3] = ld2(V(V_Y), i);
  }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    const double2 xn = fma2(s.om, v[2], fma2(s.al, v[1], v[0]));
    if (s.u0 | s.u1) st2(V(V_X), i, sel2(s.u0, s.u1, xn, v[0]));
    st2(V(V_R), i, fma2(neg2(s.om), v[3], v[2]));
  }
};
template <>
struct OpDef<OP_PG3> {  // w = y - omega (t - alpha v); (r0,r), (r0,z), (r0,w), (r0,s)
  static constexpr int ND = 4, FIN = FIN_PG3_MERGED, CTL = CTL_END_ITER, NL = 7;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) {
    v[0] = ld2(V(V_Y), i); v[1] = ld2(V(V_T), i); v[2] = ld2(V(V_V), i); v[3] = ld2(V(V_R0), i);
    v[4] = ld2(V(V_R), i); v[5] = ld2(V(V_Z), i); v[6] = ld2(V(V_S), i);
  }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&acc)[ND]) {
    const double2 w = fma2(neg2(s.om), fma2(neg2(s.al), v[2], v[1]), v[0]);
    st2(V(V_W), i, w);
    dot_acc(acc[0], v[3], v[4]);
    dot_acc(acc[1], v[3], v[5]);
    dot_acc(acc[2], v[3], w);
    dot_acc(acc[3], v[3], v[6]);
  }
};
// basic pipelined: one kernel per vector operation
template <int DST, int VR, int VOLD, int VM, bool BETA>
struct PUpd {  // DST = VR + beta (VOLD - omega VM)   or (BETA false) DST = VR - alpha VM
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = BETA ? 3 : 2;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) {
    v[0] = ld2(V(VR), i);
    v[1] = ld2(V(VM), i);
    if constexpr (BETA) v[2] = ld2(V(VOLD), i);
  }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    if constexpr (BETA)
      st2(V(DST), i, fma2(s.be, fma2(neg2(s.om), v[1], v[2]), v[0]));
    else
      st2(V(DST), i, fma2(neg2(s.al), v[1], v[0]));
  }
};
template <> struct OpDef<OP_PU_P> : PUpd<V_P, V_R, V_P, V_S, true> {};
template <> struct OpDef<OP_PU_S> : PUpd<V_S, V_W, V_S, V_Z, true> {};
template <> struct OpDef<OP_PU_Z> : PUpd<V_Z, V_T, V_Z, V_V, true> {};
template <> struct OpDef<OP_PU_Q> : PUpd<V_Q, V_R, V_R, V_S, false> {};
template <> struct OpDef<OP_PU_Y> : PUpd<V_Y, V_W, V_W, V_Z, false> {};
template <> struct OpDef<OP_DOT_QY> : DotOp<V_Q, V_Y, FIN_STORE_D0, CTL_NONE> {};
template <> struct OpDef<OP_DOT_YY> : DotOp<V_Y, V_Y, FIN_STORE_D1, CTL_NONE> {};
template <> struct OpDef<OP_DOT_QQ> : DotOp<V_Q, V_Q, FIN_PG1_PLAIN, CTL_NONE> {};
template <>
struct OpDef<OP_PU_X> {  // x += alpha p + omega q
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 3;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_X), i); v[1] = ld2(V(V_P), i); v[2] = ld2(V(V_Q), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    const double2 xn = fma2(s.om, v[2], fma2(s.al, v[1], v[0]));
    if (s.u0 | s.u1) st2(V(V_X), i, sel2(s.u0, s.u1, xn, v[0]));
  }
};
template <>
struct OpDef<OP_PU_R> {  // r = q - omega y
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 2;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_Q), i); v[1] = ld2(V(V_Y), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    st2(V(V_R), i, fma2(neg2(s.om), v[1], v[0]));
  }
};
template <>
struct OpDef<OP_PU_TMP> {  // tmp = t - alpha v   (first call of the 4-vector update)
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 2;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_T), i); v[1] = ld2(V(V_V), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    st2(V(V_TMP), i, fma2(neg2(s.al), v[1], v[0]));
  }
};
template <>
struct OpDef<OP_PU_W> {  // w = y - omega tmp   (second call)
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 2;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_Y), i); v[1] = ld2(V(V_TMP), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    st2(V(V_W), i, fma2(neg2(s.om), v[1], v[0]));
  }
};
template <> struct OpDef<OP_DOT_R0R> : DotOp<V_R0, V_R, FIN_STORE_D0, CTL_NONE> {};
template <> struct OpDef<OP_DOT_R0Z> : DotOp<V_R0, V_Z, FIN_STORE_D1, CTL_NONE> {};
template <> struct OpDef<OP_DOT_R0W> : DotOp<V_R0, V_W, FIN_STORE_D2, CTL_NONE> {};
template <> struct OpDef<OP_DOT_R0S> : DotOp<V_R0, V_S, FIN_PG3_PLAIN, CTL_END_ITER> {};

// ---- final residual norm (V_TMP holds b - A x)
template <> struct OpDef<OP_TRUE_RES> : DotOp<V_TMP, V_TMP, FIN_TRUE, CTL_NONE> {};


// ---- preconditioner application y = M^-1 x: a copy (M = I) or the Jacobi scaling x_i / a_ii
template <int SRC, int DST, int DST2 = -1>
struct PrecOp {
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 1;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(SRC), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &, double2 (&)[1]) {
    double2 y = v[0];
    if (a.invdiag) {
      const int sh = __ffs(a.kp) - 1;
      y.x *= __ldg(a.invdiag + ((2 * i) >> sh));
      y.y *= __ldg(a.invdiag + ((2 * i + 1) >> sh));
    }
    st2(V(DST), i, y);
    if constexpr (DST2 >= 0) st2(V(DST2), i, y);
  }
};
template <> struct OpDef<OP_PREC_P_Q> : PrecOp<V_P, V_Q> {};
template <> struct OpDef<OP_PREC_S_Y> : PrecOp<V_S, V_Y> {};
template <> struct OpDef<OP_PREC_R_RH> : PrecOp<V_R, V_RH> {};
template <> struct OpDef<OP_PREC_W_WH> : PrecOp<V_W, V_WH> {};
template <> struct OpDef<OP_PREC_Z_ZH> : PrecOp<V_Z, V_ZH> {};
template <> struct OpDef<OP_PREC_R_Z> : PrecOp<V_R, V_Z, V_P> {};  // Alg. 6: z_0 = M^-1 r_0, v^_0 = z_0
template <> struct OpDef<OP_PREC_V_S> : PrecOp<V_V, V_S> {};
template <> struct OpDef<OP_PREC_T_Q> : PrecOp<V_T, V_Q> {};

// X += alpha VP + omega VQ for the columns forming x_{j+1}
template <int VP, int VQ>
struct XUpd {
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 3;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_X), i); v[1] = ld2(V(VP), i); v[2] = ld2(V(VQ), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    const double2 xn = fma2(s.om, v[2], fma2(s.al, v[1], v[0]));
    if (s.u0 | s.u1) st2(V(V_X), i, sel2(s.u0, s.u1, xn, v[0]));
  }
};
// DST = VR - omega VM
template <int DST, int VR, int VM>
struct OUpd {
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 2;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(VR), i); v[1] = ld2(V(VM), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    st2(V(DST), i, fma2(neg2(s.om), v[1], v[0]));
  }
};

// ---- Algorithm 5 (p^ in V_Q, s^ in V_Y)
template <>
struct OpDef<OP5_RRHO> {  // r_{j+1} = s - omega t with rho_{j+1} = (r_{j+1}, r_0)
  static constexpr int ND = 1, FIN = FIN_RHO, CTL = CTL_END_ITER, NL = 3;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_S), i); v[1] = ld2(V(V_T), i); v[2] = ld2(V(V_R0), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&acc)[ND]) {
    const double2 r = fma2(neg2(s.om), v[1], v[0]);
    st2(V(V_R), i, r);
    dot_acc(acc[0], r, v[2]);
  }
};
template <> struct OpDef<OP5_UPD_X> : XUpd<V_Q, V_Y> {};  // x += alpha p^ + omega s^

// ---- Algorithm 7 (p^ in V_P, q^ in V_RT, s^ z^ r^ w^ in V_SH V_ZH V_RH V_WH)
template <>
struct OpDef<OP7_SETUP> {  // r^_0 := r_0 kept as r_0; step -1 vectors p^, s^, z^, s, z, v = 0
  static constexpr int ND = 2, FIN = FIN_SETUP, CTL = CTL_NONE, NL = 2;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_B), i); v[1] = ld2(V(V_R), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &, double2 (&acc)[ND]) {
    const double2 z = make_double2(0.0, 0.0);
    st2(V(V_R0), i, v[1]);
    st2(V(V_P), i, z);
    st2(V(V_SH), i, z);
    st2(V(V_ZH), i, z);
    st2(V(V_S), i, z);
    st2(V(V_Z), i, z);
    st2(V(V_V), i, z);
    dot_acc(acc[0], v[0], v[0]);
    dot_acc(acc[1], v[1], v[1]);
  }
};
template <>
struct OpDef<OP7_L1> {  // p^ = r^ + beta (p^ - omega s^); s^ = w^ + beta (s^ - omega z^); q^ = r^ - alpha s^
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 5;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) {
    v[0] = ld2(V(V_RH), i); v[1] = ld2(V(V_P), i); v[2] = ld2(V(V_SH), i); v[3] = ld2(V(V_WH), i); v[4] = ld2(V(V_ZH), i);
  }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    const double2 nom = neg2(s.om);
    st2(V(V_P), i, fma2(s.be, fma2(nom, v[2], v[1]), v[0]));
    const double2 sh = fma2(s.be, fma2(nom, v[4], v[2]), v[3]);
    st2(V(V_SH), i, sh);
    st2(V(V_RT), i, fma2(neg2(s.al), sh, v[0]));
  }
};
template <>
struct OpDef<OP7_L2> {  // s, z, q, y with theta = (q,y), phi = (y,y), pi = (q,q)
  static constexpr int ND = 3, FIN = FIN_PG1_MERGED, CTL = CTL_NONE, NL = 6;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) {
    v[0] = ld2(V(V_W), i); v[1] = ld2(V(V_S), i); v[2] = ld2(V(V_Z), i); v[3] = ld2(V(V_T), i);
    v[4] = ld2(V(V_V), i); v[5] = ld2(V(V_R), i);
  }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&acc)[ND]) {
    const double2 nom = neg2(s.om), nal = neg2(s.al);
    const double2 sn = fma2(s.be, fma2(nom, v[2], v[1]), v[0]);
    const double2 zn = fma2(s.be, fma2(nom, v[4], v[2]), v[3]);
    const double2 q = fma2(nal, sn, v[5]);
    const double2 y = fma2(nal, zn, v[0]);
    st2(V(V_S), i, sn);
    st2(V(V_Z), i, zn);
    st2(V(V_Q), i, q);
    st2(V(V_Y), i, y);
    dot_acc(acc[0], q, y);
    dot_acc(acc[1], y, y);
    dot_acc(acc[2], q, q);
  }
};
template <>
struct OpDef<OP7_L4> {  // x += alpha p^ + omega q^; r^ = q^ - omega (w^ - alpha z^)
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 5;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) {
    v[0] = ld2(V(V_X), i); v[1] = ld2(V(V_P), i); v[2] = ld2(V(V_RT), i); v[3] = ld2(V(V_WH), i); v[4] = ld2(V(V_ZH), i);
  }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    const double2 xn = fma2(s.om, v[2], fma2(s.al, v[1], v[0]));
    if (s.u0 | s.u1) st2(V(V_X), i, sel2(s.u0, s.u1, xn, v[0]));
    st2(V(V_RH), i, fma2(neg2(s.om), fma2(neg2(s.al), v[4], v[3]), v[2]));
  }
};
template <>
struct OpDef<OP7_L5> {  // r = q - omega y; w = y - omega (t - alpha v); (r0,r), (r0,z), (r0,w), (r0,s)
  static constexpr int ND = 4, FIN = FIN_PG3_MERGED, CTL = CTL_END_ITER, NL = 7;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) {
    v[0] = ld2(V(V_Q), i); v[1] = ld2(V(V_Y), i); v[2] = ld2(V(V_T), i); v[3] = ld2(V(V_V), i);
    v[4] = ld2(V(V_R0), i); v[5] = ld2(V(V_Z), i); v[6] = ld2(V(V_S), i);
  }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&acc)[ND]) {
    const double2 nom = neg2(s.om);
    const double2 r = fma2(nom, v[1], v[0]);
    const double2 w = fma2(nom, fma2(neg2(s.al), v[3], v[2]), v[1]);
    st2(V(V_R), i, r);
    st2(V(V_W), i, w);
    dot_acc(acc[0], v[4], r);
    dot_acc(acc[1], v[4], v[5]);
    dot_acc(acc[2], v[4], w);
    dot_acc(acc[3], v[4], v[6]);
  }
};
template <> struct OpDef<OP7_PU_PH> : PUpd<V_P, V_RH, V_P, V_SH, true> {};
template <> struct OpDef<OP7_PU_SH> : PUpd<V_SH, V_WH, V_SH, V_ZH, true> {};
template <> struct OpDef<OP7_PU_QH> : PUpd<V_RT, V_RH, V_RH, V_SH, false> {};
template <> struct OpDef<OP7_X> : XUpd<V_P, V_RT> {};
template <> struct OpDef<OP7_TMPH> : PUpd<V_TMP, V_WH, V_WH, V_ZH, false> {};  // 4-vector op, first call
template <> struct OpDef<OP7_RH> : OUpd<V_RH, V_RT, V_TMP> {};                 // second call

// ---- Algorithm 3 (u in V_W, f_0 = A^T r_0 in V_RT); kernels use alpha_{j+1}, beta_{j+1},
// delta_{j+1} and the coefficients cz = beta (alpha_{j+1}/alpha_j), cv = alpha_{j+1} delta_{j+1}
template <>
struct OpDef<OP3_SETUP> {  // r^_0 = r_0; q_0 = v_0 = z_0 = 0; (b,b), (r_0,r_0)
  static constexpr int ND = 2, FIN = FIN_SETUP, CTL = CTL_NONE, NL = 2;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_B), i); v[1] = ld2(V(V_R), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &, double2 (&acc)[ND]) {
    const double2 z = make_double2(0.0, 0.0);
    st2(V(V_R0), i, v[1]);
    st2(V(V_Q), i, z);
    st2(V(V_V), i, z);
    st2(V(V_Z), i, z);
    dot_acc(acc[0], v[0], v[0]);
    dot_acc(acc[1], v[1], v[1]);
  }
};
template <> struct OpDef<OP3_SIG0> : DotOp<V_R0, V_W, FIN_I_START, CTL_START> {};  // sigma_0 = (r_0, u_0)
template <>
struct OpDef<OP3_L1> {  // z = alpha r + cz z - cv v; v = u + beta v - delta q; s = r - alpha v
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 5;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) {
    v[0] = ld2(V(V_R), i); v[1] = ld2(V(V_Z), i); v[2] = ld2(V(V_V), i); v[3] = ld2(V(V_W), i); v[4] = ld2(V(V_Q), i);
  }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    const double2 ar = make_double2(s.al.x * v[0].x, s.al.y * v[0].y);
    st2(V(V_Z), i, fma2(neg2(s.cv), v[2], fma2(s.cz, v[1], ar)));
    const double2 vn = fma2(neg2(s.dl), v[4], fma2(s.be, v[2], v[3]));
    st2(V(V_V), i, vn);
    st2(V(V_S), i, fma2(neg2(s.al), vn, v[0]));
  }
};
template <>
struct OpDef<OP3_L2> {  // t = u - alpha q with the seven dot products
  static constexpr int ND = 7, FIN = FIN_I7_MERGED, CTL = CTL_END_ITER, NL = 5;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) {
    v[0] = ld2(V(V_W), i); v[1] = ld2(V(V_Q), i); v[2] = ld2(V(V_R0), i); v[3] = ld2(V(V_S), i); v[4] = ld2(V(V_RT), i);
  }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&acc)[ND]) {
    const double2 t = fma2(neg2(s.al), v[1], v[0]);
    st2(V(V_T), i, t);
    dot_acc(acc[0], v[2], v[3]);
    dot_acc(acc[1], v[2], v[1]);
    dot_acc(acc[2], v[4], v[3]);
    dot_acc(acc[3], v[4], t);
    dot_acc(acc[4], v[3], t);
    dot_acc(acc[5], t, t);
    dot_acc(acc[6], v[3], v[3]);
  }
};
template <>
struct OpDef<OP3_L3> {  // r = s - omega t; x += z + omega s
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 4;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) {
    v[0] = ld2(V(V_S), i); v[1] = ld2(V(V_T), i); v[2] = ld2(V(V_X), i); v[3] = ld2(V(V_Z), i);
  }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    st2(V(V_R), i, fma2(neg2(s.om), v[1], v[0]));
    const double2 xz = make_double2(v[2].x + v[3].x, v[2].y + v[3].y);
    const double2 xn = fma2(s.om, v[0], xz);
    if (s.u0 | s.u1) st2(V(V_X), i, sel2(s.u0, s.u1, xn, v[2]));
  }
};
template <>
struct OpDef<OP3_Z> {  // z = alpha r + cz z - cv v   (one extended-BLAS call)
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 3;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_R), i); v[1] = ld2(V(V_Z), i); v[2] = ld2(V(V_V), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    const double2 ar = make_double2(s.al.x * v[0].x, s.al.y * v[0].y);
    st2(V(V_Z), i, fma2(neg2(s.cv), v[2], fma2(s.cz, v[1], ar)));
  }
};
template <>
struct OpDef<OP3_V> {  // v = u + beta v - delta q
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 3;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_W), i); v[1] = ld2(V(V_V), i); v[2] = ld2(V(V_Q), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    st2(V(V_V), i, fma2(neg2(s.dl), v[2], fma2(s.be, v[1], v[0])));
  }
};
template <> struct OpDef<OP3_S> : PUpd<V_S, V_R, V_R, V_V, false> {};  // s = r - alpha v
template <> struct OpDef<OP3_T> : PUpd<V_T, V_W, V_W, V_Q, false> {};  // t = u - alpha q
template <> struct OpDef<OP3_D_R0S> : DotOp<V_R0, V_S, FIN_STORE_D0, CTL_NONE> {};
template <> struct OpDef<OP3_D_R0Q> : DotOp<V_R0, V_Q, FIN_STORE_D1, CTL_NONE> {};
template <> struct OpDef<OP3_D_F0S> : DotOp<V_RT, V_S, FIN_STORE_D2, CTL_NONE> {};
template <> struct OpDef<OP3_D_F0T> : DotOp<V_RT, V_T, FIN_STORE_D3, CTL_NONE> {};
template <> struct OpDef<OP3_D_ST> : DotOp<V_S, V_T, FIN_STORE_D4, CTL_NONE> {};
template <> struct OpDef<OP3_D_TT> : DotOp<V_T, V_T, FIN_STORE_D5, CTL_NONE> {};
template <> struct OpDef<OP3_D_SS> : DotOp<V_S, V_S, FIN_I7_PLAIN, CTL_END_ITER> {};
template <>
struct OpDef<OP3_X> {  // x += z + omega s
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 3;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_X), i); v[1] = ld2(V(V_Z), i); v[2] = ld2(V(V_S), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    const double2 xz = make_double2(v[0].x + v[1].x, v[0].y + v[1].y);
    const double2 xn = fma2(s.om, v[2], xz);
    if (s.u0 | s.u1) st2(V(V_X), i, sel2(s.u0, s.u1, xn, v[0]));
  }
};

// ---- mixed-precision refinement, FP32 inner solve (roles hold float arrays)
struct Op32 {
  using V2 = float2;
  using Acc = FF2;
};
template <>
struct OpDef<OP32_SETUP> : Op32 {  // d_0 = 0, r_0 = b, r^_0 = r_0, p_0 = r_0; (b,b), (r_0,r_0)
  static constexpr int ND = 2, FIN = FIN_SETUP, CTL = CTL_START, NL = 1;
  __device__ static void load(const KArgs &a, int64_t i, float2 (&v)[NL]) { v[0] = ld2f(V(V_B), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const float2 (&v)[NL], const Sc2 &, FF2 (&acc)[ND]) {
    st2f(V(V_X), i, make_float2(0.f, 0.f));
    st2f(V(V_R), i, v[0]);
    st2f(V(V_R0), i, v[0]);
    st2f(V(V_P), i, v[0]);
    dot_ff(acc[0], v[0], v[0]);
    dot_ff(acc[1], v[0], v[0]);
  }
};
template <>
struct OpDef<OP32_DELTA> : Op32 {  // delta = (v, r^_0)
  static constexpr int ND = 1, FIN = FIN_DELTA, CTL = CTL_NONE, NL = 2;
  __device__ static void load(const KArgs &a, int64_t i, float2 (&v)[NL]) { v[0] = ld2f(V(V_V), i); v[1] = ld2f(V(V_R0), i); }
  __device__ static void comp(const KArgs &, int64_t, const float2 (&v)[NL], const Sc2 &, FF2 (&acc)[ND]) {
    dot_ff(acc[0], v[0], v[1]);
  }
};
template <>
struct OpDef<OP32_UPD_S> : Op32 {  // s = r - alpha v
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 2;
  __device__ static void load(const KArgs &a, int64_t i, float2 (&v)[NL]) { v[0] = ld2f(V(V_R), i); v[1] = ld2f(V(V_V), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const float2 (&v)[NL], const Sc2 &s, FF2 (&)[1]) {
    st2f(V(V_S), i, fma2f(neg2f(s.alf), v[1], v[0]));
  }
};
template <>
struct OpDef<OP32_G1> : Op32 {  // phi = (t,s), psi = (t,t), theta = (s,s)
  static constexpr int ND = 3, FIN = FIN_G1, CTL = CTL_NONE, NL = 2;
  __device__ static void load(const KArgs &a, int64_t i, float2 (&v)[NL]) { v[0] = ld2f(V(V_T), i); v[1] = ld2f(V(V_S), i); }
  __device__ static void comp(const KArgs &, int64_t, const float2 (&v)[NL], const Sc2 &, FF2 (&acc)[ND]) {
    dot_ff(acc[0], v[0], v[1]);
    dot_ff(acc[1], v[0], v[0]);
    dot_ff(acc[2], v[1], v[1]);
  }
};
template <>
struct OpDef<OP32_G3> : Op32 {  // d += alpha p + omega s; r = s - omega t; rho = (r, r^_0)
  static constexpr int ND = 1, FIN = FIN_RHO, CTL = CTL_END_ITER, NL = 5;
  __device__ static void load(const KArgs &a, int64_t i, float2 (&v)[NL]) {
    v[0] = ld2f(V(V_X), i); v[1] = ld2f(V(V_P), i); v[2] = ld2f(V(V_S), i); v[3] = ld2f(V(V_T), i); v[4] = ld2f(V(V_R0), i);
  }
  __device__ static void comp(const KArgs &a, int64_t i, const float2 (&v)[NL], const Sc2 &s, FF2 (&acc)[ND]) {
    const float2 xn = fma2f(s.omf, v[2], fma2f(s.alf, v[1], v[0]));
    if (s.u0 | s.u1) st2f(V(V_X), i, sel2f(s.u0, s.u1, xn, v[0]));
    const float2 r = fma2f(neg2f(s.omf), v[3], v[2]);
    st2f(V(V_R), i, r);
    dot_ff(acc[0], r, v[4]);
  }
};
template <>
struct OpDef<OP32_UPD_P> : Op32 {  // p = r + beta (p - omega v)
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 3;
  __device__ static void load(const KArgs &a, int64_t i, float2 (&v)[NL]) { v[0] = ld2f(V(V_R), i); v[1] = ld2f(V(V_P), i); v[2] = ld2f(V(V_V), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const float2 (&v)[NL], const Sc2 &s, FF2 (&)[1]) {
    st2f(V(V_P), i, fma2f(s.bef, fma2f(neg2f(s.omf), v[2], v[1]), v[0]));
  }
};

// ---- mixed-precision refinement, FP64 outer steps (V_Q: FP32 b of the inner solve, V_Y: its d)
template <> struct OpDef<OP_IR_SETUP> : DotOp<V_B, V_B, FIN_IR_SETUP, CTL_NONE> {};
template <>
struct OpDef<OP_IR_RESID> {  // (r, r) of r = b - A x; the inner right-hand side b32 = fl32(r)
  static constexpr int ND = 1, FIN = FIN_IR_RESID, CTL = CTL_OUTER, NL = 1;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_R), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &, double2 (&acc)[ND]) {
    st2f(V(V_Q), i, make_float2((float)v[0].x, (float)v[0].y));
    dot_acc(acc[0], v[0], v[0]);
  }
};
template <>
struct OpDef<OP_IR_UPDATE> {  // x += d for the columns this pass refines
  static constexpr int ND = 0, FIN = FIN_NONE, CTL = CTL_NONE, NL = 1;
  __device__ static void load(const KArgs &a, int64_t i, double2 (&v)[NL]) { v[0] = ld2(V(V_X), i); }
  __device__ static void comp(const KArgs &a, int64_t i, const double2 (&v)[NL], const Sc2 &s, double2 (&)[1]) {
    if (!(s.u0 | s.u1)) return;
    const float2 d = ld2f(V(V_Y), i);
    const double2 xn = make_double2(v[0].x + (double)d.x, v[0].y + (double)d.y);
    st2(V(V_X), i, sel2(s.u0, s.u1, xn, v[0]));
  }
};

#undef V

// ------------------------------------------------------------------ the kernel

template <int ND, int NT>
struct RedSmem {
  double red[NT / 32][ND < 4 ? ND : 4][kMaxKp];  // warp partials, up to 4 dots at a time
  double sums[ND * kMaxKp];
  unsigned int ticket;
};

// NT: threads per block of the calling kernel (512 for the streaming kernels, 256 for the SpMM
// with a dot epilogue); every thread holds the partial sums of its two columns.
template <class D, int NT = kVecThreads, int ND = D::ND>
__device__ void reduce_and_finalize(const KArgs &a, double2 (&acc)[ND > 0 ? ND : 1]) {
  constexpr int NC = ND < 4 ? ND : 4;  // dots per shared-memory chunk
  __shared__ RedSmem<ND, NT> sm;
  const int kp = a.kp;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double v0[ND], v1[ND];
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    if (kp == 1) {
      v0[d] = acc[d].x + acc[d].y;
      v1[d] = 0.0;
    } else {
      v0[d] = acc[d].x;
      v1[d] = acc[d].y;
    }
  }
  // lanes l and l^m hold the same columns iff m is a multiple of kp/2 (kp >= 2)
  const int mstart = kp == 1 ? 1 : (kp >> 1);
  for (int m = mstart; m < 32; m <<= 1) {
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      v0[d] += __shfl_xor_sync(0xffffffffu, v0[d], m);
      if (kp > 1) v1[d] += __shfl_xor_sync(0xffffffffu, v1[d], m);
    }
  }
  const int nout = ND * kp;
  double *mypart = a.part + (size_t)blockIdx.x * (kMaxDots * kMaxKp);
#pragma unroll
  for (int d0 = 0; d0 < ND; d0 += NC) {
    if (kp == 1) {
      if (lane == 0)
#pragma unroll
        for (int d = 0; d < NC; ++d)
          if (d0 + d < ND) sm.red[warp][d][0] = v0[d0 + d];
    } else if (lane < (kp >> 1)) {
#pragma unroll
      for (int d = 0; d < NC; ++d)
        if (d0 + d < ND) {
          sm.red[warp][d][2 * lane] = v0[d0 + d];
          sm.red[warp][d][2 * lane + 1] = v1[d0 + d];
        }
    }
    __syncthreads();
    const int nchunk = (ND - d0 < NC ? ND - d0 : NC) * kp;
    for (int t = threadIdx.x; t < nchunk; t += blockDim.x) {
      const int d = t / kp, c = t - d * kp;
      double s = 0.0;
      for (int w = 0; w < NT / 32; ++w) s += sm.red[w][d][c];
      mypart[(d0 + d) * kMaxKp + c] = s;
    }
    __syncthreads();
  }
  // Fixed-order sum of the block partials; no block ever waits for another.  With few partial
  // sums (grid x outputs <= kOneLevelMax) the last block to arrive adds them all in block order.
  // With many, that single block's FP64 additions would dominate, so the sum goes in two
  // levels: the last block of each group of kRedGroup blocks adds its group (ascending block
  // order) into a group partial, and the last group to finish adds the group partials.
  constexpr int kStride = kMaxDots * kMaxKp;
  constexpr int kOneLevelMax = 8192;   // partial sums one final block adds at most
  constexpr int kOneLevelBlocks = 640; // ... and blocks (the streaming grids have at most 608)
  const int nblk = gridDim.x;
  const bool two_level = nblk * nout > kOneLevelMax || nblk > kOneLevelBlocks;
  const int ngrp = two_level ? (nblk + kRedGroup - 1) / kRedGroup : 1;
  const double *top = a.part;  // partials the final block adds: block partials or group partials
  // the threads that wrote partials make them visible before thread 0 takes the ticket
  if ((int)threadIdx.x < NC * kp) __threadfence();
  __syncthreads();
  if (two_level) {
    const int g = blockIdx.x / kRedGroup;
    const int g0 = g * kRedGroup;
    const int gsz = (g0 + kRedGroup < nblk) ? kRedGroup : nblk - g0;
    if (threadIdx.x == 0) sm.ticket = atomicAdd(&a.ctl->gticket[g], 1u);
    __syncthreads();
    if (sm.ticket != (unsigned)gsz - 1) return;
    __threadfence();
    double *gpart = a.part + (size_t)(nblk + g) * kStride;
    for (int t = threadIdx.x; t < nout; t += blockDim.x) {
      const int d = t / kp, c = t - d * kp;
      const double *src = a.part + (size_t)g0 * kStride + d * kMaxKp + c;
      double s = 0.0;
#pragma unroll 4
      for (int b = 0; b < gsz; ++b) s += __ldcg(src + (size_t)b * kStride);
      gpart[d * kMaxKp + c] = s;
    }
    if (threadIdx.x == 0) a.ctl->gticket[g] = 0;
    if ((int)threadIdx.x < nout) __threadfence();
    __syncthreads();
    top = a.part + (size_t)nblk * kStride;
  }
  if (threadIdx.x == 0) sm.ticket = atomicAdd(&a.ctl->ticket, 1u);
  __syncthreads();
  const int ntop = two_level ? ngrp : nblk;
  if (sm.ticket != (unsigned)ngrp - 1 + (two_level ? 0 : nblk - 1)) return;
  __threadfence();
  // few outputs (small kp): several warps per output, so that every thread loads at most a few
  // partials (one round trip to L2); their warp sums are added in warp order
  int wpo = 1;
  while (wpo * 2 * nout * 32 <= (int)blockDim.x) wpo *= 2;
  if (wpo > 1) {
    const int tpo = wpo * 32;
    const int o = threadIdx.x / tpo, sub = threadIdx.x % tpo;
    double s = 0.0;
    if (o < nout) {
      const int d = o / kp, c = o - d * kp;
#pragma unroll 4
      for (int b = sub; b < ntop; b += tpo) s += __ldcg(top + (size_t)b * kStride + d * kMaxKp + c);
    }
    for (int m = 16; m >= 1; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
    if (lane == 0) sm.red[warp][0][0] = s;
    __syncthreads();
    if ((int)threadIdx.x < nout) {
      double t = 0.0;
      for (int j = 0; j < wpo; ++j) t += sm.red[threadIdx.x * wpo + j][0][0];
      sm.sums[threadIdx.x] = t;
    }
  }
  int tpo = 32;  // lanes per output in the final sum (strided, then a butterfly)
  while (tpo > 1 && tpo * nout > (int)blockDim.x) tpo >>= 1;
  const int groups = blockDim.x / tpo;
  for (int o0 = 0; o0 < (wpo > 1 ? 0 : nout); o0 += groups) {
    const int o = o0 + threadIdx.x / tpo, sub = threadIdx.x % tpo;
    double s = 0.0;
    if (o < nout) {
      const int d = o / kp, c = o - d * kp;
#pragma unroll 4
      for (int b = sub; b < ntop; b += tpo) s += __ldcg(top + (size_t)b * kStride + d * kMaxKp + c);
    }
    for (int m = tpo >> 1; m >= 1; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
    if (o < nout && sub == 0) sm.sums[o] = s;
  }
  __syncthreads();
  if ((int)threadIdx.x < kp) fin_col<D::FIN>(a, threadIdx.x, sm.sums, kp);
  __syncthreads();
  if (threadIdx.x == 0) {
    a.ctl->ticket = 0;
    fin_ctl<D::CTL>(a);
  }
}

// Blocks of 512 threads per SM a streaming kernel is compiled for.  Two (at most 64 registers)
// suit most ops.  The fused groups of the Pipelined forms and of Algorithm 3 hold many vectors
// per chunk and spilled at 64 registers; compiled for one block of up to 128 registers they run
// 3-8 % faster at k <= 8 and the same at k = 32 (measured).  Group 3 of Algorithm 2 and the last
// group of Algorithm 6 spill too but are as fast or faster at two blocks when the two column
// groups of a solve run concurrently, so they keep two.
template <int OP>
struct VecMinBlocks {
  static constexpr int value = 2;
};
#define BICGK_ONE_BLOCK(op) \
  template <>               \
  struct VecMinBlocks<op> { \
    static constexpr int value = 1; \
  };
BICGK_ONE_BLOCK(OP_PG1)
BICGK_ONE_BLOCK(OP_PG3)
BICGK_ONE_BLOCK(OP7_L1)
BICGK_ONE_BLOCK(OP7_L2)
BICGK_ONE_BLOCK(OP7_L4)
BICGK_ONE_BLOCK(OP7_L5)
BICGK_ONE_BLOCK(OP3_L1)
BICGK_ONE_BLOCK(OP3_L2)
#undef BICGK_ONE_BLOCK

// Chunks of two doubles each thread loads before computing (memory-level parallelism): two
// for every op.  Group 3 of Algorithm 2 streams five vectors and spills 60 bytes per thread with
// two chunks under the 64-register cap, yet the four-group benchmark loop runs 0.5 % faster with
// them than with one (10,607 against 10,553 RHS-iterations/s, three runs each; the same
// per-thread order of the chunks, so the same results).
template <int OP>
struct VecChunks {
  static constexpr int value = 2;
};

template <int OP>
__global__ void __launch_bounds__(kVecThreads, VecMinBlocks<OP>::value) vec_kernel(const KArgs a) {
  using D = OpDef<OP>;
  constexpr int ND = D::ND;
  const int kp = a.kp;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int c0 = kp == 1 ? 0 : (int)((2 * gtid) & (kp - 1));
  const int c1 = kp == 1 ? 0 : c0 + 1;
  Sc2 s;
  s.al = make_double2(SC(S_ALPHA, c0), SC(S_ALPHA, c1));
  s.om = make_double2(SC(S_OMEGA, c0), SC(S_OMEGA, c1));
  s.be = make_double2(SC(S_BETA, c0), SC(S_BETA, c1));
  s.cz = make_double2(SC(S_CZ, c0), SC(S_CZ, c1));
  s.cv = make_double2(SC(S_CV, c0), SC(S_CV, c1));
  s.dl = make_double2(SC(S_DLT, c0), SC(S_DLT, c1));
  s.alf = make_float2((float)s.al.x, (float)s.al.y);
  s.omf = make_float2((float)s.om.x, (float)s.om.y);
  s.bef = make_float2((float)s.be.x, (float)s.be.y);
  // the x-update mask: columns that form x_{j+1} (refinement update: columns the pass refines)
  const int mflag = OP == OP_IR_UPDATE ? F_ACT : F_XUPD;
  s.u0 = FL(mflag, c0) != 0;
  s.u1 = FL(mflag, c1) != 0;
  using V2 = typename OpTypes<D>::V2;
  using Acc = typename OpTypes<D>::Acc;
  Acc acc[ND > 0 ? ND : 1];
#pragma unroll
  for (int d = 0; d < (ND > 0 ? ND : 1); ++d) acc_zero(acc[d]);
  // chunks of two doubles; an odd total (kp == 1, odd n) ends in a zero pad element
  const int64_t n2 = (a.n * kp + 1) >> 1;
  int64_t i = gtid;
  if constexpr (VecChunks<OP>::value == 2) {
    for (; i + stride < n2; i += 2 * stride) {
      V2 va[D::NL], vb[D::NL];
      D::load(a, i, va);
      D::load(a, i + stride, vb);
      D::comp(a, i, va, s, acc);
      D::comp(a, i + stride, vb, s, acc);
    }
  } else {
    for (; i + stride < n2; i += stride) {  // the last chunk is the tail's
      V2 va[D::NL];
      D::load(a, i, va);
      D::comp(a, i, va, s, acc);
    }
  }
  if (i < n2) {
    V2 va[D::NL];
    D::load(a, i, va);
    D::comp(a, i, va, s, acc);
  }
  if constexpr (ND > 0) {
    double2 accd[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) accd[d] = to_d2(acc[d]);
    reduce_and_finalize<D>(a, accd);
  }
}

// ------------------------------------------------------------------ SpMM with a dot epilogue
//
// y = A x (FP64) followed by the dots of the next step of the listing, taken while y is still in
// registers, then the grid reduction and that step's scalar rule (FIN) exactly as the separate
// dot kernel would run them.  Saves that kernel's launch, ramp and tail and its re-read of y.
// The row sums are those of the SpMM kernels (spmm_group_kernel with two columns per lane for
// kp >= 4, spmm_row_kernel with staged tiles for kp <= 2): one FMA per nonzero and column, in
// CSR order.  Thread -> column mapping: lane l of a row holds columns 2l, 2l+1 (kp >= 4), the
// one or two columns of its row (kp <= 2), which is the mapping reduce_and_finalize assumes.

// Epilogue policies: ND dots, the FIN rule and loop control of the dot kernel they replace, and
// the accumulation for one row's two columns (acc2, element o of the double2 view) or, at
// kp = 1, one column (acc1, element o).
struct EpiDelta {  // delta = (v, r^0): OP_DELTA
  static constexpr int ND = 1, FIN = FIN_DELTA, CTL = CTL_NONE;
  __device__ static void acc2(const KArgs &a, int64_t o, double2 y, double2 (&acc)[ND]) {
    dot_acc(acc[0], y, ld2(a.v[V_R0], o));
  }
  __device__ static void acc1(const KArgs &a, int64_t o, double y, double2 (&acc)[ND]) {
    acc[0].x = fma(y, a.v[V_R0][o], acc[0].x);
  }
};
struct EpiG1 {  // phi = (t,s), psi = (t,t), theta = (s,s): OP_G1
  static constexpr int ND = 3, FIN = FIN_G1, CTL = CTL_NONE;
  __device__ static void acc2(const KArgs &a, int64_t o, double2 t, double2 (&acc)[ND]) {
    const double2 s = ld2(a.v[V_S], o);
    dot_acc(acc[0], t, s);
    dot_acc(acc[1], t, t);
    dot_acc(acc[2], s, s);
  }
  __device__ static void acc1(const KArgs &a, int64_t o, double t, double2 (&acc)[ND]) {
    const double s = a.v[V_S][o];
    acc[0].x = fma(t, s, acc[0].x);
    acc[1].x = fma(t, t, acc[1].x);
    acc[2].x = fma(s, s, acc[2].x);
  }
};

struct EpiG1PP {  // phi = (t,s), psi = (t,t), theta from the s update: OP_G1_PP
  static constexpr int ND = 2, FIN = FIN_G1_TH, CTL = CTL_NONE;
  __device__ static void acc2(const KArgs &a, int64_t o, double2 t, double2 (&acc)[ND]) {
    dot_acc(acc[0], t, ld2(a.v[V_S], o));
    dot_acc(acc[1], t, t);
  }
  __device__ static void acc1(const KArgs &a, int64_t o, double t, double2 (&acc)[ND]) {
    acc[0].x = fma(t, a.v[V_S][o], acc[0].x);
    acc[1].x = fma(t, t, acc[1].x);
  }
};

template <int KP, class E>
__global__ void __launch_bounds__(kSpmmThreads) spmm_dot_kernel(const SpmmArgs sp, const KArgs a) {
  double2 acc[E::ND];
#pragma unroll
  for (int d = 0; d < E::ND; ++d) acc[d] = make_double2(0.0, 0.0);
  const int32_t *__restrict__ rp = sp.rowptr;
  const int32_t *__restrict__ ci = sp.colidx;
  const double *__restrict__ va = static_cast<const double *>(sp.vals);
  if constexpr (KP >= 4) {
    constexpr int L = KP / 2;  // lanes per row, two columns each
    constexpr int RPP = kSpmmThreads / L;
    const int g = threadIdx.x / L, cl = threadIdx.x % L;
    const double2 *__restrict__ x2 = static_cast<const double2 *>(sp.x);
    double2 *__restrict__ y2 = static_cast<double2 *>(sp.y);
    const int64_t stride = (int64_t)gridDim.x * RPP;
    for (int64_t r = (int64_t)blockIdx.x * RPP + g; r < sp.n; r += stride) {
      const int e0 = __ldg(rp + r), e1 = __ldg(rp + r + 1);
      double2 y = make_double2(0.0, 0.0);
      int e = e0;
      for (; e + 1 < e1; e += 2) {
        const int j0 = __ldg(ci + e), j1 = __ldg(ci + e + 1);
        const double a0 = __ldg(va + e), a1 = __ldg(va + e + 1);
        const double2 u0 = __ldg(x2 + (int64_t)j0 * L + cl), u1 = __ldg(x2 + (int64_t)j1 * L + cl);
        y.x = fma(a0, u0.x, y.x);
        y.y = fma(a0, u0.y, y.y);
        y.x = fma(a1, u1.x, y.x);
        y.y = fma(a1, u1.y, y.y);
      }
      if (e < e1) {
        const int j0 = __ldg(ci + e);
        const double a0 = __ldg(va + e);
        const double2 u0 = __ldg(x2 + (int64_t)j0 * L + cl);
        y.x = fma(a0, u0.x, y.x);
        y.y = fma(a0, u0.y, y.y);
      }
      const int64_t o = r * L + cl;
      y2[o] = y;
      E::acc2(a, o, y, acc);
    }
  } else {
    // one lane per row, each 256-row tile's CSR entries staged in shared memory
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int cap = sp.stage_cap;
    double *s_val = reinterpret_cast<double *>(smem_raw);
    int32_t *s_col = reinterpret_cast<int32_t *>(s_val + cap);
    const int64_t ntiles = (sp.n + kSpmmTileRows - 1) / kSpmmTileRows;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const int64_t r0 = t * kSpmmTileRows;
      const int64_t r1 = (r0 + kSpmmTileRows < sp.n) ? r0 + kSpmmTileRows : sp.n;
      const int te0 = __ldg(rp + r0), te1 = __ldg(rp + r1);
      const bool staged = (te1 - te0) <= cap;
      if (staged) stage_entries<double>(ci, va, te0, te1, s_val, s_col);
      __syncthreads();
      const int64_t r = r0 + threadIdx.x;
      if (r < r1) {
        const int e0 = __ldg(rp + r), e1 = __ldg(rp + r + 1);
        if constexpr (KP == 1) {
          const double *__restrict__ xs = static_cast<const double *>(sp.x);
          double y = 0.0;
          if (staged)
            y = staged_row<double>(s_val, s_col, xs, e0 - te0, e1 - te0);
          else
            for (int e = e0; e < e1; ++e) y = fma(__ldg(va + e), __ldg(xs + __ldg(ci + e)), y);
          static_cast<double *>(sp.y)[r] = y;
          E::acc1(a, r, y, acc);
        } else {
          const double2 *__restrict__ x2 = static_cast<const double2 *>(sp.x);
          double2 y = make_double2(0.0, 0.0);
          if (staged) {
            y = staged_row2<double, double2>(s_val, s_col, x2, e0 - te0, e1 - te0);
          } else {
            for (int e = e0; e < e1; ++e) {
              const double av = __ldg(va + e);
              const double2 u = __ldg(x2 + __ldg(ci + e));
              y.x = fma(av, u.x, y.x);
              y.y = fma(av, u.y, y.y);
            }
          }
          static_cast<double2 *>(sp.y)[r] = y;
          E::acc2(a, r, y, acc);
        }
      }
      __syncthreads();
    }
  }
  reduce_and_finalize<E, kSpmmThreads>(a, acc);
}

// kp <= 2 over short rows: the warp-tile product (warp_tile_rows, the kernel spmm_warp_kernel
// runs) with the same epilogue dots, then the same reduction.
template <int KP, class E>
__global__ void __launch_bounds__(kSpmmThreads) spmm_dot_warp_kernel(const SpmmArgs sp, const KArgs a) {
  static_assert(KP == 1 || KP == 2, "warp tiles: kp <= 2");
  __shared__ double s_val[kSpmmThreads / 32][kWarpCap];
  __shared__ int32_t s_col[kSpmmThreads / 32][kWarpCap];
  double2 acc[E::ND];
#pragma unroll
  for (int d = 0; d < E::ND; ++d) acc[d] = make_double2(0.0, 0.0);
  const int w = threadIdx.x >> 5;
  warp_tile_rows<double, KP>(sp, s_val[w], s_col[w], [&](int64_t row, auto y) {
    if constexpr (KP == 1) {
      static_cast<double *>(sp.y)[row] = y;
      E::acc1(a, row, y, acc);
    } else {
      static_cast<double2 *>(sp.y)[row] = y;
      E::acc2(a, row, y, acc);
    }
  });
  reduce_and_finalize<E, kSpmmThreads>(a, acc);
}

// ------------------------------------------------------------------ pack / unpack / reset

// Columns [0, ncols) of a caller block with leading dimension ld (B, X0 already offset to the
// first column of this group) into the workspace layout (ld = kp, zero padding columns).
__global__ void pack_kernel(const double *__restrict__ B, const double *__restrict__ X0, int ld, int ncols,
                            KArgs a) {
  const int kp = a.kp;
  const int64_t m = a.n * kp;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
    const int64_t i = e / kp;
    const int c = (int)(e - i * kp);
    const bool real = c < ncols;
    a.v[V_B][e] = real ? B[i * ld + c] : 0.0;
    a.v[V_X][e] = (real && X0) ? X0[i * ld + c] : 0.0;
  }
  // zero pad element of odd-length blocks (kp == 1): every role
  if ((m & 1) && blockIdx.x == 0 && threadIdx.x < V_NVEC) a.v[threadIdx.x][m] = 0.0;
}

__global__ void unpack_kernel(double *__restrict__ X, int ld, int ncols, KArgs a, int role, int use_xzero) {
  const int kp = a.kp;
  const int64_t m = a.n * ncols;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const double *src = a.v[role];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
    const int64_t i = e / ncols;
    const int c = (int)(e - i * ncols);
    X[i * ld + c] = (use_xzero && FL(F_XZERO, c)) ? 0.0 : src[i * kp + c];
  }
}

__global__ void reset_kernel(KArgs a, int64_t hist_len) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double *h = a.ctl->hist;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < hist_len; e += stride) h[e] = __longlong_as_double(0x7ff8000000000000LL);
  if (blockIdx.x == 0) {
    for (int t = threadIdx.x; t < S_NSLOT * kMaxKp; t += blockDim.x) a.sc[t] = 0.0;
    for (int t = threadIdx.x; t < F_NFLAG * kMaxKp; t += blockDim.x) a.fl[t] = 0;
  }
}

template <int OP>
cudaError_t launch_one(const KArgs &a, int grid, cudaStream_t s) {
  vec_kernel<OP><<<grid, kVecThreads, 0, s>>>(a);
  return cudaGetLastError();
}

template <int OP>
int occ_one() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, vec_kernel<OP>, kVecThreads, 0) != cudaSuccess) return 1;
  return nb > 0 ? nb : 1;
}

struct OpInfo {
  const char *name;
  int reads, writes;
  cudaError_t (*launch)(const KArgs &, int, cudaStream_t);
  int (*occ)();
  int nd;
};

#define OPI(op, name, r, w) {name, r, w, &launch_one<op>, &occ_one<op>, OpDef<op>::ND}
const OpInfo kOps[OP_COUNT] = {
    OPI(OP_SETUP_C, "setup_classical", 2, 2),
    OPI(OP_SETUP_R, "setup_reordered", 2, 3),
    OPI(OP_SETUP_P, "setup_pipelined", 2, 5),
    OPI(OP_DOT_RW0, "dot_r0_w0", 2, 0),
    OPI(OP_DELTA, "dot_delta", 2, 0),
    OPI(OP_UPD_S, "upd_s", 2, 1),
    OPI(OP_G1, "merged_phi_psi_theta", 2, 0),
    OPI(OP_G3, "merged_x_r_rho", 5, 2),
    OPI(OP_UPD_P, "upd_p", 3, 1),
    OPI(OP_DOT_TS, "dot_phi", 2, 0),
    OPI(OP_DOT_PSI, "dot_psi", 1, 0),
    OPI(OP_UPD_X_C, "upd_x", 3, 1),
    OPI(OP_UPD_R_C, "upd_r", 2, 1),
    OPI(OP_DOT_RR, "dot_rr", 1, 0),
    OPI(OP_DOT_RHO, "dot_rho", 2, 0),
    OPI(OP_COPY_SV, "precond_copy_s", 1, 1),
    OPI(OP_UPD_TH, "upd_that", 2, 1),
    OPI(OP_RG4, "merged_rtilde_4dots", 4, 1),
    OPI(OP_COPY_QT, "precond_copy_q", 1, 1),
    OPI(OP_UPD_R_R, "upd_r", 2, 1),
    OPI(OP_RFIN, "merged_x_z_vhat", 5, 3),
    OPI(OP_UPD_RT, "upd_rtilde", 2, 1),
    OPI(OP_DOT_T_RT, "dot_theta", 2, 0),
    OPI(OP_DOT_T_T, "dot_phi", 1, 0),
    OPI(OP_DOT_T_R0, "dot_psi", 2, 0),
    OPI(OP_DOT_RT_RT, "dot_eta", 1, 0),
    OPI(OP_UPD_X_R, "upd_x", 3, 1),
    OPI(OP_UPD_Z_R, "upd_z", 2, 1),
    OPI(OP_UPD_VH, "upd_vhat", 3, 1),
    OPI(OP_PG1, "merged_pszqy_3dots", 7, 5),
    OPI(OP_PG2, "merged_x_r", 4, 2),
    OPI(OP_PG3, "merged_w_4dots", 7, 1),
    OPI(OP_PU_P, "upd_p", 3, 1),
    OPI(OP_PU_S, "upd_s", 3, 1),
    OPI(OP_PU_Z, "upd_z", 3, 1),
    OPI(OP_PU_Q, "upd_q", 2, 1),
    OPI(OP_PU_Y, "upd_y", 2, 1),
    OPI(OP_DOT_QY, "dot_theta", 2, 0),
    OPI(OP_DOT_YY, "dot_phi", 1, 0),
    OPI(OP_DOT_QQ, "dot_pi", 1, 0),
    OPI(OP_PU_X, "upd_x", 3, 1),
    OPI(OP_PU_R, "upd_r", 2, 1),
    OPI(OP_PU_TMP, "upd_w_part1", 2, 1),
    OPI(OP_PU_W, "upd_w_part2", 2, 1),
    OPI(OP_DOT_R0R, "dot_rho", 2, 0),
    OPI(OP_DOT_R0Z, "dot_psi", 2, 0),
    OPI(OP_DOT_R0W, "dot_sigma", 2, 0),
    OPI(OP_DOT_R0S, "dot_delta", 2, 0),
    OPI(OP_TRUE_RES, "dot_true_residual", 1, 0),
    OPI(OP32_SETUP, "fp32_setup", 1, 4),
    OPI(OP32_DELTA, "fp32_dot_delta", 2, 0),
    OPI(OP32_UPD_S, "fp32_upd_s", 2, 1),
    OPI(OP32_G1, "fp32_merged_phi_psi_theta", 2, 0),
    OPI(OP32_G3, "fp32_merged_x_r_rho", 5, 2),
    OPI(OP32_UPD_P, "fp32_upd_p", 3, 1),
    OPI(OP_IR_SETUP, "ir_dot_b", 1, 0),
    OPI(OP_IR_RESID, "ir_resid_to_fp32", 1, 1),
    OPI(OP_IR_UPDATE, "ir_update_x", 2, 1),
    OPI(OP_PREC_P_Q, "precond_p", 1, 1),
    OPI(OP_PREC_S_Y, "precond_s", 1, 1),
    OPI(OP_PREC_R_RH, "precond_r", 1, 1),
    OPI(OP_PREC_W_WH, "precond_w", 1, 1),
    OPI(OP_PREC_Z_ZH, "precond_z", 1, 1),
    OPI(OP_PREC_R_Z, "precond_r_z", 1, 2),
    OPI(OP_PREC_V_S, "precond_copy_s", 1, 1),
    OPI(OP_PREC_T_Q, "precond_copy_q", 1, 1),
    OPI(OP5_RRHO, "merged_r_rho", 3, 1),
    OPI(OP5_UPD_X, "upd_x", 3, 1),
    OPI(OP7_SETUP, "setup_ppipe", 2, 7),
    OPI(OP7_L1, "merged_phat_shat_qhat", 5, 3),
    OPI(OP7_L2, "merged_szqy_3dots", 6, 4),
    OPI(OP7_L4, "merged_x_rhat", 5, 2),
    OPI(OP7_L5, "merged_r_w_4dots", 7, 2),
    OPI(OP7_PU_PH, "upd_phat", 3, 1),
    OPI(OP7_PU_SH, "upd_shat", 3, 1),
    OPI(OP7_PU_QH, "upd_qhat", 2, 1),
    OPI(OP7_X, "upd_x", 3, 1),
    OPI(OP7_TMPH, "upd_rhat_part1", 2, 1),
    OPI(OP7_RH, "upd_rhat_part2", 2, 1),
    OPI(OP3_SETUP, "setup_improved", 2, 4),
    OPI(OP3_SIG0, "dot_sigma0", 2, 0),
    OPI(OP3_L1, "merged_z_v_s", 5, 3),
    OPI(OP3_L2, "merged_t_7dots", 5, 1),
    OPI(OP3_L3, "merged_r_x", 4, 2),
    OPI(OP3_Z, "upd_z", 3, 1),
    OPI(OP3_V, "upd_v", 3, 1),
    OPI(OP3_S, "upd_s", 2, 1),
    OPI(OP3_T, "upd_t", 2, 1),
    OPI(OP3_D_R0S, "dot_phi", 2, 0),
    OPI(OP3_D_R0Q, "dot_pi", 2, 0),
    OPI(OP3_D_F0S, "dot_gamma", 2, 0),
    OPI(OP3_D_F0T, "dot_eta", 2, 0),
    OPI(OP3_D_ST, "dot_theta", 2, 0),
    OPI(OP3_D_TT, "dot_kappa", 1, 0),
    OPI(OP3_D_SS, "dot_nu", 1, 0),
    OPI(OP3_X, "upd_x", 3, 1),
    OPI(OP_UPD_S_TH, "upd_s_theta", 2, 1),
    OPI(OP_G1_PP, "merged_phi_psi", 2, 0),
};
#undef OPI

}  // namespace

const char *op_name(int op) { return (op >= 0 && op < OP_COUNT) ? kOps[op].name : "?"; }
void op_traffic(int op, int *reads, int *writes) {
  *reads = (op >= 0 && op < OP_COUNT) ? kOps[op].reads : 0;
  *writes = (op >= 0 && op < OP_COUNT) ? kOps[op].writes : 0;
}
int op_has_dots(int op) { return (op >= 0 && op < OP_COUNT) ? kOps[op].nd > 0 : 0; }

cudaError_t launch_vec(int op, const KArgs &a, int grid, cudaStream_t s) {
  if (op < 0 || op >= OP_COUNT) return cudaErrorInvalidValue;
  return kOps[op].launch(a, grid, s);
}
int vec_blocks_per_sm(int op) { return (op >= 0 && op < OP_COUNT) ? kOps[op].occ() : 1; }

namespace {
// Dynamic shared memory of the fused SpMM: the staged CSR entries of a tile (kp <= 2).  The
// reduction's static buffers come on top, so above 32 KB the kernel's limit is raised first.
template <int KP, class E>
cudaError_t dot_smem(int stage_cap, size_t *smem) {
  *smem = KP <= 2 ? (size_t)stage_cap * (sizeof(double) + sizeof(int32_t)) : 0;
  static size_t opened = 0;
  if (*smem > 32 * 1024 && *smem > opened) {
    cudaError_t e = cudaFuncSetAttribute(spmm_dot_kernel<KP, E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)*smem);
    if (e != cudaSuccess) return e;
    opened = *smem;
  }
  return cudaSuccess;
}
template <int KP, class E>
cudaError_t launch_dot_kp(const SpmmArgs &s, const KArgs &a, int grid, cudaStream_t st) {
  if constexpr (KP <= 2) {
    if (s.warp_rows) {
      spmm_dot_warp_kernel<KP, E><<<grid, kSpmmThreads, 0, st>>>(s, a);
      return cudaGetLastError();
    }
  }
  size_t smem = 0;
  cudaError_t e = dot_smem<KP, E>(s.stage_cap, &smem);
  if (e != cudaSuccess) return e;
  spmm_dot_kernel<KP, E><<<grid, kSpmmThreads, smem, st>>>(s, a);
  return cudaGetLastError();
}
template <int KP, class E>
int occ_dot_kp(int stage_cap, int warp_rows) {
  size_t smem = 0;
  int nb = 0;
  if constexpr (KP <= 2) {
    if (warp_rows) {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, spmm_dot_warp_kernel<KP, E>, kSpmmThreads, 0) !=
          cudaSuccess)
        return 1;
      return nb > 0 ? nb : 1;
    }
  }
  if (dot_smem<KP, E>(stage_cap, &smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, spmm_dot_kernel<KP, E>, kSpmmThreads, smem) != cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}
template <class E>
cudaError_t launch_dot_e(int kp, const SpmmArgs &s, const KArgs &a, int grid, cudaStream_t st) {
  switch (kp) {
    case 1: return launch_dot_kp<1, E>(s, a, grid, st);
    case 2: return launch_dot_kp<2, E>(s, a, grid, st);
    case 4: return launch_dot_kp<4, E>(s, a, grid, st);
    case 8: return launch_dot_kp<8, E>(s, a, grid, st);
    case 16: return launch_dot_kp<16, E>(s, a, grid, st);
    case 32: return launch_dot_kp<32, E>(s, a, grid, st);
    case 64: return launch_dot_kp<64, E>(s, a, grid, st);
    default: return cudaErrorInvalidValue;
  }
}
template <class E>
int occ_dot_e(int kp, int stage_cap, int warp_rows) {
  switch (kp) {
    case 1: return occ_dot_kp<1, E>(stage_cap, warp_rows);
    case 2: return occ_dot_kp<2, E>(stage_cap, warp_rows);
    case 4: return occ_dot_kp<4, E>(stage_cap, warp_rows);
    case 8: return occ_dot_kp<8, E>(stage_cap, warp_rows);
    case 16: return occ_dot_kp<16, E>(stage_cap, warp_rows);
    case 32: return occ_dot_kp<32, E>(stage_cap, warp_rows);
    case 64: return occ_dot_kp<64, E>(stage_cap, warp_rows);
    default: return 1;
  }
}
}  // namespace

cudaError_t launch_spmm_dot(int kp, int epi, const SpmmArgs &s, const KArgs &a, int grid, cudaStream_t st) {
  if (epi == EPI_DELTA) return launch_dot_e<EpiDelta>(kp, s, a, grid, st);
  if (epi == EPI_G1) return launch_dot_e<EpiG1>(kp, s, a, grid, st);
  if (epi == EPI_G1_PP) return launch_dot_e<EpiG1PP>(kp, s, a, grid, st);
  return cudaErrorInvalidValue;
}
int spmm_dot_blocks_per_sm(int kp, int epi, int stage_cap, int warp_rows) {
  if (epi == EPI_DELTA) return occ_dot_e<EpiDelta>(kp, stage_cap, warp_rows);
  if (epi == EPI_G1) return occ_dot_e<EpiG1>(kp, stage_cap, warp_rows);
  if (epi == EPI_G1_PP) return occ_dot_e<EpiG1PP>(kp, stage_cap, warp_rows);
  return 1;
}
const char *spmm_dot_name(int epi) {
  return epi == EPI_DELTA ? "spmm_delta" : epi == EPI_G1 ? "spmm_g1" : epi == EPI_G1_PP ? "spmm_phi_psi" : "?";
}

cudaError_t launch_pack(const double *B, const double *X0, int ld, int ncols, const KArgs &a, cudaStream_t s) {
  pack_kernel<<<1024, 256, 0, s>>>(B, X0, ld, ncols, a);
  return cudaGetLastError();
}
cudaError_t launch_unpack_role(double *X, int ld, int ncols, const KArgs &a, int role, int use_xzero,
                               cudaStream_t s) {
  unpack_kernel<<<1024, 256, 0, s>>>(X, ld, ncols, a, role, use_xzero);
  return cudaGetLastError();
}
namespace {
__global__ void pack_io_kernel(const BatchIO *io, int k, KArgs a) {
  const double *B = io->B, *X0 = io->X0;
  const int kp = a.kp;
  const int64_t m = a.n * kp;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
    const int64_t i = e / kp;
    const int c = (int)(e - i * kp);
    const bool real = c < k;
    a.v[V_B][e] = real ? B[i * k + c] : 0.0;
    a.v[V_X][e] = (real && X0) ? X0[i * k + c] : 0.0;
  }
  if ((m & 1) && blockIdx.x == 0 && threadIdx.x < V_NVEC) a.v[threadIdx.x][m] = 0.0;
}

__global__ void unpack_io_kernel(const BatchIO *io, int k, KArgs a) {
  double *X = io->X;
  const int kp = a.kp;
  const int64_t m = a.n * k;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
    const int64_t i = e / k;
    const int c = (int)(e - i * k);
    X[e] = FL(F_XZERO, c) ? 0.0 : a.v[V_X][i * kp + c];
  }
}

int small_grid(int64_t work) {  // blocks of 256 threads for a one-off pass over `work` elements
  int64_t g = (work + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 1024 ? 1024 : g));
}

__global__ void to_float_kernel(const double *__restrict__ src, float *__restrict__ dst, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) dst[e] = (float)src[e];
}
}  // namespace

cudaError_t launch_pack_io(const BatchIO *io, int k, const KArgs &a, cudaStream_t s) {
  pack_io_kernel<<<small_grid(a.n * a.kp), 256, 0, s>>>(io, k, a);
  return cudaGetLastError();
}
cudaError_t launch_unpack_io(const BatchIO *io, int k, const KArgs &a, cudaStream_t s) {
  unpack_io_kernel<<<small_grid(a.n * k), 256, 0, s>>>(io, k, a);
  return cudaGetLastError();
}

namespace {
__global__ void invdiag_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                               const double *__restrict__ va, double *__restrict__ inv, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double d = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e)
      if (ci[e] == i) d += va[e];
    inv[i] = d == 0.0 ? 1.0 : 1.0 / d;
  }
}
}  // namespace

cudaError_t launch_invdiag(const int32_t *rowptr, const int32_t *colidx, const double *vals, double *invdiag,
                           int64_t n, cudaStream_t s) {
  invdiag_kernel<<<small_grid(n), 256, 0, s>>>(rowptr, colidx, vals, invdiag, n);
  return cudaGetLastError();
}

cudaError_t launch_to_float(const double *src, float *dst, int64_t n, cudaStream_t s) {
  if (n > 0) to_float_kernel<<<1024, 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_reset(const KArgs &a, int64_t hist_len, cudaStream_t s) {
  reset_kernel<<<64, 256, 0, s>>>(a, hist_len);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ column compaction
//
// A group's loop runs until its slowest column stops, and a stopped column still costs its FP64
// FMAs in every kernel.  When at most half of a layout's columns are still active, the loop stops
// (fin_ctl) and the group continues in a layout of half the width: the active columns keep their
// order, the live vectors of the classical and preconditioned forms at the top of an iteration
// (x, r, r^0, p) are gathered into it, and everything a column reports (x, iterations, status,
// the scalars the final kernels read) leaves for final arrays indexed by the solve's column.

namespace {
__global__ void compact_plan_kernel(KArgs a, KArgs dst, int boundary, int last, cudaGraphConditionalHandle next,
                                    double *fin_sc, int *fin_fl, int *cmap_out, int *act) {
  __shared__ int s_act[kMaxKp];
  __shared__ int s_m, s_mode;
  __shared__ double s_sc[S_NSLOT][kMaxKp];
  __shared__ int s_fl[F_NFLAG][kMaxKp];
  Ctl *ctl = a.ctl;
  const int kps = a.kp, t = threadIdx.x;
  if (t == 0) {
    int mode = 0;
    if (ctl->level == boundary - 1) mode = (!last && ctl->compact_req) ? 1 : 2;
    int m = 0;
    if (mode == 1)
      for (int c = 0; c < kps; ++c)
        if (FL(F_ACT, c)) s_act[m++] = c;
    s_m = m;
    s_mode = mode;
    ctl->mode = mode;
    ctl->compact_req = 0;
    if (mode == 1) ctl->level = boundary;
    if (mode == 2) ctl->level = -1;
    if (!last) cudaGraphSetConditional(next, mode == 1 ? 1u : 0u);
  }
  __syncthreads();
  const int mode = s_mode, m = s_m;
  if (mode == 0) return;
  // the state of the columns that leave (all of them for the final values, else the stopped ones)
  if (t < kps) {
    const int orig = a.cmap ? a.cmap[t] : t;
    const bool leaving = mode == 2 || !FL(F_ACT, t);
    if (orig >= 0 && leaving) {
      for (int q = 0; q < S_NSLOT; ++q) fin_sc[q * kMaxKp + orig] = SC(q, t);
      for (int f = 0; f < F_NFLAG; ++f) fin_fl[f * kMaxKp + orig] = FL(f, t);
    }
    for (int q = 0; q < S_NSLOT; ++q) s_sc[q][t] = SC(q, t);
    for (int f = 0; f < F_NFLAG; ++f) s_fl[f][t] = FL(f, t);
  }
  __syncthreads();
  if (mode != 1) return;
  // the kept columns, in order, at the front of the narrower layout; zero padding after them
  const int kpd = dst.kp;
  if (t < kpd) {
    const int src = t < m ? s_act[t] : -1;
    for (int q = 0; q < S_NSLOT; ++q) a.sc[q * kMaxKp + t] = src >= 0 ? s_sc[q][src] : 0.0;
    for (int f = 0; f < F_NFLAG; ++f) a.fl[f * kMaxKp + t] = src >= 0 ? s_fl[f][src] : 0;
    cmap_out[t] = src >= 0 ? (a.cmap ? a.cmap[src] : src) : -1;
    act[t] = src;
  }
}

// live_mask: the roles an iteration reads before writing (gathered); loop_mask: every role the
// loop uses (its padding element is zeroed at an odd length); bit r for role r.
__global__ void compact_move_kernel(KArgs a, KArgs dst, const int *act, double *xf, unsigned live_mask,
                                    unsigned loop_mask) {
  __shared__ int s_orig[kMaxKp], s_keep[kMaxKp], s_act[kMaxKp];
  const int mode = a.ctl->mode;
  if (mode == 0) return;
  const int kps = a.kp, kpd = dst.kp, kp0 = a.kp_out;
  for (int c = threadIdx.x; c < kMaxKp; c += blockDim.x) {
    s_orig[c] = c < kps ? (a.cmap ? a.cmap[c] : c) : -1;
    s_keep[c] = 0;
  }
  __syncthreads();
  if (mode == 1)
    for (int c = threadIdx.x; c < kpd; c += blockDim.x) {
      s_act[c] = act[c];
      if (act[c] >= 0) s_keep[act[c]] = 1;
    }
  __syncthreads();
  const int64_t n = a.n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int shs = __ffs(kps) - 1, shd = __ffs(kpd) - 1;  // kp is a power of two
  // x of the columns that leave, at their place in the final block
  for (int64_t e = t0; e < n * kps; e += stride) {
    const int c = (int)(e & (kps - 1));
    const int orig = s_orig[c];
    if (orig >= 0 && !s_keep[c]) xf[(e >> shs) * kp0 + orig] = a.v[V_X][e];
  }
  if (mode != 1) return;
  for (int64_t e = t0; e < n * kpd; e += stride) {
    const int64_t i = e >> shd;
    const int src = s_act[e & (kpd - 1)];
    for (int r = 0; r < V_NVEC; ++r)
      if ((live_mask >> r) & 1u) dst.v[r][e] = src >= 0 ? a.v[r][(i << shs) + src] : 0.0;
  }
  if (((n * kpd) & 1) && t0 == 0)
    for (int r = 0; r < V_NVEC; ++r)
      if ((loop_mask >> r) & 1u) dst.v[r][n * kpd] = 0.0;
}

// In-place compaction of one role (forms whose loops leave no free slot for a second copy):
// gather the kept columns into a scratch block, then copy it back in the narrower layout (two
// launches: the gather must read the whole source before the copy overwrites it).
__global__ void compact_gather_kernel(KArgs a, int kpd, const int *act, int role, double *scratch) {
  if (a.ctl->mode != 1) return;
  __shared__ int s_act[kMaxKp];
  for (int c = threadIdx.x; c < kpd; c += blockDim.x) s_act[c] = act[c];
  __syncthreads();
  const int64_t n = a.n;
  const int shs = __ffs(a.kp) - 1, shd = __ffs(kpd) - 1;
  const double *src = a.v[role];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * kpd;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int c = s_act[e & (kpd - 1)];
    scratch[e] = c >= 0 ? src[((e >> shd) << shs) + c] : 0.0;
  }
}
__global__ void compact_copy_kernel(KArgs dst, int role, const double *scratch) {
  if (dst.ctl->mode != 1) return;
  const int64_t m = dst.n * dst.kp;
  double *d = dst.v[role];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
    d[e] = scratch[e];
  if ((m & 1) && blockIdx.x == 0 && threadIdx.x == 0) d[m] = 0.0;  // padding element of an odd length
}
}  // namespace

cudaError_t launch_compact_inplace(const KArgs &src, const KArgs &dst, const int *act, int role, double *scratch,
                                   int grid, cudaStream_t s) {
  compact_gather_kernel<<<grid, 256, 0, s>>>(src, dst.kp, act, role, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  compact_copy_kernel<<<grid, 256, 0, s>>>(dst, role, scratch);
  return cudaGetLastError();
}

cudaError_t launch_compact(const KArgs &src, const KArgs &dst, int boundary, int last,
                           cudaGraphConditionalHandle next, double *fin_sc, int *fin_fl, int *cmap_out,
                           int *act, double *xf, unsigned live_mask, unsigned loop_mask, int grid,
                           cudaStream_t s) {
  compact_plan_kernel<<<1, kMaxKp, 0, s>>>(src, dst, boundary, last, next, fin_sc, fin_fl, cmap_out, act);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  compact_move_kernel<<<grid, 256, 0, s>>>(src, dst, act, xf, live_mask, loop_mask);
  return cudaGetLastError();
}

}  // namespace bicgk
