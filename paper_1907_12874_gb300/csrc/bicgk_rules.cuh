// Per-column scalar recurrences of the listings, shared by the streaming kernels, the SpMM
// epilogues and the persistent batched solver: executed for column c by one thread after a dot
// group's grid-wide sum is final (the "finalize" rules), plus the loop control of the last
// reducing kernel of an iteration.
//
// The rules follow the oracle's (no FMA contraction: __dmul_rn / __dadd_rn / __ddiv_rn /
// __dsqrt_rn, evaluated as written):
//   R1 stop: estimate < eps_c^2, eps_c = tol*||b_c||;  R2 b_c = 0 -> x_c = 0;
//   R3 a column stops on its own; x_{j+1} is formed once omega_j is finite;
//   R5 zero denominator of omega -> omega = 0, other exact-zero divisors ->
//      BREAKDOWN, non-finite scalars -> NONFINITE;
//   R6 merged estimates (theta - omega*phi etc.) feed the stop test.
#pragma once

#include "bicgk_dev.cuh"

namespace bicgk {

namespace {

#define SC(slot, c) a.sc[(slot) * kMaxKp + (c)]
#define FL(f, c) a.fl[(f) * kMaxKp + (c)]

// ------------------------------------------------------------------ scalar rules

__device__ __forceinline__ bool fin1(double v) { return isfinite(v); }
__device__ __forceinline__ double hist_value(double est) {
  if (isnan(est)) return est;
  return est > 0.0 ? __dsqrt_rn(est) : 0.0;
}
// History entry of iteration row `row` for layout column c: rows of kp_out entries, indexed by the
// solve's column (the layouts of a compacted solve keep their columns' original places).
__device__ __forceinline__ double &hist_at(const KArgs &a, int64_t row, int c) {
  return a.ctl->hist[row * a.kp_out + (a.cmap ? a.cmap[c] : c)];
}
__device__ __forceinline__ void col_stop(const KArgs &a, int c, int st) {
  FL(F_ACT, c) = 0;
  FL(F_STATUS, c) = st;
}
__device__ __forceinline__ double sub_rn(double x, double y) { return __dadd_rn(x, -y); }

enum Fin : int {
  FIN_NONE = 0, FIN_SETUP, FIN_RW0, FIN_DELTA, FIN_G1, FIN_RHO, FIN_STORE_D0, FIN_STORE_D1, FIN_STORE_D2,
  FIN_PSI, FIN_RR, FIN_R4_MERGED, FIN_R4_PLAIN, FIN_PG1_MERGED, FIN_PG1_PLAIN, FIN_PG3_MERGED,
  FIN_PG3_PLAIN, FIN_TRUE, FIN_IR_SETUP, FIN_IR_RESID, FIN_STORE_D3, FIN_STORE_D4, FIN_STORE_D5, FIN_I_START,
  FIN_I7_MERGED, FIN_I7_PLAIN, FIN_G1_TH
};
enum Ctl_ : int { CTL_NONE = 0, CTL_START = 1, CTL_END_ITER = 2, CTL_OUTER = 3 };

// Algorithm 3, scalar lines of iteration j (state: phi_j, pi_j, sigma_j, sigma_{j-1}, tau_j, rho_j,
// alpha_j, omega_j): rho_{j+1}, delta_{j+1}, beta_{j+1}, tau_{j+1}, alpha_{j+1} and the vector
// coefficients, evaluated as written (no contraction).  Returns false if the column stopped.
__device__ bool i3_next(const KArgs &a, int c) {
  const double phi = SC(S_PHI, c), om = SC(S_OMEGA, c), sgp = SC(S_SIGP, c), al = SC(S_AOLD, c);
  const double pi = SC(S_PI, c), sg = SC(S_SIGMA, c), rho = SC(S_RHO, c), tau = SC(S_TAU, c);
  const double rho1 = __dadd_rn(sub_rn(phi, __dmul_rn(om, sgp)), __dmul_rn(__dmul_rn(om, al), pi));
  if (!fin1(rho1) || !fin1(sg)) { col_stop(a, c, ST_NONFINITE); return false; }
  if (rho == 0.0 || om == 0.0) { col_stop(a, c, ST_BREAKDOWN); return false; }
  const double de1 = __dmul_rn(__ddiv_rn(rho1, rho), al);
  const double be1 = __ddiv_rn(de1, om);
  const double tau1 = sub_rn(__dadd_rn(sg, __dmul_rn(be1, tau)), __dmul_rn(de1, pi));
  if (!fin1(de1) || !fin1(be1) || !fin1(tau1)) { col_stop(a, c, ST_NONFINITE); return false; }
  if (tau1 == 0.0) { col_stop(a, c, ST_BREAKDOWN); return false; }
  const double al1 = __ddiv_rn(rho1, tau1);
  if (!fin1(al1)) { col_stop(a, c, ST_NONFINITE); return false; }
  SC(S_ALPHA, c) = al1;
  SC(S_BETA, c) = be1;
  SC(S_DLT, c) = de1;
  SC(S_CZ, c) = __dmul_rn(be1, __ddiv_rn(al1, al));
  SC(S_CV, c) = __dmul_rn(al1, de1);
  SC(S_RHO, c) = rho1;
  SC(S_TAU, c) = tau1;
  SC(S_AOLD, c) = al1;
  return true;
}

// Algorithm 2 group 1 for column c: phi = (t,s), psi = (t,t), theta = (s,s); omega = phi/psi;
// stop test on (r_{j+1}, r_{j+1}) = theta - omega*phi.
__device__ void g1_rule(const KArgs &a, int c, double phi, double psi, double th) {
  Ctl *ctl = a.ctl;
  FL(F_XUPD, c) = 0;
  if (!FL(F_ACT, c)) return;
  if (!fin1(phi) || !fin1(psi) || !fin1(th)) { col_stop(a, c, ST_NONFINITE); return; }
  const double om = psi == 0.0 ? 0.0 : __ddiv_rn(phi, psi);
  if (!fin1(om)) { col_stop(a, c, ST_NONFINITE); return; }
  const int j = ctl->iter;
  SC(S_OMEGA, c) = om;
  FL(F_XUPD, c) = 1;
  FL(F_ITERS, c) = j + 1;
  const double est = sub_rn(th, __dmul_rn(om, phi));
  hist_at(a, j + 1, c) = hist_value(est);
  if (!fin1(est)) col_stop(a, c, ST_NONFINITE);
  else if (!(ctl->flags & 1) && est < SC(S_EPS2, c)) col_stop(a, c, ST_CONVERGED);
}

// Column c, executed by thread c of the last block.  s[d*kp + c] = dot d of column c.
template <int FIN>
__device__ void fin_col(const KArgs &a, int c, const double *s, int kp) {
  Ctl *ctl = a.ctl;
  const int nostop = ctl->flags & 1;
  if constexpr (FIN == FIN_SETUP) {
    // (b,b) and rho_0 = (r_0, r_0): set-up lines of Algorithms 1, 2, 4, 6 and readings R1, R2
    const double bn2 = s[0 * kp + c], rho = s[1 * kp + c];
    const double eps2 = __dmul_rn(__dmul_rn(ctl->tol, ctl->tol), bn2);
    SC(S_BN2, c) = bn2;
    SC(S_RHO, c) = rho;
    SC(S_EPS2, c) = eps2;
    SC(S_ALPHA, c) = 0.0;
    SC(S_OMEGA, c) = 0.0;
    SC(S_BETA, c) = 0.0;
    FL(F_ITERS, c) = 0;
    FL(F_XUPD, c) = 0;
    FL(F_XZERO, c) = 0;
    if (c >= ctl->k || (a.ext_act && !a.ext_act[c])) {  // padding column (or finished outer column)
      FL(F_ACT, c) = 0;
      FL(F_STATUS, c) = ST_CONVERGED;
      return;
    }
    double h0 = hist_value(rho);
    int st = ST_MAXIT, act = 1;
    if (bn2 == 0.0) {
      FL(F_XZERO, c) = 1;
      h0 = 0.0;
      st = ST_CONVERGED;
      act = 0;
    } else if (!fin1(bn2) || !fin1(rho)) {
      st = ST_NONFINITE;
      act = 0;
    } else if (!nostop && rho < eps2) {
      st = ST_CONVERGED;
      act = 0;
    }
    hist_at(a, 0, c) = h0;
    FL(F_ACT, c) = act;
    FL(F_STATUS, c) = st;
  } else if constexpr (FIN == FIN_RW0) {
    // Algorithm 4 set-up: alpha_0 = rho_0 / (r_0, w_0), beta_{-1} = 0, omega_{-1} = 0 (R7)
    if (!FL(F_ACT, c)) return;
    const double rw = s[c];
    if (!fin1(rw)) { col_stop(a, c, ST_NONFINITE); return; }
    if (rw == 0.0) { col_stop(a, c, ST_BREAKDOWN); return; }
    const double al = __ddiv_rn(SC(S_RHO, c), rw);
    if (!fin1(al)) { col_stop(a, c, ST_NONFINITE); return; }
    SC(S_ALPHA, c) = al;
  } else if constexpr (FIN == FIN_DELTA) {
    // delta_j = (v_j, r_0), alpha_j = rho_j / delta_j
    if (!FL(F_ACT, c)) return;
    const double de = s[c];
    if (!fin1(de)) { col_stop(a, c, ST_NONFINITE); return; }
    if (de == 0.0) { col_stop(a, c, ST_BREAKDOWN); return; }
    const double al = __ddiv_rn(SC(S_RHO, c), de);
    if (!fin1(al)) { col_stop(a, c, ST_NONFINITE); return; }
    SC(S_ALPHA, c) = al;
  } else if constexpr (FIN == FIN_G1) {
    g1_rule(a, c, s[0 * kp + c], s[1 * kp + c], s[2 * kp + c]);
  } else if constexpr (FIN == FIN_G1_TH) {
    // the same rule with theta = (s,s) stored by the s update (OP_UPD_S_TH)
    g1_rule(a, c, s[0 * kp + c], s[1 * kp + c], SC(S_D0, c));
  } else if constexpr (FIN == FIN_RHO) {
    // rho_{j+1} = (r_{j+1}, r_0), beta_j = (rho_{j+1}/rho_j)(alpha_j/omega_j)
    if (!FL(F_ACT, c)) return;
    const double r1 = s[c], rho = SC(S_RHO, c), om = SC(S_OMEGA, c);
    if (!fin1(r1)) { col_stop(a, c, ST_NONFINITE); return; }
    if (rho == 0.0 || om == 0.0) { col_stop(a, c, ST_BREAKDOWN); return; }
    const double be = __dmul_rn(__ddiv_rn(r1, rho), __ddiv_rn(SC(S_ALPHA, c), om));
    if (!fin1(be)) { col_stop(a, c, ST_NONFINITE); return; }
    SC(S_BETA, c) = be;
    SC(S_RHO, c) = r1;
  } else if constexpr (FIN == FIN_STORE_D0) {
    SC(S_D0, c) = s[c];
  } else if constexpr (FIN == FIN_STORE_D1) {
    SC(S_D1, c) = s[c];
  } else if constexpr (FIN == FIN_STORE_D2) {
    SC(S_D2, c) = s[c];
  } else if constexpr (FIN == FIN_PSI) {
    // Algorithm 1: psi_j = (t_j, t_j) (phi_j stored by the previous kernel), omega_j
    FL(F_XUPD, c) = 0;
    if (!FL(F_ACT, c)) return;
    const double phi = SC(S_D0, c), psi = s[c];
    if (!fin1(phi) || !fin1(psi)) { col_stop(a, c, ST_NONFINITE); return; }
    const double om = psi == 0.0 ? 0.0 : __ddiv_rn(phi, psi);
    if (!fin1(om)) { col_stop(a, c, ST_NONFINITE); return; }
    SC(S_OMEGA, c) = om;
    FL(F_XUPD, c) = 1;
  } else if constexpr (FIN == FIN_RR) {
    // Algorithm 1 conv-check line: (r_{j+1}, r_{j+1}) < eps^2
    if (!FL(F_XUPD, c)) return;
    const int j = ctl->iter;
    FL(F_ITERS, c) = j + 1;
    const double rr = s[c];
    hist_at(a, j + 1, c) = hist_value(rr);
    if (!fin1(rr)) col_stop(a, c, ST_NONFINITE);
    else if (!nostop && rr < SC(S_EPS2, c)) col_stop(a, c, ST_CONVERGED);
  } else if constexpr (FIN == FIN_R4_MERGED || FIN == FIN_R4_PLAIN) {
    // Algorithm 6: theta = (t, r~), phi = (t,t), psi = (t, r_0), eta = (r~, r~);
    // omega = theta/phi; stop on eta - omega*theta; rho_{j+1} = -omega*psi; beta_j
    FL(F_XUPD, c) = 0;
    if (!FL(F_ACT, c)) return;
    double th, phi, psi, eta;
    if constexpr (FIN == FIN_R4_MERGED) {
      th = s[0 * kp + c]; phi = s[1 * kp + c]; psi = s[2 * kp + c]; eta = s[3 * kp + c];
    } else {
      th = SC(S_D0, c); phi = SC(S_D1, c); psi = SC(S_D2, c); eta = s[c];
    }
    if (!fin1(th) || !fin1(phi) || !fin1(psi) || !fin1(eta)) { col_stop(a, c, ST_NONFINITE); return; }
    const double om = phi == 0.0 ? 0.0 : __ddiv_rn(th, phi);
    if (!fin1(om)) { col_stop(a, c, ST_NONFINITE); return; }
    const int j = ctl->iter;
    SC(S_OMEGA, c) = om;
    FL(F_XUPD, c) = 1;
    FL(F_ITERS, c) = j + 1;
    const double est = sub_rn(eta, __dmul_rn(om, th));
    hist_at(a, j + 1, c) = hist_value(est);
    if (!fin1(est)) { col_stop(a, c, ST_NONFINITE); return; }
    if (!nostop && est < SC(S_EPS2, c)) { col_stop(a, c, ST_CONVERGED); return; }
    const double r1 = __dmul_rn(-om, psi);
    const double rho = SC(S_RHO, c);
    if (rho == 0.0 || om == 0.0) { col_stop(a, c, ST_BREAKDOWN); return; }
    const double be = __dmul_rn(__ddiv_rn(r1, rho), __ddiv_rn(SC(S_ALPHA, c), om));
    if (!fin1(be) || !fin1(r1)) { col_stop(a, c, ST_NONFINITE); return; }
    SC(S_BETA, c) = be;
    SC(S_RHO, c) = r1;
  } else if constexpr (FIN == FIN_PG1_MERGED || FIN == FIN_PG1_PLAIN) {
    // Algorithm 4: theta = (q,y), phi = (y,y), pi = (q,q); omega = theta/phi;
    // stop on pi - omega*theta
    FL(F_XUPD, c) = 0;
    if (!FL(F_ACT, c)) return;
    double th, phi, pi;
    if constexpr (FIN == FIN_PG1_MERGED) {
      th = s[0 * kp + c]; phi = s[1 * kp + c]; pi = s[2 * kp + c];
    } else {
      th = SC(S_D0, c); phi = SC(S_D1, c); pi = s[c];
    }
    if (!fin1(th) || !fin1(phi) || !fin1(pi)) { col_stop(a, c, ST_NONFINITE); return; }
    const double om = phi == 0.0 ? 0.0 : __ddiv_rn(th, phi);
    if (!fin1(om)) { col_stop(a, c, ST_NONFINITE); return; }
    const int j = ctl->iter;
    SC(S_OMEGA, c) = om;
    FL(F_XUPD, c) = 1;
    FL(F_ITERS, c) = j + 1;
    const double est = sub_rn(pi, __dmul_rn(om, th));
    hist_at(a, j + 1, c) = hist_value(est);
    if (!fin1(est)) col_stop(a, c, ST_NONFINITE);
    else if (!nostop && est < SC(S_EPS2, c)) col_stop(a, c, ST_CONVERGED);
  } else if constexpr (FIN == FIN_PG3_MERGED || FIN == FIN_PG3_PLAIN) {
    // Algorithm 4: rho_{j+1} = (r_0, r_{j+1}), psi = (r_0, z), sigma = (r_0, w_{j+1}),
    // delta = (r_0, s); beta_j = (alpha/omega)(rho_{j+1}/rho_j);
    // alpha_{j+1} = rho_{j+1} / (sigma + beta*delta - beta*omega*psi)
    if (!FL(F_ACT, c)) return;
    double r1, psi, sg, de;
    if constexpr (FIN == FIN_PG3_MERGED) {
      r1 = s[0 * kp + c]; psi = s[1 * kp + c]; sg = s[2 * kp + c]; de = s[3 * kp + c];
    } else {
      r1 = SC(S_D0, c); psi = SC(S_D1, c); sg = SC(S_D2, c); de = s[c];
    }
    if (!fin1(r1) || !fin1(psi) || !fin1(sg) || !fin1(de)) { col_stop(a, c, ST_NONFINITE); return; }
    const double rho = SC(S_RHO, c), om = SC(S_OMEGA, c), al = SC(S_ALPHA, c);
    if (rho == 0.0 || om == 0.0) { col_stop(a, c, ST_BREAKDOWN); return; }
    const double be = __dmul_rn(__ddiv_rn(al, om), __ddiv_rn(r1, rho));
    const double den = sub_rn(__dadd_rn(sg, __dmul_rn(be, de)), __dmul_rn(__dmul_rn(be, om), psi));
    if (!fin1(be) || !fin1(den)) { col_stop(a, c, ST_NONFINITE); return; }
    if (den == 0.0) { col_stop(a, c, ST_BREAKDOWN); return; }
    const double al1 = __ddiv_rn(r1, den);
    if (!fin1(al1)) { col_stop(a, c, ST_NONFINITE); return; }
    SC(S_BETA, c) = be;
    SC(S_ALPHA, c) = al1;
    SC(S_RHO, c) = r1;
  } else if constexpr (FIN == FIN_TRUE) {
    // ||b - A x|| / ||b|| of the final iterate
    const double bn2 = SC(S_BN2, c);
    SC(S_TRUE, c) = bn2 == 0.0 ? 0.0 : __ddiv_rn(__dsqrt_rn(s[c]), __dsqrt_rn(bn2));
  } else if constexpr (FIN == FIN_IR_SETUP) {
    // refinement set-up: ||b||^2, eps^2 = tol^2 ||b||^2, zero and padding columns
    const double bn2 = s[c];
    SC(S_BN2, c) = bn2;
    SC(S_EPS2, c) = __dmul_rn(__dmul_rn(ctl->tol, ctl->tol), bn2);
    SC(S_TRUE, c) = 0.0;
    FL(F_ITERS, c) = 0;
    FL(F_XZERO, c) = 0;
    int act = 1, st = ST_MAXIT;
    if (c >= ctl->k) {
      act = 0;
      st = ST_CONVERGED;
    } else if (bn2 == 0.0) {
      FL(F_XZERO, c) = 1;
      act = 0;
      st = ST_CONVERGED;
    } else if (!fin1(bn2)) {
      act = 0;
      st = ST_NONFINITE;
    }
    FL(F_ACT, c) = act;
    FL(F_STATUS, c) = st;
  } else if constexpr (FIN == FIN_IR_RESID) {
    // refinement pass j: true residual r = b - A x in FP64; stop, or refine once more
    if (!FL(F_ACT, c)) return;
    const int j = ctl->iter;
    const double rr = s[c], bn2 = SC(S_BN2, c);
    hist_at(a, j, c) = hist_value(rr);
    SC(S_TRUE, c) = __ddiv_rn(__dsqrt_rn(rr), __dsqrt_rn(bn2));
    if (!fin1(rr)) col_stop(a, c, ST_NONFINITE);
    else if (rr < SC(S_EPS2, c)) col_stop(a, c, ST_CONVERGED);
    else if (j >= ctl->maxit) col_stop(a, c, ST_MAXIT);
    else FL(F_ITERS, c) = j + 1;
  } else if constexpr (FIN == FIN_STORE_D3) {
    SC(S_D3, c) = s[c];
  } else if constexpr (FIN == FIN_STORE_D4) {
    SC(S_D4, c) = s[c];
  } else if constexpr (FIN == FIN_STORE_D5) {
    SC(S_D5, c) = s[c];
  } else if constexpr (FIN == FIN_I_START) {
    // Algorithm 3 set-up: sigma_0 = (r_0, u_0), phi_0 = (r_0, r_0), sigma_{-1} = pi_0 = tau_0 = 0,
    // rho_0 = alpha_0 = omega_0 = 1; then the scalar lines of iteration 0
    if (!FL(F_ACT, c)) return;
    SC(S_PHI, c) = SC(S_RHO, c);
    SC(S_SIGMA, c) = s[c];
    SC(S_SIGP, c) = 0.0;
    SC(S_PI, c) = 0.0;
    SC(S_TAU, c) = 0.0;
    SC(S_RHO, c) = 1.0;
    SC(S_AOLD, c) = 1.0;
    SC(S_OMEGA, c) = 1.0;
    if (ctl->maxit > 0) i3_next(a, c);
  } else if constexpr (FIN == FIN_I7_MERGED || FIN == FIN_I7_PLAIN) {
    // Algorithm 3: phi = (r_0,s), pi = (r_0,q), gamma = (f_0,s), eta = (f_0,t), theta = (s,t),
    // kappa = (t,t), nu = (s,s); omega = theta/kappa; sigma = gamma - omega eta; stop on nu - omega theta
    FL(F_XUPD, c) = 0;
    if (!FL(F_ACT, c)) return;
    double ph, pi, ga, et, th, ka, nu;
    if constexpr (FIN == FIN_I7_MERGED) {
      ph = s[0 * kp + c]; pi = s[1 * kp + c]; ga = s[2 * kp + c]; et = s[3 * kp + c];
      th = s[4 * kp + c]; ka = s[5 * kp + c]; nu = s[6 * kp + c];
    } else {
      ph = SC(S_D0, c); pi = SC(S_D1, c); ga = SC(S_D2, c); et = SC(S_D3, c); th = SC(S_D4, c); ka = SC(S_D5, c);
      nu = s[c];
    }
    if (!fin1(ph) || !fin1(pi) || !fin1(ga) || !fin1(et) || !fin1(th) || !fin1(ka) || !fin1(nu)) {
      col_stop(a, c, ST_NONFINITE);
      return;
    }
    const double om = ka == 0.0 ? 0.0 : __ddiv_rn(th, ka);
    if (!fin1(om)) { col_stop(a, c, ST_NONFINITE); return; }
    const int j = ctl->iter;
    const double sg1 = sub_rn(ga, __dmul_rn(om, et));
    SC(S_OMEGA, c) = om;  // the r and x updates of this iteration use omega_{j+1}
    FL(F_XUPD, c) = 1;
    FL(F_ITERS, c) = j + 1;
    const double est = sub_rn(nu, __dmul_rn(om, th));
    hist_at(a, j + 1, c) = hist_value(est);
    if (!fin1(est)) { col_stop(a, c, ST_NONFINITE); return; }
    if (!nostop && est < SC(S_EPS2, c)) { col_stop(a, c, ST_CONVERGED); return; }
    SC(S_SIGP, c) = SC(S_SIGMA, c);
    SC(S_SIGMA, c) = sg1;
    SC(S_PHI, c) = ph;
    SC(S_PI, c) = pi;
    if (j + 1 < ctl->maxit) i3_next(a, c);  // the next iteration's scalar lines
  }
}

// Thread 0 of the last block, after every column's scalars are final.
template <int CTL>
__device__ void fin_ctl(const KArgs &a) {
  if constexpr (CTL == CTL_NONE) {
    return;
  } else {
    Ctl *ctl = a.ctl;
    int any = 0;
    for (int c = 0; c < a.kp; ++c) any |= FL(F_ACT, c);
    ctl->any_active = any;
    int go = 0;
    if constexpr (CTL == CTL_OUTER) {
      ctl->iter += 1;  // refinement passes: the host drives this loop
      return;
    } else if constexpr (CTL == CTL_START) {
      go = any && ctl->maxit > 0;
    } else {
      const int j = ctl->iter + 1;
      ctl->iter = j;
      ctl->loop_iters = j;
      go = any && j < ctl->maxit;
      if (go && a.compact) {  // at most half of the layout's columns left: stop to narrow it
        int cnt = 0;
        for (int c = 0; c < a.kp; ++c) cnt += FL(F_ACT, c) != 0;
        if (2 * cnt <= a.kp) {
          ctl->compact_req = 1;
          go = 0;
        }
      }
    }
    if (a.use_cond) cudaGraphSetConditional(a.cond, go ? 1u : 0u);
  }
}

}  // namespace

}  // namespace bicgk
