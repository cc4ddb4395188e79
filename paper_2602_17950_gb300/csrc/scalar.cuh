// Scalar steps of the PCG iteration (Section 3.1, Algorithms 1 and 2), run by one
// thread block per solve: either by a separate kernel or fused into the last
// block of the array pass that produced their sums.  Every thread of the block
// calls the function (block reductions); thread 0 updates the solve's state.
// Sums of block partials are taken in a fixed order (deterministic).
#pragma once

#include "gpsoc_internal.cuh"

namespace gpsoc {

// K slot totals (sums over the nb block partials of solve s); every thread gets them.
// The K partials of a block index are loaded together (one memory round trip per
// blockDim partials, not one per slot), and the first partial of a thread is taken as it
// is.  Double-word partials (X.part_dw) are added with the accurate double-word sum on
// the FP32 pipes and the totals rounded to FP64 once; FP64 partials are added in FP64.
template <int K>
__device__ __forceinline__ void slot_totals(const ScalarCtx& X, int s, const int (&slots)[K], int nb, double (&v)[K],
                                            double* scratch) {
  const double* base = X.part + (long long)s * NSLOT * X.pmax;
  int b = threadIdx.x;
  if (X.part_dw) {
    constexpr int K2 = (K < 2) ? 2 : K;
    DF w[K2];
#pragma unroll
    for (int k = 0; k < K2; ++k)
      w[k] = (k < K && b < nb) ? get_sum_partial(base + (long long)slots[k < K ? k : 0] * X.pmax + b) : DF{0.0f, 0.0f};
    for (b += blockDim.x; b < nb; b += blockDim.x) {
      DF t[K];
#pragma unroll
      for (int k = 0; k < K; ++k) t[k] = get_sum_partial(base + (long long)slots[k] * X.pmax + b);
#pragma unroll
      for (int k = 0; k < K; ++k) w[k] = dw_add(w[k], t[k]);
    }
    double r[K2];
    block_reduce_dw<K2>(w, r, scratch);
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = r[k];
    return;
  }
  const bool mx[K] = {};
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = (b < nb) ? __ldcg(base + (long long)slots[k] * X.pmax + b) : 0.0;
  for (b += blockDim.x; b < nb; b += blockDim.x) {
    double t[K];
#pragma unroll
    for (int k = 0; k < K; ++k) t[k] = __ldcg(base + (long long)slots[k] * X.pmax + b);
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] += t[k];
  }
  block_reduce<K>(v, scratch, mx);
}

__device__ __forceinline__ double slot_max(const ScalarCtx& X, int s, int slot, int nb, double* scratch) {
  double v[1] = {0.0};
  const double* p = X.part + ((long long)s * NSLOT + slot) * X.pmax;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) v[0] = fmax(v[0], __ldcg(p + b));
  const bool mx[1] = {true};
  block_reduce<1>(v, scratch, mx);
  return v[0];
}

__device__ __forceinline__ void deactivate(SolveState& S, int status) {
  S.active = 0;
  if (S.status == GPSOC_OK) S.status = status;
}

// E, mu (Eqs. energy, muphi), alpha_l (Eq. PreCnstAlpha), masses of the current iterate
// The solve state of a fused tail is copied to shared memory by the whole block
// (one round of loads), updated there by thread 0, and copied back by the block:
// thread 0 then never waits on a global-memory round trip per field, and the
// copy holds no registers of the kernel it is fused into.
__device__ __forceinline__ void state_load(SolveState& dst, const SolveState* src) {
  static_assert(sizeof(SolveState) % 8 == 0, "state is copied in 8-byte words");
  auto* d = reinterpret_cast<unsigned long long*>(&dst);
  const auto* q = reinterpret_cast<const unsigned long long*>(src);
  for (int i = threadIdx.x; i < (int)(sizeof(SolveState) / 8); i += blockDim.x) d[i] = q[i];
}
__device__ __forceinline__ void state_store(SolveState* dst, const SolveState& src) {
  auto* d = reinterpret_cast<unsigned long long*>(dst);
  const auto* q = reinterpret_cast<const unsigned long long*>(&src);
  for (int i = threadIdx.x; i < (int)(sizeof(SolveState) / 8); i += blockDim.x) d[i] = q[i];
}

__device__ __forceinline__ void obs_update(const ScalarCtx& X, int s, SolveState& S, const double (&kin)[3],
                                           const double (&v)[12], bool had_step, double dphi) {
  const PhysDev ph = X.phys[s];
  const double dV = X.dV;
  S.Q = dV * v[0];
  S.rho2 = dV * v[1];
  S.F2 = dV * v[2];
  S.E = S.Q + 0.5 * ph.c0 * S.rho2 + 0.5 * ph.c1 * S.F2;
  S.mu = S.Q + ph.c0 * S.rho2 + ph.c1 * S.F2;
  double amax = 0.0;
  for (int c = 0; c < 3; ++c) {
    S.alpha[c] = dV * (kin[c] * X.inv_npts + v[3 + c] + ph.c0 * v[6 + c]);
    S.mass[c] = dV * v[9 + c];
    amax = fmax(amax, fabs(S.alpha[c]));
  }
  const double floor_a = 1e-12 * amax + 1e-300;
  for (int c = 0; c < 3; ++c) S.alpha[c] = fmax(S.alpha[c], floor_a);
  if (had_step) S.dphi_inf = sqrt(dphi);
  S.upd_applied = had_step ? 1 : 0;
  S.pending = 0;
  if (!isfinite(S.E) || !isfinite(S.mu) || !isfinite(S.alpha[0] + S.alpha[1] + S.alpha[2]))
    deactivate(S, GPSOC_ENONFINITE);
  mirror32(S);
}

// E, mu (Eqs. energy, muphi), alpha_l (Eq. PreCnstAlpha), masses of the current iterate
__device__ __forceinline__ void sc_obs(const ScalarCtx& X, int s, double* scratch) {
  __shared__ SolveState sS;
  state_load(sS, X.st + s);      // visible after the barrier that opens the first reduction
  double kin[3], v[12];
  if (!(X.flags & 8)) {
    const int kslots[3] = {SL_KIN0, SL_KIN1, SL_KIN2};
    slot_totals<3>(X, s, kslots, X.nb_col, kin, scratch);
  }
  const int slots[12] = {SL_Q, SL_RHO2, SL_F2, SL_V0, SL_V1, SL_V2, SL_C0, SL_C1, SL_C2, SL_M0, SL_M1, SL_M2};
  slot_totals<12>(X, s, slots, X.nb_row, v, scratch);
  // GPSOC_HYBRID: the kinetic part of alpha_l is that of the last exact FP64 recomputation
  // of H_lin Phi (alpha only shifts the preconditioner; the fixed point does not depend on it)
  if (X.flags & 8)
    for (int c = 0; c < 3; ++c) kin[c] = sS.kin[c];
  const bool had_step = sS.pending != 0;
  double dphi = 0.0;
  if (had_step) dphi = slot_max(X, s, SL_DPHIINF, X.nb_row, scratch);
  if (threadIdx.x == 0) obs_update(X, s, sS, kin, v, had_step, dphi);
  __syncthreads();
  state_store(X.st + s, sS);
}

constexpr int kStallWindow = 256;

// max_l ||r_l||_inf and the stopping test (Eqs. stop1-stop3)
__device__ __forceinline__ void sc_res(const ScalarCtx& X, int s, double* scratch) {
  SolveState& S = X.st[s];
  const double rinf = slot_max(X, s, SL_RINF, X.nb_row, scratch);
  if (threadIdx.x != 0) return;
  const OptsDev& O = X.opts;
  S.res_inf = rinf;
  if (!isfinite(rinf)) { deactivate(S, GPSOC_ENONFINITE); return; }
  if (O.no_stop) return;
  // FP32 phase: once the residual is this small the FP32 rounding floor is near, so
  // the level continues in FP64 (also at iteration 0: a level that starts converged
  // takes no FP32 step)
  if (O.phase32 && O.res32 > 0.0 && rinf < O.res32) { S.active = 0; return; }
  if (S.iters >= 1 || O.stop == GPSOC_STOP_RES) {
    bool conv;
    if (O.stop == GPSOC_STOP_ENERGY) conv = fabs(S.dE_last) < O.tol + O.tol_rel * fabs(S.E);
    else if (O.stop == GPSOC_STOP_RES) conv = rinf < O.tol;
    else conv = S.dphi_inf < O.tol;
    if (conv && O.res_tol > 0.0) conv = rinf < O.res_tol;
    if (conv) { S.active = 0; return; }
  }
  // FP32 phase: per-iteration energy changes carry rounding noise that can stay
  // above tol_rel |E| for ever; hand over to FP64 once the energy fell by less
  // than tol_rel |E| per iteration on average over a window of kStallWindow.
  if (O.phase32 && S.iters - S.it_win >= kStallWindow) {
    if (!(S.E_win - S.E >= kStallWindow * O.tol_rel * fabs(S.E))) { S.active = 0; return; }
    S.E_win = S.E;
    S.it_win = S.iters;
  }
  if (S.iters >= O.max_iter) {
    if (O.phase32) S.active = 0;
    else deactivate(S, GPSOC_ENOTCONV);
  }
}

// Polak-Ribiere+ beta = max(Re<r - r_prev, P r> / Re<r_prev, P_prev r_prev>, 0), the
// tangent projection coefficient c = Re<D, Phi> of D = -P r + beta P_prev (Eq. formula-
// project) and Algorithm 2 Step 2, all from the sums of the preconditioner's last pass:
// D is linear in beta, so Re<D, Phi> = -Re<z, Phi> + beta Re<P_prev, Phi> and the slope
// Re<r, D> = -Re<r, z> + beta Re<r, P_prev> (b_n has its sign: Re<H Phi, P> = Re<r, D>
// for the tangent P).  If the slope is not negative the step restarts from D = -P r.
__device__ __forceinline__ void sc_beta(const ScalarCtx& X, int s, double* scratch) {
  SolveState& S = X.st[s];
  double w[5];
  const int wslots[5] = {SL_RZ, SL_RPZ, SL_ZPHI, SL_PPHI, SL_RP};
  slot_totals<5>(X, s, wslots, X.nb_row, w, scratch);
  if (threadIdx.x != 0) return;
  const double dV = X.dV;
  const double rz = dV * w[0], zphi = dV * w[2];
  S.s_cur = rz;
  double beta = 0.0;
  if (!S.first) {
    beta = (rz - dV * w[1]) / S.s_prev;
    if (!(beta > 0.0)) beta = 0.0;   // max(beta, 0), NaN -> 0
  }
  double cD = -zphi + beta * dV * w[3];
  if (beta != 0.0 && !(-rz + beta * dV * w[4] < 0.0)) {
    beta = 0.0;
    S.beta_resets++;
    cD = -zphi;
  }
  S.beta = beta;
  S.cproj = cD;
  S.fbeta = (float)beta;
  S.fcproj = (float)cD;
}

// |P| and the reciprocals of |P| and |P|^2: one square root and one division
// per step (FP64 square roots and divisions are long instruction sequences).
struct PNorm {
  double nP, inv_nP, inv_nP2;
};
__device__ __forceinline__ PNorm p_norm(double nP2) {
  PNorm r;
  r.inv_nP2 = 1.0 / nP2;
  r.nP = sqrt(nP2);
  r.inv_nP = r.nP * r.inv_nP2;
  return r;
}

// E(cos t Phi + sin t P/||P||) - E(Phi) from the reduced integrals (unnormalised P),
// given sn = sin t, cs = cos t: quadratic part -s^2 Q + 2cs/|P| Re<H_lin Phi,P> +
// s^2/|P|^2 <H_lin P,P>, interaction part from rho_t - rho = u rho_Phi + w1 R + w2 rho_P
// (u = -s^2, w1 = 2cs/|P|, w2 = s^2/|P|^2) and the same for the spin density
// (Section 3.1, the explicit form of E(theta)).
__device__ __forceinline__ double energy_change_sc(const SolveState& S, double c0, double c1, double sn, double cs,
                                                   const PNorm& pn) {
  const double QFP = S.HPhiP - c0 * S.I[1] - c1 * S.J[1];
  const double u = -sn * sn, w1 = 2.0 * cs * sn * pn.inv_nP, w2 = sn * sn * pn.inv_nP2;
  const double quad = u * S.Q + w1 * QFP + w2 * S.HPP;
  const double* I = S.I;
  const double* J = S.J;
  const double rl = u * I[0] + w1 * I[1] + w2 * I[2];
  const double rq = u * u * I[0] + w1 * w1 * I[3] + w2 * w2 * I[5] + 2.0 * u * w1 * I[1] + 2.0 * u * w2 * I[2] +
                    2.0 * w1 * w2 * I[4];
  const double fl = u * J[0] + w1 * J[1] + w2 * J[2];
  const double fq = u * u * J[0] + w1 * w1 * J[3] + w2 * w2 * J[5] + 2.0 * u * w1 * J[1] + 2.0 * u * w2 * J[2] +
                    2.0 * w1 * w2 * J[4];
  return quad + 0.5 * c0 * (2.0 * rl + rq) + 0.5 * c1 * (2.0 * fl + fq);
}

__device__ __forceinline__ double energy_change(const SolveState& S, double c0, double c1, double theta) {
  double sn, cs;
  sincos(theta, &sn, &cs);
  return energy_change_sc(S, c0, c1, sn, cs, p_norm(S.P2));
}

// Eq. theta: theta_n = argmin_{theta > 0} E(cos t Phi + sin t P/|P|), on the explicit
// sin/cos form of the energy change.  With u = -s^2, v = 2cs/|P|, w = s^2/|P|^2 the change
// is a quadratic polynomial in (u, v, w) (energy_change_sc); its t-derivative follows with
// du/dt = -sin 2t, dv/dt = 2 cos 2t/|P|, dw/dt = sin 2t/|P|^2.  The minimiser taken is the
// first zero of the derivative found by doubling from the quadratic model's t0 (E has
// period pi and decreases at 0+), solved by Newton steps kept inside the bracket
// (bisection when a step leaves it).  If no sign change is met up to pi, t0 is kept.
struct TrigForm {
  double lu, l1, l2;                 // linear coefficients of u, v, w
  double huu, hu1, hu2, h11, h12, h22;   // second derivatives of the change in (u, v, w)
  double inv_nP, inv_nP2;
  // derivative (g1) and second derivative (g2) of the energy change at t
  __device__ __forceinline__ void eval(double t, double& g1, double& g2) const {
    double s2, c2;
    sincos(2.0 * t, &s2, &c2);
    const double u = -0.5 * (1.0 - c2), v = s2 * inv_nP, w = 0.5 * (1.0 - c2) * inv_nP2;
    const double du = -s2, dv = 2.0 * c2 * inv_nP, dw = s2 * inv_nP2;
    const double ddu = -2.0 * c2, ddv = -4.0 * s2 * inv_nP, ddw = 2.0 * c2 * inv_nP2;
    const double Au = lu + huu * u + hu1 * v + hu2 * w;
    const double A1 = l1 + hu1 * u + h11 * v + h12 * w;
    const double A2 = l2 + hu2 * u + h12 * v + h22 * w;
    g1 = Au * du + A1 * dv + A2 * dw;
    g2 = Au * ddu + A1 * ddv + A2 * ddw + huu * du * du + h11 * dv * dv + h22 * dw * dw +
         2.0 * (hu1 * du * dv + hu2 * du * dw + h12 * dv * dw);
  }
};

__device__ __forceinline__ double exact_theta(const SolveState& S, double c0, double c1, const PNorm& pn, double t0) {
  TrigForm f;
  const double* I = S.I;
  const double* J = S.J;
  const double QFP = S.HPhiP - c0 * I[1] - c1 * J[1];
  f.lu = S.Q + c0 * I[0] + c1 * J[0];
  f.l1 = QFP + c0 * I[1] + c1 * J[1];
  f.l2 = S.HPP + c0 * I[2] + c1 * J[2];
  f.huu = c0 * I[0] + c1 * J[0]; f.hu1 = c0 * I[1] + c1 * J[1]; f.hu2 = c0 * I[2] + c1 * J[2];
  f.h11 = c0 * I[3] + c1 * J[3]; f.h12 = c0 * I[4] + c1 * J[4]; f.h22 = c0 * I[5] + c1 * J[5];
  f.inv_nP = pn.inv_nP; f.inv_nP2 = pn.inv_nP2;
  const double PI = 3.14159265358979323846;
  double lo = 0.0, hi = fmin(t0, PI), g1, g2;
  f.eval(hi, g1, g2);
  while (g1 < 0.0 && hi < PI) {
    lo = hi;
    hi = fmin(2.0 * hi, PI);
    f.eval(hi, g1, g2);
  }
  if (g1 < 0.0) return t0;
  double t = hi;   // Newton from the right end of the bracket
  for (int it = 0; it < 100; ++it) {
    f.eval(t, g1, g2);
    if (g1 == 0.0) break;
    if (g1 < 0.0) lo = t; else hi = t;
    double tn = (g2 > 0.0) ? t - g1 / g2 : 0.5 * (lo + hi);
    if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
    if (fabs(tn - t) <= 1e-15 * t || hi - lo <= 2e-16 * hi) { t = tn; break; }
    t = tn;
  }
  return t;
}

// gather the step-model sums of the P chain into S (thread 0 holds the result);
// a_n, b_n of Eqs. an, bn
__device__ __forceinline__ void step_sums(const ScalarCtx& X, int s, double* scratch, SolveState& S, PNorm& pn) {
  double v[14];
  const int slots[14] = {SL_P2, SL_HPP, SL_HPHIP, SL_RPHI, SL_IFR, SL_IFP, SL_IRR, SL_IRP, SL_IPP,
                         SL_JFR, SL_JFP, SL_JRR, SL_JRP, SL_JPP};
  slot_totals<14>(X, s, slots, X.nb_row, v, scratch);
  if (threadIdx.x != 0) return;
  const double dV = X.dV;
  const PhysDev ph = X.phys[s];
  const double c0 = ph.c0, c1 = ph.c1;
  const double P2 = dV * v[0], HPP = dV * v[1], X1 = dV * v[2], RPhi = dV * v[3];
  double I[6], J[6];
  I[0] = S.rho2; J[0] = S.F2;
  for (int k = 0; k < 5; ++k) { I[k + 1] = dV * v[4 + k]; J[k + 1] = dV * v[9 + k]; }
  const double M = S.mass[0] + S.mass[1] + S.mass[2];
  // Re<H_lin Phi, P>: from Re<H Phi, P>, or in GPSOC_HYBRID from Re<r, P> + mu Re<P, Phi>
  const double QFP = ((X.flags & 8) ? X1 + S.mu * RPhi : X1) - c0 * I[1] - c1 * J[1];
  // Exact tangent correction: the step is taken along P_t = P - a Phi, a = Re<P, Phi>/||Phi||^2,
  // which is tangent to the sphere whatever the rounding of P (an FP32 direction carries a
  // radial part of relative size 1e-7).  Every sum transforms exactly: R -> R - a rho_Phi,
  // rho_P -> rho_P - 2a R + a^2 rho_Phi, and the same for the spin vectors.
  const double a = RPhi / M, a2 = a * a;
  S.acorr = a;
  S.P2 = P2 - a * RPhi;
  S.HPP = HPP - 2.0 * a * QFP + a2 * S.Q;
  S.RPhi = 0.0;
  for (int t = 0; t < 2; ++t) {
    const double* Y = t ? J : I;
    double* Z = t ? S.J : S.I;
    Z[0] = Y[0];
    Z[1] = Y[1] - a * Y[0];
    Z[2] = Y[2] - 2.0 * a * Y[1] + a2 * Y[0];
    Z[3] = Y[3] - 2.0 * a * Y[1] + a2 * Y[0];
    Z[4] = Y[4] - 2.0 * a * Y[3] - a * Y[2] + 3.0 * a2 * Y[1] - a2 * a * Y[0];
    Z[5] = Y[5] + 4.0 * a2 * Y[3] + a2 * a2 * Y[0] - 4.0 * a * Y[4] + 2.0 * a2 * Y[2] - 4.0 * a2 * a * Y[1];
  }
  S.HPhiP = (QFP - a * S.Q) + c0 * S.I[1] + c1 * S.J[1];
  pn = p_norm(S.P2);
  // density frozen at Phi^n in H_l(P^n)
  S.a = -S.mu + (S.HPP + ph.c0 * S.I[2] + ph.c1 * S.J[2] + 2.0 * (ph.c0 * S.I[3] + ph.c1 * S.J[3])) * pn.inv_nP2;
  S.b = 2.0 * S.HPhiP * pn.inv_nP;
}

// Algorithm 2: step size from the quadratic model, backtracking on the exact
// energy change, update coefficients of Eqs. formula-pcg / update (applied by
// the next iteration's first pass).  Thread 0, on its copy S of the state.
__device__ __forceinline__ void step_decide(const ScalarCtx& X, int s, SolveState& S, const PNorm& pn) {
  const PhysDev ph = X.phys[s];
  const OptsDev& O = X.opts;
  const double a = S.a, b = S.b;
  if (!isfinite(a) || !isfinite(b)) { deactivate(S, GPSOC_ENONFINITE); return; }
  if (b > 0.0 || (b == 0.0 && a >= 0.0)) {
    if (S.beta == 0.0) {
      if (O.phase32) S.active = 0;   // rounding floor of the FP32 phase: hand over to FP64
      else deactivate(S, GPSOC_ESTAGNATED);
      return;
    }
    // the sign test before the transform missed by rounding: redo this step with
    // beta = 0 in the next iteration (same Phi, same residual: Step 2 -> Step 1)
    S.first = 1;
    S.beta_resets++;
    return;
  }
  double theta = (a > 0.0 && b < 0.0) ? -b / (2.0 * a) : O.theta_trial;
  if (O.line_search == 1) theta = exact_theta(S, ph.c0, ph.c1, pn, theta);
  bool accepted = false;
  double dE = 0.0, sn = 0.0, cs = 1.0;
  for (int h = 0; h <= O.max_halvings; ++h) {
    sincos(theta, &sn, &cs);
    dE = energy_change_sc(S, ph.c0, ph.c1, sn, cs, pn);
    if (dE < 0.0) { accepted = true; break; }
    theta *= O.sigma;
    S.halvings++;
  }
  if (!accepted) {
    if (O.phase32) S.active = 0;
    else deactivate(S, GPSOC_ESTAGNATED);
    return;
  }
  S.theta = theta;
  S.dE = dE;
  S.dE_last = dE;
  const double sp = sn * pn.inv_nP;
  const double M = S.mass[0] + S.mass[1] + S.mass[2];
  // Phi' = (cos t Phi + sin t P_t/|P_t|)/norm with P_t = P - a Phi tangent: |.|^2 = c^2 M + s'^2 |P_t|^2
  const double nrm2 = cs * cs * M + sp * sp * S.P2;
  S.upd_c = cs - sp * S.acorr; S.upd_s = sp; S.upd_scale = rsqrt(nrm2);
  if (X.flags & 8) {
    // GPSOC_HYBRID: the double-word coefficients the opening pass applies
    const double uc = S.upd_scale * S.upd_c;
    dw_split(uc, S.dw_uc);
    dw_split(S.upd_scale * S.upd_s, S.dw_ut);
    dw_split(uc - 1.0, S.dw_ucm1);
  }
  S.pending = 1;
  S.last_par = (X.flags >> 2) & 1;
  S.iters++; S.total_iters++;
  if (X.flags & 2) S.fp32_iters++; else S.fp64_iters++;
  S.first = 0;
  S.s_prev = S.s_cur;
}

__device__ __forceinline__ void sc_step(const ScalarCtx& X, int s, double* scratch) {
  __shared__ SolveState sS;
  state_load(sS, X.st + s);      // visible after the barrier that opens the reduction
  PNorm pn;
  double kq[9];
  if (X.flags & 8) {
    // GPSOC_HYBRID: kinetic sums of Phi, of P and their cross term from the column pass
    const int ks[9] = {SL_KPHI0, SL_KPHI1, SL_KPHI2, SL_KX0, SL_KX1, SL_KX2, SL_KIN0, SL_KIN1, SL_KIN2};
    slot_totals<9>(X, s, ks, X.nb_col, kq, scratch);
  }
  step_sums(X, s, scratch, sS, pn);
  if (threadIdx.x == 0) {
    step_decide(X, s, sS, pn);
    if (X.flags & 8) {
      // kinetic part of alpha_l at the next iterate, exactly: Phi' = g (c Phi + t P), so
      // |k|^2 |Phi'_hat|^2 sums to g^2 (c^2 K_Phi + 2 c t K_x + t^2 K_P) per component
      const bool acc = sS.pending != 0;
      const double g2 = sS.upd_scale * sS.upd_scale, c = sS.upd_c, t = sS.upd_s;
      for (int l = 0; l < 3; ++l)
        sS.kin[l] = acc ? g2 * (c * c * kq[l] + 2.0 * c * t * kq[3 + l] + t * t * kq[6 + l]) : kq[l];
    }
    mirror32(sS);
  }
  __syncthreads();
  state_store(X.st + s, sS);
}

}  // namespace gpsoc
