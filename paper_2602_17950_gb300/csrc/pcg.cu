// PCG scalar steps and elementwise passes (Section 3.1, Algorithms 1 and 2).
//
// Scalar kernels run one block per solve: they add the per-block partial sums
// written by the array passes in a fixed order (deterministic results), then
// update the per-solve state: observables, stopping test, Polak-Ribiere+ beta,
// tangent projection coefficient, the step-size decision of Algorithm 2 and the
// update coefficients.  Energies along the step are evaluated through the
// explicit sin/cos expansion of E(theta) (Section 3.1, after Eq. theta), whose
// coefficients are integrals reduced by the P-chain pass.
#include <math.h>

#include "gpsoc_internal.cuh"
#include "kernels.cuh"

namespace gpsoc {

static constexpr int kScalarThreads = 256;

// sum (or max) of partials of `slot` over nb blocks for solve s; result valid in thread 0
__device__ double slot_total(const double* part, int pmax, int s, int slot, int nb, bool is_max, double* scratch) {
  double v[1] = {is_max ? 0.0 : 0.0};
  const double* p = part + ((long long)s * NSLOT + slot) * pmax;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) v[0] = is_max ? fmax(v[0], p[b]) : v[0] + p[b];
  const bool mx[1] = {is_max};
  block_reduce<1>(v, scratch, mx);
  return v[0];
}

__device__ __forceinline__ bool finite(double x) { return isfinite(x); }

__device__ __forceinline__ void deactivate(SolveState& S, int status) {
  S.active = 0;
  if (S.status == GPSOC_OK) S.status = status;
}

// E(cos t Phi + sin t P/||P||) - E(Phi) from the reduced integrals (unnormalised P):
// quadratic part -s^2 Q + 2cs/|P| Re<H_lin Phi,P> + s^2/|P|^2 <H_lin P,P>, interaction
// part from rho_t - rho = u rho_Phi + w1 R + w2 rho_P (u = -s^2, w1 = 2cs/|P|, w2 = s^2/|P|^2)
// and the same for each spin density component.
__device__ double energy_change(const SolveState& S, double c0, double c1, double theta) {
  const double nP2 = S.P2, nP = sqrt(nP2);
  const double QFP = S.HPhiP - c0 * S.I[1] - c1 * S.J[1];
  double sn, cs;
  sincos(theta, &sn, &cs);
  const double u = -sn * sn, w1 = 2.0 * cs * sn / nP, w2 = sn * sn / nP2;
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

__global__ void k_scalar(ScalarArgs A) {
  __shared__ double scratch[32];
  const int s = blockIdx.x;
  if (s >= A.nsolve) return;
  SolveState& S = A.st[s];
  const bool ok = (A.phase == PH_STEP_RESET || A.phase == PH_CPROJ_RESET) ? (S.active && S.reset) : (S.active != 0);
  if (A.phase != PH_INIT && A.phase != PH_NORM && !A.force && !ok) return;
  if (A.phase == PH_INIT) {
    if (threadIdx.x == 0) {
      S.active = 1; S.status = GPSOC_OK; S.iters = 0; S.first = 1; S.reset = 0;
      S.dE_last = nan(""); S.dphi_inf = nan("");
      if (A.flags & 1) { S.total_iters = 0; S.beta_resets = 0; S.halvings = 0; S.fp32_iters = 0; S.fp64_iters = 0; }
    }
    return;
  }
  const PhysDev ph = A.phys[s];
  const double dV = A.dV;
  const OptsDev& O = A.opts;
  if (A.phase == PH_NORM) {
    double m = slot_total(A.part, A.pmax, s, SL_NORM, A.nb_row, false, scratch);
    if (threadIdx.x == 0) A.norm_scale[s] = (m > 0.0 && finite(m)) ? 1.0 / sqrt(m * dV) : 0.0;
    return;
  }
  if (A.phase == PH_OBS) {
    double kin[3], v[12];
    for (int c = 0; c < 3; ++c) kin[c] = slot_total(A.part, A.pmax, s, SL_KIN0 + c, A.nb_col, false, scratch);
    const int slots[12] = {SL_Q, SL_RHO2, SL_F2, SL_V0, SL_V1, SL_V2, SL_C0, SL_C1, SL_C2, SL_M0, SL_M1, SL_M2};
    for (int k = 0; k < 12; ++k) v[k] = slot_total(A.part, A.pmax, s, slots[k], A.nb_row, false, scratch);
    double dphi = 0.0;
    if (S.iters > 0) dphi = slot_total(A.part, A.pmax, s, SL_DPHIINF, A.nb_row, true, scratch);
    if (threadIdx.x == 0) {
      S.Q = dV * v[0];
      S.rho2 = dV * v[1];
      S.F2 = dV * v[2];
      S.E = S.Q + 0.5 * ph.c0 * S.rho2 + 0.5 * ph.c1 * S.F2;
      S.mu = S.Q + ph.c0 * S.rho2 + ph.c1 * S.F2;
      double amax = 0.0;
      for (int c = 0; c < 3; ++c) {
        S.alpha[c] = dV * (kin[c] / (double)A.npts + v[3 + c] + ph.c0 * v[6 + c]);
        S.mass[c] = dV * v[9 + c];
        amax = fmax(amax, fabs(S.alpha[c]));
      }
      const double floor = 1e-12 * amax + 1e-300;
      for (int c = 0; c < 3; ++c) S.alpha[c] = fmax(S.alpha[c], floor);
      if (S.iters > 0) S.dphi_inf = dphi;
      if (!finite(S.E) || !finite(S.mu) || !finite(S.alpha[0] + S.alpha[1] + S.alpha[2]))
        deactivate(S, GPSOC_ENONFINITE);
    }
    return;
  }
  if (A.phase == PH_RES) {
    const double rinf = slot_total(A.part, A.pmax, s, SL_RINF, A.nb_row, true, scratch);
    if (threadIdx.x == 0) {
      S.res_inf = rinf;
      if (!finite(rinf)) { deactivate(S, GPSOC_ENONFINITE); return; }
      if (O.no_stop) return;
      if (S.iters >= 1 || O.stop == GPSOC_STOP_RES) {
        bool conv;
        if (O.stop == GPSOC_STOP_ENERGY) conv = fabs(S.dE_last) < O.tol;
        else if (O.stop == GPSOC_STOP_RES) conv = rinf < O.tol;
        else conv = S.dphi_inf < O.tol;
        if (conv && O.res_tol > 0.0) conv = rinf < O.res_tol;
        if (conv) { S.active = 0; return; }
      }
      if (S.iters >= O.max_iter) deactivate(S, GPSOC_ENOTCONV);
    }
    return;
  }
  if (A.phase == PH_BETA) {
    const double rz = slot_total(A.part, A.pmax, s, SL_RZ, A.nb_row, false, scratch);
    const double rpz = slot_total(A.part, A.pmax, s, SL_RPZ, A.nb_row, false, scratch);
    if (threadIdx.x == 0) {
      S.s_cur = dV * rz;
      double beta = 0.0;
      if (!S.first) {
        beta = (dV * rz - dV * rpz) / S.s_prev;     // Polak-Ribiere with s_prev = Re<r^{n-1}, P r^{n-1}>
        if (!(beta > 0.0)) beta = 0.0;              // max(beta, 0) (also maps NaN to 0)
      }
      S.beta = beta;
      S.reset = 0;
    }
    return;
  }
  if (A.phase == PH_CPROJ || A.phase == PH_CPROJ_RESET) {
    const double dphi = slot_total(A.part, A.pmax, s, SL_DPHI, A.nb_row, false, scratch);
    if (threadIdx.x == 0) S.cproj = dV * dphi;   // Re<D, Phi>
    return;
  }
  if (A.phase == PH_STEP || A.phase == PH_STEP_RESET || A.phase == PH_MODEL) {
    double v[14];
    const int slots[14] = {SL_P2, SL_HPP, SL_HPHIP, SL_RPHI, SL_IFR, SL_IFP, SL_IRR, SL_IRP, SL_IPP,
                           SL_JFR, SL_JFP, SL_JRR, SL_JRP, SL_JPP};
    for (int k = 0; k < 14; ++k) v[k] = slot_total(A.part, A.pmax, s, slots[k], A.nb_row, false, scratch);
    if (threadIdx.x != 0) return;
    S.P2 = dV * v[0]; S.HPP = dV * v[1]; S.HPhiP = dV * v[2]; S.RPhi = dV * v[3];
    for (int k = 0; k < 5; ++k) { S.I[k + 1] = dV * v[4 + k]; S.J[k + 1] = dV * v[9 + k]; }
    S.I[0] = S.rho2; S.J[0] = S.F2;
    const double c0 = ph.c0, c1 = ph.c1;
    const double nP2 = S.P2, nP = sqrt(nP2);
    // Eqs. an, bn (density frozen at Phi^n in H_l(P^n))
    const double a = -S.mu + (S.HPP + c0 * S.I[2] + c1 * S.J[2]) / nP2 + 2.0 * (c0 * S.I[3] + c1 * S.J[3]) / nP2;
    const double b = 2.0 * S.HPhiP / nP;
    S.a = a; S.b = b;
    if (A.phase == PH_MODEL) {
      double* o = A.model_out + (long long)s * (2 + A.n_theta);
      o[0] = a; o[1] = b;
      for (int k = 0; k < A.n_theta; ++k) o[2 + k] = energy_change(S, c0, c1, A.thetas[k]);
      return;
    }
    if (!finite(a) || !finite(b)) { deactivate(S, GPSOC_ENONFINITE); return; }
    // Algorithm 2, Step 2
    if (b > 0.0 || (b == 0.0 && a >= 0.0)) {
      if (S.beta == 0.0) { deactivate(S, GPSOC_ESTAGNATED); return; }
      S.beta = 0.0; S.reset = 1; S.beta_resets++;
      return;
    }
    S.reset = 0;
    double theta = (a > 0.0 && b < 0.0) ? -b / (2.0 * a) : O.theta_trial;
    bool accepted = false;
    double dE = 0.0;
    for (int h = 0; h <= O.max_halvings; ++h) {
      dE = energy_change(S, c0, c1, theta);
      if (dE < 0.0) { accepted = true; break; }
      theta *= O.sigma;
      S.halvings++;
    }
    if (!accepted) { deactivate(S, GPSOC_ESTAGNATED); return; }
    double sn, cs;
    sincos(theta, &sn, &cs);
    S.theta = theta;
    S.dE = dE;
    S.dE_last = dE;
    const double sp = sn / nP;
    const double M = S.mass[0] + S.mass[1] + S.mass[2];
    const double nrm2 = cs * cs * M + 2.0 * cs * sp * S.RPhi + sp * sp * nP2;
    S.upd_c = cs; S.upd_s = sp; S.upd_scale = 1.0 / sqrt(nrm2);
    S.iters++; S.total_iters++;
    if (A.flags & 2) S.fp32_iters++; else S.fp64_iters++;
    S.first = 0;
    S.s_prev = S.s_cur;
    return;
  }
}

// ------------------------------------------------------------------ elementwise passes
// Same block decomposition as the row passes: block -> (solve, rows [rb*R, rb*R+R)).
template <class T, int MODE>
__global__ void k_elem(ElemArgs<T> A) {
  using C = cx_t<T>;
  __shared__ double scratch[32];
  const int bps = A.bps;
  const int s = blockIdx.x / bps, rb = blockIdx.x % bps;
  if (s >= A.nsolve) return;
  const SolveState& S = A.st[s];
  if (A.gate == GATE_ACTIVE && !S.active) return;
  if (A.gate == GATE_RESET && !(S.active && S.reset)) return;
  const long long npts = A.npts;
  const long long per = npts / bps;
  const long long sbase = (long long)s * 3 * npts + (long long)rb * per;
  double acc[1] = {0.0};
  if (MODE == EL_DIR) {
    // D = -z + beta P_prev (Section 3.1); reduce Re<D, Phi>
    const double beta = S.beta;
    for (long long e = threadIdx.x; e < per; e += blockDim.x) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const long long i = sbase + c * npts + e;
        C z = A.in0[i];
        double dr = -(double)z.x, di = -(double)z.y;
        if (beta != 0.0) { C p = A.in1[i]; dr += beta * p.x; di += beta * p.y; }
        C f = A.in2[i];
        A.out0[i] = mk<C>(dr, di);
        acc[0] += dr * f.x + di * f.y;
      }
    }
  } else if (MODE == EL_UPDATE) {
    // Phi <- (cos t Phi + sin t P/||P||) / norm (Eqs. formula-pcg, update); reduce max |dPhi|
    const double cs = S.upd_c, sp = S.upd_s, sc = S.upd_scale;
    for (long long e = threadIdx.x; e < per; e += blockDim.x) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const long long i = sbase + c * npts + e;
        C f = A.out0[i];
        C p = A.in0[i];
        const double nr = sc * (cs * f.x + sp * p.x), ni = sc * (cs * f.y + sp * p.y);
        const C o = mk<C>(nr, ni);
        A.out0[i] = o;
        const double dr = (double)o.x - f.x, di = (double)o.y - f.y;
        acc[0] = fmax(acc[0], sqrt(dr * dr + di * di));
      }
    }
  } else if (MODE == EL_MASS) {
    for (long long e = threadIdx.x; e < per; e += blockDim.x) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        C f = A.in0[sbase + c * npts + e];
        acc[0] += (double)f.x * f.x + (double)f.y * f.y;
      }
    }
  } else if (MODE == EL_SCALE) {
    const double sc = A.scalev[s];
    for (long long e = threadIdx.x; e < per; e += blockDim.x) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        C f = A.in0[sbase + c * npts + e];
        A.out0[sbase + c * npts + e] = mk<C>(sc * f.x, sc * f.y);
      }
    }
    return;
  }
  const bool mx[1] = {MODE == EL_UPDATE};
  block_reduce<1>(acc, scratch, mx);
  if (threadIdx.x == 0) {
    const int slot = (MODE == EL_DIR) ? SL_DPHI : (MODE == EL_UPDATE) ? SL_DPHIINF : SL_NORM;
    A.part[((long long)s * NSLOT + slot) * A.pmax + rb] = acc[0];
  }
}

// zero-pad the full spectrum of level N (in) into level 2N (out, zeroed first)
template <class T>
__global__ void k_pad(const cx_t<T>* in, cx_t<T>* out, Geo gc, Geo gf, int nsolve) {
  const long long totc = (long long)nsolve * 3 * gc.npts;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < totc; i += (long long)gridDim.x * blockDim.x) {
    const long long sc = i / gc.npts;          // solve*3 + component
    long long r = i - sc * gc.npts;
    const int ix = (int)(r % gc.n[0]); r /= gc.n[0];
    const int iy = (int)(r % gc.n[1]); r /= gc.n[1];
    const int iz = (int)r;
    auto map = [](int k, int nc, int nf) { return (k < (nc >> 1)) ? k : k - nc + nf; };
    const int fx = map(ix, gc.n[0], gf.n[0]);
    const int fy = map(iy, gc.n[1], gf.n[1]);
    const int fz = (gc.d == 3) ? map(iz, gc.n[2], gf.n[2]) : 0;
    const long long fi = sc * gf.npts + ((long long)fz * gf.n[1] + fy) * gf.n[0] + fx;
    out[fi] = in[i];
  }
}

template <class T>
__global__ void k_convert(const void* in, int in_fp32, cx_t<T>* out, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    if (in_fp32) { float2 v = ((const float2*)in)[i]; out[i] = mk<cx_t<T>>(v.x, v.y); }
    else { double2 v = ((const double2*)in)[i]; out[i] = mk<cx_t<T>>(v.x, v.y); }
  }
}

// Initial guesses (a)-(f) of Section 4 before normalisation of the c, d, e, f kinds:
// raw values per component; kinds needing a norm are divided by it afterwards.
__global__ void k_guess(double2* out, Geo g, TrapDev trap, const PhysDev* phys, int nsolve, int k0, int k1, int k2,
                        double muTF_base) {
  const long long tot = (long long)nsolve * 3 * g.npts;
  const double PI = 3.14159265358979323846;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const long long sc = i / g.npts;
    const int s = (int)(sc / 3), c = (int)(sc % 3);
    long long r = i - sc * g.npts;
    const int ix = (int)(r % g.n[0]); r /= g.n[0];
    const int iy = (int)(r % g.n[1]); r /= g.n[1];
    const int iz = (int)r;
    const double x = -g.L[0] + ix * g.h[0], y = -g.L[1] + iy * g.h[1];
    const double z = (g.d == 3) ? -g.L[2] + iz * g.h[2] : 0.0;
    const double r2 = x * x + y * y + z * z;
    const double pa = pow(PI, -g.d / 4.0) * exp(-r2 / 2.0);
    const double pbr = x * pa, pbi = y * pa;   // (x + i y) phi_a
    const int kind = (c == 0) ? k0 : (c == 1) ? k1 : k2;
    const double W = phys[s].Omega;
    double re = 0.0, im = 0.0;
    switch (kind) {
      case 0: re = pa; break;
      case 1: re = pbr; im = pbi; break;
      case 2: re = pbr; im = -pbi; break;
      case 3: re = pa + pbr; im = pbi; break;
      case 4: re = pa + pbr; im = -pbi; break;
      case 5: re = (1 - W) * pa + W * pbr; im = W * pbi; break;
      case 6: re = (1 - W) * pa + W * pbr; im = -W * pbi; break;
      case 7: re = W * pa + (1 - W) * pbr; im = (1 - W) * pbi; break;
      case 8: re = W * pa + (1 - W) * pbr; im = -(1 - W) * pbi; break;
      case 9: {
        const double c0 = phys[s].c0;
        const double mu = muTF_base * ((g.d == 2) ? sqrt(c0) : pow(c0, 0.4));
        const double V = trap_value(trap, g, ix, iy, iz, i - sc * g.npts);
        re = (V < mu) ? sqrt((mu - V) / c0) : 0.0;
        break;
      }
    }
    out[i] = make_double2(re, im);
  }
}

// per component mass (for normalising guesses c-f componentwise): one block per (solve, component)
__global__ void k_comp_mass(const double2* in, long long npts, double dV, double* out) {
  __shared__ double scratch[32];
  const long long base = (long long)blockIdx.x * npts;
  double v[1] = {0.0};
  for (long long e = threadIdx.x; e < npts; e += blockDim.x) {
    double2 f = in[base + e];
    v[0] += f.x * f.x + f.y * f.y;
  }
  const bool mx[1] = {false};
  block_reduce<1>(v, scratch, mx);
  if (threadIdx.x == 0) out[blockIdx.x] = v[0] * dV;
}

__global__ void k_comp_scale(double2* data, long long npts, const double* mass, int k0, int k1, int k2) {
  const int sc = blockIdx.y;
  const int c = sc % 3;
  const int kind = (c == 0) ? k0 : (c == 1) ? k1 : k2;
  // kinds a, b, b_bar are used unnormalised (closed-form unit norm); c..f are divided by their grid norm
  const double f = (kind >= 3) ? 1.0 / sqrt(mass[sc]) : 1.0;
  const double scale = f / sqrt(3.0);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < npts; e += (long long)gridDim.x * blockDim.x) {
    double2 v = data[(long long)sc * npts + e];
    data[(long long)sc * npts + e] = make_double2(v.x * scale, v.y * scale);
  }
}

// ------------------------------------------------------------------ launchers
void launch_scalar(const ScalarArgs& a, cudaStream_t st) { k_scalar<<<a.nsolve, kScalarThreads, 0, st>>>(a); }

template <class T>
void launch_elem(int mode, const ElemArgs<T>& a, cudaStream_t st) {
  const int nb = a.bps * a.nsolve;
  switch (mode) {
    case EL_DIR: k_elem<T, EL_DIR><<<nb, 256, 0, st>>>(a); break;
    case EL_UPDATE: k_elem<T, EL_UPDATE><<<nb, 256, 0, st>>>(a); break;
    case EL_MASS: k_elem<T, EL_MASS><<<nb, 256, 0, st>>>(a); break;
    case EL_SCALE: k_elem<T, EL_SCALE><<<nb, 256, 0, st>>>(a); break;
  }
}

template <class T>
void launch_pad(const cx_t<T>* in, cx_t<T>* out, const Geo& gc, const Geo& gf, int nsolve, cudaStream_t st) {
  cudaMemsetAsync(out, 0, sizeof(cx_t<T>) * (size_t)nsolve * 3 * gf.npts, st);
  k_pad<T><<<1024, 256, 0, st>>>(in, out, gc, gf, nsolve);
}

template <class T>
void launch_convert(const void* in, int in_fp32, cx_t<T>* out, long long count, cudaStream_t st) {
  k_convert<T><<<1024, 256, 0, st>>>(in, in_fp32, out, count);
}

void launch_guess(double2* out, const Geo& g, const TrapDev& trap, const PhysDev* phys, int nsolve, const int kind[3],
                  double muTF_base, double* mass_tmp, cudaStream_t st) {
  k_guess<<<1024, 256, 0, st>>>(out, g, trap, phys, nsolve, kind[0], kind[1], kind[2], muTF_base);
  k_comp_mass<<<nsolve * 3, 256, 0, st>>>(out, g.npts, g.dV, mass_tmp);
  dim3 grid(64, nsolve * 3);
  k_comp_scale<<<grid, 256, 0, st>>>(out, g.npts, mass_tmp, kind[0], kind[1], kind[2]);
}

template void launch_elem<double>(int, const ElemArgs<double>&, cudaStream_t);
template void launch_elem<float>(int, const ElemArgs<float>&, cudaStream_t);
template void launch_pad<double>(const double2*, double2*, const Geo&, const Geo&, int, cudaStream_t);
template void launch_pad<float>(const float2*, float2*, const Geo&, const Geo&, int, cudaStream_t);
template void launch_convert<double>(const void*, int, double2*, long long, cudaStream_t);
template void launch_convert<float>(const void*, int, float2*, long long, cudaStream_t);

}  // namespace gpsoc
