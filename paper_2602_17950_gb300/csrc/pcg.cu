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

#include <algorithm>

#include "gpsoc_internal.cuh"
#include "kernels.cuh"
#include "scalar.cuh"

namespace gpsoc {

static constexpr int kScalarThreads = 128;

__global__ void k_scalar(ScalarArgs A) {
  __shared__ double scratch[16 * 8 + 16];
  pdl_wait();
  const int s = blockIdx.x;
  if (s >= A.nsolve) return;
  SolveState& S = A.st[s];
  const int ph_ = A.phase;
  if (A.only >= 0 && s != A.only) return;
  if (ph_ != PH_INIT && ph_ != PH_NORM && !A.force && !S.active) return;
  ScalarCtx X{A.st, A.phys, A.part, A.pmax, A.nb_row, A.nb_col, A.npts, A.dV, A.opts, A.flags, A.inv_npts, A.part_dw};
  switch (ph_) {
    case PH_INIT:
      if (threadIdx.x == 0) {
        // flags & 4: the level continues from a direction handed over by the FP32 phase
        // (first, s_prev and the stored r_prev, P_prev are kept)
        if (!(A.flags & 4)) S.first = 1;
        S.active = 1; S.status = GPSOC_OK; S.iters = 0; S.reset = 0; S.pending = 0;
        S.dE_last = nan(""); S.dphi_inf = nan(""); S.E_win = INFINITY; S.it_win = 0;
        if (A.flags & 1) { S.total_iters = 0; S.beta_resets = 0; S.halvings = 0; S.fp32_iters = 0; S.fp64_iters = 0; }
        mirror32(S);
      }
      return;
    case PH_NORM: {
      double v[1];
      const int sl[1] = {SL_NORM};
      slot_totals<1>(X, s, sl, A.nb_row, v, scratch);
      if (threadIdx.x == 0) A.norm_scale[s] = (v[0] > 0.0 && isfinite(v[0])) ? 1.0 / sqrt(v[0] * A.dV) : 0.0;
      return;
    }
    case PH_OBS: sc_obs(X, s, scratch); return;
    case PH_RES: sc_res(X, s, scratch); return;
    case PH_BETA: sc_beta(X, s, scratch); return;
    case PH_STEP: sc_step(X, s, scratch); return;
    case PH_CLEAR: if (threadIdx.x == 0) S.pending = 0; return;
    case PH_KIN: {
      double kin[3];
      const int ks[3] = {SL_KIN0, SL_KIN1, SL_KIN2};
      slot_totals<3>(X, s, ks, A.nb_col, kin, scratch);
      if (threadIdx.x == 0) for (int c = 0; c < 3; ++c) S.kin[c] = kin[c];
      return;
    }
    case PH_MODEL: {
      SolveState L;
      if (threadIdx.x == 0) L = S;
      PNorm pn;
      step_sums(X, s, scratch, L, pn);
      if (threadIdx.x == 0) {
        S = L;
        const PhysDev ph = A.phys[s];
        double* o = A.model_out + (long long)s * (2 + A.n_theta);
        o[0] = L.a; o[1] = L.b;
        for (int k = 0; k < A.n_theta; ++k) o[2 + k] = energy_change(L, ph.c0, ph.c1, A.thetas[k]);
      }
      return;
    }
  }
}

// ------------------------------------------------------------------ elementwise passes
// Same block decomposition as the row passes: block -> (solve, rows [rb*R, rb*R+R)).
template <class T, int MODE>
__global__ void k_elem(ElemArgs<T> A) {
  using C = cx_t<T>;
  using W = T;   // working precision of the pointwise math; block sums in FP64
  __shared__ double scratch[16 * 8 + 16];
  pdl_wait();
  const int bps = A.bps;
  const int s = blockIdx.x / bps, rb = blockIdx.x % bps;
  if (s >= A.nsolve) return;
  const SolveState& S = A.st[s];
  if (A.only >= 0 && s != A.only) return;
  if (!gate_ok(A.st, A.gate, s)) return;
  const long long npts = A.npts;
  const long long per = npts / bps;
  const long long sbase = (long long)s * 3 * npts + (long long)rb * per;
  W acc = (W)0;
  if (MODE == EL_UPDATE) {
    // Phi <- (cos t Phi + sin t P/||P||) / norm (Eqs. formula-pcg, update); reduce max |dPhi|^2
    const W cs = pick<W>(S.upd_c, S.fupd_c), sp = pick<W>(S.upd_s, S.fupd_s), sc = pick<W>(S.upd_scale, S.fupd_scale);
    for (long long e = threadIdx.x; e < per; e += blockDim.x) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const long long i = sbase + c * npts + e;
        const C f = A.out0[i];
        const C p = A.in0[i];
        const C o = mk<C>(sc * (cs * f.x + sp * p.x), sc * (cs * f.y + sp * p.y));
        A.out0[i] = o;
        const W dr = o.x - f.x, di = o.y - f.y;
        acc = fmax(acc, dr * dr + di * di);
      }
    }
  } else if (MODE == EL_MASS) {
    for (long long e = threadIdx.x; e < per; e += blockDim.x) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const C f = A.in0[sbase + c * npts + e];
        acc += f.x * f.x + f.y * f.y;
      }
    }
  } else if (MODE == EL_SCALE) {
    const W sc = (W)A.scalev[s];
    for (long long e = threadIdx.x; e < per; e += blockDim.x) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const C f = A.in0[sbase + c * npts + e];
        A.out0[sbase + c * npts + e] = mk<C>(sc * f.x, sc * f.y);
      }
    }
    return;
  }
  double v[1] = {(double)acc};
  const bool mx[1] = {MODE == EL_UPDATE};
  block_reduce<1>(v, scratch, mx);
  if (threadIdx.x == 0) {
    const int slot = (MODE == EL_UPDATE) ? SL_DPHIINF : SL_NORM;
    put_partial(A.part + ((long long)s * NSLOT + slot) * A.pmax + rb, v[0], MODE == EL_UPDATE, sizeof(T) == 4);
  }
}

// GPSOC_HYBRID opening pass (see HyArgs).  The state, H_lin Phi and H(Phi) are stored in
// FP64, and every value the energy, mu, the residual and the normalisation depend on carries
// about 48 significant bits: the pointwise arithmetic runs in double words (FP32 pairs) on
// the FP32 pipes, because this part issues one FP64 warp instruction per 64 cycles per SM
// sub-partition; FP64 instructions remain only to split the loaded values and to round
// the stored ones.  The alpha_l pieces V |phi_l|^2 and rho |phi_l|^2, which only shift
// the preconditioner, are FP32 products; max |Phi' - Phi|^2 is taken from the high words.
// The block sums are double words, stored as double-word partials for the observables
// step (grid sums on the FP32 pipes, totals rounded to FP64).
constexpr int kHyThreads = 256, kHyBlocksPerSM = 2;

__global__ void __launch_bounds__(kHyThreads, kHyBlocksPerSM) k_hy_upd(HyArgs A) {
  __shared__ double scratch[16 * 8 + 16];
  pdl_wait();
  const int bps = A.bps;
  const int s = blockIdx.x / bps, rb = blockIdx.x % bps;
  if (s >= A.nsolve || !gate_ok(A.st, A.gate, s)) return;
  const SolveState& S = A.st[s];
  const long long npts = A.npts;
  // block rb of the solve takes points [rb npts / bps, (rb + 1) npts / bps)
  const long long ebase = (long long)rb * npts / bps, per = (long long)(rb + 1) * npts / bps - ebase;
  const long long sbase = (long long)s * 3 * npts;
  const bool upd = (A.flags & HY_UPD) && S.pending;
  const bool rec = upd && (A.flags & HY_REC);
  const bool red = (A.flags & HY_REDUCE) != 0;
  // Phi' = g (c Phi + t P) = uc Phi + ut P, as the change (uc - 1) Phi + ut P added to Phi
  // (uc = g c, ut = g t split into double words by the step that accepted them)
  const DF uc = DF{S.dw_uc[0], S.dw_uc[1]}, ut = DF{S.dw_ut[0], S.dw_ut[1]};
  const DF ucm1 = DF{S.dw_ucm1[0], S.dw_ucm1[1]};
  const PhysDev ph = A.phys[s];
  const DF c0 = DF{ph.fc0, ph.c0lo}, c1 = DF{ph.fc1, ph.c1lo};
  const int nx = A.g.n[0], ny = A.g.n[1];
  DF acc[6];
  float acc32[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) { acc[k] = DF{0.0f, 0.0f}; acc32[k] = 0.0f; }
  float dmax = 0.0f;
  for (long long e = threadIdx.x; e < per; e += blockDim.x) {
    const long long off = ebase + e;
    // every load of the point first (one memory round trip), then the arithmetic
    double2 f64[3], h64[3];
    float2 q[3], hq[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long i = sbase + c * npts + off;
      f64[c] = A.phi[i];
      if (red || rec) h64[c] = A.hl[i];
      if (upd) q[c] = A.p[i];
      if (rec) hq[c] = A.hlp[i];
    }
    DF fx[3], fy[3], hx[3], hy[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long i = sbase + c * npts + off;
      fx[c] = dw_of(f64[c].x);
      fy[c] = dw_of(f64[c].y);
      if (red && !rec) {
        hx[c] = dw_of(h64[c].x);
        hy[c] = dw_of(h64[c].y);
      }
      if (upd) {
        // the accepted step (Eqs. formula-pcg, update) with the exact tangent direction
        const DF dx = dw_add(dw_mul(ucm1, fx[c]), dw_mulf(ut, q[c].x));
        const DF dy = dw_add(dw_mul(ucm1, fy[c]), dw_mulf(ut, q[c].y));
        dmax = fmaxf(dmax, dx.hi * dx.hi + dy.hi * dy.hi);
        fx[c] = dw_add(fx[c], dx);
        fy[c] = dw_add(fy[c], dy);
        A.phi[i] = make_double2(dw_to_double(fx[c]), dw_to_double(fy[c]));
        if (rec) {
          // H_lin is linear: H_lin Phi' = g (c H_lin Phi + t H_lin P)
          hx[c] = dw_add(dw_mul(uc, dw_of(h64[c].x)), dw_mulf(ut, hq[c].x));
          hy[c] = dw_add(dw_mul(uc, dw_of(h64[c].y)), dw_mulf(ut, hq[c].y));
          A.hl[i] = make_double2(dw_to_double(hx[c]), dw_to_double(hy[c]));
        }
      }
    }
    if (!red) continue;
    // H(Phi) = H_lin Phi + c0 rho Phi + c1 (F.f) Phi (Eqs. eigen1-eigen3) and the sums of the
    // energy (Eq. energy) and of alpha_l (Eq. PreCnstAlpha)
    DF m[3];
    float mf[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      m[c] = dw_add(dw_mul(fx[c], fx[c]), dw_mul(fy[c], fy[c]));
      acc[0] = dw_add(acc[0], dw_add(dw_mul(fx[c], hx[c]), dw_mul(fy[c], hy[c])));
      A.phi32[sbase + c * npts + off] = make_float2(fx[c].hi, fy[c].hi);
      mf[c] = fx[c].hi * fx[c].hi + fy[c].hi * fy[c].hi;   // the alpha pieces (FP32)
    }
    const DF rho = dw_add(dw_add(m[0], m[1]), m[2]);
    // a = phi_1 conj(phi_0) + phi_0 conj(phi_-1) (components ordered 1, 0, -1), Fz = |phi_1|^2 - |phi_-1|^2
    const DF ar = dw_add(dw_add(dw_mul(fx[1], fx[0]), dw_mul(fy[1], fy[0])),
                         dw_add(dw_mul(fx[2], fx[1]), dw_mul(fy[2], fy[1])));
    const DF ai = dw_add(dw_sub(dw_mul(fx[1], fy[0]), dw_mul(fy[1], fx[0])),
                         dw_sub(dw_mul(fx[2], fy[1]), dw_mul(fy[2], fx[1])));
    const DF Fz = dw_sub(m[0], m[2]);
    DF fr[3], fi[3];
    fr[0] = dw_add(dw_mul(Fz, fx[0]), dw_sub(dw_mul(ar, fx[1]), dw_mul(ai, fy[1])));
    fi[0] = dw_add(dw_mul(Fz, fy[0]), dw_add(dw_mul(ar, fy[1]), dw_mul(ai, fx[1])));
    fr[1] = dw_add(dw_add(dw_mul(ar, fx[0]), dw_mul(ai, fy[0])), dw_sub(dw_mul(ar, fx[2]), dw_mul(ai, fy[2])));
    fi[1] = dw_add(dw_sub(dw_mul(ar, fy[0]), dw_mul(ai, fx[0])), dw_add(dw_mul(ar, fy[2]), dw_mul(ai, fx[2])));
    fr[2] = dw_sub(dw_add(dw_mul(ar, fx[1]), dw_mul(ai, fy[1])), dw_mul(Fz, fx[2]));
    fi[2] = dw_sub(dw_sub(dw_mul(ar, fy[1]), dw_mul(ai, fx[1])), dw_mul(Fz, fy[2]));
    const DF c0r = dw_mul(c0, rho);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const DF hr = dw_add(dw_add(hx[c], dw_mul(c0r, fx[c])), dw_mul(c1, fr[c]));
      const DF hi = dw_add(dw_add(hy[c], dw_mul(c0r, fy[c])), dw_mul(c1, fi[c]));
      A.hphi[sbase + c * npts + off] = make_double2(dw_to_double(hr), dw_to_double(hi));
    }
    acc[1] = dw_add(acc[1], dw_mul(rho, rho));
    const DF a2 = dw_add(dw_mul(ar, ar), dw_mul(ai, ai));
    acc[2] = dw_add(acc[2], dw_add(dw_add(a2, a2), dw_mul(Fz, Fz)));
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[3 + c] = dw_add(acc[3 + c], m[c]);
    const long long row = off / nx;
    const float V = trap_value<float>(A.trap, A.g, (int)(off - row * nx), (int)(row % ny), (int)(row / ny), off);
    const float rf = mf[0] + mf[1] + mf[2];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      acc32[c] += V * mf[c];
      acc32[3 + c] += rf * mf[c];
    }
  }
  double* P = A.part + (long long)s * NSLOT * A.pmax + rb;
  if (upd) {
    const double v = block_reduce1_f(dmax, true, scratch);
    if (threadIdx.x == 0) put_partial(P + (long long)SL_DPHIINF * A.pmax, v, true, true);
  }
  if (!red) return;
  DF all[12];
#pragma unroll
  for (int k = 0; k < 6; ++k) { all[k] = acc[k]; all[6 + k] = DF{acc32[k], 0.0f}; }
  double v[12];
  block_reduce_dw<12>(all, v, scratch);
  const int slots[12] = {SL_Q, SL_RHO2, SL_F2, SL_M0, SL_M1, SL_M2, SL_V0, SL_V1, SL_V2, SL_C0, SL_C1, SL_C2};
  const bool mx[12] = {};
  put_partials<12>(A.part, (long long)s * NSLOT, A.pmax, rb, slots, v, mx, true);
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

// End of an FP32 phase: solves that took FP32 steps get their state back in FP64
// (Phi, and r_prev, P_prev of the last accepted step into the FP64 buffers of parity 1,
// which the first FP64 iteration reads as the previous ones); a solve that took no
// FP32 step keeps its FP64 state untouched.
__global__ void k_handover(const float2* phi32, const float2* const* r32, const float2* const* p32, double2* phi64,
                           double2* r64_prev, double2* p64_prev, const SolveState* st, long long per_solve,
                           int nsolve, int carry) {
  const long long tot = (long long)nsolve * per_solve;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(i / per_solve);
    const SolveState& S = st[s];
    if (S.iters == 0) continue;
    const float2 f = phi32[i];
    phi64[i] = make_double2(f.x, f.y);
    if (carry && !S.first) {
      const float2 r = r32[S.last_par][i], q = p32[S.last_par][i];
      r64_prev[i] = make_double2(r.x, r.y);
      p64_prev[i] = make_double2(q.x, q.y);
    }
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
        const double V = trap_value<double>(trap, g, ix, iy, iz, i - sc * g.npts);
        re = (V < mu) ? sqrt((mu - V) / c0) : 0.0;
        break;
      }
    }
    out[i] = make_double2(re, im);
  }
}

// per component mass (for normalising guesses c-f componentwise): one block per (solve, component)
__global__ void k_comp_mass(const double2* in, long long npts, double dV, double* out) {
  __shared__ double scratch[16 * 8 + 16];
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
void launch_scalar(const ScalarArgs& a, cudaStream_t st) {
  launch_pdl(k_scalar, a.nsolve, kScalarThreads, 0, st, a);
}

void launch_hy_upd(const HyArgs& a, cudaStream_t st) {
  launch_pdl(k_hy_upd, a.bps * a.nsolve, kHyThreads, 0, st, a);
}

// The pass is FP64-bound: its time is that of the busiest SM.  Two 256-thread blocks
// are resident per SM, so the grid is a whole number of waves of 2 nsm blocks (split
// over the solves, rounded up), with about four points per thread at most.
int hy_blocks_per_solve(const Geo& g, int nsolve, int nsm) {
  const long long wave = (long long)kHyBlocksPerSM * std::max(nsm, 1);
  const long long work = (long long)std::max(nsolve, 1) * g.npts;
  const long long waves = std::max(1LL, (work + wave * kHyThreads * 4 - 1) / (wave * kHyThreads * 4));
  const long long b = (wave * waves + nsolve - 1) / std::max(nsolve, 1);
  return (int)std::max(1LL, std::min(b, g.npts));
}

template <class T>
void launch_elem(int mode, const ElemArgs<T>& a, cudaStream_t st) {
  const int nb = a.bps * a.nsolve;
  switch (mode) {
    case EL_UPDATE: launch_pdl(k_elem<T, EL_UPDATE>, nb, 256, 0, st, a); break;
    case EL_MASS: launch_pdl(k_elem<T, EL_MASS>, nb, 256, 0, st, a); break;
    case EL_SCALE: launch_pdl(k_elem<T, EL_SCALE>, nb, 256, 0, st, a); break;
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

void launch_handover(const float2* phi32, const float2* const* r32, const float2* const* p32, double2* phi64,
                     double2* r64_prev, double2* p64_prev, const SolveState* st, long long per_solve, int nsolve,
                     int carry, cudaStream_t stream) {
  k_handover<<<1024, 256, 0, stream>>>(phi32, r32, p32, phi64, r64_prev, p64_prev, st, per_solve, nsolve, carry);
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
