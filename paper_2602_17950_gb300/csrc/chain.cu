// Spectral passes of the Hamiltonian and preconditioner chains.
//
// A d-dimensional transform is a sequence of 1-D axis passes; each pass loads
// a tile into shared memory, runs radix-2 FFTs there and stores back with
// coalesced accesses.  Row passes (x, contiguous) take R whole rows of all
// three components; column passes (y or z, strided) take a tile of TC
// consecutive inner indices across the whole axis for all three components,
// so the 3x3 spin-orbit symbol and the pointwise spin terms see every
// component of a point in one block.
//
// Chains (Section 3.2 symbols; Section 2.2 operators; Section 3.4 preconditioner):
//   H chain 2D:  X fwd -> Y (fwd, symbol, inv, rotation pieces) -> X inv + pointwise
//   H chain 3D:  X fwd -> Y fwd -> Z (fwd, symbol, inv) -> Y inv + rotation -> X inv + pointwise
//   P_C chain:   X fwd of P_V^{1/2} r -> [Y fwd] -> last axis (fwd, divide, inv) -> [Y inv] -> X inv, P_V^{1/2}
// Rotation term -Omega Lz phi = Omega y D_x phi - Omega x D_y phi with D = -i d:
// the y D_x piece is folded into the spectral-in-x array before the last x
// inverse (y is constant along an x row), the x D_y piece is carried as a
// second array G = F_y^{-1}[v_y F_y A] and multiplied by x after the x inverse.
#include "gpsoc_internal.cuh"

namespace gpsoc {

static constexpr int kThreads = 256;

template <class T>
__device__ __forceinline__ void load_tw(cx_t<T>* s_tw, const cx_t<T>* tw, int n) {
  for (int k = threadIdx.x; k < (n >> 1); k += blockDim.x) s_tw[k] = tw[k];
}

// spin terms shared by the pointwise epilogues:
//   a = conj(p0) p1 + conj(pm) p0  so that F_-/sqrt2 = a, F_+/sqrt2 = conj(a),
//   F_x = sqrt2 Re a, F_y = -sqrt2 Im a, F_z = |p1|^2 - |pm|^2, |F|^2 = 2|a|^2 + F_z^2.
template <class C>
__device__ __forceinline__ double2 spin_a(C p1, C p0, C pm) {
  double ar = (double)p0.x * p1.x + (double)p0.y * p1.y + (double)pm.x * p0.x + (double)pm.y * p0.y;
  double ai = (double)p0.x * p1.y - (double)p0.y * p1.x + (double)pm.x * p0.y - (double)pm.y * p0.x;
  return make_double2(ar, ai);
}

// ============================================================== row passes (x axis)
template <class T, int MODE>
__global__ void __launch_bounds__(kThreads) k_row(ChainArgs<T> A, int R) {
  using C = cx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nx = A.g.n[0], Lx = A.g.log2n[0];
  const long long npts = A.g.npts;
  const int rows = (int)(npts / nx);
  const int bps = rows / R;
  const int s = blockIdx.x / bps;
  const int rb = blockIdx.x % bps;
  if (s >= A.nsolve || !gate_ok(A.st, A.gate, s)) return;
  C* s_tw = (C*)smem_raw;
  C* buf0 = s_tw + (nx >> 1);
  const int per = R * nx;             // elements of one component in the tile
  C* buf1 = buf0 + 3 * per;
  double* red = (double*)(buf1 + ((MODE == ROW_INV_H || MODE == ROW_INV_P || MODE == ROW_INV_LIN) ? 3 * per : 0));
  load_tw<T>(s_tw, A.tw[0], nx);
  const long long sbase = (long long)s * 3 * npts;
  const long long rbase = (long long)rb * R * nx;   // offset of the tile inside a component
  const SolveState& S = A.st[s];
  const PhysDev ph = A.phys[s];
  const int ny = A.g.n[1];

  if (MODE == ROW_FWD_PLAIN || MODE == ROW_FWD_PROJ || MODE == ROW_FWD_PRE) {
    double acc[1] = {0.0};
    const double cproj = S.cproj, mu = A.given_r ? 0.0 : S.mu;
    double al[3] = {S.alpha[0], S.alpha[1], S.alpha[2]};
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int r = e / nx, j = e - r * nx;
      const long long off = rbase + e;
      const int pos = r * nx + bitrev(j, Lx);
      if (MODE == ROW_FWD_PLAIN) {
#pragma unroll
        for (int c = 0; c < 3; ++c) buf0[c * per + pos] = A.in0[sbase + c * npts + off];
      } else if (MODE == ROW_FWD_PROJ) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          C d = A.in0[sbase + c * npts + off];
          C f = A.in1[sbase + c * npts + off];
          C p;
          p.x = (T)((double)d.x - cproj * (double)f.x);
          p.y = (T)((double)d.y - cproj * (double)f.y);
          A.out1[sbase + c * npts + off] = p;
          acc[0] += (double)p.x * p.x + (double)p.y * p.y;
          buf0[c * per + pos] = p;
        }
      } else {  // ROW_FWD_PRE
        C f[3], h[3];
        double rho = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          f[c] = A.in1[sbase + c * npts + off];
          h[c] = A.in0[sbase + c * npts + off];
          rho += (double)f[c].x * f[c].x + (double)f[c].y * f[c].y;
        }
        const long long gi = rbase + e;  // flat point index inside the component
        const int ix = j;
        const long long row = gi / nx;
        const int iy = (int)(row % ny), iz = (int)(row / ny);
        const double V = trap_value(A.trap, A.g, ix, iy, iz, gi);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          C r;
          r.x = (T)((double)h[c].x - mu * (double)f[c].x);
          r.y = (T)((double)h[c].y - mu * (double)f[c].y);
          A.out1[sbase + c * npts + off] = r;
          acc[0] = fmax(acc[0], sqrt((double)r.x * r.x + (double)r.y * r.y));
          double den = al[c] + V + ph.c0 * rho;
          den = fmax(den, 1e-12 * al[c]);
          const double sc = 1.0 / sqrt(den);
          buf0[c * per + pos] = mk<C>((double)r.x * sc, (double)r.y * sc);
        }
      }
    }
    __syncthreads();
    fft_dit<C, false>(buf0, Lx, 3 * R, 3 * R, 0, nx, 1, s_tw, false);
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
#pragma unroll
      for (int c = 0; c < 3; ++c) A.out0[sbase + c * npts + rbase + e] = buf0[c * per + e];
    }
    if (MODE == ROW_FWD_PROJ || MODE == ROW_FWD_PRE) {
      const bool mx[1] = {MODE == ROW_FWD_PRE};
      block_reduce<1>(acc, (double*)buf0, mx);
      if (threadIdx.x == 0) {
        const int slot = (MODE == ROW_FWD_PROJ) ? SL_P2 : SL_RINF;
        A.part[((long long)s * NSLOT + slot) * A.pmax + rb] = acc[0];
      }
    }
    return;
  }

  // ---------------------------------------------------------------- inverse passes
  // load natural order, DIF inverse -> bit-reversed positions in shared memory
  const bool two = (MODE == ROW_INV_H || MODE == ROW_INV_P || MODE == ROW_INV_LIN);
  for (int e = threadIdx.x; e < per; e += blockDim.x) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      buf0[c * per + e] = A.in0[sbase + c * npts + rbase + e];
      if (two) buf1[c * per + e] = A.in1[sbase + c * npts + rbase + e];
    }
  }
  __syncthreads();
  fft_dif<C, false>(buf0, Lx, two ? 6 * R : 3 * R, two ? 6 * R : 3 * R, 0, nx, 1, s_tw, true);

  const double inv_n = 1.0 / (double)npts;
  const double Om = ph.Omega;
  if (MODE == ROW_INV_PLAIN) {
    const double sc = A.scale;
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int r = e / nx, j = e - r * nx;
      const int pos = r * nx + bitrev(j, Lx);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        C v = buf0[c * per + pos];
        A.out0[sbase + c * npts + rbase + e] = mk<C>((double)v.x * sc, (double)v.y * sc);
      }
    }
    return;
  }
  if (MODE == ROW_INV_PRE) {
    double acc[2] = {0.0, 0.0};
    const bool use_prev = (A.in3 != nullptr) && !S.first;
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int r = e / nx, j = e - r * nx;
      const int pos = r * nx + bitrev(j, Lx);
      const long long off = rbase + e;
      C f[3];
      double rho = 0.0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        f[c] = A.in1[sbase + c * npts + off];
        rho += (double)f[c].x * f[c].x + (double)f[c].y * f[c].y;
      }
      const long long row = off / nx;
      const double V = trap_value(A.trap, A.g, j, (int)(row % ny), (int)(row / ny), off);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double den = S.alpha[c] + V + ph.c0 * rho;
        den = fmax(den, 1e-12 * S.alpha[c]);
        const double sc = inv_n / sqrt(den);
        C v = buf0[c * per + pos];
        C z = mk<C>((double)v.x * sc, (double)v.y * sc);
        A.out0[sbase + c * npts + off] = z;
        C rr = A.in2[sbase + c * npts + off];
        acc[0] += (double)rr.x * z.x + (double)rr.y * z.y;
        if (use_prev) {
          C rp = A.in3[sbase + c * npts + off];
          acc[1] += (double)rp.x * z.x + (double)rp.y * z.y;
        }
      }
    }
    const bool mx[2] = {false, false};
    block_reduce<2>(acc, red, mx);
    if (threadIdx.x == 0) {
      A.part[((long long)s * NSLOT + SL_RZ) * A.pmax + rb] = acc[0];
      A.part[((long long)s * NSLOT + SL_RPZ) * A.pmax + rb] = acc[1];
    }
    return;
  }

  // ROW_INV_H / ROW_INV_P / ROW_INV_LIN: lin = F_x^-1(T')/npts - Omega x F_x^-1(G)/npts + V u
  const double c0 = ph.c0, c1 = ph.c1;
  double acc[13];
#pragma unroll
  for (int k = 0; k < 13; ++k) acc[k] = 0.0;
  for (int e = threadIdx.x; e < per; e += blockDim.x) {
    const int r = e / nx, j = e - r * nx;
    const int pos = r * nx + bitrev(j, Lx);
    const long long off = rbase + e;
    const long long row = off / nx;
    const int iy = (int)(row % ny), iz = (int)(row / ny);
    const double x = -A.g.L[0] + j * A.g.h[0];
    const double V = trap_value(A.trap, A.g, j, iy, iz, off);
    C u[3];  // Phi for ROW_INV_H, P for ROW_INV_P / ROW_INV_LIN
    double lin_r[3], lin_i[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      u[c] = A.in2[sbase + c * npts + off];
      C t = buf0[c * per + pos];
      C gg = buf1[c * per + pos];
      lin_r[c] = ((double)t.x - Om * x * (double)gg.x) * inv_n + V * (double)u[c].x;
      lin_i[c] = ((double)t.y - Om * x * (double)gg.y) * inv_n + V * (double)u[c].y;
    }
    if (MODE == ROW_INV_LIN) {
#pragma unroll
      for (int c = 0; c < 3; ++c) A.out0[sbase + c * npts + off] = mk<C>(lin_r[c], lin_i[c]);
      continue;
    }
    if (MODE == ROW_INV_H) {
      // nonlinear terms of Eqs. eigen1-eigen3: c0 rho phi + c1 (F.f) Phi
      double m[3];
      double rho = 0.0;
#pragma unroll
      for (int c = 0; c < 3; ++c) { m[c] = (double)u[c].x * u[c].x + (double)u[c].y * u[c].y; rho += m[c]; }
      const double2 a = spin_a(u[0], u[1], u[2]);
      const double Fz = m[0] - m[2];
      // (F.f)Phi: [Fz p1 + a p0, conj(a) p1 + a pm, conj(a) p0 - Fz pm]
      double fr[3], fi[3];
      fr[0] = Fz * u[0].x + (a.x * u[1].x - a.y * u[1].y);
      fi[0] = Fz * u[0].y + (a.x * u[1].y + a.y * u[1].x);
      fr[1] = (a.x * u[0].x + a.y * u[0].y) + (a.x * u[2].x - a.y * u[2].y);
      fi[1] = (a.x * u[0].y - a.y * u[0].x) + (a.x * u[2].y + a.y * u[2].x);
      fr[2] = (a.x * u[1].x + a.y * u[1].y) - Fz * u[2].x;
      fi[2] = (a.x * u[1].y - a.y * u[1].x) - Fz * u[2].y;
      double q = 0.0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        q += (double)u[c].x * lin_r[c] + (double)u[c].y * lin_i[c];
        const double hr = lin_r[c] + c0 * rho * u[c].x + c1 * fr[c];
        const double hi = lin_i[c] + c0 * rho * u[c].y + c1 * fi[c];
        A.out0[sbase + c * npts + off] = mk<C>(hr, hi);
        acc[3 + c] += V * m[c];
        acc[6 + c] += rho * m[c];
        acc[9 + c] += m[c];
      }
      acc[0] += q;
      acc[1] += rho * rho;
      acc[2] += 2.0 * (a.x * a.x + a.y * a.y) + Fz * Fz;
    } else {  // ROW_INV_P: step-model reductions
      C f[3], h[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) { f[c] = A.in3[sbase + c * npts + off]; h[c] = A.in4[sbase + c * npts + off]; }
      double hpp = 0.0, hphip = 0.0, R = 0.0, rf = 0.0, rp = 0.0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        hpp += lin_r[c] * u[c].x + lin_i[c] * u[c].y;
        hphip += (double)h[c].x * u[c].x + (double)h[c].y * u[c].y;
        R += (double)f[c].x * u[c].x + (double)f[c].y * u[c].y;
        rf += (double)f[c].x * f[c].x + (double)f[c].y * f[c].y;
        rp += (double)u[c].x * u[c].x + (double)u[c].y * u[c].y;
      }
      // spin vectors: F(Phi), F(P) and the symmetric cross term Re F~(Phi, P)
      const double2 aF = spin_a(f[0], f[1], f[2]);
      const double2 aP = spin_a(u[0], u[1], u[2]);
      const double s2 = 1.4142135623730951;
      const double FFx = s2 * aF.x, FFy = -s2 * aF.y;
      const double FFz = ((double)f[0].x * f[0].x + (double)f[0].y * f[0].y) - ((double)f[2].x * f[2].x + (double)f[2].y * f[2].y);
      const double FPx = s2 * aP.x, FPy = -s2 * aP.y;
      const double FPz = ((double)u[0].x * u[0].x + (double)u[0].y * u[0].y) - ((double)u[2].x * u[2].x + (double)u[2].y * u[2].y);
      // cross: Re(P^dag f_alpha Phi) = 1/2 d/de F_alpha(Phi + e P): a(Phi,P) + a(P,Phi) pieces
      const double2 aX1 = spin_a(make_double2(f[0].x, f[0].y), make_double2(u[1].x, u[1].y), make_double2(f[2].x, f[2].y));
      const double2 aX2 = spin_a(make_double2(u[0].x, u[0].y), make_double2(f[1].x, f[1].y), make_double2(u[2].x, u[2].y));
      // a(Phi+eP) = a(Phi) + e (aX1 + aX2) + e^2 a(P): cross coefficient is (aX1 + aX2)
      const double FXx = 0.5 * s2 * (aX1.x + aX2.x), FXy = -0.5 * s2 * (aX1.y + aX2.y);
      const double FXz = ((double)f[0].x * u[0].x + (double)f[0].y * u[0].y) - ((double)f[2].x * u[2].x + (double)f[2].y * u[2].y);
      acc[0] += hpp;
      acc[1] += hphip;
      acc[2] += R;
      acc[3] += rf * R;
      acc[4] += rf * rp;
      acc[5] += R * R;
      acc[6] += R * rp;
      acc[7] += rp * rp;
      acc[8] += FFx * FXx + FFy * FXy + FFz * FXz;
      acc[9] += FFx * FPx + FFy * FPy + FFz * FPz;
      acc[10] += FXx * FXx + FXy * FXy + FXz * FXz;
      acc[11] += FXx * FPx + FXy * FPy + FXz * FPz;
      acc[12] += FPx * FPx + FPy * FPy + FPz * FPz;
    }
  }
  if (MODE == ROW_INV_LIN) return;
  const bool mx[13] = {false, false, false, false, false, false, false, false, false, false, false, false, false};
  block_reduce<13>(acc, red, mx);
  if (threadIdx.x == 0) {
    double* P = A.part + (long long)s * NSLOT * A.pmax + rb;
    if (MODE == ROW_INV_H) {
      const int slots[12] = {SL_Q, SL_RHO2, SL_F2, SL_V0, SL_V1, SL_V2, SL_C0, SL_C1, SL_C2, SL_M0, SL_M1, SL_M2};
      for (int k = 0; k < 12; ++k) P[(long long)slots[k] * A.pmax] = acc[k];
    } else {
      const int slots[13] = {SL_HPP, SL_HPHIP, SL_RPHI, SL_IFR, SL_IFP, SL_IRR, SL_IRP, SL_IPP,
                             SL_JFR, SL_JFP, SL_JRR, SL_JRP, SL_JPP};
      for (int k = 0; k < 13; ++k) P[(long long)slots[k] * A.pmax] = acc[k];
    }
  }
}

// ============================================================== column passes (y or z axis)
// Tile: inner indices [i0, i0 + TC) of the axis-`axis` lines at outer index o.
// Shared layout of one component: [axis position][TC].
template <class T, int MODE>
__global__ void __launch_bounds__(kThreads) k_col(ChainArgs<T> A, int axis, int TC) {
  using C = cx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int na = A.g.n[axis], La = A.g.log2n[axis];
  const long long npts = A.g.npts;
  const int ni = (axis == 1) ? A.g.n[0] : A.g.n[0] * A.g.n[1];   // inner (faster) extent
  const int no = (int)(npts / ((long long)na * ni));             // outer (slower) extent
  const int tpo = ni / TC;                                       // tiles per outer index
  const int bps = tpo * no;
  const int s = blockIdx.x / bps;
  const int tb = blockIdx.x % bps;
  if (s >= A.nsolve || !gate_ok(A.st, A.gate, s)) return;
  const int o = tb / tpo;
  const int i0 = (tb % tpo) * TC;
  C* s_tw = (C*)smem_raw;
  C* buf = s_tw + (na >> 1);
  const int per = na * TC;
  C* buf2 = buf + 3 * per;            // second 3-component buffer (YINV_H) or 1-component temp (YMID_H)
  double* red = (double*)(buf2 + 3 * per);
  load_tw<T>(s_tw, A.tw[axis], na);
  const long long sbase = (long long)s * 3 * npts;
  const long long obase = (long long)o * na * ni + i0;
  const SolveState& S = A.st[s];
  const PhysDev ph = A.phys[s];
  const double Lax = A.g.L[axis];
  const int nx = A.g.n[0];

  // load in0 tile: bit-reversed positions for forward (DIT) modes, natural for inverse (DIF)
  const bool fwd_first = (MODE != COL_INV && MODE != COL_YINV_H);
  for (int e = threadIdx.x; e < per; e += blockDim.x) {
    const int j = e / TC, t = e - j * TC;
    const int pj = fwd_first ? bitrev(j, La) : j;
#pragma unroll
    for (int c = 0; c < 3; ++c) buf[c * per + pj * TC + t] = A.in0[sbase + c * npts + obase + (long long)j * ni + t];
  }
  if (MODE == COL_YINV_H) {
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int j = e / TC, t = e - j * TC;
      const int pj = bitrev(j, La);
#pragma unroll
      for (int c = 0; c < 3; ++c) buf2[c * per + pj * TC + t] = A.in1[sbase + c * npts + obase + (long long)j * ni + t];
    }
  }
  __syncthreads();

  if (MODE == COL_FWD) {
    fft_dit<C, true>(buf, La, 3 * TC, TC, per, 1, TC, s_tw, false);
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int j = e / TC, t = e - j * TC;
#pragma unroll
      for (int c = 0; c < 3; ++c) A.out0[sbase + c * npts + obase + (long long)j * ni + t] = buf[c * per + j * TC + t];
    }
    return;
  }
  if (MODE == COL_INV) {
    fft_dif<C, true>(buf, La, 3 * TC, TC, per, 1, TC, s_tw, true);
    const double sc = A.scale;
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int j = e / TC, t = e - j * TC;
      const int pj = bitrev(j, La);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        C v = buf[c * per + pj * TC + t];
        A.out0[sbase + c * npts + obase + (long long)j * ni + t] = mk<C>((double)v.x * sc, (double)v.y * sc);
      }
    }
    return;
  }

  // inner index -> (kx [, ky]) wavenumbers (inputs are spectral along the faster axes)
  auto kinner = [&](int t, double& kx, double& ky) {
    const int ii = i0 + t;
    if (axis == 1) { kx = wavenum(ii, nx, A.g.L[0]); ky = 0.0; }
    else { kx = wavenum(ii % nx, nx, A.g.L[0]); ky = wavenum(ii / nx, A.g.n[1], A.g.L[1]); }
  };

  if (MODE == COL_YINV_H) {
    // buf: C (natural) -> DIF inverse -> bit-reversed F_y^-1 C
    // buf2: A (bit-reversed) -> DIT forward -> natural F_y A; multiply by v_y; DIF inverse -> G
    fft_dif<C, true>(buf, La, 3 * TC, TC, per, 1, TC, s_tw, true);
    fft_dit<C, true>(buf2, La, 3 * TC, TC, per, 1, TC, s_tw, false);
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int j = e / TC;
      const double vy = wavenum(j, na, Lax);
#pragma unroll
      for (int c = 0; c < 3; ++c) buf2[c * per + e] = cscale(buf2[c * per + e], (T)vy);
    }
    __syncthreads();
    fft_dif<C, true>(buf2, La, 3 * TC, TC, per, 1, TC, s_tw, true);
    const double nfac = (double)A.g.n[1] * A.g.n[2];  // ny * nz
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int j = e / TC, t = e - j * TC;
      const int pj = bitrev(j, La);
      double kx, ky;
      kinner(t, kx, ky);
      const double y = -A.g.L[1] + j * A.g.h[1];
      const double rot = nfac * ph.Omega * y * kx;
      const long long gi = sbase + obase + (long long)j * ni + t;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        C a = A.in1[gi + c * npts];
        C cv = buf[c * per + pj * TC + t];
        A.out0[gi + c * npts] = mk<C>((double)cv.x + rot * a.x, (double)cv.y + rot * a.y);
        C gv = buf2[c * per + pj * TC + t];
        A.out1[gi + c * npts] = mk<C>((double)gv.x * A.g.n[2], (double)gv.y * A.g.n[2]);
      }
    }
    return;
  }

  // forward transform along the axis: natural-order spectrum in buf
  fft_dit<C, true>(buf, La, 3 * TC, TC, per, 1, TC, s_tw, false);

  if (MODE == COL_YMID_H) {
    // G_c = F_y^-1[v_y F_y A_c], one component at a time through buf2 (1 component)
    for (int c = 0; c < 3; ++c) {
      for (int e = threadIdx.x; e < per; e += blockDim.x) {
        const int j = e / TC;
        buf2[e] = cscale(buf[c * per + e], (T)wavenum(j, na, Lax));
      }
      __syncthreads();
      fft_dif<C, true>(buf2, La, TC, TC, 0, 1, TC, s_tw, true);
      for (int e = threadIdx.x; e < per; e += blockDim.x) {
        const int j = e / TC, t = e - j * TC;
        A.out1[sbase + c * npts + obase + (long long)j * ni + t] = buf2[bitrev(j, La) * TC + t];
      }
      __syncthreads();
    }
  }

  double acc[3] = {0.0, 0.0, 0.0};
  // pointwise in k: the kinetic + SOC symbol (H chains) or the kinetic preconditioner
  for (int e = threadIdx.x; e < per; e += blockDim.x) {
    const int j = e / TC, t = e - j * TC;
    double kx, ky, kz = 0.0;
    kinner(t, kx, ky);
    if (axis == 1) ky = wavenum(j, na, Lax);
    else kz = wavenum(j, na, Lax);
    const double k2h = 0.5 * (kx * kx + ky * ky + kz * kz);
    if (MODE == COL_MID_PRE) {
#pragma unroll
      for (int c = 0; c < 3; ++c) buf[c * per + e] = cscale(buf[c * per + e], (T)(1.0 / (S.alpha[c] + k2h)));
    } else {
      C p1 = buf[e], p0 = buf[per + e], pm = buf[2 * per + e];
      // kinetic per component (Parseval): sum 1/2 |k|^2 |phat_l|^2
      acc[0] += k2h * ((double)p1.x * p1.x + (double)p1.y * p1.y);
      acc[1] += k2h * ((double)p0.x * p0.x + (double)p0.y * p0.y);
      acc[2] += k2h * ((double)pm.x * pm.x + (double)pm.y * pm.y);
      // -gamma S symbol: s0 = -kx + i ky (L0), s1 = -(kx + i ky) (L1)
      // out_1 = K p1 - g s0 p0 ; out_0 = K p0 - g (s1 p1 + s0 pm) ; out_-1 = K pm - g s1 p0
      const double g = ph.gamma;
      const double s0r = -kx, s0i = ky, s1r = -kx, s1i = -ky;
      auto mul = [](double ar, double ai, C b, double& rr, double& ri) {
        rr = ar * b.x - ai * b.y; ri = ar * b.y + ai * b.x;
      };
      double ar, ai, br, bi;
      mul(s0r, s0i, p0, ar, ai);
      const C o1 = mk<C>(k2h * p1.x - g * ar, k2h * p1.y - g * ai);
      mul(s1r, s1i, p1, ar, ai);
      mul(s0r, s0i, pm, br, bi);
      const C o0 = mk<C>(k2h * p0.x - g * (ar + br), k2h * p0.y - g * (ai + bi));
      mul(s1r, s1i, p0, ar, ai);
      const C om = mk<C>(k2h * pm.x - g * ar, k2h * pm.y - g * ai);
      buf[e] = o1; buf[per + e] = o0; buf[2 * per + e] = om;
    }
  }
  __syncthreads();
  fft_dif<C, true>(buf, La, 3 * TC, TC, per, 1, TC, s_tw, true);

  const double nrot = (double)A.g.n[1];  // 2D: T' = F_y^-1[M F_y A] + ny Omega y v_x A
  for (int e = threadIdx.x; e < per; e += blockDim.x) {
    const int j = e / TC, t = e - j * TC;
    const int pj = bitrev(j, La);
    const long long gi = sbase + obase + (long long)j * ni + t;
    if (MODE == COL_YMID_H) {
      double kx, ky;
      kinner(t, kx, ky);
      const double y = -A.g.L[1] + j * A.g.h[1];
      const double rot = nrot * ph.Omega * y * kx;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        C a = A.in0[gi + c * npts];
        C v = buf[c * per + pj * TC + t];
        A.out0[gi + c * npts] = mk<C>((double)v.x + rot * a.x, (double)v.y + rot * a.y);
      }
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) A.out0[gi + c * npts] = buf[c * per + pj * TC + t];
    }
  }
  if (MODE == COL_MID_H || MODE == COL_YMID_H) {
    const bool mx[3] = {false, false, false};
    block_reduce<3>(acc, red, mx);
    if (threadIdx.x == 0) {
      double* P = A.part + (long long)s * NSLOT * A.pmax + tb;
      P[(long long)SL_KIN0 * A.pmax] = acc[0];
      P[(long long)SL_KIN1 * A.pmax] = acc[1];
      P[(long long)SL_KIN2 * A.pmax] = acc[2];
    }
  }
}

// ============================================================== launch helpers
template <class T>
int row_rows_per_block(const Geo& g) {
  const int nx = g.n[0];
  const int rows = (int)(g.npts / nx);
  int R = 512 / nx;
  if (R < 1) R = 1;
  if (R > rows) R = rows;
  return R;
}

template <class T>
int col_tc(const Geo& g, int axis) {
  const int na = g.n[axis];
  const int ni = (axis == 1) ? g.n[0] : g.n[0] * g.n[1];
  const int target = (sizeof(T) == 8) ? 1024 : 2048;   // elements of one component per tile
  int tc = target / na;
  if (tc < 1) tc = 1;
  if (tc > ni) tc = ni;
  return tc;
}

template <class T>
int row_blocks_per_solve(const Geo& g, const Launch&) {
  return (int)(g.npts / g.n[0]) / row_rows_per_block<T>(g);
}

template <class T>
int col_blocks_per_solve(const Geo& g, int axis, const Launch&) {
  const int na = g.n[axis];
  const int ni = (axis == 1) ? g.n[0] : g.n[0] * g.n[1];
  const int no = (int)(g.npts / ((long long)na * ni));
  return (ni / col_tc<T>(g, axis)) * no;
}

template <class T>
static size_t row_smem(const Geo& g, int mode) {
  using C = cx_t<T>;
  const int R = row_rows_per_block<T>(g);
  const int per = R * g.n[0];
  const bool two = (mode == ROW_INV_H || mode == ROW_INV_P || mode == ROW_INV_LIN);
  return sizeof(C) * ((g.n[0] >> 1) + 3 * per * (two ? 2 : 1)) + 32 * 13 * sizeof(double);
}

template <class T>
static size_t col_smem(const Geo& g, int axis) {
  using C = cx_t<T>;
  const int per = g.n[axis] * col_tc<T>(g, axis);
  return sizeof(C) * ((g.n[axis] >> 1) + 6 * per) + 32 * 3 * sizeof(double);
}

template <class T, int MODE>
static void row_go(const ChainArgs<T>& a, cudaStream_t st) {
  const int R = row_rows_per_block<T>(a.g);
  const int nb = row_blocks_per_solve<T>(a.g, Launch{}) * a.nsolve;
  const size_t sm = row_smem<T>(a.g, MODE);
  k_row<T, MODE><<<nb, kThreads, sm, st>>>(a, R);
}

template <class T>
void launch_row(int mode, const ChainArgs<T>& a, int, const Launch&, cudaStream_t st) {
  switch (mode) {
    case ROW_FWD_PLAIN: row_go<T, ROW_FWD_PLAIN>(a, st); break;
    case ROW_FWD_PROJ: row_go<T, ROW_FWD_PROJ>(a, st); break;
    case ROW_FWD_PRE: row_go<T, ROW_FWD_PRE>(a, st); break;
    case ROW_INV_H: row_go<T, ROW_INV_H>(a, st); break;
    case ROW_INV_P: row_go<T, ROW_INV_P>(a, st); break;
    case ROW_INV_PRE: row_go<T, ROW_INV_PRE>(a, st); break;
    case ROW_INV_PLAIN: row_go<T, ROW_INV_PLAIN>(a, st); break;
    case ROW_INV_LIN: row_go<T, ROW_INV_LIN>(a, st); break;
  }
}

template <class T, int MODE>
static void col_go(int axis, const ChainArgs<T>& a, cudaStream_t st) {
  const int tc = col_tc<T>(a.g, axis);
  const int nb = col_blocks_per_solve<T>(a.g, axis, Launch{}) * a.nsolve;
  const size_t sm = col_smem<T>(a.g, axis);
  k_col<T, MODE><<<nb, kThreads, sm, st>>>(a, axis, tc);
}

template <class T>
void launch_col(int mode, int axis, const ChainArgs<T>& a, const Launch&, cudaStream_t st) {
  switch (mode) {
    case COL_FWD: col_go<T, COL_FWD>(axis, a, st); break;
    case COL_INV: col_go<T, COL_INV>(axis, a, st); break;
    case COL_MID_H: col_go<T, COL_MID_H>(axis, a, st); break;
    case COL_MID_PRE: col_go<T, COL_MID_PRE>(axis, a, st); break;
    case COL_YMID_H: col_go<T, COL_YMID_H>(axis, a, st); break;
    case COL_YINV_H: col_go<T, COL_YINV_H>(axis, a, st); break;
  }
}

template <class T>
cudaError_t chain_prepare() {
  const int big = 200 * 1024;
  cudaError_t e = cudaSuccess;
#define GPSOC_ATTR(K) \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  GPSOC_ATTR((k_row<T, ROW_FWD_PLAIN>)) GPSOC_ATTR((k_row<T, ROW_FWD_PROJ>)) GPSOC_ATTR((k_row<T, ROW_FWD_PRE>))
  GPSOC_ATTR((k_row<T, ROW_INV_H>)) GPSOC_ATTR((k_row<T, ROW_INV_P>)) GPSOC_ATTR((k_row<T, ROW_INV_PRE>))
  GPSOC_ATTR((k_row<T, ROW_INV_PLAIN>)) GPSOC_ATTR((k_row<T, ROW_INV_LIN>))
  GPSOC_ATTR((k_col<T, COL_FWD>)) GPSOC_ATTR((k_col<T, COL_INV>)) GPSOC_ATTR((k_col<T, COL_MID_H>))
  GPSOC_ATTR((k_col<T, COL_MID_PRE>)) GPSOC_ATTR((k_col<T, COL_YMID_H>)) GPSOC_ATTR((k_col<T, COL_YINV_H>))
#undef GPSOC_ATTR
  return e;
}

template void launch_row<double>(int, const ChainArgs<double>&, int, const Launch&, cudaStream_t);
template void launch_row<float>(int, const ChainArgs<float>&, int, const Launch&, cudaStream_t);
template void launch_col<double>(int, int, const ChainArgs<double>&, const Launch&, cudaStream_t);
template void launch_col<float>(int, int, const ChainArgs<float>&, const Launch&, cudaStream_t);
template int row_blocks_per_solve<double>(const Geo&, const Launch&);
template int row_blocks_per_solve<float>(const Geo&, const Launch&);
template int col_blocks_per_solve<double>(const Geo&, int, const Launch&);
template int col_blocks_per_solve<float>(const Geo&, int, const Launch&);
template cudaError_t chain_prepare<double>();
template cudaError_t chain_prepare<float>();

}  // namespace gpsoc
