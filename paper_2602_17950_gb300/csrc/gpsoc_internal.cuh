// Internal declarations shared by the CUDA translation units of libgpsoc.
//
// Data layout in device memory (one "3-array"): [solve][component][z][y][x],
// x fastest, complex values interleaved (double2 or float2).  Component index
// 0, 1, 2 holds phi_1, phi_0, phi_-1.
//
// Spectral conventions (Section 3.2 of arXiv 2602.17950): forward DFT along an
// axis is unnormalised, exp(-2 pi i k m / n); coefficient index k stands for
// p = k (k < n/2) or k - n (k >= n/2); wavenumber v = pi p / L.  The Nyquist
// index k = n/2 keeps v = -pi n / (2L) in every symbol, odd ones included.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include "../../include/gpsoc.h"
#include "dword.cuh"

namespace gpsoc {

// ------------------------------------------------------------------ complex helpers
template <class T> struct Cx;
template <> struct Cx<double> { using type = double2; };
template <> struct Cx<float> { using type = float2; };
template <class T> using cx_t = typename Cx<T>::type;

// build a complex of the array type from values of any real type (no detour
// through double: conversions run on the scarce FP64 pipe)
template <class C, class A, class B> __host__ __device__ __forceinline__ C mk(A re, B im) {
  C c; c.x = (decltype(c.x))re; c.y = (decltype(c.y))im; return c;
}
template <class C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <class C> __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <class C> __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <class C, class S> __device__ __forceinline__ C cscale(C a, S s) { a.x *= s; a.y *= s; return a; }

// ------------------------------------------------------------------ geometry and parameters
struct Geo {
  int d;            // 2 or 3
  int n[3];         // nx, ny, nz (nz = 1 in 2D)
  int log2n[3];
  double L[3], h[3];
  double piL[3];    // pi / L per axis: wavenumber of index k is p * piL with p = k or k - n
  long long npts;   // points of one component
  double dV;        // h^d
  float fL[3], fh[3], fpiL[3];   // FP32 copies for FP32 kernels (no per-thread FP64 conversions)
};

struct TrapDev {
  double half_g2[3];   // g_i^2 / 2
  double quad, quart;
  const double* userV; // npts doubles of the current level or nullptr
  float fhalf_g2[3], fquad, fquart;   // FP32 copies
};

struct PhysDev {
  double Omega, gamma, c0, c1;
  float fOmega, fgamma, fc0, fc1;    // FP32 copies
  float c0lo, c1lo;                  // c0 - fc0, c1 - fc1: the double-word interaction constants
};

__host__ __device__ inline PhysDev make_phys(double Omega, double gamma, double c0, double c1) {
  PhysDev p;
  p.Omega = Omega; p.gamma = gamma; p.c0 = c0; p.c1 = c1;
  p.fOmega = (float)Omega; p.fgamma = (float)gamma; p.fc0 = (float)c0; p.fc1 = (float)c1;
  p.c0lo = (float)(c0 - (double)p.fc0);
  p.c1lo = (float)(c1 - (double)p.fc1);
  return p;
}

// the copy of a scalar in the working precision W: FP32 kernels read the FP32
// copy (an FP64-to-FP32 conversion issues on the FP64 pipe, 1/64 of the FP32 rate)
template <class W> __device__ __forceinline__ W pick(double d, float f) {
  if constexpr (sizeof(W) == 4) return f; else return d;
}

// Per-solve scalar state of the PCG iteration (device resident).
struct SolveState {
  int active;       // iterating
  int status;       // gpsoc_status
  int iters;        // accepted steps on this level
  int total_iters;
  int first;        // next iteration starts with beta = 0
  int reset;        // Algorithm 2 Step 2 asked for beta = 0 in this iteration
  int beta_resets, halvings;
  int fp32_iters, fp64_iters;
  int pending;      // an accepted step waits to be applied by the next iteration's first pass
  int it_win;       // FP32 phase: iteration at which the current stall window opened
  int last_par;     // buffer parity (0/1) of the iteration whose step was accepted last
  int upd_applied;  // the opening pass of this iteration applied the step accepted before it
  // observables of the current iterate
  double E, mu, Q;          // energy, chemical potential, <H_lin Phi, Phi>
  double rho2, F2;          // sum rho^2, sum |F|^2 (times dV)
  double alpha[3], mass[3];
  double res_inf, dphi_inf;
  // PCG scalars
  double s_prev, s_cur, beta, cproj;
  double P2, HPP, HPhiP, RPhi;
  double I[6], J[6];
  double a, b, theta, dE, dE_last;
  double upd_c, upd_s, upd_scale;
  double E_win;     // FP32 phase: energy when the stall window opened
  double kin[3];    // GPSOC_HYBRID: per-component kinetic sums of the last exact recomputation of H_lin Phi
  double acorr;     // radial part Re<P, Phi>/||Phi||^2 removed from the last direction (tangent correction)
  // FP32 copies of the scalars the array passes read (refreshed by mirror32)
  float fmu, fbeta, fcproj, fupd_c, fupd_s, fupd_scale, falpha[3], fpad;
  // GPSOC_HYBRID: the accepted step as double words (hi, lo): uc = g c, ut = g t and uc - 1
  float dw_uc[2], dw_ut[2], dw_ucm1[2];
};

__device__ __forceinline__ void mirror32(SolveState& S) {
  S.fmu = (float)S.mu; S.fbeta = (float)S.beta; S.fcproj = (float)S.cproj;
  S.fupd_c = (float)S.upd_c; S.fupd_s = (float)S.upd_s; S.fupd_scale = (float)S.upd_scale;
  for (int c = 0; c < 3; ++c) S.falpha[c] = (float)S.alpha[c];
}

struct OptsDev {
  int stop;
  double tol, res_tol;
  int max_iter;
  double theta_trial, sigma;
  int max_halvings;
  int no_stop;      // gpsoc_iterate: run without stopping tests
  int phase32;      // FP32 phase of a mixed solve: stagnation / iteration cap end the phase, not the solve
  double tol_rel;   // energy stop: |dE| < tol + tol_rel * |E|
  int precond;      // GPSOC_PRECOND_*
  double res32;     // FP32 phase: ends (or never starts) once max |r| < res32 (0 = no residual rule)
  int line_search;  // 0: Algorithm 2's quadratic model; 1: the minimiser of Eq. theta
};

// reduction slots (per solve); partial sums live in part[(s * NSLOT + slot) * pmax + block]
enum Slot {
  SL_KIN0 = 0, SL_KIN1, SL_KIN2,                 // sum 1/2 |k|^2 |phat_l|^2
  SL_Q, SL_RHO2, SL_F2,                           // <H_lin phi, phi>, sum rho^2, sum |F|^2
  SL_V0, SL_V1, SL_V2, SL_C0, SL_C1, SL_C2,       // sum V|phi_l|^2, sum rho |phi_l|^2
  SL_M0, SL_M1, SL_M2,                            // masses
  SL_RINF,                                        // max |r|
  SL_RZ, SL_RPZ,                                  // Re<r, z>, Re<r_prev, z>
  SL_P2,                                          // ||P||^2
  SL_HPP, SL_HPHIP, SL_RPHI,                      // <H_lin P,P>, Re<H Phi, P>, Re<P, Phi>
  SL_IFR, SL_IFP, SL_IRR, SL_IRP, SL_IPP,         // rho cross integrals
  SL_JFR, SL_JFP, SL_JRR, SL_JRP, SL_JPP,         // spin cross integrals
  SL_DPHIINF,                                     // max |Phi_new - Phi|^2
  SL_NORM,                                        // sum |phi|^2 for normalisation
  SL_ZPHI, SL_PPHI, SL_RP,                        // Re<z, Phi>, Re<P_prev, Phi>, Re<r, P_prev>
  SL_KPHI0, SL_KPHI1, SL_KPHI2,                   // GPSOC_HYBRID: sum 1/2 |k|^2 |Phi_hat_l|^2
  SL_KX0, SL_KX1, SL_KX2,                         //   and sum 1/2 |k|^2 Re(Phi_hat_l conj P_hat_l)
  NSLOT
};

// gate of a kernel: which per-solve flag must be set for the block to run
enum Gate { GATE_ALL = 0, GATE_ACTIVE = 1, GATE_RESET = 2, GATE_PENDING = 3 };

// what the scalar steps read: state, parameters, block partial sums and sizes
struct ScalarCtx {
  SolveState* st;
  const PhysDev* phys;
  const double* part;
  int pmax;
  int nb_row, nb_col;   // blocks per solve of the row passes and of the last column pass
  long long npts;
  double dV;
  OptsDev opts;
  int flags;            // 2 = count accepted steps as FP32 iterations; bit 2 = buffer parity of the iteration;
                        // 8 = GPSOC_HYBRID iteration (kinetic part of alpha from the state, residual-based
                        //     slopes: the H Phi slots hold Re<r, .> sums)
  double inv_npts;      // 1 / npts
  int part_dw;          // the sum partials it reads are double words (written by FP32 / hybrid passes)
};

template <class T>
struct ChainArgs {
  using C = cx_t<T>;
  Geo g;
  TrapDev trap;
  const PhysDev* phys;
  SolveState* st;
  const C* in0; const C* in1; const C* in2; const C* in3; const C* in4;
  C* out0; C* out1;
  double* part; int pmax;
  const C* tw[3];     // twiddle tables exp(-2 pi i k / n_axis), k < n_axis/2
  int gate;
  int nsolve;
  double scale;       // extra scale factor (prolongation, normalisation)
  int given_r;        // ROW_FWD_PRE: in0 already holds r (mu taken as 0)
  int fuse;           // the last block of the pass runs the scalar step that consumes its sums
  unsigned* cnt;      // per-solve block arrival counters (fused scalar steps)
  ScalarCtx sc;
  // GPSOC_HYBRID passes of an FP32 chain that also read the FP64 state
  const double2* phi64;   // Phi (FP64)
  const double2* hl64;    // H(Phi) (FP64), for ROW_FWD_PRE_HY
  // GPSOC_HYBRID, last column pass of the P chain: the spectrum of Phi (advanced by the
  // step applied this iteration when khat_upd is set) and of the previous P, both updated
  // in place, for the exact per-component kinetic sums of alpha
  C* xhat; C* phat;
  int khat_upd;
};

// Programmatic dependent launch.  The iteration's kernels are launched with programmatic
// stream serialisation (launch_pdl).  pdl_wait() waits until the kernel before it in the
// stream has completed and its writes are visible (griddepcontrol.wait); every read of
// data another kernel writes comes after it, only constant tables are read before.
// pdl_trigger() (griddepcontrol.launch_dependents) lets the next kernel's blocks be
// scheduled once every block has issued it or exited.  The passes with a fused scalar
// tail issue it when a block has written its partial sums (last_block), so the next
// kernel's blocks are placed on SMs this pass has left, and wait there while the last
// block runs the tail; the others trigger at exit.  Without the launch attribute (the
// default) the wait returns at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// launch with programmatic stream serialisation when GPSOC_PDL=1 is set in the environment
// (kernels that call pdl_wait before reading what earlier kernels wrote); by default the
// kernels run in plain stream order, which measured faster for this iteration's kernels
inline bool pdl_enabled() {
  static const bool on = [] {
    const char* e = getenv("GPSOC_PDL");
    return e && e[0] == '1';
  }();
  return on;
}

template <class... KArgs, class... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

__device__ __forceinline__ bool gate_ok(const SolveState* st, int gate, int s) {
  if (gate == GATE_ALL) return true;
  if (gate == GATE_ACTIVE) return st[s].active != 0;
  if (gate == GATE_PENDING) return st[s].active != 0 && st[s].pending != 0;
  return st[s].active != 0 && st[s].reset != 0;
}

// True in every thread of the block that arrives last among the `bps` blocks of
// solve s (threadfence-reduction pattern: partial sums written before the
// arrival are visible to the last block).  The last block resets the counter.
__device__ __forceinline__ bool last_block(unsigned* cnt, int s, int bps, int* flag_smem) {
  pdl_trigger();
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(cnt + s, 1u);
    *flag_smem = (prev == (unsigned)bps - 1u);
  }
  __syncthreads();
  const bool last = *flag_smem != 0;
  if (last) {
    __threadfence();
    if (threadIdx.x == 0) cnt[s] = 0u;
  }
  return last;
}

// wavenumber v_p = pi p / L of FFT index k on an axis of n points (Section 3.2),
// evaluated in the working precision W of the kernel
template <class W>
__device__ __forceinline__ W wavenum(int k, int n, W piL) {
  const int p = (k < (n >> 1)) ? k : k - n;
  return (W)p * piL;
}
template <class W> __device__ __forceinline__ W geo_piL(const Geo& g, int a) { return pick<W>(g.piL[a], g.fpiL[a]); }
// physical coordinate -L + i h of grid index i on axis a
template <class W> __device__ __forceinline__ W coord(const Geo& g, int a, int i) {
  return -pick<W>(g.L[a], g.fL[a]) + (W)i * pick<W>(g.h[a], g.fh[a]);
}

// trapping potential at grid point (ix, iy, iz) in the working precision W
template <class W>
__device__ __forceinline__ W trap_value(const TrapDev& t, const Geo& g, int ix, int iy, int iz, long long idx) {
  const W x = coord<W>(g, 0, ix);
  const W y = coord<W>(g, 1, iy);
  W v = pick<W>(t.half_g2[0], t.fhalf_g2[0]) * x * x + pick<W>(t.half_g2[1], t.fhalf_g2[1]) * y * y;
  W r2 = x * x + y * y;
  if (g.d == 3) {
    const W z = coord<W>(g, 2, iz);
    v += pick<W>(t.half_g2[2], t.fhalf_g2[2]) * z * z;
    r2 += z * z;
  }
  v += pick<W>(t.quad, t.fquad) * r2 + pick<W>(t.quart, t.fquart) * r2 * r2;
  if (t.userV) v += (W)t.userV[idx];
  return v;
}

// ------------------------------------------------------------------ block reductions (deterministic)
// FP64 block reductions in a fixed order.  FP64 issue slots are scarce on this
// part (about 1/64 of FP32), so a multi-value reduction does not run one
// shuffle tree per value (5 adds per lane per value).  With KP = K rounded up to
// a power of two, a warp first performs a reduce-scatter over the KP value slots
// -- at each halving step a lane keeps one half of its values and adds the
// partner lane's copy of that half -- so that every lane holds one slot
// (KP - 1 adds), then the 32/KP lanes holding the same slot are added in a
// fixed butterfly (log2(32/KP) adds), and the warps are added in index order.
// scratch: >= 16 * (blockDim.x / 32) + 16 doubles.  Every thread receives the K
// results in v.  is_max is honoured for K == 1 only (multi-value calls sum).
template <int K>
__device__ __forceinline__ void block_reduce(double (&v)[K], double* scratch, const bool (&is_max)[K]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();  // scratch may alias shared memory the caller used just before
  if (K == 1) {
    double x = v[0];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double o = __shfl_down_sync(0xffffffffu, x, off);
      x = is_max[0] ? fmax(x, o) : x + o;
    }
    if (lane == 0) scratch[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
      double acc = scratch[0];
      for (int w = 1; w < nw; ++w) acc = is_max[0] ? fmax(acc, scratch[w]) : acc + scratch[w];
      scratch[nw] = acc;
    }
    __syncthreads();
    v[0] = scratch[nw];
    return;
  }
  static_assert(K <= 16, "block_reduce handles at most 16 values");
  constexpr int KP = (K <= 2) ? 2 : (K <= 4) ? 4 : (K <= 8) ? 8 : 16;
  constexpr int LB = (KP == 2) ? 1 : (KP == 4) ? 2 : (KP == 8) ? 3 : 4;
  double x[KP];
#pragma unroll
  for (int k = 0; k < KP; ++k) x[k] = (k < K) ? v[k] : 0.0;
  // reduce-scatter over the low LB lane bits
#pragma unroll
  for (int st = 0; st < LB; ++st) {
    const int ofs = 1 << st, half = (KP / 2) >> st;
    const bool up = (lane & ofs) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const double keep = up ? x[i + half] : x[i];
      const double send = up ? x[i] : x[i + half];
      x[i] = keep + __shfl_xor_sync(0xffffffffu, send, ofs);
    }
  }
  // lanes equal in the low LB bits hold the same slot: add them
#pragma unroll
  for (int ofs = KP; ofs < 32; ofs <<= 1) x[0] += __shfl_xor_sync(0xffffffffu, x[0], ofs);
  // slot of lane l: its low LB bits reversed (bit 0 chose the highest half first)
  int slot = 0;
#pragma unroll
  for (int b = 0; b < LB; ++b) slot |= ((lane >> b) & 1) << (LB - 1 - b);
  if (lane < KP) scratch[warp * 16 + slot] = x[0];
  __syncthreads();
  double* res = scratch + 16 * nw;
  if (threadIdx.x < K) {
    double acc = scratch[threadIdx.x];
    for (int w = 1; w < nw; ++w) acc += scratch[w * 16 + threadIdx.x];
    res[threadIdx.x] = acc;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = res[k];
}

// Double-float ("FP32 pair") arithmetic for the reductions of FP32 kernels: a
// value is hi + lo with |lo| <= ulp(hi)/2, about 48 significant bits.  Sums use
// Knuth's TwoSum (an error-free transformation), so adding FP32 per-thread
// partials this way is as accurate as FP64 adds while issuing on the FP32 pipes.
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb);   // TwoSum: a.hi + b.hi = s + e exactly
  const float t = a.lo + b.lo + e;
  const float h = s + t;                             // FastTwoSum(s, t): |s| >= |t|
  DF r;
  r.hi = h;
  r.lo = t - (h - s);
  return r;
}
__device__ __forceinline__ DF df_shfl_xor(DF a, int ofs) {
  DF r;
  r.hi = __shfl_xor_sync(0xffffffffu, a.hi, ofs);
  r.lo = __shfl_xor_sync(0xffffffffu, a.lo, ofs);
  return r;
}

// One FP32 block total (a sum in double-float, or a max in FP32, which is exact),
// rounded to FP64 once.  scratch: >= blockDim.x / 32 + 1 doubles.
__device__ __forceinline__ double block_reduce1_f(float a, bool is_max, double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();  // scratch may alias shared memory the caller used just before
  DF x{a, 0.0f};
#pragma unroll
  for (int ofs = 16; ofs > 0; ofs >>= 1) {
    const DF o = df_shfl_xor(x, ofs);
    if (is_max) x.hi = fmaxf(x.hi, o.hi);
    else x = df_add(x, o);
  }
  float2* sc2 = reinterpret_cast<float2*>(scratch);
  if (lane == 0) sc2[warp] = make_float2(x.hi, is_max ? 0.0f : x.lo);
  __syncthreads();
  if (threadIdx.x == 0) {
    DF acc{sc2[0].x, sc2[0].y};
    for (int w = 1; w < nw; ++w) {
      if (is_max) acc.hi = fmaxf(acc.hi, sc2[w].x);
      else acc = df_add(acc, DF{sc2[w].x, sc2[w].y});
    }
    scratch[nw] = (double)acc.hi + (double)acc.lo;
  }
  __syncthreads();
  return scratch[nw];
}

// Block sums of double-float per-thread partials, same fixed order and same
// reduce-scatter scheme as block_reduce, with the accurate double-word sum; the K
// totals are rounded to FP64 once at the end.  scratch: >= 16 * (blockDim.x / 32) + 16
// doubles.
template <int K>
__device__ __forceinline__ void block_reduce_dw(const DF (&a)[K], double (&v)[K], double* scratch) {
  static_assert(K >= 2 && K <= 16, "block_reduce_dw handles 2..16 values");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();  // scratch may alias shared memory the caller used just before
  constexpr int KP = (K <= 2) ? 2 : (K <= 4) ? 4 : (K <= 8) ? 8 : 16;
  constexpr int LB = (KP == 2) ? 1 : (KP == 4) ? 2 : (KP == 8) ? 3 : 4;
  DF x[KP];
#pragma unroll
  for (int k = 0; k < KP; ++k) {
    x[k].hi = (k < K) ? a[k].hi : 0.0f;
    x[k].lo = (k < K) ? a[k].lo : 0.0f;
  }
#pragma unroll
  for (int st = 0; st < LB; ++st) {
    const int ofs = 1 << st, half = (KP / 2) >> st;
    const bool up = (lane & ofs) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const DF keep = up ? x[i + half] : x[i];
      const DF send = up ? x[i] : x[i + half];
      x[i] = dw_add(keep, df_shfl_xor(send, ofs));
    }
  }
#pragma unroll
  for (int ofs = KP; ofs < 32; ofs <<= 1) x[0] = dw_add(x[0], df_shfl_xor(x[0], ofs));
  int slot = 0;
#pragma unroll
  for (int b = 0; b < LB; ++b) slot |= ((lane >> b) & 1) << (LB - 1 - b);
  float2* sc2 = reinterpret_cast<float2*>(scratch);
  if (lane < KP) sc2[warp * 16 + slot] = make_float2(x[0].hi, x[0].lo);
  __syncthreads();
  double* res = scratch + 16 * nw;
  if (threadIdx.x < K) {
    const float2 f = sc2[threadIdx.x];
    DF acc{f.x, f.y};
    for (int w = 1; w < nw; ++w) {
      const float2 g = sc2[w * 16 + threadIdx.x];
      acc = dw_add(acc, DF{g.x, g.y});
    }
    res[threadIdx.x] = (double)acc.hi + (double)acc.lo;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = res[k];
}
// the same for FP32 per-thread partials
template <int K>
__device__ __forceinline__ void block_reduce_df(const float (&a)[K], double (&v)[K], double* scratch) {
  DF x[K];
#pragma unroll
  for (int k = 0; k < K; ++k) { x[k].hi = a[k]; x[k].lo = 0.0f; }
  block_reduce_dw<K>(x, v, scratch);
}

// Per-block partials in the part buffer.  The FP32 and hybrid passes store a sum as a
// double word (FP32 hi, lo packed into the 8-byte slot), so that the scalar tail adding
// a solve's partials works on the FP32 pipes (it runs on one SM, where every FP64 warp
// instruction costs 64 cycles of a sub-partition); the FP64 passes store FP64 sums, and
// every pass stores maxima as FP64.  The reading tail knows the format (part_dw).
__device__ __forceinline__ void put_partial(double* p, double v, bool is_max, bool dw) {
  if (is_max || !dw) {
    *p = v;
    return;
  }
  const float hi = __double2float_rn(v);
  *reinterpret_cast<float2*>(p) = make_float2(hi, __double2float_rn(v - (double)hi));
}
__device__ __forceinline__ DF get_sum_partial(const double* p) {
  const float2 w = __ldcg(reinterpret_cast<const float2*>(p));
  DF r;
  r.hi = w.x;
  r.lo = w.y;
  return r;
}
// threads k < K of the block store slot k of the block totals v (v and slots identical
// in every thread); the value is picked by selects so that the K conversions are one
// instruction of the first warp
template <int K>
__device__ __forceinline__ void put_partials(double* part, long long sbase_slot, int pmax, int blk,
                                             const int (&slots)[K], const double (&v)[K], const bool (&mx)[K],
                                             bool dw) {
  const int t = threadIdx.x;
  if (t >= K) return;
  double vk = v[0];
  int sk = slots[0];
  bool mk_ = mx[0];
#pragma unroll
  for (int k = 1; k < K; ++k) {
    vk = (t == k) ? v[k] : vk;
    sk = (t == k) ? slots[k] : sk;
    mk_ = (t == k) ? mx[k] : mk_;
  }
  put_partial(part + (sbase_slot + sk) * pmax + blk, vk, mk_, dw);
}

// ------------------------------------------------------------------ host-side launch helpers
struct Launch {
  int rows_per_block;   // row passes
  int cols_per_tile[3]; // column passes per axis
  int threads;
};

template <class T> struct Chain;  // kernels of one precision (defined in chain.cu)

// Launchers implemented in chain.cu (explicitly instantiated for double, float).
enum RowMode {
  ROW_FWD_PLAIN = 0,   // out0 = F_x(in0); with ROW_FWD_UPD first applies a pending step to in0 (= out1)
  ROW_FWD_PROJ,        // P = in0 - cproj * in1 -> out1; out0 = F_x(P); reduce ||P||^2
  ROW_FWD_PRE,         // r = in0 - mu in1 -> out1; out0 = F_x(s * r); reduce max|r|
  ROW_INV_H,           // out0 = H(Phi) from T' (in0), G (in1), Phi (in2); energy reductions
  ROW_INV_P,           // reductions of the step model from T' (in0), G (in1), P (in2), Phi (in3), HPhi (in4)
  ROW_INV_PRE,         // z = s * F_x^-1(in0)/npts -> out0; reduce <r,z>, <r_prev,z>, <z,Phi>, <P_prev,Phi>,
                       // <r,P_prev> (in1 = Phi, in2 = r, in3 = r_prev, in4 = P_prev); fused beta and direction
  ROW_INV_PLAIN,       // out0 = scale * F_x^-1(in0)
  ROW_INV_LIN,         // out0 = H_lin(in2) from T' (in0), G (in1) (no reductions)
  ROW_FWD_UPD,         // Phi (in0, written back to out1) <- pending step with P (in2); out0 = F_x(Phi)
  ROW_FWD_PRE_HY,      // FP32 pass of GPSOC_HYBRID: r = H Phi - mu Phi in FP64 from phi64 and H(Phi)
                       // (hl64) -> out1 (FP32); out0 = F_x(P_V^{1/2} r); reduce max|r|
  ROW_INV_P_HY         // FP32 pass of GPSOC_HYBRID: as ROW_INV_P with in4 = r (slot HPHIP = Re<r, P>),
                       // out0 = H_lin P, and Re<P, Phi> summed in FP64 against phi64
};
enum ColMode {
  COL_FWD = 0,         // out0 = F_axis(in0)
  COL_INV,             // out0 = F_axis^-1(in0) (unnormalised)
  COL_MID_H,           // last axis, H chain: out0 = F^-1[M(k) F in0], reduce kinetic per component
  COL_MID_PRE,         // last axis, preconditioner: out0 = F^-1[F in0 / (alpha_l + |k|^2/2)]
  COL_YMID_H,          // 2D y pass of the H chain: out0 = T', out1 = G
  COL_YINV_H,          // 3D y inverse pass of the H chain: in0 = C, in1 = A -> out0 = T', out1 = G
  COL_MID_KIN          // last axis: reduce kinetic per component only (no output)
};

template <class T>
void launch_row(int mode, const ChainArgs<T>& a, int nblocks_total, const Launch& lc, cudaStream_t s);
template <class T>
void launch_col(int mode, int axis, const ChainArgs<T>& a, const Launch& lc, cudaStream_t s);
// blocks per solve of the row passes / column passes for a launch over nsolve solves
template <class T>
int row_blocks_per_solve(const Geo& g, int nsolve);
template <class T>
int col_blocks_per_solve(const Geo& g, int axis, int nsolve);
template <class T>
cudaError_t chain_prepare();   // sets max dynamic shared memory attributes
// tile of the axis passes: lines per tile (rows R for axis 0, columns TC otherwise),
// FFT elements per thread and threads per block, for a launch over nsolve solves
template <class T>
void tile_shape(const Geo& g, int axis, int nsolve, int& lines, int& ept, int& threads);
// tuned tiles: set (lines = 0 clears) and the list of valid candidates of an axis
template <class T>
bool tile_set(const Geo& g, int nsolve, int axis, int lines, int ept);
template <class T>
int tile_candidates(const Geo& g, int axis, int* lines, int* ept, int cap);

}  // namespace gpsoc
