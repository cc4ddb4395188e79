// Argument blocks and launchers of the scalar and elementwise kernels (pcg.cu).
#pragma once

#include "gpsoc_internal.cuh"

namespace gpsoc {

enum Phase {
  PH_INIT = 0,      // reset per-level flags (flags & 1: also reset counters)
  PH_OBS,           // E, mu, alpha, masses from the H-chain partials
  PH_RES,           // max |r| and the stopping test
  PH_BETA,          // Polak-Ribiere+ beta, Re<D, Phi> and the beta = 0 decision of Algorithm 2 Step 2
  PH_STEP,          // Algorithm 2 (step model, backtracking, update coefficients)
  PH_CLEAR,         // drop the pending-step flag
  PH_NORM,          // 1/sqrt(mass) per solve into norm_scale
  PH_MODEL,         // a_n, b_n and E(theta) - E(0) at given angles into model_out
  PH_KIN            // per-component kinetic sums of the last column pass into the state (GPSOC_HYBRID)
};

struct ScalarArgs {
  SolveState* st;
  const PhysDev* phys;
  const double* part;
  int pmax;
  int nb_row, nb_col;
  int nsolve;
  int phase;
  int flags;          // PH_INIT: 1 = reset counters, 4 = keep the direction; PH_STEP: 2 = count as an FP32 iteration
  long long npts;
  double dV;
  OptsDev opts;
  double* norm_scale;
  int force;          // process every solve regardless of its active flag
  const double* thetas; int n_theta; double* model_out;
  int only = -1;      // >= 0: act on this solve only (per-slot operations of the server)
  double inv_npts = 0.0;   // 1 / npts
  int part_dw = 0;    // the sum partials it reads are double words (FP32 passes wrote them)
};

enum ElemMode { EL_UPDATE = 0, EL_MASS, EL_SCALE };

template <class T>
struct ElemArgs {
  using C = cx_t<T>;
  SolveState* st;
  const C* in0; const C* in1; const C* in2; const C* in3;
  C* out0;
  double* part; int pmax;
  const double* scalev;
  long long npts;
  int bps;            // blocks per solve (divides npts)
  int nsolve;
  int gate;
  int only = -1;      // >= 0: act on this solve only (per-slot operations of the server)
};

// GPSOC_HYBRID: the pass that opens an iteration (FP64 state, double-word arithmetic).
// HY_UPD applies the pending step Phi <- s (c Phi + t P) (P in FP32), HY_REC advances
// H_lin Phi by the same linear combination of H_lin Phi and H_lin P, HY_REDUCE forms the
// nonlinear terms and H(Phi), the per-block energy / mu / alpha / mass sums and the FP32
// copy of Phi.  The observables step that consumes the sums runs as its own kernel after
// it when fuse is set (HY in gpsoc.cu).
enum { HY_UPD = 1, HY_REC = 2, HY_REDUCE = 4 };
struct HyArgs {
  SolveState* st;
  const PhysDev* phys;
  double* part; int pmax;
  Geo g;
  TrapDev trap;
  double2* phi;          // Phi (FP64), updated in place
  double2* hl;           // H_lin Phi (FP64), updated in place
  const float2* p;       // the pending direction P (FP32)
  const float2* hlp;     // H_lin P (FP32)
  float2* phi32;         // FP32 copy of Phi for the FP32 passes
  double2* hphi;         // H(Phi) = H_lin Phi + nonlinear terms (FP64), written by HY_REDUCE
  long long npts;
  int bps, nsolve, gate, flags;
  int fuse;              // HY: run the observables step on the sums afterwards
  ScalarCtx sc;          // scalar context of that step
};
void launch_hy_upd(const HyArgs& a, cudaStream_t st);
// blocks per solve of k_hy_upd: whole waves of its resident blocks over nsm SMs, the
// points split evenly (to one) between the blocks
int hy_blocks_per_solve(const Geo& g, int nsolve, int nsm);

void launch_scalar(const ScalarArgs& a, cudaStream_t st);
template <class T> void launch_elem(int mode, const ElemArgs<T>& a, cudaStream_t st);
template <class T> void launch_pad(const cx_t<T>* in, cx_t<T>* out, const Geo& gc, const Geo& gf, int nsolve, cudaStream_t st);
template <class T> void launch_convert(const void* in, int in_fp32, cx_t<T>* out, long long count, cudaStream_t st);
void launch_handover(const float2* phi32, const float2* const* r32, const float2* const* p32, double2* phi64,
                     double2* r64_prev, double2* p64_prev, const SolveState* st, long long per_solve, int nsolve,
                     int carry, cudaStream_t stream);
void launch_guess(double2* out, const Geo& g, const TrapDev& trap, const PhysDev* phys, int nsolve, const int kind[3],
                  double muTF_base, double* mass_tmp, cudaStream_t st);

}  // namespace gpsoc
