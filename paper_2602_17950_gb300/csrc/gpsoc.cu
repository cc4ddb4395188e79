// C ABI of libgpsoc: problem object, device memory, the PCG / CM-PCG driver.
//
// The driver keeps every solve's state on the device.  One PCG iteration
// (Algorithm 1 with Algorithm 2) is a fixed sequence of kernels over all
// solves of the batch; solves that have stopped leave every kernel at once.
// Two iterations (the residual and direction buffers swap roles) are captured
// in a CUDA graph that the host replays; the host reads the per-solve flags
// only every `check_every` iterations.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <vector>

#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define GPSOC_HAVE_NVTX 1
#else
#define GPSOC_HAVE_NVTX 0
#endif

#include "gpsoc_internal.cuh"
#include "kernels.cuh"

// NVTX ranges around the host-side phases (a solve, each multigrid level, the FP64
// lead-in, the hybrid verification, the autotuner, a server step), for timeline tools
// (ncu --nvtx, Nsight Systems); without an attached tool the calls return at once.
namespace {
struct NvtxRange {
#if GPSOC_HAVE_NVTX
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
#else
  explicit NvtxRange(const char*) {}   // toolkit without the NVTX headers: no ranges
#endif
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace

using namespace gpsoc;

namespace {

thread_local std::string g_err;

gpsoc_status fail(gpsoc_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return fail(GPSOC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}
bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// Records every kernel the host enqueues: counts launches and, when profiling,
// brackets each with CUDA events on the problem's stream.
struct Tracker {
  cudaStream_t stream = nullptr;
  uint64_t count = 0;
  bool events = false;
  std::vector<const char*> names;
  std::vector<cudaEvent_t> evs;
  void start() {
    if (events) { cudaEvent_t e; cudaEventCreate(&e); cudaEventRecord(e, stream); evs.push_back(e); }
  }
  void mark(const char* name) {
    ++count;
    if (events) {
      cudaEvent_t e; cudaEventCreate(&e); cudaEventRecord(e, stream); evs.push_back(e);
      names.push_back(name);
    }
  }
};

template <class T>
struct Bufs {
  using C = cx_t<T>;
  C *Phi = nullptr, *HPhi = nullptr, *R[2] = {nullptr, nullptr}, *P[2] = {nullptr, nullptr};
  C *Z = nullptr, *D = nullptr, *A = nullptr, *B = nullptr, *W = nullptr, *G = nullptr;
  C *Xh = nullptr, *Ph = nullptr;   // GPSOC_HYBRID (FP32 set): spectra of Phi and of the last P
};


const char* row_name(int m) {
  static const char* n[] = {"row_fwd", "row_fwd_proj", "row_fwd_pre", "row_inv_h", "row_inv_p", "row_inv_pre",
                            "row_inv_plain", "row_inv_lin", "row_fwd_upd", "row_fwd_pre_hy", "row_inv_p_hy"};
  return (m >= 0 && m < (int)(sizeof(n) / sizeof(n[0]))) ? n[m] : "row_?";
}
const char* col_name(int m, int axis) {
  static const char* n[2][7] = {{"coly_fwd", "coly_inv", "coly_mid_h", "coly_mid_pre", "coly_ymid_h", "coly_yinv_h", "coly_kin"},
                                {"colz_fwd", "colz_inv", "colz_mid_h", "colz_mid_pre", "colz_ymid_h", "colz_yinv_h", "colz_kin"}};
  return (m >= 0 && m < 7) ? n[axis == 2 ? 1 : 0][m] : "col_?";
}
const char* scalar_name(int ph) {
  static const char* n[] = {"sc_init", "sc_obs", "sc_res", "sc_beta", "sc_step", "sc_clear",
                            "sc_norm", "sc_model", "sc_kin"};
  return (ph >= 0 && ph < (int)(sizeof(n) / sizeof(n[0]))) ? n[ph] : "sc_?";
}
const char* elem_name(int m) {
  static const char* n[] = {"el_update", "el_mass", "el_scale"};
  return (m >= 0 && m < (int)(sizeof(n) / sizeof(n[0]))) ? n[m] : "el_?";
}
}  // namespace

struct gpsoc_problem {
  int dim = 2;
  int n[3] = {1, 1, 1};
  double L[3] = {1, 1, 1};
  int batch = 1;
  gpsoc_trap trap{};
  double* d_userV = nullptr;
  std::vector<gpsoc_params> params;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  PhysDev* d_phys = nullptr;
  SolveState* d_st = nullptr;
  SolveState* h_st = nullptr;   // pinned mirror
  double* d_part = nullptr;
  int pmax = 0;
  int nsm = 1;                  // SMs of the device (grid of the elementwise hybrid pass)
  unsigned* d_cnt = nullptr;    // per-solve block arrival counters of the fused scalar steps
  double* d_scale = nullptr;    // per-solve scale factors
  double* d_tmp = nullptr;      // 3*batch doubles + model outputs
  size_t tmp_len = 0;
  Bufs<double> b64;
  Bufs<float> b32;              // FP32 working set of mixed-precision solves (allocated on first use)
  std::map<int, double2*> tw64;
  std::map<int, float2*> tw32;
  int level = 0;
  bool has_state = false;
  int max_level = 0;
  // captured iteration graph (two iterations) for the current level / options
  // [0] FP64, [1] FP32, [2] hybrid, [3] hybrid opening with the exact FP64 recomputation
  cudaGraphExec_t graph[4] = {nullptr, nullptr, nullptr, nullptr};
  int graph_level[4] = {-1, -1, -1, -1};
  OptsDev graph_opts[4]{};
  uint64_t graph_kernels[4] = {0, 0, 0, 0};   // kernels per replay of the captured graph
  uint64_t launches = 0;        // kernels launched so far (graph replays included)
  Tracker* tr = nullptr;        // active tracker while enqueueing
  std::vector<std::string> prof_names;
  std::vector<std::vector<int>> level_iters;   // per solve, iterations per level of the last solve
  std::vector<std::vector<int>> level_fp32;    // per solve, FP32 iterations per level of the last solve
  std::vector<std::vector<double>> level_res32;   // per solve, max |r| where each level's FP32 phase ended
  void* d_ptrs = nullptr;       // small device table of buffer pointers (FP32 phase hand-over)
};

namespace {

void mark(gpsoc_problem* p, const char* name) {
  if (p->tr) p->tr->mark(name);
  else p->launches++;
}
template <class T>
void RL(gpsoc_problem* p, int mode, const ChainArgs<T>& a) {
  launch_row<T>(mode, a, 0, Launch{}, p->stream);
  mark(p, row_name(mode));
}
template <class T>
void CL(gpsoc_problem* p, int mode, int axis, const ChainArgs<T>& a) {
  launch_col<T>(mode, axis, a, Launch{}, p->stream);
  mark(p, col_name(mode, axis));
}
void SL(gpsoc_problem* p, const ScalarArgs& x) {
  launch_scalar(x, p->stream);
  mark(p, scalar_name(x.phase));
}
template <class T>
void EL(gpsoc_problem* p, int mode, const ElemArgs<T>& e) {
  launch_elem<T>(mode, e, p->stream);
  mark(p, elem_name(mode));
}

Geo make_geo(const gpsoc_problem* p, int level) {
  Geo g{};
  g.d = p->dim;
  g.npts = 1;
  g.dV = 1.0;
  for (int i = 0; i < 3; ++i) {
    if (i < p->dim) {
      g.n[i] = p->n[i] >> level;
      g.L[i] = p->L[i];
      g.h[i] = 2.0 * p->L[i] / g.n[i];
      g.piL[i] = 3.14159265358979323846 / p->L[i];
      g.dV *= g.h[i];
    } else {
      g.n[i] = 1;
      g.L[i] = 1.0;
      g.h[i] = 1.0;
      g.piL[i] = 0.0;
    }
    g.log2n[i] = ilog2(g.n[i]);
    g.npts *= g.n[i];
    g.fL[i] = (float)g.L[i];
    g.fh[i] = (float)g.h[i];
    g.fpiL[i] = (float)g.piL[i];
  }
  return g;
}

TrapDev make_trap(const gpsoc_problem* p, int level) {
  TrapDev t{};
  for (int i = 0; i < 3; ++i) t.half_g2[i] = (i < p->dim) ? 0.5 * p->trap.g[i] * p->trap.g[i] : 0.0;
  t.quad = (p->trap.kind == GPSOC_TRAP_HARMONIC) ? 0.0 : p->trap.quad;
  t.quart = (p->trap.kind == GPSOC_TRAP_HARMONIC) ? 0.0 : p->trap.quart;
  t.userV = (level == 0) ? p->d_userV : nullptr;
  for (int i = 0; i < 3; ++i) t.fhalf_g2[i] = (float)t.half_g2[i];
  t.fquad = (float)t.quad;
  t.fquart = (float)t.quart;
  return t;
}

gpsoc_status twiddles(gpsoc_problem* p, int n, const double2** out) {
  auto it = p->tw64.find(n);
  if (it != p->tw64.end()) { *out = it->second; return GPSOC_OK; }
  // W_n^k = exp(-2 pi i k / n), k < n; from the first octant by symmetry so that
  // W^(n/4) = -i, W^(n/2) = -1 hold exactly
  std::vector<double2> h(n);
  const double PI = 3.14159265358979323846;
  for (int k = 0; k < n; ++k) {
    int m = k;
    double sc = 1.0, ss = 1.0;
    // reduce to [0, n/4]: W^(k) = -i W^(k - n/4)
    int quad = 0;
    while (m > n / 4) { m -= n / 4; ++quad; }
    double c, sn;
    if (2 * m <= n / 4) { const double a = 2.0 * PI * m / n; c = std::cos(a); sn = std::sin(a); }
    else { const double a = 2.0 * PI * (n / 4 - m) / n; c = std::sin(a); sn = std::cos(a); }
    (void)sc; (void)ss;
    double re = c, im = -sn;   // exp(-i a)
    for (int q = 0; q < quad; ++q) { const double t = re; re = im; im = -t; }   // multiply by -i
    h[k] = make_double2(re, im);
  }
  double2* d = nullptr;
  CK(cudaMalloc(&d, sizeof(double2) * n));
  CK(cudaMemcpy(d, h.data(), sizeof(double2) * n, cudaMemcpyHostToDevice));
  p->tw64[n] = d;
  *out = d;
  return GPSOC_OK;
}

gpsoc_status twiddles(gpsoc_problem* p, int n, const float2** out) {
  auto it = p->tw32.find(n);
  if (it != p->tw32.end()) { *out = it->second; return GPSOC_OK; }
  const double2* d64;
  gpsoc_status s = twiddles(p, n, &d64);
  if (s != GPSOC_OK) return s;
  std::vector<double2> h(n);
  CK(cudaMemcpy(h.data(), d64, sizeof(double2) * n, cudaMemcpyDeviceToHost));
  std::vector<float2> f(n);
  for (int k = 0; k < n; ++k) f[k] = make_float2((float)h[k].x, (float)h[k].y);
  float2* d = nullptr;
  CK(cudaMalloc(&d, sizeof(float2) * n));
  CK(cudaMemcpy(d, f.data(), sizeof(float2) * n, cudaMemcpyHostToDevice));
  p->tw32[n] = d;
  *out = d;
  return GPSOC_OK;
}

template <class T> Bufs<T>& bufs(gpsoc_problem* p);
template <> Bufs<double>& bufs<double>(gpsoc_problem* p) { return p->b64; }
template <> Bufs<float>& bufs<float>(gpsoc_problem* p) { return p->b32; }

template <class T>
gpsoc_status chain_args(gpsoc_problem* p, int level, ChainArgs<T>& a) {
  a = ChainArgs<T>{};
  a.g = make_geo(p, level);
  a.trap = make_trap(p, level);
  a.phys = p->d_phys;
  a.st = p->d_st;
  a.part = p->d_part;
  a.pmax = p->pmax;
  a.nsolve = p->batch;
  a.gate = GATE_ACTIVE;
  a.scale = 1.0;
  a.cnt = p->d_cnt;
  for (int i = 0; i < 3; ++i) {
    if (i < p->dim) {
      const cx_t<T>* tw;
      gpsoc_status s = twiddles(p, a.g.n[i], &tw);
      if (s != GPSOC_OK) return s;
      a.tw[i] = tw;
    }
  }
  return GPSOC_OK;
}

template <class T = double>
ScalarArgs scalar_args(gpsoc_problem* p, int level, int phase, const Geo& g) {
  ScalarArgs s{};
  s.st = p->d_st;
  s.phys = p->d_phys;
  s.part = p->d_part;
  s.pmax = p->pmax;
  s.nb_row = row_blocks_per_solve<T>(g, p->batch);
  s.nb_col = col_blocks_per_solve<T>(g, p->dim - 1, p->batch);
  s.nsolve = p->batch;
  s.phase = phase;
  s.npts = g.npts;
  s.inv_npts = 1.0 / (double)g.npts;
  s.part_dw = sizeof(T) == 4 ? 1 : 0;
  s.dV = g.dV;
  s.norm_scale = p->d_scale;
  (void)level;
  return s;
}

template <class T>
ScalarCtx scalar_ctx(gpsoc_problem* p, const Geo& g, const OptsDev& o, int flags) {
  ScalarCtx c{};
  c.st = p->d_st;
  c.phys = p->d_phys;
  c.part = p->d_part;
  c.pmax = p->pmax;
  c.nb_row = row_blocks_per_solve<T>(g, p->batch);
  c.nb_col = col_blocks_per_solve<T>(g, p->dim - 1, p->batch);
  c.npts = g.npts;
  c.dV = g.dV;
  c.opts = o;
  c.flags = flags;
  c.inv_npts = 1.0 / (double)g.npts;
  c.part_dw = sizeof(T) == 4 ? 1 : 0;
  return c;
}

template <class T>
ElemArgs<T> elem_args(gpsoc_problem* p, const Geo& g, int gate) {
  ElemArgs<T> e{};
  e.st = p->d_st;
  e.part = p->d_part;
  e.pmax = p->pmax;
  e.npts = g.npts;
  e.bps = row_blocks_per_solve<T>(g, p->batch);
  e.nsolve = p->batch;
  e.gate = gate;
  e.scalev = p->d_scale;
  return e;
}

// Spectral middle of the H chain: A = F_x(u) -> (T', G) (2D: one y pass; 3D: y fwd, z symbol, y inverse)
template <class T>
void h_middle(gpsoc_problem* p, ChainArgs<T> a, Bufs<T>& B) {
  a.fuse = 0;
  if (p->dim == 2) {
    a.in0 = B.A; a.out0 = B.W; a.out1 = B.G;
    CL<T>(p, COL_YMID_H, 1, a);
  } else {
    a.in0 = B.A; a.out0 = B.B; a.out1 = nullptr;
    CL<T>(p, COL_FWD, 1, a);
    a.in0 = B.B; a.out0 = B.B;
    CL<T>(p, COL_MID_H, 2, a);
    a.in0 = B.B; a.in1 = B.A; a.out0 = B.W; a.out1 = B.G;
    CL<T>(p, COL_YINV_H, 1, a);
  }
}

// H(Phi) chain: src -> dst (H(src) with nonlinear terms) and energy reductions.
// With pending_P != nullptr the first pass applies the pending accepted step.
template <class T>
void run_h_chain(gpsoc_problem* p, ChainArgs<T> a, Bufs<T>& B, cx_t<T>* src, cx_t<T>* dst,
                 const cx_t<T>* pending_P = nullptr, int fuse_obs = 0) {
  ChainArgs<T> f = a;
  f.fuse = 0;
  if (pending_P) {
    f.in0 = src; f.in2 = pending_P; f.out1 = src; f.out0 = B.A;
    RL<T>(p, ROW_FWD_UPD, f);
  } else {
    f.in0 = src; f.out0 = B.A;
    RL<T>(p, ROW_FWD_PLAIN, f);
  }
  h_middle<T>(p, a, B);
  ChainArgs<T> g = a;
  g.fuse = fuse_obs;
  g.in0 = B.W; g.in1 = B.G; g.in2 = src; g.out0 = dst; g.out1 = nullptr;
  RL<T>(p, ROW_INV_H, g);
}

// preconditioner chain: r = in0 - mu Phi (or in0 given as r) -> rout, z = P_C r -> zout; with
// rprev and pprev the last pass also takes beta, the projection and Algorithm 2 Step 2
template <class T>
void run_pre_chain(gpsoc_problem* p, ChainArgs<T> a, Bufs<T>& B, const cx_t<T>* hphi, const cx_t<T>* phi,
                   cx_t<T>* rout, const cx_t<T>* rprev, cx_t<T>* zout, int fuse, const cx_t<T>* pprev = nullptr) {
  ChainArgs<T> f = a;
  f.fuse = fuse;
  f.in0 = hphi; f.in1 = phi; f.out0 = B.A; f.out1 = rout;
  RL<T>(p, ROW_FWD_PRE, f);
  ChainArgs<T> m = a;
  m.fuse = 0;
  m.given_r = 0;
  if (p->dim == 2) {
    m.in0 = B.A; m.out0 = B.A;
    CL<T>(p, COL_MID_PRE, 1, m);
  } else {
    m.in0 = B.A; m.out0 = B.A;
    CL<T>(p, COL_FWD, 1, m);
    CL<T>(p, COL_MID_PRE, 2, m);
    m.scale = 1.0;
    CL<T>(p, COL_INV, 1, m);
  }
  ChainArgs<T> iv = a;
  iv.fuse = fuse;
  iv.given_r = 0;
  iv.in0 = B.A; iv.in1 = phi; iv.in2 = rout; iv.in3 = rprev; iv.in4 = pprev; iv.out0 = zout;
  RL<T>(p, ROW_INV_PRE, iv);
}

// P chain: P = -z + beta P_prev - cproj Phi -> pout, step-model reductions
template <class T>
void run_p_chain(gpsoc_problem* p, ChainArgs<T> a, Bufs<T>& B, const cx_t<T>* z, const cx_t<T>* pprev,
                 const cx_t<T>* phi, const cx_t<T>* hphi, cx_t<T>* pout, int fuse_step) {
  ChainArgs<T> f = a;
  f.fuse = 0;
  f.in0 = z; f.in1 = phi; f.in2 = pprev; f.out0 = B.A; f.out1 = pout;
  RL<T>(p, ROW_FWD_PROJ, f);
  h_middle<T>(p, a, B);
  ChainArgs<T> g = a;
  g.fuse = fuse_step;
  g.in0 = B.W; g.in1 = B.G; g.in2 = pout; g.in3 = phi; g.in4 = hphi; g.out0 = nullptr; g.out1 = nullptr;
  RL<T>(p, ROW_INV_P, g);
}

// One PCG iteration for all active solves (Algorithm 1 with Algorithm 2), ten
// kernels; every scalar step runs in the last block of the pass that produces
// its sums.  The step accepted here is applied by the first pass of the next
// iteration (or by flush_pending).
template <class T>
gpsoc_status enqueue_iteration(gpsoc_problem* p, int level, Bufs<T>& B, int parity, const OptsDev& o, int fp32) {
  ChainArgs<T> a;
  gpsoc_status s = chain_args<T>(p, level, a);
  if (s != GPSOC_OK) return s;
  const Geo g = a.g;
  const int cur = parity & 1, prv = cur ^ 1;
  a.sc = scalar_ctx<T>(p, g, o, (fp32 ? 2 : 0) | (cur << 2));
  // apply the pending step, H(Phi^n), E, mu, alpha
  run_h_chain<T>(p, a, B, B.Phi, B.HPhi, B.P[prv], 1);
  // r^n, stopping test, P_C r^n, beta, Re<D, Phi> and the beta = 0 decision
  run_pre_chain<T>(p, a, B, B.HPhi, B.Phi, B.R[cur], B.R[prv], B.Z, 1, B.P[prv]);
  // P^n, step model, Algorithm 2
  run_p_chain<T>(p, a, B, B.Z, B.P[prv], B.Phi, B.HPhi, B.P[cur], 1);
  CK(cudaGetLastError());
  return GPSOC_OK;
}

// apply steps accepted by the last enqueued iteration (parity of that iteration given)
template <class T>
gpsoc_status flush_pending(gpsoc_problem* p, int level, Bufs<T>& B, int last_parity) {
  const Geo g = make_geo(p, level);
  ElemArgs<T> e = elem_args<T>(p, g, GATE_PENDING);
  e.in0 = B.P[last_parity & 1]; e.out0 = B.Phi;
  EL<T>(p, EL_UPDATE, e);
  ScalarArgs x = scalar_args<T>(p, level, PH_CLEAR, g);
  SL(p, x);
  CK(cudaGetLastError());
  return GPSOC_OK;
}

OptsDev make_opts(const gpsoc_opts* o) {
  OptsDev d{};
  d.stop = o->stop ? o->stop : GPSOC_STOP_ENERGY;
  d.tol = o->tol;
  d.res_tol = o->res_tol;
  d.max_iter = o->max_iter > 0 ? o->max_iter : 100000;
  d.theta_trial = o->theta_trial > 0 ? o->theta_trial : 0.1;
  d.sigma = (o->sigma > 0 && o->sigma < 1) ? o->sigma : 0.5;
  d.max_halvings = o->max_halvings > 0 ? o->max_halvings : 40;
  d.no_stop = 0;
  d.precond = o->precond;
  d.res32 = o->fp32_res_switch > 0 ? o->fp32_res_switch : 0.0;
  d.line_search = o->line_search == 1 ? 1 : 0;
  return d;
}

gpsoc_status init_level(gpsoc_problem* p, int level, bool reset_counters, bool keep_direction = false) {
  const Geo g = make_geo(p, level);
  ScalarArgs x = scalar_args(p, level, PH_INIT, g);
  x.flags = (reset_counters ? 1 : 0) | (keep_direction ? 4 : 0);
  SL(p, x);
  CK(cudaGetLastError());
  return GPSOC_OK;
}

gpsoc_status sync_state(gpsoc_problem* p) {
  CK(cudaMemcpyAsync(p->h_st, p->d_st, sizeof(SolveState) * p->batch, cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return GPSOC_OK;
}

template <class T>
gpsoc_status build_graph(gpsoc_problem* p, int level, const OptsDev& o) {
  const int k = (sizeof(T) == 8) ? 0 : 1;
  if (p->graph[k] && p->graph_level[k] == level && std::memcmp(&p->graph_opts[k], &o, sizeof(o)) == 0) return GPSOC_OK;
  if (p->graph[k]) { cudaGraphExecDestroy(p->graph[k]); p->graph[k] = nullptr; }
  cudaGraph_t gr;
  Tracker tr;
  tr.stream = p->stream;
  CK(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
  p->tr = &tr;
  gpsoc_status s = enqueue_iteration<T>(p, level, bufs<T>(p), 0, o, k);
  if (s == GPSOC_OK) s = enqueue_iteration<T>(p, level, bufs<T>(p), 1, o, k);
  cudaError_t e = cudaStreamEndCapture(p->stream, &gr);
  p->tr = nullptr;
  p->graph_kernels[k] = tr.count;
  if (s != GPSOC_OK) { if (e == cudaSuccess) cudaGraphDestroy(gr); return s; }
  if (e != cudaSuccess) return fail(GPSOC_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&p->graph[k], gr, 0);
  cudaGraphDestroy(gr);
  if (e != cudaSuccess) return fail(GPSOC_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  p->graph_level[k] = level;
  p->graph_opts[k] = o;
  return GPSOC_OK;
}

// replay the iteration graph of precision T until every solve has stopped
template <class T>
gpsoc_status iterate_until_done(gpsoc_problem* p, int level, const OptsDev& o, int check_every) {
  const int k = (sizeof(T) == 8) ? 0 : 1;
  gpsoc_status s = build_graph<T>(p, level, o);
  if (s != GPSOC_OK) return s;
  const int pairs = (check_every + 1) / 2;
  const long long cap = (long long)o.max_iter + 4;
  for (long long it = 0; it <= cap; it += 2 * pairs) {
    for (int r = 0; r < pairs; ++r) {
      CK(cudaGraphLaunch(p->graph[k], p->stream));
      p->launches += p->graph_kernels[k];
    }
    s = sync_state(p);
    if (s != GPSOC_OK) return s;
    bool any = false;
    for (int i = 0; i < p->batch; ++i) any |= (p->h_st[i].active != 0);
    if (!any) return GPSOC_OK;
  }
  return GPSOC_OK;
}

gpsoc_status ensure_fp32(gpsoc_problem* p) {
  if (p->b32.Phi) return GPSOC_OK;
  const Geo g = make_geo(p, 0);
  const size_t arr = sizeof(float2) * (size_t)p->batch * 3 * g.npts;
  float2** slots[] = {&p->b32.Phi, &p->b32.HPhi, &p->b32.R[0], &p->b32.R[1], &p->b32.P[0], &p->b32.P[1],
                      &p->b32.Z, &p->b32.D, &p->b32.A, &p->b32.B, &p->b32.W, &p->b32.G, &p->b32.Xh, &p->b32.Ph};
  for (float2** sl : slots) {
    if (cudaMalloc(sl, arr) != cudaSuccess) { cudaGetLastError(); return fail(GPSOC_ENOMEM, "device allocation failed (FP32 set)"); }
  }
  return GPSOC_OK;
}

// FP64 state -> FP32 working copy (or back)
gpsoc_status convert_state(gpsoc_problem* p, int level, bool to32) {
  const Geo g = make_geo(p, level);
  const long long cnt = (long long)p->batch * 3 * g.npts;
  if (to32) launch_convert<float>(p->b64.Phi, 0, p->b32.Phi, cnt, p->stream);
  else launch_convert<double>(p->b32.Phi, 1, p->b64.Phi, cnt, p->stream);
  mark(p, "convert");
  CK(cudaGetLastError());
  return GPSOC_OK;
}

// ==================================================================== GPSOC_HYBRID
// The wave function, H_lin Phi, the residual r = H(Phi) - mu Phi, every reduction of
// the state and Algorithm 2 stay FP64; the preconditioner's and the direction's
// transforms (and H_lin P) run in FP32.  H_lin Phi^{n+1} is formed from H_lin Phi^n and
// H_lin P^n by linearity (the step is a linear combination of Phi^n and P^n), and
// recomputed exactly in FP64 every few iterations and before a solve's residual is
// accepted, so the fixed point is the FP64 one: only the search directions carry FP32
// rounding.

HyArgs hy_args(gpsoc_problem* p, int level, const Geo& g, const ScalarCtx& sc, int parity, int gate, int flags) {
  HyArgs h{};
  h.st = p->d_st;
  h.phys = p->d_phys;
  h.part = p->d_part;
  h.pmax = p->pmax;
  h.g = g;
  h.trap = make_trap(p, level);
  h.phi = p->b64.Phi;
  h.hl = p->b64.HPhi;
  h.p = p->b32.P[(parity & 1) ^ 1];   // direction of the previous iteration
  h.hlp = p->b32.HPhi;                // its H_lin P
  h.phi32 = p->b32.Phi;
  h.hphi = p->b64.Z;                  // H(Phi): the FP64 Z buffer is free in hybrid iterations
  h.npts = g.npts;
  h.bps = hy_blocks_per_solve(g, p->batch, p->nsm);
  h.nsolve = p->batch;
  h.gate = gate;
  h.flags = flags;
  h.fuse = (flags & HY_REDUCE) ? 1 : 0;
  h.sc = sc;
  h.sc.nb_row = h.bps;                // the observables step sums the partials this pass wrote
  return h;
}

// The observables step (E, mu, alpha, masses from the pass's partials) runs as its own
// one-block-per-solve kernel: fused into the last block of k_hy_upd, whose code is held to
// 128 registers for two resident blocks per SM, its single SM stayed busy about 33k cycles
// (ncu, 256^2) against 11k for the same step alone; the iteration measured 1-2% faster
// with the separate launch.
void HY(gpsoc_problem* p, const HyArgs& h) {
  launch_hy_upd(h, p->stream);
  mark(p, (h.flags & HY_REDUCE) ? "hy_upd" : "hy_step");
  if (h.fuse) {
    ScalarArgs x{};
    x.st = h.st;
    x.phys = h.phys;
    x.part = h.part;
    x.pmax = h.pmax;
    x.nb_row = h.bps;
    x.nb_col = h.sc.nb_col;
    x.nsolve = h.nsolve;
    x.phase = PH_OBS;
    x.flags = h.sc.flags;
    x.npts = h.npts;
    x.dV = h.sc.dV;
    x.opts = h.sc.opts;
    x.force = (h.gate == GATE_ALL) ? 1 : 0;
    x.inv_npts = h.sc.inv_npts;
    x.part_dw = 1;
    SL(p, x);
  }
}

// exact FP64 H_lin Phi into b64.HPhi and the per-component kinetic sums into the state
gpsoc_status hy_exact_hlin(gpsoc_problem* p, int level, int gate) {
  ChainArgs<double> d;
  gpsoc_status s = chain_args<double>(p, level, d);
  if (s != GPSOC_OK) return s;
  Bufs<double>& D = p->b64;
  d.gate = gate;
  d.fuse = 0;
  d.in0 = D.Phi; d.out0 = D.A;
  RL<double>(p, ROW_FWD_PLAIN, d);
  h_middle<double>(p, d, D);
  ChainArgs<double> l = d;
  l.in0 = D.W; l.in1 = D.G; l.in2 = D.Phi; l.out0 = D.HPhi; l.out1 = nullptr;
  RL<double>(p, ROW_INV_LIN, l);
  ScalarArgs x = scalar_args<double>(p, level, PH_KIN, d.g);
  x.force = (gate == GATE_ALL) ? 1 : 0;
  SL(p, x);
  return GPSOC_OK;
}

// One GPSOC_HYBRID iteration for every active solve; `exact` opens it with the exact
// FP64 recomputation of H_lin Phi instead of the update by linearity.
gpsoc_status enqueue_iteration_hy(gpsoc_problem* p, int level, int parity, const OptsDev& o, bool exact) {
  ChainArgs<float> a;
  gpsoc_status s = chain_args<float>(p, level, a);
  if (s != GPSOC_OK) return s;
  const Geo g = a.g;
  const int cur = parity & 1, prv = cur ^ 1;
  a.sc = scalar_ctx<float>(p, g, o, 2 | (cur << 2) | 8);
  Bufs<float>& F = p->b32;
  Bufs<double>& D = p->b64;
  // apply the pending step; H_lin Phi by linearity or exactly; E, mu, alpha, masses (FP64)
  if (exact) {
    HY(p, hy_args(p, level, g, a.sc, parity, GATE_ACTIVE, HY_UPD));
    s = hy_exact_hlin(p, level, GATE_ACTIVE);
    if (s != GPSOC_OK) return s;
    HY(p, hy_args(p, level, g, a.sc, parity, GATE_ACTIVE, HY_REDUCE));
    // the spectrum of Phi, from its FP32 copy, for the kinetic sums of the P chain
    ChainArgs<float> t = a;
    t.fuse = 0;
    t.in0 = F.Phi; t.out0 = F.B;
    RL<float>(p, ROW_FWD_PLAIN, t);
    t.in0 = F.B; t.out0 = (p->dim == 2) ? F.Xh : F.B;
    CL<float>(p, COL_FWD, 1, t);
    if (p->dim == 3) {
      t.in0 = F.B; t.out0 = F.Xh;
      CL<float>(p, COL_FWD, 2, t);
    }
  } else {
    HY(p, hy_args(p, level, g, a.sc, parity, GATE_ACTIVE, HY_UPD | HY_REC | HY_REDUCE));
  }
  // r in FP64 (stored FP32), stopping test, P_C r in FP32, beta
  ChainArgs<float> f = a;
  f.fuse = 1;
  f.phi64 = D.Phi; f.hl64 = D.Z; f.out0 = F.A; f.out1 = F.R[cur];
  RL<float>(p, ROW_FWD_PRE_HY, f);
  ChainArgs<float> m = a;
  m.fuse = 0;
  m.in0 = F.A; m.out0 = F.A;
  if (p->dim == 2) {
    CL<float>(p, COL_MID_PRE, 1, m);
  } else {
    CL<float>(p, COL_FWD, 1, m);
    CL<float>(p, COL_MID_PRE, 2, m);
    m.scale = 1.0;
    CL<float>(p, COL_INV, 1, m);
  }
  ChainArgs<float> iv = a;
  iv.fuse = 1;
  iv.in0 = F.A; iv.in1 = F.Phi; iv.in2 = F.R[cur]; iv.in3 = F.R[prv]; iv.in4 = F.P[prv]; iv.out0 = F.Z;
  RL<float>(p, ROW_INV_PRE, iv);   // also beta, Re<D, Phi>, the slope Re<r, D> and Step 2
  // P, H_lin P (kept), step model with Re<r, P> and the FP64 radial part, Algorithm 2
  ChainArgs<float> pf = a;
  pf.fuse = 0;
  pf.in0 = F.Z; pf.in1 = F.Phi; pf.in2 = F.P[prv]; pf.out0 = F.A; pf.out1 = F.P[cur];
  RL<float>(p, ROW_FWD_PROJ, pf);
  ChainArgs<float> pm = a;
  pm.xhat = F.Xh; pm.phat = F.Ph; pm.khat_upd = exact ? 0 : 1;
  h_middle<float>(p, pm, F);
  ChainArgs<float> pi = a;
  pi.fuse = 1;
  pi.in0 = F.W; pi.in1 = F.G; pi.in2 = F.P[cur]; pi.in3 = F.Phi; pi.in4 = F.R[cur];
  pi.phi64 = D.Phi; pi.out0 = F.HPhi; pi.out1 = nullptr;
  RL<float>(p, ROW_INV_P_HY, pi);
  CK(cudaGetLastError());
  return GPSOC_OK;
}

gpsoc_status build_graph_hy(gpsoc_problem* p, int level, const OptsDev& o, bool exact) {
  const int k = exact ? 3 : 2;
  if (p->graph[k] && p->graph_level[k] == level && std::memcmp(&p->graph_opts[k], &o, sizeof(o)) == 0) return GPSOC_OK;
  if (p->graph[k]) { cudaGraphExecDestroy(p->graph[k]); p->graph[k] = nullptr; }
  cudaGraph_t gr;
  Tracker tr;
  tr.stream = p->stream;
  CK(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
  p->tr = &tr;
  gpsoc_status s = enqueue_iteration_hy(p, level, 0, o, exact);
  if (s == GPSOC_OK) s = enqueue_iteration_hy(p, level, 1, o, false);
  cudaError_t e = cudaStreamEndCapture(p->stream, &gr);
  p->tr = nullptr;
  p->graph_kernels[k] = tr.count;
  if (s != GPSOC_OK) { if (e == cudaSuccess) cudaGraphDestroy(gr); return s; }
  if (e != cudaSuccess) return fail(GPSOC_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&p->graph[k], gr, 0);
  cudaGraphDestroy(gr);
  if (e != cudaSuccess) return fail(GPSOC_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  p->graph_level[k] = level;
  p->graph_opts[k] = o;
  return GPSOC_OK;
}

// The stopping rule with the exact residual: for every solve that has stopped with
// status OK, recompute H_lin Phi in FP64, then E, mu, alpha and the residual; a solve
// whose exact residual misses the rule continues (*resumed counts them).  Buffer
// parity 0 is used, the parity the next iteration graph starts with.
gpsoc_status hy_verify(gpsoc_problem* p, int level, const OptsDev& o, int* resumed) {
  NvtxRange range("gpsoc hybrid verification");
  *resumed = 0;
  const Geo g = make_geo(p, level);
  OptsDev ov = o;
  ov.no_stop = 1;
  const ScalarCtx sc = scalar_ctx<float>(p, g, ov, 2 | 8);
  HY(p, hy_args(p, level, g, sc, 0, GATE_ALL, HY_UPD));
  gpsoc_status s = hy_exact_hlin(p, level, GATE_ALL);
  if (s != GPSOC_OK) return s;
  HY(p, hy_args(p, level, g, sc, 0, GATE_ALL, HY_REDUCE));
  ChainArgs<float> f;
  s = chain_args<float>(p, level, f);
  if (s != GPSOC_OK) return s;
  f.gate = GATE_ALL;
  f.sc = sc;
  f.fuse = 1;
  f.phi64 = p->b64.Phi; f.hl64 = p->b64.Z; f.out0 = p->b32.A; f.out1 = p->b32.R[0];
  RL<float>(p, ROW_FWD_PRE_HY, f);
  CK(cudaGetLastError());
  s = sync_state(p);
  if (s != GPSOC_OK) return s;
  for (int i = 0; i < p->batch; ++i) {
    SolveState& S = p->h_st[i];
    if (S.active || S.status != GPSOC_OK) continue;
    bool ok = true;
    if (o.stop == GPSOC_STOP_RES) ok = S.res_inf < o.tol;
    if (o.res_tol > 0.0) ok = ok && S.res_inf < o.res_tol;
    // resume with beta = 0: the check's residual took the buffer of one stored direction
    if (!ok) { S.active = 1; S.first = 1; ++*resumed; }
  }
  if (*resumed) {
    CK(cudaMemcpyAsync(p->d_st, p->h_st, sizeof(SolveState) * p->batch, cudaMemcpyHostToDevice, p->stream));
    CK(cudaStreamSynchronize(p->stream));
  }
  return GPSOC_OK;
}

int hy_refresh_every(const gpsoc_opts* o) { return o->hybrid_refresh > 0 ? o->hybrid_refresh : 16; }
double hy_lead_res(const gpsoc_opts* o) {
  return o->hybrid_lead_res > 0 ? o->hybrid_lead_res : (o->hybrid_lead_res < 0 ? 0.0 : 1e-4);
}

// options of an FP64 lead-in phase: the solve's own stopping rule, and the phase also ends
// (without ending the solve) once max|r| < lead_res, on stagnation or at the iteration cap
OptsDev lead_opts(const OptsDev& o, double lead_res) {
  OptsDev l = o;
  l.phase32 = 1;
  l.res32 = lead_res;
  l.tol_rel = 0.0;
  return l;
}

// replay the hybrid graphs until every solve has stopped with its exact residual
gpsoc_status iterate_until_done_hy(gpsoc_problem* p, int level, const OptsDev& o, int check_every, int refresh) {
  gpsoc_status s = build_graph_hy(p, level, o, false);
  if (s == GPSOC_OK) s = build_graph_hy(p, level, o, true);
  if (s != GPSOC_OK) return s;
  const int pairs = (check_every + 1) / 2;
  const int every = std::max(1, refresh / 2);   // pairs between exact recomputations
  for (int round = 0; round < 8; ++round) {
    long long k = 0;
    const long long cap = (long long)o.max_iter + 4;
    for (long long it = 0; it <= cap; it += 2 * pairs) {
      for (int r = 0; r < pairs; ++r, ++k) {
        const int gk = (k % every == 0) ? 3 : 2;
        CK(cudaGraphLaunch(p->graph[gk], p->stream));
        p->launches += p->graph_kernels[gk];
      }
      s = sync_state(p);
      if (s != GPSOC_OK) return s;
      bool any = false;
      for (int i = 0; i < p->batch; ++i) any |= (p->h_st[i].active != 0);
      if (!any) break;
    }
    int resumed = 0;
    s = hy_verify(p, level, o, &resumed);
    if (s != GPSOC_OK || resumed == 0) return s;
  }
  return GPSOC_OK;
}

// One multigrid level.  FP64: PCG to the stopping rule.  MIXED: PCG in FP32
// arrays (FP64 reductions and scalars) until the energy change falls below
// fp32_rel * |E| or Algorithm 2 finds no decrease (the FP32 rounding floor),
// then PCG in FP64 from that iterate (beta restarted) to the stopping rule.
gpsoc_status run_level(gpsoc_problem* p, int level, const OptsDev& o, int check_every, bool first_level,
                       int precision, double fp32_rel, bool carry, int refresh, double lead_res) {
  char rname[96];
  {
    const Geo gl = make_geo(p, level);
    const char* pn = precision == GPSOC_HYBRID ? "hybrid" : (precision == GPSOC_MIXED ? "mixed" : "fp64");
    if (p->dim == 2) snprintf(rname, sizeof rname, "gpsoc level %dx%d %s", gl.n[0], gl.n[1], pn);
    else snprintf(rname, sizeof rname, "gpsoc level %dx%dx%d %s", gl.n[0], gl.n[1], gl.n[2], pn);
  }
  NvtxRange range(rname);
  gpsoc_status s;
  if (precision == GPSOC_HYBRID) {
    s = ensure_fp32(p);
    if (s != GPSOC_OK) return s;
    s = init_level(p, level, first_level);
    if (s != GPSOC_OK) return s;
    if (lead_res > 0.0 && first_level) {
      // FP64 iterations until max|r| < lead_res on the first level (the early iterations
      // from the initial guess decide which local minimum the solve reaches; finer levels
      // start from the prolonged solution of that minimum)
      NvtxRange lead("gpsoc fp64 lead-in");
      s = iterate_until_done<double>(p, level, lead_opts(o, lead_res), check_every);
      if (s != GPSOC_OK) return s;
      s = init_level(p, level, false);
      if (s != GPSOC_OK) return s;
    }
    return iterate_until_done_hy(p, level, o, check_every, refresh);
  }
  if (precision == GPSOC_MIXED) {
    s = ensure_fp32(p);
    if (s != GPSOC_OK) return s;
    s = convert_state(p, level, true);
    if (s != GPSOC_OK) return s;
    s = init_level(p, level, first_level);
    if (s != GPSOC_OK) return s;
    OptsDev o32 = o;
    o32.stop = GPSOC_STOP_ENERGY;
    o32.res_tol = 0.0;
    o32.tol_rel = fp32_rel;
    o32.phase32 = 1;
    s = iterate_until_done<float>(p, level, o32, check_every);
    if (s != GPSOC_OK) return s;
    for (int i = 0; i < p->batch; ++i) p->level_res32[i].push_back(p->h_st[i].res_inf);
    // solves that took FP32 steps continue from their FP32 iterate and, unless the
    // options ask for a restart, from its last direction (beta carried over)
    {
      const Geo g = make_geo(p, level);
      const float2* r32[2] = {p->b32.R[0], p->b32.R[1]};
      const float2* p32[2] = {p->b32.P[0], p->b32.P[1]};
      float2** d_rp = reinterpret_cast<float2**>(p->d_ptrs);
      CK(cudaMemcpyAsync(d_rp, r32, sizeof(r32), cudaMemcpyHostToDevice, p->stream));
      CK(cudaMemcpyAsync(d_rp + 2, p32, sizeof(p32), cudaMemcpyHostToDevice, p->stream));
      launch_handover(p->b32.Phi, d_rp, d_rp + 2, p->b64.Phi, p->b64.R[1], p->b64.P[1], p->d_st, 3 * g.npts, p->batch,
                      carry ? 1 : 0, p->stream);
      mark(p, "handover");
      CK(cudaGetLastError());
    }
    s = init_level(p, level, false, carry);
    if (s != GPSOC_OK) return s;
    return iterate_until_done<double>(p, level, o, check_every);
  }
  s = init_level(p, level, first_level);
  if (s != GPSOC_OK) return s;
  return iterate_until_done<double>(p, level, o, check_every);
}

// MIXED runs an FP32 phase only where the work per iteration is large enough
// for FP32 arrays to pay (fp32_min_points, default 65536 solve-points).
long long mixed_min_points(const gpsoc_opts* opts) {
  return opts->fp32_min_points > 0 ? opts->fp32_min_points : opts->fp32_min_points < 0 ? 0 : 65536;
}

int level_precision(const gpsoc_problem* p, int level, const gpsoc_opts* opts) {
  if (opts->precision == GPSOC_HYBRID) return GPSOC_HYBRID;
  if (opts->precision != GPSOC_MIXED) return GPSOC_FP64;
  const Geo g = make_geo(p, level);
  return (long long)p->batch * g.npts >= mixed_min_points(opts) ? GPSOC_MIXED : GPSOC_FP64;
}

gpsoc_status normalize(gpsoc_problem* p, int level) {
  const Geo g = make_geo(p, level);
  ElemArgs<double> e = elem_args<double>(p, g, GATE_ALL);
  e.in0 = p->b64.Phi;
  EL<double>(p, EL_MASS, e);
  ScalarArgs x = scalar_args(p, level, PH_NORM, g);
  SL(p, x);
  e.in0 = p->b64.Phi; e.out0 = p->b64.Phi;
  EL<double>(p, EL_SCALE, e);
  CK(cudaGetLastError());
  return GPSOC_OK;
}

gpsoc_status prolong_impl(gpsoc_problem* p, int level) {
  // spectrum at level (coarse) -> zero padded at level-1 (fine) -> physical, x 2^d, renormalise
  const Geo gc = make_geo(p, level), gf = make_geo(p, level - 1);
  Bufs<double>& B = p->b64;
  ChainArgs<double> a;
  gpsoc_status s = chain_args<double>(p, level, a);
  if (s != GPSOC_OK) return s;
  a.gate = GATE_ALL;
  Launch lc{};
  a.in0 = B.Phi; a.out0 = B.A;
  RL<double>(p, ROW_FWD_PLAIN, a);
  a.in0 = B.A; a.out0 = B.A;
  for (int ax = 1; ax < p->dim; ++ax) CL<double>(p, COL_FWD, ax, a);
  launch_pad<double>(B.A, B.W, gc, gf, p->batch, p->stream);
  mark(p, "pad");
  ChainArgs<double> f;
  s = chain_args<double>(p, level - 1, f);
  if (s != GPSOC_OK) return s;
  f.gate = GATE_ALL;
  f.in0 = B.W; f.out0 = B.W; f.scale = 1.0;
  for (int ax = p->dim - 1; ax >= 1; --ax) CL<double>(p, COL_INV, ax, f);
  f.in0 = B.W; f.out0 = B.Phi;
  f.scale = (double)(1 << p->dim) / (double)gf.npts;   // 1/n_fine^d of the inverse, times 2^d
  RL<double>(p, ROW_INV_PLAIN, f);
  CK(cudaGetLastError());
  s = normalize(p, level - 1);
  if (s != GPSOC_OK) return s;
  p->level = level - 1;
  return GPSOC_OK;
}

void fill_results(const gpsoc_problem* p, gpsoc_result* r, int levels) {
  for (int i = 0; i < p->batch; ++i) {
    const SolveState& S = p->h_st[i];
    gpsoc_result& o = r[i];
    for (int k = 0; k < 8; ++k) {
      o.level_iters[k] = (i < (int)p->level_iters.size() && k < (int)p->level_iters[i].size()) ? p->level_iters[i][k] : 0;
      o.level_fp32_iters[k] = (i < (int)p->level_fp32.size() && k < (int)p->level_fp32[i].size()) ? p->level_fp32[i][k] : 0;
      o.level_res_fp32[k] = (i < (int)p->level_res32.size() && k < (int)p->level_res32[i].size()) ? p->level_res32[i][k] : 0.0;
    }
    o.status = S.status;
    if (S.status == GPSOC_OK && S.active) o.status = GPSOC_ENOTCONV;
    o.iters = S.iters;
    o.total_iters = S.total_iters;
    o.levels = levels;
    o.beta_resets = S.beta_resets;
    o.halvings = S.halvings;
    o.fp32_iters = S.fp32_iters;
    o.fp64_iters = S.fp64_iters;
    o.energy = S.E;
    o.mu = S.mu;
    for (int c = 0; c < 3; ++c) o.mass[c] = S.mass[c];
    o.res_inf = S.res_inf;
    o.dE_last = S.dE_last;
  }
}

gpsoc_status check_problem(const gpsoc_problem* p) {
  if (!p) return fail(GPSOC_EINVAL, "problem is NULL");
  return GPSOC_OK;
}

// H chain + observables for the current state without touching iteration flags, in
// the arrays of precision T (FP32: the FP64 state is first copied to the FP32 set;
// sums and scalars stay FP64 in both)
template <class T = double>
gpsoc_status observables_now(gpsoc_problem* p) {
  gpsoc_status s;
  if constexpr (sizeof(T) == 4) {
    s = ensure_fp32(p);
    if (s != GPSOC_OK) return s;
    s = convert_state(p, p->level, true);
    if (s != GPSOC_OK) return s;
  }
  Bufs<T>& B = bufs<T>(p);
  ChainArgs<T> a;
  s = chain_args<T>(p, p->level, a);
  if (s != GPSOC_OK) return s;
  a.gate = GATE_ALL;
  run_h_chain<T>(p, a, B, B.Phi, B.HPhi);
  ScalarArgs x = scalar_args<T>(p, p->level, PH_OBS, a.g);
  x.force = 1;
  SL(p, x);
  CK(cudaGetLastError());
  return sync_state(p);
}

gpsoc_status check_precision(int precision) {
  if (precision != GPSOC_FP64 && precision != GPSOC_MIXED) return fail(GPSOC_EINVAL, "unknown precision");
  return GPSOC_OK;
}

// device 3-array of precision T -> host FP64 (FP32 arrays are widened through the FP64 scratch D)
template <class T>
gpsoc_status copy_out(gpsoc_problem* p, const cx_t<T>* src, double* host) {
  const Geo g = make_geo(p, p->level);
  const long long cnt = (long long)p->batch * 3 * g.npts;
  const double2* from = reinterpret_cast<const double2*>(src);
  if constexpr (sizeof(T) == 4) {
    launch_convert<double>(src, 1, p->b64.D, cnt, p->stream);
    mark(p, "convert");
    CK(cudaGetLastError());
    from = p->b64.D;
  }
  CK(cudaMemcpyAsync(host, from, sizeof(double2) * (size_t)cnt, cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return GPSOC_OK;
}

// host FP64 3-array -> device array of precision T (FP32: through the FP64 scratch D)
template <class T>
gpsoc_status copy_in(gpsoc_problem* p, const double* host, cx_t<T>* dst) {
  const Geo g = make_geo(p, p->level);
  const long long cnt = (long long)p->batch * 3 * g.npts;
  double2* to = (sizeof(T) == 4) ? p->b64.D : reinterpret_cast<double2*>(dst);
  CK(cudaMemcpyAsync(to, host, sizeof(double2) * (size_t)cnt, cudaMemcpyHostToDevice, p->stream));
  if constexpr (sizeof(T) == 4) {
    launch_convert<float>(p->b64.D, 0, dst, cnt, p->stream);
    mark(p, "convert");
    CK(cudaGetLastError());
  }
  return GPSOC_OK;
}

template <class T>
gpsoc_status apply_h_impl(gpsoc_problem* p, double* hpsi, double* obs) {
  gpsoc_status s = observables_now<T>(p);
  if (s != GPSOC_OK) return s;
  if (hpsi) {
    s = copy_out<T>(p, bufs<T>(p).HPhi, hpsi);
    if (s != GPSOC_OK) return s;
  }
  if (obs) {
    for (int i = 0; i < p->batch; ++i) {
      const SolveState& S = p->h_st[i];
      double* o = obs + 9 * i;
      o[0] = S.E; o[1] = S.mu;
      for (int c = 0; c < 3; ++c) { o[2 + c] = S.alpha[c]; o[5 + c] = S.mass[c]; }
      o[8] = S.Q;
    }
  }
  return GPSOC_OK;
}

template <class T>
gpsoc_status apply_precond_impl(gpsoc_problem* p, const double* r, double* out) {
  gpsoc_status s = observables_now<T>(p);
  if (s != GPSOC_OK) return s;
  Bufs<T>& B = bufs<T>(p);
  s = copy_in<T>(p, r, B.D);
  if (s != GPSOC_OK) return s;
  ChainArgs<T> a;
  s = chain_args<T>(p, p->level, a);
  if (s != GPSOC_OK) return s;
  a.gate = GATE_ALL;
  a.given_r = 1;
  run_pre_chain<T>(p, a, B, B.D, B.Phi, B.R[0], nullptr, B.Z, 0);
  CK(cudaGetLastError());
  return copy_out<T>(p, B.Z, out);
}

template <class T>
gpsoc_status step_model_impl(gpsoc_problem* p, const double* P, const double* theta, int n_theta, double* out) {
  gpsoc_status s = observables_now<T>(p);
  if (s != GPSOC_OK) return s;
  const Geo g = make_geo(p, p->level);
  Bufs<T>& B = bufs<T>(p);
  // the P chain forms P = -z + beta P_prev - cproj Phi: pass z = -P with beta = cproj = 0
  std::vector<double> negP(2 * (size_t)p->batch * 3 * g.npts);
  for (size_t i = 0; i < negP.size(); ++i) negP[i] = -P[i];
  s = copy_in<T>(p, negP.data(), B.Z);
  if (s != GPSOC_OK) return s;
  double* d_theta = p->d_tmp;
  double* d_out = p->d_tmp + n_theta;
  if (n_theta) CK(cudaMemcpyAsync(d_theta, theta, sizeof(double) * n_theta, cudaMemcpyHostToDevice, p->stream));
  // cproj = 0 so that P is used as given
  for (int i = 0; i < p->batch; ++i) { p->h_st[i].cproj = 0.0; p->h_st[i].beta = 0.0; p->h_st[i].fcproj = 0.0f; p->h_st[i].fbeta = 0.0f; }
  CK(cudaMemcpyAsync(p->d_st, p->h_st, sizeof(SolveState) * p->batch, cudaMemcpyHostToDevice, p->stream));
  ChainArgs<T> a;
  s = chain_args<T>(p, p->level, a);
  if (s != GPSOC_OK) return s;
  a.gate = GATE_ALL;
  run_p_chain<T>(p, a, B, B.Z, nullptr, B.Phi, B.HPhi, B.P[0], 0);
  ScalarArgs x = scalar_args<T>(p, p->level, PH_MODEL, g);
  x.force = 1;
  x.thetas = d_theta;
  x.n_theta = n_theta;
  x.model_out = d_out;
  SL(p, x);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(out, d_out, sizeof(double) * (size_t)p->batch * (2 + n_theta), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return GPSOC_OK;
}

}  // namespace

extern "C" {

const char* gpsoc_last_error(void) { return g_err.c_str(); }
const char* gpsoc_version(void) { return "gpsoc 0.1 (sm_103a)"; }

gpsoc_status gpsoc_create(const gpsoc_grid* grid, const gpsoc_trap* trap, const gpsoc_params* params, int batch,
                          void* cuda_stream, gpsoc_problem** out) {
  g_err.clear();
  if (!grid || !trap || !params || !out) return fail(GPSOC_EINVAL, "NULL argument");
  *out = nullptr;
  if (grid->dim != 2 && grid->dim != 3) return fail(GPSOC_EINVAL, "dim must be 2 or 3");
  if (batch < 1) return fail(GPSOC_EINVAL, "batch must be >= 1");
  for (int i = 0; i < grid->dim; ++i) {
    if (!pow2(grid->n[i]) || grid->n[i] < 8 || grid->n[i] > 1024)
      return fail(GPSOC_EINVAL, "grid sizes must be powers of two in [8, 1024]");
    if (!(grid->L[i] > 0) || !std::isfinite(grid->L[i])) return fail(GPSOC_EINVAL, "box half-widths must be > 0");
  }
  if (trap->kind < 0 || trap->kind > 2) return fail(GPSOC_EINVAL, "unknown trap kind");
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(trap->g[i])) return fail(GPSOC_EINVAL, "trap frequencies must be finite");
  if (!std::isfinite(trap->quad) || !std::isfinite(trap->quart)) return fail(GPSOC_EINVAL, "trap coefficients must be finite");
  if (trap->kind == GPSOC_TRAP_USER && !trap->user_V) return fail(GPSOC_EINVAL, "user trap without user_V");
  for (int b = 0; b < batch; ++b) {
    const gpsoc_params& q = params[b];
    if (!std::isfinite(q.Omega) || !std::isfinite(q.gamma) || !std::isfinite(q.beta0) || !std::isfinite(q.beta1))
      return fail(GPSOC_EINVAL, "physical parameters must be finite");
  }
  gpsoc_problem* p = new gpsoc_problem();
  p->dim = grid->dim;
  for (int i = 0; i < 3; ++i) {
    p->n[i] = (i < grid->dim) ? grid->n[i] : 1;
    p->L[i] = (i < grid->dim) ? grid->L[i] : 1.0;
  }
  p->batch = batch;
  p->trap = *trap;
  p->trap.user_V = nullptr;
  p->params.assign(params, params + batch);
  int nmin = 1 << 30;
  for (int i = 0; i < p->dim; ++i) nmin = std::min(nmin, p->n[i]);
  p->max_level = ilog2(nmin) - 3;
  auto bail = [&](gpsoc_status s, const std::string& m) { gpsoc_destroy(p); return fail(s, m); };
  if (cuda_stream) {
    p->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(GPSOC_ECUDA, "stream create failed");
    p->own_stream = true;
  }
  if (chain_prepare<double>() != cudaSuccess || chain_prepare<float>() != cudaSuccess)
    return bail(GPSOC_ECUDA, "kernel attribute setup failed (is a GB300 / sm_103 device current?)");
  const Geo g = make_geo(p, 0);
  const size_t arr = sizeof(double2) * (size_t)batch * 3 * g.npts;
  double2** slots[] = {&p->b64.Phi, &p->b64.HPhi, &p->b64.R[0], &p->b64.R[1], &p->b64.P[0], &p->b64.P[1],
                       &p->b64.Z, &p->b64.D, &p->b64.A, &p->b64.B, &p->b64.W, &p->b64.G};
  for (double2** sl : slots) {
    if (cudaMalloc(sl, arr) != cudaSuccess) { cudaGetLastError(); return bail(GPSOC_ENOMEM, "device allocation failed"); }
  }
  // partial-sum stride: the largest blocks-per-solve of any pass at the finest level
  // the most blocks any pass can use per solve: one row, or one column line, per block
  p->pmax = (int)(g.npts / g.n[0]);
  for (int ax = 1; ax < p->dim; ++ax) p->pmax = std::max(p->pmax, (int)(g.npts / g.n[ax]));
  {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return bail(GPSOC_ECUDA, "device query failed");
  }
  // the elementwise hybrid pass: its block count grows with the points per level
  p->pmax = std::max(p->pmax, hy_blocks_per_solve(g, batch, p->nsm));
  if (cudaMalloc(&p->d_part, sizeof(double) * (size_t)batch * NSLOT * p->pmax) != cudaSuccess)
    return bail(GPSOC_ENOMEM, "device allocation failed");
  if (cudaMalloc(&p->d_st, sizeof(SolveState) * batch) != cudaSuccess) return bail(GPSOC_ENOMEM, "device allocation failed");
  if (cudaMalloc(&p->d_cnt, sizeof(unsigned) * batch) != cudaSuccess) return bail(GPSOC_ENOMEM, "device allocation failed");
  if (cudaMemset(p->d_cnt, 0, sizeof(unsigned) * batch) != cudaSuccess) return bail(GPSOC_ECUDA, "memset failed");
  if (cudaMemset(p->d_st, 0, sizeof(SolveState) * batch) != cudaSuccess) return bail(GPSOC_ECUDA, "memset failed");
  if (cudaMallocHost(&p->h_st, sizeof(SolveState) * batch) != cudaSuccess) return bail(GPSOC_ENOMEM, "host allocation failed");
  if (cudaMalloc(&p->d_scale, sizeof(double) * batch) != cudaSuccess) return bail(GPSOC_ENOMEM, "device allocation failed");
  if (cudaMalloc(&p->d_ptrs, 8 * sizeof(void*)) != cudaSuccess) return bail(GPSOC_ENOMEM, "device allocation failed");
  p->tmp_len = (size_t)batch * 64 + 4096;
  if (cudaMalloc(&p->d_tmp, sizeof(double) * p->tmp_len) != cudaSuccess) return bail(GPSOC_ENOMEM, "device allocation failed");
  std::vector<PhysDev> ph(batch);
  for (int b = 0; b < batch; ++b) ph[b] = make_phys(params[b].Omega, params[b].gamma, params[b].beta0, params[b].beta1);
  if (cudaMalloc(&p->d_phys, sizeof(PhysDev) * batch) != cudaSuccess) return bail(GPSOC_ENOMEM, "device allocation failed");
  if (cudaMemcpy(p->d_phys, ph.data(), sizeof(PhysDev) * batch, cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(GPSOC_ECUDA, "copy failed");
  // twiddle tables of every axis length of every level (no allocation later, e.g. during graph capture)
  for (int lev = 0; lev <= p->max_level; ++lev) {
    for (int i = 0; i < p->dim; ++i) {
      const double2* tw;
      const float2* tw32;
      if (twiddles(p, p->n[i] >> lev, &tw) != GPSOC_OK || twiddles(p, p->n[i] >> lev, &tw32) != GPSOC_OK)
        return bail(GPSOC_ENOMEM, "twiddle setup failed");
    }
  }
  if (trap->kind == GPSOC_TRAP_USER) {
    if (cudaMalloc(&p->d_userV, sizeof(double) * g.npts) != cudaSuccess) return bail(GPSOC_ENOMEM, "device allocation failed");
    if (cudaMemcpy(p->d_userV, trap->user_V, sizeof(double) * g.npts, cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(GPSOC_ECUDA, "copy failed");
  }
  *out = p;
  return GPSOC_OK;
}

void gpsoc_destroy(gpsoc_problem* p) {
  if (!p) return;
  if (p->stream) cudaStreamSynchronize(p->stream);
  for (int k = 0; k < 4; ++k) if (p->graph[k]) cudaGraphExecDestroy(p->graph[k]);
  double2* arrs[] = {p->b64.Phi, p->b64.HPhi, p->b64.R[0], p->b64.R[1], p->b64.P[0], p->b64.P[1],
                     p->b64.Z, p->b64.D, p->b64.A, p->b64.B, p->b64.W, p->b64.G};
  for (double2* a : arrs) if (a) cudaFree(a);
  float2* arrs32[] = {p->b32.Phi, p->b32.HPhi, p->b32.R[0], p->b32.R[1], p->b32.P[0], p->b32.P[1],
                      p->b32.Z, p->b32.D, p->b32.A, p->b32.B, p->b32.W, p->b32.G, p->b32.Xh, p->b32.Ph};
  for (float2* a : arrs32) if (a) cudaFree(a);
  for (auto& kv : p->tw64) cudaFree(kv.second);
  for (auto& kv : p->tw32) cudaFree(kv.second);
  if (p->d_part) cudaFree(p->d_part);
  if (p->d_st) cudaFree(p->d_st);
  if (p->d_cnt) cudaFree(p->d_cnt);
  if (p->h_st) cudaFreeHost(p->h_st);
  if (p->d_scale) cudaFree(p->d_scale);
  if (p->d_ptrs) cudaFree(p->d_ptrs);
  if (p->d_tmp) cudaFree(p->d_tmp);
  if (p->d_phys) cudaFree(p->d_phys);
  if (p->d_userV) cudaFree(p->d_userV);
  if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
  delete p;
}

size_t gpsoc_solve_size(const gpsoc_problem* p, int level) {
  if (!p || level < 0 || level > p->max_level) return 0;
  return (size_t)3 * make_geo(p, level).npts;
}

gpsoc_status gpsoc_set_initial(gpsoc_problem* p, const double* psi, int level) {
  g_err.clear();
  if (check_problem(p) != GPSOC_OK) return GPSOC_EINVAL;
  if (!psi) return fail(GPSOC_EINVAL, "psi is NULL");
  if (level < 0 || level > p->max_level) return fail(GPSOC_EINVAL, "level out of range");
  const Geo g = make_geo(p, level);
  CK(cudaMemcpyAsync(p->b64.Phi, psi, sizeof(double2) * (size_t)p->batch * 3 * g.npts, cudaMemcpyHostToDevice, p->stream));
  p->level = level;
  gpsoc_status s = normalize(p, level);
  if (s != GPSOC_OK) return s;
  CK(cudaStreamSynchronize(p->stream));
  p->has_state = true;
  return GPSOC_OK;
}

gpsoc_status gpsoc_set_initial_device(gpsoc_problem* p, const void* dptr, int is_fp32, int level) {
  g_err.clear();
  if (check_problem(p) != GPSOC_OK) return GPSOC_EINVAL;
  if (!dptr) return fail(GPSOC_EINVAL, "dptr is NULL");
  if (level < 0 || level > p->max_level) return fail(GPSOC_EINVAL, "level out of range");
  const Geo g = make_geo(p, level);
  launch_convert<double>(dptr, is_fp32, p->b64.Phi, (long long)p->batch * 3 * g.npts, p->stream);
  mark(p, "convert");
  CK(cudaGetLastError());
  p->level = level;
  gpsoc_status s = normalize(p, level);
  if (s != GPSOC_OK) return s;
  CK(cudaStreamSynchronize(p->stream));
  p->has_state = true;
  return GPSOC_OK;
}

gpsoc_status gpsoc_set_initial_kind(gpsoc_problem* p, const int kind[3], int level) {
  g_err.clear();
  if (check_problem(p) != GPSOC_OK) return GPSOC_EINVAL;
  if (!kind) return fail(GPSOC_EINVAL, "kind is NULL");
  if (level < 0 || level > p->max_level) return fail(GPSOC_EINVAL, "level out of range");
  for (int c = 0; c < 3; ++c) {
    if (kind[c] < 0 || kind[c] > 9) return fail(GPSOC_EINVAL, "guess kind must be in 0..9");
    if (kind[c] == 9) {
      if (p->trap.kind != GPSOC_TRAP_HARMONIC) return fail(GPSOC_EINVAL, "guess (f) needs a harmonic trap");
      for (int b = 0; b < p->batch; ++b)
        if (!(p->params[b].beta0 > 0)) return fail(GPSOC_EINVAL, "guess (f) needs beta0 > 0");
    }
  }
  const Geo g = make_geo(p, level);
  const double PI = 3.14159265358979323846;
  double base;
  if (p->dim == 2) base = 0.5 * std::sqrt(4.0 * p->trap.g[0] * p->trap.g[1] / PI);
  else base = 0.5 * std::pow(15.0 * p->trap.g[0] * p->trap.g[1] * p->trap.g[2] / (4.0 * PI), 0.4);
  TrapDev t = make_trap(p, level);
  launch_guess(p->b64.Phi, g, t, p->d_phys, p->batch, kind, base, p->d_tmp, p->stream);
  p->launches += 3;
  CK(cudaGetLastError());
  p->level = level;
  gpsoc_status s = normalize(p, level);
  if (s != GPSOC_OK) return s;
  CK(cudaStreamSynchronize(p->stream));
  p->has_state = true;
  return GPSOC_OK;
}

gpsoc_status gpsoc_solve(gpsoc_problem* p, const gpsoc_opts* opts, gpsoc_result* results) {
  NvtxRange range("gpsoc_solve");
  g_err.clear();
  if (check_problem(p) != GPSOC_OK) return GPSOC_EINVAL;
  if (!opts) return fail(GPSOC_EINVAL, "opts is NULL");
  if (!p->has_state) return fail(GPSOC_ESTATE, "no initial guess set");
  if (opts->precision != GPSOC_FP64 && opts->precision != GPSOC_MIXED && opts->precision != GPSOC_HYBRID)
    return fail(GPSOC_EINVAL, "unknown precision");
  if (opts->stop < 0 || opts->stop > 3) return fail(GPSOC_EINVAL, "unknown stopping criterion");
  if (opts->precond < 0 || opts->precond > 3) return fail(GPSOC_EINVAL, "unknown preconditioner");
  if (!(opts->tol > 0)) return fail(GPSOC_EINVAL, "tol must be > 0");
  const int levels = opts->cm_levels > 0 ? opts->cm_levels : 1;
  if (levels - 1 > p->max_level) return fail(GPSOC_EINVAL, "too many multigrid levels for this grid");
  if (p->level != levels - 1) return fail(GPSOC_ESTATE, "initial guess is not on the coarsest multigrid level");
  if (levels > 1 && p->d_userV) return fail(GPSOC_EINVAL, "user potentials support single-level solves only");
  const OptsDev o = make_opts(opts);
  const int check = opts->check_every > 0 ? opts->check_every : 16;
  gpsoc_status s = GPSOC_OK;
  p->level_iters.assign(p->batch, std::vector<int>());
  p->level_fp32.assign(p->batch, std::vector<int>());
  p->level_res32.assign(p->batch, std::vector<double>());
  std::vector<int> done(p->batch, 0), done32(p->batch, 0);
  for (int lev = levels - 1; lev >= 0; --lev) {
    if (lev < p->level) {
      s = prolong_impl(p, lev + 1);
      if (s != GPSOC_OK) return s;
    }
    const int lp = level_precision(p, lev, opts);
    s = run_level(p, lev, o, check, lev == levels - 1, lp, opts->fp32_switch > 0 ? opts->fp32_switch : 1e-10,
                  opts->fp32_carry != 0, hy_refresh_every(opts), hy_lead_res(opts));
    if (lp != GPSOC_MIXED)
      for (int i = 0; i < p->batch; ++i) p->level_res32[i].push_back(0.0);
    if (s != GPSOC_OK) return s;
    for (int i = 0; i < p->batch; ++i) {
      p->level_iters[i].push_back(p->h_st[i].total_iters - done[i]);
      p->level_fp32[i].push_back(p->h_st[i].fp32_iters - done32[i]);
      done[i] = p->h_st[i].total_iters;
      done32[i] = p->h_st[i].fp32_iters;
    }
  }
  s = sync_state(p);
  if (s != GPSOC_OK) return s;
  std::vector<gpsoc_result> tmp(p->batch);
  fill_results(p, tmp.data(), levels);
  if (results) std::memcpy(results, tmp.data(), sizeof(gpsoc_result) * p->batch);
  for (int i = 0; i < p->batch; ++i)
    if (tmp[i].status != GPSOC_OK) return fail((gpsoc_status)tmp[i].status, "solve " + std::to_string(i) + " did not converge");
  return GPSOC_OK;
}

gpsoc_status gpsoc_iterate(gpsoc_problem* p, const gpsoc_opts* opts, int iters, int restart, gpsoc_result* results) {
  g_err.clear();
  if (check_problem(p) != GPSOC_OK) return GPSOC_EINVAL;
  if (!opts || iters < 0) return fail(GPSOC_EINVAL, "bad arguments");
  if (opts->precond < 0 || opts->precond > 3) return fail(GPSOC_EINVAL, "unknown preconditioner");
  if (!p->has_state) return fail(GPSOC_ESTATE, "no initial guess set");
  if (opts->precision == GPSOC_HYBRID) {
    // exact FP64 H_lin Phi on the first iteration and every hybrid_refresh iterations
    OptsDev o = make_opts(opts);
    o.no_stop = 1;
    gpsoc_status s = ensure_fp32(p);
    if (s != GPSOC_OK) return s;
    if (restart) {
      s = init_level(p, p->level, true);
      if (s != GPSOC_OK) return s;
    }
    const int every = hy_refresh_every(opts);
    for (int k = 0; k < iters; ++k) {
      s = enqueue_iteration_hy(p, p->level, k & 1, o, k % every == 0);
      if (s != GPSOC_OK) return s;
    }
    if (iters > 0) {
      const Geo g = make_geo(p, p->level);
      HY(p, hy_args(p, p->level, g, scalar_ctx<float>(p, g, o, 2 | 8), iters & 1, GATE_PENDING, HY_UPD));
      ScalarArgs x = scalar_args<float>(p, p->level, PH_CLEAR, g);
      SL(p, x);
      CK(cudaGetLastError());
    }
    s = sync_state(p);
    if (s != GPSOC_OK) return s;
    p->level_iters.assign(p->batch, std::vector<int>());
    p->level_fp32.assign(p->batch, std::vector<int>());
    p->level_res32.assign(p->batch, std::vector<double>());
    if (results) fill_results(p, results, 1);
    return GPSOC_OK;
  }
  if (check_precision(opts->precision) != GPSOC_OK) return GPSOC_EINVAL;
  OptsDev o = make_opts(opts);
  o.no_stop = 1;
  gpsoc_status s;
  const bool f32 = opts->precision == GPSOC_MIXED;
  if (f32) {
    // FP32 arrays (FP64 sums and scalars), from the FP64 state
    s = ensure_fp32(p);
    if (s == GPSOC_OK) s = convert_state(p, p->level, true);
    if (s != GPSOC_OK) return s;
  }
  if (restart) {
    s = init_level(p, p->level, true);
    if (s != GPSOC_OK) return s;
  }
  for (int k = 0; k < iters; ++k) {
    s = f32 ? enqueue_iteration<float>(p, p->level, p->b32, k & 1, o, 1)
            : enqueue_iteration<double>(p, p->level, p->b64, k & 1, o, 0);
    if (s != GPSOC_OK) return s;
  }
  if (iters > 0) {
    s = f32 ? flush_pending<float>(p, p->level, p->b32, (iters - 1) & 1)
            : flush_pending<double>(p, p->level, p->b64, (iters - 1) & 1);
    if (s != GPSOC_OK) return s;
  }
  if (f32) {
    s = convert_state(p, p->level, false);
    if (s != GPSOC_OK) return s;
  }
  s = sync_state(p);
  if (s != GPSOC_OK) return s;
  p->level_iters.assign(p->batch, std::vector<int>());
  p->level_fp32.assign(p->batch, std::vector<int>());
  if (results) fill_results(p, results, 1);
  return GPSOC_OK;
}

gpsoc_status gpsoc_get_psi(const gpsoc_problem* p, double* psi_out) {
  g_err.clear();
  if (!p || !psi_out) return fail(GPSOC_EINVAL, "NULL argument");
  const Geo g = make_geo(p, p->level);
  CK(cudaMemcpyAsync(psi_out, p->b64.Phi, sizeof(double2) * (size_t)p->batch * 3 * g.npts, cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return GPSOC_OK;
}

gpsoc_status gpsoc_get_psi_device(const gpsoc_problem* p, void* dptr) {
  g_err.clear();
  if (!p || !dptr) return fail(GPSOC_EINVAL, "NULL argument");
  const Geo g = make_geo(p, p->level);
  CK(cudaMemcpyAsync(dptr, p->b64.Phi, sizeof(double2) * (size_t)p->batch * 3 * g.npts, cudaMemcpyDeviceToDevice, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return GPSOC_OK;
}

gpsoc_status gpsoc_get_observables(gpsoc_problem* p, double* E, double* mu, double* mass) {
  g_err.clear();
  if (check_problem(p) != GPSOC_OK) return GPSOC_EINVAL;
  if (!p->has_state) return fail(GPSOC_ESTATE, "no state");
  gpsoc_status s = observables_now(p);
  if (s != GPSOC_OK) return s;
  for (int i = 0; i < p->batch; ++i) {
    if (E) E[i] = p->h_st[i].E;
    if (mu) mu[i] = p->h_st[i].mu;
    if (mass) for (int c = 0; c < 3; ++c) mass[3 * i + c] = p->h_st[i].mass[c];
  }
  return GPSOC_OK;
}

gpsoc_status gpsoc_apply_h(gpsoc_problem* p, int precision, double* hpsi, double* obs) {
  g_err.clear();
  if (check_problem(p) != GPSOC_OK) return GPSOC_EINVAL;
  if (check_precision(precision) != GPSOC_OK) return GPSOC_EINVAL;
  if (!p->has_state) return fail(GPSOC_ESTATE, "no state");
  return precision == GPSOC_MIXED ? apply_h_impl<float>(p, hpsi, obs) : apply_h_impl<double>(p, hpsi, obs);
}

gpsoc_status gpsoc_apply_precond(gpsoc_problem* p, int precision, const double* r, double* out) {
  g_err.clear();
  if (check_problem(p) != GPSOC_OK) return GPSOC_EINVAL;
  if (!r || !out) return fail(GPSOC_EINVAL, "NULL argument");
  if (check_precision(precision) != GPSOC_OK) return GPSOC_EINVAL;
  if (!p->has_state) return fail(GPSOC_ESTATE, "no state");
  return precision == GPSOC_MIXED ? apply_precond_impl<float>(p, r, out) : apply_precond_impl<double>(p, r, out);
}

gpsoc_status gpsoc_step_model(gpsoc_problem* p, int precision, const double* P, const double* theta, int n_theta,
                              double* out) {
  g_err.clear();
  if (check_problem(p) != GPSOC_OK) return GPSOC_EINVAL;
  if (!P || !out || n_theta < 0 || (n_theta > 0 && !theta)) return fail(GPSOC_EINVAL, "bad arguments");
  if (check_precision(precision) != GPSOC_OK) return GPSOC_EINVAL;
  if (!p->has_state) return fail(GPSOC_ESTATE, "no state");
  if ((size_t)p->batch * (2 + n_theta) + n_theta > p->tmp_len) return fail(GPSOC_EINVAL, "too many angles");
  return precision == GPSOC_MIXED ? step_model_impl<float>(p, P, theta, n_theta, out)
                                  : step_model_impl<double>(p, P, theta, n_theta, out);
}

gpsoc_status gpsoc_prolong(gpsoc_problem* p, int level) {
  g_err.clear();
  if (check_problem(p) != GPSOC_OK) return GPSOC_EINVAL;
  if (!p->has_state) return fail(GPSOC_ESTATE, "no state");
  if (level < 1 || level > p->max_level || level != p->level) return fail(GPSOC_EINVAL, "level must be the current level and >= 1");
  gpsoc_status s = prolong_impl(p, level);
  if (s != GPSOC_OK) return s;
  CK(cudaStreamSynchronize(p->stream));
  return GPSOC_OK;
}

gpsoc_status gpsoc_profile(gpsoc_problem* p, const gpsoc_opts* opts, int iters, double* ms, int cap, int* n_kernels) {
  g_err.clear();
  if (check_problem(p) != GPSOC_OK) return GPSOC_EINVAL;
  if (!opts || iters < 1 || !ms || !n_kernels) return fail(GPSOC_EINVAL, "bad arguments");
  if (!p->has_state) return fail(GPSOC_ESTATE, "no initial guess set");
  OptsDev o = make_opts(opts);
  o.no_stop = 1;
  gpsoc_status s = init_level(p, p->level, true);
  if (s != GPSOC_OK) return s;
  Tracker tr;
  tr.stream = p->stream;
  tr.events = true;
  p->tr = &tr;
  size_t per = 0;
  std::vector<size_t> starts;
  const bool f32 = (opts->precision == GPSOC_MIXED);
  const bool hy = (opts->precision == GPSOC_HYBRID);
  if (f32 || hy) {
    p->tr = nullptr;
    s = ensure_fp32(p);
    if (s == GPSOC_OK && f32) s = convert_state(p, p->level, true);
    // hybrid: an untimed opening iteration with the exact H_lin Phi, then the timed ones
    if (s == GPSOC_OK && hy) s = enqueue_iteration_hy(p, p->level, 0, o, true);
    p->tr = &tr;
  }
  for (int k = 0; k < iters && s == GPSOC_OK; ++k) {
    starts.push_back(tr.evs.size());
    tr.start();
    if (hy) s = enqueue_iteration_hy(p, p->level, (k + 1) & 1, o, false);
    else if (f32) s = enqueue_iteration<float>(p, p->level, p->b32, k & 1, o, 1);
    else s = enqueue_iteration<double>(p, p->level, p->b64, k & 1, o, 0);
  }
  const int last_par = hy ? (iters & 1) : ((iters - 1) & 1);
  p->tr = nullptr;
  p->launches += tr.count;
  if (s == GPSOC_OK && cudaStreamSynchronize(p->stream) != cudaSuccess) s = fail(GPSOC_ECUDA, "profile sync failed");
  if (s == GPSOC_OK) {
    per = tr.names.size() / iters;
    *n_kernels = (int)per;
    p->prof_names.assign(tr.names.begin(), tr.names.begin() + per);
    for (size_t k = 0; k < per && (int)k < cap; ++k) {
      double acc = 0.0;
      for (int it = 0; it < iters; ++it) {
        float t = 0.f;
        cudaEventElapsedTime(&t, tr.evs[starts[it] + k], tr.evs[starts[it] + k + 1]);
        acc += t;
      }
      ms[k] = acc / iters;
    }
  }
  for (cudaEvent_t e : tr.evs) cudaEventDestroy(e);
  if (s == GPSOC_OK) {
    if (hy) {
      const Geo g = make_geo(p, p->level);
      HY(p, hy_args(p, p->level, g, scalar_ctx<float>(p, g, o, 2 | 8), last_par ^ 1, GATE_PENDING, HY_UPD));
      ScalarArgs x = scalar_args<float>(p, p->level, PH_CLEAR, g);
      SL(p, x);
      CK(cudaGetLastError());
    } else {
      s = f32 ? flush_pending<float>(p, p->level, p->b32, last_par) : flush_pending<double>(p, p->level, p->b64, last_par);
      if (s == GPSOC_OK && f32) s = convert_state(p, p->level, false);
    }
  }
  return s;
}

const char* gpsoc_profile_name(const gpsoc_problem* p, int k) {
  if (!p || k < 0 || k >= (int)p->prof_names.size()) return "";
  return p->prof_names[k].c_str();
}

uint64_t gpsoc_kernel_launches(const gpsoc_problem* p) { return p ? p->launches : 0; }

gpsoc_status gpsoc_tile_candidates(const gpsoc_problem* p, int level, int axis, int precision, int* lines,
                                   int* elems_per_thread, int cap, int* count) {
  g_err.clear();
  if (!p || !count || cap < 0 || (cap > 0 && (!lines || !elems_per_thread))) return fail(GPSOC_EINVAL, "bad arguments");
  if (level < 0 || level > p->max_level || axis < 0 || axis >= p->dim) return fail(GPSOC_EINVAL, "bad level or axis");
  if (precision != GPSOC_FP64 && precision != GPSOC_MIXED && precision != GPSOC_HYBRID)
    return fail(GPSOC_EINVAL, "unknown precision");
  const Geo g = make_geo(p, level);
  *count = (precision == GPSOC_FP64) ? tile_candidates<double>(g, axis, lines, elems_per_thread, cap)
                                     : tile_candidates<float>(g, axis, lines, elems_per_thread, cap);
  return GPSOC_OK;
}

gpsoc_status gpsoc_tuning_set(const gpsoc_problem* p, int level, int axis, int precision, int lines,
                              int elems_per_thread) {
  g_err.clear();
  if (!p) return fail(GPSOC_EINVAL, "NULL problem");
  if (level < 0 || level > p->max_level || axis < 0 || axis >= p->dim) return fail(GPSOC_EINVAL, "bad level or axis");
  if (precision != GPSOC_FP64 && precision != GPSOC_MIXED && precision != GPSOC_HYBRID)
    return fail(GPSOC_EINVAL, "unknown precision");
  if (lines < 0) return fail(GPSOC_EINVAL, "lines must be >= 0");
  const Geo g = make_geo(p, level);
  const bool ok = (precision == GPSOC_FP64) ? tile_set<double>(g, p->batch, axis, lines, elems_per_thread)
                                            : tile_set<float>(g, p->batch, axis, lines, elems_per_thread);
  if (!ok) return fail(GPSOC_EINVAL, "tile does not fit (see gpsoc_tile_candidates)");
  gpsoc_problem* q = const_cast<gpsoc_problem*>(p);
  for (int k = 0; k < 4; ++k)
    if (q->graph[k]) { cudaGraphExecDestroy(q->graph[k]); q->graph[k] = nullptr; }   // captured with the old tiles
  return GPSOC_OK;
}

gpsoc_status gpsoc_autotune(gpsoc_problem* p, const gpsoc_opts* opts, int iters, int* lines, int* elems_per_thread) {
  NvtxRange range("gpsoc_autotune");
  g_err.clear();
  if (check_problem(p) != GPSOC_OK) return GPSOC_EINVAL;
  if (!opts) return fail(GPSOC_EINVAL, "opts is NULL");
  if (!p->has_state) return fail(GPSOC_ESTATE, "no initial guess set");
  if (opts->precision != GPSOC_FP64 && opts->precision != GPSOC_MIXED && opts->precision != GPSOC_HYBRID)
    return fail(GPSOC_EINVAL, "unknown precision");
  if (iters < 1) iters = 6;
  const int prec = opts->precision;
  const int level = p->level;
  const Geo g = make_geo(p, level);
  const size_t bytes = sizeof(double2) * (size_t)p->batch * 3 * g.npts;
  // every candidate starts from the same state (kept in the FP64 scratch D)
  CK(cudaMemcpyAsync(p->b64.D, p->b64.Phi, bytes, cudaMemcpyDeviceToDevice, p->stream));
  std::vector<double> ms(128);
  // average time per iteration of the passes whose tile the axis sets: the column passes
  // of that axis, or (axis 0) every other pass (row tiles also set the elementwise blocks)
  auto time_axis = [&](int axis, double* t) -> gpsoc_status {
    CK(cudaMemcpyAsync(p->b64.Phi, p->b64.D, bytes, cudaMemcpyDeviceToDevice, p->stream));
    int nk = 0;
    const gpsoc_status st = gpsoc_profile(p, opts, iters, ms.data(), (int)ms.size(), &nk);
    if (st != GPSOC_OK) return st;
    *t = 0.0;
    for (int k = 0; k < nk && k < (int)ms.size(); ++k) {
      const std::string& nm = p->prof_names[k];
      const bool col = nm.compare(0, 3, "col") == 0;
      const bool mine = (axis == 0) ? !col : nm.compare(0, 4, axis == 1 ? "coly" : "colz") == 0;
      if (mine) *t += ms[k];
    }
    return GPSOC_OK;
  };
  gpsoc_status s = GPSOC_OK;
  for (int axis = 0; axis < p->dim && s == GPSOC_OK; ++axis) {
    int cl[64], ce[64];
    const int nc = std::min(64, (prec == GPSOC_FP64) ? tile_candidates<double>(g, axis, cl, ce, 64)
                                                     : tile_candidates<float>(g, axis, cl, ce, 64));
    s = gpsoc_tuning_set(p, level, axis, prec, 0, 0);            // the rule first
    double best = 0.0;
    if (s == GPSOC_OK) s = time_axis(axis, &best);
    int bl = 0, be = 0;
    for (int c = 0; c < nc && s == GPSOC_OK; ++c) {
      s = gpsoc_tuning_set(p, level, axis, prec, cl[c], ce[c]);
      double t = 0.0;
      if (s == GPSOC_OK) s = time_axis(axis, &t);
      if (s == GPSOC_OK && t < best) { best = t; bl = cl[c]; be = ce[c]; }
    }
    if (s == GPSOC_OK) s = gpsoc_tuning_set(p, level, axis, prec, bl, be);
  }
  cudaMemcpyAsync(p->b64.Phi, p->b64.D, bytes, cudaMemcpyDeviceToDevice, p->stream);
  if (s != GPSOC_OK) return s;
  CK(cudaStreamSynchronize(p->stream));
  for (int axis = 0; axis < 3; ++axis) {
    int l = 0, e = 0, th = 0;
    if (axis < p->dim) {
      if (prec == GPSOC_FP64) tile_shape<double>(g, axis, p->batch, l, e, th);
      else tile_shape<float>(g, axis, p->batch, l, e, th);
    }
    if (lines) lines[axis] = l;
    if (elems_per_thread) elems_per_thread[axis] = e;
  }
  return GPSOC_OK;
}

gpsoc_status gpsoc_tile_shape(const gpsoc_problem* p, int level, int axis, int precision, int* lines,
                              int* elems_per_thread, int* threads) {
  g_err.clear();
  if (!p || !lines || !elems_per_thread || !threads) return fail(GPSOC_EINVAL, "NULL argument");
  if (level < 0 || level > p->max_level || axis < 0 || axis >= p->dim) return fail(GPSOC_EINVAL, "bad level or axis");
  if (precision != GPSOC_FP64 && precision != GPSOC_MIXED && precision != GPSOC_HYBRID)
    return fail(GPSOC_EINVAL, "unknown precision");
  const Geo g = make_geo(p, level);
  if (precision != GPSOC_FP64) tile_shape<float>(g, axis, p->batch, *lines, *elems_per_thread, *threads);
  else tile_shape<double>(g, axis, p->batch, *lines, *elems_per_thread, *threads);
  return GPSOC_OK;
}

gpsoc_status gpsoc_fft_axis(gpsoc_problem* p, void* data, int count, int axis, int inverse) {
  g_err.clear();
  if (check_problem(p) != GPSOC_OK) return GPSOC_EINVAL;
  if (!data || count < 1 || axis < 0 || axis >= p->dim) return fail(GPSOC_EINVAL, "bad arguments");
  if (count % 3 != 0 || count / 3 > p->batch) return fail(GPSOC_EINVAL, "count must be 3 * k with k <= batch");
  ChainArgs<double> a;
  gpsoc_status s = chain_args<double>(p, 0, a);
  if (s != GPSOC_OK) return s;
  a.gate = GATE_ALL;
  a.nsolve = count / 3;
  double2* d = (double2*)data;
  Launch lc{};
  const double sc = inverse ? 1.0 / a.g.n[axis] : 1.0;
  a.in0 = d; a.out0 = d; a.scale = sc;
  if (axis == 0) RL<double>(p, inverse ? ROW_INV_PLAIN : ROW_FWD_PLAIN, a);
  else CL<double>(p, inverse ? COL_INV : COL_FWD, axis, a);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(p->stream));
  return GPSOC_OK;
}

}  // extern "C"

// =====================================================================================
// Served form: continuous batching of ground-state requests.
//
// Requests are grouped into buckets by (grid, trap, stopping rule, precision
// stage); a bucket is a problem whose batch entries are slots.  Every step
// advances each non-empty bucket by a fixed number of PCG iterations (one graph
// replay per two iterations, each bucket on its own stream so buckets overlap on
// the device), then retires the slots whose solve stopped and refills free
// slots from the queue.  New buckets are created while the device-memory budget
// allows; empty buckets are released when queued requests need the room.
// With GPSOC_MIXED a request first runs in an FP32-stage bucket (FP32 arrays,
// FP64 sums) and then, from its FP32 iterate, in an FP64 bucket to the stopping rule.
// =====================================================================================
namespace {

struct ServerReq {
  uint64_t ticket = 0;
  gpsoc_grid grid{};
  gpsoc_trap trap{};
  gpsoc_params par{};
  gpsoc_opts opts{};
  std::vector<double> psi;     // initial guess, later the state handed from the FP32 stage, finally the result
  int stage = 0;               // 1 = FP32 stage, 2 = FP64 stage, 3 = finished
  int fp32_iters = 0;
  gpsoc_result res{};
};

struct Bucket {
  gpsoc_problem* p = nullptr;
  std::string key;
  int stage = 2;
  OptsDev o{};
  std::vector<int64_t> slot;   // ticket per slot, -1 = free
  size_t bytes = 0;
  cudaEvent_t done = nullptr;  // recorded after the last launched round of iterations
  bool in_flight = false;
  uint64_t launched = 0;       // launch sequence number of the round in flight
  bool hybrid = false;         // GPSOC_HYBRID graphs (FP64 state, FP32 directions)
  bool fp32_phase = false;     // GPSOC_MIXED first stage: FP32 arrays
  int refresh = 16;            // hybrid: iterations between exact recomputations of H_lin Phi
};

bool bucket_empty(const Bucket* b) {
  for (int64_t t : b->slot)
    if (t >= 0) return false;
  return true;
}

void bucket_free(Bucket* b) {
  if (b->done) cudaEventDestroy(b->done);
  gpsoc_destroy(b->p);
  delete b;
}

std::string bucket_key(const ServerReq& r, int stage) {
  char buf[512];
  std::snprintf(buf, sizeof buf, "%d|%d,%d,%d|%.17g,%.17g,%.17g|%d|%.17g,%.17g,%.17g|%.17g|%.17g|%d|%.17g|%.17g|%d|%d|%d",
                r.grid.dim, r.grid.n[0], r.grid.n[1], r.grid.n[2], r.grid.L[0], r.grid.L[1], r.grid.L[2], r.trap.kind,
                r.trap.g[0], r.trap.g[1], r.trap.g[2], r.trap.quad, r.trap.quart, r.opts.stop, r.opts.tol,
                r.opts.res_tol, r.opts.max_iter, r.opts.precond, stage);
  return buf;
}

size_t solve_points(const gpsoc_grid& g) {
  size_t n = 1;
  for (int i = 0; i < g.dim; ++i) n *= (size_t)g.n[i];
  return n;
}

}  // namespace

struct gpsoc_server {
  gpsoc_server_opts opts{};
  std::vector<Bucket*> buckets;
  std::map<uint64_t, ServerReq*> reqs;
  std::vector<uint64_t> queue;   // FIFO of tickets waiting for a slot
  size_t bytes = 0;
  uint64_t next = 1;
  uint64_t rounds = 0;           // rounds of iterations launched, over all buckets
};

namespace {

size_t bucket_bytes(const gpsoc_grid& g, int slots, int stage) {
  const size_t per = sizeof(double2) * 3 * solve_points(g);
  size_t b = 12 * per * (size_t)slots;                     // FP64 working set
  if (stage == 1) b += 14 * (per / 2) * (size_t)slots;     // FP32 working set (FP32 phase or hybrid)
  return b + (4u << 20);
}

gpsoc_status load_slot(Bucket* b, int s, const ServerReq& r) {
  gpsoc_problem* p = b->p;
  const Geo g = make_geo(p, 0);
  const size_t off = (size_t)s * 3 * g.npts;
  CK(cudaMemcpyAsync(p->b64.Phi + off, r.psi.data(), sizeof(double2) * 3 * g.npts, cudaMemcpyHostToDevice, p->stream));
  const PhysDev ph = make_phys(r.par.Omega, r.par.gamma, r.par.beta0, r.par.beta1);
  CK(cudaMemcpyAsync(p->d_phys + s, &ph, sizeof(PhysDev), cudaMemcpyHostToDevice, p->stream));
  ElemArgs<double> e = elem_args<double>(p, g, GATE_ALL);
  e.only = s;
  e.in0 = p->b64.Phi;
  EL<double>(p, EL_MASS, e);
  ScalarArgs x = scalar_args(p, 0, PH_NORM, g);
  x.only = s;
  SL(p, x);
  e.out0 = p->b64.Phi;
  EL<double>(p, EL_SCALE, e);
  ScalarArgs in = scalar_args(p, 0, PH_INIT, g);
  in.only = s;
  in.flags = 1;
  SL(p, in);
  if (b->fp32_phase) {
    launch_convert<float>(p->b64.Phi + off, 0, p->b32.Phi + off, (long long)3 * g.npts, p->stream);
    mark(p, "convert");
  }
  CK(cudaGetLastError());
  // the PCG state of this slot is per solve (first = 1 restarts beta); host parameters follow
  p->params[s] = r.par;
  return GPSOC_OK;
}

gpsoc_status read_slot(Bucket* b, int s, ServerReq& r) {
  gpsoc_problem* p = b->p;
  const Geo g = make_geo(p, 0);
  const size_t off = (size_t)s * 3 * g.npts;
  if (b->fp32_phase) {
    launch_convert<double>(p->b32.Phi + off, 1, p->b64.Phi + off, (long long)3 * g.npts, p->stream);
    mark(p, "convert");
    CK(cudaGetLastError());
  }
  CK(cudaMemcpyAsync(r.psi.data(), p->b64.Phi + off, sizeof(double2) * 3 * g.npts, cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return GPSOC_OK;
}

Bucket* find_or_make_bucket(gpsoc_server* sv, ServerReq& r, int stage, gpsoc_status* err) {
  const std::string key = bucket_key(r, stage);
  for (Bucket* b : sv->buckets) {
    if (b->key != key) continue;
    for (int64_t t : b->slot)
      if (t < 0) return b;
  }
  const int slots = sv->opts.slots_per_bucket > 0 ? sv->opts.slots_per_bucket : 32;
  // FP32 working set: the hybrid stage of GPSOC_HYBRID, the FP32 phase of GPSOC_MIXED
  const bool with32 = (sv->opts.precision == GPSOC_HYBRID) ? (stage == 2) : (stage == 1);
  const size_t need = bucket_bytes(r.grid, slots, with32 ? 1 : 2);
  // release idle empty buckets while the budget is short
  for (size_t i = 0; i < sv->buckets.size() && sv->bytes + need > (size_t)sv->opts.hbm_budget_bytes;) {
    Bucket* b = sv->buckets[i];
    if (bucket_empty(b) && !b->in_flight) {
      sv->bytes -= b->bytes;
      bucket_free(b);
      sv->buckets.erase(sv->buckets.begin() + i);
    } else {
      ++i;
    }
  }
  if (sv->bytes + need > (size_t)sv->opts.hbm_budget_bytes) return nullptr;   // wait for room
  Bucket* b = new Bucket();
  std::vector<gpsoc_params> pars(slots, r.par);
  gpsoc_status s = gpsoc_create(&r.grid, &r.trap, pars.data(), slots, nullptr, &b->p);
  if (s != GPSOC_OK) { delete b; *err = s; return nullptr; }
  // GPSOC_MIXED: stage 1 = FP32 phase; GPSOC_HYBRID: stage 1 = FP64 lead-in, stage 2 = hybrid
  const bool hy_server = (sv->opts.precision == GPSOC_HYBRID);
  b->hybrid = hy_server && stage == 2;
  b->fp32_phase = !hy_server && stage == 1;
  if ((b->fp32_phase || b->hybrid) && ensure_fp32(b->p) != GPSOC_OK) { bucket_free(b); *err = GPSOC_ENOMEM; return nullptr; }
  b->refresh = hy_refresh_every(&r.opts);
  if (cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess) {
    b->done = nullptr;
    bucket_free(b);
    *err = fail(GPSOC_ECUDA, "event create failed");
    return nullptr;
  }
  b->key = key;
  b->stage = stage;
  b->slot.assign(slots, -1);
  b->bytes = need;
  b->o = make_opts(&r.opts);
  if (b->fp32_phase) {
    b->o.stop = GPSOC_STOP_ENERGY;
    b->o.res_tol = 0.0;
    b->o.tol_rel = r.opts.fp32_switch > 0 ? r.opts.fp32_switch : 1e-10;
    b->o.phase32 = 1;
  } else if (hy_server && stage == 1) {
    b->o = lead_opts(b->o, hy_lead_res(&r.opts));
  }
  // every slot starts inactive (gpsoc_create zeroes the per-solve states)
  b->p->level = 0;
  b->p->has_state = true;
  sv->bytes += need;
  sv->buckets.push_back(b);
  return b;
}

}  // namespace

extern "C" {

gpsoc_status gpsoc_server_create(const gpsoc_server_opts* opts, gpsoc_server** out) {
  g_err.clear();
  if (!opts || !out) return fail(GPSOC_EINVAL, "NULL argument");
  if (!(opts->hbm_budget_bytes > 0)) return fail(GPSOC_EINVAL, "hbm_budget_bytes must be > 0");
  if (opts->precision != GPSOC_FP64 && opts->precision != GPSOC_MIXED && opts->precision != GPSOC_HYBRID)
    return fail(GPSOC_EINVAL, "unknown precision");
  gpsoc_server* s = new gpsoc_server();
  s->opts = *opts;
  *out = s;
  return GPSOC_OK;
}

void gpsoc_server_destroy(gpsoc_server* s) {
  if (!s) return;
  for (Bucket* b : s->buckets) bucket_free(b);
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
}

gpsoc_status gpsoc_server_submit(gpsoc_server* s, const gpsoc_grid* grid, const gpsoc_trap* trap,
                                 const gpsoc_params* params, const double* psi0, const gpsoc_opts* opts,
                                 uint64_t* ticket) {
  g_err.clear();
  if (!s || !grid || !trap || !params || !psi0 || !opts || !ticket) return fail(GPSOC_EINVAL, "NULL argument");
  if (trap->kind == GPSOC_TRAP_USER) return fail(GPSOC_EINVAL, "the server takes analytic traps only");
  if (opts->cm_levels > 1) return fail(GPSOC_EINVAL, "the server runs single-level solves (cm_levels = 1)");
  if (!(opts->tol > 0)) return fail(GPSOC_EINVAL, "tol must be > 0");
  if (opts->precond < 0 || opts->precond > 3) return fail(GPSOC_EINVAL, "unknown preconditioner");
  for (int i = 0; i < grid->dim; ++i)
    if (!pow2(grid->n[i]) || grid->n[i] < 8 || grid->n[i] > 1024) return fail(GPSOC_EINVAL, "grid sizes must be powers of two in [8, 1024]");
  if (grid->dim != 2 && grid->dim != 3) return fail(GPSOC_EINVAL, "dim must be 2 or 3");
  ServerReq* r = new ServerReq();
  r->ticket = s->next++;
  r->grid = *grid;
  for (int i = grid->dim; i < 3; ++i) { r->grid.n[i] = 1; r->grid.L[i] = 1.0; }
  r->trap = *trap;
  r->trap.user_V = nullptr;
  r->par = *params;
  r->opts = *opts;
  r->psi.assign(psi0, psi0 + 2 * 3 * solve_points(r->grid));
  const int slots = s->opts.slots_per_bucket > 0 ? s->opts.slots_per_bucket : 32;
  const bool fp32_pays = (long long)slots * (long long)solve_points(r->grid) >= mixed_min_points(opts);
  const bool lead = (s->opts.precision == GPSOC_HYBRID && hy_lead_res(opts) > 0.0);
  r->stage = ((s->opts.precision == GPSOC_MIXED && fp32_pays) || lead) ? 1 : 2;
  s->reqs[r->ticket] = r;
  s->queue.push_back(r->ticket);
  *ticket = r->ticket;
  return GPSOC_OK;
}

}  // extern "C"

namespace {

using Clock = std::chrono::steady_clock;

// One server step (retire, admit, launch).  If no round has finished it waits
// for the earliest-launched one: without limit when `bounded` is false, else
// until `deadline`, after which it goes on to admission and launches without
// retiring anything.
gpsoc_status server_step_impl(gpsoc_server* s, int* busy, bool bounded, Clock::time_point deadline) {
  NvtxRange range("gpsoc server step");
  gpsoc_status err = GPSOC_OK;
  // 1. buckets whose round of iterations finished: retire the solves that stopped.
  //    If no bucket has finished yet, wait for the one launched first.
  bool any_done = false;
  Bucket* oldest = nullptr;
  for (Bucket* b : s->buckets) {
    if (!b->in_flight) continue;
    const cudaError_t q = cudaEventQuery(b->done);
    if (q == cudaSuccess) { any_done = true; continue; }
    if (q != cudaErrorNotReady) return fail(GPSOC_ECUDA, std::string("bucket event: ") + cudaGetErrorString(q));
    if (!oldest || b->launched < oldest->launched) oldest = b;
  }
  if (!any_done && oldest) {
    if (!bounded) {
      CK(cudaEventSynchronize(oldest->done));
    } else {
      for (;;) {
        const cudaError_t q = cudaEventQuery(oldest->done);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) return fail(GPSOC_ECUDA, std::string("bucket event: ") + cudaGetErrorString(q));
        if (Clock::now() >= deadline) break;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
      }
    }
  }
  for (Bucket* b : s->buckets) {
    if (!b->in_flight || cudaEventQuery(b->done) != cudaSuccess) continue;
    b->in_flight = false;
    gpsoc_status st = sync_state(b->p);
    if (st != GPSOC_OK) return st;
    if (b->hybrid) {
      // solves that stopped are accepted on their exact FP64 residual (or resumed)
      bool stopped = false;
      for (size_t k = 0; k < b->slot.size(); ++k)
        stopped |= (b->slot[k] >= 0 && !b->p->h_st[k].active && b->p->h_st[k].status == GPSOC_OK);
      int resumed = 0;
      if (stopped) st = hy_verify(b->p, 0, b->o, &resumed);
      if (st != GPSOC_OK) return st;
    }
    for (size_t k = 0; k < b->slot.size(); ++k) {
      if (b->slot[k] < 0) continue;
      const SolveState& S = b->p->h_st[k];
      if (S.active) continue;
      ServerReq* r = s->reqs[(uint64_t)b->slot[k]];
      st = read_slot(b, (int)k, *r);
      if (st != GPSOC_OK) return st;
      b->slot[k] = -1;
      if (b->stage == 1) {                 // first stage done: continue in the second from this iterate
        r->fp32_iters = S.iters;
        r->stage = 2;
        s->queue.push_back(r->ticket);
        continue;
      }
      gpsoc_result& o = r->res;
      o.status = S.status;
      o.iters = S.iters;
      o.total_iters = S.iters + r->fp32_iters;
      o.levels = 1;
      o.beta_resets = S.beta_resets;
      o.halvings = S.halvings;
      // first-stage iterations: FP32 (GPSOC_MIXED) or the FP64 lead-in (GPSOC_HYBRID)
      o.fp32_iters = b->hybrid ? S.iters : r->fp32_iters;
      o.fp64_iters = b->hybrid ? r->fp32_iters : S.iters;
      o.energy = S.E;
      o.mu = S.mu;
      for (int c = 0; c < 3; ++c) o.mass[c] = S.mass[c];
      o.res_inf = S.res_inf;
      o.dE_last = S.dE_last;
      o.level_iters[0] = o.total_iters;
      o.level_fp32_iters[0] = o.fp32_iters;
      r->stage = 3;
    }
  }
  // 2. admission: fill free slots from the queue, in arrival order (a slot load is
  //    stream-ordered after any round still running in its bucket)
  std::vector<uint64_t> waiting;
  for (uint64_t t : s->queue) {
    ServerReq* r = s->reqs[t];
    Bucket* b = find_or_make_bucket(s, *r, r->stage, &err);
    if (err != GPSOC_OK) return err;
    if (!b) { waiting.push_back(t); continue; }
    int slot = -1;
    for (size_t k = 0; k < b->slot.size(); ++k)
      if (b->slot[k] < 0) { slot = (int)k; break; }
    gpsoc_status st = load_slot(b, slot, *r);
    if (st != GPSOC_OK) return st;
    b->slot[slot] = (int64_t)t;
  }
  s->queue.swap(waiting);
  // 3. every idle bucket that holds work starts its next round on its own stream
  const int iters = s->opts.iters_per_step > 0 ? s->opts.iters_per_step : 32;
  const int pairs = (iters + 1) / 2;
  int n_busy = (int)s->queue.size();
  for (Bucket* b : s->buckets) {
    for (int64_t t : b->slot) n_busy += (t >= 0);
    if (b->in_flight || bucket_empty(b)) continue;
    if (b->hybrid) {
      gpsoc_status st = build_graph_hy(b->p, 0, b->o, false);
      if (st == GPSOC_OK) st = build_graph_hy(b->p, 0, b->o, true);
      if (st != GPSOC_OK) return st;
      const int every = std::max(1, b->refresh / 2);
      for (int r = 0; r < pairs; ++r) {
        const int gk = (r % every == 0) ? 3 : 2;   // every round opens with the exact H_lin Phi
        CK(cudaGraphLaunch(b->p->graph[gk], b->p->stream));
        b->p->launches += b->p->graph_kernels[gk];
      }
    } else {
      const int k = b->fp32_phase ? 1 : 0;
      gpsoc_status st = (k == 1) ? build_graph<float>(b->p, 0, b->o) : build_graph<double>(b->p, 0, b->o);
      if (st != GPSOC_OK) return st;
      for (int r = 0; r < pairs; ++r) {
        CK(cudaGraphLaunch(b->p->graph[k], b->p->stream));
        b->p->launches += b->p->graph_kernels[k];
      }
    }
    CK(cudaEventRecord(b->done, b->p->stream));
    b->in_flight = true;
    b->launched = ++s->rounds;
  }
  if (busy) *busy = n_busy;
  return GPSOC_OK;
}

}  // namespace

extern "C" {

gpsoc_status gpsoc_server_step(gpsoc_server* s, int* busy) {
  g_err.clear();
  if (!s) return fail(GPSOC_EINVAL, "NULL server");
  return server_step_impl(s, busy, false, Clock::now());
}

gpsoc_status gpsoc_server_poll(gpsoc_server* s, uint64_t ticket, int timeout_ms, gpsoc_result* res, double* psi_out) {
  g_err.clear();
  if (!s) return fail(GPSOC_EINVAL, "NULL server");
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return fail(GPSOC_EINVAL, "unknown ticket");
  ServerReq* r = it->second;
  if (r->stage != 3 && timeout_ms != 0) {
    // drive the server until this request finishes or the wait runs out
    const bool bounded = timeout_ms > 0;
    const Clock::time_point deadline = Clock::now() + std::chrono::milliseconds(bounded ? timeout_ms : 0);
    while (r->stage != 3) {
      if (bounded && Clock::now() >= deadline) break;
      int busy = 0;
      const gpsoc_status st = server_step_impl(s, &busy, bounded, deadline);
      if (st != GPSOC_OK) return st;
      if (busy == 0 && r->stage != 3) return fail(GPSOC_ESTATE, "request neither queued nor running");
    }
  }
  if (r->stage != 3) return GPSOC_ETIMEOUT;   // still queued or running (no message: polling is routine)
  if (res) *res = r->res;
  if (psi_out && r->res.status != GPSOC_ECANCELED) std::memcpy(psi_out, r->psi.data(), sizeof(double) * r->psi.size());
  delete r;
  s->reqs.erase(it);
  return GPSOC_OK;
}

gpsoc_status gpsoc_server_cancel(gpsoc_server* s, uint64_t ticket) {
  g_err.clear();
  if (!s) return fail(GPSOC_EINVAL, "NULL server");
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return fail(GPSOC_EINVAL, "unknown ticket");
  ServerReq* r = it->second;
  if (r->stage == 3) return fail(GPSOC_ESTATE, "request already finished");
  bool found = false;
  for (size_t q = 0; q < s->queue.size(); ++q) {
    if (s->queue[q] == ticket) { s->queue.erase(s->queue.begin() + q); found = true; break; }
  }
  for (Bucket* b : s->buckets) {
    if (found) break;
    for (size_t k = 0; k < b->slot.size(); ++k) {
      if (b->slot[k] != (int64_t)ticket) continue;
      // stop the slot's solve on the device, stream-ordered after any round in flight;
      // the slot is free for admission at once (a later load is ordered after this too)
      CK(cudaMemsetAsync(&b->p->d_st[k].active, 0, sizeof(int), b->p->stream));
      b->slot[k] = -1;
      found = true;
      break;
    }
  }
  if (!found) return fail(GPSOC_ESTATE, "request neither queued nor running");
  r->res = gpsoc_result{};
  r->res.status = GPSOC_ECANCELED;
  r->stage = 3;
  return GPSOC_OK;
}

gpsoc_status gpsoc_server_stats(const gpsoc_server* s, double* bytes_in_use, int* buckets, int* queued) {
  if (!s) return GPSOC_EINVAL;
  if (bytes_in_use) *bytes_in_use = (double)s->bytes;
  if (buckets) *buckets = (int)s->buckets.size();
  if (queued) *queued = (int)s->queue.size();
  return GPSOC_OK;
}

}  // extern "C"
