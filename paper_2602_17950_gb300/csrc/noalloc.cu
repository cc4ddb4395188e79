// Allocation-free variant of gpsoc_apply_h.
//
// Some callers cannot allocate device memory at the point where they need the
// Hamiltonian: a host framework that has already handed all device memory to its
// own pool, a real-time loop that must not pay for (or synchronise on)
// cudaMalloc/cudaFree, or code running under a fixed memory budget that has been
// reserved up front.  gpsoc_apply_h_noalloc serves them: it takes the wave
// functions and the output buffer from the caller and keeps every intermediate
// array, partial sum, twiddle table and per-solve scalar in one file-scope device
// array of fixed size, kNoAllocScratchBytes, that exists once per GPU from the
// moment the library is loaded until the process exits.
//
// Nothing here allocates: no cudaMalloc, cudaFree, cudaMallocHost or host heap
// (failures are reported through the returned status only; gpsoc_last_error
// is not updated by this call).
// The device address of the array is looked up once per device with
// cudaGetSymbolAddress (the host-side name of a __device__ array is only a
// stand-in and must never be handed to a kernel).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "gpsoc_internal.cuh"
#include "kernels.cuh"

using namespace gpsoc;

static constexpr size_t kNoAllocScratchBytes = 16u << 20;   // 16 MiB per device

// the scratch of every call; in host code this name is a stand-in, not a device address
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;

unsigned char* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// device address of the scratch array on the current device (set up on first use)
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    e = chain_prepare<double>();   // kernel attributes (idempotent)
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = (unsigned char*)p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

__global__ void k_gather_obs(const SolveState* st, int batch, double* out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= batch) return;
  const SolveState& S = st[s];
  double* o = out + 9 * s;
  o[0] = S.E; o[1] = S.mu;
  for (int c = 0; c < 3; ++c) { o[2 + c] = S.alpha[c]; o[5 + c] = S.mass[c]; }
  o[8] = S.Q;
}

__global__ void k_init_state(SolveState* st, int batch) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= batch) return;
  SolveState z{};
  z.active = 1;
  st[s] = z;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int ilog2i(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }

}  // namespace

extern "C" gpsoc_status gpsoc_apply_h_noalloc(const gpsoc_grid* grid, const gpsoc_trap* trap,
                                              const gpsoc_params* params, int batch, const void* d_psi,
                                              void* d_hpsi, double* obs, void* cuda_stream) {
  if (!grid || !trap || !params || !d_psi || !d_hpsi || batch < 1) return GPSOC_EINVAL;
  if (grid->dim != 2 && grid->dim != 3) return GPSOC_EINVAL;
  // the same trap checks as gpsoc_create; user potentials would need device memory of their own
  if (trap->kind != GPSOC_TRAP_HARMONIC && trap->kind != GPSOC_TRAP_HARMONIC_QUARTIC) return GPSOC_EINVAL;
  for (int i = 0; i < grid->dim; ++i)
    if (!std::isfinite(trap->g[i])) return GPSOC_EINVAL;
  if (!std::isfinite(trap->quad) || !std::isfinite(trap->quart)) return GPSOC_EINVAL;
  Geo g{};
  g.d = grid->dim;
  g.npts = 1;
  g.dV = 1.0;
  for (int i = 0; i < 3; ++i) {
    if (i < grid->dim) {
      const int n = grid->n[i];
      if (n < 8 || n > 1024 || (n & (n - 1))) return GPSOC_EINVAL;
      if (!(grid->L[i] > 0) || !std::isfinite(grid->L[i])) return GPSOC_EINVAL;
      g.n[i] = n;
      g.L[i] = grid->L[i];
      g.h[i] = 2.0 * grid->L[i] / n;
      g.piL[i] = 3.14159265358979323846 / grid->L[i];
      g.dV *= g.h[i];
    } else {
      g.n[i] = 1; g.L[i] = 1.0; g.h[i] = 1.0; g.piL[i] = 0.0;
    }
    g.log2n[i] = ilog2i(g.n[i]);
    g.npts *= g.n[i];
  }
  // scratch layout: A, B, W, G arrays | partial sums | states | parameters | twiddles | observables
  const size_t arr = sizeof(double2) * (size_t)batch * 3 * g.npts;
  const int nb_row = row_blocks_per_solve<double>(g, batch);
  int pmax = nb_row;
  for (int ax = 1; ax < g.d; ++ax) pmax = std::max(pmax, col_blocks_per_solve<double>(g, ax, batch));
  size_t off = 0;
  const size_t o_arr = off; off += align256(4 * arr);
  const size_t o_part = off; off += align256(sizeof(double) * (size_t)batch * NSLOT * pmax);
  const size_t o_st = off; off += align256(sizeof(SolveState) * batch);
  const size_t o_ph = off; off += align256(sizeof(PhysDev) * batch);
  size_t o_tw[3];
  for (int i = 0; i < g.d; ++i) { o_tw[i] = off; off += align256(sizeof(double2) * g.n[i]); }
  const size_t o_obs = off; off += align256(sizeof(double) * 9 * batch);
  if (off > kNoAllocScratchBytes) {
    return GPSOC_EBUDGET;
  }
  unsigned char* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return GPSOC_ECUDA;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double2* A = (double2*)(base + o_arr);
  double2* Bb = A + (size_t)batch * 3 * g.npts;
  double2* W = Bb + (size_t)batch * 3 * g.npts;
  double2* G = W + (size_t)batch * 3 * g.npts;
  double* part = (double*)(base + o_part);
  SolveState* sst = (SolveState*)(base + o_st);
  PhysDev* ph = (PhysDev*)(base + o_ph);
  double* dobs = (double*)(base + o_obs);
  // parameters and twiddle tables from stack buffers (copied before cudaMemcpyAsync returns)
  PhysDev phs[64];
  for (int b0 = 0; b0 < batch; b0 += 64) {
    const int nb = std::min(64, batch - b0);
    for (int k = 0; k < nb; ++k) {
      const gpsoc_params& q = params[b0 + k];
      if (!std::isfinite(q.Omega) || !std::isfinite(q.gamma) || !std::isfinite(q.beta0) || !std::isfinite(q.beta1)) {
        return GPSOC_EINVAL;
      }
      phs[k] = make_phys(q.Omega, q.gamma, q.beta0, q.beta1);
    }
    e = cudaMemcpyAsync(ph + b0, phs, sizeof(PhysDev) * nb, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return GPSOC_ECUDA;
  }
  double2 tw[1024];
  const double PI = 3.14159265358979323846;
  ChainArgs<double> a{};
  for (int i = 0; i < g.d; ++i) {
    const int n = g.n[i];
    for (int k = 0; k < n; ++k) {
      // exp(-2 pi i k / n) from the first octant by symmetry (exact at multiples of n/4)
      int m = k, quad = 0;
      while (m > n / 4) { m -= n / 4; ++quad; }
      double c, sn;
      if (2 * m <= n / 4) { const double ang = 2.0 * PI * m / n; c = std::cos(ang); sn = std::sin(ang); }
      else { const double ang = 2.0 * PI * (n / 4 - m) / n; c = std::sin(ang); sn = std::cos(ang); }
      double re = c, im = -sn;
      for (int q = 0; q < quad; ++q) { const double t = re; re = im; im = -t; }
      tw[k] = make_double2(re, im);
    }
    e = cudaMemcpyAsync(base + o_tw[i], tw, sizeof(double2) * n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return GPSOC_ECUDA;
    a.tw[i] = (const double2*)(base + o_tw[i]);
  }
  k_init_state<<<(batch + 127) / 128, 128, 0, st>>>(sst, batch);
  a.g = g;
  for (int i = 0; i < 3; ++i) a.trap.half_g2[i] = (i < g.d) ? 0.5 * trap->g[i] * trap->g[i] : 0.0;
  a.trap.quad = (trap->kind == GPSOC_TRAP_HARMONIC) ? 0.0 : trap->quad;
  a.trap.quart = (trap->kind == GPSOC_TRAP_HARMONIC) ? 0.0 : trap->quart;
  a.trap.userV = nullptr;
  a.phys = ph;
  a.st = sst;
  a.part = part;
  a.pmax = pmax;
  a.gate = GATE_ALL;
  a.nsolve = batch;
  a.scale = 1.0;
  // the Hamiltonian chain of gpsoc_apply_h, on the caller's buffers and the scratch
  const double2* src = (const double2*)d_psi;
  a.in0 = src; a.out0 = A;
  launch_row<double>(ROW_FWD_PLAIN, a, 0, Launch{}, st);
  if (g.d == 2) {
    a.in0 = A; a.out0 = W; a.out1 = G;
    launch_col<double>(COL_YMID_H, 1, a, Launch{}, st);
  } else {
    a.in0 = A; a.out0 = Bb; a.out1 = nullptr;
    launch_col<double>(COL_FWD, 1, a, Launch{}, st);
    a.in0 = Bb; a.out0 = Bb;
    launch_col<double>(COL_MID_H, 2, a, Launch{}, st);
    a.in0 = Bb; a.in1 = A; a.out0 = W; a.out1 = G;
    launch_col<double>(COL_YINV_H, 1, a, Launch{}, st);
  }
  a.in0 = W; a.in1 = G; a.in2 = src; a.out0 = (double2*)d_hpsi; a.out1 = nullptr;
  launch_row<double>(ROW_INV_H, a, 0, Launch{}, st);
  ScalarArgs x{};
  x.st = sst; x.phys = ph; x.part = part; x.pmax = pmax;
  x.nb_row = nb_row;
  x.nb_col = col_blocks_per_solve<double>(g, g.d - 1, batch);
  x.nsolve = batch; x.phase = PH_OBS; x.npts = g.npts; x.dV = g.dV; x.force = 1;
  x.inv_npts = 1.0 / (double)g.npts;
  launch_scalar(x, st);
  k_gather_obs<<<(batch + 127) / 128, 128, 0, st>>>(sst, batch, dobs);
  e = cudaGetLastError();
  if (e != cudaSuccess) return GPSOC_ECUDA;
  if (obs) {
    e = cudaMemcpyAsync(obs, dobs, sizeof(double) * 9 * batch, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return GPSOC_ECUDA;
  }
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return GPSOC_ECUDA;
  return GPSOC_OK;
}
