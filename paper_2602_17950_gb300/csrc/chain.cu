// Spectral passes of the Hamiltonian and preconditioner chains.
//
// A d-dimensional transform is a sequence of 1-D axis passes; each pass loads
// a tile into shared memory, runs Stockham FFTs there and stores back with
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
#include <map>
#include <mutex>

#include "gpsoc_internal.cuh"
#include "scalar.cuh"
#include "fft.cuh"

namespace gpsoc {

static constexpr int kThreads = 384;
// reduction scratch (doubles) behind the tiles: block_reduce needs 16 per warp + 16
static constexpr int kRedDoubles = 16 * (kThreads / 32) + 16;

// Twiddle table in shared memory for transforms with E elements per thread:
// entry (r, j) = W_n^(r j), r < E, j < n/E, at the padded index fft_pad(r n/E + j).
// The last pass (radix E, Ns = n/E) reads j = k for consecutive groups k:
// consecutive addresses; earlier passes read j = k n/(Ns E) for few distinct k.
template <class T>
__device__ __forceinline__ void load_tw(cx_t<T>* s_tw, const cx_t<T>* tw, int n, int ept) {
  const int lc = __ffs(n / ept) - 1;   // log2(n / E): n and E are powers of two
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int r = i >> lc, j = i & ((1 << lc) - 1);
    s_tw[fft_pad<cx_t<T>>(i)] = tw[r * j];
  }
}

// Row tiles: nlines lines of padded length NP; thread -> (line q, group g0), E
// elements per thread.  NI = 2 transforms the same line of buf0 and buf1 together.
template <class C, bool INV, int NI, int E>
__device__ __forceinline__ void row_fft_e(C* buf0, C* buf1, int nlines, int NP, int L, const C* tw) {
  const int G = (1 << L) / E;
  const int q = threadIdx.x / G, g0 = threadIdx.x - q * G;
  const bool act = q < nlines;
  const int qq = act ? q : 0;
  if constexpr (NI == 2) {
    C* const l2[2] = {buf0 + qq * NP, buf1 + qq * NP};
    const bool a2[2] = {act, act};
    stockham_fft<C, INV, E, 2>(l2, a2, g0, 1, L, tw);
  } else {
    C* const l1[1] = {buf0 + qq * NP};
    const bool a1[1] = {act};
    stockham_fft<C, INV, E, 1>(l1, a1, g0, 1, L, tw);
  }
}

// R16: the kernel may run radix-16 passes (FP32 column passes only: the code path
// sets the register allocation of the whole kernel, and FP64 or two-line row
// tiles would lose occupancy to it)
template <class C, bool INV, int NI, bool R16 = false>
__device__ __forceinline__ void row_fft(C* buf0, C* buf1, int nlines, int NP, int L, const C* tw, int ept) {
  if constexpr (R16 && sizeof(C) == 8) {
    if (ept == 16) { row_fft_e<C, INV, NI, 16>(buf0, buf1, nlines, NP, L, tw); return; }
  }
  if (ept == 8) row_fft_e<C, INV, NI, 8>(buf0, buf1, nlines, NP, L, tw);
  else if (ept == 4) row_fft_e<C, INV, NI, 4>(buf0, buf1, nlines, NP, L, tw);
  else row_fft_e<C, INV, NI, 2>(buf0, buf1, nlines, NP, L, tw);
}

// padded length of a column line in shared memory
template <class C> __host__ __device__ __forceinline__ int col_line_len(int n, int tc) {
  // tiles are loaded with consecutive threads on consecutive columns, then on
  // consecutive rows: S complex values fill a 128-byte wavefront, so the line
  // stride is made S / tc modulo S (tc < S) or odd (tc >= S), which puts the
  // values one half-warp (FP32) or quarter-warp (FP64) touches on distinct banks
  constexpr int S = (sizeof(C) == 8) ? 16 : 8;
  const int base = fft_padded_len<C>(n);
  if (tc >= S) return base | 1;
  const int want = S / tc;
  return base + ((want - base % S) + S) % S;
}

// spin terms shared by the pointwise epilogues (working precision W):
//   a = conj(p0) p1 + conj(pm) p0  so that F_-/sqrt2 = a, F_+/sqrt2 = conj(a),
//   F_x = sqrt2 Re a, F_y = -sqrt2 Im a, F_z = |p1|^2 - |pm|^2, |F|^2 = 2|a|^2 + F_z^2.
template <class W, class C1, class C2, class C3>
__device__ __forceinline__ void spin_a(C1 p1, C2 p0, C3 pm, W& ar, W& ai) {
  ar = (W)p0.x * (W)p1.x + (W)p0.y * (W)p1.y + (W)pm.x * (W)p0.x + (W)pm.y * (W)p0.y;
  ai = (W)p0.x * (W)p1.y - (W)p0.y * (W)p1.x + (W)pm.x * (W)p0.y - (W)pm.y * (W)p0.x;
}

template <class W> __device__ __forceinline__ W rsqrt_w(W x);
template <> __device__ __forceinline__ double rsqrt_w<double>(double x) { return rsqrt(x); }
template <> __device__ __forceinline__ float rsqrt_w<float>(float x) { return rsqrtf(x); }

// write per-thread partial sums (working precision) as a deterministic block total in FP64
// (FP32 partials are added in double-float, which carries more bits than the partials hold)
template <int K, class W>
__device__ __forceinline__ void store_partials(const W (&acc)[K], const int (&slots)[K], const bool (&mx)[K],
                                               double* red, double* part, long long sbase_slot, int pmax, int blk) {
  double v[K];
  if constexpr (sizeof(W) == 4 && K >= 2) {
    block_reduce_df<K>(acc, v, red);     // FP32 partials: double-float sums on the FP32 pipes
  } else if constexpr (sizeof(W) == 4) {
    v[0] = block_reduce1_f(acc[0], mx[0], red);
  } else {
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = (double)acc[k];
    block_reduce<K>(v, red, mx);
  }
  put_partials<K>(part, sbase_slot, pmax, blk, slots, v, mx, sizeof(W) == 4);
}

// ============================================================== row passes (x axis)
// Working precision W = T: FP64 kernels compute in double, FP32 kernels in float
// (per-thread partial sums in T, block and grid reductions in FP64).
template <class T, int MODE>
__device__ __forceinline__ void row_pass(const ChainArgs<T>& A, int R, int ept) {
  using C = cx_t<T>;
  using W = T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int last_flag;
  const int nx = A.g.n[0], Lx = A.g.log2n[0];
  const long long npts = A.g.npts;
  const int rows = (int)(npts / nx);
  const int bps = rows / R;
  const int s = blockIdx.x / bps;
  const int rb = blockIdx.x % bps;
  C* s_tw = (C*)smem_raw;
  load_tw<T>(s_tw, A.tw[0], nx, ept);   // constant table: before the wait on the previous kernel
  pdl_wait();
  if (s >= A.nsolve || !gate_ok(A.st, A.gate, s)) return;
  C* buf0 = s_tw + fft_padded_len<C>(nx);
  const int per = R * nx;             // elements of one component in the tile
  const int NP = fft_padded_len<C>(nx), CP = R * NP;   // padded line length, component stride in smem
  constexpr bool two = (MODE == ROW_INV_H || MODE == ROW_INV_P || MODE == ROW_INV_LIN || MODE == ROW_INV_P_HY);
  C* buf1 = buf0 + 3 * CP;
  double* red = (double*)(buf1 + (two ? 3 * CP : 0));
  const long long sbase = (long long)s * 3 * npts;
  const long long rbase = (long long)rb * R * nx;   // offset of the tile inside a component
  const long long sslot = (long long)s * NSLOT;
  const SolveState& S = A.st[s];
  const PhysDev ph = A.phys[s];
  const int ny = A.g.n[1];

  if (MODE == ROW_FWD_PLAIN || MODE == ROW_FWD_UPD || MODE == ROW_FWD_PROJ || MODE == ROW_FWD_PRE ||
      MODE == ROW_FWD_PRE_HY) {
    W acc[1] = {(W)0};
    const W cproj = pick<W>(S.cproj, S.fcproj), mu = A.given_r ? (W)0 : pick<W>(S.mu, S.fmu), beta = pick<W>(S.beta, S.fbeta);
    const bool use_prev = (MODE == ROW_FWD_PROJ) && pick<W>(S.beta, S.fbeta) != (W)0;
    const bool upd = (MODE == ROW_FWD_UPD) && S.pending != 0;
    const W uc = pick<W>(S.upd_c, S.fupd_c), us = pick<W>(S.upd_s, S.fupd_s), usc = pick<W>(S.upd_scale, S.fupd_scale);
    const W al[3] = {pick<W>(S.alpha[0], S.falpha[0]), pick<W>(S.alpha[1], S.falpha[1]), pick<W>(S.alpha[2], S.falpha[2])};
    const W c0 = pick<W>(ph.c0, ph.fc0);
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int r = e / nx, j = e - r * nx;
      const long long off = rbase + e;
      const int pos = r * NP + fft_pad<C>(j);
      if (MODE == ROW_FWD_PLAIN) {
#pragma unroll
        for (int c = 0; c < 3; ++c) buf0[c * CP + pos] = A.in0[sbase + c * npts + off];
      } else if (MODE == ROW_FWD_UPD) {
        // the step accepted by the previous iteration: Phi <- (cos t Phi + sin t P/|P|)/norm
        // (Eqs. formula-pcg, update); reduce max |dPhi|^2 for the stop1 test
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          C f = A.in0[sbase + c * npts + off];
          if (upd) {
            const C p = A.in2[sbase + c * npts + off];
            const C o = mk<C>(usc * (uc * f.x + us * p.x), usc * (uc * f.y + us * p.y));
            const W dr = o.x - f.x, di = o.y - f.y;
            acc[0] = fmax(acc[0], dr * dr + di * di);
            A.out1[sbase + c * npts + off] = o;
            f = o;
          }
          buf0[c * CP + pos] = f;
        }
      } else if (MODE == ROW_FWD_PROJ) {
        // D = -z + beta P_prev, P = D - Re<D, Phi> Phi (Eq. formula-project); reduce ||P||^2
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const C z = A.in0[sbase + c * npts + off];
          const C f = A.in1[sbase + c * npts + off];
          W dr = -z.x, di = -z.y;
          if (use_prev) { const C q = A.in2[sbase + c * npts + off]; dr += beta * q.x; di += beta * q.y; }
          C p;
          p.x = dr - cproj * f.x;
          p.y = di - cproj * f.y;
          A.out1[sbase + c * npts + off] = p;
          acc[0] += p.x * p.x + p.y * p.y;
          buf0[c * CP + pos] = p;
        }
      } else if (MODE == ROW_FWD_PRE_HY) {
        // GPSOC_HYBRID: r = H Phi - mu Phi in FP64 from the FP64 state and H(Phi) (the residual
        // keeps FP64 accuracy), stored as FP32; the preconditioner's transforms then run on
        // P_V^{1/2} r in FP32
        const int pk = A.sc.opts.precond;
        const bool use_pv = (pk == GPSOC_PRECOND_COMBINED || pk == GPSOC_PRECOND_POTENTIAL);
        const double mu64 = S.mu;
        double2 f[3];
        double rho = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          f[c] = A.phi64[sbase + c * npts + off];
          rho += f[c].x * f[c].x + f[c].y * f[c].y;
        }
        const long long row = off / nx;
        const W V = trap_value<W>(A.trap, A.g, j, (int)(row % ny), (int)(row / ny), off);
        const W rhow = (W)rho;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const double2 h = A.hl64[sbase + c * npts + off];
          const double rr = h.x - mu64 * f[c].x, ri = h.y - mu64 * f[c].y;
          const C rc = mk<C>(rr, ri);
          A.out1[sbase + c * npts + off] = rc;
          acc[0] = fmax(acc[0], (W)sqrt((W)(rr * rr + ri * ri)));
          W den = al[c] + V + c0 * rhow;
          den = fmax(den, (W)1e-12 * al[c]);
          const W sc = use_pv ? rsqrt_w<W>(den) : (W)1;
          buf0[c * CP + pos] = mk<C>(rc.x * sc, rc.y * sc);
        }
      } else {  // ROW_FWD_PRE: r = H Phi - mu Phi, then P_V^{1/2} r (Eq. PreCondPot)
        const int pk = A.sc.opts.precond;
        const bool use_pv = (pk == GPSOC_PRECOND_COMBINED || pk == GPSOC_PRECOND_POTENTIAL);
        C f[3], h[3];
        W rho = (W)0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          f[c] = A.in1[sbase + c * npts + off];
          h[c] = A.in0[sbase + c * npts + off];
          rho += f[c].x * f[c].x + f[c].y * f[c].y;
        }
        const long long row = off / nx;
        const W V = trap_value<W>(A.trap, A.g, j, (int)(row % ny), (int)(row / ny), off);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          C rr;
          rr.x = h[c].x - mu * f[c].x;
          rr.y = h[c].y - mu * f[c].y;
          A.out1[sbase + c * npts + off] = rr;
          acc[0] = fmax(acc[0], sqrt(rr.x * rr.x + rr.y * rr.y));
          W den = al[c] + V + c0 * rho;
          den = fmax(den, (W)1e-12 * al[c]);
          const W sc = use_pv ? rsqrt_w<W>(den) : (W)1;
          buf0[c * CP + pos] = mk<C>(rr.x * sc, rr.y * sc);
        }
      }
    }
    __syncthreads();
    row_fft<C, false, 1>(buf0, buf1, 3 * R, NP, Lx, s_tw, ept);
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int pos = (e / nx) * NP + fft_pad<C>(e % nx);
#pragma unroll
      for (int c = 0; c < 3; ++c) A.out0[sbase + c * npts + rbase + e] = buf0[c * CP + pos];
    }
    if (MODE == ROW_FWD_PROJ || MODE == ROW_FWD_PRE || MODE == ROW_FWD_PRE_HY || (MODE == ROW_FWD_UPD && upd)) {
      const bool mx[1] = {MODE != ROW_FWD_PROJ};
      const int slots[1] = {(MODE == ROW_FWD_PROJ) ? (int)SL_P2
                            : (MODE == ROW_FWD_PRE || MODE == ROW_FWD_PRE_HY) ? (int)SL_RINF : (int)SL_DPHIINF};
      store_partials<1, W>(acc, slots, mx, red, A.part, sslot, A.pmax, rb);
    }
    if ((MODE == ROW_FWD_PRE || MODE == ROW_FWD_PRE_HY) && A.fuse && last_block(A.cnt, s, bps, &last_flag))
      sc_res(A.sc, s, red);
    return;
  }

  // ---------------------------------------------------------------- inverse passes
  // natural order in shared memory, inverse transform in place
  for (int e = threadIdx.x; e < per; e += blockDim.x) {
    const int pos = (e / nx) * NP + fft_pad<C>(e % nx);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      buf0[c * CP + pos] = A.in0[sbase + c * npts + rbase + e];
      if (two) buf1[c * CP + pos] = A.in1[sbase + c * npts + rbase + e];
    }
  }
  __syncthreads();
  if (two) row_fft<C, true, 2>(buf0, buf1, 3 * R, NP, Lx, s_tw, ept);
  else row_fft<C, true, 1>(buf0, buf1, 3 * R, NP, Lx, s_tw, ept);

  const W inv_n = (W)1 / (W)npts;
  const W Om = pick<W>(ph.Omega, ph.fOmega);
  if (MODE == ROW_INV_PLAIN) {
    const W sc = (W)A.scale;
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int r = e / nx, j = e - r * nx;
      const int pos = r * NP + fft_pad<C>(j);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const C v = buf0[c * CP + pos];
        A.out0[sbase + c * npts + rbase + e] = mk<C>(v.x * sc, v.y * sc);
      }
    }
    return;
  }
  if (MODE == ROW_INV_PRE) {
    // z = P_V^{1/2} F^-1[...] (Eq. PreCondMix); reduce Re<r, z>, Re<r_prev, z> (beta) and
    // Re<z, Phi>, Re<P_prev, Phi>, Re<r, P_prev> (the direction's projection and slope)
    W acc[5] = {(W)0, (W)0, (W)0, (W)0, (W)0};
    const bool use_prev = (A.in3 != nullptr) && !S.first;
    const int pk = A.sc.opts.precond;
    const bool use_pv = (pk == GPSOC_PRECOND_COMBINED || pk == GPSOC_PRECOND_POTENTIAL);
    const W al[3] = {pick<W>(S.alpha[0], S.falpha[0]), pick<W>(S.alpha[1], S.falpha[1]), pick<W>(S.alpha[2], S.falpha[2])};
    const W c0 = pick<W>(ph.c0, ph.fc0);
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int r = e / nx, j = e - r * nx;
      const int pos = r * NP + fft_pad<C>(j);
      const long long off = rbase + e;
      W rho = (W)0;
      C f[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        f[c] = A.in1[sbase + c * npts + off];
        rho += f[c].x * f[c].x + f[c].y * f[c].y;
      }
      const long long row = off / nx;
      const W V = trap_value<W>(A.trap, A.g, j, (int)(row % ny), (int)(row / ny), off);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        W den = al[c] + V + c0 * rho;
        den = fmax(den, (W)1e-12 * al[c]);
        const W sc = use_pv ? inv_n * rsqrt_w<W>(den) : inv_n;
        const C v = buf0[c * CP + pos];
        const C z = mk<C>(v.x * sc, v.y * sc);
        A.out0[sbase + c * npts + off] = z;
        const C rr = A.in2[sbase + c * npts + off];
        acc[0] += rr.x * z.x + rr.y * z.y;
        acc[2] += z.x * f[c].x + z.y * f[c].y;
        if (use_prev) {
          const C rp = A.in3[sbase + c * npts + off];
          const C pp = A.in4[sbase + c * npts + off];
          acc[1] += rp.x * z.x + rp.y * z.y;
          acc[3] += pp.x * f[c].x + pp.y * f[c].y;
          acc[4] += rr.x * pp.x + rr.y * pp.y;
        }
      }
    }
    const bool mx[5] = {false, false, false, false, false};
    const int slots[5] = {SL_RZ, SL_RPZ, SL_ZPHI, SL_PPHI, SL_RP};
    store_partials<5, W>(acc, slots, mx, red, A.part, sslot, A.pmax, rb);
    if (A.fuse && last_block(A.cnt, s, bps, &last_flag)) sc_beta(A.sc, s, red);
    return;
  }

  // ROW_INV_H / ROW_INV_P / ROW_INV_LIN: lin = F_x^-1(T')/npts - Omega x F_x^-1(G)/npts + V u
  const W c0 = pick<W>(ph.c0, ph.fc0), c1 = pick<W>(ph.c1, ph.fc1);
  double rphi = 0.0, pp64 = 0.0;   // ROW_INV_P_HY: Re<P, Phi> against the FP64 Phi and ||P||^2, summed in FP64
  W acc[13];
#pragma unroll
  for (int k = 0; k < 13; ++k) acc[k] = (W)0;
  for (int e = threadIdx.x; e < per; e += blockDim.x) {
    const int r = e / nx, j = e - r * nx;
    const int pos = r * NP + fft_pad<C>(j);
    const long long off = rbase + e;
    const long long row = off / nx;
    const int iy = (int)(row % ny), iz = (int)(row / ny);
    const W x = coord<W>(A.g, 0, j);
    const W V = trap_value<W>(A.trap, A.g, j, iy, iz, off);
    C u[3];  // Phi for ROW_INV_H, P for ROW_INV_P / ROW_INV_LIN
    W lin_r[3], lin_i[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      u[c] = A.in2[sbase + c * npts + off];
      const C t = buf0[c * CP + pos];
      const C gg = buf1[c * CP + pos];
      lin_r[c] = (t.x - Om * x * gg.x) * inv_n + V * u[c].x;
      lin_i[c] = (t.y - Om * x * gg.y) * inv_n + V * u[c].y;
    }
    if (MODE == ROW_INV_LIN) {
#pragma unroll
      for (int c = 0; c < 3; ++c) A.out0[sbase + c * npts + off] = mk<C>(lin_r[c], lin_i[c]);
      continue;
    }
    if (MODE == ROW_INV_H) {
      // nonlinear terms of Eqs. eigen1-eigen3: c0 rho phi + c1 (F.f) Phi
      W m[3];
      W rho = (W)0;
#pragma unroll
      for (int c = 0; c < 3; ++c) { m[c] = u[c].x * u[c].x + u[c].y * u[c].y; rho += m[c]; }
      W ax, ay;
      spin_a<W>(u[0], u[1], u[2], ax, ay);
      const W Fz = m[0] - m[2];
      // (F.f)Phi: [Fz p1 + a p0, conj(a) p1 + a pm, conj(a) p0 - Fz pm]
      W fr[3], fi[3];
      fr[0] = Fz * u[0].x + (ax * u[1].x - ay * u[1].y);
      fi[0] = Fz * u[0].y + (ax * u[1].y + ay * u[1].x);
      fr[1] = (ax * u[0].x + ay * u[0].y) + (ax * u[2].x - ay * u[2].y);
      fi[1] = (ax * u[0].y - ay * u[0].x) + (ax * u[2].y + ay * u[2].x);
      fr[2] = (ax * u[1].x + ay * u[1].y) - Fz * u[2].x;
      fi[2] = (ax * u[1].y - ay * u[1].x) - Fz * u[2].y;
      W q = (W)0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        q += u[c].x * lin_r[c] + u[c].y * lin_i[c];
        const W hr = lin_r[c] + c0 * rho * u[c].x + c1 * fr[c];
        const W hi = lin_i[c] + c0 * rho * u[c].y + c1 * fi[c];
        A.out0[sbase + c * npts + off] = mk<C>(hr, hi);
        acc[3 + c] += V * m[c];
        acc[6 + c] += rho * m[c];
        acc[9 + c] += m[c];
      }
      acc[0] += q;
      acc[1] += rho * rho;
      acc[2] += (W)2 * (ax * ax + ay * ay) + Fz * Fz;
    } else {  // ROW_INV_P: step-model reductions (Eqs. an, bn and the sin/cos form of E(theta))
      C f[3], h[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) { f[c] = A.in3[sbase + c * npts + off]; h[c] = A.in4[sbase + c * npts + off]; }
      if constexpr (MODE == ROW_INV_P_HY) {
        // H_lin P kept for the update of H_lin Phi by linearity; the radial part of P
        // in FP64 (P's FP32 values against the FP64 Phi) for the exact tangent correction
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          A.out0[sbase + c * npts + off] = mk<C>(lin_r[c], lin_i[c]);
          const double2 g = A.phi64[sbase + c * npts + off];
          const double ux = (double)u[c].x, uy = (double)u[c].y;
          rphi += g.x * ux + g.y * uy;
          pp64 += ux * ux + uy * uy;
        }
      }
      W hpp = (W)0, hphip = (W)0, Rv = (W)0, rf = (W)0, rp = (W)0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        hpp += lin_r[c] * u[c].x + lin_i[c] * u[c].y;
        hphip += h[c].x * u[c].x + h[c].y * u[c].y;
        Rv += f[c].x * u[c].x + f[c].y * u[c].y;
        rf += f[c].x * f[c].x + f[c].y * f[c].y;
        rp += u[c].x * u[c].x + u[c].y * u[c].y;
      }
      // spin vectors F(Phi), F(P) and the symmetric cross term Re F~(Phi, P)
      const W s2 = (W)1.4142135623730951;
      W aFx, aFy, aPx, aPy, a1x, a1y, a2x, a2y;
      spin_a<W>(f[0], f[1], f[2], aFx, aFy);
      spin_a<W>(u[0], u[1], u[2], aPx, aPy);
      // a(Phi + e P) = a(Phi) + e (a1 + a2) + e^2 a(P); Re F~ is half the e coefficient of F
      spin_a<W>(f[0], u[1], f[2], a1x, a1y);
      spin_a<W>(u[0], f[1], u[2], a2x, a2y);
      const W FFx = s2 * aFx, FFy = -s2 * aFy;
      const W FFz = (f[0].x * f[0].x + f[0].y * f[0].y) - (f[2].x * f[2].x + f[2].y * f[2].y);
      const W FPx = s2 * aPx, FPy = -s2 * aPy;
      const W FPz = (u[0].x * u[0].x + u[0].y * u[0].y) - (u[2].x * u[2].x + u[2].y * u[2].y);
      const W FXx = (W)0.5 * s2 * (a1x + a2x), FXy = -(W)0.5 * s2 * (a1y + a2y);
      const W FXz = (f[0].x * u[0].x + f[0].y * u[0].y) - (f[2].x * u[2].x + f[2].y * u[2].y);
      acc[0] += hpp;
      acc[1] += hphip;
      acc[2] += Rv;
      acc[3] += rf * Rv;
      acc[4] += rf * rp;
      acc[5] += Rv * Rv;
      acc[6] += Rv * rp;
      acc[7] += rp * rp;
      acc[8] += FFx * FXx + FFy * FXy + FFz * FXz;
      acc[9] += FFx * FPx + FFy * FPy + FFz * FPz;
      acc[10] += FXx * FXx + FXy * FXy + FXz * FXz;
      acc[11] += FXx * FPx + FXy * FPy + FXz * FPz;
      acc[12] += FPx * FPx + FPy * FPy + FPz * FPz;
    }
  }
  if (MODE == ROW_INV_LIN) return;
  const bool mx[13] = {};
  if (MODE == ROW_INV_H) {
    const W a12[12] = {acc[0], acc[1], acc[2], acc[3], acc[4], acc[5], acc[6], acc[7], acc[8], acc[9], acc[10], acc[11]};
    const bool mx12[12] = {};
    const int slots[12] = {SL_Q, SL_RHO2, SL_F2, SL_V0, SL_V1, SL_V2, SL_C0, SL_C1, SL_C2, SL_M0, SL_M1, SL_M2};
    store_partials<12, W>(a12, slots, mx12, red, A.part, sslot, A.pmax, rb);
    if (A.fuse && last_block(A.cnt, s, bps, &last_flag)) sc_obs(A.sc, s, red);
  } else {
    const int slots[13] = {SL_HPP, SL_HPHIP, SL_RPHI, SL_IFR, SL_IFP, SL_IRR, SL_IRP, SL_IPP,
                           SL_JFR, SL_JFP, SL_JRR, SL_JRP, SL_JPP};
    store_partials<13, W>(acc, slots, mx, red, A.part, sslot, A.pmax, rb);
    if constexpr (MODE == ROW_INV_P_HY) {
      // the normalisation of the step needs these two to FP64 accuracy
      double v2[2] = {rphi, pp64};
      const bool mx2[2] = {false, false};
      block_reduce<2>(v2, red, mx2);
      const int slots2[2] = {SL_RPHI, SL_P2};
      __syncthreads();   // thread 0 of store_partials wrote SL_RPHI's FP32 sum before
      put_partials<2>(A.part, sslot, A.pmax, rb, slots2, v2, mx2, true);
    }
    if (A.fuse && last_block(A.cnt, s, bps, &last_flag)) sc_step(A.sc, s, red);
  }
}

template <class T, int MODE>
__global__ void __launch_bounds__(kThreads) k_row(ChainArgs<T> A, int R, int ept) {
  row_pass<T, MODE>(A, R, ept);
}

// The FP32 inverse passes with fused reductions (the heaviest epilogues) are
// compiled for three blocks of kThreads per SM (at most 56 registers, a few values
// spilled): six 192-thread tiles per SM instead of four.
template <class T, int MODE>
__global__ void __launch_bounds__(kThreads, 3) k_row_lean(ChainArgs<T> A, int R, int ept) {
  row_pass<T, MODE>(A, R, ept);
}

template <class T, int MODE>
constexpr bool row_lean() {
  return sizeof(T) == 4 && (MODE == ROW_INV_H || MODE == ROW_INV_P || MODE == ROW_INV_PRE);
}

// ============================================================== column passes (y or z axis)
// Tile: inner indices [i0, i0 + TC) of the axis-`axis` lines at outer index o, all
// three components.  Shared memory holds every (component, column) line
// contiguously, line (c, t) at (c TC + t) NPL with the padded length NPL of
// col_line_len, so the transforms run exactly as in the row passes and the
// transposing accesses (consecutive threads on consecutive columns) fall on
// distinct banks.
template <class T, int MODE>
__global__ void __launch_bounds__(kThreads) k_col(ChainArgs<T> A, int axis, int TC, int ept) {
  using C = cx_t<T>;
  using W = T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int na = A.g.n[axis], La = A.g.log2n[axis];
  const long long npts = A.g.npts;
  const int ni = (axis == 1) ? A.g.n[0] : A.g.n[0] * A.g.n[1];   // inner (faster) extent
  const int no = (int)(npts / ((long long)na * ni));             // outer (slower) extent
  const int tpo = ni / TC;                                       // tiles per outer index
  const int bps = tpo * no;
  const int s = blockIdx.x / bps;
  const int tb = blockIdx.x % bps;
  C* s_tw = (C*)smem_raw;
  load_tw<T>(s_tw, A.tw[axis], na, ept);   // constant table: before the wait on the previous kernel
  pdl_wait();
  if (s >= A.nsolve || !gate_ok(A.st, A.gate, s)) return;
  const int o = tb / tpo;
  const int i0 = (tb % tpo) * TC;
  C* buf = s_tw + fft_padded_len<C>(na);
  const int per = na * TC;
  const int NPL = col_line_len<C>(na, TC);        // padded line length
  const int CS = TC * NPL;                     // component stride in smem
  C* buf2 = buf + 3 * CS;            // second 3-component tile (YMID_H, YINV_H)
  double* red = (double*)(buf2 + 3 * CS);
  const long long sbase = (long long)s * 3 * npts;
  const long long obase = (long long)o * na * ni + i0;
  const SolveState& S = A.st[s];
  const PhysDev ph = A.phys[s];
  const W piA = geo_piL<W>(A.g, axis);
  const int nx = A.g.n[0];
  // smem index of element j of column t, component c: c * CS + t * NPL + pad(j)
  auto sidx = [&](int c, int t, int j) { return c * CS + t * NPL + fft_pad<C>(j); };

  // load the in0 tile (and in1 for YINV_H) in natural order; global reads coalesced over t
  for (int e = threadIdx.x; e < per; e += blockDim.x) {
    const int j = e / TC, t = e - j * TC;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      buf[sidx(c, t, j)] = A.in0[sbase + c * npts + obase + (long long)j * ni + t];
      if (MODE == COL_YINV_H) buf2[sidx(c, t, j)] = A.in1[sbase + c * npts + obase + (long long)j * ni + t];
    }
  }
  __syncthreads();

  if (MODE == COL_FWD) {
    row_fft<C, false, 1, true>(buf, buf, 3 * TC, NPL, La, s_tw, ept);
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int j = e / TC, t = e - j * TC;
#pragma unroll
      for (int c = 0; c < 3; ++c) A.out0[sbase + c * npts + obase + (long long)j * ni + t] = buf[sidx(c, t, j)];
    }
    return;
  }
  if (MODE == COL_INV) {
    row_fft<C, true, 1, true>(buf, buf, 3 * TC, NPL, La, s_tw, ept);
    const W sc = (W)A.scale;
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int j = e / TC, t = e - j * TC;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const C v = buf[sidx(c, t, j)];
        A.out0[sbase + c * npts + obase + (long long)j * ni + t] = mk<C>(v.x * sc, v.y * sc);
      }
    }
    return;
  }

  // inner index -> (kx [, ky]) wavenumbers (inputs are spectral along the faster axes)
  auto kinner = [&](int t, W& kx, W& ky) {
    const int ii = i0 + t;
    if (axis == 1) { kx = wavenum<W>(ii, nx, geo_piL<W>(A.g, 0)); ky = (W)0; }
    else { kx = wavenum<W>(ii % nx, nx, geo_piL<W>(A.g, 0)); ky = wavenum<W>(ii / nx, A.g.n[1], geo_piL<W>(A.g, 1)); }
  };

  if (MODE == COL_YINV_H) {
    // buf: C -> F_y^-1 C;  buf2: A -> F_y A, times v_y, F_y^-1 -> G
    row_fft<C, true, 1, true>(buf, buf, 3 * TC, NPL, La, s_tw, ept);
    row_fft<C, false, 1, true>(buf2, buf2, 3 * TC, NPL, La, s_tw, ept);
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int j = e / TC, t = e - j * TC;
      const W vy = wavenum<W>(j, na, piA);
#pragma unroll
      for (int c = 0; c < 3; ++c) buf2[sidx(c, t, j)] = cscale(buf2[sidx(c, t, j)], vy);
    }
    __syncthreads();
    row_fft<C, true, 1, true>(buf2, buf2, 3 * TC, NPL, La, s_tw, ept);
    const W nfac = (W)A.g.n[1] * (W)A.g.n[2];  // ny * nz
    const W nz = (W)A.g.n[2];
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int j = e / TC, t = e - j * TC;
      W kx, ky;
      kinner(t, kx, ky);
      const W y = coord<W>(A.g, 1, j);
      const W rot = nfac * pick<W>(ph.Omega, ph.fOmega) * y * kx;
      const long long gi = sbase + obase + (long long)j * ni + t;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const C a = A.in1[gi + c * npts];
        const C cv = buf[sidx(c, t, j)];
        A.out0[gi + c * npts] = mk<C>(cv.x + rot * a.x, cv.y + rot * a.y);
        const C gv = buf2[sidx(c, t, j)];
        A.out1[gi + c * npts] = mk<C>(gv.x * nz, gv.y * nz);
      }
    }
    return;
  }

  // forward transform along the axis: natural-order spectrum in buf
  row_fft<C, false, 1, true>(buf, buf, 3 * TC, NPL, La, s_tw, ept);

  if ((MODE == COL_YMID_H || MODE == COL_MID_H) && A.xhat) {
    // GPSOC_HYBRID P chain: buf holds the full spectrum of P.  Advance the stored spectrum
    // of Phi by the step applied this iteration (Phi_hat <- g (c Phi_hat + t P_hat_prev)),
    // keep this P_hat, and sum 1/2 |k|^2 |Phi_hat_l|^2 and 1/2 |k|^2 Re(Phi_hat_l conj P_hat_l)
    const bool upd = A.khat_upd && S.upd_applied;
    const W uc = pick<W>(S.upd_c, S.fupd_c), us = pick<W>(S.upd_s, S.fupd_s), usc = pick<W>(S.upd_scale, S.fupd_scale);
    W kacc[6] = {(W)0, (W)0, (W)0, (W)0, (W)0, (W)0};
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int j = e / TC, t = e - j * TC;
      W kx, ky, kz = (W)0;
      kinner(t, kx, ky);
      if (axis == 1) ky = wavenum<W>(j, na, piA);
      else kz = wavenum<W>(j, na, piA);
      const W k2h = (W)0.5 * (kx * kx + ky * ky + kz * kz);
      const long long gi = sbase + obase + (long long)j * ni + t;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const C pv = buf[sidx(c, t, j)];
        C xv = A.xhat[gi + c * npts];
        if (upd) {
          const C po = A.phat[gi + c * npts];
          xv = mk<C>(usc * (uc * xv.x + us * po.x), usc * (uc * xv.y + us * po.y));
          A.xhat[gi + c * npts] = xv;
        }
        A.phat[gi + c * npts] = pv;
        kacc[c] += k2h * (xv.x * xv.x + xv.y * xv.y);
        kacc[3 + c] += k2h * (xv.x * pv.x + xv.y * pv.y);
      }
    }
    const bool kmx[6] = {false, false, false, false, false, false};
    const int kslots[6] = {SL_KPHI0, SL_KPHI1, SL_KPHI2, SL_KX0, SL_KX1, SL_KX2};
    store_partials<6, W>(kacc, kslots, kmx, red, A.part, (long long)s * NSLOT, A.pmax, tb);
  }

  if (MODE == COL_YMID_H) {
    // G_c = F_y^-1[v_y F_y A_c] for the three components at once (buf2)
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int j = e / TC, t = e - j * TC;
      const W vy = wavenum<W>(j, na, piA);
#pragma unroll
      for (int c = 0; c < 3; ++c) buf2[sidx(c, t, j)] = cscale(buf[sidx(c, t, j)], vy);
    }
    __syncthreads();
    row_fft<C, true, 1, true>(buf2, buf2, 3 * TC, NPL, La, s_tw, ept);
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int j = e / TC, t = e - j * TC;
#pragma unroll
      for (int c = 0; c < 3; ++c) A.out1[sbase + c * npts + obase + (long long)j * ni + t] = buf2[sidx(c, t, j)];
    }
  }

  W acc[3] = {(W)0, (W)0, (W)0};
  // pointwise in k: the kinetic + SOC symbol (H chains) or the kinetic preconditioner
  const W al[3] = {pick<W>(S.alpha[0], S.falpha[0]), pick<W>(S.alpha[1], S.falpha[1]), pick<W>(S.alpha[2], S.falpha[2])};
  const W g = pick<W>(ph.gamma, ph.fgamma);
  const bool use_pd = (A.sc.opts.precond == GPSOC_PRECOND_COMBINED || A.sc.opts.precond == GPSOC_PRECOND_KINETIC);
  for (int e = threadIdx.x; e < per; e += blockDim.x) {
    const int j = e / TC, t = e - j * TC;
    const int i1 = sidx(0, t, j), i2 = sidx(1, t, j), i3 = sidx(2, t, j);
    W kx, ky, kz = (W)0;
    kinner(t, kx, ky);
    if (axis == 1) ky = wavenum<W>(j, na, piA);
    else kz = wavenum<W>(j, na, piA);
    const W k2h = (W)0.5 * (kx * kx + ky * ky + kz * kz);
    if (MODE == COL_MID_PRE) {
      // P_Delta (Eq. PreCondKin); the potential-only and no-preconditioner variants keep
      // the coefficients (the transform pair is then the identity up to rounding)
      if (use_pd) {
        // the three reciprocals from one division (an FP64 division is a long
        // instruction sequence): 1/d0 = d1 d2 / (d0 d1 d2), and so on
        const W d0 = al[0] + k2h, d1 = al[1] + k2h, d2 = al[2] + k2h;
        const W d01 = d0 * d1;
        const W inv = (W)1 / (d01 * d2);
        const W r01 = d2 * inv;
        buf[i1] = cscale(buf[i1], d1 * r01);
        buf[i2] = cscale(buf[i2], d0 * r01);
        buf[i3] = cscale(buf[i3], d01 * inv);
      }
    } else {
      const C p1 = buf[i1], p0 = buf[i2], pm = buf[i3];
      // kinetic per component (Parseval): sum 1/2 |k|^2 |phat_l|^2
      acc[0] += k2h * (p1.x * p1.x + p1.y * p1.y);
      acc[1] += k2h * (p0.x * p0.x + p0.y * p0.y);
      acc[2] += k2h * (pm.x * pm.x + pm.y * pm.y);
      // -gamma S symbol: s0 = -kx + i ky (L0), s1 = -(kx + i ky) (L1)
      // out_1 = K p1 - g s0 p0 ; out_0 = K p0 - g (s1 p1 + s0 pm) ; out_-1 = K pm - g s1 p0
      const W s0r = -kx, s0i = ky, s1r = -kx, s1i = -ky;
      const W a_r = s0r * p0.x - s0i * p0.y, a_i = s0r * p0.y + s0i * p0.x;   // s0 p0
      const W b_r = s1r * p1.x - s1i * p1.y, b_i = s1r * p1.y + s1i * p1.x;   // s1 p1
      const W c_r = s0r * pm.x - s0i * pm.y, c_i = s0r * pm.y + s0i * pm.x;   // s0 pm
      const W d_r = s1r * p0.x - s1i * p0.y, d_i = s1r * p0.y + s1i * p0.x;   // s1 p0
      buf[i1] = mk<C>(k2h * p1.x - g * a_r, k2h * p1.y - g * a_i);
      buf[i2] = mk<C>(k2h * p0.x - g * (b_r + c_r), k2h * p0.y - g * (b_i + c_i));
      buf[i3] = mk<C>(k2h * pm.x - g * d_r, k2h * pm.y - g * d_i);
    }
  }
  __syncthreads();
  row_fft<C, true, 1, true>(buf, buf, 3 * TC, NPL, La, s_tw, ept);

  const W nrot = (W)A.g.n[1];  // 2D: T' = F_y^-1[M F_y A] + ny Omega y v_x A
  const W Om = pick<W>(ph.Omega, ph.fOmega);
  for (int e = threadIdx.x; e < per; e += blockDim.x) {
    const int j = e / TC, t = e - j * TC;
    const long long gi = sbase + obase + (long long)j * ni + t;
    if (MODE == COL_YMID_H) {
      W kx, ky;
      kinner(t, kx, ky);
      const W y = coord<W>(A.g, 1, j);
      const W rot = nrot * Om * y * kx;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const C a = A.in0[gi + c * npts];
        const C v = buf[sidx(c, t, j)];
        A.out0[gi + c * npts] = mk<C>(v.x + rot * a.x, v.y + rot * a.y);
      }
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) A.out0[gi + c * npts] = buf[sidx(c, t, j)];
    }
  }
  if (MODE == COL_MID_H || MODE == COL_YMID_H) {
    const bool mx[3] = {false, false, false};
    const int slots[3] = {SL_KIN0, SL_KIN1, SL_KIN2};
    store_partials<3, W>(acc, slots, mx, red, A.part, (long long)s * NSLOT, A.pmax, tb);
  }
}

// ============================================================== launch helpers
// Tile shapes: the largest tile (up to 512 elements per row tile, 1024 per
// column tile and component) that still gives the launch at least kTargetBlocks
// blocks over all solves, so small grids and single solves spread over the SMs
// while large batches keep long coalesced line segments.
static constexpr int kTargetBlocks = 304;   // two blocks per SM of a 152-SM GB300

// Tuned tiles (gpsoc_tuning_set / gpsoc_autotune) override the rule below for one
// grid, batch and precision; every launch and every block count of that key reads the
// same table entry, so the passes feeding one fused scalar step always agree.
namespace {
struct TileKey {
  int n0, n1, n2, nsolve, fp32;
  bool operator<(const TileKey& o) const {
    if (n0 != o.n0) return n0 < o.n0;
    if (n1 != o.n1) return n1 < o.n1;
    if (n2 != o.n2) return n2 < o.n2;
    if (nsolve != o.nsolve) return nsolve < o.nsolve;
    return fp32 < o.fp32;
  }
};
struct TileEntry { int lines[3] = {0, 0, 0}, ept[3] = {0, 0, 0}; };
std::map<TileKey, TileEntry> g_tiles;
std::mutex g_tiles_mu;

template <class T> TileKey tile_key(const Geo& g, int nsolve) {
  return TileKey{g.n[0], g.n[1], g.n[2], nsolve, sizeof(T) == 4 ? 1 : 0};
}
// tuned (lines, ept) of an axis, or (0, 0)
template <class T> void tuned(const Geo& g, int axis, int nsolve, int& lines, int& ept) {
  std::lock_guard<std::mutex> lk(g_tiles_mu);
  auto it = g_tiles.find(tile_key<T>(g, nsolve));
  lines = 0; ept = 0;
  if (it != g_tiles.end()) { lines = it->second.lines[axis]; ept = it->second.ept[axis]; }
}
}  // namespace

template <class T>
int row_rows_per_block(const Geo& g, int nsolve) {
  int tl, te;
  tuned<T>(g, 0, nsolve, tl, te);
  if (tl > 0) return tl;
  const int nx = g.n[0];
  const int rows = (int)(g.npts / nx);
  int R = 512 / nx;
  if (R < 1) R = 1;
  if (R > rows) R = rows;
  while (R > 1 && (long long)nsolve * (rows / R) < kTargetBlocks) R >>= 1;
  return R;
}

template <class T>
int col_tc(const Geo& g, int axis, int nsolve) {
  int tl, te;
  tuned<T>(g, axis, nsolve, tl, te);
  if (tl > 0) return tl;
  const int na = g.n[axis];
  const int ni = (axis == 1) ? g.n[0] : g.n[0] * g.n[1];
  const int no = (int)(g.npts / ((long long)na * ni));
  int tc = 1024 / na;
  if (tc < 1) tc = 1;
  if (tc > ni) tc = ni;
  while (tc > 1 && (long long)nsolve * (ni / tc) * no < kTargetBlocks) tc >>= 1;
  return tc;
}

// elements per thread of the FFT passes: 16 (radix-16 passes, FP32 column passes) or 8,
// unless the tile would then have fewer than 128 threads or a line is shorter,
// in which case fewer (more threads, more passes); and the matching thread
// count (multiple of 32, >= 64)
template <class T>
static int pick_ept(int work /* complex elements of the three components */, int n /* line length */,
                    bool r16 = true) {
  int e = (sizeof(T) == 4 && r16) ? 16 : 8;
  while (e > 2 && (work / e < 128 || e > n)) e >>= 1;
  return e;
}
static int round_threads(int t) {
  if (t < 64) t = 64;
  return (t + 31) & ~31;
}

template <class T>
static int row_ept(const Geo& g, int nsolve) {
  int tl, te;
  tuned<T>(g, 0, nsolve, tl, te);
  if (tl > 0 && te > 0) return te;
  return pick_ept<T>(3 * row_rows_per_block<T>(g, nsolve) * g.n[0], g.n[0], false);
}

template <class T>
static void col_cfg(const Geo& g, int axis, int nsolve, int& tc, int& ept, int& threads) {
  tc = col_tc<T>(g, axis, nsolve);
  const int work = 3 * tc * g.n[axis];
  int tl, te;
  tuned<T>(g, axis, nsolve, tl, te);
  ept = (tl > 0 && te > 0) ? te : pick_ept<T>(work, g.n[axis]);
  threads = round_threads(work / ept);
}

template <class T>
void tile_shape(const Geo& g, int axis, int nsolve, int& lines, int& ept, int& threads) {
  if (axis == 0) {
    lines = row_rows_per_block<T>(g, nsolve);
    ept = row_ept<T>(g, nsolve);
    threads = round_threads(3 * lines * g.n[0] / ept);
  } else {
    col_cfg<T>(g, axis, nsolve, lines, ept, threads);
  }
}

// A tile (lines, ept) for the passes along `axis` is valid when the FFT layout fits
// (ept a supported radix no longer than the line; every line of the tile has its
// threads), the block stays within the kernels' thread bound and the shared memory
// of its largest mode stays within the attribute chain_prepare sets.
template <class T>
bool tile_valid(const Geo& g, int axis, int lines, int ept) {
  using C = cx_t<T>;
  const int n = g.n[axis];
  if (lines < 1 || (lines & (lines - 1)) || n < 2) return false;
  const bool r16 = (sizeof(T) == 4 && axis > 0);
  if (!(ept == 2 || ept == 4 || ept == 8 || (ept == 16 && r16)) || ept > n) return false;
  const long long work = 3LL * lines * n;
  if (work / ept > kThreads) return false;
  size_t sm;
  if (axis == 0) {
    const int rows = (int)(g.npts / n);
    if (lines > rows) return false;
    sm = sizeof(C) * (fft_padded_len<C>(n) + 6 * (size_t)lines * fft_padded_len<C>(n)) + kRedDoubles * sizeof(double);
  } else {
    const int ni = (axis == 1) ? g.n[0] : g.n[0] * g.n[1];
    if (lines > ni) return false;
    sm = sizeof(C) * (fft_padded_len<C>(n) + 6 * (size_t)lines * col_line_len<C>(n, lines)) + kRedDoubles * sizeof(double);
  }
  return sm <= 200 * 1024;
}

// set (lines > 0) or clear (lines = 0) the tuned tile of one axis
template <class T>
bool tile_set(const Geo& g, int nsolve, int axis, int lines, int ept) {
  if (axis < 0 || axis >= g.d) return false;
  if (lines > 0 && !tile_valid<T>(g, axis, lines, ept)) return false;
  std::lock_guard<std::mutex> lk(g_tiles_mu);
  TileEntry& e = g_tiles[tile_key<T>(g, nsolve)];
  e.lines[axis] = lines > 0 ? lines : 0;
  e.ept[axis] = lines > 0 ? ept : 0;
  return true;
}

// every valid tile of an axis: powers of two for the lines, each supported radix
template <class T>
int tile_candidates(const Geo& g, int axis, int* lines, int* ept, int cap) {
  int k = 0;
  for (int l = 1; l <= 4096; l <<= 1)
    for (int e = 2; e <= 16; e <<= 1)
      if (tile_valid<T>(g, axis, l, e)) {
        if (k < cap) { lines[k] = l; ept[k] = e; }
        ++k;
      }
  return k;
}

template <class T>
int row_blocks_per_solve(const Geo& g, int nsolve) {
  return (int)(g.npts / g.n[0]) / row_rows_per_block<T>(g, nsolve);
}

template <class T>
int col_blocks_per_solve(const Geo& g, int axis, int nsolve) {
  const int na = g.n[axis];
  const int ni = (axis == 1) ? g.n[0] : g.n[0] * g.n[1];
  const int no = (int)(g.npts / ((long long)na * ni));
  return (ni / col_tc<T>(g, axis, nsolve)) * no;
}

template <class T>
static size_t row_smem(const Geo& g, int mode, int nsolve) {
  using C = cx_t<T>;
  const int R = row_rows_per_block<T>(g, nsolve);
  const int per = R * g.n[0];
  const bool two = (mode == ROW_INV_H || mode == ROW_INV_P || mode == ROW_INV_LIN || mode == ROW_INV_P_HY);
  (void)per;
  const int CP = R * fft_padded_len<C>(g.n[0]);
  return sizeof(C) * (fft_padded_len<C>(g.n[0]) + 3 * CP * (two ? 2 : 1)) + kRedDoubles * sizeof(double);
}

template <class T>
static size_t col_smem(const Geo& g, int axis, int nsolve) {
  using C = cx_t<T>;
  const int tc = col_tc<T>(g, axis, nsolve);
  const int CS = col_line_len<C>(g.n[axis], tc) * tc;
  return sizeof(C) * (fft_padded_len<C>(g.n[axis]) + 6 * CS) + kRedDoubles * sizeof(double);
}

template <class T, int MODE>
static void row_go(const ChainArgs<T>& a, cudaStream_t st) {
  const int R = row_rows_per_block<T>(a.g, a.nsolve);
  const int nb = row_blocks_per_solve<T>(a.g, a.nsolve) * a.nsolve;
  const size_t sm = row_smem<T>(a.g, MODE, a.nsolve);
  const int ept = row_ept<T>(a.g, a.nsolve);
  const int threads = round_threads(3 * R * a.g.n[0] / ept);
  if constexpr (row_lean<T, MODE>())
    launch_pdl(k_row_lean<T, MODE>, nb, threads, sm, st, a, R, ept);
  else
    launch_pdl(k_row<T, MODE>, nb, threads, sm, st, a, R, ept);
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
    case ROW_FWD_UPD: row_go<T, ROW_FWD_UPD>(a, st); break;
    case ROW_FWD_PRE_HY: row_go<T, ROW_FWD_PRE_HY>(a, st); break;
    case ROW_INV_P_HY: row_go<T, ROW_INV_P_HY>(a, st); break;
  }
}

template <class T, int MODE>
static void col_go(int axis, const ChainArgs<T>& a, cudaStream_t st) {
  int tc, ept, threads;
  col_cfg<T>(a.g, axis, a.nsolve, tc, ept, threads);
  const int nb = col_blocks_per_solve<T>(a.g, axis, a.nsolve) * a.nsolve;
  const size_t sm = col_smem<T>(a.g, axis, a.nsolve);
  launch_pdl(k_col<T, MODE>, nb, threads, sm, st, a, axis, tc, ept);
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
  GPSOC_ATTR((k_row<T, ROW_INV_PLAIN>)) GPSOC_ATTR((k_row<T, ROW_INV_LIN>)) GPSOC_ATTR((k_row<T, ROW_FWD_UPD>))
  GPSOC_ATTR((k_row<T, ROW_FWD_PRE_HY>)) GPSOC_ATTR((k_row<T, ROW_INV_P_HY>))
  GPSOC_ATTR((k_col<T, COL_FWD>)) GPSOC_ATTR((k_col<T, COL_INV>)) GPSOC_ATTR((k_col<T, COL_MID_H>))
  GPSOC_ATTR((k_col<T, COL_MID_PRE>)) GPSOC_ATTR((k_col<T, COL_YMID_H>)) GPSOC_ATTR((k_col<T, COL_YINV_H>))
  if constexpr (sizeof(T) == 4) {
    GPSOC_ATTR((k_row_lean<T, ROW_INV_H>)) GPSOC_ATTR((k_row_lean<T, ROW_INV_P>)) GPSOC_ATTR((k_row_lean<T, ROW_INV_PRE>))
  }
#undef GPSOC_ATTR
  return e;
}

template void launch_row<double>(int, const ChainArgs<double>&, int, const Launch&, cudaStream_t);
template void launch_row<float>(int, const ChainArgs<float>&, int, const Launch&, cudaStream_t);
template void launch_col<double>(int, int, const ChainArgs<double>&, const Launch&, cudaStream_t);
template void launch_col<float>(int, int, const ChainArgs<float>&, const Launch&, cudaStream_t);
template bool tile_set<double>(const Geo&, int, int, int, int);
template bool tile_set<float>(const Geo&, int, int, int, int);
template int tile_candidates<double>(const Geo&, int, int*, int*, int);
template int tile_candidates<float>(const Geo&, int, int*, int*, int);
template void tile_shape<double>(const Geo&, int, int, int&, int&, int&);
template void tile_shape<float>(const Geo&, int, int, int&, int&, int&);
template int row_blocks_per_solve<double>(const Geo&, int);
template int row_blocks_per_solve<float>(const Geo&, int);
template int col_blocks_per_solve<double>(const Geo&, int, int);
template int col_blocks_per_solve<float>(const Geo&, int, int);
template cudaError_t chain_prepare<double>();
template cudaError_t chain_prepare<float>();

}  // namespace gpsoc
