// Shared-memory Stockham FFTs, radix 16 or 8 (plus one smaller pass when log2 N
// is not a multiple of 4 or 3), natural order in and out.
//
// Transform convention (Section 3.2): forward X_k = sum_m x_m exp(-2 pi i k m / N),
// inverse with exp(+...) and no 1/N (callers fold the 1/N into their epilogues).
//
// A pass of radix R with Ns = product of the radices of the earlier passes
// treats group g in [0, N/R): it reads x[g + r N/R] (r < R), multiplies element r
// by W_N^(r k N / (Ns R)) with k = g mod Ns, takes the R-point DFT and writes
// output q to x[(g / Ns) Ns R + k + q Ns].  Every pass reads all values into
// registers, synchronises, then writes: the transform runs in place.
//
// Lines are padded in shared memory, element e at e + (e >> 4) for 8-byte and
// e + (e >> 3) for 16-byte complex values: the contiguous reads of every pass
// and the strided writes of the first pass then avoid bank conflicts.  tw holds
// W_N^(r j) = exp(-2 pi i r j / N) for r < E, j < N/E at the padded index
// fft_pad(r N/E + j) (E = elements per thread, the radix of the last pass).
#pragma once

#include "gpsoc_internal.cuh"

namespace gpsoc {

// one gap per 16 elements for 8-byte complex values (a half-warp's 16 consecutive
// elements fill one 128-byte wavefront), one per 8 for 16-byte values
template <class C> constexpr int kPadShift = (sizeof(C) == 8) ? 4 : 3;
template <class C> __host__ __device__ __forceinline__ int fft_pad(int e) { return e + (e >> kPadShift<C>); }
template <class C> __host__ __device__ __forceinline__ int fft_padded_len(int n) { return n + (n >> kPadShift<C>); }

template <class C> __device__ __forceinline__ C cmul_conj_if(C a, C w, bool conj) {
  if (conj) w.y = -w.y;
  return cmul(a, w);
}

// multiply by -i (forward) or +i (inverse)
template <class C, bool INV> __device__ __forceinline__ C mul_mi(C a) {
  C r;
  if (INV) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
  return r;
}

template <class C, bool INV> __device__ __forceinline__ void dft2(C& a, C& b) {
  const C t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

// 4-point DFT of (v0, v1, v2, v3) in place, natural output order
template <class C, bool INV> __device__ __forceinline__ void dft4(C& v0, C& v1, C& v2, C& v3) {
  const C a0 = cadd(v0, v2), a1 = csub(v0, v2);
  const C a2 = cadd(v1, v3), a3 = mul_mi<C, INV>(csub(v1, v3));
  v0 = cadd(a0, a2);
  v2 = csub(a0, a2);
  v1 = cadd(a1, a3);
  v3 = csub(a1, a3);
}

// 8-point DFT in place: two 4-point DFTs (even / odd inputs) combined with W_8^q
template <class C, bool INV> __device__ __forceinline__ void dft8(C (&v)[8]) {
  using R = decltype(v[0].x);
  C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<C, INV>(e0, e1, e2, e3);
  dft4<C, INV>(o0, o1, o2, o3);
  const R h = (R)0.70710678118654752440;
  // W_8^1 = (1 - i)/sqrt2, W_8^2 = -i, W_8^3 = (-1 - i)/sqrt2 (conjugated for the inverse)
  C t1, t3;
  if (INV) {
    t1.x = h * (o1.x - o1.y); t1.y = h * (o1.y + o1.x);
    t3.x = -h * (o3.x + o3.y); t3.y = h * (o3.x - o3.y);
  } else {
    t1.x = h * (o1.x + o1.y); t1.y = h * (o1.y - o1.x);
    t3.x = h * (o3.y - o3.x); t3.y = -h * (o3.x + o3.y);
  }
  const C t2 = mul_mi<C, INV>(o2);
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[1] = cadd(e1, t1); v[5] = csub(e1, t1);
  v[2] = cadd(e2, t2); v[6] = csub(e2, t2);
  v[3] = cadd(e3, t3); v[7] = csub(e3, t3);
}

// v * exp(-i a) (forward) or v * exp(+i a) (inverse) for a constant angle with
// cos a = c, sin a = s
template <class C, bool INV, class R> __device__ __forceinline__ C rot_const(C v, R c, R s) {
  C r;
  if (INV) { r.x = v.x * c - v.y * s; r.y = v.y * c + v.x * s; }
  else { r.x = v.x * c + v.y * s; r.y = v.y * c - v.x * s; }
  return r;
}

// 16-point DFT in place: four 4-point DFTs over n1 (stride 4), the twiddles
// W_16^(n2 k1), four 4-point DFTs over n2; output k = k1 + 4 k2 in natural order
template <class C, bool INV> __device__ __forceinline__ void dft16(C (&v)[16]) {
  using R = decltype(v[0].x);
  const R c1 = (R)0.92387953251128675613, s1 = (R)0.38268343236508977173, h = (R)0.70710678118654752440;
  C a[4][4];   // a[n2][k1]
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    C x0 = v[n2], x1 = v[4 + n2], x2 = v[8 + n2], x3 = v[12 + n2];
    dft4<C, INV>(x0, x1, x2, x3);
    a[n2][0] = x0; a[n2][1] = x1; a[n2][2] = x2; a[n2][3] = x3;
  }
  // W_16^m for m = n2 k1: 1, 2, 3 (n2 = 1); 2, 4, 6 (n2 = 2); 3, 6, 9 (n2 = 3)
  a[1][1] = rot_const<C, INV>(a[1][1], c1, s1);
  a[1][2] = rot_const<C, INV>(a[1][2], h, h);
  a[1][3] = rot_const<C, INV>(a[1][3], s1, c1);
  a[2][1] = rot_const<C, INV>(a[2][1], h, h);
  a[2][2] = mul_mi<C, INV>(a[2][2]);
  a[2][3] = rot_const<C, INV>(a[2][3], -h, h);
  a[3][1] = rot_const<C, INV>(a[3][1], s1, c1);
  a[3][2] = rot_const<C, INV>(a[3][2], -h, h);
  a[3][3] = rot_const<C, INV>(a[3][3], -c1, -s1);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    C y0 = a[0][k1], y1 = a[1][k1], y2 = a[2][k1], y3 = a[3][k1];
    dft4<C, INV>(y0, y1, y2, y3);
    v[k1] = y0; v[k1 + 4] = y1; v[k1 + 8] = y2; v[k1 + 12] = y3;
  }
}

// DFT of radix R on the R values starting at v[off] (R in {2, 4, 8, 16})
template <class C, bool INV, int R, int E> __device__ __forceinline__ void dftR(C (&v)[E], int off) {
  if constexpr (R == 16) {
    C w[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) w[r] = v[off + r];
    dft16<C, INV>(w);
#pragma unroll
    for (int r = 0; r < 16; ++r) v[off + r] = w[r];
  } else if constexpr (R == 8) {
    C w[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) w[r] = v[off + r];
    dft8<C, INV>(w);
#pragma unroll
    for (int r = 0; r < 8; ++r) v[off + r] = w[r];
  } else if constexpr (R == 4) {
    dft4<C, INV>(v[off], v[off + 1], v[off + 2], v[off + 3]);
  } else {
    dft2<C, INV>(v[off], v[off + 1]);
  }
}

// One Stockham pass of radix R for NI work items per thread holding E elements
// each (E >= R).  Item it of this thread covers line lines[it] (element stride
// es, padded indices) and the E/R groups g0 + u N/E (u < E/R).  Inactive items
// only take part in the barriers.
template <class C, bool INV, int R, int E, int NI>
__device__ __forceinline__ void stockham_pass(C* const (&lines)[NI], const bool (&active)[NI], int g0, int es, int N,
                                              int Ns, const C* tw) {
  constexpr int PER = E / R;   // radix-R groups handled by one item
  C v[NI][E];
  const int NR = N / R;
#pragma unroll
  for (int it = 0; it < NI; ++it) {
    if (!active[it]) continue;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int g = g0 + u * (N / E);
#pragma unroll
      for (int r = 0; r < R; ++r) v[it][u * R + r] = lines[it][fft_pad<C>(g + r * NR) * es];
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < NI; ++it) {
    if (!active[it]) continue;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int g = g0 + u * (N / E);
      const int k = g % Ns;
      if (k != 0) {
        // W_N^(r k N / (Ns R)): entry (r, k N / (Ns R)) of the table (R = E here:
        // only the first pass, with k = 0, can have a smaller radix)
        const int j = k * (N / (Ns * R));
#pragma unroll
        for (int r = 1; r < R; ++r)
          v[it][u * R + r] = cmul_conj_if(v[it][u * R + r], tw[fft_pad<C>(r * (N / E) + j)], INV);
      }
      dftR<C, INV, R, E>(v[it], u * R);
      const int ob = (g / Ns) * Ns * R + k;
#pragma unroll
      for (int q = 0; q < R; ++q) lines[it][fft_pad<C>(ob + q * Ns) * es] = v[it][u * R + q];
    }
  }
  __syncthreads();
}

// Full transform of length N = 2^L (N >= E) for the NI lines of this thread, E
// elements per thread and pass (E in {2, 4, 8, 16}: radix-E passes plus one smaller
// pass when log2 N is not a multiple of log2 E).  Threads with g0 >= N/E (or
// inactive items) only join the barriers.
template <class C, bool INV, int E, int NI>
__device__ __forceinline__ void stockham_fft(C* const (&lines)[NI], const bool (&active_in)[NI], int g0, int es, int L,
                                             const C* tw) {
  const int N = 1 << L;
  bool active[NI];
#pragma unroll
  for (int it = 0; it < NI; ++it) active[it] = active_in[it] && g0 < (N / E);
  int Ns = 1;
  constexpr int LE = (E == 16) ? 4 : (E == 8) ? 3 : (E == 4) ? 2 : 1;
  const int rem = L % LE;
  if (rem == 1) { stockham_pass<C, INV, 2, E, NI>(lines, active, g0, es, N, Ns, tw); Ns *= 2; }
  else if (rem == 2) { stockham_pass<C, INV, 4, E, NI>(lines, active, g0, es, N, Ns, tw); Ns *= 4; }
  else if constexpr (E == 16) {
    if (rem == 3) { stockham_pass<C, INV, 8, E, NI>(lines, active, g0, es, N, Ns, tw); Ns *= 8; }
  }
  for (int p = 0; p < L / LE; ++p) { stockham_pass<C, INV, E, E, NI>(lines, active, g0, es, N, Ns, tw); Ns *= E; }
}

}  // namespace gpsoc
