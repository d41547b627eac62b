// Batched shared-memory FFT of short pencils (N <= 128, radices 4, 2, 3, 5),
// with register-resident pencils for the common sizes in FP32 (below).
//
// Self-sorting Stockham formulation: stage s with radix r and span Ns (the
// product of the earlier radices) takes butterfly j in [0, N/r):
//     k   = j mod Ns
//     a_q = x[j + q N/r] * w^(k q N / (Ns r)),   q = 0..r-1,  w = exp(sign 2 pi i / N)
//     y   = DFT_r(a)
//     x'[(j div Ns) Ns r + k + p Ns] = y_p
// After the last stage x' holds the DFT in natural order.  All threads of the
// block share the butterflies of all pencils of the tile; stages ping-pong
// between two shared-memory buffers.
#pragma once

#include "gw_common.cuh"

namespace gw {

template <typename V>
__device__ __forceinline__ V mul_i(V a, int sign) {  // a * (sign * i)
  V r;
  if (sign > 0) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
  return r;
}

template <typename T, int SIGN>
__device__ __forceinline__ void butterfly(cpx<T>* a, int r) {
  using V = cpx<T>;
  if (r == 2) {
    V t = a[0];
    a[0] = cadd(t, a[1]);
    a[1] = csub(t, a[1]);
  } else if (r == 4) {
    V t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
    V t2 = cadd(a[1], a[3]), t3 = mul_i(csub(a[1], a[3]), SIGN);
    a[0] = cadd(t0, t2);
    a[2] = csub(t0, t2);
    a[1] = cadd(t1, t3);
    a[3] = csub(t1, t3);
  } else if (r == 3) {
    const T h = (T)0.86602540378443864676;  // sqrt(3)/2
    V t = cadd(a[1], a[2]);
    V d = mul_i(cscale(csub(a[1], a[2]), h), SIGN);
    V m = csub(a[0], cscale(t, (T)0.5));
    a[0] = cadd(a[0], t);
    a[1] = cadd(m, d);
    a[2] = csub(m, d);
  } else {  // r == 5
    const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;
    const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;
    V t1 = cadd(a[1], a[4]), t2 = cadd(a[2], a[3]);
    V d1 = csub(a[1], a[4]), d2 = csub(a[2], a[3]);
    V m1 = cadd(a[0], cadd(cscale(t1, c1), cscale(t2, c2)));
    V m2 = cadd(a[0], cadd(cscale(t1, c2), cscale(t2, c1)));
    V e1 = mul_i(cadd(cscale(d1, s1), cscale(d2, s2)), SIGN);
    V e2 = mul_i(csub(cscale(d1, s2), cscale(d2, s1)), SIGN);
    a[0] = cadd(a[0], cadd(t1, t2));
    a[1] = cadd(m1, e1);
    a[4] = csub(m1, e1);
    a[2] = cadd(m2, e2);
    a[3] = csub(m2, e2);
  }
}

// Butterfly of a compile-time radix R (2, 3, 4 or 5).
template <typename T, int SIGN, int R>
__device__ __forceinline__ void butterfly_r(cpx<T>* a) {
  butterfly<T, SIGN>(a, R);
}

// One Stockham stage of radix R over npen pencils (see fft_tile2).
template <typename T, int SIGN, bool PFAST, int R>
__device__ __forceinline__ void fft_stage(const cpx<T>* __restrict__ a, cpx<T>* __restrict__ b, int npen, int ps,
                                          int es, int nb, int Ns, int tstep, const FastDiv& dpen,
                                          const FastDiv& dnb, const FastDiv& dns, const cpx<T>* tw) {
  using V = cpx<T>;
  const int total = npen * nb;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    int p, j;
    if (PFAST) { j = dpen.div(t); p = t - j * npen; }
    else { p = dnb.div(t); j = t - p * nb; }
    const int jq = dns.div(j);
    const int k = j - jq * Ns;
    const V* src = a + p * ps;
    V* dst = b + p * ps;
    V v[R];
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = src[(j + q * nb) * es];
    if (k > 0) {
#pragma unroll
      for (int q = 1; q < R; ++q) {
        V w = tw[k * q * tstep];
        if (SIGN > 0) w.y = -w.y;
        v[q] = cmul(v[q], w);
      }
    }
    butterfly_r<T, SIGN, R>(v);
    const int base = jq * Ns * R + k;
#pragma unroll
    for (int q = 0; q < R; ++q) dst[(base + q * Ns) * es] = v[q];
  }
}

// Register-resident pencils for N = L M (M lanes per pencil, L values per
// lane; L in 1..5, M a power of two dividing 32): lane m holds x[m + M l].
// Cooley-Tukey with n = m + M l, k = k1 + L k2:
//   X[k1 + L k2] = sum_m w_M^(m k2) [ w_N^(m k1) sum_l x[m + M l] w_L^(l k1) ],
// the L-point DFTs in each lane's registers, the M-point DFTs across the
// lanes as radix-2 decimation-in-frequency stages with warp shuffles (lane m
// ends with output k2 = bitreverse(m)).  No barrier between stages; the
// result goes to the other buffer.  Every lane of a warp takes part in every
// shuffle (pencils beyond npen run on zeros and store nothing).
template <typename T, int SIGN, int N, int M>
__device__ __forceinline__ cpx<T>* fft_tile_reg(const cpx<T>* __restrict__ a, cpx<T>* __restrict__ b, int npen,
                                                int ps, int es, const cpx<T>* tw) {
  using V = cpx<T>;
  constexpr int L = N / M;
  static_assert(L * M == N && L >= 1 && L <= 5 && (M & (M - 1)) == 0 && M <= 32, "unsupported split");
  constexpr int LOGM = (M >= 32) ? 5 : (M >= 16) ? 4 : (M >= 8) ? 3 : (M >= 4) ? 2 : (M >= 2) ? 1 : 0;
  const int lane = threadIdx.x & (M - 1);
  const int grp = threadIdx.x / M, ngrp = blockDim.x / M;
  const int k2 = (LOGM > 0) ? (int)(__brev((unsigned)lane) >> (32 - LOGM)) : 0;
  for (int base = 0; base < npen; base += ngrp) {
    const int p = base + grp;
    const bool on = p < npen;
    V v[L];
#pragma unroll
    for (int l = 0; l < L; ++l) v[l] = on ? a[p * ps + (lane + M * l) * es] : mk<T>(0, 0);
    if (L > 1) butterfly<T, SIGN>(v, L);
#pragma unroll
    for (int k1 = 1; k1 < L; ++k1) {
      V w = tw[(lane * k1) % N];
      if (SIGN > 0) w.y = -w.y;
      v[k1] = cmul(v[k1], w);
    }
#pragma unroll
    for (int h = M / 2; h >= 1; h >>= 1) {
      const bool bot = (lane & h) != 0;
      V w = tw[(lane & (h - 1)) * (N / (2 * h))];
      if (SIGN > 0) w.y = -w.y;
#pragma unroll
      for (int k1 = 0; k1 < L; ++k1) {
        V o;
        o.x = __shfl_xor_sync(0xffffffffu, v[k1].x, h);
        o.y = __shfl_xor_sync(0xffffffffu, v[k1].y, h);
        v[k1] = bot ? cmul(csub(o, v[k1]), w) : cadd(v[k1], o);
      }
    }
    if (on) {
#pragma unroll
      for (int k1 = 0; k1 < L; ++k1) b[p * ps + (k1 + L * k2) * es] = v[k1];
    }
  }
  __syncthreads();
  return b;
}

// Generalised tile FFT: npen pencils, pencil p element k at buf[p * ps + k * es].
// PFAST selects the thread mapping: consecutive threads take consecutive
// pencils (PFAST, for pencils adjacent in memory: es > 1, ps = 1) or
// consecutive butterflies of one pencil (contiguous pencils: es = 1).  Each
// stage runs a loop specialised for its radix; the index divisions use the
// plan's precomputed multiply-shift divisors.
// Returns the buffer holding the result (a or b).  Ends with __syncthreads().
template <typename T, int SIGN, bool PFAST>
__device__ cpx<T>* fft_tile2(cpx<T>* a, cpx<T>* b, int npen, int ps, int es, const FftPlan& pl,
                             const cpx<T>* tw) {
  using V = cpx<T>;
  const int N = pl.N;
  if (sizeof(T) == 4 && (blockDim.x & 31) == 0) {
    // register-resident pencils for the common grid sizes (FP32: in FP64 the
    // shuffle stages' extra twiddle products cost more than the barriers they
    // save, on this GPU's FP64 rate)
    switch (N) {
      case 16: return fft_tile_reg<T, SIGN, 16, 16>(a, b, npen, ps, es, tw);
      case 24: return fft_tile_reg<T, SIGN, 24, 8>(a, b, npen, ps, es, tw);
      case 32: return fft_tile_reg<T, SIGN, 32, 16>(a, b, npen, ps, es, tw);
      case 40: return fft_tile_reg<T, SIGN, 40, 8>(a, b, npen, ps, es, tw);
      case 48: return fft_tile_reg<T, SIGN, 48, 16>(a, b, npen, ps, es, tw);
      case 64: return fft_tile_reg<T, SIGN, 64, 16>(a, b, npen, ps, es, tw);
      default: break;
    }
  }
  FastDiv dpen = pl.dN;
  if (PFAST && npen != N) dpen.set((unsigned)npen);
  for (int s = 0; s < pl.nst; ++s) {
    const int nb = pl.nb[s];
    const int Ns = pl.ns[s];
    const int tstep = pl.dns[s].div(nb);          // N / (Ns r)
    const FastDiv dnb = pl.dnb[s], dns = pl.dns[s];
    switch (pl.rad[s]) {
      case 4: fft_stage<T, SIGN, PFAST, 4>(a, b, npen, ps, es, nb, Ns, tstep, dpen, dnb, dns, tw); break;
      case 2: fft_stage<T, SIGN, PFAST, 2>(a, b, npen, ps, es, nb, Ns, tstep, dpen, dnb, dns, tw); break;
      case 3: fft_stage<T, SIGN, PFAST, 3>(a, b, npen, ps, es, nb, Ns, tstep, dpen, dnb, dns, tw); break;
      default: fft_stage<T, SIGN, PFAST, 5>(a, b, npen, ps, es, nb, Ns, tstep, dpen, dnb, dns, tw); break;
    }
    __syncthreads();
    V* tmp = a; a = b; b = tmp;
  }
  return a;
}

// npen contiguous pencils of length pl.N at buf[p * ld + k]; tw[k] = exp(-2 pi i k / N).
template <typename T, int SIGN>
__device__ cpx<T>* fft_tile(cpx<T>* a, cpx<T>* b, int npen, int ld, const FftPlan& pl, const cpx<T>* tw) {
  return fft_tile2<T, SIGN, false>(a, b, npen, ld, 1, pl, tw);
}

}  // namespace gw
