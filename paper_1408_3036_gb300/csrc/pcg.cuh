// Device helpers shared by the persistent and the cluster CG kernels.
#pragma once

#include "gw_common.cuh"

namespace gw {

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ double dsum_block_f(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
  return r;   // thread 0
}

// Partial sums of one plane (entries s0 .. s0+ns-1 of the sphere):
//   dp[v] = <C_v|Ap>, dp[nocc + v] = <C_v|p> (v < nocc), dp[2 nocc] = p^H Ap,
// with the plane's Ap (W) and p (P) in shared memory (ACC: add the sums to dp
// instead of storing them).  Warp w takes the
// occupied states v = w, w + warps, ...; its lanes stride over the entries
// with four loads of C in flight, then reduce with shuffles.
template <typename T, bool ACC>
__device__ __forceinline__ void plane_dots(const cpx<T>* __restrict__ C, int npw, int nocc, const cpx<T>* P,
                                           const cpx<T>* W, int s0, int ns, double2* __restrict__ dp,
                                           double* red) {
  using V = cpx<T>;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int v = warp; v < nocc; v += nw) {
    const V* Cv = C + (size_t)v * npw + s0;
    T ax = 0, ay = 0, bx = 0, by = 0;
    int e = lane;
    for (; e + 96 < ns; e += 128) {
      V cv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) cv[u] = Cv[e + 32 * u];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const V y = W[e + 32 * u], q = P[e + 32 * u];
        ax += cv[u].x * y.x + cv[u].y * y.y;        // conj(C) Ap
        ay += cv[u].x * y.y - cv[u].y * y.x;
        bx += cv[u].x * q.x + cv[u].y * q.y;        // conj(C) p
        by += cv[u].x * q.y - cv[u].y * q.x;
      }
    }
    for (; e < ns; e += 32) {
      const V cv = Cv[e], y = W[e], q = P[e];
      ax += cv.x * y.x + cv.y * y.y;
      ay += cv.x * y.y - cv.y * y.x;
      bx += cv.x * q.x + cv.y * q.y;
      by += cv.x * q.y - cv.y * q.x;
    }
    double r0 = ax, r1 = ay, r2 = bx, r3 = by;
    for (int o = 16; o > 0; o >>= 1) {
      r0 += __shfl_xor_sync(0xffffffffu, r0, o);
      r1 += __shfl_xor_sync(0xffffffffu, r1, o);
      r2 += __shfl_xor_sync(0xffffffffu, r2, o);
      r3 += __shfl_xor_sync(0xffffffffu, r3, o);
    }
    if (lane == 0) {
      if (ACC) {
        dp[v].x += r0; dp[v].y += r1;
        dp[nocc + v].x += r2; dp[nocc + v].y += r3;
      } else {
        dp[v] = make_double2(r0, r1);
        dp[nocc + v] = make_double2(r2, r3);
      }
    }
  }
  double t = 0.0;
  for (int e = threadIdx.x; e < ns; e += blockDim.x) {
    const V y = W[e], q = P[e];
    t += (double)(q.x * y.x + q.y * y.y);
  }
  t = dsum_block_f(t, red);
  if (threadIdx.x == 0) {
    if (ACC) dp[2 * nocc].x += t;
    else dp[2 * nocc] = make_double2(t, 0.0);
  }
  __syncthreads();
}

}  // namespace gw
