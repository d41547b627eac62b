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
// instead of storing them).  Warp w takes the occupied states v = w and
// w + warps (then w + 2 warps, ...); its lanes stride over the entries with
// the loads of C for both states and eight entries in flight together, then
// reduce with shuffles.
template <typename T, bool ACC>
__device__ __forceinline__ void plane_dots(const cpx<T>* __restrict__ C, int npw, int nocc, const cpx<T>* P,
                                           const cpx<T>* W, int s0, int ns, double2* __restrict__ dp,
                                           double* red) {
  using V = cpx<T>;
  constexpr int UE = 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int v0 = warp; v0 < nocc; v0 += 2 * nw) {
    const int v1 = v0 + nw;
    const bool two = v1 < nocc;
    const V* C0 = C + (size_t)v0 * npw + s0;
    const V* C1 = C + (size_t)(two ? v1 : v0) * npw + s0;
    T a0x = 0, a0y = 0, b0x = 0, b0y = 0, a1x = 0, a1y = 0, b1x = 0, b1y = 0;
    for (int e0 = lane; e0 < ns; e0 += 32 * UE) {
      V c0[UE], c1[UE];
#pragma unroll
      for (int u = 0; u < UE; ++u) {
        const int e = e0 + 32 * u;
        c0[u] = (e < ns) ? C0[e] : mk<T>(0, 0);
        c1[u] = (e < ns && two) ? C1[e] : mk<T>(0, 0);
      }
#pragma unroll
      for (int u = 0; u < UE; ++u) {
        const int e = e0 + 32 * u;
        if (e < ns) {
          const V y = W[e], q = P[e];
          a0x += c0[u].x * y.x + c0[u].y * y.y;      // conj(C) Ap
          a0y += c0[u].x * y.y - c0[u].y * y.x;
          b0x += c0[u].x * q.x + c0[u].y * q.y;      // conj(C) p
          b0y += c0[u].x * q.y - c0[u].y * q.x;
          a1x += c1[u].x * y.x + c1[u].y * y.y;
          a1y += c1[u].x * y.y - c1[u].y * y.x;
          b1x += c1[u].x * q.x + c1[u].y * q.y;
          b1y += c1[u].x * q.y - c1[u].y * q.x;
        }
      }
    }
    double r[8] = {(double)a0x, (double)a0y, (double)b0x, (double)b0y,
                   (double)a1x, (double)a1y, (double)b1x, (double)b1y};
#pragma unroll
    for (int k = 0; k < 8; ++k)
      for (int o = 16; o > 0; o >>= 1) r[k] += __shfl_xor_sync(0xffffffffu, r[k], o);
    if (lane == 0) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h == 1 && !two) break;
        const int v = h ? v1 : v0;
        if (ACC) {
          dp[v].x += r[4 * h]; dp[v].y += r[4 * h + 1];
          dp[nocc + v].x += r[4 * h + 2]; dp[nocc + v].y += r[4 * h + 3];
        } else {
          dp[v] = make_double2(r[4 * h], r[4 * h + 1]);
          dp[nocc + v] = make_double2(r[4 * h + 2], r[4 * h + 3]);
        }
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

// Block sum in the precision T of the vectors (result in thread 0).  For the
// positive sums of a CG update (|r|^2, r^H K r over a chunk) FP32 keeps the
// relative accuracy of its terms; FP64 arithmetic is scarce on this GPU.
template <typename T>
__device__ __forceinline__ T tsum_block(T v, T* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  T r = (T)0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
  return r;   // thread 0
}

// Record of one plane's partial sums for the grid-wide kernel: the 2 nocc
// projector sums <C_v|Ap>, <C_v|p> in the precision T of the vectors, then
// p^H Ap in FP64 (the one sum whose value can be much smaller than its terms
// when H - e_v is badly conditioned).
__host__ __device__ inline size_t plane_rec_bytes(int nocc, int csize) {
  return ((2 * (size_t)nocc * csize + 15) & ~(size_t)15) + 16;
}

// As plane_dots, writing one record (plane_rec_bytes): the projector sums
// reduced over the warp in T, p^H Ap accumulated per thread in T over the
// thread's one or two entries and reduced over the block in FP64.
template <typename T>
__device__ __forceinline__ void plane_dots_rec(const cpx<T>* __restrict__ C, int npw, int nocc, const cpx<T>* P,
                                               const cpx<T>* W, int s0, int ns, unsigned char* __restrict__ rec,
                                               double* red) {
  using V = cpx<T>;
  constexpr int UE = 8;
  V* pc = reinterpret_cast<V*>(rec);
  double* pap = reinterpret_cast<double*>(rec + plane_rec_bytes(nocc, (int)sizeof(V)) - 16);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int v0 = warp; v0 < nocc; v0 += 2 * nw) {
    const int v1 = v0 + nw;
    const bool two = v1 < nocc;
    const V* C0 = C + (size_t)v0 * npw + s0;
    const V* C1 = C + (size_t)(two ? v1 : v0) * npw + s0;
    T r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int e0 = lane; e0 < ns; e0 += 32 * UE) {
      V c0[UE], c1[UE];
#pragma unroll
      for (int u = 0; u < UE; ++u) {
        const int e = e0 + 32 * u;
        c0[u] = (e < ns) ? C0[e] : mk<T>(0, 0);
        c1[u] = (e < ns && two) ? C1[e] : mk<T>(0, 0);
      }
#pragma unroll
      for (int u = 0; u < UE; ++u) {
        const int e = e0 + 32 * u;
        if (e < ns) {
          const V y = W[e], q = P[e];
          r[0] += c0[u].x * y.x + c0[u].y * y.y;      // conj(C) Ap
          r[1] += c0[u].x * y.y - c0[u].y * y.x;
          r[2] += c0[u].x * q.x + c0[u].y * q.y;      // conj(C) p
          r[3] += c0[u].x * q.y - c0[u].y * q.x;
          r[4] += c1[u].x * y.x + c1[u].y * y.y;
          r[5] += c1[u].x * y.y - c1[u].y * y.x;
          r[6] += c1[u].x * q.x + c1[u].y * q.y;
          r[7] += c1[u].x * q.y - c1[u].y * q.x;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k)
      for (int o = 16; o > 0; o >>= 1) r[k] += __shfl_xor_sync(0xffffffffu, r[k], o);
    if (lane == 0) {
      pc[v0] = mk<T>(r[0], r[1]);
      pc[nocc + v0] = mk<T>(r[2], r[3]);
      if (two) {
        pc[v1] = mk<T>(r[4], r[5]);
        pc[nocc + v1] = mk<T>(r[6], r[7]);
      }
    }
  }
  T t = (T)0;
  for (int e = threadIdx.x; e < ns; e += blockDim.x) {
    const V y = W[e], q = P[e];
    t += q.x * y.x + q.y * y.y;
  }
  const double tt = dsum_block_f((double)t, red);
  if (threadIdx.x == 0) *pap = tt;
  __syncthreads();
}

}  // namespace gw
