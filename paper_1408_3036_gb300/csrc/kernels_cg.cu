// Persistent conjugate-gradient solver for the Sternheimer equations
// (Eq. P2: (H - e_v -/+ w) x = P_c psi_v* dV, projected on the conduction
// space at every step as in Sec. Avoiding summations).
//
// One cooperative launch runs a whole CG pass for every column (occupied
// state x field x frequency) with per-column convergence masks.  The CTAs are
// all resident and step through four phases per iteration, separated by a
// grid barrier (bounded spin: a barrier that waits too long sets an error flag
// and every CTA returns):
//   A  per (column, plane i0): p = K r + beta p on the plane's sphere entries
//      (K: kinetic preconditioner, 1 without one),
//      scatter, z-IFFT of the disc rows, y-IFFT of the plane (all in shared
//      memory), store the plane
//   B  per (column, i1, 16 i2): x-IFFT, * V(r)/N_g, x-FFT (planes of the sphere)
//   C  per (column, plane): y-FFT, z-FFT of the disc rows, gather the sphere
//      entries, Ap = (Vp)_G + (|G|^2/2 - E) p_G, the plane's partial sums
//      <C_v|Ap>, <C_v|p> and p^H Ap
//   E  per (column, 1024 entries): coef = sum of the plane partials,
//      p^H P_c A p = p^H A p - sum_v conj(<C_v|p>) coef_v, alpha = r^H K r /
//      p^H P_c A p, x += alpha p, r -= alpha (Ap - C coef) (P_c on the fly),
//      partials |r|^2 and r^H K r
// After E every CTA sums the partials of every column in the same order, so
// all CTAs take the same convergence decisions without another barrier.
#include <algorithm>
#include <cstdio>

#include <mutex>

#include "fft.cuh"
#include "gw_common.cuh"
#include "linalg.cuh"
#include "pcg.cuh"

namespace gw {

constexpr int kPT = 256;        // threads per CTA

template <typename T>
struct PcgArgs {
  Geometry g;
  FftPlan pl;
  const cpx<T>* tw;
  const T* kin;
  const T* vloc_s;
  const cpx<T>* C;
  int nocc, npw, ncol, nchunk, chunk;   // phases 0 and E: nchunk tasks of chunk entries per column
  const double2* b64;
  const int* outer_active;
  const double2* E;
  const double* rr_abs;
  double tol_in2;
  int maxit;
  cpx<T>* x;
  cpx<T>* r;
  cpx<T>* p;
  cpx<T>* Ap;
  cpx<T>* grid;
  double2* dpart;   // [ncol][nplanes][2 nocc + 1] plane partial sums
  double* ppart;    // [ncol][nchunk]: entry 0 of a column holds p^H P_c A p
  double* rpart;    // [ncol][nchunk]
  double* zpart;    // [ncol][nchunk] partial r^H K r
  const double* tk; // per-column T_ref of the kinetic preconditioner, or null (none)
  unsigned* bar;
  int* err;
  int* iters_out;
  int* flag_out;
  double* rr_out;
  unsigned long long* ptime;   // optional [16] phase timing (see the kernel)
  unsigned long long spin_limit;   // spins of one barrier wait before the error flag is set
};

__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* err, unsigned nblk,
                                             unsigned long long limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned old = atomicAdd(bar, 1u);
    const unsigned target = (old / nblk + 1u) * nblk;
    unsigned long long spins = 0;
    int good = 1;
    while (*(volatile unsigned*)bar < target) {
      if (*(volatile int*)err) { good = 0; break; }
      if (++spins > limit) { atomicExch(err, 1); good = 0; break; }
      __nanosleep(64);
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

template <typename T>
__device__ __forceinline__ double dsum_block(double v, double* sh) {
  return dsum_block_f(v, sh);
}

// Copies n elements (e = 0..n-1, strided over the block) with U loads in
// flight per thread: every load of a round is issued before the first store.
constexpr int kLd = 4;
template <int U, typename X, typename Ld, typename St>
__device__ __forceinline__ void staged_copy(int n, Ld ld, St st) {
  for (int e0 = threadIdx.x; e0 < n; e0 += U * (int)blockDim.x) {
    X t[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * (int)blockDim.x;
      if (e < n) t[u] = ld(e);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * (int)blockDim.x;
      if (e < n) st(e, t[u]);
    }
  }
}

// Per column c: s[c] = sum of rp[c][0 .. n), z[c] = sum of zp[c][0 .. n), one
// warp per column (lane l adds records l, l + 32, ... in order, then a fixed
// shuffle tree; lane 0's value is kept), so that every CTA gets the same bits.
__device__ __forceinline__ void column_sums(const double* __restrict__ rp, const double* __restrict__ zp, int n,
                                            int ncol, double* s, double* z) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int c = warp; c < ncol; c += nw) {
    double a = 0.0, b = 0.0;
    for (int k = lane; k < n; k += 32) {
      a += rp[(size_t)c * n + k];
      b += zp[(size_t)c * n + k];
    }
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) { s[c] = a; z[c] = b; }
  }
  __syncthreads();
}

struct PcgLayout {
  size_t dbl, ints, red, coef, tv, tw, A, B, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline PcgLayout pcg_layout(int N, int ncol, int nocc, int vsize) {
  PcgLayout L;
  L.dbl = 0;
  L.ints = align16(L.dbl + (size_t)8 * ncol * sizeof(double));
  L.red = align16(L.ints + (size_t)(4 * ncol + N) * sizeof(int));
  L.coef = align16(L.red + 32 * sizeof(double));
  L.tv = align16(L.coef + (size_t)(2 * nocc + 1) * 2 * sizeof(double));
  L.tw = align16(L.tv + align16((size_t)(ncol + 1) * (vsize / 2)) + (size_t)2 * nocc * vsize);
  L.A = align16(L.tw + (size_t)N * vsize);
  L.B = align16(L.A + (size_t)N * (N + 1) * vsize);
  L.total = align16(L.B + (size_t)N * (N + 1) * vsize);
  return L;
}

template <typename T>
__global__ void __launch_bounds__(kPT, 2) k_cg_persistent(PcgArgs<T> a) {
  using V = cpx<T>;
  extern __shared__ unsigned char smem_raw[];
  const Geometry& g = a.g;
  const int N = g.N, LDp = N + 1;
  const int ncol = a.ncol;
  // ---- shared memory: column state, then the FFT work area (offsets: pcg_layout)
  const PcgLayout L = pcg_layout(N, ncol, a.nocc, (int)sizeof(V));
  double* st_rr = reinterpret_cast<double*>(smem_raw + L.dbl);
  double* st_min = st_rr + ncol;
  double* st_stop = st_min + ncol;
  double* st_beta = st_stop + ncol;
  double* st_rz = st_beta + ncol;                             // r^H K r
  double* st_best = st_rz + ncol;                             // stagnation guard
  double* st_s = st_best + ncol;                              // this iteration's |r|^2 and r^H K r
  double* st_z = st_s + ncol;
  int* st_act = reinterpret_cast<int*>(smem_raw + L.ints);
  int* st_it = st_act + ncol;
  int* st_flag = st_it + ncol;
  int* st_itb = st_flag + ncol;
  int* rowmap = st_itb + ncol;                                // [N]
  double* red = reinterpret_cast<double*>(smem_raw + L.red);  // [32] block sums
  double2* coef = reinterpret_cast<double2*>(smem_raw + L.coef);  // [2 nocc + 1] plane sums
  T* st_rtk = reinterpret_cast<T*>(smem_raw + L.tv);          // [ncol] 1 / T_ref (0: no preconditioner)
  T* s_al = st_rtk + ncol;                                    // alpha of the current column
  V* coefT = reinterpret_cast<V*>(smem_raw + L.tv + align16((size_t)(ncol + 1) * sizeof(T)));   // [2 nocc]
  T* redT = reinterpret_cast<T*>(red);
  V* stw = reinterpret_cast<V*>(smem_raw + L.tw);             // [N]
  V* A = reinterpret_cast<V*>(smem_raw + L.A);                // [N][LDp]
  V* B = reinterpret_cast<V*>(smem_raw + L.B);                // [N][LDp]
  __shared__ double bcast;

  for (int k = threadIdx.x; k < N; k += blockDim.x) stw[k] = a.tw[k];
  for (int c = threadIdx.x; c < ncol; c += blockDim.x) st_rtk[c] = a.tk ? (T)1 / (T)a.tk[c] : (T)0;
  __syncthreads();
  const unsigned nblk = gridDim.x;
  const int npl = g.nplanes;

  // ---- phase 0: r = b, x = 0, partial |b|^2
  for (int task = blockIdx.x; task < ncol * a.nchunk; task += gridDim.x) {
    const int c = task / a.nchunk, ch = task - c * a.nchunk;
    const bool on = !a.outer_active || a.outer_active[c];
    const int g0 = ch * a.chunk, g1 = min(a.npw, g0 + a.chunk);
    const T rtk = st_rtk[c];
    T acc = 0, accz = 0;
    for (int G = g0 + threadIdx.x; G < g1; G += blockDim.x) {
      const size_t i = (size_t)c * a.npw + G;
      const V bv = on ? from_d<T>(a.b64[i]) : mk<T>(0, 0);
      a.r[i] = bv;
      a.x[i] = mk<T>(0, 0);
      const T n2 = bv.x * bv.x + bv.y * bv.y;
      acc += n2;
      accz += (rtk != (T)0 ? tpa<T>(a.kin[G] * rtk) : (T)1) * n2;
    }
    acc = tsum_block<T>(acc, redT);
    if (threadIdx.x == 0) a.rpart[(size_t)c * a.nchunk + ch] = (double)acc;
    accz = tsum_block<T>(accz, redT);
    if (threadIdx.x == 0) a.zpart[(size_t)c * a.nchunk + ch] = (double)accz;
  }
  if (!grid_barrier(a.bar, a.err, nblk, a.spin_limit)) return;
  column_sums(a.rpart, a.zpart, a.nchunk, ncol, st_s, st_z);
  for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
    const double s = st_s[c], z = st_z[c];
    const bool on = !a.outer_active || a.outer_active[c];
    st_rr[c] = s;
    st_rz[c] = z;
    st_min[c] = s;
    st_best[c] = s;
    st_itb[c] = 0;
    st_stop[c] = fmax(a.tol_in2 * s, a.rr_abs ? a.rr_abs[c] : 0.0);
    st_beta[c] = -1.0;
    st_act[c] = (on && s > 0.0) ? 1 : 0;
    st_it[c] = 0;
    st_flag[c] = 0;
  }
  __syncthreads();

  unsigned long long tprev = gtimer(), tphase = tprev;
  // Optional timing (a.ptime): [ph] wall time of phase ph seen by CTA 0,
  // [8 + ph] work time of phase ph summed over CTAs (before its barrier).
  auto work = [&](int ph) {
    if (a.ptime && threadIdx.x == 0) atomicAdd(&a.ptime[8 + ph], gtimer() - tphase);
  };
  auto mark = [&](int ph) {
    if (a.ptime && threadIdx.x == 0) {
      const unsigned long long t = gtimer();
      if (blockIdx.x == 0) a.ptime[ph] += t - tprev;
      tprev = t;
      tphase = t;
    }
  };
  for (int it = 0; it < a.maxit; ++it) {
    int any = 0;
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) any |= st_act[c];
    if (!__syncthreads_or(any)) break;

    // ---- phase A: p update, scatter, z-IFFT (disc rows), y-IFFT (plane)
    for (int task = blockIdx.x; task < ncol * npl; task += gridDim.x) {
      const int c = task / npl, pi = task - c * npl;
      if (!st_act[c]) continue;
      const int i0 = g.planes[pi];
      const int s0 = g.plane_sph[pi], s1 = g.plane_sph[pi + 1];
      const int q0 = g.plane_pen[pi], npp = g.plane_pen[pi + 1] - q0;
      const double bt = st_beta[c];
      const T btT = (T)bt;
      const T rtk = st_rtk[c];
      const size_t sc = (size_t)c * a.npw;
      for (int e = threadIdx.x; e < npp * LDp; e += blockDim.x) A[e] = mk<T>(0, 0);
      for (int k = threadIdx.x; k < N; k += blockDim.x) rowmap[k] = -1;
      __syncthreads();
      for (int k = threadIdx.x; k < npp; k += blockDim.x) rowmap[g.pencils[q0 + k].y] = k;
      for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
        V rv = a.r[sc + s];
        if (rtk != (T)0) {                         // z = K r
          const T k = tpa<T>(a.kin[s] * rtk);
          rv.x *= k;
          rv.y *= k;
        }
        V val = rv;
        if (bt >= 0.0) {
          const V pv = a.p[sc + s];
          val = mk<T>(rv.x + btT * pv.x, rv.y + btT * pv.y);
        }
        a.p[sc + s] = val;
        A[(g.sph_pen[s] - q0) * LDp + g.sph_i2[s]] = val;
      }
      __syncthreads();
      V* R = fft_tile2<T, +1, false>(A, B, npp, LDp, 1, a.pl, stw);
      V* Q = (R == A) ? B : A;
      for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
        const int i1 = a.pl.dN.div(e), i2 = e - i1 * N;
        const int k = rowmap[i1];
        Q[i1 * LDp + i2] = (k >= 0) ? R[k * LDp + i2] : mk<T>(0, 0);
      }
      __syncthreads();
      V* S = fft_tile2<T, +1, true>(Q, R, N, 1, LDp, a.pl, stw);
      const size_t base = (size_t)c * g.N3 + (size_t)i0 * g.N2;
      for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
        const int i1 = a.pl.dN.div(e), i2 = e - i1 * N;
        a.grid[base + e] = S[i1 * LDp + i2];
      }
      __syncthreads();
    }
    work(0);
    if (!grid_barrier(a.bar, a.err, nblk, a.spin_limit)) return;
    mark(0);

    // ---- phase B: x-IFFT, * V / N_g, x-FFT on (column, i1) slabs: pencils along i0
    // for every i2, element (i0, i2) at A[i0 * LDp + i2] (consecutive threads take
    // consecutive i2: coalesced global rows, conflict-free shared accesses)
    for (int task = blockIdx.x; task < ncol * N; task += gridDim.x) {
      const int c = task / N, i1 = task - c * N;
      if (!st_act[c]) continue;
      const size_t base = (size_t)c * g.N3 + (size_t)i1 * N;
#pragma unroll 4
      for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
        const int i0 = a.pl.dN.div(e), i2 = e - i0 * N;
        A[i0 * LDp + i2] = g.plane_mask[i0] ? a.grid[base + (size_t)i0 * g.N2 + i2] : mk<T>(0, 0);
      }
      __syncthreads();
      V* R = fft_tile2<T, +1, true>(A, B, N, 1, LDp, a.pl, stw);
      V* Q = (R == A) ? B : A;
#pragma unroll 4
      for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
        const int i0 = a.pl.dN.div(e), i2 = e - i0 * N;
        const T m = a.vloc_s[(size_t)i0 * g.N2 + (size_t)i1 * N + i2];
        const V v = R[i0 * LDp + i2];
        R[i0 * LDp + i2] = mk<T>(v.x * m, v.y * m);
      }
      __syncthreads();
      V* S = fft_tile2<T, -1, true>(R, Q, N, 1, LDp, a.pl, stw);
      for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
        const int i0 = a.pl.dN.div(e), i2 = e - i0 * N;
        if (g.plane_mask[i0]) a.grid[base + (size_t)i0 * g.N2 + i2] = S[i0 * LDp + i2];
      }
      __syncthreads();
    }
    work(1);
    if (!grid_barrier(a.bar, a.err, nblk, a.spin_limit)) return;
    mark(1);

    // ---- phase C: y-FFT, z-FFT of the disc rows, gather + kinetic + shift, and
    // the plane's partial sums <C_v|Ap>, <C_v|p> and p^H Ap (Ap before P_c)
    const size_t rbytes = plane_rec_bytes(a.nocc, (int)sizeof(V));
    for (int task = blockIdx.x; task < ncol * npl; task += gridDim.x) {
      const int c = task / npl, pi = task - c * npl;
      if (!st_act[c]) continue;
      const int i0 = g.planes[pi];
      const int s0 = g.plane_sph[pi], s1 = g.plane_sph[pi + 1];
      const int q0 = g.plane_pen[pi], npp = g.plane_pen[pi + 1] - q0;
      const size_t sc = (size_t)c * a.npw;
      const size_t base = (size_t)c * g.N3 + (size_t)i0 * g.N2;
#pragma unroll 4
      for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
        const int i1 = a.pl.dN.div(e), i2 = e - i1 * N;
        A[i1 * LDp + i2] = a.grid[base + e];
      }
      __syncthreads();
      V* R = fft_tile2<T, -1, true>(A, B, N, 1, LDp, a.pl, stw);
      V* Q = (R == A) ? B : A;
      for (int e = threadIdx.x; e < npp * N; e += blockDim.x) {
        const int k = a.pl.dN.div(e), i2 = e - k * N;
        Q[k * LDp + i2] = R[g.pencils[q0 + k].y * LDp + i2];
      }
      __syncthreads();
      V* S = fft_tile2<T, -1, false>(Q, R, npp, LDp, 1, a.pl, stw);
      V* Wv = (S == Q) ? R : Q;                     // free buffer: the plane's Ap values
      const V Ec = from_d<T>(a.E[c]);
      const int ns = s1 - s0;
      for (int e = threadIdx.x; e < ns; e += blockDim.x) {
        const int s = s0 + e;
        V val = S[(g.sph_pen[s] - q0) * LDp + g.sph_i2[s]];
        const V pv = a.p[sc + s];
        const T dr = a.kin[s] - Ec.x, di = -Ec.y;
        val.x += dr * pv.x - di * pv.y;
        val.y += dr * pv.y + di * pv.x;
        a.Ap[sc + s] = val;
        Wv[e] = val;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < ns; e += blockDim.x) S[e] = a.p[sc + s0 + e];   // the plane's p values
      __syncthreads();
      unsigned char* rec = reinterpret_cast<unsigned char*>(a.dpart) + ((size_t)c * npl + pi) * rbytes;
      plane_dots_rec<T>(a.C, a.npw, a.nocc, S, Wv, s0, ns, rec, red);
    }
    work(2);
    if (!grid_barrier(a.bar, a.err, nblk, a.spin_limit)) return;
    mark(2);

    // ---- phase E: coef = sum of the plane partials, p^H P_c A p, alpha;
    // x += alpha p, r -= alpha P_c Ap (P_c applied on the fly), partials
    // |r|^2 and r^H K r
    for (int task = blockIdx.x; task < ncol * a.nchunk; task += gridDim.x) {
      const int c = task / a.nchunk, ch = task - c * a.nchunk;
      if (!st_act[c]) continue;
      {
        // stage the column's plane records in shared memory (every thread
        // loading: independent loads in flight), then add them in plane
        // order: the projector sums in T, p^H Ap in FP64 (one warp, planes
        // strided over the lanes, a fixed shuffle tree)
        const unsigned char* src = reinterpret_cast<const unsigned char*>(a.dpart) + (size_t)c * npl * rbytes;
        const size_t nb16 = (size_t)npl * rbytes / 16;
        const bool staged = nb16 * 16 <= 2 * (size_t)N * LDp * sizeof(V);
        const unsigned char* stage = staged ? reinterpret_cast<const unsigned char*>(A) : src;
        if (staged) {
          const float4* s4 = reinterpret_cast<const float4*>(src);
          float4* d4 = reinterpret_cast<float4*>(A);
          staged_copy<kLd, float4>((int)nb16, [&](int e) { return s4[e]; }, [&](int e, float4 v) { d4[e] = v; });
        }
        __syncthreads();
        for (int j = threadIdx.x; j < 2 * a.nocc; j += blockDim.x) {
          T sx = 0, sy = 0;
          for (int q = 0; q < npl; ++q) {
            const V v = reinterpret_cast<const V*>(stage + (size_t)q * rbytes)[j];
            sx += v.x;
            sy += v.y;
          }
          coefT[j] = mk<T>(sx, sy);
        }
        if (threadIdx.x < 32) {
          double t = 0.0;
          for (int q = threadIdx.x; q < npl; q += 32)
            t += *reinterpret_cast<const double*>(stage + (size_t)q * rbytes + rbytes - 16);
          for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
          if (threadIdx.x == 0) bcast = t;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          // p^H P_c A p = p^H A p - sum_v conj(<C_v|p>) <C_v|Ap>  (the correction
          // is of the order of the rounding of p's occupied components: T)
          T corr = 0;
          for (int v = 0; v < a.nocc; ++v) {
            const V k = coefT[v], q = coefT[a.nocc + v];
            corr += q.x * k.x + q.y * k.y;
          }
          const double pap = bcast - (double)corr;
          *s_al = (T)((pap > 0.0) ? st_rz[c] / pap : 0.0);
          if (ch == 0) a.ppart[(size_t)c * a.nchunk] = pap;
        }
        __syncthreads();
      }
      const T al = *s_al;
      const int g0 = ch * a.chunk, g1 = min(a.npw, g0 + a.chunk);
      const size_t sc = (size_t)c * a.npw;
      const T rtk = st_rtk[c];
      T acc = 0, accz = 0;
      for (int G = g0 + threadIdx.x; G < g1; G += blockDim.x) {
        const size_t i = sc + G;
        V y = a.Ap[i];
        const V pv = a.p[i];
        V xv = a.x[i], rv = a.r[i];
        const T kin = a.kin[G];
        int v = 0;
        for (; v + 4 <= a.nocc; v += 4) {          // four independent loads in flight
          V cv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) cv[u] = a.C[(size_t)(v + u) * a.npw + G];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const V k = coefT[v + u];
            y.x -= cv[u].x * k.x - cv[u].y * k.y;
            y.y -= cv[u].x * k.y + cv[u].y * k.x;
          }
        }
        for (; v < a.nocc; ++v) {
          const V cv = a.C[(size_t)v * a.npw + G];
          const V k = coefT[v];
          y.x -= cv.x * k.x - cv.y * k.y;
          y.y -= cv.x * k.y + cv.y * k.x;
        }
        xv.x += al * pv.x;
        xv.y += al * pv.y;
        rv.x -= al * y.x;
        rv.y -= al * y.y;
        a.x[i] = xv;
        a.r[i] = rv;
        const T n2 = rv.x * rv.x + rv.y * rv.y;
        acc += n2;
        accz += (rtk != (T)0 ? tpa<T>(kin * rtk) : (T)1) * n2;
      }
      acc = tsum_block<T>(acc, redT);
      if (threadIdx.x == 0) a.rpart[(size_t)c * a.nchunk + ch] = (double)acc;
      accz = tsum_block<T>(accz, redT);
      if (threadIdx.x == 0) a.zpart[(size_t)c * a.nchunk + ch] = (double)accz;
      __syncthreads();
    }
    work(4);
    if (!grid_barrier(a.bar, a.err, nblk, a.spin_limit)) return;
    mark(4);

    // ---- convergence decisions (identical in every CTA)
    column_sums(a.rpart, a.zpart, a.nchunk, ncol, st_s, st_z);
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
      if (!st_act[c]) continue;
      const double s = st_s[c], z = st_z[c];
      const double pp = a.ppart[(size_t)c * a.nchunk];
      const int itc = st_it[c] + 1;
      st_it[c] = itc;
      st_beta[c] = z / st_rz[c];
      st_rz[c] = z;
      st_rr[c] = s;
      st_min[c] = fmin(st_min[c], s);
      if (s < 0.25 * st_best[c]) { st_best[c] = s; st_itb[c] = itc; }
      int stop = 0;
      if (!(pp > 0.0) || !isfinite(s)) { st_flag[c] = 2; stop = 1; }
      else if (s <= st_stop[c]) { st_flag[c] = 0; stop = 1; }
      else if (s > 1e4 * st_min[c]) { st_flag[c] = 3; stop = 1; }
      else if (itc >= a.maxit) { st_flag[c] = 1; stop = 1; }
      else if (itc - st_itb[c] > max(kCgStagWindow, 2 * st_itb[c])) { st_flag[c] = 4; stop = 1; }
      if (stop) st_act[c] = 0;
    }
    __syncthreads();
    mark(5);
  }
  if (blockIdx.x == 0) {
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
      a.iters_out[c] = st_it[c];
      a.flag_out[c] = st_act[c] ? 1 : st_flag[c];
      a.rr_out[c] = st_rr[c];
    }
  }
}

template <typename T>
static size_t pcg_smem(int N, int ncol, int nocc) {
  return pcg_layout(N, ncol, nocc, (int)sizeof(cpx<T>)).total;
}

template <typename T>
cudaError_t launch_cg_persistent(cudaStream_t s, const Geometry& g, const FftPlan& pl, const Prec<T>& P, int nocc,
                                 int npw, int ncol, const double2* b64, const int* outer_active, const double2* E,
                                 const double* rr_abs, double tol_in2, int maxit, cpx<T>* x, cpx<T>* r, cpx<T>* p,
                                 cpx<T>* Ap, cpx<T>* grid, double2* dpart, double* ppart, double* rpart,
                                 double* zpart, const double* tk, unsigned* bar, int* err, int* iters, int* flags,
                                 double* rr_out, int* grid_used, unsigned long long* ptime, int cta_div,
                                 int max_chunks, unsigned long long spin_limit) {
  PcgArgs<T> a;
  a.g = g; a.pl = pl; a.tw = P.tw; a.kin = P.kin; a.vloc_s = P.vloc_s; a.C = P.C;
  a.nocc = nocc; a.npw = npw; a.ncol = ncol;
  a.b64 = b64; a.outer_active = outer_active; a.E = E; a.rr_abs = rr_abs; a.tol_in2 = tol_in2; a.maxit = maxit;
  a.x = x; a.r = r; a.p = p; a.Ap = Ap; a.grid = grid; a.dpart = dpart; a.ppart = ppart; a.rpart = rpart;
  a.zpart = zpart; a.tk = tk;
  a.bar = bar; a.err = err; a.iters_out = iters; a.flag_out = flags; a.rr_out = rr_out; a.ptime = ptime;
  a.spin_limit = spin_limit;
  const size_t sm = pcg_smem<T>(g.N, ncol, nocc);
  cudaError_t e = cudaSuccess;
  {
    // The attribute is per function and per process: only ever raise it, so a
    // context on another host thread never sees its limit lowered under it.
    static std::mutex mu;
    static size_t raised = 0;
    std::lock_guard<std::mutex> lock(mu);
    if (sm > raised) {
      e = cudaFuncSetAttribute(k_cg_persistent<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
      raised = sm;
    }
  }
  int dev = 0, nsm = 0, per = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cg_persistent<T>, kPT, sm)) != cudaSuccess)
    return e;
  if (per < 1) return cudaErrorInvalidConfiguration;
  const int ntask = ncol * std::max(g.N, g.nplanes);
  // cta_div contexts run concurrently (batch mode): each takes an equal share
  // of the resident slots, so all their grids can be co-resident at once.
  const int cap = std::max(1, per * nsm / std::max(cta_div, 1));
  const int nblk = std::min(cap, std::max(ntask, 1));
  *grid_used = nblk;
  // phases 0 and E: one round of tasks (columns x chunks <= CTAs), chunks a
  // multiple of 32 entries, at most max_chunks per column (partial-sum slots)
  a.nchunk = std::max(1, std::min(max_chunks, nblk / std::max(ncol, 1)));
  a.chunk = (((npw + a.nchunk - 1) / a.nchunk) + 31) / 32 * 32;
  a.nchunk = (npw + a.chunk - 1) / a.chunk;
  void* args[] = {&a};
  ++g_launches;
  return cudaLaunchCooperativeKernel((const void*)k_cg_persistent<T>, dim3(nblk), dim3(kPT), args, sm, s);
}

template cudaError_t launch_cg_persistent<float>(cudaStream_t, const Geometry&, const FftPlan&, const Prec<float>&,
                                                 int, int, int, const double2*, const int*, const double2*,
                                                 const double*, double, int, float2*, float2*, float2*, float2*,
                                                 float2*, double2*, double*, double*, double*, const double*,
                                                 unsigned*, int*, int*, int*, double*, int*, unsigned long long*,
                                                 int, int, unsigned long long);
template cudaError_t launch_cg_persistent<double>(cudaStream_t, const Geometry&, const FftPlan&, const Prec<double>&,
                                                  int, int, int, const double2*, const int*, const double2*,
                                                  const double*, double, int, double2*, double2*, double2*,
                                                  double2*, double2*, double2*, double*, double*, double*,
                                                  const double*, unsigned*, int*, int*, int*, double*, int*,
                                                  unsigned long long*, int, int, unsigned long long);

}  // namespace gw
