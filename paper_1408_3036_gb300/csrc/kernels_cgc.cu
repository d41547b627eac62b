// Cluster conjugate-gradient solver for the Sternheimer equations
// (Eq. P2: (H - e_v -/+ w) x = P_c psi_v* dV, projected on the conduction
// space at every step as in Sec. Avoiding summations).
//
// One thread-block cluster of Q CTAs (8 or 16) runs the whole CG pass of one
// column, so columns never wait on one another and no grid-wide barrier is
// needed.  The column's sphere-pruned real-space grid (its P0 planes i0 that
// hold sphere points, N x N each) lives in the distributed shared memory of
// the cluster: plane pi belongs to CTA pi mod Q.  Each iteration:
//   A  own planes: p = K r + beta p on the plane's sphere entries (K: kinetic
//      preconditioner, 1 without one), scatter, z-IFFT of the disc rows,
//      y-IFFT of the plane, into the plane's shared-memory slot
//   B  slabs i1 = rank, rank + Q, ...: gather row i1 of every plane from the
//      owning CTAs, x-IFFT, * V(r)/N_g, x-FFT, scatter the rows back
//   C  own planes: y-FFT, z-FFT of the disc rows, gather the sphere entries,
//      Ap = (Vp)_G + (|G|^2/2 - E) p_G, plane sums <C_v|Ap>, <C_v|p>, p^H Ap
//   E  every CTA adds the Q partial sums in rank order (identical in every
//      CTA): coef, p^H P_c A p = p^H A p - sum_v conj(<C_v|p>) coef_v, alpha;
//      its 1/Q of the sphere: x += alpha p, r -= alpha (Ap - C coef),
//      partials |r|^2 and r^H K r, summed over the cluster in rank order
// The four phases are separated by cluster barriers (hardware barriers of the
// cluster: no spinning), and every CTA takes the same convergence decision.
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>

#include "fft.cuh"
#include "gw_common.cuh"
#include "linalg.cuh"
#include "pcg.cuh"

namespace cgrp = cooperative_groups;

namespace gw {

constexpr int kCT = 256;   // threads per CTA

template <typename T>
struct CcgArgs {
  Geometry g;
  FftPlan pl;
  const cpx<T>* tw;
  const T* kin;
  const T* vloc_s;
  const cpx<T>* C;
  int nocc, npw, Q, nown;
  const double2* b64;
  const int* outer_active;
  const double2* E;
  const double* rr_abs;
  const double* tk;
  double tol_in2;
  int maxit;
  cpx<T>* x;
  cpx<T>* r;
  cpx<T>* p;
  cpx<T>* Ap;
  int* iters_out;
  int* flag_out;
  double* rr_out;
  unsigned long long* ptime;   // optional [16]: wall time per phase seen by CTA 0 (ns)
};

struct CcgLayout {
  size_t planes, A, B, tw, red, loc, tot, locE, pidx, rowmap, total;
};

__host__ __device__ inline size_t ccg_al16(size_t x) { return (x + 15) & ~(size_t)15; }

// Shared-memory layout of one CTA (offsets in bytes).
__host__ __device__ inline CcgLayout ccg_layout(int N, int nocc, int nown, int vsize) {
  CcgLayout L;
  const size_t ndp = 2 * (size_t)nocc + 1;
  L.planes = 0;
  L.A = ccg_al16(L.planes + (size_t)nown * N * N * vsize);
  L.B = ccg_al16(L.A + (size_t)N * (N + 1) * vsize);
  L.tw = ccg_al16(L.B + (size_t)N * (N + 1) * vsize);
  L.red = ccg_al16(L.tw + (size_t)N * vsize);
  L.loc = ccg_al16(L.red + 32 * sizeof(double));
  L.tot = ccg_al16(L.loc + ndp * sizeof(double2));
  L.locE = ccg_al16(L.tot + ndp * sizeof(double2));
  L.pidx = ccg_al16(L.locE + 4 * sizeof(double));
  L.rowmap = ccg_al16(L.pidx + (size_t)N * sizeof(int));
  L.total = ccg_al16(L.rowmap + (size_t)N * sizeof(int));
  return L;
}

template <typename T>
__global__ void __launch_bounds__(kCT) k_cg_cluster(CcgArgs<T> a) {
  using V = cpx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cgrp::cluster_group cl = cgrp::this_cluster();
  const int Q = a.Q;
  const int rank = (int)cl.block_rank();
  const int c = blockIdx.x / Q;                 // the column of this cluster
  const Geometry& g = a.g;
  const int N = g.N, LDp = N + 1, N2 = N * N, npl = g.nplanes;
  const int nocc = a.nocc, ndp = 2 * nocc + 1;
  const CcgLayout L = ccg_layout(N, nocc, a.nown, (int)sizeof(V));
  V* planes = reinterpret_cast<V*>(smem_raw + L.planes);   // [nown][N][N]
  V* A = reinterpret_cast<V*>(smem_raw + L.A);             // [N][LDp]
  V* B = reinterpret_cast<V*>(smem_raw + L.B);             // [N][LDp]
  V* stw = reinterpret_cast<V*>(smem_raw + L.tw);          // [N]
  double* red = reinterpret_cast<double*>(smem_raw + L.red);
  double2* loc = reinterpret_cast<double2*>(smem_raw + L.loc);   // [ndp] this CTA's plane sums
  double2* tot = reinterpret_cast<double2*>(smem_raw + L.tot);   // [ndp] cluster sums
  double* locE = reinterpret_cast<double*>(smem_raw + L.locE);   // [2] this CTA's |r|^2, r^H K r
  int* pidx = reinterpret_cast<int*>(smem_raw + L.pidx);         // [N] plane index of i0, or -1
  int* rowmap = reinterpret_cast<int*>(smem_raw + L.rowmap);     // [N]
  __shared__ double s_rr, s_rz, s_min, s_stop, s_beta, s_pap, s_best;
  __shared__ int s_act, s_it, s_flag, s_itb;

  const bool on = !a.outer_active || a.outer_active[c];
  if (!on) {                                    // the whole cluster leaves together
    if (rank == 0 && threadIdx.x == 0) {
      a.iters_out[c] = 0;
      a.flag_out[c] = 0;
      a.rr_out[c] = 0.0;
    }
    return;
  }
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    stw[k] = a.tw[k];
    pidx[k] = -1;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < npl; q += blockDim.x) pidx[g.planes[q]] = q;

  const size_t sc = (size_t)c * a.npw;
  const int chunk = (a.npw + Q - 1) / Q;
  const int g0 = min(a.npw, rank * chunk), g1 = min(a.npw, g0 + chunk);
  const T rtk = a.tk ? (T)(1.0 / a.tk[c]) : (T)0;
  const double2 Ec = a.E[c];

  // ---- phase 0: r = b, x = 0 on this CTA's part; |b|^2 and b^H K b
  {
    double acc = 0.0, accz = 0.0;
    for (int G = g0 + threadIdx.x; G < g1; G += blockDim.x) {
      const V bv = from_d<T>(a.b64[sc + G]);
      a.r[sc + G] = bv;
      a.x[sc + G] = mk<T>(0, 0);
      const double2 bd = to_d(bv);
      const double n2 = bd.x * bd.x + bd.y * bd.y;
      acc += n2;
      accz += (rtk != (T)0 ? (double)tpa<T>(a.kin[G] * rtk) : 1.0) * n2;
    }
    acc = dsum_block_f(acc, red);
    accz = dsum_block_f(accz, red);
    if (threadIdx.x == 0) {
      locE[0] = acc;
      locE[1] = accz;
    }
  }
  cl.sync();
  if (threadIdx.x == 0) {
    double s = 0.0, z = 0.0;
    for (int q = 0; q < Q; ++q) {
      const double* le = cl.map_shared_rank(locE, q);
      s += le[0];
      z += le[1];
    }
    s_rr = s;
    s_rz = z;
    s_min = s;
    s_best = s;
    s_itb = 0;
    s_stop = fmax(a.tol_in2 * s, a.rr_abs ? a.rr_abs[c] : 0.0);
    s_beta = -1.0;
    s_act = (s > 0.0) ? 1 : 0;
    s_it = 0;
    s_flag = 0;
  }
  __syncthreads();

  unsigned long long tprev = gtimer();
  auto mark = [&](int ph) {
    if (a.ptime && blockIdx.x == 0 && threadIdx.x == 0) {
      const unsigned long long t = gtimer();
      a.ptime[ph] += t - tprev;
      tprev = t;
    }
  };
  for (int it = 0; it < a.maxit && s_act; ++it) {
    // ---- phase A: p update, scatter, z-IFFT, y-IFFT of the own planes
    const double bt = s_beta;
    for (int j = 0; j < a.nown; ++j) {
      const int pi = rank + j * Q;
      if (pi >= npl) break;
      const int s0 = g.plane_sph[pi], s1 = g.plane_sph[pi + 1];
      const int q0 = g.plane_pen[pi], npp = g.plane_pen[pi + 1] - q0;
      for (int e = threadIdx.x; e < npp * LDp; e += blockDim.x) A[e] = mk<T>(0, 0);
      for (int k = threadIdx.x; k < N; k += blockDim.x) rowmap[k] = -1;
      __syncthreads();
      for (int k = threadIdx.x; k < npp; k += blockDim.x) rowmap[g.pencils[q0 + k].y] = k;
      for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
        V rv = a.r[sc + s];
        if (rtk != (T)0) {                      // z = K r
          const T k = tpa<T>(a.kin[s] * rtk);
          rv.x *= k;
          rv.y *= k;
        }
        V val = rv;
        if (bt >= 0.0) {
          const V pv = a.p[sc + s];
          val = mk<T>(rv.x + (T)bt * pv.x, rv.y + (T)bt * pv.y);
        }
        a.p[sc + s] = val;
        A[(g.sph_pen[s] - q0) * LDp + g.sph_i2[s]] = val;
      }
      __syncthreads();
      V* R = fft_tile2<T, +1, false>(A, B, npp, LDp, 1, a.pl, stw);
      V* Qb = (R == A) ? B : A;
      for (int e = threadIdx.x; e < N2; e += blockDim.x) {
        const int i1 = a.pl.dN.div(e), i2 = e - i1 * N;
        const int k = rowmap[i1];
        Qb[i1 * LDp + i2] = (k >= 0) ? R[k * LDp + i2] : mk<T>(0, 0);
      }
      __syncthreads();
      V* S = fft_tile2<T, +1, true>(Qb, R, N, 1, LDp, a.pl, stw);
      V* dst = planes + (size_t)j * N2;
      for (int e = threadIdx.x; e < N2; e += blockDim.x) {
        const int i1 = a.pl.dN.div(e), i2 = e - i1 * N;
        dst[e] = S[i1 * LDp + i2];
      }
      __syncthreads();
    }
    cl.sync();
    mark(0);

    // ---- phase B: x-IFFT, * V / N_g, x-FFT on the slabs i1 = rank + Q k
    for (int i1 = rank; i1 < N; i1 += Q) {
#pragma unroll 4
      for (int e = threadIdx.x; e < N2; e += blockDim.x) {
        const int i0 = a.pl.dN.div(e), i2 = e - i0 * N;
        const int pi = pidx[i0];
        V v = mk<T>(0, 0);
        if (pi >= 0) v = cl.map_shared_rank(planes, pi % Q)[(size_t)(pi / Q) * N2 + i1 * N + i2];
        A[i0 * LDp + i2] = v;
      }
      __syncthreads();
      V* R = fft_tile2<T, +1, true>(A, B, N, 1, LDp, a.pl, stw);
#pragma unroll 4
      for (int e = threadIdx.x; e < N2; e += blockDim.x) {
        const int i0 = a.pl.dN.div(e), i2 = e - i0 * N;
        const T m = a.vloc_s[(size_t)i0 * N2 + (size_t)i1 * N + i2];
        V& v = R[i0 * LDp + i2];
        v.x *= m;
        v.y *= m;
      }
      __syncthreads();
      V* Qb = (R == A) ? B : A;
      V* S = fft_tile2<T, -1, true>(R, Qb, N, 1, LDp, a.pl, stw);
      for (int e = threadIdx.x; e < N2; e += blockDim.x) {
        const int i0 = a.pl.dN.div(e), i2 = e - i0 * N;
        const int pi = pidx[i0];
        if (pi >= 0) cl.map_shared_rank(planes, pi % Q)[(size_t)(pi / Q) * N2 + i1 * N + i2] = S[i0 * LDp + i2];
      }
      __syncthreads();
    }
    cl.sync();
    mark(1);

    // ---- phase C: y-FFT, z-FFT, gather + kinetic + shift, plane sums
    for (int k = threadIdx.x; k < ndp; k += blockDim.x) loc[k] = make_double2(0.0, 0.0);
    for (int j = 0; j < a.nown; ++j) {
      const int pi = rank + j * Q;
      if (pi >= npl) break;
      const int s0 = g.plane_sph[pi], s1 = g.plane_sph[pi + 1];
      const int q0 = g.plane_pen[pi], npp = g.plane_pen[pi + 1] - q0;
      const V* src = planes + (size_t)j * N2;
      for (int e = threadIdx.x; e < N2; e += blockDim.x) {
        const int i1 = a.pl.dN.div(e), i2 = e - i1 * N;
        A[i1 * LDp + i2] = src[e];
      }
      __syncthreads();
      V* R = fft_tile2<T, -1, true>(A, B, N, 1, LDp, a.pl, stw);
      V* Qb = (R == A) ? B : A;
      for (int e = threadIdx.x; e < npp * N; e += blockDim.x) {
        const int k = a.pl.dN.div(e), i2 = e - k * N;
        Qb[k * LDp + i2] = R[g.pencils[q0 + k].y * LDp + i2];
      }
      __syncthreads();
      V* S = fft_tile2<T, -1, false>(Qb, R, npp, LDp, 1, a.pl, stw);
      V* Wv = (S == Qb) ? R : Qb;                   // the plane's Ap values
      const int ns = s1 - s0;
      for (int e = threadIdx.x; e < ns; e += blockDim.x) {
        const int s = s0 + e;
        V val = S[(g.sph_pen[s] - q0) * LDp + g.sph_i2[s]];
        const V pv = a.p[sc + s];
        const T dr = a.kin[s] - (T)Ec.x, di = -(T)Ec.y;
        val.x += dr * pv.x - di * pv.y;
        val.y += dr * pv.y + di * pv.x;
        a.Ap[sc + s] = val;
        Wv[e] = val;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < ns; e += blockDim.x) S[e] = a.p[sc + s0 + e];
      __syncthreads();
      plane_dots<T, true>(a.C, a.npw, nocc, S, Wv, s0, ns, loc, red);
    }
    cl.sync();
    mark(2);

    // ---- phase E: cluster sums, alpha, x and r on this CTA's part
    for (int k = threadIdx.x; k < ndp; k += blockDim.x) {
      double sx = 0.0, sy = 0.0;
      for (int q = 0; q < Q; ++q) {
        const double2 v = cl.map_shared_rank(loc, q)[k];
        sx += v.x;
        sy += v.y;
      }
      tot[k] = make_double2(sx, sy);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      // p^H P_c A p = p^H A p - sum_v conj(<C_v|p>) <C_v|Ap>
      double pap = tot[2 * nocc].x;
      for (int v = 0; v < nocc; ++v) {
        const double2 k = tot[v], q = tot[nocc + v];
        pap -= q.x * k.x + q.y * k.y;
      }
      s_pap = pap;
    }
    __syncthreads();
    const double pap = s_pap;
    const T al = (T)((pap > 0.0) ? s_rz / pap : 0.0);
    double acc = 0.0, accz = 0.0;
    for (int G = g0 + threadIdx.x; G < g1; G += blockDim.x) {
      const size_t i = sc + G;
      V y = a.Ap[i];
      const V pv = a.p[i];
      V xv = a.x[i], rv = a.r[i];
      const T kin = a.kin[G];
      int v = 0;
      for (; v + 4 <= nocc; v += 4) {              // four independent loads in flight
        V cv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) cv[u] = a.C[(size_t)(v + u) * a.npw + G];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const V k = from_d<T>(tot[v + u]);
          y.x -= cv[u].x * k.x - cv[u].y * k.y;
          y.y -= cv[u].x * k.y + cv[u].y * k.x;
        }
      }
      for (; v < nocc; ++v) {
        const V cv = a.C[(size_t)v * a.npw + G];
        const V k = from_d<T>(tot[v]);
        y.x -= cv.x * k.x - cv.y * k.y;
        y.y -= cv.x * k.y + cv.y * k.x;
      }
      xv.x += al * pv.x;
      xv.y += al * pv.y;
      rv.x -= al * y.x;
      rv.y -= al * y.y;
      a.x[i] = xv;
      a.r[i] = rv;
      const double2 rd = to_d(rv);
      const double n2 = rd.x * rd.x + rd.y * rd.y;
      acc += n2;
      accz += (rtk != (T)0 ? (double)tpa<T>(kin * rtk) : 1.0) * n2;
    }
    acc = dsum_block_f(acc, red);
    accz = dsum_block_f(accz, red);
    if (threadIdx.x == 0) {
      locE[0] = acc;
      locE[1] = accz;
    }
    cl.sync();
    mark(4);

    // ---- convergence decision (identical in every CTA of the cluster)
    if (threadIdx.x == 0) {
      double s = 0.0, z = 0.0;
      for (int q = 0; q < Q; ++q) {
        const double* le = cl.map_shared_rank(locE, q);
        s += le[0];
        z += le[1];
      }
      const int itc = s_it + 1;
      s_it = itc;
      s_beta = z / s_rz;
      s_rz = z;
      s_rr = s;
      s_min = fmin(s_min, s);
      if (s < 0.25 * s_best) { s_best = s; s_itb = itc; }
      int stop = 0;
      if (!(pap > 0.0) || !isfinite(s)) { s_flag = 2; stop = 1; }
      else if (s <= s_stop) { s_flag = 0; stop = 1; }
      else if (s > 1e4 * s_min) { s_flag = 3; stop = 1; }
      else if (itc >= a.maxit) { s_flag = 1; stop = 1; }
      else if (itc - s_itb > max(kCgStagWindow, 2 * s_itb)) { s_flag = 4; stop = 1; }
      if (stop) s_act = 0;
    }
    __syncthreads();
    mark(5);
  }
  if (rank == 0 && threadIdx.x == 0) {
    a.iters_out[c] = s_it;
    a.flag_out[c] = s_act ? 1 : s_flag;
    a.rr_out[c] = s_rr;
  }
  cl.sync();   // no CTA leaves while another may still read its shared memory
}

template <typename T>
cudaError_t launch_cg_cluster(cudaStream_t s, const Geometry& g, const FftPlan& pl, const Prec<T>& P, int nocc,
                              int npw, int ncol, const double2* b64, const int* outer_active, const double2* E,
                              const double* rr_abs, const double* tk, double tol_in2, int maxit, cpx<T>* x,
                              cpx<T>* r, cpx<T>* p, cpx<T>* Ap, int* iters, int* flags, double* rr_out,
                              int* q_used, unsigned long long* ptime) {
  *q_used = 0;
  if (ncol < 1 || g.nplanes < 1) return cudaErrorInvalidValue;
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  const void* fn = (const void*)k_cg_cluster<T>;
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, fn)) != cudaSuccess) return e;
  optin -= (int)fa.sharedSizeBytes;           // room left for dynamic shared memory
  {
    // Raise the function's limits once per process (never lowered: contexts
    // on other host threads launch the same function).
    static std::mutex mu;
    static bool done = false;
    std::lock_guard<std::mutex> lock(mu);
    if (!done) {
      if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin)) != cudaSuccess)
        return e;
      if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess) return e;
      done = true;
    }
  }
  // Cluster size: the one that finishes soonest, counting waves of clusters
  // (time ~ waves x work per CTA ~ waves / Q); larger Q on ties.
  int best_q = 0;
  double best_cost = 0.0;
  size_t best_sm = 0;
  for (int Q : {16, 8}) {
    const int nown = (g.nplanes + Q - 1) / Q;
    const size_t sm = ccg_layout(g.N, nocc, nown, (int)sizeof(cpx<T>)).total;
    if (sm > (size_t)optin) continue;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = Q;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(ncol * Q);
    cfg.blockDim = dim3(kCT);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclu = 0;
    if (cudaOccupancyMaxActiveClusters(&nclu, fn, &cfg) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (nclu < 1) continue;
    const double cost = (double)((ncol + nclu - 1) / nclu) / Q;
    if (best_q == 0 || cost < best_cost) {
      best_q = Q;
      best_cost = cost;
      best_sm = sm;
    }
  }
  if (best_q == 0) return cudaErrorNotSupported;
  CcgArgs<T> a;
  a.g = g; a.pl = pl; a.tw = P.tw; a.kin = P.kin; a.vloc_s = P.vloc_s; a.C = P.C;
  a.nocc = nocc; a.npw = npw; a.Q = best_q; a.nown = (g.nplanes + best_q - 1) / best_q;
  a.b64 = b64; a.outer_active = outer_active; a.E = E; a.rr_abs = rr_abs; a.tk = tk;
  a.tol_in2 = tol_in2; a.maxit = maxit;
  a.x = x; a.r = r; a.p = p; a.Ap = Ap;
  a.iters_out = iters; a.flag_out = flags; a.rr_out = rr_out; a.ptime = ptime;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = best_q;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(ncol * best_q);
  cfg.blockDim = dim3(kCT);
  cfg.dynamicSmemBytes = best_sm;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  *q_used = best_q;
  ++g_launches;
  return cudaLaunchKernelEx(&cfg, k_cg_cluster<T>, a);
}

template cudaError_t launch_cg_cluster<float>(cudaStream_t, const Geometry&, const FftPlan&, const Prec<float>&, int,
                                              int, int, const double2*, const int*, const double2*, const double*,
                                              const double*, double, int, float2*, float2*, float2*, float2*, int*,
                                              int*, double*, int*, unsigned long long*);
template cudaError_t launch_cg_cluster<double>(cudaStream_t, const Geometry&, const FftPlan&, const Prec<double>&,
                                               int, int, int, const double2*, const int*, const double2*,
                                               const double*, const double*, double, int, double2*, double2*,
                                               double2*, double2*, int*, int*, double*, int*,
                                               unsigned long long*);

}  // namespace gw
