// Vector kernels of the Sternheimer solver and of the Lanczos recursion:
// the conduction projector P_c (Sec. Avoiding summations: orthogonalisation
// against the valence space at every solver step), conjugate-gradient updates
// with per-column convergence masks, FP64 residuals of the refinement loop,
// the Lanczos re-orthogonalisation (Sec. Lanczos: Gram-Schmidt against all
// previous vectors) and the inverse of the tridiagonal Lanczos matrix.
//
// Reductions are deterministic: blocks write partial sums, the last block to
// finish (atomic ticket) adds them in a fixed order.  Dot products accumulate
// in FP64 for both precisions.
#include <algorithm>
#include <cstdio>

#include "gw_common.cuh"
#include "linalg.cuh"

namespace gw {

constexpr int kLT = 256;   // threads per block
constexpr int kChunk = 1024; // sphere / grid entries per block in vector kernels
constexpr int kCT = 8;     // columns per block in the projector dots

template <typename R>
__device__ __forceinline__ R block_sum(R v) {
  __shared__ R sh[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  R r = 0;
  if (threadIdx.x < 32) {
    r = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : (R)0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  return r;  // valid in thread 0
}

// ---------------------------------------------------------------------------
// P_c y = y - sum_v c_v <c_v|y>: coefficients (a) then update (b).
// ---------------------------------------------------------------------------
constexpr int kChunkP = 128;  // sphere entries per block in the projector coefficients (spreads over all SMs)

// (a) coef[v * ncol + b] = sum_G conj(C[v][G]) Y[b][G]; grid (nchunk, ceil(ncol / kCT)).
// REAL: rows and columns real in real space (x(-G) = conj x(G)), so every
// coefficient is real: only Re is summed (half the products and reductions)
// and Im is 0.
template <typename T, bool REAL>
__global__ void __launch_bounds__(kLT)
k_proj_dots(const cpx<T>* __restrict__ C, int nocc, int npw, const cpx<T>* __restrict__ Y, int ncol,
            const int* __restrict__ active, double2* __restrict__ partial, unsigned* __restrict__ cnt,
            double2* __restrict__ coef) {
  // partial sums, their shuffles and the sum over chunks in the precision of
  // the vectors (FP64 arithmetic is scarce on this GPU); coef in FP64
  cpx<T>* part = reinterpret_cast<cpx<T>*>(partial);
  const int nchunk = gridDim.x;
  const int g0 = blockIdx.x * kChunkP, g1 = min(npw, g0 + kChunkP);
  const int b0 = blockIdx.y * kCT;
  const int nb = min(kCT, ncol - b0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  for (int v = warp; v < nocc; v += nw) {
    T ax[kCT], ay[kCT];
#pragma unroll
    for (int j = 0; j < kCT; ++j) { ax[j] = 0; ay[j] = 0; }
    for (int G = g0 + lane; G < g1; G += 32) {
      const cpx<T> c = C[(size_t)v * npw + G];
#pragma unroll
      for (int j = 0; j < kCT; ++j) {
        if (j < nb) {
          const cpx<T> y = Y[(size_t)(b0 + j) * npw + G];
          ax[j] += c.x * y.x + c.y * y.y;
          if (!REAL) ay[j] += c.x * y.y - c.y * y.x;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kCT; ++j) {
      T sx = ax[j], sy = ay[j];
      for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        if (!REAL) sy += __shfl_xor_sync(0xffffffffu, sy, o);
      }
      if (lane == 0 && j < nb) part[((size_t)blockIdx.x * nocc + v) * ncol + b0 + j] = mk<T>(sx, sy);
    }
  }
  if (!last_block(&cnt[blockIdx.y], nchunk)) return;
  for (int t = threadIdx.x; t < nocc * nb; t += blockDim.x) {
    const int v = t / nb, j = t - v * nb;
    T q[2];
    sum_records<2, T>(reinterpret_cast<const T*>(part + (size_t)v * ncol + b0 + j), nchunk,
                      2 * (size_t)nocc * ncol, q);
    coef[(size_t)v * ncol + b0 + j] = make_double2((double)q[0], (double)q[1]);
  }
}

// (b) Y[b] -= sum_v C[v] coef[v][b] (precision T); optionally pap[b] = Re <P[b]|Y[b]> (new Y),
// accumulated in FP64.  grid (nchunk, ncol)
template <typename T, bool REAL>
__global__ void __launch_bounds__(kLT)
k_proj_update(const cpx<T>* __restrict__ C, int nocc, int npw, cpx<T>* __restrict__ Y, int ncol,
              const int* __restrict__ active, const double2* __restrict__ coef,
              const cpx<T>* __restrict__ Pv, double* __restrict__ partial, unsigned* __restrict__ cnt,
              double* __restrict__ pap) {
  __shared__ cpx<T> sc[kMaxOcc];
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  for (int v = threadIdx.x; v < nocc; v += blockDim.x) sc[v] = from_d<T>(coef[(size_t)v * ncol + b]);
  __syncthreads();
  const int g0 = blockIdx.x * kChunk, g1 = min(npw, g0 + kChunk);
  double acc = 0.0;
  for (int G = g0 + threadIdx.x; G < g1; G += blockDim.x) {
    cpx<T> y = Y[(size_t)b * npw + G];
    for (int v = 0; v < nocc; ++v) {
      const cpx<T> c = C[(size_t)v * npw + G];
      const cpx<T> a = sc[v];
      if (REAL) {                   // real coefficient
        y.x -= c.x * a.x;
        y.y -= c.y * a.x;
      } else {
        y.x -= c.x * a.x - c.y * a.y;
        y.y -= c.x * a.y + c.y * a.x;
      }
    }
    Y[(size_t)b * npw + G] = y;
    if (Pv) {
      const cpx<T> p = Pv[(size_t)b * npw + G];
      acc += (double)(p.x * y.x + p.y * y.y);
    }
  }
  if (!Pv) return;
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[(size_t)blockIdx.x * ncol + b] = acc;
  if (!last_block(&cnt[b], gridDim.x)) return;
  if (threadIdx.x == 0) {
    double s;
    sum_records<1>(partial + b, gridDim.x, ncol, &s);
    pap[b] = s;
  }
}

template <typename T>
void launch_proj(cudaStream_t s, const cpx<T>* C, int nocc, int npw, cpx<T>* Y, int ncol, const int* active,
                 Work& w, const cpx<T>* Pv, double* pap, bool real) {
  if (ncol == 0 || nocc == 0) return;
  const int nchunk = (npw + kChunkP - 1) / kChunkP;
  dim3 g1(nchunk, (ncol + kCT - 1) / kCT);
  ++g_launches;
  if (real) k_proj_dots<T, true><<<g1, kLT, 0, s>>>(C, nocc, npw, Y, ncol, active, w.part2, w.cnt_a, w.coef);
  else k_proj_dots<T, false><<<g1, kLT, 0, s>>>(C, nocc, npw, Y, ncol, active, w.part2, w.cnt_a, w.coef);
  launch_proj_update<T>(s, C, nocc, npw, Y, ncol, active, w.coef, w, Pv, pap, real);
}

// Gram matrix only: coef[v * ncol + b] = sum_G conj(C[v][G]) Y[b][G]
template <typename T>
void launch_gram(cudaStream_t s, const cpx<T>* C, int nocc, int npw, const cpx<T>* Y, int ncol, Work& w,
                 double2* out, bool real) {
  if (ncol == 0 || nocc == 0) return;
  const int nchunk = (npw + kChunkP - 1) / kChunkP;
  dim3 g1(nchunk, (ncol + kCT - 1) / kCT);
  ++g_launches;
  if (real) k_proj_dots<T, true><<<g1, kLT, 0, s>>>(C, nocc, npw, Y, ncol, nullptr, w.part2, w.cnt_a, out);
  else k_proj_dots<T, false><<<g1, kLT, 0, s>>>(C, nocc, npw, Y, ncol, nullptr, w.part2, w.cnt_a, out);
}

// ---------------------------------------------------------------------------
// adjoint (derivative of <phi|eps~^-1(0)|phi> w.r.t. V_loc) grid kernels
// ---------------------------------------------------------------------------
// W[v][v'] = (1/N_g) sum_r conj(U_v) w U_v'; grid (nchunk over N_g, nocc*nocc)
__global__ void __launch_bounds__(kLT)
k_wmat(const double2* __restrict__ U, const double* __restrict__ w, int n, int nocc,
       double2* __restrict__ partial, unsigned* __restrict__ cnt, double2* __restrict__ W) {
  const int pair = blockIdx.y;
  const int v = pair / nocc, vp = pair - v * nocc;
  const int g0 = blockIdx.x * kChunk, g1 = min(n, g0 + kChunk);
  double ax = 0.0, ay = 0.0;
  for (int r = g0 + threadIdx.x; r < g1; r += blockDim.x) {
    const double2 a = U[(size_t)v * n + r], b = U[(size_t)vp * n + r];
    const double wr = w[r];
    ax += wr * (a.x * b.x + a.y * b.y);
    ay += wr * (a.x * b.y - a.y * b.x);
  }
  ax = block_sum(ax);
  ay = block_sum(ay);
  const int np = nocc * nocc;
  if (threadIdx.x == 0) partial[(size_t)blockIdx.x * np + pair] = make_double2(ax, ay);
  if (!last_block(&cnt[pair], gridDim.x)) return;
  if (threadIdx.x == 0) {
    double q[2];
    sum_records<2>(reinterpret_cast<const double*>(partial + pair), gridDim.x, 2 * (size_t)np, q);
    W[pair] = make_double2(q[0] / n, q[1] / n);
  }
}

void launch_wmat(cudaStream_t s, const double2* U, const double* w, int n, int nocc, Work& wk, double2* W) {
  dim3 g((n + kChunk - 1) / kChunk, nocc * nocc);
  ++g_launches;
  k_wmat<<<g, kLT, 0, s>>>(U, w, n, nocc, wk.part2, wk.cnt_c, W);
}

// g1[r] = (sum_v |dU_v|^2 - sum_{v v'} S[v][v'] conj(U_v'(r)) U_v(r)) / vol
__global__ void k_g1(const double2* __restrict__ dU, const double2* __restrict__ U, const double2* __restrict__ S,
                     int n, int nocc, double inv_vol, double* __restrict__ g1) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int v = 0; v < nocc; ++v) {
      const double2 d = dU[(size_t)v * n + r];
      acc += d.x * d.x + d.y * d.y;
      const double2 uv = U[(size_t)v * n + r];
      for (int vp = 0; vp < nocc; ++vp) {
        const double2 uvp = U[(size_t)vp * n + r];
        const double2 sv = S[(size_t)v * nocc + vp];
        // Re( S[v][v'] conj(U_v') U_v )
        const double cx = uvp.x * uv.x + uvp.y * uv.y;   // conj(uvp) * uv
        const double cy = uvp.x * uv.y - uvp.y * uv.x;
        acc -= sv.x * cx - sv.y * cy;
      }
    }
    g1[r] = acc * inv_vol;
  }
}

void launch_g1(cudaStream_t s, const double2* dU, const double2* U, const double2* S, int n, int nocc,
               double inv_vol, double* g1) {
  const int nb = std::min((n + kLT - 1) / kLT, 152 * 8);
  ++g_launches;
  k_g1<<<nb, kLT, 0, s>>>(dU, U, S, n, nocc, inv_vol, g1);
}

// grad = wgt (4 g1 + 8 g2)
__global__ void k_grad_combine(int n, const double* __restrict__ g1, const double* __restrict__ g2, double wgt,
                               double* __restrict__ grad) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
    grad[r] = wgt * (4.0 * g1[r] + 8.0 * g2[r]);
}

void launch_grad_combine(cudaStream_t s, int n, const double* g1, const double* g2, double wgt, double* grad) {
  const int nb = std::min((n + kLT - 1) / kLT, 152 * 8);
  ++g_launches;
  k_grad_combine<<<nb, kLT, 0, s>>>(n, g1, g2, wgt, grad);
}

// Ap += w2[c] p (the shift of (H - E)^2 + w^2); optionally pap[c] = Re <p|Ap>
// (FP64, deterministic two-level sum).  grid (nchunk, ncol)
template <typename T>
__global__ void __launch_bounds__(kLT)
k_sq_shift(int npw, cpx<T>* __restrict__ Ap, const cpx<T>* __restrict__ p, const double* __restrict__ w2,
           const int* __restrict__ active, double* __restrict__ partial, unsigned* __restrict__ cnt,
           double* __restrict__ pap, int ncol) {
  const int c = blockIdx.y;
  if (active && !active[c]) return;
  const T s2 = (T)w2[c];
  const int g0 = blockIdx.x * kChunk, g1 = min(npw, g0 + kChunk);
  double acc = 0.0;
  for (int G = g0 + threadIdx.x; G < g1; G += blockDim.x) {
    const size_t i = (size_t)c * npw + G;
    const cpx<T> pv = p[i];
    cpx<T> a = Ap[i];
    a.x += s2 * pv.x;
    a.y += s2 * pv.y;
    Ap[i] = a;
    acc += (double)(pv.x * a.x + pv.y * a.y);
  }
  if (!pap) return;
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[(size_t)blockIdx.x * ncol + c] = acc;
  if (!last_block(&cnt[c], gridDim.x)) return;
  if (threadIdx.x == 0) {
    double q;
    sum_records<1>(partial + c, gridDim.x, ncol, &q);
    pap[c] = q;
  }
}

template <typename T>
void launch_sq_shift(cudaStream_t s, int npw, int ncol, cpx<T>* Ap, const cpx<T>* p, const double* w2,
                     const int* active, Work& w, double* pap) {
  dim3 g((npw + kChunk - 1) / kChunk, ncol);
  ++g_launches;
  k_sq_shift<T><<<g, kLT, 0, s>>>(npw, Ap, p, w2, active, w.part1, w.cnt_c, pap, ncol);
}

template <typename T>
void launch_proj_update(cudaStream_t s, const cpx<T>* C, int nocc, int npw, cpx<T>* Y, int ncol,
                        const int* active, const double2* coef, Work& w, const cpx<T>* Pv, double* pap, bool real) {
  if (ncol == 0 || nocc == 0) return;
  const int nchunk = (npw + kChunk - 1) / kChunk;
  dim3 g2(nchunk, ncol);
  ++g_launches;
  if (real) k_proj_update<T, true><<<g2, kLT, 0, s>>>(C, nocc, npw, Y, ncol, active, coef, Pv, w.part1, w.cnt_b, pap);
  else k_proj_update<T, false><<<g2, kLT, 0, s>>>(C, nocc, npw, Y, ncol, active, coef, Pv, w.part1, w.cnt_b, pap);
}

// ---------------------------------------------------------------------------
// conjugate gradients (Hermitian positive definite A = P_c (H - E) P_c)
// ---------------------------------------------------------------------------
// Preconditioner factor of sphere entry G for column c (1 without one).
template <typename T>
__device__ __forceinline__ T precond(const T* kin, const double* tk, int c, int G) {
  return tk ? tpa<T>(kin[G] * (T)(1.0 / tk[c])) : (T)1;
}
// The CG's preconditioner: K, or K^2 for the squared operator (H - E)^2 + w^2.
template <typename T>
__device__ __forceinline__ T precond_cg(const T* kin, const CgState& st, int c, int G) {
  const T k = precond<T>(kin, st.tk, c, G);
  return st.ppow == 2 ? k * k : k;
}

// init: x = 0, r = b (converted), rr = rr0 = |b|^2, rz = r^H K r, beta = -1 (first p = K r)
template <typename T, typename U>
__global__ void __launch_bounds__(kLT)
k_cg_init(int npw, const cpx<U>* __restrict__ b, cpx<T>* __restrict__ x, cpx<T>* __restrict__ r,
          const int* __restrict__ outer_active, double2* __restrict__ partial, const T* __restrict__ kin,
          CgState st, int ncol, double tol_in2, double tol_abs2) {
  const int c = blockIdx.y;
  const int g0 = blockIdx.x * kChunk, g1 = min(npw, g0 + kChunk);
  double acc = 0.0, accz = 0.0;
  const bool on = !outer_active || outer_active[c];
  for (int G = g0 + threadIdx.x; G < g1; G += blockDim.x) {
    const size_t i = (size_t)c * npw + G;
    cpx<T> bv = on ? from_d<T>(to_d(b[i])) : mk<T>(0, 0);
    r[i] = bv;
    x[i] = mk<T>(0, 0);
    const double2 bd = to_d(bv);
    const double n2 = bd.x * bd.x + bd.y * bd.y;
    acc += n2;
    accz += (double)precond_cg<T>(kin, st, c, G) * n2;
  }
  acc = block_sum(acc);
  accz = block_sum(accz);
  if (threadIdx.x == 0) partial[(size_t)blockIdx.x * ncol + c] = make_double2(acc, accz);
  if (!last_block(&st.cnt[c], gridDim.x)) return;
  if (threadIdx.x == 0) {
    double q[2];
    sum_records<2>(reinterpret_cast<const double*>(partial + c), gridDim.x, 2 * (size_t)ncol, q);
    const double s = q[0], z = q[1];
    st.rr[c] = s;
    st.rr0[c] = s;
    st.rr_min[c] = s;
    st.rr_best[c] = s;
    st.it_best[c] = 0;
    st.rz[c] = z;
    // relative target of this pass, but never below what the refinement needs
    // overall (a fraction of the final tolerance on the original right-hand side)
    st.rr_stop[c] = fmax(tol_in2 * s, st.rr_abs ? st.rr_abs[c] : tol_abs2 * s);
    st.beta[c] = -1.0;
    st.iters[c] = 0;
    st.flag[c] = 0;
    st.active[c] = (on && s > 0.0) ? 1 : 0;
    if (!st.active[c]) atomicAdd(st.n_done, 1);
  }
}

// alpha = rz / pap; x += alpha p; r -= alpha Ap; rr' = |r|^2, rz' = r^H K r;
// beta = rz'/rz (the next p = K r + beta p is fused into the scatter); masks
template <typename T>
__global__ void __launch_bounds__(kLT)
k_cg_update(int npw, cpx<T>* __restrict__ x, cpx<T>* __restrict__ r, const cpx<T>* __restrict__ p,
            const cpx<T>* __restrict__ Ap, const double* __restrict__ pap, double2* __restrict__ partial,
            const T* __restrict__ kin, CgState st, double tol2, int maxit, int ncol) {
  const int c = blockIdx.y;
  if (!st.active[c]) return;
  const double pp = pap[c];
  const double alpha = (pp > 0.0) ? st.rz[c] / pp : 0.0;
  const T a = (T)alpha;
  const int g0 = blockIdx.x * kChunk, g1 = min(npw, g0 + kChunk);
  double acc = 0.0, accz = 0.0;
  for (int G = g0 + threadIdx.x; G < g1; G += blockDim.x) {
    const size_t i = (size_t)c * npw + G;
    const cpx<T> pv = p[i], av = Ap[i];
    cpx<T> xv = x[i], rv = r[i];
    xv.x += a * pv.x; xv.y += a * pv.y;
    rv.x -= a * av.x; rv.y -= a * av.y;
    x[i] = xv;
    r[i] = rv;
    const double2 rd = to_d(rv);
    const double n2 = rd.x * rd.x + rd.y * rd.y;
    acc += n2;
    accz += (double)precond_cg<T>(kin, st, c, G) * n2;
  }
  acc = block_sum(acc);
  accz = block_sum(accz);
  if (threadIdx.x == 0) partial[(size_t)blockIdx.x * ncol + c] = make_double2(acc, accz);
  if (!last_block(&st.cnt[c], gridDim.x)) return;
  if (threadIdx.x == 0) {
    double q[2];
    sum_records<2>(reinterpret_cast<const double*>(partial + c), gridDim.x, 2 * (size_t)ncol, q);
    const double s = q[0], z = q[1];
    const int it = st.iters[c] + 1;
    st.iters[c] = it;
    st.beta[c] = z / st.rz[c];
    st.rz[c] = z;
    st.rr[c] = s;
    bool stop = false;
    st.rr_min[c] = fmin(st.rr_min[c], s);
    if (s < 0.25 * st.rr_best[c]) { st.rr_best[c] = s; st.it_best[c] = it; }
    if (!(pp > 0.0) || !isfinite(s)) { st.flag[c] = 2; stop = true; }     // breakdown / not SPD
    else if (s <= st.rr_stop[c]) { st.flag[c] = 0; stop = true; }
    else if (s > 1e4 * st.rr_min[c]) { st.flag[c] = 3; stop = true; }      // past the round-off floor
    else if (it >= maxit) { st.flag[c] = 1; stop = true; }
    else if (it - st.it_best[c] > max(kCgStagWindow, 2 * st.it_best[c])) { st.flag[c] = 4; stop = true; }
    if (stop) { st.active[c] = 0; atomicAdd(st.n_done, 1); }
  }
}

template <typename T, typename U>
void launch_cg_init(cudaStream_t s, int npw, int ncol, const cpx<U>* b, cpx<T>* x, cpx<T>* r,
                    const int* outer_active, Work& w, CgState st, const T* kin, double tol_in2, double tol_abs2) {
  dim3 g((npw + kChunk - 1) / kChunk, ncol);
  ++g_launches;
  k_cg_init<T, U><<<g, kLT, 0, s>>>(npw, b, x, r, outer_active, w.part2, kin, st, ncol, tol_in2, tol_abs2);
}

template <typename T>
void launch_cg_update(cudaStream_t s, int npw, int ncol, cpx<T>* x, cpx<T>* r, const cpx<T>* p,
                      const cpx<T>* Ap, const double* pap, Work& w, CgState st, const T* kin, double tol2,
                      int maxit) {
  dim3 g((npw + kChunk - 1) / kChunk, ncol);
  ++g_launches;
  k_cg_update<T><<<g, kLT, 0, s>>>(npw, x, r, p, Ap, pap, w.part2, kin, st, tol2, maxit, ncol);
}

// ---------------------------------------------------------------------------
// simplified QMR (Freund-Nachtigal) for complex-symmetric A = P_c (H - E) P_c
// with the bilinear form [x, y] = sum_r x(r) y(r) = sum_G x(-G) y(G)
// (Sec. "Avoiding summations": SQMR replaces CG when (H - e_v -/+ w) is not
// positive definite; unpreconditioned it equals MINRES for real symmetric A)
// with the symmetric kinetic preconditioner K applied on the right (K = 1
// without one):
//   init: r = b, q = K b, x = d = 0, tau = |b|, rho = [b, K b], theta = 0
//   loop: t = A q; sigma = [q, t]; alpha = rho / sigma; r -= alpha t
//         theta' = |r| / tau; c2 = 1 / (1 + theta'^2); tau = tau theta' sqrt(c2)
//         d = c2 theta^2 d + c2 alpha q; x += d
//         rho' = [r, K r]; beta = rho' / rho; q = K r + beta q
//   stop when tau^2 <= rr_stop (tau: the quasi-residual norm)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double den = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}

template <typename T>
__global__ void __launch_bounds__(kLT)
k_qmr_init(int npw, const double2* __restrict__ b, cpx<T>* __restrict__ x, cpx<T>* __restrict__ r,
           cpx<T>* __restrict__ q, cpx<T>* __restrict__ d, const int* __restrict__ neg,
           const int* __restrict__ outer_active, double* __restrict__ partial, const T* __restrict__ kin,
           QmrState st, int ncol, double tol_in2) {
  const int c = blockIdx.y;
  const int g0 = blockIdx.x * kChunk, g1 = min(npw, g0 + kChunk);
  const bool on = !outer_active || outer_active[c];
  double a1 = 0.0, ax = 0.0, ay = 0.0;
  for (int G = g0 + threadIdx.x; G < g1; G += blockDim.x) {
    const size_t i = (size_t)c * npw + G;
    const cpx<T> bv = on ? from_d<T>(b[i]) : mk<T>(0, 0);
    const cpx<T> bn = on ? from_d<T>(b[(size_t)c * npw + neg[G]]) : mk<T>(0, 0);
    const T k = precond<T>(kin, st.tk, c, G);
    r[i] = bv;
    q[i] = mk<T>(k * bv.x, k * bv.y);               // q = K b
    x[i] = mk<T>(0, 0);
    d[i] = mk<T>(0, 0);
    const double2 u = to_d(bv), w = to_d(bn);
    a1 += u.x * u.x + u.y * u.y;
    ax += (double)k * (w.x * u.x - w.y * u.y);       // rho = [b, K b]
    ay += (double)k * (w.x * u.y + w.y * u.x);
  }
  a1 = block_sum(a1);
  ax = block_sum(ax);
  ay = block_sum(ay);
  if (threadIdx.x == 0) {
    double* pp = partial + 3 * ((size_t)blockIdx.x * ncol + c);
    pp[0] = a1; pp[1] = ax; pp[2] = ay;
  }
  if (!last_block(&st.cnt[c], gridDim.x)) return;
  if (threadIdx.x == 0) {
    double q[3];
    sum_records<3>(partial + 3 * (size_t)c, gridDim.x, 3 * (size_t)ncol, q);
    const double s1 = q[0], sx = q[1], sy = q[2];
    st.tau[c] = sqrt(s1);
    st.rho[c] = make_double2(sx, sy);
    st.theta[c] = 0.0;
    st.iters[c] = 0;
    st.flag[c] = 0;
    st.rr_stop[c] = fmax(tol_in2 * s1, st.rr_abs ? st.rr_abs[c] : 0.0);
    st.qbest[c] = s1;
    st.itbest[c] = 0;
    st.active[c] = (on && s1 > 0.0) ? 1 : 0;
    if (!st.active[c]) atomicAdd(st.n_done, 1);
  }
}

constexpr int kQmrStagWindow = 1000;

// sigma = [q, t]; alpha = rho / sigma
template <typename T>
__global__ void __launch_bounds__(kLT)
k_qmr_sigma(int npw, const cpx<T>* __restrict__ q, const cpx<T>* __restrict__ t, const int* __restrict__ neg,
            double* __restrict__ partial, QmrState st, int ncol) {
  const int c = blockIdx.y;
  if (!st.active[c]) return;
  const int g0 = blockIdx.x * kChunk, g1 = min(npw, g0 + kChunk);
  double ax = 0.0, ay = 0.0;
  for (int G = g0 + threadIdx.x; G < g1; G += blockDim.x) {
    const double2 a = to_d(q[(size_t)c * npw + neg[G]]), u = to_d(t[(size_t)c * npw + G]);
    ax += a.x * u.x - a.y * u.y;
    ay += a.x * u.y + a.y * u.x;
  }
  ax = block_sum(ax);
  ay = block_sum(ay);
  if (threadIdx.x == 0) {
    double* pp = partial + 2 * ((size_t)blockIdx.x * ncol + c);
    pp[0] = ax; pp[1] = ay;
  }
  if (!last_block(&st.cnt[c], gridDim.x)) return;
  if (threadIdx.x == 0) {
    double q[2];
    sum_records<2>(partial + 2 * (size_t)c, gridDim.x, 2 * (size_t)ncol, q);
    const double sx = q[0], sy = q[1];
    const double2 sg = make_double2(sx, sy);
    const double2 rho = st.rho[c];
    if (!(sx * sx + sy * sy > 1e-300 * (rho.x * rho.x + rho.y * rho.y)) || !isfinite(sx) || !isfinite(sy)) {
      st.alpha[c] = make_double2(0, 0);
      st.flag[c] = 2;                                  // serious breakdown: [q, A q] = 0
    } else {
      st.alpha[c] = cdiv(rho, sg);
    }
  }
}

// r -= alpha t; theta', c2, tau
template <typename T>
__global__ void __launch_bounds__(kLT)
k_qmr_r(int npw, cpx<T>* __restrict__ r, const cpx<T>* __restrict__ t, double* __restrict__ partial, QmrState st,
        int ncol) {
  const int c = blockIdx.y;
  if (!st.active[c]) return;
  const double2 al = st.alpha[c];
  const cpx<T> a = from_d<T>(al);
  const int g0 = blockIdx.x * kChunk, g1 = min(npw, g0 + kChunk);
  double acc = 0.0;
  for (int G = g0 + threadIdx.x; G < g1; G += blockDim.x) {
    const size_t i = (size_t)c * npw + G;
    cpx<T> rv = r[i];
    const cpx<T> tv = t[i];
    rv.x -= a.x * tv.x - a.y * tv.y;
    rv.y -= a.x * tv.y + a.y * tv.x;
    r[i] = rv;
    const double2 rd = to_d(rv);
    acc += rd.x * rd.x + rd.y * rd.y;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[(size_t)blockIdx.x * ncol + c] = acc;
  if (!last_block(&st.cnt[c], gridDim.x)) return;
  if (threadIdx.x == 0) {
    double s;
    sum_records<1>(partial + c, gridDim.x, ncol, &s);
    const double th = sqrt(s) / st.tau[c];
    const double c2 = 1.0 / (1.0 + th * th);
    st.dcoef[c] = c2 * st.theta[c] * st.theta[c];   // multiplies the old d
    st.qcoef[c] = make_double2(c2 * al.x, c2 * al.y);
    st.tau[c] = st.tau[c] * th * sqrt(c2);
    st.theta[c] = th;
  }
}

// d = dcoef d + qcoef q; x += d; rho' = [r, r]; beta
template <typename T>
__global__ void __launch_bounds__(kLT)
k_qmr_dx(int npw, cpx<T>* __restrict__ x, cpx<T>* __restrict__ d, const cpx<T>* __restrict__ q,
         const cpx<T>* __restrict__ r, const int* __restrict__ neg, double* __restrict__ partial,
         const T* __restrict__ kin, QmrState st, int ncol, int maxit) {
  const int c = blockIdx.y;
  if (!st.active[c]) return;
  const T dc = (T)st.dcoef[c];
  const cpx<T> qc = from_d<T>(st.qcoef[c]);
  const int g0 = blockIdx.x * kChunk, g1 = min(npw, g0 + kChunk);
  double ax = 0.0, ay = 0.0;
  for (int G = g0 + threadIdx.x; G < g1; G += blockDim.x) {
    const size_t i = (size_t)c * npw + G;
    const cpx<T> qv = q[i];
    cpx<T> dv = d[i];
    dv.x = dc * dv.x + (qc.x * qv.x - qc.y * qv.y);
    dv.y = dc * dv.y + (qc.x * qv.y + qc.y * qv.x);
    d[i] = dv;
    cpx<T> xv = x[i];
    xv.x += dv.x;
    xv.y += dv.y;
    x[i] = xv;
    const double2 a = to_d(r[(size_t)c * npw + neg[G]]), u = to_d(r[i]);
    const double k = (double)precond<T>(kin, st.tk, c, G);
    ax += k * (a.x * u.x - a.y * u.y);              // rho' = [r, K r]
    ay += k * (a.x * u.y + a.y * u.x);
  }
  ax = block_sum(ax);
  ay = block_sum(ay);
  if (threadIdx.x == 0) {
    double* pp = partial + 2 * ((size_t)blockIdx.x * ncol + c);
    pp[0] = ax; pp[1] = ay;
  }
  if (!last_block(&st.cnt[c], gridDim.x)) return;
  if (threadIdx.x == 0) {
    double q[2];
    sum_records<2>(partial + 2 * (size_t)c, gridDim.x, 2 * (size_t)ncol, q);
    const double sx = q[0], sy = q[1];
    const double2 rn = make_double2(sx, sy);
    const double2 rho = st.rho[c];
    st.beta[c] = (rho.x * rho.x + rho.y * rho.y > 0.0) ? cdiv(rn, rho) : make_double2(0, 0);
    st.rho[c] = rn;
    const int it = st.iters[c] + 1;
    st.iters[c] = it;
    const double tau = st.tau[c];
    // tau is the quasi-residual norm: for a Hermitian system (real frequency)
    // it is the minimal-residual norm of the iterate, and the usual estimate of
    // |b - A x| in the complex-symmetric case.  The FP64 refinement around the
    // solve checks the true residual.
    const double qb = tau * tau;
    if (qb < 0.25 * st.qbest[c]) { st.qbest[c] = qb; st.itbest[c] = it; }
    bool stop = false;
    if (st.flag[c] == 2 || !isfinite(tau)) { st.flag[c] = 2; stop = true; }
    else if (qb <= st.rr_stop[c]) { st.flag[c] = 0; stop = true; }
    else if (!(rn.x * rn.x + rn.y * rn.y > 0.0)) { st.flag[c] = 2; stop = true; }
    else if (it >= maxit) { st.flag[c] = 1; stop = true; }
    else if (it - st.itbest[c] > max(kQmrStagWindow, 2 * st.itbest[c])) {
      // The estimate has not halved for a long stretch: the recurrence has reached
      // the accuracy its working precision allows for this (nearly singular,
      // indefinite) system.  Stop; the FP64 refinement around the solve
      // continues from the iterate reached.
      st.flag[c] = 4;
      stop = true;
    }
    if (stop) { st.active[c] = 0; atomicAdd(st.n_done, 1); }
  }
}

// q = K r + beta q
template <typename T>
__global__ void k_qmr_q(int npw, cpx<T>* __restrict__ q, const cpx<T>* __restrict__ r, const T* __restrict__ kin,
                        QmrState st) {
  const int c = blockIdx.y;
  if (!st.active[c]) return;
  const cpx<T> b = from_d<T>(st.beta[c]);
  for (int G = blockIdx.x * blockDim.x + threadIdx.x; G < npw; G += gridDim.x * blockDim.x) {
    const size_t i = (size_t)c * npw + G;
    const T k = precond<T>(kin, st.tk, c, G);
    const cpx<T> qv = q[i], rv = r[i];
    q[i] = mk<T>(k * rv.x + b.x * qv.x - b.y * qv.y, k * rv.y + b.x * qv.y + b.y * qv.x);
  }
}

template <typename T>
void launch_qmr(cudaStream_t s, int step, int npw, int ncol, const double2* b, cpx<T>* x, cpx<T>* r, cpx<T>* q,
                cpx<T>* d, const cpx<T>* t, const int* neg, const int* outer_active, Work& w, QmrState st,
                const T* kin, double tol_in2, int maxit) {
  dim3 g((npw + kChunk - 1) / kChunk, ncol);
  double* part = reinterpret_cast<double*>(w.part2);
  ++g_launches;
  switch (step) {
    case 0:
      k_qmr_init<T><<<g, kLT, 0, s>>>(npw, b, x, r, q, d, neg, outer_active, part, kin, st, ncol, tol_in2);
      break;
    case 1: k_qmr_sigma<T><<<g, kLT, 0, s>>>(npw, q, t, neg, part, st, ncol); break;
    case 2: k_qmr_r<T><<<g, kLT, 0, s>>>(npw, r, t, part, st, ncol); break;
    case 3: k_qmr_dx<T><<<g, kLT, 0, s>>>(npw, x, d, q, r, neg, part, kin, st, ncol, maxit); break;
    default: {
      dim3 g2((npw + kLT - 1) / kLT, ncol);
      k_qmr_q<T><<<g2, kLT, 0, s>>>(npw, q, r, kin, st);
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 refinement helpers
// ---------------------------------------------------------------------------
// x64 += d (converted), for active columns
template <typename T>
__global__ void k_add_conv(size_t npw, const cpx<T>* __restrict__ d, double2* __restrict__ x,
                           const int* __restrict__ active) {
  const int c = blockIdx.y;
  if (active && !active[c]) return;
  for (size_t G = blockIdx.x * (size_t)blockDim.x + threadIdx.x; G < npw; G += (size_t)gridDim.x * blockDim.x) {
    const size_t i = (size_t)c * npw + G;
    const double2 dv = to_d(d[i]);
    double2 xv = x[i];
    xv.x += dv.x; xv.y += dv.y;
    x[i] = xv;
  }
}

template <typename T>
void launch_add_conv(cudaStream_t s, int npw, int ncol, const cpx<T>* d, double2* x, const int* active) {
  dim3 g((npw + kLT - 1) / kLT, ncol);
  ++g_launches;
  k_add_conv<T><<<g, kLT, 0, s>>>((size_t)npw, d, x, active);
}

// x += (d(G) + conj d(-G)) / 2: the correction of a column whose solution is
// real in real space, with any antisymmetric rounding of d dropped.
template <typename T>
__global__ void k_add_conv_sym(size_t npw, const cpx<T>* __restrict__ d, double2* __restrict__ x,
                               const int* __restrict__ active, const int* __restrict__ neg) {
  const int c = blockIdx.y;
  if (active && !active[c]) return;
  for (size_t G = blockIdx.x * (size_t)blockDim.x + threadIdx.x; G < npw; G += (size_t)gridDim.x * blockDim.x) {
    const size_t i = (size_t)c * npw + G;
    const double2 dv = to_d(d[i]);
    const double2 dn = to_d(d[(size_t)c * npw + neg[G]]);
    double2 xv = x[i];
    xv.x += 0.5 * (dv.x + dn.x);
    xv.y += 0.5 * (dv.y - dn.y);
    x[i] = xv;
  }
}

template <typename T>
void launch_add_conv_sym(cudaStream_t s, int npw, int ncol, const cpx<T>* d, double2* x, const int* active,
                         const int* neg) {
  dim3 g((npw + kLT - 1) / kLT, ncol);
  ++g_launches;
  k_add_conv_sym<T><<<g, kLT, 0, s>>>((size_t)npw, d, x, active, neg);
}

// Two columns that are real in real space in one complex vector:
//   out[j](G) = x[ia[j]](G) + i x[ib[j]](G)   (ib[j] < 0: the first alone)
__global__ void k_pack_pairs(size_t npw, const double2* __restrict__ x, const int* __restrict__ ia,
                             const int* __restrict__ ib, const int* __restrict__ active, double2* __restrict__ out) {
  const int j = blockIdx.y;
  if (active && !active[j]) return;
  const int a = ia[j], b = ib[j];
  for (size_t G = blockIdx.x * (size_t)blockDim.x + threadIdx.x; G < npw; G += (size_t)gridDim.x * blockDim.x) {
    const double2 u = x[(size_t)a * npw + G];
    const double2 v = (b >= 0) ? x[(size_t)b * npw + G] : make_double2(0.0, 0.0);
    out[(size_t)j * npw + G] = make_double2(u.x - v.y, u.y + v.x);
  }
}

void launch_pack_pairs(cudaStream_t s, int npw, int npair, const double2* x, const int* ia, const int* ib,
                       const int* active, double2* out) {
  dim3 g((npw + kLT - 1) / kLT, npair);
  ++g_launches;
  k_pack_pairs<<<g, kLT, 0, s>>>((size_t)npw, x, ia, ib, active, out);
}

// The two parts of a packed transform Y_j = F(f_a) + i F(f_b) of real fields:
//   out[ia[j]](G) = (Y_j(G) + conj Y_j(-G)) / 2,  out[ib[j]](G) = (Y_j(G) - conj Y_j(-G)) / 2i,
// plus (kin(G) - E_c) x_c(G) when kin is given (the kinetic part of (H - E) x).
__global__ void k_unpack_pairs(size_t npw, const double2* __restrict__ Y, const int* __restrict__ neg,
                               const int* __restrict__ ia, const int* __restrict__ ib, const int* __restrict__ active,
                               const double* __restrict__ kin, const double2* __restrict__ E,
                               const double2* __restrict__ x, double2* __restrict__ out) {
  const int j = blockIdx.y;
  if (active && !active[j]) return;
  const int a = ia[j], b = ib[j];
  for (size_t G = blockIdx.x * (size_t)blockDim.x + threadIdx.x; G < npw; G += (size_t)gridDim.x * blockDim.x) {
    const double2 y1 = Y[(size_t)j * npw + G];
    const double2 yn = Y[(size_t)j * npw + neg[G]];
    double2 o0 = make_double2(0.5 * (y1.x + yn.x), 0.5 * (y1.y - yn.y));
    double2 o1 = make_double2(0.5 * (y1.y + yn.y), -0.5 * (y1.x - yn.x));
    if (kin) {
      const double2 xa = x[(size_t)a * npw + G];
      const double dr = kin[G] - E[a].x, di = -E[a].y;
      o0.x += dr * xa.x - di * xa.y;
      o0.y += dr * xa.y + di * xa.x;
      if (b >= 0) {
        const double2 xb = x[(size_t)b * npw + G];
        const double er = kin[G] - E[b].x, ei = -E[b].y;
        o1.x += er * xb.x - ei * xb.y;
        o1.y += er * xb.y + ei * xb.x;
      }
    }
    out[(size_t)a * npw + G] = o0;
    if (b >= 0) out[(size_t)b * npw + G] = o1;
  }
}

void launch_unpack_pairs(cudaStream_t s, int npw, int npair, const double2* Y, const int* neg, const int* ia,
                         const int* ib, const int* active, const double* kin, const double2* E, const double2* x,
                         double2* out) {
  dim3 g((npw + kLT - 1) / kLT, npair);
  ++g_launches;
  k_unpack_pairs<<<g, kLT, 0, s>>>((size_t)npw, Y, neg, ia, ib, active, kin, E, x, out);
}

// out[c] = max_G |b(G) - conj b(-G)|, out[ncol + c] = max_G |b(G)| (one block per column)
__global__ void __launch_bounds__(kLT) k_sym_check(int npw, const double2* __restrict__ b, const int* __restrict__ neg,
                                                   double* __restrict__ out, int ncol) {
  __shared__ double sa[kLT / 32], sb[kLT / 32];
  const int c = blockIdx.x;
  double ma = 0.0, mb = 0.0;
  for (int G = threadIdx.x; G < npw; G += blockDim.x) {
    const double2 v = b[(size_t)c * npw + G], w = b[(size_t)c * npw + neg[G]];
    ma = fmax(ma, fabs(v.x - w.x) + fabs(v.y + w.y));
    mb = fmax(mb, fabs(v.x) + fabs(v.y));
  }
  for (int o = 16; o > 0; o >>= 1) {
    ma = fmax(ma, __shfl_xor_sync(0xffffffffu, ma, o));
    mb = fmax(mb, __shfl_xor_sync(0xffffffffu, mb, o));
  }
  if ((threadIdx.x & 31) == 0) { sa[threadIdx.x >> 5] = ma; sb[threadIdx.x >> 5] = mb; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) { ma = fmax(ma, sa[k]); mb = fmax(mb, sb[k]); }
    out[c] = fmax(ma, sa[0]);
    out[ncol + c] = fmax(mb, sb[0]);
  }
}

void launch_sym_check(cudaStream_t s, int npw, int ncol, const double2* b, const int* neg, double* out) {
  ++g_launches;
  k_sym_check<<<ncol, kLT, 0, s>>>(npw, b, neg, out, ncol);
}

// r = b - Ax (in place over Ax), res2[c] = |r|^2, bb[c] = |b|^2, xx[c] = |x|^2.
// With C: r = P_c (b - Ax) = b - Ax - sum_v C_v (cb[v][c] - cax[v][c]), where
// cb = C^H b and cax = C^H Ax (coefficients [nocc][ncol]).
__global__ void __launch_bounds__(kLT)
k_residual(int npw, const double2* __restrict__ b, double2* __restrict__ ax, const double2* __restrict__ x,
           const int* __restrict__ active, double* __restrict__ partial, unsigned* __restrict__ cnt,
           double* __restrict__ res2, double* __restrict__ bb, double* __restrict__ xx, int ncol,
           const double2* __restrict__ C, int nocc, const double2* __restrict__ cb,
           const double2* __restrict__ cax, int real) {
  __shared__ double2 sc[kMaxOcc];
  const int c = blockIdx.y;
  if (active && !active[c]) return;
  if (C) {
    for (int v = threadIdx.x; v < nocc; v += blockDim.x) {
      const double2 u = cb[(size_t)v * ncol + c], w = cax[(size_t)v * ncol + c];
      sc[v] = make_double2(u.x - w.x, u.y - w.y);
    }
    __syncthreads();
  }
  const int g0 = blockIdx.x * kChunk, g1 = min(npw, g0 + kChunk);
  double a1 = 0.0, a2 = 0.0, a3 = 0.0;
  for (int G = g0 + threadIdx.x; G < g1; G += blockDim.x) {
    const size_t i = (size_t)c * npw + G;
    const double2 bv = b[i];
    double2 r = ax[i];
    r.x = bv.x - r.x;
    r.y = bv.y - r.y;
    if (C && real) {               // real coefficients (real-in-real-space columns)
      for (int v = 0; v < nocc; ++v) {
        const double2 cv = C[(size_t)v * npw + G];
        const double k = sc[v].x;
        r.x -= cv.x * k;
        r.y -= cv.y * k;
      }
    } else if (C) {
      for (int v = 0; v < nocc; ++v) {
        const double2 cv = C[(size_t)v * npw + G], k = sc[v];
        r.x -= cv.x * k.x - cv.y * k.y;
        r.y -= cv.x * k.y + cv.y * k.x;
      }
    }
    ax[i] = r;
    a1 += r.x * r.x + r.y * r.y;
    a2 += bv.x * bv.x + bv.y * bv.y;
    if (x) { const double2 xv = x[i]; a3 += xv.x * xv.x + xv.y * xv.y; }
  }
  a1 = block_sum(a1);
  a2 = block_sum(a2);
  a3 = block_sum(a3);
  if (threadIdx.x == 0) {
    double* pp = partial + 3 * ((size_t)blockIdx.x * ncol + c);
    pp[0] = a1; pp[1] = a2; pp[2] = a3;
  }
  if (!last_block(&cnt[c], gridDim.x)) return;
  if (threadIdx.x == 0) {
    double q[3];
    sum_records<3>(partial + 3 * (size_t)c, gridDim.x, 3 * (size_t)ncol, q);
    const double s1 = q[0], s2 = q[1], s3 = q[2];
    res2[c] = s1;
    bb[c] = s2;
    if (xx) xx[c] = s3;
  }
}

void launch_residual(cudaStream_t s, int npw, int ncol, const double2* b, double2* ax, const double2* x,
                     const int* active, Work& w, double* res2, double* bb, double* xx, const double2* C, int nocc,
                     const double2* cb, const double2* cax, bool real) {
  dim3 g((npw + kChunk - 1) / kChunk, ncol);
  ++g_launches;
  k_residual<<<g, kLT, 0, s>>>(npw, b, ax, x, active, reinterpret_cast<double*>(w.part2), w.cnt_b, res2, bb,
                                xx, ncol, C, nocc, cb, cax, real ? 1 : 0);
}

// Deflated components of a Sternheimer pass: coef[d][c] = <D_d|r_c> on entry;
// on exit -<D_d|r_c> / (eps_d - E_c), the negated coefficients of
// sum_d D_d <D_d|r_c> / (eps_d - E_c) for launch_proj_update (which subtracts).
__global__ void k_defl_scale(double2* __restrict__ coef, const double* __restrict__ eps,
                             const double2* __restrict__ E, int ndef, int ncol, const int* __restrict__ active) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ndef * ncol) return;
  const int d = t / ncol, c = t - d * ncol;
  if (active && !active[c]) return;
  const double2 den = make_double2(eps[d] - E[c].x, -E[c].y);
  const double2 q = cdiv(coef[t], den);
  coef[t] = make_double2(-q.x, -q.y);
}

void launch_defl_scale(cudaStream_t s, double2* coef, const double* eps, const double2* E, int ndef, int ncol,
                       const int* active) {
  const int n = ndef * ncol;
  if (n == 0) return;
  ++g_launches;
  k_defl_scale<<<(n + 255) / 256, 256, 0, s>>>(coef, eps, E, ndef, ncol, active);
}

// ---------------------------------------------------------------------------
// sphere-vector helpers
// ---------------------------------------------------------------------------
// out[j] = w_pair (in[src0[j]] + in[src1[j]])  or  w_single in[src0[j]] when src1[j] < 0
__global__ void k_combine(int npw, const double2* __restrict__ in, const int* __restrict__ src0,
                          const int* __restrict__ src1, double w_pair, double w_single, double2* __restrict__ out) {
  const int j = blockIdx.y;
  const int a = src0[j], b = src1[j];
  for (int G = blockIdx.x * blockDim.x + threadIdx.x; G < npw; G += gridDim.x * blockDim.x) {
    double2 v = in[(size_t)a * npw + G];
    if (b >= 0) {
      const double2 u = in[(size_t)b * npw + G];
      v.x = w_pair * (v.x + u.x);
      v.y = w_pair * (v.y + u.y);
    } else {
      v.x *= w_single;
      v.y *= w_single;
    }
    out[(size_t)j * npw + G] = v;
  }
}

void launch_combine(cudaStream_t s, int npw, int nout, const double2* in, const int* src0, const int* src1,
                    double w_pair, double w_single, double2* out) {
  dim3 g((npw + kLT - 1) / kLT, nout);
  ++g_launches;
  k_combine<<<g, kLT, 0, s>>>(npw, in, src0, src1, w_pair, w_single, out);
}

// Kinetic denominators of the model operator (Sec. Dielectric model, Eq.
// model_eq): out[j][G] = (1/(|G|^2/2 - Em_j) + 1/(|G|^2/2 - Ep_j)) in[src_j][G]
// with Em = e_v + omega, Ep = e_v - omega (complex).  A reciprocal whose
// denominator is exactly zero is taken as 0 (the pseudo-inverse of the
// diagonal; such an entry of a projected right-hand side is zero).
template <typename T>
__device__ __forceinline__ cpx<T> pinv_shift(T t, cpx<T> e) {
  const T dr = t - e.x, di = -e.y;
  const T d2 = dr * dr + di * di;
  if (d2 == (T)0) return mk<T>(0, 0);
  const T r = (T)1 / d2;
  return mk<T>(dr * r, -di * r);
}

// (in the precision T of the vectors)
template <typename T>
__global__ void k_model_scale(int npw, const T* __restrict__ kin, const cpx<T>* __restrict__ in,
                              const int* __restrict__ src, const double2* __restrict__ Em,
                              const double2* __restrict__ Ep, cpx<T>* __restrict__ out) {
  const int j = blockIdx.y;
  const int a = src[j];
  const cpx<T> em = from_d<T>(Em[j]), ep = from_d<T>(Ep[j]);
  for (int G = blockIdx.x * blockDim.x + threadIdx.x; G < npw; G += gridDim.x * blockDim.x) {
    const T t = kin[G];
    const cpx<T> w = cadd(pinv_shift<T>(t, em), pinv_shift<T>(t, ep));
    out[(size_t)j * npw + G] = cmul(w, in[(size_t)a * npw + G]);
  }
}

template <typename T>
void launch_model_scale(cudaStream_t s, int npw, int nout, const T* kin, const cpx<T>* in, const int* src,
                        const double2* Em, const double2* Ep, cpx<T>* out) {
  if (nout == 0) return;
  dim3 g((npw + kLT - 1) / kLT, nout);
  ++g_launches;
  k_model_scale<T><<<g, kLT, 0, s>>>(npw, kin, in, src, Em, Ep, out);
}
template void launch_model_scale<double>(cudaStream_t, int, int, const double*, const double2*, const int*,
                                         const double2*, const double2*, double2*);
template void launch_model_scale<float>(cudaStream_t, int, int, const float*, const float2*, const int*,
                                        const double2*, const double2*, float2*);

// precision changes at the boundary of an FP32 pipeline; out = x - z (FP64 result)
// Eq. subs_epsilon in the two bases: out[i][j] = sum_ab a_ia (Ti_ab - (M^-1)_ab) a_jb
// + sum_ab am_ia (Tmi_ab - delta_ab) am_jb; one block per (i, j), rows a over
// the threads, then an ordered block sum.  Mi holds the inverse of M^T, i.e.
// (M^-1)_ab = Re Mi[b][a]; the matrices are read column-wise (X[b][a] for row a)
// so that the threads' loads are contiguous (Ti and Tmi are symmetric).
__global__ void __launch_bounds__(kLT)
k_split_form(int m, int k, int km, const double* __restrict__ a, const double* __restrict__ Ti,
             const double2* __restrict__ Mi, const double* __restrict__ am, const double* __restrict__ Tmi,
             double* __restrict__ out) {
  const int i = blockIdx.x, j = blockIdx.y;
  const double* ai = a + (size_t)i * k;
  const double* aj = a + (size_t)j * k;
  const double* bi = am + (size_t)i * km;
  const double* bj = am + (size_t)j * km;
  double acc = 0.0;
  for (int r = threadIdx.x; r < k; r += blockDim.x) {
    double t = 0.0;
    for (int c = 0; c < k; ++c) t += (Ti[(size_t)c * k + r] - Mi[(size_t)c * k + r].x) * aj[c];
    acc += ai[r] * t;
  }
  for (int r = threadIdx.x; r < km; r += blockDim.x) {
    double t = -bj[r];
    for (int c = 0; c < km; ++c) t += Tmi[(size_t)c * km + r] * bj[c];
    acc += bi[r] * t;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) out[(size_t)i * m + j] = acc;
}

void launch_split_form(cudaStream_t s, int m, int k, int km, const double* a, const double* Ti,
                       const double2* Mi, const double* am, const double* Tmi, double* out) {
  ++g_launches;
  k_split_form<<<dim3(m, m), kLT, 0, s>>>(m, k, km, a, Ti, Mi, am, Tmi, out);
}

// real -> complex square matrix (imaginary part zero)
__global__ void k_to_cplx(size_t n, const double* __restrict__ x, double2* __restrict__ y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = make_double2(x[i], 0.0);
}

void launch_to_cplx(cudaStream_t s, size_t n, const double* x, double2* y) {
  ++g_launches;
  k_to_cplx<<<(int)std::min<size_t>((n + kLT - 1) / kLT, 152 * 8), kLT, 0, s>>>(n, x, y);
}

// gather rows: out[j] = in[idx[j]] (sphere vectors, with precision conversion)
template <typename T, typename U>
__global__ void k_gather_rows(int npw, const cpx<U>* __restrict__ in, const int* __restrict__ idx,
                              cpx<T>* __restrict__ out) {
  const int j = blockIdx.y;
  const int a = idx ? idx[j] : j;
  for (int G = blockIdx.x * blockDim.x + threadIdx.x; G < npw; G += gridDim.x * blockDim.x)
    out[(size_t)j * npw + G] = from_d<T>(to_d(in[(size_t)a * npw + G]));
}

template <typename T, typename U>
void launch_gather_rows(cudaStream_t s, int npw, int nout, const cpx<U>* in, const int* idx, cpx<T>* out) {
  dim3 g((npw + kLT - 1) / kLT, nout);
  ++g_launches;
  k_gather_rows<T, U><<<g, kLT, 0, s>>>(npw, in, idx, out);
}

// ---------------------------------------------------------------------------
// Lanczos vectors (real FP64 grid fields, weighted inner product)
// ---------------------------------------------------------------------------
// out[j] = wgt * sum_r Q[j][r] w[r], j < k; grid (nchunk, k)
__global__ void __launch_bounds__(kLT)
k_gemv_t(const double* __restrict__ Q, size_t ld, int n, const double* __restrict__ w, double wgt,
         double* __restrict__ partial, unsigned* __restrict__ cnt, double* __restrict__ out, int k) {
  const int j = blockIdx.y;
  const int g0 = blockIdx.x * kChunk, g1 = min(n, g0 + kChunk);
  double acc = 0.0;
  for (int r = g0 + threadIdx.x; r < g1; r += blockDim.x) acc += Q[(size_t)j * ld + r] * w[r];
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[(size_t)blockIdx.x * k + j] = acc;
  if (!last_block(&cnt[j], gridDim.x)) return;
  if (threadIdx.x == 0) {
    double s;
    sum_records<1>(partial + j, gridDim.x, k, &s);
    out[j] = wgt * s;
  }
}

// w[r] -= sum_j Q[j][r] h[j]
__global__ void k_gemv_n(const double* __restrict__ Q, size_t ld, int n, const double* __restrict__ h, int k,
                         double* __restrict__ w) {
  extern __shared__ double sh[];
  for (int j = threadIdx.x; j < k; j += blockDim.x) sh[j] = h[j];
  __syncthreads();
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < k; ++j) acc += Q[(size_t)j * ld + r] * sh[j];
    w[r] -= acc;
  }
}

void launch_gemv_t(cudaStream_t s, const double* Q, size_t ld, int n, const double* w, double wgt, int k,
                   Work& wk, double* out) {
  dim3 g((n + kChunk - 1) / kChunk, k);
  ++g_launches;
  k_gemv_t<<<g, kLT, 0, s>>>(Q, ld, n, w, wgt, wk.part1, wk.cnt_c, out, k);
}

void launch_gemv_n(cudaStream_t s, const double* Q, size_t ld, int n, const double* h, int k, double* w) {
  const int nb = (n + kLT - 1) / kLT;
  ++g_launches;
  k_gemv_n<<<nb, kLT, k * sizeof(double), s>>>(Q, ld, n, h, k, w);
}

// Lanczos scalar steps on device:
//   op 0: w -= beta[k-1] * qprev                          (k > 0)
//   op 1: w -= alpha[k] * q
//   op 2: q_next = w / beta[k]
__global__ void k_lz_axpy(int n, int op, const double* __restrict__ sc, double* __restrict__ w,
                          const double* __restrict__ q, double* __restrict__ qn) {
  const double a = *sc;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    if (op == 2) qn[r] = w[r] / a;
    else w[r] -= a * q[r];
  }
}

void launch_lz_axpy(cudaStream_t s, int n, int op, const double* sc, double* w, const double* q, double* qn) {
  const int nb = min((n + kLT - 1) / kLT, 4 * 152);
  ++g_launches;
  k_lz_axpy<<<nb, kLT, 0, s>>>(n, op, sc, w, q, qn);
}

// out = wgt * sum x*y (sqrt if want_sqrt); single block reduce over a grid of blocks
__global__ void __launch_bounds__(kLT)
k_dot(int n, const double* __restrict__ x, const double* __restrict__ y, double wgt, int want_sqrt,
      double* __restrict__ partial, unsigned* __restrict__ cnt, double* __restrict__ out) {
  double acc = 0.0;
  const int g0 = blockIdx.x * kChunk, g1 = min(n, g0 + kChunk);
  for (int r = g0 + threadIdx.x; r < g1; r += blockDim.x) acc += x[r] * y[r];
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
  if (!last_block(cnt, gridDim.x)) return;
  if (threadIdx.x == 0) {
    double s;
    sum_records<1>(partial, gridDim.x, 1, &s);
    s *= wgt;
    *out = want_sqrt ? sqrt(s) : s;
  }
}

void launch_dot(cudaStream_t s, int n, const double* x, const double* y, double wgt, int want_sqrt, Work& w,
                double* out) {
  const int nb = (n + kChunk - 1) / kChunk;
  ++g_launches;
  k_dot<<<nb, kLT, 0, s>>>(n, x, y, wgt, want_sqrt, w.part1, w.cnt_c, out);
}

// ---------------------------------------------------------------------------
// T_K^-1 for the symmetric tridiagonal Lanczos matrix (Sec. Lanczos: cost ~K^2).
// LU without pivoting (T is positive definite at omega = 0: eps~ >= 1), then one
// forward/backward substitution per unit column, one thread per column.
// ---------------------------------------------------------------------------
__global__ void k_tridiag_inv(int K, const double* __restrict__ alpha, const double* __restrict__ beta,
                              double* __restrict__ d, double* __restrict__ l, double* __restrict__ out,
                              int* __restrict__ status) {
  if (threadIdx.x == 0) {
    int bad = 0;
    d[0] = alpha[0];
    if (d[0] == 0.0) bad = 1;
    for (int i = 1; i < K && !bad; ++i) {
      l[i] = beta[i - 1] / d[i - 1];
      d[i] = alpha[i] - l[i] * beta[i - 1];
      if (d[i] == 0.0 || !isfinite(d[i])) bad = 1;
    }
    *status = bad;
  }
  __syncthreads();
  if (*status) return;
  for (int j = threadIdx.x; j < K; j += blockDim.x) {
    double* x = out + (size_t)j * K;   // column j (symmetric: also row j)
    // forward: L y = e_j
    for (int i = 0; i < K; ++i) x[i] = 0.0;
    x[j] = 1.0;
    for (int i = j + 1; i < K; ++i) x[i] = -l[i] * x[i - 1];
    // backward: U x = y
    x[K - 1] = x[K - 1] / d[K - 1];
    for (int i = K - 2; i >= 0; --i) x[i] = (x[i] - beta[i] * x[i + 1]) / d[i];
  }
}

void launch_tridiag_inv(cudaStream_t s, int K, const double* alpha, const double* beta, double* d, double* l,
                        double* out, int* status) {
  ++g_launches;
  k_tridiag_inv<<<1, 256, 0, s>>>(K, alpha, beta, d, l, out, status);
}

#define GW_LINST(T)                                                                                        \
  template void launch_qmr<T>(cudaStream_t, int, int, int, const double2*, cpx<T>*, cpx<T>*, cpx<T>*,       \
                              cpx<T>*, const cpx<T>*, const int*, const int*, Work&, QmrState, const T*, double,   \
                              int);                                                                        \
  template void launch_gram<T>(cudaStream_t, const cpx<T>*, int, int, const cpx<T>*, int, Work&, double2*, \
                               bool);                                                                      \
  template void launch_proj_update<T>(cudaStream_t, const cpx<T>*, int, int, cpx<T>*, int, const int*,     \
                                      const double2*, Work&, const cpx<T>*, double*, bool);                \
  template void launch_proj<T>(cudaStream_t, const cpx<T>*, int, int, cpx<T>*, int, const int*, Work&,     \
                               const cpx<T>*, double*, bool);                                              \
  template void launch_cg_init<T, double>(cudaStream_t, int, int, const double2*, cpx<T>*, cpx<T>*,       \
                                          const int*, Work&, CgState, const T*, double, double);           \
  template void launch_cg_update<T>(cudaStream_t, int, int, cpx<T>*, cpx<T>*, const cpx<T>*,              \
                                    const cpx<T>*, const double*, Work&, CgState, const T*, double, int); \
  template void launch_add_conv<T>(cudaStream_t, int, int, const cpx<T>*, double2*, const int*);        \
  template void launch_sq_shift<T>(cudaStream_t, int, int, cpx<T>*, const cpx<T>*, const double*, const int*, \
                                   Work&, double*);                                                      \
  template void launch_add_conv_sym<T>(cudaStream_t, int, int, const cpx<T>*, double2*, const int*, const int*);

GW_LINST(double)
GW_LINST(float)
template void launch_gather_rows<double, double>(cudaStream_t, int, int, const double2*, const int*, double2*);
template void launch_gather_rows<float, double>(cudaStream_t, int, int, const double2*, const int*, float2*);
template void launch_gather_rows<double, float>(cudaStream_t, int, int, const float2*, const int*, double2*);

}  // namespace gw

namespace gw {

// ---------------------------------------------------------------------------
// block Lanczos on complex grid fields (Sec. Lanczos, block form; bilinear
// form at complex frequency): Gram matrices and small-matrix combinations
// ---------------------------------------------------------------------------
constexpr int kGT = 8;          // Y columns per block

// out[i * my + j] = wgt * sum_r op(X[i][r]) Y[j][r], op = conj (Hermitian) or identity (bilinear)
// grid (nchunk, ceil(my / kGT)), chunk entries per CTA; one warp per i (strided), lanes over r
__global__ void __launch_bounds__(kLT)
k_cgram(const double2* __restrict__ X, int mx, const double2* __restrict__ Y, int my, size_t n, int conj_x,
        double wgt, double2* __restrict__ partial, unsigned* __restrict__ cnt, double2* __restrict__ out,
        size_t chunk) {
  const int nchunk = gridDim.x;
  const size_t r0 = (size_t)blockIdx.x * chunk, r1 = min(n, r0 + chunk);
  const int j0 = blockIdx.y * kGT;
  const int nj = min(kGT, my - j0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = warp; i < mx; i += nw) {
    double ax[kGT], ay[kGT];
#pragma unroll
    for (int j = 0; j < kGT; ++j) { ax[j] = 0.0; ay[j] = 0.0; }
    for (size_t r = r0 + lane; r < r1; r += 32) {
      double2 x = X[(size_t)i * n + r];
      if (conj_x) x.y = -x.y;
#pragma unroll
      for (int j = 0; j < kGT; ++j) {
        if (j < nj) {
          const double2 y = Y[(size_t)(j0 + j) * n + r];
          ax[j] += x.x * y.x - x.y * y.y;
          ay[j] += x.x * y.y + x.y * y.x;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kGT; ++j) {
      double sx = ax[j], sy = ay[j];
      for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
      }
      if (lane == 0 && j < nj) partial[((size_t)blockIdx.x * mx + i) * my + j0 + j] = make_double2(sx, sy);
    }
  }
  if (!last_block(&cnt[blockIdx.y], nchunk)) return;
  for (int t = threadIdx.x; t < mx * nj; t += blockDim.x) {
    const int i = t / nj, j = t - i * nj;
    double q[2];
    sum_records<2>(reinterpret_cast<const double*>(partial + (size_t)i * my + j0 + j), nchunk,
                   2 * (size_t)mx * my, q);
    out[(size_t)i * my + j0 + j] = make_double2(wgt * q[0], wgt * q[1]);
  }
}

void launch_cgram(cudaStream_t s, const double2* X, int mx, const double2* Y, int my, size_t n, int conj_x,
                  double wgt, double2* partial, unsigned* cnt, double2* out) {
  const size_t chunk = cgram_chunk(n, my);
  const int nchunk = (int)((n + chunk - 1) / chunk);
  dim3 g(nchunk, (my + kGT - 1) / kGT);
  ++g_launches;
  k_cgram<<<g, kLT, 0, s>>>(X, mx, Y, my, n, conj_x, wgt, partial, cnt, out, chunk);
}

// Y[j][r] = (accumulate ? Y[j][r] : 0) + sign * sum_i M[j * mx + i] X[i][r],  j < my (<= 16)
constexpr int kMT = 64;   // coefficients staged per pass
__global__ void __launch_bounds__(kLT)
k_cgemm_n(const double2* __restrict__ M, int my, int mx, const double2* __restrict__ X, size_t n,
          double2* __restrict__ Y, int accumulate, double sign) {
  __shared__ double2 sm[16 * kMT];
  for (size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x; r - threadIdx.x < n;
       r += (size_t)gridDim.x * blockDim.x) {
    double2 acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = make_double2(0, 0);
    for (int i0 = 0; i0 < mx; i0 += kMT) {
      const int ni = min(kMT, mx - i0);
      __syncthreads();
      for (int t = threadIdx.x; t < my * ni; t += blockDim.x) {
        const int j = t / ni, i = t - j * ni;
        sm[j * kMT + i] = M[(size_t)j * mx + i0 + i];
      }
      __syncthreads();
      if (r < n) {
        for (int i = 0; i < ni; ++i) {
          const double2 x = X[(size_t)(i0 + i) * n + r];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            if (j < my) {
              const double2 m = sm[j * kMT + i];
              acc[j].x += m.x * x.x - m.y * x.y;
              acc[j].y += m.x * x.y + m.y * x.x;
            }
          }
        }
      }
    }
    if (r < n) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        if (j < my) {
          double2 y = accumulate ? Y[(size_t)j * n + r] : make_double2(0, 0);
          y.x += sign * acc[j].x;
          y.y += sign * acc[j].y;
          Y[(size_t)j * n + r] = y;
        }
      }
    }
  }
}

void launch_cgemm_n(cudaStream_t s, const double2* M, int my, int mx, const double2* X, size_t n, double2* Y,
                    int accumulate, double sign) {
  const int nb = (int)std::min<size_t>((n + kLT - 1) / kLT, 152 * 8);
  ++g_launches;
  k_cgemm_n<<<nb, kLT, 0, s>>>(M, my, mx, X, n, Y, accumulate, sign);
}

// ---------------------------------------------------------------------------
// inverse of a small dense complex matrix (the block-tridiagonal Lanczos
// matrix) by Gauss-Jordan elimination with partial pivoting, one CTA.
// Work: a [n][n] (destroyed), out [n][n] (starts as the identity).
// ---------------------------------------------------------------------------
__global__ void k_cinv(int n, double2* __restrict__ a, double2* __restrict__ out, int* __restrict__ status) {
  __shared__ int piv;
  __shared__ double2 pv;
  for (size_t t = threadIdx.x; t < (size_t)n * n; t += blockDim.x) {
    const size_t i = t / n, j = t - i * n;
    out[t] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  if (threadIdx.x == 0) *status = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      int best = k;
      double bm = -1.0;
      for (int i = k; i < n; ++i) {
        const double2 v = a[(size_t)i * n + k];
        const double m = v.x * v.x + v.y * v.y;
        if (m > bm) { bm = m; best = i; }
      }
      piv = best;
      if (!(bm > 0.0) || !isfinite(bm)) *status = 1;
    }
    __syncthreads();
    if (*status) return;
    if (piv != k) {
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double2 t1 = a[(size_t)k * n + j]; a[(size_t)k * n + j] = a[(size_t)piv * n + j]; a[(size_t)piv * n + j] = t1;
        double2 t2 = out[(size_t)k * n + j]; out[(size_t)k * n + j] = out[(size_t)piv * n + j]; out[(size_t)piv * n + j] = t2;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) pv = a[(size_t)k * n + k];
    __syncthreads();
    const double den = pv.x * pv.x + pv.y * pv.y;
    const double2 inv = make_double2(pv.x / den, -pv.y / den);
    for (int j = threadIdx.x; j < n; j += blockDim.x) {      // scale the pivot row
      const double2 x = a[(size_t)k * n + j], y = out[(size_t)k * n + j];
      a[(size_t)k * n + j] = make_double2(x.x * inv.x - x.y * inv.y, x.x * inv.y + x.y * inv.x);
      out[(size_t)k * n + j] = make_double2(y.x * inv.x - y.y * inv.y, y.x * inv.y + y.y * inv.x);
    }
    __syncthreads();
    for (size_t t = threadIdx.x; t < (size_t)n * n; t += blockDim.x) {   // eliminate column k elsewhere
      const int i = (int)(t / n), j = (int)(t - (size_t)i * n);
      if (i == k) continue;
      const double2 f = a[(size_t)i * n + k];
      if (j == k) continue;
      const double2 x = a[(size_t)k * n + j], y = out[(size_t)k * n + j];
      double2 ai = a[(size_t)i * n + j], oi = out[(size_t)i * n + j];
      ai.x -= f.x * x.x - f.y * x.y; ai.y -= f.x * x.y + f.y * x.x;
      oi.x -= f.x * y.x - f.y * y.y; oi.y -= f.x * y.y + f.y * y.x;
      a[(size_t)i * n + j] = ai;
      out[(size_t)i * n + j] = oi;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {      // column k of the inverse part
      if (i == k) continue;
      const double2 f = a[(size_t)i * n + k];
      const double2 y = out[(size_t)k * n + k];
      double2 oi = out[(size_t)i * n + k];
      oi.x -= f.x * y.x - f.y * y.y; oi.y -= f.x * y.y + f.y * y.x;
      out[(size_t)i * n + k] = oi;
      a[(size_t)i * n + k] = make_double2(0, 0);
    }
    __syncthreads();
  }
}

void launch_cinv(cudaStream_t s, int n, double2* a, double2* out, int* status) {
  ++g_launches;
  k_cinv<<<1, 1024, 0, s>>>(n, a, out, status);
}

// assemble the block-tridiagonal T: diagonal A_k, B_k below, B_k^H (Hermitian)
// or B_k^T (bilinear) above; T [n][n] with n = K blk
__global__ void k_block_tridiag(int K, int blk, const double2* __restrict__ A, const double2* __restrict__ B,
                                int bilinear, double2* __restrict__ T) {
  const int n = K * blk;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (size_t)n * n;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / n), j = (int)(t - (size_t)i * n);
    const int bi = i / blk, bj = j / blk, ii = i - bi * blk, jj = j - bj * blk;
    double2 v = make_double2(0, 0);
    if (bi == bj) v = A[((size_t)bi * blk + ii) * blk + jj];
    else if (bi == bj + 1) v = B[((size_t)bj * blk + ii) * blk + jj];
    else if (bj == bi + 1) {
      const double2 b = B[((size_t)bi * blk + jj) * blk + ii];
      v = bilinear ? b : make_double2(b.x, -b.y);
    }
    T[t] = v;
  }
}

void launch_block_tridiag(cudaStream_t s, int K, int blk, const double2* A, const double2* B, int bilinear,
                          double2* T) {
  const size_t n2 = (size_t)K * blk * K * blk;
  const int nb = (int)std::min<size_t>((n2 + 255) / 256, 152 * 8);
  ++g_launches;
  k_block_tridiag<<<nb, 256, 0, s>>>(K, blk, A, B, bilinear, T);
}

}  // namespace gw
