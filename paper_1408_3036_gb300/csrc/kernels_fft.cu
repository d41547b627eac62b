// Pencil passes of the batched, sphere-pruned 3D FFT and the operators fused
// into them (Sec. Scaling: H is applied through FFTs at N_FFT ln N_FFT cost).
//
// Layout: a column's grid is N^3 complex values, C order [i0][i1][i2]; a batch
// of columns is contiguous.  Each CTA loads a tile of P = 16 pencils into
// shared memory (leading dimension N + 1), transforms them with fft_tile and
// writes them back.  Three pass kinds:
//   Z: pencils along i2 (contiguous), one per (i0, i1)
//   Y: pencils along i1 for one plane i0 and 16 consecutive i2
//   X: pencils along i0 for one i1 and 16 consecutive i2
// Pruning: after the scatter of sphere coefficients only the pencils of the
// sphere's (i0, i1) disc are non-zero, and only the planes i0 that cut the
// sphere; passes read zeros instead of memory there and write only what the
// next pass reads.  Inverse transforms are unnormalised (u(r) = sum_G c_G
// e^{iGr}); the forward 1/N_g is folded into the multipliers.
#include <algorithm>
#include <cstdio>

#include "fft.cuh"
#include "gw_common.cuh"

namespace gw {

std::atomic<unsigned long long> g_launches{0};

constexpr int kP = 16;          // pencils per tile
constexpr int kThreads = 256;

template <typename T>
__device__ __forceinline__ void load_tw(cpx<T>* stw, const cpx<T>* tw, int N) {
  for (int k = threadIdx.x; k < N; k += blockDim.x) stw[k] = tw[k];
}

template <typename T>
static size_t tile_smem(int N, int nbuf) {
  return (size_t)(nbuf * kP * (N + 1) + N) * sizeof(cpx<T>);
}

// ---------------------------------------------------------------------------
// Z pass
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_zpass(int mode, Geometry g, Prec<T> P, FftPlan pl, cpx<T>* __restrict__ grid,
        cpx<T>* __restrict__ sph, const cpx<T>* __restrict__ sph_r, const double* __restrict__ beta,
        const cpx<T>* __restrict__ sph_p, const double2* __restrict__ E, const int* __restrict__ active,
        const T* __restrict__ real_in, T* __restrict__ real_out, GatherDots dots, const double* __restrict__ tk,
        int ppow) {
  using V = cpx<T>;
  extern __shared__ unsigned char smem_raw[];
  const int N = g.N, LD = N + 1;
  V* A = reinterpret_cast<V*>(smem_raw);
  V* B = A + kP * LD;
  V* stw = B + kP * LD;
  const int col = blockIdx.y;
  if (active && !active[col]) return;
  const bool disc_list = (mode == Z_SCATTER_INV || mode == Z_SCATTER_INV_PUPD || mode == Z_GATHER_FWD ||
                          mode == Z_GATHER_FWD_H);
  const int npen_total = disc_list ? g.npen : g.N2;
  const int p0 = blockIdx.x * kP;
  const int np = min(kP, npen_total - p0);
  load_tw<T>(stw, P.tw, N);
  const size_t gcol = (size_t)col * g.N3;
  const size_t scol = (size_t)col * g.npw;

  // ---- load
  if (mode == Z_SCATTER_INV || mode == Z_SCATTER_INV_PUPD) {
    for (int e = threadIdx.x; e < kP * LD; e += blockDim.x) A[e] = mk<T>(0, 0);
    __syncthreads();
    double bt = 0.0;
    T rtk = (T)0;                                    // 1 / T_ref of the column (0: no preconditioner)
    if (mode == Z_SCATTER_INV_PUPD) {
      bt = beta[col];
      if (tk) rtk = (T)(1.0 / tk[col]);
    }
    const int4 pa = g.pencils[p0], pb = g.pencils[p0 + np - 1];
    const int s0 = pa.z, s1 = pb.z + pb.w;          // sphere entries of the tile are contiguous
    for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
      V val;
      if (mode == Z_SCATTER_INV_PUPD) {
        V rv = sph_r[scol + s];
        if (rtk != (T)0) {                           // z = K r  (K^2 r for a squared operator)
          T k = tpa<T>(P.kin[s] * rtk);
          if (ppow == 2) k *= k;
          rv.x *= k;
          rv.y *= k;
        }
        if (bt < 0.0) {
          val = rv;                                  // first iteration: p = z
        } else {
          const V pv = sph[scol + s];
          val = mk<T>(rv.x + (T)bt * pv.x, rv.y + (T)bt * pv.y);
        }
        sph[scol + s] = val;
      } else {
        val = sph[scol + s];
      }
      A[(g.sph_pen[s] - p0) * LD + g.sph_i2[s]] = val;
    }
  } else {
    for (int e = threadIdx.x; e < np * N; e += blockDim.x) {
      const int p = pl.dN.div(e), k = e - p * N;
      int i0, i1;
      if (disc_list) { const int4 pc = g.pencils[p0 + p]; i0 = pc.x; i1 = pc.y; }
      else { i0 = (p0 + p) / N; i1 = (p0 + p) - i0 * N; }
      const size_t off = gcol + ((size_t)i0 * N + i1) * N + k;
      V val;
      if (real_in && mode == Z_G2G_FWD) val = mk<T>(real_in[off], (T)0);
      else val = grid[off];
      A[p * LD + k] = val;
    }
  }
  __syncthreads();

  // ---- transform
  const bool inv = (mode == Z_SCATTER_INV || mode == Z_SCATTER_INV_PUPD || mode == Z_G2G_INV ||
                    mode == Z_G2G_INV_SUB);
  V* R = inv ? fft_tile<T, +1>(A, B, np, LD, pl, stw) : fft_tile<T, -1>(A, B, np, LD, pl, stw);

  // ---- store
  if (mode == Z_GATHER_FWD || mode == Z_GATHER_FWD_H) {
    double2 Ec = make_double2(0, 0);
    if (mode == Z_GATHER_FWD_H) Ec = E[col];
    const int4 pa = g.pencils[p0], pb = g.pencils[p0 + np - 1];
    const int s0 = pa.z, s1 = pb.z + pb.w;
    for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
      V val = R[(g.sph_pen[s] - p0) * LD + g.sph_i2[s]];
      if (mode == Z_GATHER_FWD_H) {
        const V pv = sph_p[scol + s];
        const T dr = P.kin[s] - (T)Ec.x, di = -(T)Ec.y;      // (kin - E) p
        val.x += dr * pv.x - di * pv.y;
        val.y += dr * pv.y + di * pv.x;
      }
      sph[scol + s] = val;
    }
    if (dots.C) {
      // <C_v | out> over this tile's sphere entries: one warp per v, lanes over G
      __syncthreads();
      const cpx<T>* Cv = reinterpret_cast<const cpx<T>*>(dots.C);
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
      const int nblk = gridDim.x;
      for (int v = warp; v < dots.nocc; v += nw) {
        T ax = 0, ay = 0;
        for (int s = s0 + lane; s < s1; s += 32) {
          const V c = Cv[(size_t)v * g.npw + s];
          const V y = sph[scol + s];
          ax += c.x * y.x + c.y * y.y;
          ay += c.x * y.y - c.y * y.x;
        }
        for (int o = 16; o > 0; o >>= 1) {
          ax += __shfl_xor_sync(0xffffffffu, ax, o);
          ay += __shfl_xor_sync(0xffffffffu, ay, o);
        }
        if (lane == 0) dots.part[((size_t)col * nblk + blockIdx.x) * dots.nocc + v] = make_double2(ax, ay);
      }
      if (last_block(&dots.cnt[col], nblk)) {
        for (int v = threadIdx.x; v < dots.nocc; v += blockDim.x) {
          double q[2];
          sum_records<2>(reinterpret_cast<const double*>(dots.part + (size_t)col * nblk * dots.nocc + v), nblk,
                         2 * (size_t)dots.nocc, q);
          dots.coef[(size_t)v * dots.ncol + col] = make_double2(q[0], q[1]);
        }
      }
    }
  } else {
    for (int e = threadIdx.x; e < np * N; e += blockDim.x) {
      const int p = pl.dN.div(e), k = e - p * N;
      int i0, i1;
      if (disc_list) { const int4 pc = g.pencils[p0 + p]; i0 = pc.x; i1 = pc.y; }
      else { i0 = (p0 + p) / N; i1 = (p0 + p) - i0 * N; }
      const size_t off = gcol + ((size_t)i0 * N + i1) * N + k;
      const V val = R[p * LD + k];
      if (mode == Z_G2G_INV_SUB) real_out[off] = real_in[off] - val.x;
      else if (real_out && mode == Z_G2G_INV) real_out[off] = val.x;
      else grid[off] = val;
    }
  }
}

template <typename T>
void launch_zpass(cudaStream_t s, int mode, const Geometry& g, const Prec<T>& P, const FftPlan& pl,
                  cpx<T>* grid, cpx<T>* sph, const cpx<T>* sph_r, const double* beta,
                  const cpx<T>* sph_p, const double2* E, const int* active, const T* real_in,
                  T* real_out, int ncol, const GatherDots* dots, const double* tk, int ppow) {
  const bool disc_list = (mode == Z_SCATTER_INV || mode == Z_SCATTER_INV_PUPD || mode == Z_GATHER_FWD ||
                          mode == Z_GATHER_FWD_H);
  const int npen = disc_list ? g.npen : g.N2;
  if (npen == 0 || ncol == 0) return;
  dim3 grd((npen + kP - 1) / kP, ncol);
  const size_t sm = tile_smem<T>(g.N, 2);
  ++g_launches;
  GatherDots d;
  if (dots) d = *dots;
  k_zpass<T><<<grd, kThreads, sm, s>>>(mode, g, P, pl, grid, sph, sph_r, beta, sph_p, E, active,
                                        real_in, real_out, d, tk, ppow);
}

// ---------------------------------------------------------------------------
// Y pass: planes x 16-wide i2 chunks
// ---------------------------------------------------------------------------
template <typename T, int SIGN>
__global__ void __launch_bounds__(kThreads)
k_ypass(Geometry g, Prec<T> P, FftPlan pl, cpx<T>* __restrict__ grid, const int* __restrict__ planes,
        int nchunk, const uint8_t* __restrict__ ldmask, const uint8_t* __restrict__ stmask,
        const int* __restrict__ active) {
  using V = cpx<T>;
  extern __shared__ unsigned char smem_raw[];
  const int N = g.N, LD = N + 1;
  V* A = reinterpret_cast<V*>(smem_raw);
  V* B = A + kP * LD;
  V* stw = B + kP * LD;
  const int col = blockIdx.y;
  if (active && !active[col]) return;
  const int pi = blockIdx.x / nchunk;
  const int c0 = (blockIdx.x - pi * nchunk) * kP;
  const int i0 = planes[pi];
  const int np = min(kP, N - c0);
  load_tw<T>(stw, P.tw, N);
  const size_t base = (size_t)col * g.N3 + (size_t)i0 * g.N2 + c0;
  for (int e = threadIdx.x; e < N * kP; e += blockDim.x) {
    const int i1 = e / kP, dz = e - i1 * kP;
    if (dz < np) {
      V val = mk<T>(0, 0);
      if (!ldmask || ldmask[i0 * N + i1]) val = grid[base + (size_t)i1 * N + dz];
      A[dz * LD + i1] = val;
    }
  }
  __syncthreads();
  V* R = fft_tile<T, SIGN>(A, B, np, LD, pl, stw);
  for (int e = threadIdx.x; e < N * kP; e += blockDim.x) {
    const int i1 = e / kP, dz = e - i1 * kP;
    if (dz < np && (!stmask || stmask[i0 * N + i1])) grid[base + (size_t)i1 * N + dz] = R[dz * LD + i1];
  }
}

template <typename T>
void launch_ypass(cudaStream_t s, int inverse, int pruned_in, int pruned_out, const Geometry& g,
                  const Prec<T>& P, const FftPlan& pl, cpx<T>* grid, const int* active, int ncol,
                  int full_planes) {
  const int nchunk = (g.N + kP - 1) / kP;
  const int npl = full_planes ? g.N : g.nplanes;
  const int* planes = full_planes ? g.all_planes : g.planes;
  if (ncol == 0 || npl == 0) return;
  dim3 grd(npl * nchunk, ncol);
  const size_t sm = tile_smem<T>(g.N, 2);
  const uint8_t* lm = pruned_in ? g.disc : nullptr;
  const uint8_t* sm_ = pruned_out ? g.disc : nullptr;
  ++g_launches;
  if (inverse)
    k_ypass<T, +1><<<grd, kThreads, sm, s>>>(g, P, pl, grid, planes, nchunk, lm, sm_, active);
  else
    k_ypass<T, -1><<<grd, kThreads, sm, s>>>(g, P, pl, grid, planes, nchunk, lm, sm_, active);
}

// ---------------------------------------------------------------------------
// X pass with a pointwise multiplier between two transforms:
//   first_inverse = 1: IFFT_x, * mul(r), FFT_x      (H: V(r)/N_g)
//   first_inverse = 0: FFT_x,  * mul(G), IFFT_x     (v^1/2: sqrt(v(G))/N_g)
// mul == nullptr: the first transform only.
// ---------------------------------------------------------------------------
template <typename T, int FIRST>
__global__ void __launch_bounds__(kThreads)
k_xpass_mul(Geometry g, Prec<T> P, FftPlan pl, cpx<T>* __restrict__ grid, const T* __restrict__ mul,
            int nchunk, const uint8_t* __restrict__ ldpl, const uint8_t* __restrict__ stpl,
            const int* __restrict__ active) {
  using V = cpx<T>;
  extern __shared__ unsigned char smem_raw[];
  const int N = g.N, LD = N + 1;
  V* A = reinterpret_cast<V*>(smem_raw);
  V* B = A + kP * LD;
  V* stw = B + kP * LD;
  const int col = blockIdx.y;
  if (active && !active[col]) return;
  const int i1 = blockIdx.x / nchunk;
  const int c0 = (blockIdx.x - i1 * nchunk) * kP;
  const int np = min(kP, N - c0);
  load_tw<T>(stw, P.tw, N);
  const size_t base = (size_t)col * g.N3 + (size_t)i1 * N + c0;
  for (int e = threadIdx.x; e < N * kP; e += blockDim.x) {
    const int i0 = e / kP, dz = e - i0 * kP;
    if (dz < np) {
      V val = mk<T>(0, 0);
      if (!ldpl || ldpl[i0]) val = grid[base + (size_t)i0 * g.N2 + dz];
      A[dz * LD + i0] = val;
    }
  }
  __syncthreads();
  V* R = fft_tile<T, FIRST>(A, B, np, LD, pl, stw);
  V* Q = (R == A) ? B : A;
  if (mul == nullptr) {                       // single transform, no multiplier
    for (int e = threadIdx.x; e < N * kP; e += blockDim.x) {
      const int i0 = e / kP, dz = e - i0 * kP;
      if (dz < np && (!stpl || stpl[i0])) grid[base + (size_t)i0 * g.N2 + dz] = R[dz * LD + i0];
    }
    return;
  }
  for (int e = threadIdx.x; e < N * kP; e += blockDim.x) {
    const int i0 = e / kP, dz = e - i0 * kP;
    if (dz < np) {
      const T m = mul[(size_t)i0 * g.N2 + (size_t)i1 * N + c0 + dz];
      V val = R[dz * LD + i0];
      R[dz * LD + i0] = mk<T>(val.x * m, val.y * m);
    }
  }
  __syncthreads();
  V* S = fft_tile<T, -FIRST>(R, Q, np, LD, pl, stw);
  for (int e = threadIdx.x; e < N * kP; e += blockDim.x) {
    const int i0 = e / kP, dz = e - i0 * kP;
    if (dz < np && (!stpl || stpl[i0])) grid[base + (size_t)i0 * g.N2 + dz] = S[dz * LD + i0];
  }
}

template <typename T>
void launch_xpass_mul(cudaStream_t s, int first_inverse, int pruned_in, int pruned_out, const Geometry& g,
                      const Prec<T>& P, const FftPlan& pl, cpx<T>* grid, const T* mul, const int* active,
                      int ncol) {
  const int nchunk = (g.N + kP - 1) / kP;
  if (ncol == 0) return;
  dim3 grd(g.N * nchunk, ncol);
  const size_t sm = tile_smem<T>(g.N, 2);
  const uint8_t* lp = pruned_in ? g.plane_mask : nullptr;
  const uint8_t* sp = pruned_out ? g.plane_mask : nullptr;
  ++g_launches;
  if (first_inverse)
    k_xpass_mul<T, +1><<<grd, kThreads, sm, s>>>(g, P, pl, grid, mul, nchunk, lp, sp, active);
  else
    k_xpass_mul<T, -1><<<grd, kThreads, sm, s>>>(g, P, pl, grid, mul, nchunk, lp, sp, active);
}

// ---------------------------------------------------------------------------
// X pass, forward, of a pointwise product (first pass of Sphere(FFT(a* y))):
//   out[col] = FFT_x( A[col_a[col]]^(*) * Y[col_y[col]] ) / N_g, planes of the sphere only
// A is either the occupied u_v(r) (a_per_col = 0: index = col_a) or a grid column.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_xpass_prod_fwd(Geometry g, Prec<T> P, FftPlan pl, const cpx<T>* __restrict__ Y, int y_complex,
                 const cpx<T>* __restrict__ Aarr, int conj_a, const int* __restrict__ col_a,
                 const int* __restrict__ col_y, cpx<T>* __restrict__ out, int nchunk,
                 const int* __restrict__ col_a2, const int* __restrict__ col_y2) {
  using V = cpx<T>;
  extern __shared__ unsigned char smem_raw[];
  const int N = g.N, LD = N + 1;
  V* A = reinterpret_cast<V*>(smem_raw);
  V* B = A + kP * LD;
  V* stw = B + kP * LD;
  const int col = blockIdx.y;
  const int i1 = blockIdx.x / nchunk;
  const int c0 = (blockIdx.x - i1 * nchunk) * kP;
  const int np = min(kP, N - c0);
  load_tw<T>(stw, P.tw, N);
  const size_t off1 = (size_t)i1 * N + c0;
  const size_t abase = (size_t)col_a[col] * g.N3 + off1;
  const size_t ybase = (size_t)col_y[col] * g.N3 + off1;
  const T* Yr = reinterpret_cast<const T*>(Y);
  const T sc = (T)(1.0 / (double)g.N3);
  // pair mode (col_a2 given; real A and real Y): the products of two columns
  // packed as a + i b, each real in real space
  const int a2 = col_a2 ? col_a2[col] : -1;
  const size_t a2base = (size_t)(a2 >= 0 ? a2 : 0) * g.N3 + off1;
  const size_t y2base = (size_t)(col_y2 ? col_y2[col] : 0) * g.N3 + off1;
  for (int e = threadIdx.x; e < N * kP; e += blockDim.x) {
    const int i0 = e / kP, dz = e - i0 * kP;
    if (dz < np) {
      const size_t o = (size_t)i0 * g.N2 + dz;
      if (col_a2) {
        const T p1 = Aarr[abase + o].x * Yr[ybase + o];
        const T p2 = (a2 >= 0) ? Aarr[a2base + o].x * Yr[y2base + o] : (T)0;
        A[dz * LD + i0] = mk<T>(p1 * sc, p2 * sc);
      } else {
        V a = Aarr[abase + o];
        if (conj_a) a.y = -a.y;
        V y = y_complex ? Y[ybase + o] : mk<T>(Yr[ybase + o], (T)0);
        V p = cmul(a, y);
        A[dz * LD + i0] = mk<T>(p.x * sc, p.y * sc);
      }
    }
  }
  __syncthreads();
  V* R = fft_tile<T, -1>(A, B, np, LD, pl, stw);
  const size_t obase = (size_t)col * g.N3 + off1;
  for (int e = threadIdx.x; e < N * kP; e += blockDim.x) {
    const int i0 = e / kP, dz = e - i0 * kP;
    if (dz < np && g.plane_mask[i0]) out[obase + (size_t)i0 * g.N2 + dz] = R[dz * LD + i0];
  }
}

template <typename T>
void launch_xpass_prod_fwd(cudaStream_t s, const Geometry& g, const Prec<T>& P, const FftPlan& pl,
                           const cpx<T>* Y, int y_complex, const cpx<T>* A, int /*a_per_col*/, int conj_a,
                           const int* col_a, const int* col_y, cpx<T>* out, int ncol, const int* col_a2,
                           const int* col_y2) {
  const int nchunk = (g.N + kP - 1) / kP;
  if (ncol == 0) return;
  dim3 grd(g.N * nchunk, ncol);
  const size_t sm = tile_smem<T>(g.N, 2);
  ++g_launches;
  k_xpass_prod_fwd<T><<<grd, kThreads, sm, s>>>(g, P, pl, Y, y_complex, A, conj_a, col_a, col_y, out, nchunk,
                                                 col_a2, col_y2);
}

// ---------------------------------------------------------------------------
// X pass, inverse, with the product by u_v and the sum over occupied states
// (last pass of the density reduction, Eq. P1):
//   out[o](r) (+)= scale * sum_{col in group o} U[col_v[col]](r) * IFFT_x(grid[col])(r)
// ---------------------------------------------------------------------------
// With ngrp > 1 the columns of a group are split into ngrp contiguous parts
// (blockIdx.z), each summed into its own partial field part[z][o] (unscaled);
// k_reduce_parts then adds the parts in order: more CTAs in flight for the
// few groups of a Lanczos step.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_xpass_inv_reduce(Geometry g, Prec<T> P, FftPlan pl, const cpx<T>* __restrict__ grid,
                   const int* __restrict__ gstart, const int* __restrict__ col_v, double scale,
                   T* __restrict__ out_real, cpx<T>* __restrict__ out_c, int accumulate, int nchunk,
                   int ngrp, cpx<T>* __restrict__ part, const int* __restrict__ col_v2) {
  using V = cpx<T>;
  extern __shared__ unsigned char smem_raw[];
  const int N = g.N, LD = N + 1;
  V* A = reinterpret_cast<V*>(smem_raw);
  V* B = A + kP * LD;
  V* Acc = B + kP * LD;
  V* stw = Acc + kP * LD;
  const int o = blockIdx.y;
  const int i1 = blockIdx.x / nchunk;
  const int c0 = (blockIdx.x - i1 * nchunk) * kP;
  const int np = min(kP, N - c0);
  load_tw<T>(stw, P.tw, N);
  for (int e = threadIdx.x; e < kP * LD; e += blockDim.x) Acc[e] = mk<T>(0, 0);
  const size_t off1 = (size_t)i1 * N + c0;
  const int cg0 = gstart[o], len = gstart[o + 1] - cg0, z = blockIdx.z;
  const int col_lo = cg0 + (int)(((long long)len * z) / ngrp);
  const int col_hi = cg0 + (int)(((long long)len * (z + 1)) / ngrp);
  for (int col = col_lo; col < col_hi; ++col) {
    __syncthreads();
    const size_t base = (size_t)col * g.N3 + off1;
    for (int e = threadIdx.x; e < N * kP; e += blockDim.x) {
      const int i0 = e / kP, dz = e - i0 * kP;
      if (dz < np) {
        V val = mk<T>(0, 0);
        if (g.plane_mask[i0]) val = grid[base + (size_t)i0 * g.N2 + dz];
        A[dz * LD + i0] = val;
      }
    }
    __syncthreads();
    V* R = fft_tile<T, +1>(A, B, np, LD, pl, stw);
    const size_t ubase = (size_t)col_v[col] * g.N3 + off1;
    const int v2 = col_v2 ? col_v2[col] : -1;
    const size_t u2base = (size_t)(v2 >= 0 ? v2 : 0) * g.N3 + off1;
    for (int e = threadIdx.x; e < N * kP; e += blockDim.x) {
      const int i0 = e / kP, dz = e - i0 * kP;
      if (dz < np) {
        const V x = R[dz * LD + i0];
        V a = Acc[dz * LD + i0];
        if (col_v2) {
          // pair mode: x = f_1 + i f_2 of two real fields, real u_v (real output)
          const T u1 = P.U[ubase + (size_t)i0 * g.N2 + dz].x;
          const T u2 = (v2 >= 0) ? P.U[u2base + (size_t)i0 * g.N2 + dz].x : (T)0;
          a.x += u1 * x.x + u2 * x.y;
        } else {
          const V u = P.U[ubase + (size_t)i0 * g.N2 + dz];
          a.x += u.x * x.x - u.y * x.y;
          a.y += u.x * x.y + u.y * x.x;
        }
        Acc[dz * LD + i0] = a;
      }
    }
  }
  __syncthreads();
  const size_t obase = (size_t)o * g.N3 + off1;
  if (ngrp > 1) {
    const size_t pbase = ((size_t)z * gridDim.y + o) * g.N3 + off1;
    for (int e = threadIdx.x; e < N * kP; e += blockDim.x) {
      const int i0 = e / kP, dz = e - i0 * kP;
      if (dz < np) part[pbase + (size_t)i0 * g.N2 + dz] = Acc[dz * LD + i0];
    }
    return;
  }
  for (int e = threadIdx.x; e < N * kP; e += blockDim.x) {
    const int i0 = e / kP, dz = e - i0 * kP;
    if (dz < np) {
      const size_t idx = obase + (size_t)i0 * g.N2 + dz;
      V a = Acc[dz * LD + i0];
      a.x *= (T)scale;
      a.y *= (T)scale;
      if (out_real) {
        out_real[idx] = accumulate ? out_real[idx] + a.x : a.x;
      } else {
        if (accumulate) { V b0 = out_c[idx]; a.x += b0.x; a.y += b0.y; }
        out_c[idx] = a;
      }
    }
  }
}

// out[o][r] (+)= scale * sum_z part[z][o][r]  (z in order)
template <typename T>
__global__ void k_reduce_parts(size_t n3, int ngroups, int ngrp, const cpx<T>* __restrict__ part, double scale,
                               T* __restrict__ out_real, cpx<T>* __restrict__ out_c, int accumulate) {
  const size_t n = n3 * ngroups;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    cpx<T> a = part[i];
    for (int z = 1; z < ngrp; ++z) {
      const cpx<T> b = part[(size_t)z * n + i];
      a.x += b.x;
      a.y += b.y;
    }
    a.x *= (T)scale;
    a.y *= (T)scale;
    if (out_real) {
      out_real[i] = accumulate ? out_real[i] + a.x : a.x;
    } else {
      if (accumulate) { const cpx<T> b0 = out_c[i]; a.x += b0.x; a.y += b0.y; }
      out_c[i] = a;
    }
  }
}

template <typename T>
void launch_xpass_inv_reduce(cudaStream_t s, const Geometry& g, const Prec<T>& P, const FftPlan& pl,
                             const cpx<T>* grid, const int* group_start, const int* col_v, int ngroups,
                             double scale, T* out_real, cpx<T>* out_cplx, int accumulate, cpx<T>* scratch,
                             size_t scratch_elems, int max_cols, const int* col_v2) {
  const int nchunk = (g.N + kP - 1) / kP;
  if (ngroups == 0) return;
  // split the column sums until about four CTAs per SM are in flight
  const int base = g.N * nchunk * ngroups;
  int ngrp = 1;
  if (scratch) {
    ngrp = std::min(std::min(kMaxReduceParts, std::max(max_cols, 1)), (4 * 152 + base - 1) / base);
    ngrp = (int)std::min<size_t>((size_t)std::max(ngrp, 1), scratch_elems / ((size_t)ngroups * g.N3));
    ngrp = std::max(ngrp, 1);
  }
  dim3 grd(g.N * nchunk, ngroups, ngrp);
  const size_t sm = tile_smem<T>(g.N, 3);
  ++g_launches;
  k_xpass_inv_reduce<T><<<grd, kThreads, sm, s>>>(g, P, pl, grid, group_start, col_v, scale, out_real,
                                                   out_cplx, accumulate, nchunk, ngrp, scratch, col_v2);
  if (ngrp > 1) {
    const size_t n = (size_t)g.N3 * ngroups;
    ++g_launches;
    k_reduce_parts<T><<<(int)std::min<size_t>((n + 255) / 256, 152 * 8), 256, 0, s>>>(
        (size_t)g.N3, ngroups, ngrp, scratch, scale, out_real, out_cplx, accumulate);
  }
}

// ---------------------------------------------------------------------------
// opt-in to > 48 KB dynamic shared memory for the larger grids
// ---------------------------------------------------------------------------
template <typename T>
cudaError_t fft_set_smem_limits() {
  const int mx = (int)tile_smem<T>(kMaxN, 3);
  cudaError_t e = cudaSuccess;
  e = cudaFuncSetAttribute(k_zpass<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx); if (e) return e;
  e = cudaFuncSetAttribute(k_ypass<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx); if (e) return e;
  e = cudaFuncSetAttribute(k_ypass<T, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx); if (e) return e;
  e = cudaFuncSetAttribute(k_xpass_mul<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx); if (e) return e;
  e = cudaFuncSetAttribute(k_xpass_mul<T, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx); if (e) return e;
  e = cudaFuncSetAttribute(k_xpass_prod_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx); if (e) return e;
  e = cudaFuncSetAttribute(k_xpass_inv_reduce<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  return e;
}

#define GW_INST(T)                                                                                         \
  template void launch_zpass<T>(cudaStream_t, int, const Geometry&, const Prec<T>&, const FftPlan&,      \
                                cpx<T>*, cpx<T>*, const cpx<T>*, const double*, const cpx<T>*,           \
                                const double2*, const int*, const T*, T*, int, const GatherDots*,        \
                                const double*, int);                                                          \
  template void launch_ypass<T>(cudaStream_t, int, int, int, const Geometry&, const Prec<T>&,            \
                                const FftPlan&, cpx<T>*, const int*, int, int);                          \
  template void launch_xpass_mul<T>(cudaStream_t, int, int, int, const Geometry&, const Prec<T>&,        \
                                    const FftPlan&, cpx<T>*, const T*, const int*, int);                 \
  template void launch_xpass_prod_fwd<T>(cudaStream_t, const Geometry&, const Prec<T>&, const FftPlan&,  \
                                         const cpx<T>*, int, const cpx<T>*, int, int, const int*,        \
                                         const int*, cpx<T>*, int, const int*, const int*);              \
  template void launch_xpass_inv_reduce<T>(cudaStream_t, const Geometry&, const Prec<T>&,                \
                                           const FftPlan&, const cpx<T>*, const int*, const int*, int,   \
                                           double, T*, cpx<T>*, int, cpx<T>*, size_t, int, const int*);  \
  template cudaError_t fft_set_smem_limits<T>();

GW_INST(double)
GW_INST(float)

}  // namespace gw
