// Shared definitions for the GB300 (sm_103a) Lanczos / Sternheimer dielectric
// library: complex helpers, the per-cell geometry of the plane-wave sphere, and
// the launch interfaces between the translation units.
#pragma once

#include <atomic>

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

namespace gw {

// ---------------------------------------------------------------------------
// complex arithmetic on double2 / float2
// ---------------------------------------------------------------------------
template <typename T> struct CT;
template <> struct CT<double> { using type = double2; };
template <> struct CT<float> { using type = float2; };
template <typename T> using cpx = typename CT<T>::type;

template <typename T> __host__ __device__ __forceinline__ cpx<T> mk(T x, T y) {
  cpx<T> r; r.x = x; r.y = y; return r;
}
template <typename V> __host__ __device__ __forceinline__ V cadd(V a, V b) { V r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename V> __host__ __device__ __forceinline__ V csub(V a, V b) { V r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename V> __host__ __device__ __forceinline__ V cmul(V a, V b) {
  V r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// conj(a) * b
template <typename V> __host__ __device__ __forceinline__ V cmulc(V a, V b) {
  V r; r.x = a.x * b.x + a.y * b.y; r.y = a.x * b.y - a.y * b.x; return r;
}
template <typename V, typename S> __host__ __device__ __forceinline__ V cscale(V a, S s) {
  V r; r.x = a.x * s; r.y = a.y * s; return r;
}
template <typename V> __host__ __device__ __forceinline__ V cconj(V a) { V r; r.x = a.x; r.y = -a.y; return r; }

__host__ __device__ __forceinline__ double2 to_d(float2 a) { return make_double2(a.x, a.y); }
__host__ __device__ __forceinline__ double2 to_d(double2 a) { return a; }
template <typename T> __host__ __device__ __forceinline__ cpx<T> from_d(double2 a);
template <> __host__ __device__ __forceinline__ double2 from_d<double>(double2 a) { return a; }
template <> __host__ __device__ __forceinline__ float2 from_d<float>(double2 a) { return make_float2((float)a.x, (float)a.y); }

// ---------------------------------------------------------------------------
// FFT plan: radices of a length-N transform (Stockham, mixed radix 4/2/3/5)
// ---------------------------------------------------------------------------
// Division by a runtime divisor 1 <= d < 2^31 as multiply-high, add and
// shift (Granlund and Montgomery, PLDI 1994): with s = ceil(log2 d) and
// m = floor(2^32 (2^s - d) / d) + 1, q = (umulhi(x, m) + x) >> s = floor(x / d)
// for 0 <= x < 2^31.  Set on the host (the 64-bit division is slow on the GPU).
struct FastDiv {
  unsigned m = 1, s = 0;
  __host__ __device__ void set(unsigned d) {
    s = 0;
    while ((1ull << s) < d) ++s;
    m = (unsigned)(((1ull << 32) * ((1ull << s) - d)) / d + 1);
  }
  __host__ __device__ __forceinline__ int div(int x) const {
    const unsigned long long hi = ((unsigned long long)(unsigned)x * m) >> 32;
    return (int)((hi + (unsigned)x) >> s);
  }
};

constexpr int kMaxStages = 10;
constexpr int kMaxN = 128;
struct FftPlan {
  int N;
  int nst;
  int rad[kMaxStages];
  int nb[kMaxStages];       // N / rad: butterflies per pencil of each stage
  int ns[kMaxStages];       // span Ns (product of the earlier radices)
  FastDiv dN;               // division by N
  FastDiv dnb[kMaxStages];  // by nb[s]
  FastDiv dns[kMaxStages];  // by ns[s]
};
bool make_plan(int N, FftPlan* p);

// kernel launches issued by this library since it was loaded (host counter)
extern std::atomic<unsigned long long> g_launches;

// ---------------------------------------------------------------------------
// geometry of one cell's sphere on its grid (device arrays)
// ---------------------------------------------------------------------------
struct Geometry {
  int N = 0, N2 = 0, N3 = 0, npw = 0;
  int npen = 0;            // pencils (i0, i1) holding sphere points
  int nplanes = 0;         // planes i0 holding sphere points
  int* sph_i2 = nullptr;   // [npw] z index of each sphere point
  int* sph_pen = nullptr;  // [npw] disc pencil holding each sphere point
  int4* pencils = nullptr; // [npen] (i0, i1, first sphere index, count)
  uint8_t* disc = nullptr; // [N2] 1 where pencil (i0, i1) holds sphere points
  uint8_t* ones = nullptr; // [N2] all ones
  int* planes = nullptr;   // [nplanes] i0 values
  int* plane_sph = nullptr;  // [nplanes + 1] first sphere entry of each plane (entries are i0-major)
  int* plane_mirror = nullptr;  // [nplanes] the plane holding -G of a plane's entries
  int* plane_pen = nullptr;  // [nplanes + 1] first disc pencil of each plane
  int* sph_i1 = nullptr;     // [npw] y index of each sphere point
  int* sph_neg = nullptr;    // [npw] sphere index of -G (bilinear form sum_G x(-G) y(G))
  int* all_planes = nullptr; // [N] 0..N-1
  uint8_t* plane_mask = nullptr; // [N]
};

// Per-precision device data of a cell.
template <typename T> struct Prec {
  cpx<T>* tw = nullptr;      // [N] exp(-2 pi i k / N)
  T* kin = nullptr;          // [npw] |G|^2/2
  T* vloc_s = nullptr;       // [N3] V(r) / N_g
  T* sqv_s = nullptr;        // [N3] sqrt(v(G)) / N_g
  cpx<T>* C = nullptr;       // [nocc][npw] occupied coefficients
  cpx<T>* U = nullptr;       // [nocc][N3] u_v(r) = sum_G c_G e^{iGr}
};

// Kinetic preconditioner of the Sternheimer solvers (Teter, Payne and Allan,
// Phys. Rev. B 40, 12255 (1989)): for x = (|G|^2/2) / T_ref, with T_ref the
// kinetic energy of the occupied state of the column,
//   K(x) = (27 + 18x + 12x^2 + 8x^3) / (27 + 18x + 12x^2 + 8x^3 + 16x^4),
// 1 for x << 1 and 1/(2x) for x >> 1: a smooth inverse of the kinetic energy
// that leaves the low-lying components alone.  K(-G) = K(G), so it is symmetric
// in the bilinear form as well.
template <typename T>
__device__ __forceinline__ T tpa(T x) {
  const T p = (T)27 + x * ((T)18 + x * ((T)12 + x * (T)8));
  return p / (p + (T)16 * (x * x) * (x * x));
}

// Adds n records of W doubles (record k at p + k * stride) in index order --
// the rounding of a plain loop -- with the loads of eight records in flight
// (the last block of a reduction otherwise waits one memory round trip per
// record).
template <int W, typename X = double>
__device__ __forceinline__ void sum_records(const X* __restrict__ p, int n, size_t stride, X* s) {
#pragma unroll
  for (int w = 0; w < W; ++w) s[w] = (X)0;
  int k = 0;
  for (; k + 8 <= n; k += 8) {
    X t[8][W];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int w = 0; w < W; ++w) t[u][w] = p[(size_t)(k + u) * stride + w];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int w = 0; w < W; ++w) s[w] += t[u][w];
  }
  for (; k < n; ++k)
#pragma unroll
    for (int w = 0; w < W; ++w) s[w] += p[(size_t)k * stride + w];
}

// Deterministic cross-block reduction: every block writes its partial sums,
// then takes a ticket; the block drawing the last ticket sees all partials
// (after the fences) and resets the ticket for the next launch.
__device__ __forceinline__ bool last_block(unsigned* cnt, unsigned nblk) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(cnt, 1u);
    is_last = (t == nblk - 1);
    if (is_last) *cnt = 0u;
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// Projector coefficients fused into a gather pass: coef[v * ncol + col] =
// <C_v|out_col> = sum_G conj(C[v][G]) out[col][G].
struct GatherDots {
  const void* C = nullptr;     // cpx<T> [nocc][npw]
  int nocc = 0;
  int ncol = 0;
  double2* part = nullptr;     // [ncol][blocks per column][nocc]
  unsigned* cnt = nullptr;     // [ncol] tickets
  double2* coef = nullptr;     // [nocc][ncol]
};

// ---------------------------------------------------------------------------
// kernel launchers (kernels_fft.cu)
// ---------------------------------------------------------------------------
// Which grid points a pass loads / stores; see kernels_fft.cu.
enum ZMode { Z_SCATTER_INV = 0, Z_GATHER_FWD = 1, Z_G2G_FWD = 2, Z_G2G_INV = 3, Z_SCATTER_INV_PUPD = 4,
             Z_GATHER_FWD_H = 5, Z_G2G_INV_SUB = 6 };

template <typename T>
void launch_zpass(cudaStream_t s, int mode, const Geometry& g, const Prec<T>& P, const FftPlan& pl,
                  cpx<T>* grid, cpx<T>* sph, const cpx<T>* sph_r, const double* beta,
                  const cpx<T>* sph_p, const double2* E, const int* active, const T* real_in,
                  T* real_out, int ncol, const GatherDots* dots = nullptr, const double* tk = nullptr,
                  int ppow = 1);
template <typename T>
void launch_ypass(cudaStream_t s, int inverse, int pruned_in, int pruned_out, const Geometry& g,
                  const Prec<T>& P, const FftPlan& pl, cpx<T>* grid, const int* active, int ncol, int full_planes);
template <typename T>
void launch_xpass_mul(cudaStream_t s, int first_inverse, int pruned_in, int pruned_out, const Geometry& g,
                      const Prec<T>& P, const FftPlan& pl, cpx<T>* grid, const T* mul, const int* active,
                      int ncol);
// out(v,b) = FFT_x(conj(U[v]) * Y[b]) / N_g   (first pass of a pruned forward transform)
// Pair mode (col_a2, col_y2 given; A and Y real): out = FFT_x(A[a] Y[y] + i A[a2] Y[y2]) / N_g
// (col_a2[col] < 0: the first product alone).
template <typename T>
void launch_xpass_prod_fwd(cudaStream_t s, const Geometry& g, const Prec<T>& P, const FftPlan& pl,
                           const cpx<T>* Y, int y_complex, const cpx<T>* A, int a_per_col, int conj_a,
                           const int* col_a, const int* col_y, cpx<T>* out, int ncol,
                           const int* col_a2 = nullptr, const int* col_y2 = nullptr);
// dn[o] += scale * sum_{v} U[v] * IFFT_x(grid[col])   for col in group o (last pass of inverse);
// pair mode (col_v2 given, real output): grid[col] holds f_1 + i f_2 of two
// real fields and the sum takes Re U[col_v] f_1 + Re U[col_v2] f_2.
// scratch (optional, scratch_elems complex entries) lets the sum over the at
// most max_cols columns of a group be split over several CTAs.
constexpr int kMaxReduceParts = 8;
template <typename T>
void launch_xpass_inv_reduce(cudaStream_t s, const Geometry& g, const Prec<T>& P, const FftPlan& pl,
                             const cpx<T>* grid, const int* group_start, const int* col_v, int ngroups,
                             double scale, T* out_real, cpx<T>* out_cplx, int accumulate,
                             cpx<T>* scratch = nullptr, size_t scratch_elems = 0, int max_cols = 1,
                             const int* col_v2 = nullptr);

}  // namespace gw
