// Persistent conjugate-gradient solver for the Sternheimer equations
// (Eq. P2: (H - e_v) x = P_c psi_v* dV, projected on the conduction space at
// every step as in Sec. Avoiding summations).
//
// One cooperative launch runs a whole CG pass for every column (occupied
// state x field) with per-column convergence masks.  The work of an iteration
// is cut into tasks that the CTAs draw, in one fixed global order, from an
// atomic ticket counter; a task waits only for the tasks of its own group that
// it depends on (per-group completion counters), and loads what it can while
// it waits.  Every wait is bounded and, when the bound runs out, sets an error
// flag on which every CTA returns.  No grid-wide barrier: a group whose
// columns converge early stops holding the others, and the tasks of different
// groups overlap.  (A dataflow variant -- tasks queued by the last task of the
// phase they depend on -- measured slower: the solve is bound by each group's
// chain of dependent tasks, and the queue adds a hop to every link of it.)
//
// Groups: two columns whose right-hand sides are real in real space
// (b(-G) = conj b(G), true for real fields at omega = 0) share one complex
// transform, z = u_1 + i u_2; V(r) is real, so F(V z)(G) = F(V u_1)(G) +
// i F(V u_2)(G) and each part is recovered from G and -G:
//   F(V u_1)(G) = (Y(G) + conj Y(-G)) / 2,  F(V u_2)(G) = (Y(G) - conj Y(-G)) / 2i.
// The vectors of such a pair stay exactly Hermitian-symmetric in floating
// point (the right-hand side is symmetrised on entry, the projector rows are
// symmetric, every update combines G and -G the same way).  Other columns run
// one per group.
//
// Recurrences: the one-reduction form of preconditioned CG of Chronopoulos and
// Gear (J. Comput. Appl. Math. 25, 153 (1989)): with u = K r and
// w = P_c (H - E) u,
//   gamma = r^H u,  delta = u^H w,  beta = gamma / gamma_prev,
//   alpha = gamma / (delta - beta gamma / alpha_prev),
//   p = u + beta p,  s = w + beta s,  x += alpha p,  r -= alpha s,
// so both inner products of an iteration come out of the one reduction that
// follows the operator application (K: kinetic preconditioner, 1 without one).
//
// Tasks of iteration it for group g (tickets: all A tasks of the iteration,
// then all B, then all C; group by group):
//   A (g, plane i0)  sum the group's C records of it - 1 (projector
//      coefficients, delta) and A partials (gamma, |r|^2) in plane order,
//      decide per column (the same bits in every A task of the group), update
//      x, r, p, s on the plane's sphere entries, u = K r, the plane's partial
//      gamma and |r|^2; scatter the packed u, z-IFFT of the disc rows and
//      y-IFFT of the plane in shared memory, store the plane.
//      Depends on every C task of the group at it - 1 (none at it = 0: the
//      launch before sets r = b, x = p = s = 0).
//   B (g, i1)  x-IFFT, * V(r)/N_g, x-FFT on the (i0, i2) slab.  Depends on the
//      group's A tasks of it.
//   C (g, plane)  y-FFT, z-FFT of the disc rows, gather Y = F(V z) on the
//      plane's entries, and the plane's record: <C_v|Y>, <C_v|kin u_c>,
//      <C_v|u_c>, u_c^H Y, sum kin |u_c|^2, sum |u_c|^2.  Depends on the
//      group's B tasks of it.
// Data read across CTAs goes through L2 (ld.global.cg).
#include <algorithm>
#include <cstdio>

#include <mutex>

#include "fft.cuh"
#include "gw_common.cuh"
#include "linalg.cuh"
#include "pcg.cuh"

namespace gw {

// Control words: [0] ticket, [1] groups done, [2] error flag, [3] unused;
// then per group the completed A, B and C tasks and done + 1 (the iteration
// + 1 at which the group finished).
constexpr int kCtlHead = 4;

template <typename T>
struct PcgArgs {
  Geometry g;
  FftPlan pl;
  const cpx<T>* tw;
  const T* kin;
  const T* vloc_s;
  const cpx<T>* C;
  int nocc, npw, ncol, ngrp, W, maxplane;
  const T* cin;               // [ncol][4] per column, in T: E, 1 / T_ref (0: no preconditioner), |r|^2 floor,
                              // 1 when the column is solved (written by k_pcg_prep)
  T tol2;
  int maxit;
  int pf;                     // 1: the A tasks prefetch r, p, s, x into shared memory
  int crs;                    // 1: A and C tasks stage the plane's occupied rows C in shared memory
  cpx<T>* x;
  cpx<T>* r;
  cpx<T>* p;
  cpx<T>* s;
  cpx<T>* Y;                  // [ngrp][npw]
  cpx<T>* grid;               // [ngrp][N3]
  unsigned char* rec;         // [ngrp][nplanes] records of the C tasks
  size_t rec_bytes;
  unsigned char* apart;       // [2][ngrp][nplanes][W][2] Acc<T>: partial gamma, |r|^2 of the A tasks
  unsigned char* cst;         // [2][ncol] PcgColT<T> column state, by iteration parity
  unsigned* ctl;              // control words (above)
  int* iters_out;
  int* flag_out;
  double* rr_out;
  unsigned long long spin_limit;
  unsigned long long* ptask;  // optional [3][12]: per task kind A, B, C: tasks run, busy ns, wait ns, skipped,
                              // then the busy time of up to eight sub-phases (ns)
};

template <typename V> __device__ __forceinline__ V ldcg(const V* p);
template <> __device__ __forceinline__ float2 ldcg<float2>(const float2* p) { return __ldcg(p); }
template <> __device__ __forceinline__ double2 ldcg<double2>(const double2* p) { return __ldcg(p); }

// Scalar sums of the CG (inner products, |r|^2, the plane records): FP64 in
// the FP64 kernel; in the FP32 kernel a pair of floats hi + lo whose
// additions are error-free transformations (Knuth's TwoSum, then a
// renormalising FastTwoSum; products by Dekker's splitting through an FMA),
// which keeps the sums close to FP64 accuracy with FP32 instructions only --
// this GPU runs FP64 at a small fraction of its FP32 rate.
template <typename T> struct AccOf { using type = double; };
template <> struct AccOf<float> { using type = float2; };
template <typename T> using Acc = typename AccOf<T>::type;

__device__ __forceinline__ double acc_add(double a, double b) { return a + b; }
__device__ __forceinline__ float2 acc_add(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float bb = __fsub_rn(s, a.x);
  const float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
  const float t = __fadd_rn(e, __fadd_rn(a.y, b.y));
  const float h = __fadd_rn(s, t);
  return make_float2(h, __fsub_rn(t, __fsub_rn(h, s)));
}
__device__ __forceinline__ double acc_scale(double a, double c) { return a * c; }
__device__ __forceinline__ float2 acc_scale(float2 a, float c) {
  const float p = __fmul_rn(a.x, c);
  const float e = fmaf(a.y, c, fmaf(a.x, c, -p));
  const float h = __fadd_rn(p, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, p)));
}
__device__ __forceinline__ double acc_of(double x) { return x; }
__device__ __forceinline__ float2 acc_of(float x) { return make_float2(x, 0.f); }
__device__ __forceinline__ double acc_val(double a) { return a; }
__device__ __forceinline__ float acc_val(float2 a) { return __fadd_rn(a.x, a.y); }
__device__ __forceinline__ double acc_shfl(double a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
__device__ __forceinline__ float2 acc_shfl(float2 a, int o) {
  return make_float2(__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o));
}
__device__ __forceinline__ double acc_ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float2 acc_ldcg(const float2* p) { return __ldcg(p); }

// Per-column CG state, in the precision of the vectors.
template <typename T>
struct PcgColT {
  T gam, alpha, stop, rmin, rbest;
  int it, itb, active, flag;
};

// Column state written by another CTA: read through L2.
template <typename T>
__device__ __forceinline__ PcgColT<T> ld_col(const PcgColT<T>* p) {
  PcgColT<T> c;
  c.gam = __ldcg(&p->gam);
  c.alpha = __ldcg(&p->alpha);
  c.stop = __ldcg(&p->stop);
  c.rmin = __ldcg(&p->rmin);
  c.rbest = __ldcg(&p->rbest);
  c.it = __ldcg(&p->it);
  c.itb = __ldcg(&p->itb);
  c.active = __ldcg(&p->active);
  c.flag = __ldcg(&p->flag);
  return c;
}

// Sums over the block of NV values per thread, in Acc (the NV sums land in
// out[0 .. NV), visible to every thread after the call); up to 16 warps.
template <int NV, typename A>
__device__ __forceinline__ void block_sum_n(A (&v)[NV], A* sh, A* out) {
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] = acc_add(v[k], acc_shfl(v[k], o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k * 16 + w] = v[k];
  __syncthreads();
  if (threadIdx.x < NV) {
    A t = sh[threadIdx.x * 16];
    for (int q = 1; q < nw; ++q) t = acc_add(t, sh[threadIdx.x * 16 + q]);
    out[threadIdx.x] = t;
  }
  __syncthreads();
}

struct PcgLayout {
  size_t A, B, U, K, tw, rowmap, red, S, coef, dsum, ap, col, pre, IX, X, CR, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Shared memory of one CTA: two FFT tiles N x (N+1), the plane's u_c (C
// tasks) or Y(G), conj Y(-G) (A tasks), |G|^2/2 on the plane's entries,
// twiddles, the row map of a plane's disc pencils, reduction scratch, the
// summed records, the group's projector coefficients and <C_v|u_c> (A tasks),
// scalar sums, the staged per-plane partials of the A tasks, per-column
// scalars, the plane's -G indices and scatter positions (A tasks), with pf
// the plane's r, p, s, x prefetched by the A tasks, and with crs the plane's
// occupied rows C staged by the A and C tasks.
__host__ __device__ inline PcgLayout pcg_layout(int N, int nocc, int W, int maxplane, int vsize, bool pf,
                                                bool crs) {
  PcgLayout L;
  L.A = 0;
  L.B = align16(L.A + (size_t)N * (N + 1) * vsize);
  L.U = align16(L.B + (size_t)N * (N + 1) * vsize);
  L.K = align16(L.U + (size_t)W * maxplane * vsize);
  L.tw = align16(L.K + (size_t)maxplane * (vsize / 2));
  L.rowmap = align16(L.tw + (size_t)N * vsize);
  L.red = align16(L.rowmap + (size_t)N * sizeof(int));
  L.S = align16(L.red + 8 * 16 * sizeof(double));
  L.coef = align16(L.S + (size_t)(1 + 2 * W) * nocc * vsize);
  L.dsum = align16(L.coef + (size_t)2 * W * nocc * vsize);
  L.ap = align16(L.dsum + 24 * sizeof(double));
  L.col = align16(L.ap + (size_t)N * 2 * W * sizeof(double));
  L.pre = align16(L.col + 2 * 8 * sizeof(double));
  L.IX = align16(L.pre + 2 * (4 * sizeof(double) + sizeof(PcgCol)));
  L.X = align16(L.IX + (size_t)2 * maxplane * sizeof(int));
  L.CR = align16(L.X + (pf ? (size_t)W * 4 * maxplane * vsize : 0));
  L.total = align16(L.CR + (crs ? (size_t)nocc * maxplane * vsize : 0));
  return L;
}

// Record of one (group, plane) C task:
//   V [nocc]        D_v   = sum conj(C_v) Y
//   V [W][nocc]     K_c,v = sum conj(C_v) kin u_c
//   V [W][nocc]     U_c,v = sum conj(C_v) u_c
//   Acc<T> [W][4]   Re, Im of u_c^H Y, sum kin |u_c|^2, sum |u_c|^2 (8 bytes each)
__host__ __device__ inline size_t pcg_rec_bytes(int nocc, int W, int vsize) {
  return align16((size_t)(1 + 2 * W) * nocc * vsize) + (size_t)32 * W;
}

// Bounded wait of thread 0 for cnt >= target.  Returns 0 to run the task, 1 to
// skip it (the group finished at an A task of iteration done1 - 1 with
// done1 <= skip_le), 2 on error (the bound ran out here or elsewhere).
__device__ __forceinline__ int wait_dep(const unsigned* cnt, unsigned target, const unsigned* done1, unsigned skip_le,
                                        unsigned* ctl, unsigned long long limit) {
  unsigned long long spins = 0;
  while (true) {
    // the three words loaded back to back: one L2 round trip per poll
    const unsigned d = *(volatile const unsigned*)done1;
    const unsigned c = *(volatile const unsigned*)cnt;
    const unsigned e = *(volatile const unsigned*)&ctl[2];
    if (d != 0u && d <= skip_le) return 1;
    if (c >= target) break;
    if (e) return 2;
    if (++spins > limit) { atomicExch(&ctl[2], 1u); return 2; }
    if (spins > 8) __nanosleep(32);
  }
  __threadfence();
  const unsigned d = *(volatile const unsigned*)done1;
  return (d != 0u && d <= skip_le) ? 1 : 0;
}

// Completion of a task: every thread's writes fenced, then one count.
__device__ __forceinline__ void signal_done(unsigned* cnt) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(cnt, 1u);
}

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Optional task timing (thread 0): wait from t0 to t1, work from t1 to now.
__device__ __forceinline__ void task_time(unsigned long long* pt, int kind, unsigned long long t0,
                                          unsigned long long t1, bool ran) {
  if (!pt || threadIdx.x != 0) return;
  unsigned long long* q = pt + 12 * kind;
  if (ran) {
    atomicAdd(q + 0, 1ull);
    atomicAdd(q + 1, gtime() - t1);
  } else {
    atomicAdd(q + 3, 1ull);
  }
  atomicAdd(q + 2, t1 - t0);
}

// Optional sub-phase mark (thread 0): adds now - *t to slot 4 + k of the task
// kind and moves *t to now.
__device__ __forceinline__ void task_mark(unsigned long long* pt, int kind, int k, unsigned long long* t) {
  if (!pt || threadIdx.x != 0) return;
  const unsigned long long now = gtime();
  atomicAdd(pt + 12 * kind + 4 + k, now - *t);
  *t = now;
}


// Rows of n contiguous complex values between device memory (row k at
// g + k * stride) and a shared tile (row k at t + k * LDp), for k < nrow;
// rows whose mask entry is 0 are zero in the tile and left alone in memory.
// FP32 values move in pairs (16-byte accesses) when every row start is even.
template <typename T>
__device__ __forceinline__ void load_rows(cpx<T>* t, int LDp, const cpx<T>* g, size_t stride, int nrow, int n,
                                          const unsigned char* mask) {
  using V = cpx<T>;
  if (sizeof(T) == 4 && (n & 1) == 0 && (stride & 1) == 0 && ((reinterpret_cast<size_t>(g) & 15) == 0)) {
    const int h = n >> 1, tot = nrow * h;
#pragma unroll 4
    for (int f = threadIdx.x; f < tot; f += blockDim.x) {
      const int k = f / h, j = 2 * (f - k * h);
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (!mask || mask[k]) v = __ldcg(reinterpret_cast<const float4*>(g + (size_t)k * stride + j));
      t[k * LDp + j] = mk<T>((T)v.x, (T)v.y);
      t[k * LDp + j + 1] = mk<T>((T)v.z, (T)v.w);
    }
  } else {
    const int tot = nrow * n;
#pragma unroll 8
    for (int f = threadIdx.x; f < tot; f += blockDim.x) {
      const int k = f / n, j = f - k * n;
      t[k * LDp + j] = (!mask || mask[k]) ? ldcg(g + (size_t)k * stride + j) : mk<T>(0, 0);
    }
  }
}

template <typename T>
__device__ __forceinline__ void store_rows(cpx<T>* g, size_t stride, const cpx<T>* t, int LDp, int nrow, int n,
                                           const unsigned char* mask) {
  if (sizeof(T) == 4 && (n & 1) == 0 && (stride & 1) == 0 && ((reinterpret_cast<size_t>(g) & 15) == 0)) {
    const int h = n >> 1, tot = nrow * h;
#pragma unroll 4
    for (int f = threadIdx.x; f < tot; f += blockDim.x) {
      const int k = f / h, j = 2 * (f - k * h);
      if (mask && !mask[k]) continue;
      const cpx<T> u = t[k * LDp + j], v = t[k * LDp + j + 1];
      *reinterpret_cast<float4*>(g + (size_t)k * stride + j) = make_float4((float)u.x, (float)u.y, (float)v.x,
                                                                           (float)v.y);
    }
  } else {
    const int tot = nrow * n;
    for (int f = threadIdx.x; f < tot; f += blockDim.x) {
      const int k = f / n, j = f - k * n;
      if (!mask || mask[k]) g[(size_t)k * stride + j] = t[k * LDp + j];
    }
  }
}

// The plane's occupied rows C[v][s0 .. s0 + ns) into CR[v][0 .. ns) (static
// data: loaded at the start of a task, before its waits).
template <typename T>
__device__ __forceinline__ void stage_rows(cpx<T>* CR, int maxplane, const cpx<T>* C, int npw, int nocc, int s0,
                                           int ns) {
  const int tot = nocc * ns;
#pragma unroll 8
  for (int f = threadIdx.x; f < tot; f += blockDim.x) {
    const int v = f / ns, e = f - v * ns;
    CR[(size_t)v * maxplane + e] = C[(size_t)v * npw + s0 + e];
  }
}

// ---------------------------------------------------------------------------
// A task
// ---------------------------------------------------------------------------
template <typename T>
__device__ void task_A(const PcgArgs<T>& a, int it, int gi, int pi, unsigned char* sm, const PcgLayout& L,
                       int* s_ctl) {
  using V = cpx<T>;
  using SA = Acc<T>;
  const Geometry& g = a.g;
  const int N = g.N, LDp = N + 1, P = g.nplanes, W = a.W, nocc = a.nocc;
  const int c0 = gi * W, nc = min(W, a.ncol - c0);
  unsigned* gc = a.ctl + kCtlHead + 4 * gi;
  V* Ab = reinterpret_cast<V*>(sm + L.A);
  V* Bb = reinterpret_cast<V*>(sm + L.B);
  const V* stw = reinterpret_cast<const V*>(sm + L.tw);
  int* rowmap = reinterpret_cast<int*>(sm + L.rowmap);
  SA* red = reinterpret_cast<SA*>(sm + L.red);
  V* Ssum = reinterpret_cast<V*>(sm + L.S);            // the records' projector sums over planes
  V* coefT = reinterpret_cast<V*>(sm + L.coef);        // [W][nocc] coefficients, then [W][nocc] <C_v|u_c>
  SA* dsum = reinterpret_cast<SA*>(sm + L.dsum);
  T* colv = reinterpret_cast<T*>(sm + L.col);          // [c * 8 + k]: alpha, beta, active, E, 1 / T_ref
  const int i0 = g.planes[pi];
  const int s0 = g.plane_sph[pi], s1 = g.plane_sph[pi + 1];
  const int q0 = g.plane_pen[pi], npp = g.plane_pen[pi + 1] - q0;
  const int ns = s1 - s0;
  const size_t rb = a.rec_bytes;
  const int nv = (1 + 2 * W) * nocc;
  const bool pf = a.pf != 0;
  V* X = reinterpret_cast<V*>(sm + L.X);              // [W][4][maxplane]: r, p, s, x (pf)
  int* IXn = reinterpret_cast<int*>(sm + L.IX);       // [maxplane]: position of -G in the mirror plane
  int* IXs = IXn + a.maxplane;                        // [maxplane]: position in tile A
  T* Ks = reinterpret_cast<T*>(sm + L.K);             // [maxplane]: |G|^2/2
  V* Ys = reinterpret_cast<V*>(sm + L.U);             // [maxplane]: Y on the plane, then (W = 2) on its mirror
  const int pm = g.plane_mirror[pi];
  const int s0m = g.plane_sph[pm];
  V* CR = reinterpret_cast<V*>(sm + L.CR);            // [nocc][maxplane]: the plane's rows of C (crs)
  unsigned long long t0 = 0, t1 = 0;
  // First wait (it > 0, pf): the group's A tasks of it - 1 are done, so the
  // plane's r, p, s, x are final; they and the plane's static per-entry values
  // are loaded while the C tasks of it - 1 finish (second wait).
  if (threadIdx.x == 0) {
    int w = 0;
    if (a.ptask) t0 = gtime();
    if (it > 0 && pf) w = wait_dep(gc + 0, (unsigned)(it * P), gc + 3, (unsigned)it, a.ctl, a.spin_limit);
    if (a.ptask) t1 = gtime();
    s_ctl[0] = w;
  }
  __syncthreads();
  if (s_ctl[0] == 2) return;
  if (s_ctl[0] == 1) {                 // the group finished earlier: nothing left to do
    task_time(a.ptask, 0, t0, t1, false);
    return;
  }
  for (int e = threadIdx.x; e < ns; e += blockDim.x) {
    const int G = s0 + e;
    Ks[e] = a.kin[G];
    IXn[e] = g.sph_neg[G] - s0m;
    IXs[e] = (g.sph_pen[G] - q0) * LDp + g.sph_i2[G];
  }
  if (a.crs) stage_rows<T>(CR, a.maxplane, a.C, a.npw, nocc, s0, ns);
  if (pf) {
    const int nvec = (it == 0) ? 1 : 4, tot = nc * nvec * ns;
#pragma unroll 8
    for (int f = threadIdx.x; f < tot; f += blockDim.x) {
      const int cv = f / ns, e = f - cv * ns;
      const int c = cv / nvec, k = cv - c * nvec;
      const V* src = (k == 0) ? a.r : (k == 1) ? a.p : (k == 2) ? a.s : a.x;
      X[((size_t)c * 4 + k) * a.maxplane + e] = ldcg(src + (size_t)(c0 + c) * a.npw + s0 + e);
    }
  }
  // Second wait (it > 0): the group's C tasks of it - 1 are done.
  if (threadIdx.x == 0) {
    int w = 0;
    if (it > 0) w = wait_dep(gc + 2, (unsigned)(it * P), gc + 3, (unsigned)it, a.ctl, a.spin_limit);
    if (a.ptask) t1 = gtime();
    s_ctl[0] = w;
  }
  __syncthreads();
  if (s_ctl[0] == 2) return;
  if (s_ctl[0] == 1) {
    task_time(a.ptask, 0, t0, t1, false);
    return;
  }
  unsigned long long tm = t1;

  // ---- column scalars
  if (it == 0) {
    for (int c = threadIdx.x; c < W; c += blockDim.x) {
      const bool present = c < nc;
      colv[c * 8 + 0] = (T)0;
      colv[c * 8 + 1] = (T)0;
      colv[c * 8 + 2] = present ? (T)1 : (T)0;
      colv[c * 8 + 3] = present ? a.cin[(c0 + c) * 4 + 0] : (T)0;
      colv[c * 8 + 4] = present ? a.cin[(c0 + c) * 4 + 1] : (T)0;
    }
  } else {
    // One round of loads: the group's P records (shared-memory tiles A and B,
    // when they fit), the A partials of the previous iteration, and each
    // column's state and inputs; then every sum from shared memory.
    const unsigned char* src = a.rec + (size_t)gi * P * rb;
    const size_t nb16 = (size_t)P * rb / 16;
    const bool staged = nb16 * 16 <= L.U - L.A;
    const unsigned char* stg = staged ? sm + L.A : src;
    if (staged) {
      const float4* s4 = reinterpret_cast<const float4*>(src);
      float4* d4 = reinterpret_cast<float4*>(sm + L.A);
#pragma unroll 4
      for (size_t e = threadIdx.x; e < nb16; e += blockDim.x) d4[e] = __ldcg(s4 + e);
    }
    {
      const V* Yg = a.Y + (size_t)gi * a.npw;
#pragma unroll 4
      for (int e = threadIdx.x; e < ns; e += blockDim.x) {
        Ys[e] = ldcg(Yg + s0 + e);
        if (W == 2) Ys[a.maxplane + e] = ldcg(Yg + s0m + e);     // the mirror plane, in its own order
      }
    }
    const SA* ap = reinterpret_cast<const SA*>(a.apart) + ((size_t)((it - 1) & 1) * a.ngrp + gi) * P * W * 2;
    SA* aps = reinterpret_cast<SA*>(sm + L.ap);
    for (int j = threadIdx.x; j < P * W * 2; j += blockDim.x) aps[j] = acc_ldcg(ap + j);
    T* pre = reinterpret_cast<T*>(sm + L.pre);                            // [W][4]: E, 1/T_ref, floor, on
    PcgColT<T>* pcs = reinterpret_cast<PcgColT<T>*>(sm + L.pre + 2 * 4 * sizeof(double));
    if (threadIdx.x < nc) {
      const int col = c0 + threadIdx.x;
#pragma unroll
      for (int k = 0; k < 4; ++k) pre[threadIdx.x * 4 + k] = a.cin[col * 4 + k];
      if (it > 1)
        pcs[threadIdx.x] = ld_col(reinterpret_cast<const PcgColT<T>*>(a.cst) + (size_t)((it - 1) & 1) * a.ncol + col);
    }
    __syncthreads();
    task_mark(a.ptask, 0, 0, &tm);     // loads
    // projector sums in T over the planes in order (threads j < nv)
    const size_t dbase = align16((size_t)nv * sizeof(V));
    for (int j = threadIdx.x; j < nv; j += blockDim.x) {
      T sx = 0, sy = 0;
      for (int q = 0; q < P; ++q) {
        const V v = staged ? reinterpret_cast<const V*>(stg + (size_t)q * rb)[j]
                           : ldcg(reinterpret_cast<const V*>(stg + (size_t)q * rb) + j);
        sx += v.x;
        sy += v.y;
      }
      Ssum[j] = mk<T>(sx, sy);
    }
    // the 6 W scalar sums in Acc (per column: Re/Im u^H Y, kin |u|^2, |u|^2 of
    // the records, gamma and |r|^2 of the A partials) by the block's last
    // warps: eight threads per value, each over every eighth plane, then a
    // shuffle reduction (a fixed order: the same bits in every A task)
    {
      const int nval = 6 * W, R = (8 * nval + 31) & ~31;
      const int t = (int)threadIdx.x - ((int)blockDim.x - R);
      if (t >= 0) {
        const int j = t >> 3, part = t & 7;
        SA acc = acc_of((T)0);
        if (j < 4 * W) {
          for (int q = part; q < P; q += 8) {
            const SA* d = reinterpret_cast<const SA*>(stg + (size_t)q * rb + dbase);
            acc = acc_add(acc, staged ? d[j] : acc_ldcg(d + j));
          }
        } else if (j < nval) {
          const int k = j - 4 * W;          // c * 2 + (0 gamma, 1 |r|^2)
          for (int q = part; q < P; q += 8) acc = acc_add(acc, aps[(size_t)q * W * 2 + k]);
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) acc = acc_add(acc, acc_shfl(acc, o));
        if (part == 0 && j < nval) dsum[j] = acc;
      }
    }
    __syncthreads();
    // coefficients per column c: coef_v = FV_c,v + K_c,v - E_c U_c,v, with
    // FV = Re D (c = 0) or Im D (c = 1) for a packed pair (real: taken real), D otherwise
    for (int j = threadIdx.x; j < W * nocc; j += blockDim.x) {
      const int c = j / nocc, v = j - c * nocc;
      const T Ec = (c < nc) ? pre[c * 4 + 0] : (T)0;
      const V D = Ssum[v], K = Ssum[(1 + c) * nocc + v], U = Ssum[(1 + W + c) * nocc + v];
      V cf;
      if (W == 2) {
        const T fv = (c == 0) ? D.x : D.y;
        cf = mk<T>(fv + K.x - Ec * U.x, (T)0);
      } else {
        cf = mk<T>(D.x + K.x - Ec * U.x, D.y + K.y - Ec * U.y);
      }
      coefT[j] = cf;
      coefT[W * nocc + j] = U;
    }
    __syncthreads();
    // delta correction sum_v Re(conj(U_v) coef_v), one warp per column
    {
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
      if (warp < W) {
        SA t = acc_of((T)0);
        for (int v = lane; v < nocc; v += 32) {
          const V cf = coefT[warp * nocc + v], U = coefT[W * nocc + warp * nocc + v];
          t = acc_add(t, acc_of(U.x * cf.x + U.y * cf.y));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t = acc_add(t, acc_shfl(t, o));
        if (lane == 0) red[warp] = t;
      }
    }
    __syncthreads();
    // decisions (thread c for column c; identical in every A task of the group)
    if (threadIdx.x < W) {
      const int c = threadIdx.x;
      T* cv = colv + c * 8;
      cv[2] = (T)0;
      if (c < nc) {
        const int col = c0 + c;
        const T Ec = pre[c * 4 + 0];
        const SA uY = (W == 2) ? dsum[c * 4 + ((c == 0) ? 0 : 1)] : dsum[c * 4];
        const SA dl = acc_add(acc_add(uY, dsum[c * 4 + 2]),
                             acc_add(acc_scale(dsum[c * 4 + 3], -Ec), acc_scale(red[c], (T)-1)));
        const T delta = acc_val(dl);
        const T gam = acc_val(dsum[4 * W + c * 2]), rr = acc_val(dsum[4 * W + c * 2 + 1]);
        PcgColT<T> st;
        if (it == 1) {
          const bool on = pre[c * 4 + 3] != (T)0;
          const T s1v = a.tol2 * rr, s2v = pre[c * 4 + 2];
          st.gam = (T)0;
          st.alpha = (T)0;
          st.stop = s1v > s2v ? s1v : s2v;
          st.rmin = rr;
          st.rbest = rr;
          st.it = 0;
          st.itb = 0;
          st.active = (on && rr > (T)0) ? 1 : 0;
          st.flag = 0;
        } else {
          st = pcs[c];
        }
        const bool was = st.active != 0;
        if (st.active) {
          const int itc = it - 1;               // updates done so far
          st.rmin = rr < st.rmin ? rr : st.rmin;
          if (rr < (T)0.25 * st.rbest) { st.rbest = rr; st.itb = itc; }
          int stop = 0;
          if (!isfinite(rr)) { st.flag = 2; stop = 1; }
          else if (rr <= st.stop) { st.flag = 0; stop = 1; }
          else if (rr > (T)1e4 * st.rmin) { st.flag = 3; stop = 1; }
          else if (itc >= a.maxit) { st.flag = 1; stop = 1; }
          else if (itc - st.itb > max(kCgStagWindow, 2 * st.itb)) { st.flag = 4; stop = 1; }
          T al = 0, bt = 0;
          if (!stop) {
            T den = delta;
            if (it > 1) {
              bt = gam / st.gam;
              den = delta - bt * gam / st.alpha;
            }
            if (!(den > (T)0) || !isfinite(den) || !(gam > (T)0)) { st.flag = 2; stop = 1; }
            else al = gam / den;
          }
          st.it = itc;
          if (stop) {
            st.active = 0;
          } else {
            st.gam = gam;
            st.alpha = al;
            cv[0] = al;
            cv[1] = bt;
            cv[2] = (T)1;
          }
        }
        cv[3] = Ec;
        cv[4] = pre[c * 4 + 1];
        if (pi == 0) {
          reinterpret_cast<PcgColT<T>*>(a.cst)[(size_t)(it & 1) * a.ncol + col] = st;
          if (!st.active && (was || it == 1)) {
            a.iters_out[col] = st.it;
            a.flag_out[col] = st.flag;
            a.rr_out[col] = (double)rr;
          }
        }
      }
    }
    __syncthreads();
    // group finished: mark it (plane-0 task) and stop here
    {
      int any = 0;
      for (int c = 0; c < W; ++c) any |= (colv[c * 8 + 2] != (T)0);
      if (!any) {
        if (pi == 0 && threadIdx.x == 0) {
          __threadfence();
          atomicExch(gc + 3, (unsigned)(it + 1));
          atomicAdd(&a.ctl[1], 1u);
        }
        signal_done(gc + 0);
        task_time(a.ptask, 0, t0, t1, true);
        return;
      }
    }
  }

  task_mark(a.ptask, 0, 1, &tm);       // sums and decisions
  // ---- update the plane's entries and scatter the packed u = K r
  for (int e = threadIdx.x; e < npp * LDp; e += blockDim.x) Ab[e] = mk<T>(0, 0);
  for (int k = threadIdx.x; k < N; k += blockDim.x) rowmap[k] = -1;
  __syncthreads();
  for (int k = threadIdx.x; k < npp; k += blockDim.x) rowmap[g.pencils[q0 + k].y] = k;
  T gacc[2] = {0, 0}, racc[2] = {0, 0};
  T c_al[2], c_bt[2], c_E[2], c_rtk[2];
  bool c_act[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int cc = (c < W) ? c : 0;
    c_al[c] = colv[cc * 8 + 0];
    c_bt[c] = colv[cc * 8 + 1];
    c_act[c] = (c < nc) && colv[cc * 8 + 2] != (T)0;
    c_E[c] = colv[cc * 8 + 3];
    c_rtk[c] = colv[cc * 8 + 4];
  }
  for (int e = threadIdx.x; e < ns; e += blockDim.x) {
    const int G = s0 + e;
    const T kinG = Ks[e];
    V z = mk<T>(0, 0);
    if (it == 0) {
      // r = b (symmetrised), x = p = s = 0: written by k_pcg_prep
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (c >= nc) break;
        const V rv = pf ? X[(size_t)c * 4 * a.maxplane + e] : a.r[(size_t)(c0 + c) * a.npw + G];
        const T rtk = c_rtk[c];
        const T K = (rtk != (T)0) ? tpa<T>(kinG * rtk) : (T)1;
        const V u = mk<T>(K * rv.x, K * rv.y);
        const T n2 = rv.x * rv.x + rv.y * rv.y;
        racc[c] += n2;
        gacc[c] += K * n2;
        if (W == 2 && c == 1) z = mk<T>(z.x - u.y, z.y + u.x);
        else z = mk<T>(z.x + u.x, z.y + u.y);
      }
    } else {
      // every load of the entry (both columns, the rows of C) before any store
      const V y1 = Ys[e];
      V y2 = mk<T>(0, 0);
      if (W == 2) {
        y2 = Ys[a.maxplane + IXn[e]];
        y2.y = -y2.y;                                 // conj Y(-G)
      }
      V rv[2], pv[2], sv[2], xv[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (c_act[c] && pf) {
          const V* xc = X + (size_t)c * 4 * a.maxplane + e;
          rv[c] = xc[0];
          pv[c] = xc[a.maxplane];
          sv[c] = xc[2 * a.maxplane];
          xv[c] = xc[3 * a.maxplane];
        } else if (c_act[c]) {
          const size_t i = (size_t)(c0 + c) * a.npw + G;
          rv[c] = ldcg(a.r + i);
          pv[c] = ldcg(a.p + i);
          sv[c] = ldcg(a.s + i);
          xv[c] = ldcg(a.x + i);
        } else {
          rv[c] = pv[c] = sv[c] = xv[c] = mk<T>(0, 0);
        }
      }
      V w[2];
      T Kc[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const T rtk = c_rtk[c];
        Kc[c] = (rtk != (T)0) ? tpa<T>(kinG * rtk) : (T)1;
        const V u = mk<T>(Kc[c] * rv[c].x, Kc[c] * rv[c].y);
        V fv;
        if (W == 2) {
          if (c == 0) fv = mk<T>((T)0.5 * (y1.x + y2.x), (T)0.5 * (y1.y + y2.y));
          else fv = mk<T>((T)0.5 * (y1.y - y2.y), (T)-0.5 * (y1.x - y2.x));
        } else {
          fv = y1;
        }
        const T kd = kinG - c_E[c];
        w[c] = mk<T>(fv.x + kd * u.x, fv.y + kd * u.y);
      }
      // w_c -= sum_v C_v(G) coef_c,v: the rows of C read once for both columns
      constexpr int RB = (sizeof(T) == 4) ? 16 : 4;   // rows of C in flight
      for (int v = 0; v < nocc; v += RB) {
        V cv[RB];
#pragma unroll
        for (int q = 0; q < RB; ++q)
          cv[q] = (v + q < nocc) ? (a.crs ? CR[(size_t)(v + q) * a.maxplane + e] : a.C[(size_t)(v + q) * a.npw + G])
                                 : mk<T>(0, 0);
#pragma unroll
        for (int q = 0; q < RB; ++q) {
          if (v + q < nocc) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              if (c < W) {
                const V k = coefT[c * nocc + v + q];
                w[c].x -= cv[q].x * k.x - cv[q].y * k.y;
                w[c].y -= cv[q].x * k.y + cv[q].y * k.x;
              }
            }
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (!c_act[c]) continue;
        const size_t i = (size_t)(c0 + c) * a.npw + G;
        const T al = c_al[c], bt = c_bt[c], K = Kc[c];
        const V u = mk<T>(K * rv[c].x, K * rv[c].y);
        const V pn = mk<T>(u.x + bt * pv[c].x, u.y + bt * pv[c].y);
        const V sn = mk<T>(w[c].x + bt * sv[c].x, w[c].y + bt * sv[c].y);
        const V xn = mk<T>(xv[c].x + al * pn.x, xv[c].y + al * pn.y);
        const V rn = mk<T>(rv[c].x - al * sn.x, rv[c].y - al * sn.y);
        a.p[i] = pn;
        a.s[i] = sn;
        a.x[i] = xn;
        a.r[i] = rn;
        const V un = mk<T>(K * rn.x, K * rn.y);
        const T n2 = rn.x * rn.x + rn.y * rn.y;
        racc[c] += n2;
        gacc[c] += K * n2;
        if (W == 2 && c == 1) z = mk<T>(z.x - un.y, z.y + un.x);
        else z = mk<T>(z.x + un.x, z.y + un.y);
      }
    }
    Ab[IXs[e]] = z;
  }
  {
    SA v4[4] = {acc_of(gacc[0]), acc_of(racc[0]), acc_of(gacc[1]), acc_of(racc[1])};
    block_sum_n<4>(v4, red, dsum + 16);
    if (threadIdx.x < 2 * W) {
      SA* ap = reinterpret_cast<SA*>(a.apart) + (((size_t)(it & 1) * a.ngrp + gi) * P + pi) * W * 2;
      ap[threadIdx.x] = dsum[16 + threadIdx.x];
    }
  }
  __syncthreads();
  task_mark(a.ptask, 0, 2, &tm);       // update and scatter
  // ---- z-IFFT of the disc rows, transpose into the plane, y-IFFT, store
  V* R = fft_tile2<T, +1, false>(Ab, Bb, npp, LDp, 1, a.pl, stw);
  V* Q = (R == Ab) ? Bb : Ab;
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int i1 = a.pl.dN.div(e), i2 = e - i1 * N;
    const int k = rowmap[i1];
    Q[i1 * LDp + i2] = (k >= 0) ? R[k * LDp + i2] : mk<T>(0, 0);
  }
  __syncthreads();
  V* S = fft_tile2<T, +1, true>(Q, R, N, 1, LDp, a.pl, stw);
  task_mark(a.ptask, 0, 3, &tm);       // transforms
  const size_t base = (size_t)gi * g.N3 + (size_t)i0 * g.N2;
  store_rows<T>(a.grid + base, N, S, LDp, N, N, nullptr);
  signal_done(gc + 0);
  task_time(a.ptask, 0, t0, t1, true);
}

// ---------------------------------------------------------------------------
// B task: x-IFFT, * V / N_g, x-FFT on the (group, i1) slab: pencils along i0
// for every i2, element (i0, i2) at tile[i0 * LDp + i2]
// ---------------------------------------------------------------------------
template <typename T>
__device__ void task_B(const PcgArgs<T>& a, int it, int gi, int i1, unsigned char* sm, const PcgLayout& L,
                       int* s_ctl) {
  using V = cpx<T>;
  const Geometry& g = a.g;
  const int N = g.N, LDp = N + 1, P = g.nplanes;
  unsigned* gc = a.ctl + kCtlHead + 4 * gi;
  V* Ab = reinterpret_cast<V*>(sm + L.A);
  V* Bb = reinterpret_cast<V*>(sm + L.B);
  const V* stw = reinterpret_cast<const V*>(sm + L.tw);
  // V(r)/N_g on the slab (static) goes to shared memory before the wait when
  // the prefetch region holds it
  T* Vs = reinterpret_cast<T*>(sm + L.X);
  const bool vpf = L.total - L.X >= (size_t)N * N * sizeof(T);
  if (vpf) {
#pragma unroll 8
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
      const int i0 = a.pl.dN.div(e), i2 = e - i0 * N;
      Vs[e] = a.vloc_s[(size_t)i0 * g.N2 + (size_t)i1 * N + i2];
    }
  }
  unsigned long long t0 = 0, t1 = 0;
  if (threadIdx.x == 0) {
    if (a.ptask) t0 = gtime();
    s_ctl[0] = wait_dep(gc + 0, (unsigned)((it + 1) * P), gc + 3, (unsigned)(it + 1), a.ctl, a.spin_limit);
    if (a.ptask) t1 = gtime();
  }
  __syncthreads();
  if (s_ctl[0] == 1) task_time(a.ptask, 1, t0, t1, false);
  if (s_ctl[0] != 0) return;
  const size_t base = (size_t)gi * g.N3 + (size_t)i1 * N;
  load_rows<T>(Ab, LDp, a.grid + base, g.N2, N, N, g.plane_mask);
  __syncthreads();
  unsigned long long tm = t1;
  task_mark(a.ptask, 1, 0, &tm);       // slab load
  V* R = fft_tile2<T, +1, true>(Ab, Bb, N, 1, LDp, a.pl, stw);
  V* Q = (R == Ab) ? Bb : Ab;
#pragma unroll 4
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int i0 = a.pl.dN.div(e), i2 = e - i0 * N;
    const T m = vpf ? Vs[e] : a.vloc_s[(size_t)i0 * g.N2 + (size_t)i1 * N + i2];
    const V v = R[i0 * LDp + i2];
    R[i0 * LDp + i2] = mk<T>(v.x * m, v.y * m);
  }
  __syncthreads();
  V* S = fft_tile2<T, -1, true>(R, Q, N, 1, LDp, a.pl, stw);
  task_mark(a.ptask, 1, 1, &tm);       // transforms and V
  store_rows<T>(a.grid + base, g.N2, S, LDp, N, N, g.plane_mask);
  signal_done(gc + 1);
  task_mark(a.ptask, 1, 2, &tm);       // store and signal
  task_time(a.ptask, 1, t0, t1, true);
}

// ---------------------------------------------------------------------------
// C task: y-FFT, z-FFT of the disc rows, gather Y, the plane's record
// ---------------------------------------------------------------------------
template <typename T>
__device__ void task_C(const PcgArgs<T>& a, int it, int gi, int pi, unsigned char* sm, const PcgLayout& L,
                       int* s_ctl) {
  using V = cpx<T>;
  const Geometry& g = a.g;
  const int N = g.N, LDp = N + 1, W = a.W, nocc = a.nocc;
  const int c0 = gi * W, nc = min(W, a.ncol - c0);
  unsigned* gc = a.ctl + kCtlHead + 4 * gi;
  V* Ab = reinterpret_cast<V*>(sm + L.A);
  V* Bb = reinterpret_cast<V*>(sm + L.B);
  V* Us = reinterpret_cast<V*>(sm + L.U);          // [W][maxplane] u_c on the plane's entries
  T* Ks = reinterpret_cast<T*>(sm + L.K);          // [maxplane] |G|^2/2 on the plane's entries
  const V* stw = reinterpret_cast<const V*>(sm + L.tw);
  Acc<T>* red = reinterpret_cast<Acc<T>*>(sm + L.red);
  Acc<T>* dsum = reinterpret_cast<Acc<T>*>(sm + L.dsum);
  V* CR = reinterpret_cast<V*>(sm + L.CR);            // [nocc][maxplane]: the plane's rows of C (crs)
  unsigned long long t0 = 0, t1 = 0;
  // First wait: the group's A tasks of it are done (r is final): u = K r and
  // |G|^2/2 on the plane's entries are loaded while the B tasks finish.
  if (threadIdx.x == 0) {
    if (a.ptask) t0 = gtime();
    s_ctl[0] = wait_dep(gc + 0, (unsigned)((it + 1) * g.nplanes), gc + 3, (unsigned)(it + 1), a.ctl,
                        a.spin_limit);
    if (a.ptask) t1 = gtime();
  }
  __syncthreads();
  if (s_ctl[0] == 1) task_time(a.ptask, 2, t0, t1, false);
  if (s_ctl[0] != 0) return;
  const int i0 = g.planes[pi];
  const int s0 = g.plane_sph[pi], s1 = g.plane_sph[pi + 1];
  const int q0 = g.plane_pen[pi], npp = g.plane_pen[pi + 1] - q0;
  const int ns = s1 - s0;
  const size_t base = (size_t)gi * g.N3 + (size_t)i0 * g.N2;
  if (a.crs) stage_rows<T>(CR, a.maxplane, a.C, a.npw, nocc, s0, ns);
  // u_c = K r_c on the plane's entries (0 for an absent column)
  T c_rtk[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) c_rtk[c] = (c < nc) ? a.cin[(c0 + c) * 4 + 1] : (T)0;
  for (int e = threadIdx.x; e < ns; e += blockDim.x) {
    const int G = s0 + e;
    const T kinG = a.kin[G];
    Ks[e] = kinG;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (c >= W) break;
      V u = mk<T>(0, 0);
      if (c < nc) {
        const int col = c0 + c;
        const T rtk = c_rtk[c];
        const T K = (rtk != (T)0) ? tpa<T>(kinG * rtk) : (T)1;
        const V rv = ldcg(a.r + (size_t)col * a.npw + G);
        u = mk<T>(K * rv.x, K * rv.y);
      }
      Us[c * a.maxplane + e] = u;
    }
  }
  // Second wait: the group's B tasks of it are done; the plane.
  if (threadIdx.x == 0) {
    s_ctl[0] = wait_dep(gc + 1, (unsigned)((it + 1) * N), gc + 3, (unsigned)(it + 1), a.ctl, a.spin_limit);
    if (a.ptask) t1 = gtime();
  }
  __syncthreads();
  if (s_ctl[0] == 1) task_time(a.ptask, 2, t0, t1, false);
  if (s_ctl[0] != 0) return;
  load_rows<T>(Ab, LDp, a.grid + base, N, N, N, nullptr);
  __syncthreads();
  unsigned long long tm = t1;
  task_mark(a.ptask, 2, 0, &tm);       // plane and u loads
  V* R = fft_tile2<T, -1, true>(Ab, Bb, N, 1, LDp, a.pl, stw);
  V* Q = (R == Ab) ? Bb : Ab;
  for (int e = threadIdx.x; e < npp * N; e += blockDim.x) {
    const int k = a.pl.dN.div(e), i2 = e - k * N;
    Q[k * LDp + i2] = R[g.pencils[q0 + k].y * LDp + i2];
  }
  __syncthreads();
  V* S = fft_tile2<T, -1, false>(Q, R, npp, LDp, 1, a.pl, stw);
  V* Wv = (S == Q) ? R : Q;                       // free tile: the plane's Y values
  V* Yg = a.Y + (size_t)gi * a.npw;
  for (int e = threadIdx.x; e < ns; e += blockDim.x) {
    const int s = s0 + e;
    const V val = S[(g.sph_pen[s] - q0) * LDp + g.sph_i2[s]];
    Yg[s] = val;
    Wv[e] = val;
  }
  __syncthreads();
  task_mark(a.ptask, 2, 1, &tm);       // transforms and gather
  // ---- the record: projector sums (warp per pair of occupied states, lanes
  // over entries, eight entries in flight), then the FP64 scalar sums
  unsigned char* rec = a.rec + ((size_t)gi * g.nplanes + pi) * a.rec_bytes;
  V* rv = reinterpret_cast<V*>(rec);
  {
    // a warp takes the occupied states v and v + nw together, its lanes UE
    // entries each with all their loads of C in flight before the products
    constexpr int UE = (sizeof(T) == 4) ? 8 : 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const V* U0 = Us;
    const V* U1 = Us + a.maxplane;
    for (int v0 = warp; v0 < nocc; v0 += 2 * nw) {
      const int v1 = v0 + nw;
      const bool two = v1 < nocc;
      const V* C0 = a.crs ? CR + (size_t)v0 * a.maxplane : a.C + (size_t)v0 * a.npw + s0;
      const V* C1 = a.crs ? CR + (size_t)(two ? v1 : v0) * a.maxplane : a.C + (size_t)(two ? v1 : v0) * a.npw + s0;
      T acc[2][10];
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int k = 0; k < 10; ++k) acc[h][k] = (T)0;
      for (int e0 = lane; e0 < ns; e0 += 32 * UE) {
        V cv[2][UE];
#pragma unroll
        for (int u = 0; u < UE; ++u) {
          const int e = e0 + 32 * u;
          cv[0][u] = (e < ns) ? C0[e] : mk<T>(0, 0);
          cv[1][u] = (e < ns && two) ? C1[e] : mk<T>(0, 0);
        }
#pragma unroll
        for (int u = 0; u < UE; ++u) {
          const int e = e0 + 32 * u;
          if (e < ns) {
            const V y = Wv[e];
            const T kk = Ks[e];
            const V u0 = U0[e];
            const V u1 = (W == 2) ? U1[e] : mk<T>(0, 0);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const V c = cv[h][u];
              T* A = acc[h];
              A[0] += c.x * y.x + c.y * y.y;            // conj(C) Y
              A[1] += c.x * y.y - c.y * y.x;
              A[2] += kk * (c.x * u0.x + c.y * u0.y);   // conj(C) kin u_0
              A[3] += kk * (c.x * u0.y - c.y * u0.x);
              A[4] += c.x * u0.x + c.y * u0.y;          // conj(C) u_0
              A[5] += c.x * u0.y - c.y * u0.x;
              if (W == 2) {
                A[6] += kk * (c.x * u1.x + c.y * u1.y);
                A[7] += kk * (c.x * u1.y - c.y * u1.x);
                A[8] += c.x * u1.x + c.y * u1.y;
                A[9] += c.x * u1.y - c.y * u1.x;
              }
            }
          }
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int k = 0; k < 10; ++k)
          for (int o = 16; o > 0; o >>= 1) acc[h][k] += __shfl_xor_sync(0xffffffffu, acc[h][k], o);
      if (lane == 0) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (h == 1 && !two) break;
          const int v = h ? v1 : v0;
          const T* A = acc[h];
          rv[v] = mk<T>(A[0], A[1]);
          rv[(1 + 0) * nocc + v] = mk<T>(A[2], A[3]);
          rv[(1 + W + 0) * nocc + v] = mk<T>(A[4], A[5]);
          if (W == 2) {
            rv[(1 + 1) * nocc + v] = mk<T>(A[6], A[7]);
            rv[(1 + W + 1) * nocc + v] = mk<T>(A[8], A[9]);
          }
        }
      }
    }
  }
  task_mark(a.ptask, 2, 2, &tm);       // projector dots
  {
    T t[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int e = threadIdx.x; e < ns; e += blockDim.x) {
      const V y = Wv[e];
      const T kk = Ks[e];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (c >= W) break;
        const V u = Us[c * a.maxplane + e];
        t[c * 4 + 0] += u.x * y.x + u.y * y.y;        // conj(u) Y
        t[c * 4 + 1] += u.x * y.y - u.y * y.x;
        const T n2 = u.x * u.x + u.y * u.y;
        t[c * 4 + 2] += kk * n2;
        t[c * 4 + 3] += n2;
      }
    }
    Acc<T> v8[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v8[k] = acc_of(t[k]);
    block_sum_n<8>(v8, red, dsum);
    Acc<T>* rd = reinterpret_cast<Acc<T>*>(rec + align16((size_t)(1 + 2 * W) * nocc * sizeof(V)));
    if (threadIdx.x < 4 * W) rd[threadIdx.x] = dsum[threadIdx.x];
  }
  signal_done(gc + 2);
  task_mark(a.ptask, 2, 3, &tm);       // scalar sums, record and signal
  task_time(a.ptask, 2, t0, t1, true);
}

// TPB threads per CTA: 256 (two CTAs per SM) or 512 (one CTA per SM, twice
// the threads on each task: shorter tasks, fewer tasks in flight).
template <typename T, int TPB>
__global__ void __launch_bounds__(TPB, 512 / TPB) k_cg_persistent(PcgArgs<T> a) {
  using V = cpx<T>;
  extern __shared__ unsigned char smem_raw[];
  const Geometry& g = a.g;
  const int N = g.N;
  const PcgLayout L = pcg_layout(N, a.nocc, a.W, a.maxplane, (int)sizeof(V), a.pf != 0, a.crs != 0);
  __shared__ int s_task[4];
  __shared__ int s_ctl[2];
  V* stw = reinterpret_cast<V*>(smem_raw + L.tw);
  for (int k = threadIdx.x; k < N; k += blockDim.x) stw[k] = a.tw[k];
  __syncthreads();
  const int P = g.nplanes;
  const unsigned nA = (unsigned)a.ngrp * P, nB = (unsigned)a.ngrp * N;
  const unsigned per_it = 2u * nA + nB;
  while (true) {
    if (threadIdx.x == 0) {
      int ph = -1;
      if (!*(volatile unsigned*)&a.ctl[2] && *(volatile unsigned*)&a.ctl[1] < (unsigned)a.ngrp) {
        const unsigned t = atomicAdd(&a.ctl[0], 1u);
        const unsigned it = t / per_it;
        unsigned rem = t - it * per_it;
        if (rem < nA) { ph = 0; s_task[2] = rem / P; s_task[3] = rem % P; }
        else if ((rem -= nA) < nB) { ph = 1; s_task[2] = rem / N; s_task[3] = rem % N; }
        else { rem -= nB; ph = 2; s_task[2] = rem / P; s_task[3] = rem % P; }
        s_task[0] = (int)it;
      }
      s_task[1] = ph;
    }
    __syncthreads();
    const int ph = s_task[1], it = s_task[0], gi = s_task[2], k = s_task[3];
    __syncthreads();
    if (ph < 0) break;
    if (ph == 0) task_A<T>(a, it, gi, k, smem_raw, L, s_ctl);
    else if (ph == 1) task_B<T>(a, it, gi, k, smem_raw, L, s_ctl);
    else task_C<T>(a, it, gi, k, smem_raw, L, s_ctl);
    __syncthreads();
  }
}

template <typename T>
static size_t pcg_smem(int N, int nocc, int W, int maxplane, bool pf, bool crs) {
  return pcg_layout(N, nocc, W, maxplane, (int)sizeof(cpx<T>), pf, crs).total;
}

PcgSizes pcg_sizes(int nocc, int npw, int ncol, int W, int nplanes, int N, int csize) {
  const int N3 = N * N * N;
  PcgSizes z;
  z.W = W;
  z.ngrp = (ncol + W - 1) / W;

  z.rec_bytes = pcg_rec_bytes(nocc, W, csize);
  z.rec_total = z.rec_bytes * (size_t)z.ngrp * nplanes;
  z.apart = (size_t)2 * z.ngrp * nplanes * W * 2;
  z.cst = (size_t)2 * ncol;
  z.ctl = (size_t)kCtlHead + 4 * (size_t)z.ngrp;
  z.Y = (size_t)z.ngrp * npw;
  z.grid = (size_t)z.ngrp * N3;
  return z;
}

template <typename T, int TPB>
static cudaError_t launch_pcg_tpb(cudaStream_t s, const PcgArgs<T>& a0, size_t sm, int cta_div, int per_it,
                                  int* grid_used) {
  cudaError_t e = cudaSuccess;
  {
    // The attribute is per function and per process: only ever raise it, so a
    // context on another host thread never sees its limit lowered under it.
    static std::mutex mu;
    static size_t raised = 0;
    std::lock_guard<std::mutex> lock(mu);
    if (sm > raised) {
      e = cudaFuncSetAttribute(k_cg_persistent<T, TPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
      raised = sm;
    }
  }
  int dev = 0, nsm = 0, per = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cg_persistent<T, TPB>, TPB, sm)) != cudaSuccess)
    return e;
  if (per < 1) return cudaErrorNotSupported;
  // cta_div contexts run concurrently (batch mode): each takes an equal share
  // of the resident slots, so all their grids can be co-resident at once.
  const int cap = std::max(1, per * nsm / std::max(cta_div, 1));
  const int nblk = std::min(cap, std::max(per_it, 1));
  *grid_used = nblk;
  PcgArgs<T> a = a0;
  void* args[] = {&a};
  ++g_launches;
  return cudaLaunchCooperativeKernel((const void*)k_cg_persistent<T, TPB>, dim3(nblk), dim3(TPB), args, sm, s);
}

// r = b (two packed columns: b symmetrised, b(G) <- (b(G) + conj b(-G)) / 2),
// x = p = s = 0, and the per-column inputs in T; absent or finished columns
// (outer_active 0) get r = 0.
template <typename T>
__global__ void k_pcg_prep(int npw, int ncol, int W, const double2* __restrict__ b64, const int* outer_active,
                           const double2* E, const double* rr_abs, const double* tk, const int* __restrict__ sph_neg,
                           cpx<T>* x, cpx<T>* r, cpx<T>* p, cpx<T>* sv, T* cin) {
  const size_t n = (size_t)npw * ncol;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int col = (int)(i / (size_t)npw), G = (int)(i - (size_t)col * npw);
    const bool on = !outer_active || outer_active[col];
    double2 b = on ? b64[i] : make_double2(0.0, 0.0);
    if (W == 2 && on) {
      const double2 bn = b64[(size_t)col * npw + sph_neg[G]];
      b = make_double2(0.5 * (b.x + bn.x), 0.5 * (b.y - bn.y));
    }
    r[i] = from_d<T>(b);
    x[i] = mk<T>(0, 0);
    p[i] = mk<T>(0, 0);
    sv[i] = mk<T>(0, 0);
    if (G == 0) {
      cin[col * 4 + 0] = (T)E[col].x;
      cin[col * 4 + 1] = (tk && tk[col] != 0.0) ? (T)(1.0 / tk[col]) : (T)0;
      cin[col * 4 + 2] = rr_abs ? (T)rr_abs[col] : (T)0;
      cin[col * 4 + 3] = on ? (T)1 : (T)0;
    }
  }
}

template <typename T>
cudaError_t launch_cg_persistent(cudaStream_t s, const Geometry& g, const FftPlan& pl, const Prec<T>& P, int nocc,
                                 int npw, int ncol, const PcgSizes& z, int maxplane, const double2* b64,
                                 const int* outer_active, const double2* E, const double* rr_abs, const double* tk,
                                 double tol_in2, int maxit, cpx<T>* x, cpx<T>* r, cpx<T>* p, cpx<T>* sv, cpx<T>* Y,
                                 cpx<T>* grid, unsigned char* rec, double* apart, PcgCol* cst, unsigned* ctl,
                                 T* cin, int* iters, int* flags, double* rr_out, int* grid_used, int cta_div,
                                 unsigned long long spin_limit, unsigned long long* ptask, int tpb) {
  // the A tasks' prefetch of r, p, s, x when it fits beside the rest; with one
  // CTA per SM (512 threads) also the plane's occupied rows, when they fit
  const bool pf = pcg_smem<T>(g.N, nocc, z.W, maxplane, true, false) <= 227 * 1024;
  const bool crs = pf && tpb == 512 && pcg_smem<T>(g.N, nocc, z.W, maxplane, true, true) <= 227 * 1024;
  const size_t sm = pcg_smem<T>(g.N, nocc, z.W, maxplane, pf, crs);
  if (sm > 227 * 1024) return cudaErrorNotSupported;
  {
    const size_t n = (size_t)npw * ncol;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 4096);
    ++g_launches;
    k_pcg_prep<T><<<blocks, 256, 0, s>>>(npw, ncol, z.W, b64, outer_active, E, rr_abs, tk, g.sph_neg, x, r, p, sv,
                                         cin);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  PcgArgs<T> a;
  a.g = g; a.pl = pl; a.tw = P.tw; a.kin = P.kin; a.vloc_s = P.vloc_s; a.C = P.C;
  a.nocc = nocc; a.npw = npw; a.ncol = ncol; a.ngrp = z.ngrp; a.W = z.W; a.maxplane = maxplane;
  a.cin = cin; a.tol2 = (T)tol_in2; a.pf = pf ? 1 : 0; a.crs = crs ? 1 : 0;
  a.maxit = maxit;
  a.x = x; a.r = r; a.p = p; a.s = sv; a.Y = Y; a.grid = grid; a.rec = rec; a.rec_bytes = z.rec_bytes;
  a.apart = reinterpret_cast<unsigned char*>(apart);
  a.cst = reinterpret_cast<unsigned char*>(cst);
  a.ctl = ctl;
  a.iters_out = iters; a.flag_out = flags; a.rr_out = rr_out; a.spin_limit = spin_limit; a.ptask = ptask;
  const int per_it = z.ngrp * (2 * g.nplanes + g.N);
  if (tpb == 512) return launch_pcg_tpb<T, 512>(s, a, sm, cta_div, per_it, grid_used);
  return launch_pcg_tpb<T, 256>(s, a, sm, cta_div, per_it, grid_used);
}

#define GW_PCG_INST(T)                                                                                      \
  template cudaError_t launch_cg_persistent<T>(                                                            \
      cudaStream_t, const Geometry&, const FftPlan&, const Prec<T>&, int, int, int, const PcgSizes&, int,    \
      const double2*, const int*, const double2*, const double*, const double*, double, int, cpx<T>*,       \
      cpx<T>*, cpx<T>*, cpx<T>*, cpx<T>*, cpx<T>*, unsigned char*, double*, PcgCol*, unsigned*, T*, int*,    \
      int*, double*, int*, int, unsigned long long, unsigned long long*, int);
GW_PCG_INST(float)
GW_PCG_INST(double)

}  // namespace gw
