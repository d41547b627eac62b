// Persistent conjugate-gradient solver for the Sternheimer equations
// (Eq. P2: (H - e_v) x = P_c psi_v* dV, projected on the conduction space at
// every step as in Sec. Avoiding summations).
//
// One cooperative launch runs a whole CG pass for every column (occupied
// state x field) with per-column convergence masks.  The work of an iteration
// is cut into tasks that the CTAs draw, in one fixed global order, from an
// atomic ticket counter; a task waits only for the tasks of its own group that
// it depends on (per-group completion counters; every wait is bounded and, when
// the bound runs out, sets an error flag on which every CTA returns).  No
// grid-wide barrier: a group whose columns converge early stops holding the
// others, and the tasks of different groups overlap.
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
//      Depends on every C task of the group at it - 1 (none at it = 0, which
//      sets r = b, x = p = s = 0).
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

constexpr int kCtlHead = 4;     // control words: ticket, groups done, error flag, unused

template <typename T>
struct PcgArgs {
  Geometry g;
  FftPlan pl;
  const cpx<T>* tw;
  const T* kin;
  const T* vloc_s;
  const cpx<T>* C;
  int nocc, npw, ncol, ngrp, W, maxplane;
  const double2* b64;
  const int* outer_active;
  const double2* E;           // per-column shift (real)
  const double* rr_abs;
  const double* tk;           // per-column T_ref of the kinetic preconditioner, or null (none)
  double tol_in2;
  int maxit;
  cpx<T>* x;
  cpx<T>* r;
  cpx<T>* p;
  cpx<T>* s;
  cpx<T>* Y;                  // [ngrp][npw]
  cpx<T>* grid;               // [ngrp][N3]
  unsigned char* rec;         // [ngrp][nplanes] records of the C tasks
  size_t rec_bytes;
  double* apart;              // [2][ngrp][nplanes][W][2] partial gamma, |r|^2 of the A tasks
  PcgCol* cst;                // [2][ncol] column state, by iteration parity
  unsigned* ctl;              // kCtlHead words, then per group: count A, count B, count C, done + 1
  int* iters_out;
  int* flag_out;
  double* rr_out;
  unsigned long long spin_limit;
  unsigned long long* ptask;  // optional [3][8]: per task kind A, B, C: tasks run, busy ns, wait ns, skipped,
                              // then the busy time of up to three sub-phases (ns)
};

template <typename V> __device__ __forceinline__ V ldcg(const V* p);
template <> __device__ __forceinline__ float2 ldcg<float2>(const float2* p) { return __ldcg(p); }
template <> __device__ __forceinline__ double2 ldcg<double2>(const double2* p) { return __ldcg(p); }

// Column state written by another CTA: read through L2.
__device__ __forceinline__ PcgCol ld_col(const PcgCol* p) {
  PcgCol c;
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

// Sums over the block of NV values per thread, in FP64 (the NV sums land in
// out[0 .. NV), visible to every thread after the call); up to 16 warps.
template <int NV>
__device__ __forceinline__ void block_sum_n(double (&v)[NV], double* sh, double* out) {
#pragma unroll
  for (int k = 0; k < NV; ++k)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k * 16 + w] = v[k];
  __syncthreads();
  if (threadIdx.x < NV) {
    double t = 0.0;
    for (int q = 0; q < nw; ++q) t += sh[threadIdx.x * 16 + q];
    out[threadIdx.x] = t;
  }
  __syncthreads();
}

struct PcgLayout {
  size_t A, B, U, K, tw, rowmap, red, S, coef, dsum, ap, col, pre, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Shared memory of one CTA: two FFT tiles N x (N+1), the plane's u_c and
// |G|^2/2 (C tasks), twiddles, the row map of a plane's disc pencils,
// reduction scratch, the summed records, the group's projector coefficients
// and <C_v|u_c> (A tasks), FP64 sums, the staged per-plane partials of the A
// tasks, and per-column scalars.
__host__ __device__ inline PcgLayout pcg_layout(int N, int nocc, int W, int maxplane, int vsize) {
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
  L.total = align16(L.pre + 2 * (4 * sizeof(double) + sizeof(PcgCol)));
  return L;
}

// Record of one (group, plane) C task:
//   V [nocc]        D_v   = sum conj(C_v) Y
//   V [W][nocc]     K_c,v = sum conj(C_v) kin u_c
//   V [W][nocc]     U_c,v = sum conj(C_v) u_c
//   double [W][4]   Re, Im of u_c^H Y, sum kin |u_c|^2, sum |u_c|^2
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
    const unsigned d = *(volatile const unsigned*)done1;
    if (d != 0u && d <= skip_le) return 1;
    if (*(volatile const unsigned*)cnt >= target) break;
    if (*(volatile unsigned*)&ctl[2]) return 2;
    if (++spins > limit) { atomicExch(&ctl[2], 1u); return 2; }
    __nanosleep(32);
  }
  __threadfence();
  const unsigned d = *(volatile const unsigned*)done1;
  return (d != 0u && d <= skip_le) ? 1 : 0;
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
  unsigned long long* q = pt + 8 * kind;
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
  atomicAdd(pt + 8 * kind + 4 + k, now - *t);
  *t = now;
}

// Completion of a task: every thread's writes fenced, then one count.
__device__ __forceinline__ void signal_done(unsigned* cnt) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(cnt, 1u);
}

// ---------------------------------------------------------------------------
// A task
// ---------------------------------------------------------------------------
template <typename T>
__device__ void task_A(const PcgArgs<T>& a, int it, int gi, int pi, unsigned char* sm, const PcgLayout& L,
                       int* s_ctl) {
  using V = cpx<T>;
  const Geometry& g = a.g;
  const int N = g.N, LDp = N + 1, P = g.nplanes, W = a.W, nocc = a.nocc;
  const int c0 = gi * W, nc = min(W, a.ncol - c0);
  unsigned* gc = a.ctl + kCtlHead + 4 * gi;
  V* Ab = reinterpret_cast<V*>(sm + L.A);
  V* Bb = reinterpret_cast<V*>(sm + L.B);
  const V* stw = reinterpret_cast<const V*>(sm + L.tw);
  int* rowmap = reinterpret_cast<int*>(sm + L.rowmap);
  double* red = reinterpret_cast<double*>(sm + L.red);
  V* Ssum = reinterpret_cast<V*>(sm + L.S);            // the records' projector sums over planes
  V* coefT = reinterpret_cast<V*>(sm + L.coef);        // [W][nocc] coefficients, then [W][nocc] <C_v|u_c>
  double* dsum = reinterpret_cast<double*>(sm + L.dsum);
  double* colv = reinterpret_cast<double*>(sm + L.col);   // [c * 8 + k]: alpha, beta, active, E, rtk
  unsigned long long t0 = 0, t1 = 0;
  if (threadIdx.x == 0) {
    int w = 0;
    if (a.ptask) t0 = gtime();
    if (it > 0) w = wait_dep(gc + 2, (unsigned)(it * P), gc + 3, (unsigned)it, a.ctl, a.spin_limit);
    if (a.ptask) t1 = gtime();
    s_ctl[0] = w;
  }
  __syncthreads();
  if (s_ctl[0] == 2) return;
  if (s_ctl[0] == 1) {                 // the group finished earlier: nothing left to do
    task_time(a.ptask, 0, t0, t1, false);
    return;
  }
  const int i0 = g.planes[pi];
  const int s0 = g.plane_sph[pi], s1 = g.plane_sph[pi + 1];
  const int q0 = g.plane_pen[pi], npp = g.plane_pen[pi + 1] - q0;
  const int ns = s1 - s0;
  const size_t rb = a.rec_bytes;
  const int nv = (1 + 2 * W) * nocc;

  // ---- column scalars
  if (it == 0) {
    for (int c = threadIdx.x; c < W; c += blockDim.x) {
      const bool present = c < nc;
      colv[c * 8 + 0] = 0.0;
      colv[c * 8 + 1] = 0.0;
      colv[c * 8 + 2] = present ? 1.0 : 0.0;
      colv[c * 8 + 3] = present ? a.E[c0 + c].x : 0.0;
      colv[c * 8 + 4] = (present && a.tk) ? 1.0 / a.tk[c0 + c] : 0.0;
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
      for (size_t e = threadIdx.x; e < nb16; e += blockDim.x) d4[e] = __ldcg(s4 + e);
    }
    const double* ap = a.apart + ((size_t)((it - 1) & 1) * a.ngrp + gi) * P * W * 2;
    double* aps = reinterpret_cast<double*>(sm + L.ap);
    for (int j = threadIdx.x; j < P * W * 2; j += blockDim.x) aps[j] = __ldcg(ap + j);
    double* pre = reinterpret_cast<double*>(sm + L.pre);                  // [W][4]: E, T_ref, on, |r|^2 target
    PcgCol* pcs = reinterpret_cast<PcgCol*>(sm + L.pre + 2 * 4 * sizeof(double));
    if (threadIdx.x < nc) {
      const int col = c0 + threadIdx.x;
      pre[threadIdx.x * 4 + 0] = a.E[col].x;
      pre[threadIdx.x * 4 + 1] = a.tk ? a.tk[col] : 0.0;
      pre[threadIdx.x * 4 + 2] = (!a.outer_active || a.outer_active[col]) ? 1.0 : 0.0;
      pre[threadIdx.x * 4 + 3] = a.rr_abs ? a.rr_abs[col] : 0.0;
      if (it > 1) pcs[threadIdx.x] = ld_col(a.cst + (size_t)((it - 1) & 1) * a.ncol + col);
    }
    __syncthreads();
    // projector sums in T (threads j < nv) and the FP64 sums (the next 6 W
    // threads: per column Re/Im u^H Y, kin|u|^2, |u|^2 of the records, gamma
    // and |r|^2 of the A partials), each over the planes in order
    const size_t dbase = align16((size_t)nv * sizeof(V));
    for (int j = threadIdx.x; j < nv + 6 * W; j += blockDim.x) {
      if (j < nv) {
        T sx = 0, sy = 0;
        for (int q = 0; q < P; ++q) {
          const V v = staged ? reinterpret_cast<const V*>(stg + (size_t)q * rb)[j]
                             : ldcg(reinterpret_cast<const V*>(stg + (size_t)q * rb) + j);
          sx += v.x;
          sy += v.y;
        }
        Ssum[j] = mk<T>(sx, sy);
      } else {
        const int jj = j - nv;
        double t = 0.0;
        if (jj < 4 * W) {
          for (int q = 0; q < P; ++q) {
            const double* d = reinterpret_cast<const double*>(stg + (size_t)q * rb + dbase);
            t += staged ? d[jj] : __ldcg(d + jj);
          }
        } else {
          const int k = jj - 4 * W;        // c * 2 + (0 gamma, 1 |r|^2)
          for (int q = 0; q < P; ++q) t += aps[(size_t)q * W * 2 + k];
        }
        dsum[jj] = t;
      }
    }
    __syncthreads();
    // coefficients per column c: coef_v = FV_c,v + K_c,v - E_c U_c,v, with
    // FV = Re D (c = 0) or Im D (c = 1) for a packed pair (real: taken real), D otherwise
    for (int j = threadIdx.x; j < W * nocc; j += blockDim.x) {
      const int c = j / nocc, v = j - c * nocc;
      const T Ec = (T)((c < nc) ? pre[c * 4 + 0] : 0.0);
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
        double t = 0.0;
        for (int v = lane; v < nocc; v += 32) {
          const V cf = coefT[warp * nocc + v], U = coefT[W * nocc + warp * nocc + v];
          t += (double)(U.x * cf.x + U.y * cf.y);
        }
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) red[warp] = t;
      }
    }
    __syncthreads();
    // decisions (thread c for column c; identical in every A task of the group)
    if (threadIdx.x < W) {
      const int c = threadIdx.x;
      double* cv = colv + c * 8;
      cv[2] = 0.0;
      if (c < nc) {
        const int col = c0 + c;
        const double Ec = pre[c * 4 + 0];
        const double uY = (W == 2) ? dsum[c * 4 + ((c == 0) ? 0 : 1)] : dsum[c * 4];
        const double delta = uY + dsum[c * 4 + 2] - Ec * dsum[c * 4 + 3] - red[c];
        const double gam = dsum[4 * W + c * 2], rr = dsum[4 * W + c * 2 + 1];
        PcgCol st;
        if (it == 1) {
          const bool on = pre[c * 4 + 2] != 0.0;
          st.gam = 0.0;
          st.alpha = 0.0;
          st.stop = fmax(a.tol_in2 * rr, pre[c * 4 + 3]);
          st.rmin = rr;
          st.rbest = rr;
          st.it = 0;
          st.itb = 0;
          st.active = (on && rr > 0.0) ? 1 : 0;
          st.flag = 0;
          if (!st.active) st.flag = 0;
        } else {
          st = pcs[c];
        }
        const bool was = st.active != 0;
        if (st.active) {
          const int itc = it - 1;               // updates done so far
          st.rmin = fmin(st.rmin, rr);
          if (rr < 0.25 * st.rbest) { st.rbest = rr; st.itb = itc; }
          int stop = 0;
          if (!isfinite(rr)) { st.flag = 2; stop = 1; }
          else if (rr <= st.stop) { st.flag = 0; stop = 1; }
          else if (rr > 1e4 * st.rmin) { st.flag = 3; stop = 1; }
          else if (itc >= a.maxit) { st.flag = 1; stop = 1; }
          else if (itc - st.itb > max(kCgStagWindow, 2 * st.itb)) { st.flag = 4; stop = 1; }
          double al = 0.0, bt = 0.0;
          if (!stop) {
            double den = delta;
            if (it > 1) {
              bt = gam / st.gam;
              den = delta - bt * gam / st.alpha;
            }
            if (!(den > 0.0) || !isfinite(den) || !(gam > 0.0)) { st.flag = 2; stop = 1; }
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
            cv[2] = 1.0;
          }
        }
        cv[3] = Ec;
        cv[4] = pre[c * 4 + 1] != 0.0 ? 1.0 / pre[c * 4 + 1] : 0.0;
        if (pi == 0) {
          a.cst[(size_t)(it & 1) * a.ncol + col] = st;
          if (!st.active && (was || it == 1)) {
            a.iters_out[col] = st.it;
            a.flag_out[col] = st.flag;
            a.rr_out[col] = rr;
          }
        }
      }
    }
    __syncthreads();
    // group finished: mark it (plane-0 task) and stop here
    {
      int any = 0;
      for (int c = 0; c < W; ++c) any |= (colv[c * 8 + 2] != 0.0);
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

  unsigned long long tm = t1;
  task_mark(a.ptask, 0, 0, &tm);       // sums and decisions
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
    c_al[c] = (T)colv[cc * 8 + 0];
    c_bt[c] = (T)colv[cc * 8 + 1];
    c_act[c] = (c < W) && colv[cc * 8 + 2] != 0.0;
    c_E[c] = (T)colv[cc * 8 + 3];
    c_rtk[c] = (T)colv[cc * 8 + 4];
  }
  const V* Yg = a.Y + (size_t)gi * a.npw;
  for (int e = threadIdx.x; e < ns; e += blockDim.x) {
    const int G = s0 + e;
    const T kinG = a.kin[G];
    V z = mk<T>(0, 0);
    if (it == 0) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (c >= nc) break;
        const int col = c0 + c;
        const size_t i = (size_t)col * a.npw + G;
        const bool on = !a.outer_active || a.outer_active[col];
        double2 b = on ? a.b64[i] : make_double2(0.0, 0.0);
        if (W == 2 && on) {
          const double2 bn = a.b64[(size_t)col * a.npw + g.sph_neg[G]];
          b = make_double2(0.5 * (b.x + bn.x), 0.5 * (b.y - bn.y));
        }
        const V rv = from_d<T>(b);
        a.r[i] = rv;
        a.x[i] = mk<T>(0, 0);
        a.p[i] = mk<T>(0, 0);
        a.s[i] = mk<T>(0, 0);
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
      const V y1 = ldcg(Yg + G);
      V y2 = ldcg(Yg + g.sph_neg[G]);
      y2.y = -y2.y;                                   // conj Y(-G)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (c >= nc || !c_act[c]) continue;
        const int col = c0 + c;
        const size_t i = (size_t)col * a.npw + G;
        const T al = c_al[c], bt = c_bt[c], Ec = c_E[c];
        const T rtk = c_rtk[c];
        const T K = (rtk != (T)0) ? tpa<T>(kinG * rtk) : (T)1;
        V rv = ldcg(a.r + i), pv = ldcg(a.p + i), sv = ldcg(a.s + i), xv = ldcg(a.x + i);
        const V u = mk<T>(K * rv.x, K * rv.y);
        V fv;
        if (W == 2) {
          if (c == 0) fv = mk<T>((T)0.5 * (y1.x + y2.x), (T)0.5 * (y1.y + y2.y));
          else fv = mk<T>((T)0.5 * (y1.y - y2.y), (T)-0.5 * (y1.x - y2.x));
        } else {
          fv = y1;
        }
        const T kd = kinG - Ec;
        V w = mk<T>(fv.x + kd * u.x, fv.y + kd * u.y);
        const V* cf = coefT + c * nocc;
        constexpr int RB = (sizeof(T) == 4) ? 16 : 8;   // rows of C in flight
        for (int v = 0; v < nocc; v += RB) {
          V cv[RB];
#pragma unroll
          for (int q = 0; q < RB; ++q) cv[q] = (v + q < nocc) ? a.C[(size_t)(v + q) * a.npw + G] : mk<T>(0, 0);
#pragma unroll
          for (int q = 0; q < RB; ++q) {
            if (v + q < nocc) {
              const V k = cf[v + q];
              w.x -= cv[q].x * k.x - cv[q].y * k.y;
              w.y -= cv[q].x * k.y + cv[q].y * k.x;
            }
          }
        }
        pv = mk<T>(u.x + bt * pv.x, u.y + bt * pv.y);
        sv = mk<T>(w.x + bt * sv.x, w.y + bt * sv.y);
        xv = mk<T>(xv.x + al * pv.x, xv.y + al * pv.y);
        rv = mk<T>(rv.x - al * sv.x, rv.y - al * sv.y);
        a.p[i] = pv;
        a.s[i] = sv;
        a.x[i] = xv;
        a.r[i] = rv;
        const V un = mk<T>(K * rv.x, K * rv.y);
        const T n2 = rv.x * rv.x + rv.y * rv.y;
        racc[c] += n2;
        gacc[c] += K * n2;
        if (W == 2 && c == 1) z = mk<T>(z.x - un.y, z.y + un.x);
        else z = mk<T>(z.x + un.x, z.y + un.y);
      }
    }
    Ab[(g.sph_pen[G] - q0) * LDp + g.sph_i2[G]] = z;
  }
  {
    double v4[4] = {(double)gacc[0], (double)racc[0], (double)gacc[1], (double)racc[1]};
    block_sum_n<4>(v4, red, dsum + 16);
    if (threadIdx.x < 2 * W) {
      double* ap = a.apart + (((size_t)(it & 1) * a.ngrp + gi) * P + pi) * W * 2;
      ap[threadIdx.x] = dsum[16 + threadIdx.x];
    }
  }
  __syncthreads();
  task_mark(a.ptask, 0, 1, &tm);       // update and scatter
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
  task_mark(a.ptask, 0, 2, &tm);       // transforms
  const size_t base = (size_t)gi * g.N3 + (size_t)i0 * g.N2;
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int i1 = a.pl.dN.div(e), i2 = e - i1 * N;
    a.grid[base + e] = S[i1 * LDp + i2];
  }
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
#pragma unroll 8
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int i0 = a.pl.dN.div(e), i2 = e - i0 * N;
    Ab[i0 * LDp + i2] = g.plane_mask[i0] ? ldcg(a.grid + base + (size_t)i0 * g.N2 + i2) : mk<T>(0, 0);
  }
  __syncthreads();
  unsigned long long tm = t1;
  task_mark(a.ptask, 1, 0, &tm);       // slab load
  V* R = fft_tile2<T, +1, true>(Ab, Bb, N, 1, LDp, a.pl, stw);
  V* Q = (R == Ab) ? Bb : Ab;
#pragma unroll 4
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int i0 = a.pl.dN.div(e), i2 = e - i0 * N;
    const T m = a.vloc_s[(size_t)i0 * g.N2 + (size_t)i1 * N + i2];
    const V v = R[i0 * LDp + i2];
    R[i0 * LDp + i2] = mk<T>(v.x * m, v.y * m);
  }
  __syncthreads();
  V* S = fft_tile2<T, -1, true>(R, Q, N, 1, LDp, a.pl, stw);
  task_mark(a.ptask, 1, 1, &tm);       // transforms and V
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int i0 = a.pl.dN.div(e), i2 = e - i0 * N;
    if (g.plane_mask[i0]) a.grid[base + (size_t)i0 * g.N2 + i2] = S[i0 * LDp + i2];
  }
  signal_done(gc + 1);
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
  double* red = reinterpret_cast<double*>(sm + L.red);
  double* dsum = reinterpret_cast<double*>(sm + L.dsum);
  unsigned long long t0 = 0, t1 = 0;
  if (threadIdx.x == 0) {
    if (a.ptask) t0 = gtime();
    s_ctl[0] = wait_dep(gc + 1, (unsigned)((it + 1) * N), gc + 3, (unsigned)(it + 1), a.ctl, a.spin_limit);
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
#pragma unroll 8
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int i1 = a.pl.dN.div(e), i2 = e - i1 * N;
    Ab[i1 * LDp + i2] = ldcg(a.grid + base + e);
  }
  // u_c = K r_c on the plane's entries (0 for an absent column)
  T c_rtk[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) c_rtk[c] = (a.tk && c < nc) ? (T)(1.0 / a.tk[c0 + c]) : (T)0;
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
      const V* C0 = a.C + (size_t)v0 * a.npw + s0;
      const V* C1 = a.C + (size_t)(two ? v1 : v0) * a.npw + s0;
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
    double v8[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v8[k] = (double)t[k];
    block_sum_n<8>(v8, red, dsum);
    double* rd = reinterpret_cast<double*>(rec + align16((size_t)(1 + 2 * W) * nocc * sizeof(V)));
    if (threadIdx.x < 4 * W) rd[threadIdx.x] = dsum[threadIdx.x];
  }
  signal_done(gc + 2);
  task_time(a.ptask, 2, t0, t1, true);
}

// TPB threads per CTA: 256 (two CTAs per SM) or 512 (one CTA per SM, twice
// the threads on each task: shorter tasks, fewer tasks in flight).
template <typename T, int TPB>
__global__ void __launch_bounds__(TPB, 512 / TPB) k_cg_persistent(PcgArgs<T> a) {
  using V = cpx<T>;
  extern __shared__ unsigned char smem_raw[];
  const Geometry& g = a.g;
  const int N = g.N, P = g.nplanes;
  const PcgLayout L = pcg_layout(N, a.nocc, a.W, a.maxplane, (int)sizeof(V));
  __shared__ int s_task[4];
  __shared__ int s_ctl[2];
  V* stw = reinterpret_cast<V*>(smem_raw + L.tw);
  for (int k = threadIdx.x; k < N; k += blockDim.x) stw[k] = a.tw[k];
  __syncthreads();
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
static size_t pcg_smem(int N, int nocc, int W, int maxplane) {
  return pcg_layout(N, nocc, W, maxplane, (int)sizeof(cpx<T>)).total;
}

PcgSizes pcg_sizes(int nocc, int npw, int ncol, int W, int nplanes, int N3, int csize) {
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

template <typename T>
cudaError_t launch_cg_persistent(cudaStream_t s, const Geometry& g, const FftPlan& pl, const Prec<T>& P, int nocc,
                                 int npw, int ncol, const PcgSizes& z, int maxplane, const double2* b64,
                                 const int* outer_active, const double2* E, const double* rr_abs, const double* tk,
                                 double tol_in2, int maxit, cpx<T>* x, cpx<T>* r, cpx<T>* p, cpx<T>* sv, cpx<T>* Y,
                                 cpx<T>* grid, unsigned char* rec, double* apart, PcgCol* cst, unsigned* ctl,
                                 int* iters, int* flags, double* rr_out, int* grid_used, int cta_div,
                                 unsigned long long spin_limit, unsigned long long* ptask, int tpb) {
  PcgArgs<T> a;
  a.g = g; a.pl = pl; a.tw = P.tw; a.kin = P.kin; a.vloc_s = P.vloc_s; a.C = P.C;
  a.nocc = nocc; a.npw = npw; a.ncol = ncol; a.ngrp = z.ngrp; a.W = z.W; a.maxplane = maxplane;
  a.b64 = b64; a.outer_active = outer_active; a.E = E; a.rr_abs = rr_abs; a.tk = tk; a.tol_in2 = tol_in2;
  a.maxit = maxit;
  a.x = x; a.r = r; a.p = p; a.s = sv; a.Y = Y; a.grid = grid; a.rec = rec; a.rec_bytes = z.rec_bytes;
  a.apart = apart; a.cst = cst; a.ctl = ctl;
  a.iters_out = iters; a.flag_out = flags; a.rr_out = rr_out; a.spin_limit = spin_limit; a.ptask = ptask;
  const size_t sm = pcg_smem<T>(g.N, nocc, z.W, maxplane);
  if (sm > 227 * 1024) return cudaErrorNotSupported;
  const int per_it = z.ngrp * (2 * g.nplanes + g.N);
  if (tpb == 512) return launch_pcg_tpb<T, 512>(s, a, sm, cta_div, per_it, grid_used);
  return launch_pcg_tpb<T, 256>(s, a, sm, cta_div, per_it, grid_used);
}

#define GW_PCG_INST(T)                                                                                      \
  template cudaError_t launch_cg_persistent<T>(                                                            \
      cudaStream_t, const Geometry&, const FftPlan&, const Prec<T>&, int, int, int, const PcgSizes&, int,    \
      const double2*, const int*, const double2*, const double*, const double*, double, int, cpx<T>*,       \
      cpx<T>*, cpx<T>*, cpx<T>*, cpx<T>*, cpx<T>*, unsigned char*, double*, PcgCol*, unsigned*, int*, int*,  \
      double*, int*, int, unsigned long long, unsigned long long*, int);
GW_PCG_INST(float)
GW_PCG_INST(double)

}  // namespace gw
