// Launch interfaces of the solver / Lanczos kernels (kernels_linalg.cu).
#pragma once

#include <vector>

#include "gw_common.cuh"

namespace gw {

constexpr int kMaxOcc = 256;   // occupied states supported by the projector kernels

// Scratch for deterministic reductions, owned by the context.
struct Work {
  double* part1 = nullptr;    // partial sums (double)
  double2* part2 = nullptr;   // partial sums (double2)
  double2* coef = nullptr;    // projector coefficients [nocc][ncol]
  unsigned* cnt_a = nullptr;  // tickets (zero between launches)
  unsigned* cnt_b = nullptr;
  unsigned* cnt_c = nullptr;
  unsigned* cnt_d = nullptr;  // tickets of the dots fused into the gather pass
  double2* part_d = nullptr;  // their partial sums
};

// Per-column state of a batched CG solve (device arrays).
struct CgState {
  double* rr = nullptr;     // current |r|^2
  double* rr0 = nullptr;    // |b|^2
  double* beta = nullptr;   // next p = r + beta p (beta < 0: p = r)
  int* iters = nullptr;
  int* flag = nullptr;      // 0 converged, 1 max iterations, 2 breakdown, 3 diverging (round-off floor),
                            // 4 stagnated (no 4x drop of |r|^2 in max(kCgStagWindow, 2 k_best) iterations)
  int* active = nullptr;
  double* rr_stop = nullptr;  // stop when |r|^2 <= rr_stop
  double* rr_min = nullptr;   // smallest |r|^2 seen (divergence guard)
  double* rr_best = nullptr;  // |r|^2 at the last 4x improvement (stagnation guard)
  int* it_best = nullptr;     // iteration of that improvement
  const double* rr_abs = nullptr;   // per-column absolute |r|^2 target of the refinement
  double* rz = nullptr;     // current r^H K r (K = kinetic preconditioner; = rr without one)
  const double* tk = nullptr;       // per-column T_ref of the preconditioner, or null (none)
  int* n_done = nullptr;    // columns that stopped (atomic)
  unsigned* cnt = nullptr;  // tickets [ncol]
  int ppow = 1;             // preconditioner K (1) or K^2 (2: squared operator)
};

// Per-column state of a batched simplified-QMR solve (device arrays).
struct QmrState {
  double2* rho = nullptr;    // [r, r]
  double2* alpha = nullptr;
  double2* beta = nullptr;
  double2* qcoef = nullptr;  // c^2 alpha
  double* dcoef = nullptr;   // c^2 theta_old^2
  double* theta = nullptr;
  double* tau = nullptr;
  double* rr_stop = nullptr;
  const double* rr_abs = nullptr;
  const double* tk = nullptr;   // per-column T_ref of the preconditioner, or null (none)
  double* qbest = nullptr;   // smallest tau^2 so far (to within a factor 4)
  int* itbest = nullptr;     // iteration at which qbest was last lowered
  int* iters = nullptr;
  int* flag = nullptr;       // 0 converged, 1 max iterations, 2 breakdown, 4 stagnated
  int* active = nullptr;
  int* n_done = nullptr;
  unsigned* cnt = nullptr;
};

template <typename T>
void launch_proj(cudaStream_t s, const cpx<T>* C, int nocc, int npw, cpx<T>* Y, int ncol, const int* active,
                 Work& w, const cpx<T>* Pv, double* pap, bool real = false);
// step 0 init, 1 sigma/alpha, 2 residual, 3 d/x/rho/beta + stop test, 4 q update
template <typename T>
void launch_qmr(cudaStream_t s, int step, int npw, int ncol, const double2* b, cpx<T>* x, cpx<T>* r, cpx<T>* q,
                cpx<T>* d, const cpx<T>* t, const int* neg, const int* outer_active, Work& w, QmrState st,
                const T* kin, double tol_in2, int maxit);
template <typename T>
void launch_proj_update(cudaStream_t s, const cpx<T>* C, int nocc, int npw, cpx<T>* Y, int ncol,
                        const int* active, const double2* coef, Work& w, const cpx<T>* Pv, double* pap, bool real = false);
// Ap += w2[c] p per column; pap[c] = Re <p|Ap> when pap is given
template <typename T>
void launch_sq_shift(cudaStream_t s, int npw, int ncol, cpx<T>* Ap, const cpx<T>* p, const double* w2,
                     const int* active, Work& w, double* pap);
template <typename T>
void launch_gram(cudaStream_t s, const cpx<T>* C, int nocc, int npw, const cpx<T>* Y, int ncol, Work& w,
                 double2* out, bool real = false);
void launch_wmat(cudaStream_t s, const double2* U, const double* w, int n, int nocc, Work& wk, double2* W);
void launch_g1(cudaStream_t s, const double2* dU, const double2* U, const double2* S, int n, int nocc,
               double inv_vol, double* g1);
void launch_grad_combine(cudaStream_t s, int n, const double* g1, const double* g2, double wgt, double* grad);
template <typename T, typename U>
void launch_cg_init(cudaStream_t s, int npw, int ncol, const cpx<U>* b, cpx<T>* x, cpx<T>* r,
                    const int* outer_active, Work& w, CgState st, const T* kin, double tol_in2, double tol_abs2);
template <typename T>
void launch_cg_update(cudaStream_t s, int npw, int ncol, cpx<T>* x, cpx<T>* r, const cpx<T>* p,
                      const cpx<T>* Ap, const double* pap, Work& w, CgState st, const T* kin, double tol2,
                      int maxit);
template <typename T>
void launch_add_conv(cudaStream_t s, int npw, int ncol, const cpx<T>* d, double2* x, const int* active);
template <typename T>
void launch_add_conv_sym(cudaStream_t s, int npw, int ncol, const cpx<T>* d, double2* x, const int* active,
                         const int* neg);
// Packed pairs of real-in-real-space columns (see kernels_linalg.cu):
// out[j] = x[ia[j]] + i x[ib[j]]; and the inverse split of a transform of such
// a pair, optionally adding (kin - E_c) x_c.
void launch_pack_pairs(cudaStream_t s, int npw, int npair, const double2* x, const int* ia, const int* ib,
                       const int* active, double2* out);
void launch_unpack_pairs(cudaStream_t s, int npw, int npair, const double2* Y, const int* neg, const int* ia,
                         const int* ib, const int* active, const double* kin, const double2* E, const double2* x,
                         double2* out);
// out[c] = max |b(G) - conj b(-G)|, out[ncol + c] = max |b(G)| per column
void launch_sym_check(cudaStream_t s, int npw, int ncol, const double2* b, const int* neg, double* out);
void launch_defl_scale(cudaStream_t s, double2* coef, const double* eps, const double2* E, int ndef, int ncol,
                       const int* active);
void launch_residual(cudaStream_t s, int npw, int ncol, const double2* b, double2* ax, const double2* x,
                     const int* active, Work& w, double* res2, double* bb, double* xx, const double2* C = nullptr,
                     int nocc = 0, const double2* cb = nullptr, const double2* cax = nullptr, bool real = false);
void launch_combine(cudaStream_t s, int npw, int nout, const double2* in, const int* src0, const int* src1,
                    double w_pair, double w_single, double2* out);
// Eq. model_eq: out[j] = (pinv(T - Em_j) + pinv(T - Ep_j)) in[src_j] on the sphere
template <typename T>
void launch_model_scale(cudaStream_t s, int npw, int nout, const T* kin, const cpx<T>* in, const int* src,
                        const double2* Em, const double2* Ep, cpx<T>* out);
// Eq. subs_epsilon: out[m][m] from the coefficients a [m][k], am [m][km] and the
// inverses Ti (exact basis), Mi (model in the exact basis, complex), Tmi (model basis)
void launch_split_form(cudaStream_t s, int m, int k, int km, const double* a, const double* Ti,
                       const double2* Mi, const double* am, const double* Tmi, double* out);
void launch_to_cplx(cudaStream_t s, size_t n, const double* x, double2* y);
template <typename T, typename U>
void launch_gather_rows(cudaStream_t s, int npw, int nout, const cpx<U>* in, const int* idx, cpx<T>* out);
void launch_gemv_t(cudaStream_t s, const double* Q, size_t ld, int n, const double* w, double wgt, int k,
                   Work& wk, double* out);
void launch_gemv_n(cudaStream_t s, const double* Q, size_t ld, int n, const double* h, int k, double* w);
void launch_lz_axpy(cudaStream_t s, int n, int op, const double* sc, double* w, const double* q, double* qn);
void launch_dot(cudaStream_t s, int n, const double* x, const double* y, double wgt, int want_sqrt, Work& w,
                double* out);
void launch_tridiag_inv(cudaStream_t s, int K, const double* alpha, const double* beta, double* d, double* l,
                        double* out, int* status);

template <typename T> cudaError_t fft_set_smem_limits();

// small dense FP64 algebra of the recycled bases (kernels_small.cu)
void launch_normalize_rows(cudaStream_t s, double2* rows, int nrows, size_t n);
void launch_real_part(cudaStream_t s, size_t n, const double2* src, double* dst);
void launch_symmetrize(cudaStream_t s, int nb, int m, double* A);
cudaError_t launch_jacobi_sym(cudaStream_t s, int nb, int m, double* A, double* V, double tol, int max_sweeps,
                              int* sweeps);
void launch_gemm_small(cudaStream_t s, int nb, int r, int k, int c, const double* A, int ta, const double* B, int tb,
                       double* C);
void launch_orth_transform(cudaStream_t s, int nb, int m, const double* S, const double* W, double rel, double* T,
                           int* kept);
void launch_recycled_form(cudaStream_t s, int nbat, int m, int nl, int nw, const double* L, const double* c,
                          const double* w, double* out);
void launch_eig_function(cudaStream_t s, int nb, int m, const double* L, const double* V, int mode, double* out);
void launch_add_identity(cudaStream_t s, int nb, int m, double* A);
void launch_shift_quadrature(cudaStream_t s, int m, int b, const double* L, const double* U, const double* R,
                             const double* w, int nw, double* G, double* out);
void launch_pe_form(cudaStream_t s, int nocc, int nl, const double2* a, const double* eps, double c, double alpha,
                    double* out);
void launch_frob_forms(cudaStream_t s, int nj, int n, const double* A, const int* ia, const double* fa,
                       const double* B, const int* ib, const double* C, const int* ic, double* out);

// block Lanczos helpers (complex grid fields)
// Entries per CTA of the complex Gram kernel for vectors of length n and my
// columns: halved from 4096 (down to 256) while fewer than 128 CTAs would run
// and the sum over chunks stays under 64 records; cgram_partials is the
// partial-sum storage (double2 entries) a launch with mx rows needs.
inline size_t cgram_chunk(size_t n, int my) {
  const size_t groups = ((size_t)my + 7) / 8;
  size_t chunk = 4096;
  while (chunk > 256) {
    const size_t nc = (n + chunk - 1) / chunk;
    if (nc * groups >= 128 || 2 * nc > 64) break;
    chunk /= 2;
  }
  return chunk;
}
inline size_t cgram_partials(size_t n, int mx, int my) {
  const size_t chunk = cgram_chunk(n, my);
  return ((n + chunk - 1) / chunk) * (size_t)mx * (size_t)my;
}
void launch_cgram(cudaStream_t s, const double2* X, int mx, const double2* Y, int my, size_t n, int conj_x,
                  double wgt, double2* partial, unsigned* cnt, double2* out);
void launch_cgemm_n(cudaStream_t s, const double2* M, int my, int mx, const double2* X, size_t n, double2* Y,
                    int accumulate, double sign);
void launch_cinv(cudaStream_t s, int n, double2* a, double2* out, int* status);
void launch_block_tridiag(cudaStream_t s, int K, int blk, const double2* A, const double2* B, int bilinear,
                          double2* T);

// whole CG pass in one cooperative launch (kernels_cg.cu)
// Tensor-core projector coefficients (kernels_tc.cu): coef[v * ncol + j] =
// <C_v|Y_j> for FP32 columns Y [ncol][npw] and up to 64 occupied rows, from
// the rows split once into TF32 hi / lo parts (A [128][kpad], FP32, device),
// described by two TMA tensor maps.
struct TcMaps {
  alignas(64) unsigned char hi[128];   // CUtensorMap of A_hi
  alignas(64) unsigned char lo[128];   // CUtensorMap of A_lo
  int kpad = 0;
};
int tc_kpad(int npw);
void tc_split_rows(const std::vector<double2>& C, int nocc, int npw, std::vector<float>* hi, std::vector<float>* lo);
cudaError_t tc_maps(const float* Ahi, const float* Alo, int npw, TcMaps* maps);
size_t tc_part_elems(int npw, int ncol);     // FP32 scratch of launch_tc_dots
cudaError_t tc_prepare();                    // kernel attributes (once, before any capture)
constexpr int kTcMinCols = 256;              // solver columns from which the tensor cores take the dots
cudaError_t launch_tc_dots(cudaStream_t s, const TcMaps& maps, const float2* Y, int npw, int ncol, int nocc,
                           float* part, double2* coef, int* err, unsigned long long limit);

// Per-column state of the persistent CG carried between iterations.
struct PcgCol {
  double gam, alpha, stop, rmin, rbest;
  int it, itb, active, flag;
};
// Sizes of the persistent CG's work buffers for ncol columns in groups of W
// (2: packed pairs of real-in-real-space columns; 1: one column per group).
struct PcgSizes {
  int W = 1, ngrp = 0;
  size_t rec_bytes = 0, rec_total = 0;   // bytes of one plane record, of all
  size_t apart = 0, cst = 0, ctl = 0;    // doubles, PcgCol entries, control words
  size_t Y = 0, grid = 0;                // complex entries
};
PcgSizes pcg_sizes(int nocc, int npw, int ncol, int W, int nplanes, int N, int csize);
// One cooperative launch = one CG pass over ncol columns (kernels_cg.cu), after
// a small launch that sets r = b, x = p = s = 0 and the per-column inputs cin
// ([ncol][4] in T); ctl (z.ctl words) must be zero at launch.  cudaErrorNotSupported when the
// kernel's shared memory does not fit (the caller then uses the multi-launch CG).
template <typename T>
cudaError_t launch_cg_persistent(cudaStream_t s, const Geometry& g, const FftPlan& pl, const Prec<T>& P, int nocc,
                                 int npw, int ncol, const PcgSizes& z, int maxplane, const double2* b64,
                                 const int* outer_active, const double2* E, const double* rr_abs, const double* tk,
                                 double tol_in2, int maxit, cpx<T>* x, cpx<T>* r, cpx<T>* p, cpx<T>* sv, cpx<T>* Y,
                                 cpx<T>* grid, unsigned char* rec, double* apart, PcgCol* cst, unsigned* ctl,
                                 T* cin, int* iters, int* flags, double* rr_out, int* grid_used, int cta_div,
                                 unsigned long long spin_limit, unsigned long long* ptask = nullptr,
                                 int tpb = 256);
// One thread-block cluster per column (kernels_cgc.cu); cudaErrorNotSupported
// when the column's planes do not fit in the shared memory of a cluster.
template <typename T>
cudaError_t launch_cg_cluster(cudaStream_t s, const Geometry& g, const FftPlan& pl, const Prec<T>& P, int nocc,
                              int npw, int ncol, const double2* b64, const int* outer_active, const double2* E,
                              const double* rr_abs, const double* tk, double tol_in2, int maxit, cpx<T>* x,
                              cpx<T>* r, cpx<T>* p, cpx<T>* Ap, int* iters, int* flags, double* rr_out,
                              int* q_used, unsigned long long* ptime = nullptr);
constexpr int kPersistentMaxCols = 256;
constexpr int kPcgChunkMin = 64;   // smallest chunk (sphere entries) of the persistent CG's update phase
// A CG pass whose |r|^2 has not dropped 4x for max(kCgStagWindow, 2 k_best)
// iterations has reached the accuracy of its working precision: it stops, and
// the FP64 refinement around it continues from there.
constexpr int kCgStagWindow = 100;   // sphere entries per task in the persistent CG's update phase

}  // namespace gw
