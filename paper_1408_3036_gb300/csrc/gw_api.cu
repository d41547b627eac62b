// C ABI of libgw (declared in include/gw.h) and the host drivers of the hot
// path: cell set-up, the Sternheimer solver with FP64 iterative refinement,
// the chi0 / eps~ application (Eqs. epsilon, P, P1, P2) and the Lanczos
// recursion with full re-orthogonalisation (Sec. Lanczos).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <type_traits>
#include <vector>

#include "gw.h"
#include "gw_common.cuh"
#include "linalg.cuh"
#include "tune.h"

using namespace gw;

struct gw_ctx {
  double L = 0, ecut = 0, vol = 0;
  int N = 0, N3 = 0, npw = 0, coulomb = 0;
  cudaStream_t user = nullptr, st = nullptr;
  bool own_stream = true;
  cudaEvent_t ev = nullptr;
  FftPlan plan{};
  Geometry geo;
  Prec<double> P64;
  Prec<float> P32;
  std::vector<int> miller;      // [npw][3]
  std::vector<int> sph_index;   // linear grid index
  std::vector<double> kin;
  int nocc = 0;
  std::vector<double> eps;
  std::vector<std::complex<double>> c_occ;   // realified occupied coefficients (host) [nocc][npw]
  int ndef = 0;                  // deflation states (lowest conduction states) after the occupied rows of C
  std::vector<double> eps_def;
  std::map<std::string, std::pair<void*, size_t>> bufs;
  std::map<std::string, std::vector<unsigned char>> tables;   // last contents of read-only index tables
  Work work;
  size_t work_cols = 0;
  double tol = 1e-13, tol_mixed = 1e-10, tol_inner = 1e-5;   // backward errors (FP64 / mixed), inner
  double anorm = 1.0;           // bound on |H - E| used by the backward error
  int cg_kernel = GW_CG_PERSISTENT;   // kernel of the CG passes (gw_set_cg_kernel)
  int maxplane = 0;                   // most sphere entries in one plane i0
  bool use_graphs = true;             // SQMR iterations replayed from a captured CUDA graph
  int imag_route = GW_IMAG_SQMR;      // solver of purely imaginary frequencies (gw_set_imaginary_route)
  double recycle_w0 = 0.0;            // > 0: recycled bases augmented with x(i w0)
  bool use_tc = false;                // tensor-core projector coefficients where they apply (opt-in)
  bool tune = true;                   // launch shapes picked by timing (tune.cu)
  int pcg_tpb = 0;                    // CTA width of the last persistent CG launch
  bool tc_ok = false;                 // the split occupied rows and their tensor maps are ready
  TcMaps tc_maps;
  long long graph_replays = 0;        // replays in the last SQMR solve
  unsigned long long wait_limit = 1ull << 24;   // spins of one device wait before GW_E_TIMEOUT
  long long pcg_iters = 0;      // iterations run by persistent launches
  int pcg_launch_blocks = 0;
  int* pcg_pin = nullptr;       // pinned read-back of the last persistent launch: iterations, flags, error
  size_t pcg_pin_n = 0;
  struct PcgPending {           // that launch, until the caller's next synchronisation (pcg_finish)
    bool on = false;
    int ncol = 0, used = 0, tune_tpb = 0;
    bool fp64 = false;
    std::string tune_key;
  } pcg_pend;
  int pcg_cluster = 0;          // cluster size of the last persistent launch (0: grid-wide kernel)
  int cta_div = 1;              // contexts sharing the GPU concurrently (batch mode)
  int precond = 1;              // 1: kinetic (TPA) preconditioner in the Sternheimer solvers; 0: none
  int op = GW_OP_STERNHEIMER;   // operator of the chi0 / eps~ entries (GW_OP_MODEL: Eq. model_eq)
  std::vector<double> tkin;     // kinetic energy of each occupied state (preconditioner reference)
  bool ptime_init = false;
  double vmax = 0.0;            // max |V_loc|
  int max_iter = 20000, max_outer = 12;
  double stats[6] = {0, 0, 0, 0, 0, 0};
  int* host_pin = nullptr;      // pinned scratch for small read-backs
  unsigned char* stage = nullptr;  // pinned staging ring for small uploads (no stream sync on copy)
  size_t stage_off = 0;
  std::string err;
  // optional per-kernel-class timing with CUDA events on the work stream
  unsigned prof_mask = 0;
  unsigned long long* ptask = nullptr;   // device [36] task timing of the persistent CG (PC_TASKS)
  cudaEvent_t tune_ev[2] = {nullptr, nullptr};   // autotuner timing events
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<int, int>>> ev_used;   // (class, (start, end))
  size_t ev_next = 0;
};

namespace {

// Rows of C the inner solvers project out: the occupied states and, when set,
// the deflation states (whose components the solver adds analytically).
inline int nproj(const gw_ctx* ctx) { return ctx->nocc + ctx->ndef; }

gw_status fail(gw_ctx* ctx, gw_status s, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return s;
}

#define CK(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) {                                                                       \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? GW_E_NOMEM : GW_E_CUDA,                   \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                             \
    }                                                                                              \
  } while (0)

#define TRY(call)                                                                                  \
  do {                                                                                             \
    gw_status s_ = (call);                                                                         \
    if (s_ != GW_OK) return s_;                                                                    \
  } while (0)

// As TRY, except that GW_E_NOCONV is kept in `var` and the work goes on, so
// that the outputs of a solve that missed its tolerance are still written
// (the best iterate) before the status is returned.
#define SOFT(var, call)                                                                            \
  do {                                                                                             \
    gw_status s_ = (call);                                                                         \
    if (s_ == GW_E_NOCONV) var = s_;                                                               \
    else if (s_ != GW_OK) return s_;                                                               \
  } while (0)

template <class X>
gw_status getbuf(gw_ctx* ctx, const std::string& name, size_t count, X** out) {
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(X);
  auto& b = ctx->bufs[name];
  if (b.second < bytes) {
    if (b.first) CK(cudaFree(b.first));
    b.first = nullptr;
    b.second = 0;
    CK(cudaMalloc(&b.first, bytes));
    b.second = bytes;
  }
  *out = reinterpret_cast<X*>(b.first);
  return GW_OK;
}

// Small uploads go through a pinned staging ring: a copy from pageable host
// memory makes the runtime wait for the stream first, one from pinned memory
// is queued like a kernel.  A slot is reused only after the stream has passed
// every copy out of it (the ring wraps with a stream synchronisation).
constexpr size_t kStageBytes = 1 << 20, kStageMax = 64 << 10;

template <class X>
gw_status upload(gw_ctx* ctx, const std::string& name, const std::vector<X>& v, X** out) {
  TRY(getbuf(ctx, name, v.size(), out));
  if (v.empty()) return GW_OK;
  const size_t bytes = v.size() * sizeof(X);
  if (bytes <= kStageMax) {
    if (!ctx->stage) {
      void* p = nullptr;
      if (cudaMallocHost(&p, kStageBytes) != cudaSuccess) {
        cudaGetLastError();
        CK(cudaMemcpyAsync(*out, v.data(), bytes, cudaMemcpyHostToDevice, ctx->st));
        return GW_OK;
      }
      ctx->stage = static_cast<unsigned char*>(p);
      ctx->stage_off = 0;
    }
    const size_t len = (bytes + 255) & ~(size_t)255;
    if (ctx->stage_off + len > kStageBytes) {
      CK(cudaStreamSynchronize(ctx->st));        // every earlier copy out of the ring is done
      ctx->stage_off = 0;
    }
    unsigned char* slot = ctx->stage + ctx->stage_off;
    ctx->stage_off += len;
    std::memcpy(slot, v.data(), bytes);
    CK(cudaMemcpyAsync(*out, slot, bytes, cudaMemcpyHostToDevice, ctx->st));
    return GW_OK;
  }
  CK(cudaMemcpyAsync(*out, v.data(), bytes, cudaMemcpyHostToDevice, ctx->st));
  return GW_OK;
}

// Upload of a read-only table that kernels never write: skipped when the same
// bytes were uploaded last under this name (the per-call column tables of an
// application repeat from one Lanczos step to the next).
template <class X>
gw_status upload_table(gw_ctx* ctx, const std::string& name, const std::vector<X>& v, X** out) {
  const size_t bytes = v.size() * sizeof(X);
  auto& last = ctx->tables[name];
  auto it = ctx->bufs.find(name);
  if (bytes > 0 && it != ctx->bufs.end() && it->second.first && it->second.second >= bytes &&
      last.size() == bytes && std::memcmp(last.data(), v.data(), bytes) == 0) {
    *out = reinterpret_cast<X*>(it->second.first);
    return GW_OK;
  }
  TRY(upload(ctx, name, v, out));
  const unsigned char* p = reinterpret_cast<const unsigned char*>(v.data());
  last.assign(p, p + bytes);
  return GW_OK;
}

gw_status launch_check(gw_ctx* ctx, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, GW_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return GW_OK;
}

gw_status sync(gw_ctx* ctx, const char* where) {
  cudaError_t e = cudaStreamSynchronize(ctx->st);
  if (e != cudaSuccess) return fail(ctx, GW_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return launch_check(ctx, where);
}

// reduction scratch for up to `cols` columns (or Lanczos vectors)
gw_status ensure_work(gw_ctx* ctx, size_t cols) {
  cols = std::max<size_t>(cols, 64);
  if (cols <= ctx->work_cols) return GW_OK;
  // enough partial slots for chunks of 1024 grid points and of 128 sphere entries
  const size_t nch = std::max<size_t>((size_t)ctx->N3 / 1024, (size_t)ctx->npw / 128) + 2;
  const size_t occ = std::max(ctx->nocc + ctx->ndef, 1);
  TRY(getbuf(ctx, "w_part1", nch * cols, &ctx->work.part1));
  TRY(getbuf(ctx, "w_part2", nch * cols * std::max<size_t>(occ, 1), &ctx->work.part2));
  TRY(getbuf(ctx, "w_coef", occ * cols, &ctx->work.coef));
  TRY(getbuf(ctx, "w_cnt_a", cols, &ctx->work.cnt_a));
  TRY(getbuf(ctx, "w_cnt_b", cols, &ctx->work.cnt_b));
  TRY(getbuf(ctx, "w_cnt_c", cols, &ctx->work.cnt_c));
  TRY(getbuf(ctx, "w_cnt_d", cols, &ctx->work.cnt_d));
  TRY(getbuf(ctx, "w_part_d", cols * ((size_t)ctx->geo.npen / 16 + 2) * occ, &ctx->work.part_d));
  CK(cudaMemsetAsync(ctx->work.cnt_d, 0, cols * sizeof(unsigned), ctx->st));
  CK(cudaMemsetAsync(ctx->work.cnt_a, 0, cols * sizeof(unsigned), ctx->st));
  CK(cudaMemsetAsync(ctx->work.cnt_b, 0, cols * sizeof(unsigned), ctx->st));
  CK(cudaMemsetAsync(ctx->work.cnt_c, 0, cols * sizeof(unsigned), ctx->st));
  ctx->work_cols = cols;
  return GW_OK;
}


// ---------------------------------------------------------------------------
// per-kernel-class timing (gw_profile): an event pair around each launch of a
// selected class, resolved by gw_profile_read
// ---------------------------------------------------------------------------
enum ProfClass { PC_ZSCAT = 0, PC_YINV = 1, PC_XH = 2, PC_YFWD = 3, PC_ZGATH = 4, PC_PROJ = 5, PC_CGUPD = 6,
                 PC_REFINE = 7, PC_PCG = 8, PC_TASKS = 9, PC_N = 10 };
// PC_TASKS: the persistent CG's task kinds A, B, C, read back as six
// pseudo-classes after PC_TASKS: busy and wait milliseconds summed over tasks
// (counts: tasks run, and tasks skipped / waits)

int prof_begin(gw_ctx* ctx, int cls) {
  if (!(ctx->prof_mask & (1u << cls))) return -1;
  if (ctx->ev_next + 2 > ctx->ev_pool.size()) {
    for (int i = 0; i < 256; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      ctx->ev_pool.push_back(e);
    }
  }
  const int a = (int)ctx->ev_next;
  ctx->ev_next += 2;
  cudaEventRecord(ctx->ev_pool[a], ctx->st);
  return a;
}

void prof_end(gw_ctx* ctx, int cls, int a) {
  if (a < 0) return;
  cudaEventRecord(ctx->ev_pool[a + 1], ctx->st);
  ctx->ev_used.push_back({cls, {a, a + 1}});
}

#define PROF(cls, stmt)                  \
  do {                                   \
    const int pa_ = prof_begin(ctx, cls); \
    stmt;                                \
    prof_end(ctx, cls, pa_);             \
  } while (0)

template <typename T> Prec<T>& prec_of(gw_ctx* ctx);
template <> Prec<double>& prec_of<double>(gw_ctx* ctx) { return ctx->P64; }
template <> Prec<float>& prec_of<float>(gw_ctx* ctx) { return ctx->P32; }
template <typename T> const char* tname();
template <> const char* tname<double>() { return "64"; }
template <> const char* tname<float>() { return "32"; }

// ---------------------------------------------------------------------------
// elementwise conversion of real arrays
// ---------------------------------------------------------------------------
template <typename A, typename B>
__global__ void k_conv_real(size_t n, const A* __restrict__ in, B* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (B)in[i];
}
template <typename A, typename B>
void conv_real(cudaStream_t s, size_t n, const A* in, B* out) {
  const int nb = (int)std::min<size_t>((n + 255) / 256, 152 * 8);
  ++g_launches;
  k_conv_real<A, B><<<nb, 256, 0, s>>>(n, in, out);
}

// ---------------------------------------------------------------------------
// v^1/2 on real fields: out = v^1/2 in   (or out = sub - v^1/2 in)
// ---------------------------------------------------------------------------
template <typename T>
gw_status sqrtv(gw_ctx* ctx, const T* in, int nb, T* out, const T* sub) {
  cpx<T>* grid;
  TRY(getbuf(ctx, std::string("g_sqv") + tname<T>(), (size_t)nb * ctx->N3, &grid));
  auto& P = prec_of<T>(ctx);
  const Geometry& g = ctx->geo;
  launch_zpass<T>(ctx->st, Z_G2G_FWD, g, P, ctx->plan, grid, nullptr, nullptr, nullptr, nullptr, nullptr,
                  nullptr, in, nullptr, nb);
  launch_ypass<T>(ctx->st, 0, 0, 0, g, P, ctx->plan, grid, nullptr, nb, 1);
  launch_xpass_mul<T>(ctx->st, 0, 0, 0, g, P, ctx->plan, grid, P.sqv_s, nullptr, nb);
  launch_ypass<T>(ctx->st, 1, 0, 0, g, P, ctx->plan, grid, nullptr, nb, 1);
  launch_zpass<T>(ctx->st, sub ? Z_G2G_INV_SUB : Z_G2G_INV, g, P, ctx->plan, grid, nullptr, nullptr, nullptr,
                  nullptr, nullptr, nullptr, sub, out, nb);
  return launch_check(ctx, "sqrtv");
}

// ---------------------------------------------------------------------------
// H applied to FP64 sphere vectors with shift: out = P_c? (H - E) x
// ---------------------------------------------------------------------------
template <typename T>
gw_status h_apply(gw_ctx* ctx, cpx<T>* x, int ncol, const double2* E, const int* active, cpx<T>* out,
                  const GatherDots* dots = nullptr) {
  cpx<T>* grid;
  TRY(getbuf(ctx, std::string("g_h") + tname<T>(), (size_t)ncol * ctx->N3, &grid));
  auto& P = prec_of<T>(ctx);
  const Geometry& g = ctx->geo;
  launch_zpass<T>(ctx->st, Z_SCATTER_INV, g, P, ctx->plan, grid, x, nullptr, nullptr, nullptr, nullptr, active,
                  nullptr, nullptr, ncol);
  launch_ypass<T>(ctx->st, 1, 1, 0, g, P, ctx->plan, grid, active, ncol, 0);
  launch_xpass_mul<T>(ctx->st, 1, 1, 1, g, P, ctx->plan, grid, P.vloc_s, active, ncol);
  launch_ypass<T>(ctx->st, 0, 0, 1, g, P, ctx->plan, grid, active, ncol, 0);
  launch_zpass<T>(ctx->st, Z_GATHER_FWD_H, g, P, ctx->plan, grid, out, nullptr, nullptr, x, E, active, nullptr,
                  nullptr, ncol, dots);
  return launch_check(ctx, "h_apply");
}

// (H - E) x in FP64 for columns that are real in real space, two per complex
// transform (pack, the pruned passes, split through G and -G with the kinetic
// part added); act: host mask of the columns wanted (a pair runs when one of
// its columns is wanted, and both of its outputs are written).
gw_status h_apply_sym(gw_ctx* ctx, const double2* x, int ncol, const double2* E, const std::vector<int>& act,
                      double2* out) {
  const int npw = ctx->npw, npair = (ncol + 1) / 2;
  std::vector<int> ia(npair), ib(npair), pact(npair);
  for (int j = 0; j < npair; ++j) {
    ia[j] = 2 * j;
    ib[j] = (2 * j + 1 < ncol) ? 2 * j + 1 : -1;
    pact[j] = act[2 * j] || (ib[j] >= 0 && act[2 * j + 1]);
  }
  int *dia, *dib, *dpact;
  TRY(upload_table(ctx, "hs_ia", ia, &dia));
  TRY(upload_table(ctx, "hs_ib", ib, &dib));
  TRY(upload(ctx, "hs_act", pact, &dpact));
  double2 *xp, *yp, *grid;
  TRY(getbuf(ctx, "hs_xp", (size_t)npair * npw, &xp));
  TRY(getbuf(ctx, "hs_yp", (size_t)npair * npw, &yp));
  TRY(getbuf(ctx, "g_hs", (size_t)npair * ctx->N3, &grid));
  auto& P = ctx->P64;
  const Geometry& g = ctx->geo;
  launch_pack_pairs(ctx->st, npw, npair, x, dia, dib, dpact, xp);
  launch_zpass<double>(ctx->st, Z_SCATTER_INV, g, P, ctx->plan, grid, xp, nullptr, nullptr, nullptr, nullptr, dpact,
                       nullptr, nullptr, npair);
  launch_ypass<double>(ctx->st, 1, 1, 0, g, P, ctx->plan, grid, dpact, npair, 0);
  launch_xpass_mul<double>(ctx->st, 1, 1, 1, g, P, ctx->plan, grid, P.vloc_s, dpact, npair);
  launch_ypass<double>(ctx->st, 0, 0, 1, g, P, ctx->plan, grid, dpact, npair, 0);
  launch_zpass<double>(ctx->st, Z_GATHER_FWD, g, P, ctx->plan, grid, yp, nullptr, nullptr, nullptr, nullptr, dpact,
                       nullptr, nullptr, npair);
  launch_unpack_pairs(ctx->st, npw, npair, yp, g.sph_neg, dia, dib, dpact, P.kin, E, x, out);
  return launch_check(ctx, "h_apply_sym");
}

// ---------------------------------------------------------------------------
// batched CG on P_c (H - E) P_c x = b, precision T, rhs FP64
// ---------------------------------------------------------------------------
template <typename T>
gw_status cg_solve(gw_ctx* ctx, int ncol, const double2* b64, const double2* E, const int* outer_active,
                   cpx<T>* x, double tol, const double* rr_abs, const double* tk, long long* it_sum, int* it_max,
                   const double* w2 = nullptr) {
  const int npw = ctx->npw;
  const std::string t = tname<T>();
  cpx<T>*r, *p, *Ap, *grid;
  TRY(getbuf(ctx, "cg_r" + t, (size_t)ncol * npw, &r));
  TRY(getbuf(ctx, "cg_p" + t, (size_t)ncol * npw, &p));
  TRY(getbuf(ctx, "cg_Ap" + t, (size_t)ncol * npw, &Ap));
  TRY(getbuf(ctx, "g_cg" + t, (size_t)ncol * ctx->N3, &grid));
  CgState st;
  double* pap;
  TRY(getbuf(ctx, "cg_rr", ncol, &st.rr));
  TRY(getbuf(ctx, "cg_rr0", ncol, &st.rr0));
  TRY(getbuf(ctx, "cg_beta", ncol, &st.beta));
  TRY(getbuf(ctx, "cg_pap", ncol, &pap));
  TRY(getbuf(ctx, "cg_iters", ncol, &st.iters));
  TRY(getbuf(ctx, "cg_flag", ncol, &st.flag));
  TRY(getbuf(ctx, "cg_active", ncol, &st.active));
  TRY(getbuf(ctx, "cg_ndone", 1, &st.n_done));
  TRY(getbuf(ctx, "cg_cnt", ncol, &st.cnt));
  TRY(getbuf(ctx, "cg_rrstop", ncol, &st.rr_stop));
  TRY(getbuf(ctx, "cg_rrmin", ncol, &st.rr_min));
  TRY(getbuf(ctx, "cg_rz", ncol, &st.rz));
  TRY(getbuf(ctx, "cg_rrbest", ncol, &st.rr_best));
  TRY(getbuf(ctx, "cg_itbest", ncol, &st.it_best));
  st.rr_abs = rr_abs;
  st.tk = tk;
  st.ppow = w2 ? 2 : 1;        // (H - E)^2 + w^2: the kinetic preconditioner squared
  cpx<T>* Ap2 = nullptr;
  if (w2) TRY(getbuf(ctx, "cg_Ap2" + t, (size_t)ncol * npw, &Ap2));
  TRY(ensure_work(ctx, ncol));
  CK(cudaMemsetAsync(st.cnt, 0, ncol * sizeof(unsigned), ctx->st));
  CK(cudaMemsetAsync(ctx->work.cnt_c, 0, ncol * sizeof(unsigned), ctx->st));
  CK(cudaMemsetAsync(st.n_done, 0, sizeof(int), ctx->st));
  auto& P = prec_of<T>(ctx);
  const Geometry& g = ctx->geo;
  launch_cg_init<T, double>(ctx->st, npw, ncol, b64, x, r, outer_active, ctx->work, st, P.kin, tol * tol, 0.0);
  GatherDots dots;
  dots.C = P.C;
  dots.nocc = nproj(ctx);
  dots.ncol = ncol;
  dots.part = ctx->work.part_d;
  dots.cnt = ctx->work.cnt_d;
  dots.coef = ctx->work.coef;
  const double tol2 = tol * tol;
  const int check = 8;
  for (int it = 0; it < ctx->max_iter; ++it) {
    PROF(PC_ZSCAT, launch_zpass<T>(ctx->st, Z_SCATTER_INV_PUPD, g, P, ctx->plan, grid, p, r, st.beta, nullptr,
                                   nullptr, st.active, nullptr, nullptr, ncol, nullptr, tk, st.ppow));
    PROF(PC_YINV, launch_ypass<T>(ctx->st, 1, 1, 0, g, P, ctx->plan, grid, st.active, ncol, 0));
    PROF(PC_XH, launch_xpass_mul<T>(ctx->st, 1, 1, 1, g, P, ctx->plan, grid, P.vloc_s, st.active, ncol));
    PROF(PC_YFWD, launch_ypass<T>(ctx->st, 0, 0, 1, g, P, ctx->plan, grid, st.active, ncol, 0));
    PROF(PC_ZGATH, launch_zpass<T>(ctx->st, Z_GATHER_FWD_H, g, P, ctx->plan, grid, Ap, nullptr, nullptr, p, E,
                                   st.active, nullptr, nullptr, ncol, &dots));
    if (w2) {
      // Eq. P2+: A p = P_c (H - E) P_c (H - E) p + w^2 p, two H applications
      PROF(PC_PROJ, launch_proj_update<T>(ctx->st, P.C, nproj(ctx), npw, Ap, ncol, st.active, ctx->work.coef,
                                          ctx->work, nullptr, nullptr));
      launch_zpass<T>(ctx->st, Z_SCATTER_INV, g, P, ctx->plan, grid, Ap, nullptr, nullptr, nullptr, nullptr,
                      st.active, nullptr, nullptr, ncol);
      launch_ypass<T>(ctx->st, 1, 1, 0, g, P, ctx->plan, grid, st.active, ncol, 0);
      launch_xpass_mul<T>(ctx->st, 1, 1, 1, g, P, ctx->plan, grid, P.vloc_s, st.active, ncol);
      launch_ypass<T>(ctx->st, 0, 0, 1, g, P, ctx->plan, grid, st.active, ncol, 0);
      launch_zpass<T>(ctx->st, Z_GATHER_FWD_H, g, P, ctx->plan, grid, Ap2, nullptr, nullptr, Ap, E, st.active,
                      nullptr, nullptr, ncol, &dots);
      launch_proj_update<T>(ctx->st, P.C, nproj(ctx), npw, Ap2, ncol, st.active, ctx->work.coef, ctx->work,
                            nullptr, nullptr);
      launch_sq_shift<T>(ctx->st, npw, ncol, Ap2, p, w2, st.active, ctx->work, pap);
      PROF(PC_CGUPD, launch_cg_update<T>(ctx->st, npw, ncol, x, r, p, Ap2, pap, ctx->work, st, P.kin, tol2,
                                             ctx->max_iter));
    } else {
    PROF(PC_PROJ, launch_proj_update<T>(ctx->st, P.C, nproj(ctx), npw, Ap, ncol, st.active, ctx->work.coef,
                                        ctx->work, p, pap));
    PROF(PC_CGUPD, launch_cg_update<T>(ctx->st, npw, ncol, x, r, p, Ap, pap, ctx->work, st, P.kin, tol2,
                                           ctx->max_iter));
    }
    if ((it % check) == check - 1 || it == ctx->max_iter - 1) {
      CK(cudaMemcpyAsync(ctx->host_pin, st.n_done, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
      TRY(sync(ctx, "cg_solve"));
      if (ctx->host_pin[0] >= ncol) break;
    }
  }
  std::vector<int> its(ncol), flags(ncol);
  CK(cudaMemcpyAsync(its.data(), st.iters, ncol * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(flags.data(), st.flag, ncol * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  TRY(sync(ctx, "cg_solve stats"));
  for (int c = 0; c < ncol; ++c) {
    *it_sum += its[c];
    *it_max = std::max(*it_max, its[c]);
  }
  // FP32 inner solves of the refinement loop stop at a breakdown (p^H A p
  // <= 0 from rounding once the FP32 recursion has gone as far as it can);
  // the FP64 outer residual decides.  In FP64 a breakdown is an error.
  for (int c = 0; c < ncol; ++c)
    if (flags[c] == 2 && std::is_same<T, double>::value) {
      double2 hE;
      double hrr = 0, hrr0 = 0, hpap = 0;
      CK(cudaMemcpy(&hE, E + c, sizeof(double2), cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(&hrr, st.rr + c, sizeof(double), cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(&hrr0, st.rr0 + c, sizeof(double), cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(&hpap, pap + c, sizeof(double), cudaMemcpyDeviceToHost));
      char buf[256];
      std::snprintf(buf, sizeof(buf),
                    "CG breakdown in column %d (shift E = %.6g) after %d iterations (|r|^2 = %.3e of %.3e, "
                    "p^H A p = %.3e): (H - E) is not positive definite on P_c", c, hE.x, its[c], hrr, hrr0, hpap);
      return fail(ctx, GW_E_BREAKDOWN, buf);
    }
  return GW_OK;
}

// ---------------------------------------------------------------------------
// the same CG pass as cg_solve in one cooperative launch (kernels_cg.cu)
// ---------------------------------------------------------------------------
template <typename T>
gw_status cg_solve_persistent(gw_ctx* ctx, int ncol, const double2* b64, const double2* E, const int* outer_active,
                              cpx<T>* x, double tol, const double* rr_abs, const double* tk, bool sym,
                              long long* it_sum, int* it_max, bool* ran) {
  const int npw = ctx->npw;
  const std::string t = tname<T>();
  *ran = true;
  int *iters, *flags;
  double* rr_out;
  TRY(getbuf(ctx, "pcg_rr", ncol, &rr_out));
  TRY(getbuf(ctx, "pcg_iters", ncol, &iters));
  TRY(getbuf(ctx, "pcg_flags", ncol, &flags));
  int used = 0;
  const int pa = prof_begin(ctx, PC_PCG);
  cudaError_t le = cudaErrorNotSupported;
  unsigned* ctl = nullptr;
  std::string tune_key;
  int tune_tpb = 0;
  if (ctx->cg_kernel == GW_CG_CLUSTER) {
    // opt-in: one thread-block cluster per column when the column's planes
    // fit in the cluster's shared memory
    cpx<T>*r, *p, *Ap;
    TRY(getbuf(ctx, "cg_r" + t, (size_t)ncol * npw, &r));
    TRY(getbuf(ctx, "cg_p" + t, (size_t)ncol * npw, &p));
    TRY(getbuf(ctx, "cg_Ap" + t, (size_t)ncol * npw, &Ap));
    int q = 0;
    le = launch_cg_cluster<T>(ctx->st, ctx->geo, ctx->plan, prec_of<T>(ctx), nproj(ctx), npw, ncol, b64, outer_active,
                              E, rr_abs, tk, tol * tol, ctx->max_iter, x, r, p, Ap, iters, flags, rr_out, &q, nullptr);
    used = ncol * q;
    ctx->pcg_cluster = q;
  }
  if (le == cudaErrorNotSupported) {
    cudaGetLastError();
    ctx->pcg_cluster = 0;
    // the grid-wide task-queue kernel: real-in-real-space columns in packed pairs
    const PcgSizes z = pcg_sizes(nproj(ctx), npw, ncol, sym ? 2 : 1, ctx->geo.nplanes, ctx->N,
                                 (int)sizeof(cpx<T>));
    cpx<T>*r, *p, *sv, *Y, *grid;
    unsigned char* rec;
    double* apart;
    PcgCol* cst;
    TRY(getbuf(ctx, "cg_r" + t, (size_t)ncol * npw, &r));
    TRY(getbuf(ctx, "cg_p" + t, (size_t)ncol * npw, &p));
    TRY(getbuf(ctx, "cg_Ap" + t, (size_t)ncol * npw, &sv));
    TRY(getbuf(ctx, "pcg_Y" + t, z.Y, &Y));
    TRY(getbuf(ctx, "g_cg" + t, z.grid, &grid));
    TRY(getbuf(ctx, "pcg_rec", z.rec_total, &rec));
    TRY(getbuf(ctx, "pcg_apart", z.apart, &apart));
    TRY(getbuf(ctx, "pcg_cst", z.cst, &cst));
    TRY(getbuf(ctx, "pcg_ctl", z.ctl, &ctl));
    T* cin;
    TRY(getbuf(ctx, "pcg_cin" + t, (size_t)4 * ncol, &cin));
    CK(cudaMemsetAsync(ctl, 0, z.ctl * sizeof(unsigned), ctx->st));
    unsigned long long* ptask = nullptr;
    if (ctx->prof_mask & (1u << PC_TASKS)) {
      if (!ctx->ptask) {
        TRY(getbuf(ctx, "pcg_ptask", 36, &ctx->ptask));
        CK(cudaMemsetAsync(ctx->ptask, 0, 36 * sizeof(unsigned long long), ctx->st));
      }
      ptask = ctx->ptask;
    }
    // CTA width: 256 (two per SM) or 512 (one per SM), tuned per shape
    char key[160];
    std::snprintf(key, sizeof(key), "pcg1_tpb:%s:N%d:npw%d:nproj%d:ncol%d:W%d:div%d", tname<T>(), ctx->N, npw,
                  nproj(ctx), ncol, z.W, ctx->cta_div);
    const int tpb = tune_pick(key, {256, 512}, ctx->tune && ctx->cta_div == 1);
    if (!ctx->tune_ev[0]) {
      CK(cudaEventCreate(&ctx->tune_ev[0]));
      CK(cudaEventCreate(&ctx->tune_ev[1]));
    }
    const bool timing = ctx->tune && ctx->cta_div == 1 && !tune_known(key);
    if (timing) CK(cudaEventRecord(ctx->tune_ev[0], ctx->st));
    le = launch_cg_persistent<T>(ctx->st, ctx->geo, ctx->plan, prec_of<T>(ctx), nproj(ctx), npw, ncol, z,
                                 ctx->maxplane, b64, outer_active, E, rr_abs, tk, tol * tol, ctx->max_iter, x, r, p,
                                 sv, Y, grid, rec, apart, cst, ctl, cin, iters, flags, rr_out, &used, ctx->cta_div,
                                 ctx->wait_limit, ptask, tpb);
    if (timing && le == cudaSuccess) CK(cudaEventRecord(ctx->tune_ev[1], ctx->st));
    ctx->pcg_tpb = tpb;
    tune_key = key;
    tune_tpb = timing ? tpb : 0;
    if (le == cudaErrorNotSupported) {      // shared memory beyond one SM: the multi-launch CG
      cudaGetLastError();
      prof_end(ctx, PC_PCG, pa);
      *ran = false;
      return GW_OK;
    }
  }
  CK(le);
  prof_end(ctx, PC_PCG, pa);
  // Iteration counts, flags and the error word come back into pinned memory
  // and are read at the caller's next synchronisation (pcg_finish): no stream
  // synchronisation of its own per pass.
  if (ctx->pcg_pin_n < (size_t)(2 * ncol + 1)) {
    if (ctx->pcg_pin) CK(cudaFreeHost(ctx->pcg_pin));
    ctx->pcg_pin = nullptr;
    ctx->pcg_pin_n = 0;
    CK(cudaMallocHost(&ctx->pcg_pin, (size_t)(2 * ncol + 1) * sizeof(int)));
    ctx->pcg_pin_n = (size_t)(2 * ncol + 1);
  }
  CK(cudaMemcpyAsync(ctx->pcg_pin, iters, ncol * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(ctx->pcg_pin + ncol, flags, ncol * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  ctx->pcg_pin[2 * ncol] = 0;
  if (ctl) CK(cudaMemcpyAsync(ctx->pcg_pin + 2 * ncol, ctl + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->st));
  ctx->pcg_pend.on = true;
  ctx->pcg_pend.ncol = ncol;
  ctx->pcg_pend.used = used;
  ctx->pcg_pend.fp64 = std::is_same<T, double>::value;
  ctx->pcg_pend.tune_key = tune_key;
  ctx->pcg_pend.tune_tpb = tune_tpb;
  (void)it_sum;
  (void)it_max;
  return GW_OK;
}

// The read-back of the last persistent launch, after the stream has been
// synchronised: a bounded wait that gave up (GW_E_TIMEOUT), an FP64 breakdown,
// the iteration statistics and the autotuner's sample.
gw_status pcg_finish(gw_ctx* ctx, long long* it_sum, int* it_max) {
  if (!ctx->pcg_pend.on) return GW_OK;
  ctx->pcg_pend.on = false;
  const int ncol = ctx->pcg_pend.ncol;
  const int* its = ctx->pcg_pin;
  const int* fl = ctx->pcg_pin + ncol;
  if (ctx->pcg_pin[2 * ncol]) return fail(ctx, GW_E_TIMEOUT, "persistent CG: a bounded device wait gave up");
  int imax = 0;
  for (int c = 0; c < ncol; ++c) {
    *it_sum += its[c];
    *it_max = std::max(*it_max, its[c]);
    imax = std::max(imax, its[c]);
    if (fl[c] == 2 && ctx->pcg_pend.fp64)
      return fail(ctx, GW_E_BREAKDOWN, "CG breakdown: (H - E) is not positive definite on P_c");
  }
  ctx->pcg_iters += imax;       // iterations of the whole launch (bounded by the slowest column)
  ctx->pcg_launch_blocks = ctx->pcg_pend.used;
  if (ctx->pcg_pend.tune_tpb && imax > 0) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->tune_ev[0], ctx->tune_ev[1]) == cudaSuccess)
      tune_report(ctx->pcg_pend.tune_key, ctx->pcg_pend.tune_tpb, (double)ms / imax);
  }
  return GW_OK;
}

// ---------------------------------------------------------------------------
// batched simplified QMR on P_c (H - E) P_c x = b (complex or indefinite shifts)
// ---------------------------------------------------------------------------
template <typename T>
gw_status qmr_solve(gw_ctx* ctx, int ncol, const double2* b64, const double2* E, const int* outer_active,
                    cpx<T>* x, double tol, const double* rr_abs, const double* tk, long long* it_sum, int* it_max) {
  const int npw = ctx->npw;
  const std::string t = tname<T>();
  cpx<T>*r, *q, *dd, *tt, *grid;
  TRY(getbuf(ctx, "cg_r" + t, (size_t)ncol * npw, &r));
  TRY(getbuf(ctx, "cg_p" + t, (size_t)ncol * npw, &q));
  TRY(getbuf(ctx, "cg_Ap" + t, (size_t)ncol * npw, &tt));
  TRY(getbuf(ctx, "qmr_d" + t, (size_t)ncol * npw, &dd));
  TRY(getbuf(ctx, "g_cg" + t, (size_t)ncol * ctx->N3, &grid));
  QmrState st;
  TRY(getbuf(ctx, "qmr_rho", ncol, &st.rho));
  TRY(getbuf(ctx, "qmr_alpha", ncol, &st.alpha));
  TRY(getbuf(ctx, "qmr_beta", ncol, &st.beta));
  TRY(getbuf(ctx, "qmr_qc", ncol, &st.qcoef));
  TRY(getbuf(ctx, "qmr_dc", ncol, &st.dcoef));
  TRY(getbuf(ctx, "qmr_theta", ncol, &st.theta));
  TRY(getbuf(ctx, "qmr_tau", ncol, &st.tau));
  TRY(getbuf(ctx, "qmr_stop", ncol, &st.rr_stop));
  TRY(getbuf(ctx, "qmr_qbest", ncol, &st.qbest));
  TRY(getbuf(ctx, "qmr_itbest", ncol, &st.itbest));
  TRY(getbuf(ctx, "cg_iters", ncol, &st.iters));
  TRY(getbuf(ctx, "cg_flag", ncol, &st.flag));
  TRY(getbuf(ctx, "cg_active", ncol, &st.active));
  TRY(getbuf(ctx, "cg_ndone", 1, &st.n_done));
  TRY(getbuf(ctx, "cg_cnt", ncol, &st.cnt));
  st.rr_abs = rr_abs;
  st.tk = tk;
  TRY(ensure_work(ctx, ncol));
  CK(cudaMemsetAsync(st.cnt, 0, ncol * sizeof(unsigned), ctx->st));
  CK(cudaMemsetAsync(st.n_done, 0, sizeof(int), ctx->st));
  auto& P = prec_of<T>(ctx);
  const Geometry& g = ctx->geo;
  const int* neg = g.sph_neg;
  launch_qmr<T>(ctx->st, 0, npw, ncol, b64, x, r, q, dd, tt, neg, outer_active, ctx->work, st, P.kin, tol * tol,
                ctx->max_iter);
  GatherDots dots;
  dots.C = P.C;
  dots.nocc = nproj(ctx);
  dots.ncol = ncol;
  dots.part = ctx->work.part_d;
  dots.cnt = ctx->work.cnt_d;
  dots.coef = ctx->work.coef;
  // Mixed path with many columns: the projector coefficients <C_v|t> on the
  // tensor cores (kernels_tc.cu) instead of the dots fused into the gather
  const bool tc = std::is_same<T, float>::value && ctx->use_tc && ctx->tc_ok && ncol >= kTcMinCols;
  float* tc_part = nullptr;
  int* tc_err = nullptr;
  if (tc) {
    TRY(getbuf(ctx, "tc_part", tc_part_elems(npw, ncol), &tc_part));
    TRY(getbuf(ctx, "tc_err", 1, &tc_err));
    CK(cudaMemsetAsync(tc_err, 0, sizeof(int), ctx->st));
  }
  const int check = 8;
  // One iteration: t = P_c (H - E) q, then the four update steps.  Its ten
  // launches read all per-column state from device memory, so the same
  // sequence serves every iteration: it is captured once into a CUDA graph
  // and replayed (one launch instead of ten per iteration); the direct
  // launches remain for a stream that cannot be captured.
  auto iteration = [&]() {
    launch_zpass<T>(ctx->st, Z_SCATTER_INV, g, P, ctx->plan, grid, q, nullptr, nullptr, nullptr, nullptr, st.active,
                    nullptr, nullptr, ncol);
    launch_ypass<T>(ctx->st, 1, 1, 0, g, P, ctx->plan, grid, st.active, ncol, 0);
    launch_xpass_mul<T>(ctx->st, 1, 1, 1, g, P, ctx->plan, grid, P.vloc_s, st.active, ncol);
    launch_ypass<T>(ctx->st, 0, 0, 1, g, P, ctx->plan, grid, st.active, ncol, 0);
    launch_zpass<T>(ctx->st, Z_GATHER_FWD_H, g, P, ctx->plan, grid, tt, nullptr, nullptr, q, E, st.active, nullptr,
                    nullptr, ncol, tc ? nullptr : &dots);
    if constexpr (std::is_same<T, float>::value) {
      if (tc)
        launch_tc_dots(ctx->st, ctx->tc_maps, tt, npw, ncol, nproj(ctx), tc_part, ctx->work.coef, tc_err,
                       std::max<unsigned long long>(ctx->wait_limit / 16, 1024));
    }
    launch_proj_update<T>(ctx->st, P.C, nproj(ctx), npw, tt, ncol, st.active, ctx->work.coef, ctx->work, nullptr,
                          nullptr);
    for (int step = 1; step <= 4; ++step)
      launch_qmr<T>(ctx->st, step, npw, ncol, b64, x, r, q, dd, tt, neg, outer_active, ctx->work, st, P.kin,
                    tol * tol, ctx->max_iter);
  };
  struct ExecGuard {
    cudaGraphExec_t e = nullptr;
    ~ExecGuard() { if (e) cudaGraphExecDestroy(e); }
  } guard;
  cudaGraphExec_t& exec = guard.e;
  unsigned long long per_iter = 0;
  ctx->graph_replays = 0;
  if (ctx->use_graphs) {
    const unsigned long long l0 = g_launches;
    if (cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      iteration();
      cudaGraph_t graph = nullptr;
      if (cudaStreamEndCapture(ctx->st, &graph) == cudaSuccess && graph) {
        if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) exec = nullptr;
        cudaGraphDestroy(graph);
      }
    }
    cudaGetLastError();
    per_iter = g_launches - l0;
    g_launches = l0;           // nothing ran during the capture
  }
  for (int it = 0; it < ctx->max_iter; ++it) {
    if (exec) {
      CK(cudaGraphLaunch(exec, ctx->st));
      g_launches += per_iter;
      ++ctx->graph_replays;
    } else {
      iteration();
    }
    if ((it % check) == check - 1 || it == ctx->max_iter - 1) {
      CK(cudaMemcpyAsync(ctx->host_pin, st.n_done, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
      TRY(sync(ctx, "qmr_solve"));
      if (ctx->host_pin[0] >= ncol) break;
    }
  }
  std::vector<int> its(ncol), flags(ncol);
  int herr = 0;
  CK(cudaMemcpyAsync(its.data(), st.iters, ncol * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(flags.data(), st.flag, ncol * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  if (tc) CK(cudaMemcpyAsync(&herr, tc_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  TRY(sync(ctx, "qmr_solve stats"));
  if (herr) return fail(ctx, GW_E_TIMEOUT, "tensor-core projector: a bounded device wait gave up");
  for (int c = 0; c < ncol; ++c) {
    *it_sum += its[c];
    *it_max = std::max(*it_max, its[c]);
  }
  for (int c = 0; c < ncol; ++c)
    if (flags[c] == 2 && std::is_same<T, double>::value)
      return fail(ctx, GW_E_BREAKDOWN, "SQMR serious breakdown: [q, A q] = 0");
  return GW_OK;
}

// ---------------------------------------------------------------------------
// Sternheimer solves with FP64 iterative refinement:
//   x64 = 0; repeat { d = CG_T(b - A64 x64); x64 += d } until the normwise
//   backward error |b - A64 x64| / (|A| |x64| + |b|) <= tol for every column.
// |A| is bounded by max |G|^2/2 + max |V| + max |E| (set with the occupied
// states).  Each inner solve stops at tol_inner relative to its own right-hand
// side, or at a tenth of the final target, whichever is larger.
// ---------------------------------------------------------------------------
// One inner solve in precision U: simplified QMR, or CG (one persistent launch
// when the columns fit, else the multi-launch form).
template <typename U>
gw_status inner_solve(gw_ctx* ctx, bool qmr, int ncol, const double2* r64, const double2* E, const int* oact,
                      cpx<U>* d, double tol_in, const double* rra, const double* tk, bool sym, long long* it_sum,
                      int* it_max, const double* w2 = nullptr) {
  if (w2) return cg_solve<U>(ctx, ncol, r64, E, oact, d, tol_in, rra, tk, it_sum, it_max, w2);
  if (qmr) return qmr_solve<U>(ctx, ncol, r64, E, oact, d, tol_in, rra, tk, it_sum, it_max);
  if (ncol <= kPersistentMaxCols && ctx->cg_kernel != GW_CG_MULTI_LAUNCH) {
    bool ran = false;
    TRY(cg_solve_persistent<U>(ctx, ncol, r64, E, oact, d, tol_in, rra, tk, sym, it_sum, it_max, &ran));
    if (ran) return GW_OK;
  }
  return cg_solve<U>(ctx, ncol, r64, E, oact, d, tol_in, rra, tk, it_sum, it_max);
}

// w2 (optional, device [ncol]): solve the squared system of Eq. P2+,
// (P_c (H - E) P_c)^2 x + w2 x = b, by CG (w2max: the largest w2, for |A|).
template <typename T>
gw_status solve(gw_ctx* ctx, int ncol, const double2* b64, const double2* E, double2* x64, bool qmr = false,
                const double* tk = nullptr, const double* w2 = nullptr, double w2max = 0.0, int sym_hint = -1) {
  const int npw = ctx->npw;
  const bool mixed = !std::is_same<T, double>::value;
  ctx->pcg_pend.on = false;
  const double tol = mixed ? ctx->tol_mixed : ctx->tol;
  const double tol_in = mixed ? ctx->tol_inner : std::max(1e2 * ctx->tol, 1e-11);
  double2 *r64, *ax;
  cpx<T>* d;
  int* oact;
  double *res2, *bb, *xx, *rra;
  TRY(getbuf(ctx, "sv_r64", (size_t)ncol * npw, &r64));
  TRY(getbuf(ctx, "sv_ax", (size_t)ncol * npw, &ax));
  TRY(getbuf(ctx, std::string("sv_d") + tname<T>(), (size_t)ncol * npw, &d));
  TRY(getbuf(ctx, "sv_oact", ncol, &oact));
  TRY(getbuf(ctx, "sv_res2", ncol, &res2));
  TRY(getbuf(ctx, "sv_bb", ncol, &bb));
  TRY(getbuf(ctx, "sv_xx", ncol, &xx));
  double2 *cb, *cax;
  TRY(getbuf(ctx, "sv_cb", (size_t)ctx->nocc * ncol, &cb));
  TRY(getbuf(ctx, "sv_cax", (size_t)ctx->nocc * ncol, &cax));
  TRY(ensure_work(ctx, ncol));
  double2* cdef = nullptr;
  double* edef = nullptr;
  if (ctx->ndef > 0) {
    TRY(getbuf(ctx, "sv_cdef", (size_t)ctx->ndef * ncol, &cdef));
    TRY(upload(ctx, "sv_edef", ctx->eps_def, &edef));
  }
  CK(cudaMemsetAsync(x64, 0, (size_t)ncol * npw * sizeof(double2), ctx->st));
  CK(cudaMemcpyAsync(r64, b64, (size_t)ncol * npw * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->st));
  // Right-hand sides that are real in real space (b(-G) = conj b(G): real
  // fields, realified occupied states) have real-in-real-space solutions; the
  // CG then packs two columns into one complex transform.  Given by the caller
  // when it knows (sym_hint 0 or 1), else decided from the data, to the FP64
  // rounding of the right-hand sides.
  bool sym = false;
  if (!qmr && sym_hint >= 0) {
    sym = sym_hint != 0;             // known to the caller (real fields and states)
  } else if (!qmr) {
    double* symv;
    TRY(getbuf(ctx, "sv_sym", (size_t)2 * ncol, &symv));
    launch_sym_check(ctx->st, npw, ncol, b64, ctx->geo.sph_neg, symv);
    std::vector<double> hs(2 * ncol);
    CK(cudaMemcpyAsync(hs.data(), symv, 2 * ncol * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    TRY(sync(ctx, "symmetry check"));
    sym = true;
    for (int c = 0; c < ncol; ++c) sym = sym && (hs[c] <= 1e-12 * hs[ncol + c]);
  }
  // C^H b (real coefficients for real-in-real-space columns: the occupied rows are too)
  launch_gram<double>(ctx->st, ctx->P64.C, ctx->nocc, npw, b64, ncol, ctx->work, cb, sym);
  std::vector<int> act(ncol, 1);
  TRY(upload(ctx, "sv_oact", act, &oact));
  std::vector<double> hr(ncol, 0.0), hb(ncol, 0.0), hx(ncol, 0.0), habs(ncol, 0.0);
  TRY(upload(ctx, "sv_rra", habs, &rra));
  long long it_sum = 0;
  int it_max = 0, outer = 0;
  bool done = false;
  double prev_worst = 1e300;
  // Mixed path: a pass in which some column far from convergence does not
  // drop its residual by 10x means the FP32 recurrence cannot resolve that
  // system (a nearly singular, indefinite shift close to a transition); the
  // remaining passes then run the inner solver in FP64.
  bool esc = false;
  double2* d64 = nullptr;
  std::vector<double> hprev;
  for (outer = 0; outer < ctx->max_outer && !done; ++outer) {
    if (ctx->ndef > 0) {
      // Deflation: the inner pass solves on the complement of the occupied and
      // the deflation states, so the deflation components leave its right-hand
      // side (r -= D <D|r>); they are added to x exactly after the pass:
      // x += sum_d D_d <D_d|r> / (eps_d - E)
      const double2* D = ctx->P64.C + (size_t)ctx->nocc * npw;
      launch_gram<double>(ctx->st, D, ctx->ndef, npw, r64, ncol, ctx->work, cdef);
      launch_proj_update<double>(ctx->st, D, ctx->ndef, npw, r64, ncol, oact, cdef, ctx->work, nullptr, nullptr);
      launch_defl_scale(ctx->st, cdef, edef, E, ctx->ndef, ncol, oact);
    }
    if (esc) {
      if (!d64) TRY(getbuf(ctx, "sv_d64", (size_t)ncol * npw, &d64));
      TRY(inner_solve<double>(ctx, qmr, ncol, r64, E, oact, reinterpret_cast<cpx<double>*>(d64),
                              std::max(1e2 * ctx->tol, 1e-11), rra, tk, sym, &it_sum, &it_max, w2));
      if (sym) launch_add_conv_sym<double>(ctx->st, npw, ncol, reinterpret_cast<cpx<double>*>(d64), x64, oact,
                                           ctx->geo.sph_neg);
      else launch_add_conv<double>(ctx->st, npw, ncol, reinterpret_cast<cpx<double>*>(d64), x64, oact);
    } else {
      TRY(inner_solve<T>(ctx, qmr, ncol, r64, E, oact, d, tol_in, rra, tk, sym, &it_sum, &it_max, w2));
      if (sym) launch_add_conv_sym<T>(ctx->st, npw, ncol, d, x64, oact, ctx->geo.sph_neg);
      else launch_add_conv<T>(ctx->st, npw, ncol, d, x64, oact);
    }
    if (ctx->ndef > 0)                // the deflated components, exactly
      launch_proj_update<double>(ctx->st, ctx->P64.C + (size_t)ctx->nocc * npw, ctx->ndef, npw, x64, ncol, oact,
                                 cdef, ctx->work, nullptr, nullptr);
    // r64 = P_c (b - (H - E) x64): C^H (H - E) x64 from the dots fused into the
    // last transform pass, C^H b computed once per solve
    if (w2) {
      // Eq. P2+ residual in FP64: ax = P_c (H - E) P_c (H - E) x + w2 x
      const int pa = prof_begin(ctx, PC_REFINE);
      double2* ax1;
      TRY(getbuf(ctx, "sv_ax1", (size_t)ncol * npw, &ax1));
      GatherDots dots;
      dots.C = ctx->P64.C;
      dots.nocc = ctx->nocc;
      dots.ncol = ncol;
      dots.part = ctx->work.part_d;
      dots.cnt = ctx->work.cnt_d;
      dots.coef = cax;
      TRY(h_apply<double>(ctx, x64, ncol, E, oact, ax1, &dots));
      launch_proj_update<double>(ctx->st, ctx->P64.C, ctx->nocc, npw, ax1, ncol, oact, cax, ctx->work, nullptr,
                                 nullptr);
      TRY(h_apply<double>(ctx, ax1, ncol, E, oact, ax, &dots));
      launch_sq_shift<double>(ctx->st, npw, ncol, ax, x64, w2, oact, ctx->work, nullptr);
      launch_gram<double>(ctx->st, ctx->P64.C, ctx->nocc, npw, ax, ncol, ctx->work, cax);
      prof_end(ctx, PC_REFINE, pa);
    } else {
      const int pa = prof_begin(ctx, PC_REFINE);
      if (sym) {
        // two real-in-real-space columns per FP64 transform
        TRY(h_apply_sym(ctx, x64, ncol, E, act, ax));
        launch_gram<double>(ctx->st, ctx->P64.C, ctx->nocc, npw, ax, ncol, ctx->work, cax, true);
      } else {
        GatherDots dots;
        dots.C = ctx->P64.C;
        dots.nocc = ctx->nocc;
        dots.ncol = ncol;
        dots.part = ctx->work.part_d;
        dots.cnt = ctx->work.cnt_d;
        dots.coef = cax;
        TRY(h_apply<double>(ctx, x64, ncol, E, oact, ax, &dots));
      }
      prof_end(ctx, PC_REFINE, pa);
    }
    launch_residual(ctx->st, npw, ncol, b64, ax, x64, oact, ctx->work, res2, bb, xx, ctx->P64.C, ctx->nocc, cb,
                    cax, sym && !w2);
    CK(cudaMemcpyAsync(r64, ax, (size_t)ncol * npw * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaMemcpyAsync(hr.data(), res2, ncol * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(hb.data(), bb, ncol * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(hx.data(), xx, ncol * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    TRY(sync(ctx, "solve"));
    TRY(pcg_finish(ctx, &it_sum, &it_max));
    if (hprev.empty()) hprev = hb;
    int nact = 0;
    const double anorm = w2 ? ctx->anorm * ctx->anorm + w2max : ctx->anorm;
    for (int c = 0; c < ncol; ++c) {
      if (!act[c]) continue;
      const double scale = anorm * std::sqrt(hx[c]) + std::sqrt(hb[c]);
      const double be = scale > 0 ? std::sqrt(hr[c]) / scale : 0.0;
      if (!std::isfinite(be)) return fail(ctx, GW_E_NONFINITE, "non-finite Sternheimer residual");
      habs[c] = 0.01 * tol * tol * scale * scale;
      if (be > tol) {
        ++nact;
        if (mixed && be > 1e3 * tol && hr[c] > 1e-2 * hprev[c]) esc = true;
      } else {
        act[c] = 0;
      }
      hprev[c] = hr[c];
    }
    // stagnation: a pass that does not halve the worst backward error ends the
    // refinement (accepted within 10x of the target: the floor set by rounding
    // and by the accuracy of the occupied states)
    double worst = 0.0;
    for (int c = 0; c < ncol; ++c) {
      const double scale = anorm * std::sqrt(hx[c]) + std::sqrt(hb[c]);
      if (act[c] && scale > 0) worst = std::max(worst, std::sqrt(hr[c]) / scale);
    }
    done = (nact == 0) || (outer > 0 && worst > 0.5 * prev_worst && worst <= 10.0 * tol);
    prev_worst = worst;
    if (!done) {
      TRY(upload(ctx, "sv_oact", act, &oact));
      TRY(upload(ctx, "sv_rra", habs, &rra));
    }
  }
  // The solution lies in P_c.  Inner passes in FP32 leave valence components
  // at the FP32 rounding level that the residual cannot see (P_c removes them
  // from A x) but the density reduction would: project them out in FP64.
  launch_proj<double>(ctx->st, ctx->P64.C, ctx->nocc, npw, x64, ncol, nullptr, ctx->work, nullptr, nullptr, sym);
  {
    double fin = 0.0;        // final relative FP64 residual |b - A x| / |b| over all columns
    for (int c = 0; c < ncol; ++c) fin = std::max(fin, hb[c] > 0 ? std::sqrt(hr[c] / hb[c]) : 0.0);
    ctx->stats[4] = std::max(ctx->stats[4], fin);
  }
  ctx->stats[0] += ncol;
  ctx->stats[1] = std::max<double>(ctx->stats[1], it_max);
  ctx->stats[2] += (double)it_sum;
  ctx->stats[3] = std::max<double>(ctx->stats[3], outer);
  ctx->stats[5] += (double)it_sum + ncol * outer;
  if (!done) {
    int wc = -1;
    double wbe = -1.0;
    const double anorm = w2 ? ctx->anorm * ctx->anorm + w2max : ctx->anorm;
    for (int c = 0; c < ncol; ++c) {
      if (!act[c]) continue;
      const double scale = anorm * std::sqrt(hx[c]) + std::sqrt(hb[c]);
      const double be = scale > 0 ? std::sqrt(hr[c]) / scale : 0.0;
      if (be > wbe) { wbe = be; wc = c; }
    }
    char buf[256];
    std::snprintf(buf, sizeof(buf),
                  "Sternheimer solve did not converge: column %d backward error %.3e (tol %.1e), |r|/|b| = %.3e, "
                  "|x|/|b| = %.3e after %d passes", wc, wbe, tol,
                  wc >= 0 ? std::sqrt(hr[wc] / hb[wc]) : 0.0, wc >= 0 ? std::sqrt(hx[wc] / hb[wc]) : 0.0, outer);
    return fail(ctx, GW_E_NOCONV, buf);
  }
  return GW_OK;
}

// ---------------------------------------------------------------------------
// chi0 application (Eqs. P1, P2):
//   rhs_{v,b}   = P_c Sphere(FFT(conj(u_v) y_b))
//   x_{o,b,v,s} = (H - e_v - s omega_o)^-1 rhs   (s = +/-; one solve at omega = 0)
//   dn_{o,b}    = -(2/Omega) sum_v u_v IFFT(x^- + x^+)
// The right-hand sides and the density reduction (a few transforms per
// column) run in FP64; the Sternheimer solves (hundreds of H applications per
// column) run with inner precision S and FP64 refinement: CG at omega = 0,
// simplified QMR for any other (real or complex) frequency.
// Fields y are real (y_cplx = false) or complex; dn is complex when dn_cplx.
// ---------------------------------------------------------------------------
gw_status chi0_reduce(gw_ctx* ctx, const double2* sol64, int nb, int nom, void* dn, bool dn_cplx);

// Right-hand sides of Eqs. P1, P2 in FP64: rhs[b * nocc + v] = P_c Sphere(FFT(conj(u_v) y_b))
// for nb fields y (real, or complex when y_cplx), in the context buffer "rhs64".
gw_status rhs_core(gw_ctx* ctx, const void* y, bool y_cplx, int nb, double2** out) {
  using T = double;
  const int npw = ctx->npw, nocc = ctx->nocc, N3 = ctx->N3;
  auto& P = ctx->P64;
  const Geometry& g = ctx->geo;
  const std::string t = tname<T>();
  const int nr = nocc * nb;
  std::vector<int> ca(nr), cy(nr);
  for (int b = 0; b < nb; ++b)
    for (int v = 0; v < nocc; ++v) { ca[b * nocc + v] = v; cy[b * nocc + v] = b; }
  int *dca, *dcy;
  TRY(upload_table(ctx, "rhs_ca", ca, &dca));
  TRY(upload_table(ctx, "rhs_cy", cy, &dcy));
  double2* rhs64;
  TRY(getbuf(ctx, "rhs64", (size_t)nr * npw, &rhs64));
  TRY(ensure_work(ctx, std::max(nr, 1)));
  if (!y_cplx) {
    // real fields and real u_v: the products of states 2k and 2k+1 with the
    // same field share one complex transform, split afterwards through G, -G
    const int hp = (nocc + 1) / 2, npair = hp * nb;
    std::vector<int> pa(npair), py(npair), pa2(npair), ia(npair), ib(npair);
    for (int b = 0; b < nb; ++b)
      for (int k = 0; k < hp; ++k) {
        const int j = b * hp + k;
        const bool two = 2 * k + 1 < nocc;
        pa[j] = 2 * k;
        py[j] = b;
        pa2[j] = two ? 2 * k + 1 : -1;
        ia[j] = b * nocc + 2 * k;
        ib[j] = two ? b * nocc + 2 * k + 1 : -1;
      }
    int *dpa, *dpy, *dpa2, *dia, *dib;
    TRY(upload_table(ctx, "rhsp_a", pa, &dpa));
    TRY(upload_table(ctx, "rhsp_y", py, &dpy));
    TRY(upload_table(ctx, "rhsp_a2", pa2, &dpa2));
    TRY(upload_table(ctx, "rhsp_ia", ia, &dia));
    TRY(upload_table(ctx, "rhsp_ib", ib, &dib));
    cpx<T>* grid;
    double2* yp;
    TRY(getbuf(ctx, "g_rhs" + t, (size_t)npair * N3, &grid));
    TRY(getbuf(ctx, "rhs_pk", (size_t)npair * npw, &yp));
    launch_xpass_prod_fwd<T>(ctx->st, g, P, ctx->plan, reinterpret_cast<const cpx<T>*>(y), 0, P.U, 0, 0, dpa, dpy,
                             grid, npair, dpa2, dpy);
    launch_ypass<T>(ctx->st, 0, 0, 1, g, P, ctx->plan, grid, nullptr, npair, 0);
    launch_zpass<T>(ctx->st, Z_GATHER_FWD, g, P, ctx->plan, grid, yp, nullptr, nullptr, nullptr, nullptr, nullptr,
                    nullptr, nullptr, npair);
    launch_unpack_pairs(ctx->st, npw, npair, yp, g.sph_neg, dia, dib, nullptr, nullptr, nullptr, nullptr, rhs64);
  } else {
    cpx<T>* grid;
    TRY(getbuf(ctx, "g_rhs" + t, (size_t)nr * N3, &grid));
    launch_xpass_prod_fwd<T>(ctx->st, g, P, ctx->plan, reinterpret_cast<const cpx<T>*>(y), 1, P.U, 0, 1, dca, dcy,
                             grid, nr);
    launch_ypass<T>(ctx->st, 0, 0, 1, g, P, ctx->plan, grid, nullptr, nr, 0);
    launch_zpass<T>(ctx->st, Z_GATHER_FWD, g, P, ctx->plan, grid, rhs64, nullptr, nullptr, nullptr, nullptr, nullptr,
                    nullptr, nullptr, nr);
  }
  // P_c once: psi_v* y has a large component along the occupied states (e.g.
  // <psi_v|y psi_v>) and one pass leaves |C C^H - 1| times it behind; the
  // solver's FP64 residual P_c (b - A x) removes that remnant
  launch_proj<double>(ctx->st, ctx->P64.C, nocc, npw, rhs64, nr, nullptr, ctx->work, nullptr, nullptr, !y_cplx);
  *out = rhs64;
  return launch_check(ctx, "rhs");
}

// ---------------------------------------------------------------------------
// The model operator (Sec. Dielectric model, Eq. model_eq), every step in
// precision T: H -> T in Eq. P2a turns each Sternheimer solve into one
// division by the kinetic denominators,
//   rhs_{b,v}  = P_c Sphere(FFT(conj(u_v) y_b))
//   sol_{o,b,v} = P_c [ (pinv(|G|^2/2 - e_v - w_o) + pinv(|G|^2/2 - e_v + w_o)) rhs_{b,v} ]
//   dn_{o,b}   = -(2/Omega) sum_v u_v IFFT(sol_{o,b,v})
// (the two signs summed before the second projector, which is linear).
// y: [nb][N_g] real or complex (interleaved) in T; dn: [nom][nb][N_g] in T.
// ---------------------------------------------------------------------------
template <typename T>
gw_status chi0_model_core(gw_ctx* ctx, const T* y, bool y_cplx, int nb, const std::vector<double2>& omega, T* dn,
                          bool dn_cplx) {
  const int npw = ctx->npw, nocc = ctx->nocc;
  const int nom = (int)omega.size();
  const int nr = nocc * nb, nsol = nom * nr;
  auto& P = prec_of<T>(ctx);
  const Geometry& g = ctx->geo;
  const std::string t = tname<T>();
  std::vector<int> ca(nr), cy(nr), src(nsol), gstart(nom * nb + 1), colv(nsol);
  std::vector<double2> Em(nsol), Ep(nsol);
  for (int b = 0; b < nb; ++b)
    for (int v = 0; v < nocc; ++v) { ca[b * nocc + v] = v; cy[b * nocc + v] = b; }
  for (int o = 0; o < nom; ++o)
    for (int b = 0; b < nb; ++b)
      for (int v = 0; v < nocc; ++v) {
        const int j = (o * nb + b) * nocc + v;
        src[j] = b * nocc + v;
        colv[j] = v;
        Em[j] = make_double2(ctx->eps[v] + omega[o].x, omega[o].y);     // T - e_v - w
        Ep[j] = make_double2(ctx->eps[v] - omega[o].x, -omega[o].y);    // T - e_v + w
      }
  for (int j = 0; j <= nom * nb; ++j) gstart[j] = j * nocc;
  int *dca, *dcy, *dsrc, *dgs, *dcv;
  double2 *dEm, *dEp;
  TRY(upload_table(ctx, "mod_ca", ca, &dca));
  TRY(upload_table(ctx, "mod_cy", cy, &dcy));
  TRY(upload_table(ctx, "mod_src", src, &dsrc));
  TRY(upload_table(ctx, "mod_em", Em, &dEm));
  TRY(upload_table(ctx, "mod_ep", Ep, &dEp));
  TRY(upload_table(ctx, "mod_gs", gstart, &dgs));
  TRY(upload_table(ctx, "mod_cv", colv, &dcv));
  cpx<T> *grid, *rhs, *sol;
  TRY(getbuf(ctx, "mod_grid" + t, (size_t)std::max(nr, nsol) * ctx->N3, &grid));
  TRY(getbuf(ctx, "mod_rhs" + t, (size_t)nr * npw, &rhs));
  TRY(getbuf(ctx, "mod_sol" + t, (size_t)nsol * npw, &sol));
  TRY(ensure_work(ctx, std::max(nsol, 1)));
  launch_xpass_prod_fwd<T>(ctx->st, g, P, ctx->plan, reinterpret_cast<const cpx<T>*>(y), y_cplx ? 1 : 0, P.U, 0,
                           1, dca, dcy, grid, nr);
  launch_ypass<T>(ctx->st, 0, 0, 1, g, P, ctx->plan, grid, nullptr, nr, 0);
  launch_zpass<T>(ctx->st, Z_GATHER_FWD, g, P, ctx->plan, grid, rhs, nullptr, nullptr, nullptr, nullptr, nullptr,
                  nullptr, nullptr, nr);
  // real fields and realified states: real-in-real-space right-hand sides and,
  // at real frequencies (denominators even in G), solutions: real coefficients
  bool real_w = !y_cplx;
  for (const double2& w : omega) real_w = real_w && w.y == 0.0;
  launch_proj<T>(ctx->st, P.C, nocc, npw, rhs, nr, nullptr, ctx->work, nullptr, nullptr, !y_cplx);
  launch_model_scale<T>(ctx->st, npw, nsol, P.kin, rhs, dsrc, dEm, dEp, sol);
  launch_proj<T>(ctx->st, P.C, nocc, npw, sol, nsol, nullptr, ctx->work, nullptr, nullptr, real_w);
  launch_zpass<T>(ctx->st, Z_SCATTER_INV, g, P, ctx->plan, grid, sol, nullptr, nullptr, nullptr, nullptr, nullptr,
                  nullptr, nullptr, nsol);
  launch_ypass<T>(ctx->st, 1, 1, 0, g, P, ctx->plan, grid, nullptr, nsol, 0);
  cpx<T>* parts;
  const size_t nparts = (size_t)kMaxReduceParts * ctx->N3;   // enough whenever a split pays (few groups)
  TRY(getbuf(ctx, "mod_parts" + t, nparts, &parts));
  launch_xpass_inv_reduce<T>(ctx->st, g, P, ctx->plan, grid, dgs, dcv, nom * nb, -2.0 / ctx->vol,
                             dn_cplx ? nullptr : dn, dn_cplx ? reinterpret_cast<cpx<T>*>(dn) : nullptr, 0, parts,
                             nparts, nocc);
  for (int i = 0; i < 6; ++i) ctx->stats[i] = 0;
  return launch_check(ctx, "chi0 model");
}

template <typename S>
gw_status chi0_core(gw_ctx* ctx, const void* y, bool y_cplx, int nb, const std::vector<double2>& omega, void* dn,
                    bool dn_cplx) {
  if (ctx->op == GW_OP_MODEL)
    return chi0_model_core<double>(ctx, reinterpret_cast<const double*>(y), y_cplx, nb, omega,
                                   reinterpret_cast<double*>(dn), dn_cplx);
  const int npw = ctx->npw, nocc = ctx->nocc;
  const int nom = (int)omega.size();
  double2* rhs64;
  TRY(rhs_core(ctx, y, y_cplx, nb, &rhs64));
  double2* sol64;
  const int nsol = nom * nb * nocc;
  TRY(getbuf(ctx, "sol64", (size_t)nsol * npw, &sol64));
  // -- solver columns: the frequencies solved as Eq. P2 (CG at 0, SQMR
  // otherwise) first, then the purely imaginary ones when the squared route of
  // Eq. P2+ is selected (one Hermitian positive definite solve per state)
  std::vector<int> src, s0(nsol, -1), s1(nsol, -1);
  std::vector<double2> E;
  std::vector<double> tk, w2v;
  bool qmr = false;
  const bool sq_route = ctx->imag_route == GW_IMAG_SQUARED;
  auto squared = [&](int o) { return sq_route && omega[o].x == 0.0 && omega[o].y != 0.0; };
  int nstd = 0;
  double w2max = 0.0;
  for (int pass = 0; pass < 2; ++pass) {
    for (int o = 0; o < nom; ++o) {
      if (squared(o) != (pass == 1)) continue;
      const bool zero = (omega[o].x == 0.0 && omega[o].y == 0.0);
      if (pass == 0) qmr |= !zero;
      const int ns = (zero || pass == 1) ? 1 : 2;
      for (int b = 0; b < nb; ++b)
        for (int v = 0; v < nocc; ++v) {
          const int k = (o * nb + b) * nocc + v;
          const int first = (int)src.size();
          for (int sg = 0; sg < ns; ++sg) {
            src.push_back(b * nocc + v);
            const double sgn = (sg == 0) ? 1.0 : -1.0;     // x^-: H - e_v - w;  x^+: H - e_v + w
            if (pass == 0) E.push_back(make_double2(ctx->eps[v] + sgn * omega[o].x, sgn * omega[o].y));
            else E.push_back(make_double2(ctx->eps[v], 0.0));
            tk.push_back(ctx->tkin[v]);
            if (pass == 1) {
              w2v.push_back(omega[o].y * omega[o].y);
              w2max = std::max(w2max, omega[o].y * omega[o].y);
            }
          }
          s0[k] = first;
          s1[k] = ns == 2 ? first + 1 : -1;
        }
    }
    if (pass == 0) nstd = (int)src.size();
  }
  const int ncol = (int)src.size(), nsq = ncol - nstd;
  int *dsrc, *ds0, *ds1;
  double2* dE;
  TRY(upload_table(ctx, "col_src", src, &dsrc));
  TRY(upload_table(ctx, "col_s0", s0, &ds0));
  TRY(upload_table(ctx, "col_s1", s1, &ds1));
  TRY(upload_table(ctx, "col_E", E, &dE));
  double* dtk = nullptr;
  if (ctx->precond) TRY(upload_table(ctx, "col_tk", tk, &dtk));
  double2 *bcol, *xcol;
  TRY(getbuf(ctx, "bcol", (size_t)ncol * npw, &bcol));
  TRY(getbuf(ctx, "xcol", (size_t)ncol * npw, &xcol));
  launch_gather_rows<double, double>(ctx->st, npw, ncol, rhs64, dsrc, bcol);
  gw_status sv = GW_OK;
  // real fields at omega = 0: right-hand sides real in real space by construction
  if (nstd > 0) SOFT(sv, (solve<S>(ctx, nstd, bcol, dE, xcol, qmr, dtk, nullptr, 0.0, (!qmr && !y_cplx) ? 1 : -1)));
  if (nsq > 0) {
    // Eq. P2+: ((H - e_v)^2 + w^2) y = 2 (H - e_v) b gives y = x^- + x^+ at
    // omega = i w; solved for x = y / 2 from the right-hand side P_c (H - e_v) b
    double2* bs = bcol + (size_t)nstd * npw;
    double2* hb;
    double* dw2;
    TRY(getbuf(ctx, "sq_hb", (size_t)nsq * npw, &hb));
    TRY(upload(ctx, "sq_w2", w2v, &dw2));
    TRY(h_apply<double>(ctx, bs, nsq, dE + nstd, nullptr, hb, nullptr));
    launch_proj<double>(ctx->st, ctx->P64.C, nocc, npw, hb, nsq, nullptr, ctx->work, nullptr, nullptr);
    CK(cudaMemcpyAsync(bs, hb, (size_t)nsq * npw * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->st));
    SOFT(sv, (solve<S>(ctx, nsq, bs, dE + nstd, xcol + (size_t)nstd * npw, false, dtk ? dtk + nstd : nullptr, dw2,
                       w2max)));
  }
  // -- combine: x^- + x^+, or 2 x at omega = 0 (x^- = x^+) and on the squared route
  launch_combine(ctx->st, npw, nsol, xcol, ds0, ds1, 1.0, 2.0, sol64);
  TRY(chi0_reduce(ctx, sol64, nb, nom, dn, dn_cplx));
  return sv;
}

// density reduction of Eq. P1: dn_{o,b} = -(2/Omega) sum_v u_v IFFT(sol_{o,b,v}),
// sol [nom][nb][nocc][npw] (x^- + x^+ per occupied state)
gw_status chi0_reduce(gw_ctx* ctx, const double2* sol64, int nb, int nom, void* dn, bool dn_cplx) {
  using T = double;
  const int nocc = ctx->nocc, N3 = ctx->N3;
  const int nsol = nom * nb * nocc;
  auto& P = ctx->P64;
  const Geometry& g = ctx->geo;
  const std::string t = tname<T>();
  cpx<T>* parts;
  const size_t nparts = (size_t)kMaxReduceParts * N3;   // enough whenever a split pays (few groups)
  TRY(getbuf(ctx, "dn_parts" + t, nparts, &parts));
  if (!dn_cplx) {
    // real densities: the solutions of states 2k and 2k+1 (real in real
    // space) share one inverse transform, f_2k + i f_2k+1
    const int hp = (nocc + 1) / 2, ng = nom * nb, npair = hp * ng;
    std::vector<int> ia(npair), ib(npair), gs(ng + 1), cv(npair), cv2(npair);
    for (int o = 0; o < ng; ++o)
      for (int k = 0; k < hp; ++k) {
        const int j = o * hp + k;
        const bool two = 2 * k + 1 < nocc;
        ia[j] = o * nocc + 2 * k;
        ib[j] = two ? o * nocc + 2 * k + 1 : -1;
        cv[j] = 2 * k;
        cv2[j] = two ? 2 * k + 1 : -1;
      }
    for (int o = 0; o <= ng; ++o) gs[o] = o * hp;
    int *dia, *dib, *dgs, *dcv, *dcv2;
    TRY(upload_table(ctx, "dnp_ia", ia, &dia));
    TRY(upload_table(ctx, "dnp_ib", ib, &dib));
    TRY(upload_table(ctx, "dnp_gs", gs, &dgs));
    TRY(upload_table(ctx, "dnp_cv", cv, &dcv));
    TRY(upload_table(ctx, "dnp_cv2", cv2, &dcv2));
    double2* xp;
    cpx<T>* gd;
    TRY(getbuf(ctx, "dn_pk", (size_t)npair * ctx->npw, &xp));
    TRY(getbuf(ctx, "g_dn" + t, (size_t)npair * N3, &gd));
    launch_pack_pairs(ctx->st, ctx->npw, npair, sol64, dia, dib, nullptr, xp);
    launch_zpass<T>(ctx->st, Z_SCATTER_INV, g, P, ctx->plan, gd, xp, nullptr, nullptr, nullptr, nullptr, nullptr,
                    nullptr, nullptr, npair);
    launch_ypass<T>(ctx->st, 1, 1, 0, g, P, ctx->plan, gd, nullptr, npair, 0);
    launch_xpass_inv_reduce<T>(ctx->st, g, P, ctx->plan, gd, dgs, dcv, ng, -2.0 / ctx->vol,
                               reinterpret_cast<double*>(dn), nullptr, 0, parts, nparts, hp, dcv2);
    return launch_check(ctx, "chi0");
  }
  cpx<T>* gd;
  TRY(getbuf(ctx, "g_dn" + t, (size_t)nsol * N3, &gd));
  launch_zpass<T>(ctx->st, Z_SCATTER_INV, g, P, ctx->plan, gd, const_cast<double2*>(sol64), nullptr, nullptr,
                  nullptr, nullptr, nullptr, nullptr, nullptr, nsol);
  launch_ypass<T>(ctx->st, 1, 1, 0, g, P, ctx->plan, gd, nullptr, nsol, 0);
  std::vector<int> gstart(nom * nb + 1), colv(nsol);
  for (int j = 0; j <= nom * nb; ++j) gstart[j] = j * nocc;
  for (int j = 0; j < nsol; ++j) colv[j] = j % nocc;
  int *dgs, *dcv;
  TRY(upload_table(ctx, "dn_gs", gstart, &dgs));
  TRY(upload_table(ctx, "dn_cv", colv, &dcv));
  launch_xpass_inv_reduce<T>(ctx->st, g, P, ctx->plan, gd, dgs, dcv, nom * nb, -2.0 / ctx->vol,
                             dn_cplx ? nullptr : reinterpret_cast<double*>(dn),
                             dn_cplx ? reinterpret_cast<double2*>(dn) : nullptr, 0, parts, nparts, nocc);
  return launch_check(ctx, "chi0");
}

// <r|p* e> = conj(u_p(r)) u_e(r) / Omega for the pole states p, split into the
// real and imaginary parts: out[j][0][r], out[j][1][r]
__global__ void k_pair_product(size_t n3, int np, const double2* __restrict__ up, const double2* __restrict__ ue,
                               double inv_vol, double* __restrict__ out) {
  const size_t n = n3 * np;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t j = i / n3, r = i - j * n3;
    const double2 a = up[i], b = ue[r];
    out[(2 * j) * n3 + r] = (a.x * b.x + a.y * b.y) * inv_vol;
    out[(2 * j + 1) * n3 + r] = (a.x * b.y - a.y * b.x) * inv_vol;
  }
}

// complex fields: out = v^1/2 in  (or out = sub - v^1/2 in)
__global__ void k_csub(size_t n, const double2* __restrict__ a, const double2* __restrict__ b,
                       double2* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double2 x = a[i], y = b[i];
    out[i] = make_double2(x.x - y.x, x.y - y.y);
  }
}

// real -> complex (imaginary part zero)
__global__ void k_promote(size_t n, const double* __restrict__ a, double2* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = make_double2(a[i], 0.0);
}

gw_status sqrtv_c(gw_ctx* ctx, const double2* in, int nb, double2* out, const double2* sub) {
  double2* grid;
  TRY(getbuf(ctx, "g_sqvc", (size_t)nb * ctx->N3, &grid));
  auto& P = ctx->P64;
  const Geometry& g = ctx->geo;
  const size_t n = (size_t)nb * ctx->N3;
  CK(cudaMemcpyAsync(grid, in, n * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->st));
  launch_zpass<double>(ctx->st, Z_G2G_FWD, g, P, ctx->plan, grid, nullptr, nullptr, nullptr, nullptr, nullptr,
                       nullptr, nullptr, nullptr, nb);
  launch_ypass<double>(ctx->st, 0, 0, 0, g, P, ctx->plan, grid, nullptr, nb, 1);
  launch_xpass_mul<double>(ctx->st, 0, 0, 0, g, P, ctx->plan, grid, P.sqv_s, nullptr, nb);
  launch_ypass<double>(ctx->st, 1, 0, 0, g, P, ctx->plan, grid, nullptr, nb, 1);
  launch_zpass<double>(ctx->st, Z_G2G_INV, g, P, ctx->plan, grid, nullptr, nullptr, nullptr, nullptr, nullptr,
                       nullptr, nullptr, nullptr, nb);
  const int nblk = (int)std::min<size_t>((n + 255) / 256, 152 * 8);
  if (sub) {
    ++g_launches;
    k_csub<<<nblk, 256, 0, ctx->st>>>(n, sub, grid, out);
  } else {
    CK(cudaMemcpyAsync(out, grid, n * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->st));
  }
  return launch_check(ctx, "sqrtv_c");
}

// eps~ (or chi0 when chi0_only) on nb fields; x real or complex; out complex
// when x is complex or a frequency is complex, real otherwise
template <typename S>
gw_status eps_core(gw_ctx* ctx, const void* x, bool x_cplx, int nb, const std::vector<double2>& omega, void* out,
                   bool chi0_only) {
  const int N3 = ctx->N3;
  const int nom = (int)omega.size();
  bool out_cplx = x_cplx;
  for (auto& o : omega) out_cplx |= (o.y != 0.0);
  if (!out_cplx) {
    const double* x64 = reinterpret_cast<const double*>(x);
    double* out64 = reinterpret_cast<double*>(out);
    if (chi0_only) return chi0_core<S>(ctx, x64, false, nb, omega, out64, false);
    double *y, *dn;
    TRY(getbuf(ctx, "eps_y", (size_t)nb * N3, &y));
    TRY(getbuf(ctx, "eps_dn", (size_t)nom * nb * N3, &dn));
    TRY(sqrtv<double>(ctx, x64, nb, y, nullptr));
    gw_status sv = GW_OK;
    SOFT(sv, (chi0_core<S>(ctx, y, false, nb, omega, dn, false)));
    for (int k = 0; k < nom; ++k)
      TRY(sqrtv<double>(ctx, dn + (size_t)k * nb * N3, nb, out64 + (size_t)k * nb * N3, x64));
    TRY(launch_check(ctx, "eps out"));
    return sv;
  }
  // complex pipeline: promote a real input
  const double2* xc = reinterpret_cast<const double2*>(x);
  if (!x_cplx) {
    double2* tmp;
    TRY(getbuf(ctx, "eps_xc", (size_t)nb * N3, &tmp));
    const size_t n = (size_t)nb * N3;
    ++g_launches;
    k_promote<<<(int)std::min<size_t>((n + 255) / 256, 152 * 8), 256, 0, ctx->st>>>(
        n, reinterpret_cast<const double*>(x), tmp);
    xc = tmp;
  }
  double2* outc = reinterpret_cast<double2*>(out);
  if (chi0_only) return chi0_core<S>(ctx, xc, true, nb, omega, outc, true);
  double2 *y, *dn;
  TRY(getbuf(ctx, "eps_yc", (size_t)nb * N3, &y));
  TRY(getbuf(ctx, "eps_dnc", (size_t)nom * nb * N3, &dn));
  TRY(sqrtv_c(ctx, xc, nb, y, nullptr));
  gw_status sv = GW_OK;
  SOFT(sv, (chi0_core<S>(ctx, y, true, nb, omega, dn, true)));
  for (int k = 0; k < nom; ++k)
    TRY(sqrtv_c(ctx, dn + (size_t)k * nb * N3, nb, outc + (size_t)k * nb * N3, xc));
  TRY(launch_check(ctx, "eps out"));
  return sv;
}

gw_status check_omega(gw_ctx* ctx, const double* omega, int n, std::vector<double2>* out) {
  out->clear();
  for (int i = 0; i < n; ++i) {
    const double re = omega[2 * i], im = omega[2 * i + 1];
    if (!std::isfinite(re) || !std::isfinite(im)) return fail(ctx, GW_E_NONFINITE, "non-finite omega");
    out->push_back(make_double2(re, im));
  }
  return GW_OK;
}

gw_status begin(gw_ctx* ctx) {
  if (!ctx) return GW_E_ARG;
  ctx->err.clear();
  return GW_OK;
}

gw_status finish(gw_ctx* ctx, gw_status s) {
  cudaError_t e = cudaStreamSynchronize(ctx->st);
  if (s == GW_OK && e != cudaSuccess) return fail(ctx, GW_E_CUDA, cudaGetErrorString(e));
  return s;
}

// input staging: returns a device pointer holding `bytes` of the caller's data
gw_status stage_in(gw_ctx* ctx, const char* name, const void* p, size_t bytes, int dev, const void** out) {
  if (dev) { *out = p; return GW_OK; }
  unsigned char* b;
  TRY(getbuf(ctx, name, bytes, &b));
  CK(cudaMemcpyAsync(b, p, bytes, cudaMemcpyHostToDevice, ctx->st));
  *out = b;
  return GW_OK;
}
gw_status stage_out(gw_ctx* ctx, const char* name, void* p, size_t bytes, int dev, void** out) {
  if (dev) { *out = p; return GW_OK; }
  unsigned char* b;
  TRY(getbuf(ctx, name, bytes, &b));
  *out = b;
  return GW_OK;
}
gw_status copy_back(gw_ctx* ctx, void* host, const void* devp, size_t bytes, int dev) {
  if (dev) return GW_OK;
  CK(cudaMemcpyAsync(host, devp, bytes, cudaMemcpyDeviceToHost, ctx->st));
  return GW_OK;
}

gw_status need_occ(gw_ctx* ctx) {
  if (ctx->nocc <= 0) return fail(ctx, GW_E_ARG, "gw_set_occupied has not been called");
  return GW_OK;
}

// ---------------------------------------------------------------------------
// Lanczos (Sec. Lanczos) on real fields, FP64 vectors and inner products
// ---------------------------------------------------------------------------
// width = 2: the vectors are pairs (real part, imaginary part) of complex
// fields stacked into one real vector of 2 N_g entries: for a real symmetric
// eps~ (real omega) this is the Lanczos recursion of a complex start vector in
// the Hermitian inner product.  *done (optional) receives the steps completed
// (fewer than K at an invariant subspace, where GW_E_BREAKDOWN is returned).
template <typename T>
// k0 > 0: resume at step k0 from rows 0..k0 of Q and alpha[0..k0), beta[0..k0)
// (x0 unused).
gw_status lanczos_core(gw_ctx* ctx, const double* x0, int K, const std::vector<double2>& omega, double* alpha,
                       double* beta, double* Q, int width = 1, int* done = nullptr, int k0 = 0) {
  const int N3 = width * ctx->N3;
  const double wgt = ctx->vol / ctx->N3;
  if (done) *done = 0;
  double *w, *h, *nrm;
  TRY(getbuf(ctx, "lz_w", N3, &w));
  TRY(getbuf(ctx, "lz_h", K + 1, &h));
  TRY(getbuf(ctx, "lz_nrm", 1, &nrm));
  TRY(ensure_work(ctx, (size_t)width * (K + 1)));   // partial sums of the stacked length
  if (k0 == 0) {
    launch_dot(ctx->st, N3, x0, x0, wgt, 1, ctx->work, nrm);
    launch_lz_axpy(ctx->st, N3, 2, nrm, const_cast<double*>(x0), nullptr, Q);
  }
  for (int k = k0; k < K; ++k) {
    double* qk = Q + (size_t)k * N3;
    TRY(eps_core<T>(ctx, qk, false, width, omega, w, false));
    if (done) *done = k + 1;
    if (k > 0) launch_lz_axpy(ctx->st, N3, 0, beta + (k - 1), w, Q + (size_t)(k - 1) * N3, nullptr);
    launch_dot(ctx->st, N3, qk, w, wgt, 0, ctx->work, alpha + k);
    launch_lz_axpy(ctx->st, N3, 1, alpha + k, w, qk, nullptr);
    for (int pass = 0; pass < 2; ++pass) {
      launch_gemv_t(ctx->st, Q, N3, N3, w, wgt, k + 1, ctx->work, h);
      launch_gemv_n(ctx->st, Q, N3, N3, h, k + 1, w);
    }
    if (k == K - 1) break;
    launch_dot(ctx->st, N3, w, w, wgt, 1, ctx->work, beta + k);
    launch_lz_axpy(ctx->st, N3, 2, beta + k, w, nullptr, Q + (size_t)(k + 1) * N3);
    double hb[2];
    CK(cudaMemcpyAsync(hb, beta + k, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(hb + 1, alpha + k, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    TRY(sync(ctx, "lanczos"));
    if (!std::isfinite(hb[0]) || !std::isfinite(hb[1])) return fail(ctx, GW_E_NONFINITE, "non-finite Lanczos coefficient");
    if (hb[0] <= 1e-14 * std::fabs(hb[1])) return fail(ctx, GW_E_BREAKDOWN, "Lanczos breakdown: invariant subspace");
  }
  return launch_check(ctx, "lanczos");
}

// ---------------------------------------------------------------------------
// Block Lanczos on eps~(omega) (Sec. Lanczos, block form) on complex fields.
// Hermitian inner product at real omega, bilinear form sum_r x(r) y(r) at
// complex omega (eps~ is then complex symmetric).  Rows are vectors:
//   W = eps~(Q_k) - B'_{k-1} Q_{k-1};  A_k = <Q_k|W>;  W -= A_k^T Q_k
//   W -= H^T Q_all, H = <Q_all|W>   (twice: full re-orthogonalisation)
//   W = R^T Q_{k+1} with G = <W|W> = R^H R (Hermitian) or R^T R (bilinear)
// B' = conj(B) (Hermitian) or B (bilinear).  The block-sized factorisations run
// on the host in FP64 (blk <= 16); everything N_g-sized runs on the GPU.
// ---------------------------------------------------------------------------
using zcd = std::complex<double>;

// upper R with G = R^H R (herm) or G = R^T R (bilinear, principal square roots)
static bool chol_upper(const std::vector<zcd>& G, int b, bool bilinear, std::vector<zcd>* R) {
  R->assign((size_t)b * b, zcd(0, 0));
  auto r = [&](int i, int j) -> zcd& { return (*R)[(size_t)i * b + j]; };
  for (int i = 0; i < b; ++i) {
    zcd s = G[(size_t)i * b + i];
    for (int k = 0; k < i; ++k) s -= bilinear ? r(k, i) * r(k, i) : std::conj(r(k, i)) * r(k, i);
    if (bilinear) {
      if (!(std::abs(s) > 1e-300)) return false;
      r(i, i) = std::sqrt(s);
    } else {
      if (!(s.real() > 0.0)) return false;
      r(i, i) = std::sqrt(s.real());
    }
    for (int j = i + 1; j < b; ++j) {
      zcd t = G[(size_t)i * b + j];
      for (int k = 0; k < i; ++k) t -= bilinear ? r(k, i) * r(k, j) : std::conj(r(k, i)) * r(k, j);
      r(i, j) = t / r(i, i);
    }
  }
  return true;
}

// M = R^{-T} (rows of W R^{-1}), R upper triangular
static std::vector<zcd> inv_transpose_upper(const std::vector<zcd>& R, int b) {
  std::vector<zcd> inv((size_t)b * b, zcd(0, 0));   // inv = R^{-1}, upper
  for (int j = 0; j < b; ++j) {
    inv[(size_t)j * b + j] = 1.0 / R[(size_t)j * b + j];
    for (int i = j - 1; i >= 0; --i) {
      zcd s = 0.0;
      for (int k = i + 1; k <= j; ++k) s += R[(size_t)i * b + k] * inv[(size_t)k * b + j];
      inv[(size_t)i * b + j] = -s / R[(size_t)i * b + i];
    }
  }
  std::vector<zcd> M((size_t)b * b);
  for (int i = 0; i < b; ++i)
    for (int j = 0; j < b; ++j) M[(size_t)i * b + j] = inv[(size_t)j * b + i];
  return M;
}

// The block recursion on vectors of length n with inner-product weight wgt
// (Hermitian, or bilinear when bil), for any operator op(Qk, W) applied to blk
// rows: Q [K blk][n] receives the basis (Q_0 from the complex start block X0,
// which is overwritten), A/B the block coefficients, R0 (optional) the factor
// of the start block, X0 rows = sum_i R0[i][l] q_i.
template <class Op>
gw_status block_lanczos_run(gw_ctx* ctx, size_t n, double wgt, bool bil, int blk, int K, double2* X0, double2* Q,
                            Op op, std::vector<zcd>* Aout, std::vector<zcd>* Bout, std::vector<zcd>* R0) {
  const int cj = bil ? 0 : 1;
  const int mmax = K * blk;
  double2 *W, *gram, *part, *M;
  unsigned* cnt;
  TRY(getbuf(ctx, "bl_W", (size_t)blk * n, &W));
  TRY(getbuf(ctx, "bl_gram", (size_t)mmax * blk, &gram));
  TRY(getbuf(ctx, "bl_part", cgram_partials(n, mmax, blk), &part));
  TRY(getbuf(ctx, "bl_M", (size_t)blk * mmax, &M));
  TRY(getbuf(ctx, "bl_cnt", (size_t)(blk + 7) / 8 + 1, &cnt));
  CK(cudaMemsetAsync(cnt, 0, ((size_t)(blk + 7) / 8 + 1) * sizeof(unsigned), ctx->st));
  auto gram_host = [&](const double2* X, int mx, const double2* Y, std::vector<zcd>* out) -> gw_status {
    launch_cgram(ctx->st, X, mx, Y, blk, n, cj, wgt, part, cnt, gram);
    std::vector<double2> h((size_t)mx * blk);
    CK(cudaMemcpyAsync(h.data(), gram, h.size() * sizeof(double2), cudaMemcpyDeviceToHost, ctx->st));
    TRY(sync(ctx, "block gram"));
    out->resize(h.size());
    for (size_t i = 0; i < h.size(); ++i) (*out)[i] = zcd(h[i].x, h[i].y);
    return GW_OK;
  };
  auto combine = [&](const std::vector<zcd>& Mh, int my, int mx, const double2* X, double2* Y, int acc,
                     double sign) -> gw_status {
    std::vector<double2> h(Mh.size());
    for (size_t i = 0; i < h.size(); ++i) h[i] = make_double2(Mh[i].real(), Mh[i].imag());
    CK(cudaMemcpyAsync(M, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice, ctx->st));
    launch_cgemm_n(ctx->st, M, my, mx, X, n, Y, acc, sign);
    return launch_check(ctx, "block combine");
  };
  {
    std::vector<zcd> G, R;
    TRY(gram_host(X0, blk, X0, &G));
    if (!chol_upper(G, blk, bil, &R)) return fail(ctx, GW_E_BREAKDOWN, "start block is rank deficient");
    TRY(combine(inv_transpose_upper(R, blk), blk, blk, X0, Q, 0, 1.0));
    if (R0) *R0 = R;
  }
  Aout->assign((size_t)K * blk * blk, zcd(0, 0));
  Bout->assign((size_t)std::max(K - 1, 1) * blk * blk, zcd(0, 0));
  for (int k = 0; k < K; ++k) {
    double2* Qk = Q + (size_t)k * blk * n;
    TRY(op(Qk, W));
    if (k > 0) {
      std::vector<zcd> Bp(Bout->begin() + (size_t)(k - 1) * blk * blk, Bout->begin() + (size_t)k * blk * blk);
      if (!bil)
        for (auto& z : Bp) z = std::conj(z);
      TRY(combine(Bp, blk, blk, Q + (size_t)(k - 1) * blk * n, W, 1, -1.0));
    }
    std::vector<zcd> Ak;
    TRY(gram_host(Qk, blk, W, &Ak));
    std::vector<zcd> AkT((size_t)blk * blk);
    for (int i = 0; i < blk; ++i)
      for (int j = 0; j < blk; ++j) AkT[(size_t)j * blk + i] = Ak[(size_t)i * blk + j];
    TRY(combine(AkT, blk, blk, Qk, W, 1, -1.0));
    const int m = (k + 1) * blk;
    for (int pass = 0; pass < 2; ++pass) {
      std::vector<zcd> H, HT((size_t)blk * m);
      TRY(gram_host(Q, m, W, &H));
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < blk; ++j) HT[(size_t)j * m + i] = H[(size_t)i * blk + j];
      TRY(combine(HT, blk, m, Q, W, 1, -1.0));
    }
    std::copy(Ak.begin(), Ak.end(), Aout->begin() + (size_t)k * blk * blk);
    if (k == K - 1) break;
    std::vector<zcd> G, R;
    TRY(gram_host(W, blk, W, &G));
    if (!chol_upper(G, blk, bil, &R)) return fail(ctx, GW_E_BREAKDOWN, "block Lanczos breakdown (rank loss)");
    std::copy(R.begin(), R.end(), Bout->begin() + (size_t)k * blk * blk);
    TRY(combine(inv_transpose_upper(R, blk), blk, blk, W, Q + (size_t)(k + 1) * blk * n, 0, 1.0));
  }
  return launch_check(ctx, "block lanczos");
}

template <typename S>
gw_status block_lanczos_core(gw_ctx* ctx, const double* start, int blk, int K, double2 omega,
                             std::vector<zcd>* Aout, std::vector<zcd>* Bout, double2* Q) {
  const int N3 = ctx->N3;
  const size_t n = (size_t)N3;
  double2* X0;
  TRY(getbuf(ctx, "bl_X0", (size_t)blk * n, &X0));
  const size_t tot = (size_t)blk * n;
  ++g_launches;
  k_promote<<<(int)std::min<size_t>((tot + 255) / 256, 152 * 8), 256, 0, ctx->st>>>(tot, start, X0);
  const std::vector<double2> om(1, omega);
  auto op = [&](double2* Qk, double2* W) -> gw_status { return eps_core<S>(ctx, Qk, true, blk, om, W, false); };
  return block_lanczos_run(ctx, n, ctx->vol / N3, omega.y != 0.0, blk, K, X0, Q, op, Aout, Bout, nullptr);
}

// ---------------------------------------------------------------------------
// Derivative of s = <phi|eps~^-1(0)|phi> with respect to V_loc(r_i) (not in the
// paper; third-order perturbation theory, see include/gw.h):
//   Lanczos from phi -> T^-1, s = |phi|^2 (T^-1)_11, u = |phi| Q T^-1 e_1
//   w = v^1/2 u;  dpsi_v = -G_v P_c (w psi_v)          (Sternheimer solves)
//   g1 = sum |dpsi_v|^2 - sum S_vv' psi_v'* psi_v,  S = <dpsi|dpsi>
//   eta_v = P_c [w dpsi_v - sum_v' W_v'v dpsi_v'],  W = <psi|w|psi>
//   lambda_v = G_v eta_v                                (adjoint solves)
//   g2 = -sum_v lambda_v* psi_v;  grad = (Omega/N_g)(4 g1 + 8 Re g2)
// The occupied states are real in real space, so conj(u_v) = u_v and
// Re(lambda* u) = Re(lambda u).  Lanczos vectors are kept (checkpointed) and
// dpsi is recomputed from them rather than stored across the Lanczos run.
// ---------------------------------------------------------------------------
template <typename S>
gw_status grad_from_basis(gw_ctx* ctx, const double* phi, const double* Q, const double* a, const double* b, int K,
                          double* s_out, double* grad);

template <typename S>
gw_status grad_core(gw_ctx* ctx, const double* phi, int K, double* s_out, double* grad) {
  const int N3 = ctx->N3;
  TRY(ensure_work(ctx, std::max(K + 1, ctx->nocc * ctx->nocc)));
  // -- Lanczos from phi with the basis kept
  double *a, *b, *Q, *x0c;
  TRY(getbuf(ctx, "gr_alpha", K, &a));
  TRY(getbuf(ctx, "gr_beta", std::max(K - 1, 1), &b));
  TRY(getbuf(ctx, "gr_Q", (size_t)K * N3, &Q));
  TRY(getbuf(ctx, "gr_x0", N3, &x0c));
  CK(cudaMemcpyAsync(x0c, phi, (size_t)N3 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
  std::vector<double2> om(1, make_double2(0.0, 0.0));
  gw_status st = lanczos_core<S>(ctx, x0c, K, om, a, b, Q);
  if (st != GW_OK && st != GW_E_BREAKDOWN) return st;
  return grad_from_basis<S>(ctx, phi, Q, a, b, K, s_out, grad);
}

// The gradient from a kept Lanczos basis Q [K][N_g] of eps~(0) started at phi
// (alpha [K], beta [K-1] on the device): T^-1, s, u = |phi| Q T^-1 e_1, then
// the Sternheimer and adjoint solves (dpsi is computed here, never stored
// with the basis).
template <typename S>
gw_status grad_from_basis(gw_ctx* ctx, const double* phi, const double* Q, const double* a, const double* b, int K,
                          double* s_out, double* grad) {
  const int N3 = ctx->N3, npw = ctx->npw, nocc = ctx->nocc;
  const double vol = ctx->vol, wgt = vol / N3;
  const Geometry& g = ctx->geo;
  auto& P = ctx->P64;
  TRY(ensure_work(ctx, std::max(K + 1, nocc * nocc)));
  double *Ti, *d, *l, *u, *w, *h;
  int* stat;
  // -- T^-1 and s
  TRY(getbuf(ctx, "gr_Ti", (size_t)K * K, &Ti));
  TRY(getbuf(ctx, "gr_d", K, &d));
  TRY(getbuf(ctx, "gr_l", K, &l));
  TRY(getbuf(ctx, "gr_stat", 1, &stat));
  launch_tridiag_inv(ctx->st, K, a, b, d, l, Ti, stat);
  std::vector<double> t0(K);
  double pn2 = 0.0;
  {
    double* nrm;
    TRY(getbuf(ctx, "gr_nrm", 1, &nrm));
    launch_dot(ctx->st, N3, phi, phi, wgt, 0, ctx->work, nrm);
    CK(cudaMemcpyAsync(t0.data(), Ti, K * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));  // column 0
    CK(cudaMemcpyAsync(&pn2, nrm, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(ctx->host_pin, stat, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    TRY(sync(ctx, "grad T^-1"));
    if (ctx->host_pin[0]) return fail(ctx, GW_E_BREAKDOWN, "zero pivot in the tridiagonal inverse");
  }
  *s_out = pn2 * t0[0];
  // u = |phi| sum_k Q_k (T^-1)_k0
  std::vector<double> hm(K);
  for (int k = 0; k < K; ++k) hm[k] = -std::sqrt(pn2) * t0[k];
  TRY(upload(ctx, "gr_h", hm, &h));
  TRY(getbuf(ctx, "gr_u", N3, &u));
  TRY(getbuf(ctx, "gr_w", N3, &w));
  CK(cudaMemsetAsync(u, 0, (size_t)N3 * sizeof(double), ctx->st));
  launch_gemv_n(ctx->st, Q, N3, N3, h, K, u);
  TRY(sqrtv<double>(ctx, u, 1, w, nullptr));
  // -- first-order orbitals: (H - e_v) x_v = P_c(u_v w), dpsi_v = -x_v (sphere coefficients)
  std::vector<int> cv(nocc), cz(nocc, 0), src(nocc);
  std::vector<double2> E(nocc);
  for (int v = 0; v < nocc; ++v) { cv[v] = v; src[v] = v; E[v] = make_double2(ctx->eps[v], 0.0); }
  int *dcv, *dcz;
  double2* dE;
  TRY(upload(ctx, "gr_cv", cv, &dcv));
  TRY(upload(ctx, "gr_cz", cz, &dcz));
  TRY(upload(ctx, "gr_E", E, &dE));
  double* dtk = nullptr;
  if (ctx->precond) TRY(upload(ctx, "gr_tk", ctx->tkin, &dtk));
  double2 *grid, *rhs, *dC, *dU, *eta, *lam, *Sg, *Wm;
  TRY(getbuf(ctx, "gr_grid", (size_t)nocc * N3, &grid));
  TRY(getbuf(ctx, "gr_rhs", (size_t)nocc * npw, &rhs));
  TRY(getbuf(ctx, "gr_dC", (size_t)nocc * npw, &dC));
  TRY(getbuf(ctx, "gr_dU", (size_t)nocc * N3, &dU));
  TRY(getbuf(ctx, "gr_eta", (size_t)nocc * npw, &eta));
  TRY(getbuf(ctx, "gr_lam", (size_t)nocc * npw, &lam));
  TRY(getbuf(ctx, "gr_S", (size_t)nocc * nocc, &Sg));
  TRY(getbuf(ctx, "gr_W", (size_t)nocc * nocc, &Wm));
  auto sphere_of_product = [&](const double2* A, int a_conj, double2* out) {
    // out[v] = P_c Sphere(FFT(A_v w)) (twice projected)
    launch_xpass_prod_fwd<double>(ctx->st, g, P, ctx->plan, reinterpret_cast<const double2*>(w), 0, A, 0, a_conj,
                                  dcv, dcz, grid, nocc);
    launch_ypass<double>(ctx->st, 0, 0, 1, g, P, ctx->plan, grid, nullptr, nocc, 0);
    launch_zpass<double>(ctx->st, Z_GATHER_FWD, g, P, ctx->plan, grid, out, nullptr, nullptr, nullptr, nullptr,
                         nullptr, nullptr, nullptr, nocc);
  };
  sphere_of_product(P.U, 0, rhs);
  launch_proj<double>(ctx->st, P.C, nocc, npw, rhs, nocc, nullptr, ctx->work, nullptr, nullptr);
  launch_proj<double>(ctx->st, P.C, nocc, npw, rhs, nocc, nullptr, ctx->work, nullptr, nullptr);
  TRY(launch_check(ctx, "grad rhs"));
  TRY(solve<S>(ctx, nocc, rhs, dE, dC, false, dtk));
  // dC = -x  (dpsi coefficients); dU_v = IFFT(dC_v) on the grid
  {
    std::vector<int> one(nocc, -1);
    int* dnone;
    TRY(upload(ctx, "gr_none", one, &dnone));
    int* dsrc;
    TRY(upload(ctx, "gr_src", src, &dsrc));
    launch_combine(ctx->st, npw, nocc, dC, dsrc, dnone, 1.0, -1.0, dC);
  }
  launch_zpass<double>(ctx->st, Z_SCATTER_INV, g, P, ctx->plan, dU, dC, nullptr, nullptr, nullptr, nullptr, nullptr,
                       nullptr, nullptr, nocc);
  launch_ypass<double>(ctx->st, 1, 1, 0, g, P, ctx->plan, dU, nullptr, nocc, 0);
  launch_xpass_mul<double>(ctx->st, 1, 1, 0, g, P, ctx->plan, dU, nullptr, nullptr, nocc);
  // S = <dpsi|dpsi> (sphere), W = <psi|w|psi> (grid)
  launch_gram<double>(ctx->st, dC, nocc, npw, dC, nocc, ctx->work, Sg);
  launch_wmat(ctx->st, P.U, w, N3, nocc, ctx->work, Wm);
  // g1 on the grid
  double *g1, *g2;
  TRY(getbuf(ctx, "gr_g1", N3, &g1));
  TRY(getbuf(ctx, "gr_g2", N3, &g2));
  launch_g1(ctx->st, dU, P.U, Sg, N3, nocc, 1.0 / vol, g1);
  // eta_v = P_c [Sphere(FFT(w dU_v)) - sum_v' W[v'][v] dC_v']
  {
    std::vector<int> cself(nocc);
    for (int v = 0; v < nocc; ++v) cself[v] = v;
    int* dself;
    TRY(upload(ctx, "gr_cself", cself, &dself));
    launch_xpass_prod_fwd<double>(ctx->st, g, P, ctx->plan, reinterpret_cast<const double2*>(w), 0, dU, 1, 0, dself,
                                  dcz, grid, nocc);
    launch_ypass<double>(ctx->st, 0, 0, 1, g, P, ctx->plan, grid, nullptr, nocc, 0);
    launch_zpass<double>(ctx->st, Z_GATHER_FWD, g, P, ctx->plan, grid, eta, nullptr, nullptr, nullptr, nullptr,
                         nullptr, nullptr, nullptr, nocc);
    // eta_v -= sum_v' dC_v' W[v'][v]: the projector update with C := dC and coef[v' * ncol + v] = W[v'][v]
    launch_proj_update<double>(ctx->st, dC, nocc, npw, eta, nocc, nullptr, Wm, ctx->work, nullptr, nullptr);
    launch_proj<double>(ctx->st, P.C, nocc, npw, eta, nocc, nullptr, ctx->work, nullptr, nullptr);
    launch_proj<double>(ctx->st, P.C, nocc, npw, eta, nocc, nullptr, ctx->work, nullptr, nullptr);
  }
  TRY(launch_check(ctx, "grad eta"));
  TRY(solve<S>(ctx, nocc, eta, dE, lam, false, dtk));
  // Re g2 = -(1/Omega) Re sum_v lambda_v(r) u_v(r)
  launch_zpass<double>(ctx->st, Z_SCATTER_INV, g, P, ctx->plan, grid, lam, nullptr, nullptr, nullptr, nullptr,
                       nullptr, nullptr, nullptr, nocc);
  launch_ypass<double>(ctx->st, 1, 1, 0, g, P, ctx->plan, grid, nullptr, nocc, 0);
  {
    std::vector<int> gs(2);
    gs[0] = 0;
    gs[1] = nocc;
    int* dgs;
    TRY(upload(ctx, "gr_gs", gs, &dgs));
    launch_xpass_inv_reduce<double>(ctx->st, g, P, ctx->plan, grid, dgs, dcv, 1, -1.0 / vol, g2, nullptr, 0);
  }
  launch_grad_combine(ctx->st, N3, g1, g2, wgt, grad);
  return launch_check(ctx, "grad");
}

// host sphere, pencils, planes
gw_status build_geometry(gw_ctx* ctx) {
  const int N = ctx->N;
  const double gg = 2.0 * M_PI / ctx->L;
  std::vector<int> i2s, pen;
  std::vector<int4> pencils;
  std::vector<uint8_t> disc(N * N, 0), ones(N * N, 1), pmask(N, 0);
  int maxn = 0;
  for (int i0 = 0; i0 < N; ++i0)
    for (int i1 = 0; i1 < N; ++i1)
      for (int i2 = 0; i2 < N; ++i2) {
        const int n0 = (2 * i0 < N) ? i0 : i0 - N;
        const int n1 = (2 * i1 < N) ? i1 : i1 - N;
        const int n2 = (2 * i2 < N) ? i2 : i2 - N;
        const long nn = (long)n0 * n0 + (long)n1 * n1 + (long)n2 * n2;
        const double kin = 0.5 * (gg * gg) * (double)nn;
        if (kin <= ctx->ecut) {
          const int s = (int)ctx->sph_index.size();
          ctx->sph_index.push_back((i0 * N + i1) * N + i2);
          ctx->miller.push_back(n0);
          ctx->miller.push_back(n1);
          ctx->miller.push_back(n2);
          ctx->kin.push_back(kin);
          maxn = std::max(maxn, std::max(std::abs(n0), std::max(std::abs(n1), std::abs(n2))));
          if (pencils.empty() || pencils.back().x != i0 || pencils.back().y != i1)
            pencils.push_back(make_int4(i0, i1, s, 0));
          pencils.back().w += 1;
          i2s.push_back(i2);
          pen.push_back((int)pencils.size() - 1);
          disc[i0 * N + i1] = 1;
          pmask[i0] = 1;
        }
      }
  if (2 * maxn >= N) return fail(ctx, GW_E_ARG, "the plane-wave sphere does not fit in the FFT grid");
  ctx->npw = (int)ctx->kin.size();
  if (ctx->npw == 0) return fail(ctx, GW_E_ARG, "empty plane-wave sphere");
  std::vector<int> planes, allp(N);
  for (int i = 0; i < N; ++i) {
    allp[i] = i;
    if (pmask[i]) planes.push_back(i);
  }
  // first sphere entry / disc pencil of every plane (sphere order is i0-major)
  std::vector<int> plane_sph, plane_pen, i1s(ctx->npw);
  for (size_t pi = 0; pi < planes.size(); ++pi) {
    int s0 = -1, p0 = -1;
    for (size_t k = 0; k < pencils.size(); ++k)
      if (pencils[k].x == planes[pi]) { p0 = (int)k; s0 = pencils[k].z; break; }
    plane_sph.push_back(s0);
    plane_pen.push_back(p0);
  }
  plane_sph.push_back(ctx->npw);
  plane_pen.push_back((int)pencils.size());
  for (int s = 0; s < ctx->npw; ++s) i1s[s] = pencils[pen[s]].y;
  // sphere index of -G (the sphere is symmetric: 2 max|n| < N)
  std::vector<int> negs(ctx->npw, -1);
  {
    std::map<long, int> where;
    auto key = [&](int a, int b, int c) { return ((long)(a + N) * (2 * N + 1) + (b + N)) * (2 * N + 1) + (c + N); };
    for (int s = 0; s < ctx->npw; ++s)
      where[key(ctx->miller[3 * s], ctx->miller[3 * s + 1], ctx->miller[3 * s + 2])] = s;
    for (int s = 0; s < ctx->npw; ++s) {
      auto it = where.find(key(-ctx->miller[3 * s], -ctx->miller[3 * s + 1], -ctx->miller[3 * s + 2]));
      if (it == where.end()) return fail(ctx, GW_E_ARG, "sphere not symmetric");
      negs[s] = it->second;
    }
  }
  Geometry& g = ctx->geo;
  g.N = N; g.N2 = N * N; g.N3 = N * N * N; g.npw = ctx->npw;
  g.npen = (int)pencils.size();
  g.nplanes = (int)planes.size();
  TRY(upload(ctx, "geo_i2", i2s, &g.sph_i2));
  TRY(upload(ctx, "geo_pen", pen, &g.sph_pen));
  TRY(upload(ctx, "geo_pencils", pencils, &g.pencils));
  TRY(upload(ctx, "geo_disc", disc, &g.disc));
  TRY(upload(ctx, "geo_ones", ones, &g.ones));
  TRY(upload(ctx, "geo_planes", planes, &g.planes));
  TRY(upload(ctx, "geo_allp", allp, &g.all_planes));
  TRY(upload(ctx, "geo_pmask", pmask, &g.plane_mask));
  TRY(upload(ctx, "geo_plane_sph", plane_sph, &g.plane_sph));
  {
    // the plane holding -G of each plane's entries (i0 -> -i0 mod N)
    std::vector<int> mirror(planes.size(), -1);
    for (size_t pi = 0; pi < planes.size(); ++pi)
      for (size_t q = 0; q < planes.size(); ++q)
        if (planes[q] == (N - planes[pi]) % N) mirror[pi] = (int)q;
    for (size_t pi = 0; pi < planes.size(); ++pi)
      if (mirror[pi] < 0 || plane_sph[mirror[pi] + 1] - plane_sph[mirror[pi]] != plane_sph[pi + 1] - plane_sph[pi])
        return fail(ctx, GW_E_ARG, "sphere planes not symmetric");
    TRY(upload(ctx, "geo_plane_mirror", mirror, &g.plane_mirror));
  }
  ctx->maxplane = 0;
  for (size_t q = 0; q + 1 < plane_sph.size(); ++q) ctx->maxplane = std::max(ctx->maxplane, plane_sph[q + 1] - plane_sph[q]);
  TRY(upload(ctx, "geo_plane_pen", plane_pen, &g.plane_pen));
  TRY(upload(ctx, "geo_i1", i1s, &g.sph_i1));
  TRY(upload(ctx, "geo_neg", negs, &g.sph_neg));
  return GW_OK;
}

template <typename T>
gw_status upload_prec(gw_ctx* ctx, const std::vector<double>& vloc, const std::vector<double>& sqv) {
  const int N = ctx->N, N3 = ctx->N3;
  Prec<T>& P = prec_of<T>(ctx);
  const std::string t = tname<T>();
  std::vector<cpx<T>> tw(N);
  for (int k = 0; k < N; ++k) tw[k] = mk<T>((T)std::cos(2.0 * M_PI * k / N), (T)(-std::sin(2.0 * M_PI * k / N)));
  std::vector<T> kin(ctx->npw), vs(N3), sq(N3);
  for (int s = 0; s < ctx->npw; ++s) kin[s] = (T)ctx->kin[s];
  for (int r = 0; r < N3; ++r) {
    vs[r] = (T)(vloc[r] / (double)N3);
    sq[r] = (T)(sqv[r] / (double)N3);
  }
  TRY(upload(ctx, "p_tw" + t, tw, &P.tw));
  TRY(upload(ctx, "p_kin" + t, kin, &P.kin));
  TRY(upload(ctx, "p_v" + t, vs, &P.vloc_s));
  TRY(upload(ctx, "p_sqv" + t, sq, &P.sqv_s));
  return GW_OK;
}

// complex helpers on the host
using zc = std::complex<double>;

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
namespace {
// Real-in-real-space basis for a block of eigenstates (see the comments in
// the body); with prior rows given, the block is also made orthogonal to them.
// R receives the rows, e the energies (shell means inside degenerate shells).
gw_status realify_block(gw_ctx* ctx, int n_occ, const double* psi, const double* eps,
                        const std::vector<zc>* prior, int n_prior, std::vector<zc>* Rout,
                        std::vector<double>* eout, const char* what) {
  const int npw = ctx->npw, N = ctx->N;
  // index of -G for every sphere point
  std::map<long, int> where;
  auto key = [&](int a, int b, int c) { return ((long)(a + N) * (2 * N + 1) + (b + N)) * (2 * N + 1) + (c + N); };
  for (int s = 0; s < npw; ++s) where[key(ctx->miller[3 * s], ctx->miller[3 * s + 1], ctx->miller[3 * s + 2])] = s;
  std::vector<int> neg(npw);
  for (int s = 0; s < npw; ++s) {
    auto it = where.find(key(-ctx->miller[3 * s], -ctx->miller[3 * s + 1], -ctx->miller[3 * s + 2]));
    if (it == where.end()) return fail(ctx, GW_E_ARG, "sphere not symmetric");
    neg[s] = it->second;
  }
  // Real-in-real-space basis: (K c)_G = conj(c_{-G}), H K = K H.
  //  * a state that is K-symmetric up to a phase (|<c|Kc>| ~ 1: the usual,
  //    non-degenerate case) is multiplied by that phase and its K-symmetric
  //    part kept;
  //  * a degenerate shell (consecutive energies within 1e-6 Ha) whose states
  //    are mixed is re-spanned by the K-symmetric parts (c + Kc)/2 and
  //    (c - Kc)/2i, picked by pivoted Gram-Schmidt (inner products of
  //    K-symmetric vectors are real), energies set to the shell mean;
  //  * finally all states are re-orthonormalised (modified Gram-Schmidt).
  auto kdot = [&](const zc* c) {       // <c|Kc> = sum_G conj(c_G) conj(c_{-G})
    zc z = 0.0;
    for (int s = 0; s < npw; ++s) z += std::conj(c[s]) * std::conj(c[neg[s]]);
    return z;
  };
  std::vector<zc> C((size_t)n_occ * npw);
  for (size_t i = 0; i < C.size(); ++i) C[i] = zc(psi[2 * i], psi[2 * i + 1]);
  std::vector<zc> R((size_t)n_occ * npw);
  std::vector<double> e(n_occ);
  int v0 = 0;
  while (v0 < n_occ) {
    const zc z = kdot(&C[(size_t)v0 * npw]);
    if (std::abs(z) > 1.0 - 1e-3) {
      const zc ph = std::exp(zc(0.0, 0.5 * std::arg(z)));   // c = ph^-1 * (K-symmetric)
      zc* out = &R[(size_t)v0 * npw];
      for (int s = 0; s < npw; ++s) out[s] = ph * C[(size_t)v0 * npw + s];
      for (int s = 0; s < npw; ++s)
        if (neg[s] > s) {
          const zc a = 0.5 * (out[s] + std::conj(out[neg[s]]));
          out[s] = a;
          out[neg[s]] = std::conj(a);
        } else if (neg[s] == s) {
          out[s] = zc(out[s].real(), 0.0);
        }
      e[v0] = eps[v0];
      ++v0;
      continue;
    }
    int v1 = v0 + 1;
    while (v1 < n_occ && std::fabs(eps[v1] - eps[v1 - 1]) < 1e-6) ++v1;
    const int m = v1 - v0;
    std::vector<std::vector<zc>> cand;
    double norm0 = 0.0;
    for (int v = v0; v < v1; ++v) {
      std::vector<zc> a(npw), b(npw);
      for (int s = 0; s < npw; ++s) {
        const zc c = C[(size_t)v * npw + s], kc = std::conj(C[(size_t)v * npw + neg[s]]);
        a[s] = 0.5 * (c + kc);
        b[s] = (c - kc) / zc(0.0, 2.0);
        norm0 += std::norm(c);
      }
      cand.push_back(a);
      cand.push_back(b);
    }
    double mean = 0.0;
    for (int v = v0; v < v1; ++v) mean += eps[v];
    mean /= m;
    std::vector<bool> used(cand.size(), false);
    for (int k = 0; k < m; ++k) {
      int best = -1;
      double bn = -1.0;
      for (size_t j = 0; j < cand.size(); ++j) {
        if (used[j]) continue;
        double n2 = 0.0;
        for (int s = 0; s < npw; ++s) n2 += std::norm(cand[j][s]);
        if (n2 > bn) { bn = n2; best = (int)j; }
      }
      if (best < 0 || bn < 1e-8) return fail(ctx, GW_E_ARG, std::string(what) + " space is not closed under conjugation");
      used[best] = true;
      const double inv = 1.0 / std::sqrt(bn);
      for (int s = 0; s < npw; ++s) cand[best][s] *= inv;
      for (size_t j = 0; j < cand.size(); ++j) {
        if (used[j]) continue;
        zc d = 0.0;
        for (int s = 0; s < npw; ++s) d += std::conj(cand[best][s]) * cand[j][s];
        const double dr = d.real();
        for (int s = 0; s < npw; ++s) cand[j][s] -= dr * cand[best][s];
      }
      for (int s = 0; s < npw; ++s) R[(size_t)(v0 + k) * npw + s] = cand[best][s];
      e[v0 + k] = mean;
    }
    // what is left must be (numerically) inside the span of the shell
    for (size_t j = 0; j < cand.size(); ++j) {
      if (used[j]) continue;
      double n2 = 0.0;
      for (int s = 0; s < npw; ++s) n2 += std::norm(cand[j][s]);
      if (n2 > 1e-8 * norm0) return fail(ctx, GW_E_ARG, std::string(what) + " space is not closed under conjugation");
    }
    v0 = v1;
  }
  for (int v = 0; v < n_occ; ++v) {     // modified Gram-Schmidt, twice (real inner products)
    zc* a = &R[(size_t)v * npw];
    for (int u2 = 0; u2 < 2 * (v + n_prior); ++u2) {
      const int u = u2 % (v + n_prior);
      const zc* b = (u < n_prior) ? &(*prior)[(size_t)u * npw] : &R[(size_t)(u - n_prior) * npw];
      zc d = 0.0;
      for (int s = 0; s < npw; ++s) d += std::conj(b[s]) * a[s];
      const double dr = d.real();
      for (int s = 0; s < npw; ++s) a[s] -= dr * b[s];
    }
    double n2 = 0.0;
    for (int s = 0; s < npw; ++s) n2 += std::norm(a[s]);
    if (!(n2 > 0.5)) return fail(ctx, GW_E_ARG, std::string(what) + " states are not orthonormal");
    const double inv = 1.0 / std::sqrt(n2);
    for (int s = 0; s < npw; ++s) a[s] *= inv;
  }
  // exact K-symmetry of every row (c_{-G} = conj c_G to the last bit), so that
  // solver vectors built from these rows stay exactly real in real space
  for (int v = 0; v < n_occ; ++v) {
    zc* a = &R[(size_t)v * npw];
    for (int s = 0; s < npw; ++s) {
      if (neg[s] > s) {
        const zc h = 0.5 * (a[s] + std::conj(a[neg[s]]));
        a[s] = h;
        a[neg[s]] = std::conj(h);
      } else if (neg[s] == s) {
        a[s] = zc(a[s].real(), 0.0);
      }
    }
  }
  *Rout = std::move(R);
  *eout = std::move(e);
  return GW_OK;
}

// C on the device (FP64 and FP32): the occupied rows, then the deflation rows.
gw_status upload_projector(gw_ctx* ctx, const std::vector<zc>& cdef) {
  const size_t n = ctx->c_occ.size() + cdef.size();
  std::vector<double2> c64(n);
  std::vector<float2> c32(n);
  for (size_t i = 0; i < n; ++i) {
    const zc z = (i < ctx->c_occ.size()) ? ctx->c_occ[i] : cdef[i - ctx->c_occ.size()];
    c64[i] = make_double2(z.real(), z.imag());
    c32[i] = make_float2((float)z.real(), (float)z.imag());
  }
  TRY(upload(ctx, "occ_C64", c64, &ctx->P64.C));
  TRY(upload(ctx, "occ_C32", c32, &ctx->P32.C));
  // the rows split into TF32 hi / lo parts for the tensor-core projector
  // coefficients (up to 64 rows); without a tensor-map encoder the CUDA-core
  // dots remain
  ctx->tc_ok = false;
  const int rows = (int)(n / std::max(ctx->npw, 1));
  if (rows >= 1 && rows <= 64 && tc_prepare() == cudaSuccess) {
    std::vector<float> hi, lo;
    tc_split_rows(c64, rows, ctx->npw, &hi, &lo);
    float *dhi, *dlo;
    TRY(upload(ctx, "tc_Ahi", hi, &dhi));
    TRY(upload(ctx, "tc_Alo", lo, &dlo));
    ctx->tc_ok = (tc_maps(dhi, dlo, ctx->npw, &ctx->tc_maps) == cudaSuccess);
  }
  cudaGetLastError();
  return GW_OK;
}

}  // namespace

// Eq. recy_eq: <l|eps~(i w) - 1|l'> = 4 sum_v <b_{l,v}|A_v^-1(i w)|b_{l',v}> with A_v^-1
// applied in the recycled basis of state v (the static solutions x(0) and the
// high-frequency directions x(i inf) = P_c (H - e_v) b, orthonormalised through
// the eigendecomposition of their Gram matrix).  F [nl][N_g] real fields on
// the device; out [nw][nl][nl] on the device.
template <typename S>
gw_status recycle_core(gw_ctx* ctx, const double* F, int nl, const double* dw, int nw, double rtol, double* out,
                       int* kept_min) {
  const int npw = ctx->npw, nocc = ctx->nocc, N3 = ctx->N3;
  const double w0 = ctx->recycle_w0;                 // > 0: x(i w0) joins the basis
  const int nblk = (w0 > 0.0) ? 3 : 2;
  const int m = nblk * nl, nc = nl * nocc, nx = nocc * m;
  auto& P = ctx->P64;
  // right-hand sides b[l * nocc + v]
  double* y;
  TRY(getbuf(ctx, "rc_y", (size_t)nl * N3, &y));
  TRY(sqrtv<double>(ctx, F, nl, y, nullptr));
  double2* b;
  TRY(rhs_core(ctx, y, false, nl, &b));
  double2* bcp;
  TRY(getbuf(ctx, "rc_b", (size_t)nc * npw, &bcp));
  CK(cudaMemcpyAsync(bcp, b, (size_t)nc * npw * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->st));
  // x(0) (rows 0 .. nc-1 of xc) and x(i inf) (rows nc .. 2 nc - 1)
  std::vector<double2> E(nc);
  std::vector<double> tk(nc);
  for (int j = 0; j < nc; ++j) {
    E[j] = make_double2(ctx->eps[j % nocc], 0.0);
    tk[j] = ctx->tkin[j % nocc];
  }
  double2* dE;
  double* dtk = nullptr;
  TRY(upload_table(ctx, "rc_E", E, &dE));
  if (ctx->precond) TRY(upload_table(ctx, "rc_tk", tk, &dtk));
  double2* xc;
  TRY(getbuf(ctx, "rc_x", (size_t)nblk * nc * npw, &xc));
  for (int j0 = 0; j0 < nc; j0 += kPersistentMaxCols) {
    const int nj = std::min(kPersistentMaxCols, nc - j0);
    TRY(solve<S>(ctx, nj, bcp + (size_t)j0 * npw, dE + j0, xc + (size_t)j0 * npw, false, dtk ? dtk + j0 : nullptr));
  }
  TRY(h_apply<double>(ctx, bcp, nc, dE, nullptr, xc + (size_t)nc * npw));
  TRY(ensure_work(ctx, std::max(nx, nc)));
  launch_proj<double>(ctx->st, P.C, nocc, npw, xc + (size_t)nc * npw, nc, nullptr, ctx->work, nullptr, nullptr);
  if (w0 > 0.0) {
    // x(i w0) = ((H - e_v)^2 + w0^2)^-1 (H - e_v) b (Eq. P2+), the right-hand
    // side being the high-frequency rows P_c (H - e_v) b just computed
    std::vector<double> w2(nc, w0 * w0);
    double* dw2;
    TRY(upload_table(ctx, "rc_w2", w2, &dw2));
    double2* rhs_sq;
    TRY(getbuf(ctx, "rc_rsq", (size_t)nc * npw, &rhs_sq));
    CK(cudaMemcpyAsync(rhs_sq, xc + (size_t)nc * npw, (size_t)nc * npw * sizeof(double2), cudaMemcpyDeviceToDevice,
                       ctx->st));
    for (int j0 = 0; j0 < nc; j0 += kPersistentMaxCols) {
      const int nj = std::min(kPersistentMaxCols, nc - j0);
      TRY(solve<S>(ctx, nj, rhs_sq + (size_t)j0 * npw, dE + j0, xc + (size_t)(2 * nc + j0) * npw, false,
                   dtk ? dtk + j0 : nullptr, dw2 + j0, w0 * w0));
    }
  }
  // per state v: X_v rows [x_{l,v}(0); x_{l,v}(i inf); x_{l,v}(i w0)] normalised, and b_v rows
  std::vector<int> ix(nx), ib(nc), vrow(nx);
  for (int v = 0; v < nocc; ++v)
    for (int i = 0; i < m; ++i) {
      ix[v * m + i] = (i / nl) * nc + (i % nl) * nocc + v;
      vrow[v * m + i] = v;
    }
  for (int v = 0; v < nocc; ++v)
    for (int l = 0; l < nl; ++l) ib[v * nl + l] = l * nocc + v;
  int *dix, *dib;
  TRY(upload_table(ctx, "rc_ix", ix, &dix));
  TRY(upload_table(ctx, "rc_ib", ib, &dib));
  double2 *X, *HX, *B;
  TRY(getbuf(ctx, "rc_X", (size_t)nx * npw, &X));
  TRY(getbuf(ctx, "rc_HX", (size_t)nx * npw, &HX));
  TRY(getbuf(ctx, "rc_B", (size_t)nc * npw, &B));
  launch_gather_rows<double, double>(ctx->st, npw, nx, xc, dix, X);
  launch_gather_rows<double, double>(ctx->st, npw, nc, bcp, dib, B);
  launch_normalize_rows(ctx->st, X, nx, npw);
  std::vector<double2> Ex(nx);
  for (int j = 0; j < nx; ++j) Ex[j] = make_double2(ctx->eps[vrow[j]], 0.0);
  double2* dEx;
  TRY(upload_table(ctx, "rc_Ex", Ex, &dEx));
  TRY(h_apply<double>(ctx, X, nx, dEx, nullptr, HX));
  // Gram, Hamiltonian and right-hand-side matrices of every state (real: the
  // fields and the occupied states are real in real space)
  double2 *cg, *gpart;
  unsigned* gcnt;
  TRY(getbuf(ctx, "rc_cg", (size_t)m * m, &cg));
  TRY(getbuf(ctx, "rc_gpart", std::max(cgram_partials(npw, m, m), cgram_partials(npw, m, nl)), &gpart));
  if (!ctx->bufs.count("rc_gcnt") || ctx->bufs["rc_gcnt"].second < (size_t)m * sizeof(unsigned)) {
    TRY(getbuf(ctx, "rc_gcnt", (size_t)m, &gcnt));
    CK(cudaMemsetAsync(gcnt, 0, (size_t)m * sizeof(unsigned), ctx->st));
  } else {
    TRY(getbuf(ctx, "rc_gcnt", (size_t)m, &gcnt));
  }
  double *Sm, *Hm, *Bm, *W, *T, *Hg, *Bg, *U, *C, *tmp;
  const size_t mm = (size_t)m * m, mb = (size_t)m * nl;
  TRY(getbuf(ctx, "rc_S", nocc * mm, &Sm));
  TRY(getbuf(ctx, "rc_H", nocc * mm, &Hm));
  TRY(getbuf(ctx, "rc_Bm", nocc * mb, &Bm));
  TRY(getbuf(ctx, "rc_W", nocc * mm, &W));
  TRY(getbuf(ctx, "rc_T", nocc * mm, &T));
  TRY(getbuf(ctx, "rc_Hg", nocc * mm, &Hg));
  TRY(getbuf(ctx, "rc_Bg", nocc * mb, &Bg));
  TRY(getbuf(ctx, "rc_U", nocc * mm, &U));
  TRY(getbuf(ctx, "rc_C", nocc * mb, &C));
  TRY(getbuf(ctx, "rc_tmp", nocc * mm, &tmp));
  for (int v = 0; v < nocc; ++v) {
    const double2* Xv = X + (size_t)v * m * npw;
    launch_cgram(ctx->st, Xv, m, Xv, m, npw, 1, 1.0, gpart, gcnt, cg);
    launch_real_part(ctx->st, mm, cg, Sm + v * mm);
    launch_cgram(ctx->st, Xv, m, HX + (size_t)v * m * npw, m, npw, 1, 1.0, gpart, gcnt, cg);
    launch_real_part(ctx->st, mm, cg, Hm + v * mm);
    launch_cgram(ctx->st, Xv, m, B + (size_t)v * nl * npw, nl, npw, 1, 1.0, gpart, gcnt, cg);
    launch_real_part(ctx->st, mb, cg, Bm + v * mb);
  }
  launch_symmetrize(ctx->st, nocc, m, Sm);
  launch_symmetrize(ctx->st, nocc, m, Hm);
  int *sweeps, *kept;
  TRY(getbuf(ctx, "rc_sweeps", (size_t)2 * nocc, &sweeps));
  TRY(getbuf(ctx, "rc_kept", (size_t)nocc, &kept));
  constexpr int kSweeps = 40;
  CK(launch_jacobi_sym(ctx->st, nocc, m, Sm, W, 1e-14, kSweeps, sweeps));
  launch_orth_transform(ctx->st, nocc, m, Sm, W, rtol * rtol, T, kept);
  // H_gamma = T^T H T, b_gamma = T^T B; eigenvectors U of H_gamma; c = U^T b_gamma
  launch_gemm_small(ctx->st, nocc, m, m, m, Hm, 0, T, 0, tmp);
  launch_gemm_small(ctx->st, nocc, m, m, m, T, 1, tmp, 0, Hg);
  launch_gemm_small(ctx->st, nocc, m, m, nl, T, 1, Bm, 0, Bg);
  launch_symmetrize(ctx->st, nocc, m, Hg);
  CK(launch_jacobi_sym(ctx->st, nocc, m, Hg, U, 1e-14, kSweeps, sweeps + nocc));
  launch_gemm_small(ctx->st, nocc, m, m, nl, U, 1, Bg, 0, C);
  launch_recycled_form(ctx->st, nocc, m, nl, nw, Hg, C, dw, out);
  TRY(launch_check(ctx, "recycle"));
  std::vector<int> hs(2 * nocc), hk(nocc);
  CK(cudaMemcpyAsync(hs.data(), sweeps, 2 * nocc * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(hk.data(), kept, nocc * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  TRY(sync(ctx, "recycle"));
  for (int v = 0; v < 2 * nocc; ++v)
    if (hs[v] > kSweeps) return fail(ctx, GW_E_NOCONV, "Jacobi eigensolver did not converge in the recycled basis");
  *kept_min = *std::min_element(hk.begin(), hk.end());
  return GW_OK;
}

// Eq. pe for candidate states given on the device (psi_e [N_PW], psi [n][N_PW]
// complex) with host energies and occupations; *total and (*terms)[n] out.
gw_status sigma_p_core(gw_ctx* ctx, const double2* psi_e, double eps_e, double delta, int n, const double2* psi,
                       const std::vector<double>& he, const std::vector<int>& ho, int k, gw_prec prec,
                       double* total_out, std::vector<double>* terms) {
  const int npw = ctx->npw, N3 = ctx->N3;
  const double wgt = ctx->vol / N3;
  // the poles that Theta keeps, with their weights -Theta(w) (occupied) or Theta(-w)
  std::vector<int> pole;
  std::vector<double> pw_, pom;
  for (int j = 0; j < n; ++j) {
    if (!std::isfinite(he[j])) return fail(ctx, GW_E_NONFINITE, "non-finite energy");
    const double om = he[j] - eps_e - delta;
    const double th = ho[j] ? (om > 0 ? 1.0 : (om == 0 ? 0.5 : 0.0)) : (om < 0 ? 1.0 : (om == 0 ? 0.5 : 0.0));
    if (th == 0.0) continue;
    pole.push_back(j);
    pw_.push_back(ho[j] ? -th : th);
    pom.push_back(om);
  }
  std::vector<double>& hterms = *terms;
  hterms.assign(n, 0.0);
  double total = 0.0;
  const int np = (int)pole.size();
  if (np > 0) {
    // grids u_e and u_p of the states (sphere -> grid, FP64), then the pair products
    const double2* pe = psi_e;
    const double2* pp = psi;
    double2 *cs, *ug;
    double *seeds, *al, *be, *Q, *n2, *Ti, *d, *l;
    int* stat;
    TRY(getbuf(ctx, "sgp_cs", (size_t)(np + 1) * npw, &cs));
    TRY(getbuf(ctx, "sgp_ug", (size_t)(np + 1) * N3, &ug));
    for (int i = 0; i < np; ++i)
      CK(cudaMemcpyAsync(cs + (size_t)i * npw, pp + (size_t)pole[i] * npw,
                         npw * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaMemcpyAsync(cs + (size_t)np * npw, pe, npw * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->st));
    const Geometry& g = ctx->geo;
    launch_zpass<double>(ctx->st, Z_SCATTER_INV, g, ctx->P64, ctx->plan, ug, cs, nullptr, nullptr, nullptr, nullptr,
                         nullptr, nullptr, nullptr, np + 1);
    launch_ypass<double>(ctx->st, 1, 1, 0, g, ctx->P64, ctx->plan, ug, nullptr, np + 1, 0);
    launch_xpass_mul<double>(ctx->st, 1, 1, 0, g, ctx->P64, ctx->plan, ug, nullptr, nullptr, np + 1);
    double* prod;
    TRY(getbuf(ctx, "sgp_prod", (size_t)2 * np * N3, &prod));
    {
      const size_t nn = (size_t)np * N3;
      ++g_launches;
      k_pair_product<<<(int)std::min<size_t>((nn + 255) / 256, 152 * 8), 256, 0, ctx->st>>>(
          (size_t)N3, np, ug, ug + (size_t)np * N3, 1.0 / ctx->vol, prod);
    }
    // phi = v^1/2 |p* e> (real and imaginary parts as real fields), [np][2][N3]
    TRY(getbuf(ctx, "sgp_seeds", (size_t)2 * np * N3, &seeds));
    TRY(sqrtv<double>(ctx, prod, 2 * np, seeds, nullptr));
    TRY(getbuf(ctx, "sgp_n2", 2 * np, &n2));
    TRY(ensure_work(ctx, 64));
    for (int j = 0; j < 2 * np; ++j)
      launch_dot(ctx->st, N3, seeds + (size_t)j * N3, seeds + (size_t)j * N3, wgt, 0, ctx->work, n2 + j);
    std::vector<double> hn2(2 * np);
    CK(cudaMemcpyAsync(hn2.data(), n2, 2 * np * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    TRY(sync(ctx, "sigma_p seeds"));
    TRY(getbuf(ctx, "sgp_al", k, &al));
    TRY(getbuf(ctx, "sgp_be", k, &be));
    TRY(getbuf(ctx, "sgp_Q", (size_t)2 * k * N3, &Q));
    TRY(getbuf(ctx, "sgp_Ti", (size_t)k * k, &Ti));
    TRY(getbuf(ctx, "sgp_d", k, &d));
    TRY(getbuf(ctx, "sgp_l", k, &l));
    TRY(getbuf(ctx, "sgp_stat", 1, &stat));
    double* x0;
    TRY(getbuf(ctx, "sgp_x0", (size_t)2 * N3, &x0));
    for (int i = 0; i < np; ++i) {
      const double nr = hn2[2 * i], ni = hn2[2 * i + 1];
      const double nt = nr + ni;
      if (!(nt > 0.0)) continue;                       // a vanishing seed: the term is 0
      // a real seed (states real in real space) runs on N_g entries, a complex one on 2 N_g
      const bool cplx = ni > 1e-24 * nt;
      const double* src = seeds + (size_t)(2 * i + (cplx || nr > 0.0 ? 0 : 1)) * N3;
      const int width = cplx ? 2 : 1;
      CK(cudaMemcpyAsync(x0, src, (size_t)width * N3 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
      const std::vector<double2> om{make_double2(pom[i], 0.0)};
      int steps = 0;
      gw_status st = (prec == GW_FP64) ? lanczos_core<double>(ctx, x0, k, om, al, be, Q, width, &steps)
                                       : lanczos_core<float>(ctx, x0, k, om, al, be, Q, width, &steps);
      if (st != GW_OK && st != GW_E_BREAKDOWN) return st;
      ctx->err.clear();
      launch_tridiag_inv(ctx->st, steps, al, be, d, l, Ti, stat);
      double t11 = 0.0;
      int hs = 0;
      CK(cudaMemcpyAsync(&t11, Ti, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
      CK(cudaMemcpyAsync(&hs, stat, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
      TRY(sync(ctx, "sigma_p element"));
      if (hs) return fail(ctx, GW_E_BREAKDOWN, "singular Lanczos matrix in a Sigma^P element");
      hterms[pole[i]] = pw_[i] * (cplx ? nt : (nr > 0.0 ? nr : ni)) * (t11 - 1.0);
    }
    for (int j = 0; j < n; ++j) total += hterms[j];
  }
  *total_out = total;
  return GW_OK;
}

// Gauss-Legendre nodes (ascending) and weights on [-1, 1]: Newton iteration on
// P_n from the three-term recurrence, P_n'(x) = n (x P_n - P_{n-1}) / (x^2 - 1).
static void gauss_legendre(int n, std::vector<double>* t, std::vector<double>* w) {
  t->assign(n, 0.0);
  w->assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double x = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
      const double dx = p1 / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= n; ++k) {
      const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = (n == 1) ? 1.0 : n * (x * p1 - p0) / (x * x - 1.0);
    (*t)[n - 1 - i] = x;
    (*w)[n - 1 - i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
}

// Eq. e_c in the basis of the fields F (see gw_sigma_c in include/gw.h):
// out = {Sigma^c, frequency integral, Sigma^A, Sigma^P}.
template <typename S>
gw_status sigma_c_core(gw_ctx* ctx, int e, double delta, double alpha, int nf, const double* F, int nl, int kh,
                       int kp, gw_prec prec, double* out) {
  const int npw = ctx->npw, nocc = ctx->nocc, N3 = ctx->N3;
  const double c = ctx->eps[e] + delta;
  const double pi = 3.14159265358979323846;
  // frequency nodes w = (1 + t)/(1 - t) with weights of (1/pi) int_0^inf dw
  std::vector<double> t, wt, wall(1, 0.0), Wt(nf);
  gauss_legendre(nf, &t, &wt);
  for (int i = 0; i < nf; ++i) {
    wall.push_back((1.0 + t[i]) / (1.0 - t[i]));
    Wt[i] = wt[i] * 2.0 / ((1.0 - t[i]) * (1.0 - t[i])) / pi;
  }
  double* dw;
  TRY(upload_table(ctx, "sc_w", wall, &dw));
  // M(i w) = (1 + E(i w))^-1 - 1 in the basis, E from the recycled bases
  double *E, *V, *M;
  int* sw;
  const size_t nn = (size_t)nl * nl;
  TRY(getbuf(ctx, "sc_E", (nf + 1) * nn, &E));
  TRY(getbuf(ctx, "sc_V", (nf + 1) * nn, &V));
  TRY(getbuf(ctx, "sc_M", (nf + 1) * nn, &M));
  TRY(getbuf(ctx, "sc_sw", (size_t)nf + 2, &sw));
  int kept = 0;
  TRY(recycle_core<S>(ctx, F, nl, dw, nf + 1, 1e-6, E, &kept));
  launch_add_identity(ctx->st, nf + 1, nl, E);
  launch_symmetrize(ctx->st, nf + 1, nl, E);
  CK(launch_jacobi_sym(ctx->st, nf + 1, nl, E, V, 1e-14, 40, sw));
  launch_eig_function(ctx->st, nf + 1, nl, E, V, 0, M);
  // z_l = Sphere(u_e (v^1/2 F_l)): the phase-space vectors Phi_e v^1/2 |l*>
  double* y;
  TRY(getbuf(ctx, "sc_y", (size_t)nl * N3, &y));
  TRY(sqrtv<double>(ctx, F, nl, y, nullptr));
  std::vector<int> ca(nl, e), cy(nl);
  for (int l = 0; l < nl; ++l) cy[l] = l;
  int *dca, *dcy;
  TRY(upload_table(ctx, "sc_ca", ca, &dca));
  TRY(upload_table(ctx, "sc_cy", cy, &dcy));
  double2 *grid, *Z, *X0, *Qh;
  TRY(getbuf(ctx, "sc_grid", (size_t)nl * N3, &grid));
  TRY(getbuf(ctx, "sc_Z", (size_t)nl * npw, &Z));
  TRY(getbuf(ctx, "sc_X0", (size_t)nl * npw, &X0));
  TRY(getbuf(ctx, "sc_Q", (size_t)kh * nl * npw, &Qh));
  const Geometry& g = ctx->geo;
  launch_xpass_prod_fwd<double>(ctx->st, g, ctx->P64, ctx->plan, reinterpret_cast<const double2*>(y), 0,
                                ctx->P64.U, 0, 0, dca, dcy, grid, nl);
  launch_ypass<double>(ctx->st, 0, 0, 1, g, ctx->P64, ctx->plan, grid, nullptr, nl, 0);
  launch_zpass<double>(ctx->st, Z_GATHER_FWD, g, ctx->P64, ctx->plan, grid, Z, nullptr, nullptr, nullptr, nullptr,
                       nullptr, nullptr, nullptr, nl);
  CK(cudaMemcpyAsync(X0, Z, (size_t)nl * npw * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->st));
  // shift-Lanczos: one block recursion on H - c serves every frequency
  std::vector<double2> Ec(nl, make_double2(c, 0.0));
  double2* dEc;
  TRY(upload_table(ctx, "sc_Ec", Ec, &dEc));
  auto op = [&](double2* Qk, double2* W) -> gw_status { return h_apply<double>(ctx, Qk, nl, dEc, nullptr, W); };
  std::vector<zcd> Ah, Bh, R0;
  TRY(block_lanczos_run(ctx, (size_t)npw, 1.0, false, nl, kh, X0, Qh, op, &Ah, &Bh, &R0));
  const int m = kh * nl;
  std::vector<double> T((size_t)m * m, 0.0), R(nn);
  for (int k = 0; k < kh; ++k)
    for (int i = 0; i < nl; ++i)
      for (int j = 0; j < nl; ++j) {
        T[(size_t)(k * nl + i) * m + k * nl + j] = Ah[(size_t)k * nn + i * nl + j].real();
        if (k + 1 < kh) {
          const double b = Bh[(size_t)k * nn + i * nl + j].real();
          T[(size_t)((k + 1) * nl + i) * m + k * nl + j] = b;
          T[(size_t)(k * nl + j) * m + (k + 1) * nl + i] = b;
        }
      }
  for (size_t i = 0; i < nn; ++i) R[i] = R0[i].real();
  double *dT, *dU, *dR, *G, *K;
  TRY(upload(ctx, "sc_T", T, &dT));
  TRY(upload(ctx, "sc_R", R, &dR));
  TRY(getbuf(ctx, "sc_U", (size_t)m * m, &dU));
  TRY(getbuf(ctx, "sc_G", (size_t)nf * nn, &G));
  TRY(getbuf(ctx, "sc_K", (size_t)nf * nn, &K));
  launch_symmetrize(ctx->st, 1, m, dT);
  CK(launch_jacobi_sym(ctx->st, 1, m, dT, dU, 1e-14, 40, sw + nf + 1));
  launch_shift_quadrature(ctx->st, m, nl, dT, dU, dR, dw + 1, nf, G, K);
  // Sigma^A: h+ = alpha (H - c + alpha)^-1 P_c z in the conduction space; P_e part in closed form
  double2 *bz, *hp, *cg, *gpart, *a;
  unsigned* gcnt;
  TRY(getbuf(ctx, "sc_bz", (size_t)nl * npw, &bz));
  TRY(getbuf(ctx, "sc_hp", (size_t)nl * npw, &hp));
  CK(cudaMemcpyAsync(bz, Z, (size_t)nl * npw * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->st));
  TRY(ensure_work(ctx, std::max(nl, 64)));
  launch_proj<double>(ctx->st, ctx->P64.C, nocc, npw, bz, nl, nullptr, ctx->work, nullptr, nullptr);
  std::vector<double2> Ea(nl, make_double2(c - alpha, 0.0));
  std::vector<double> tk(nl, ctx->tkin[e]);
  double2* dEa;
  double* dtk = nullptr;
  TRY(upload_table(ctx, "sc_Ea", Ea, &dEa));
  if (ctx->precond) TRY(upload_table(ctx, "sc_tk", tk, &dtk));
  TRY(solve<S>(ctx, nl, bz, dEa, hp, false, dtk));
  double *Hp, *Hm, *deps, *forms;
  TRY(getbuf(ctx, "sc_cg", nn, &cg));
  TRY(getbuf(ctx, "sc_gpart", cgram_partials(npw, nl, nl), &gpart));
  if (!ctx->bufs.count("sc_gcnt") || ctx->bufs["sc_gcnt"].second < (size_t)nl * sizeof(unsigned)) {
    TRY(getbuf(ctx, "sc_gcnt", (size_t)nl, &gcnt));
    CK(cudaMemsetAsync(gcnt, 0, (size_t)nl * sizeof(unsigned), ctx->st));
  } else {
    TRY(getbuf(ctx, "sc_gcnt", (size_t)nl, &gcnt));
  }
  TRY(getbuf(ctx, "sc_Hp", nn, &Hp));
  TRY(getbuf(ctx, "sc_Hm", nn, &Hm));
  TRY(getbuf(ctx, "sc_a", (size_t)nocc * nl, &a));
  launch_cgram(ctx->st, Z, nl, hp, nl, npw, 1, alpha, gpart, gcnt, cg);
  launch_real_part(ctx->st, nn, cg, Hp);
  launch_gram<double>(ctx->st, ctx->P64.C, nocc, npw, Z, nl, ctx->work, a);
  TRY(upload(ctx, "sc_eps", ctx->eps, &deps));
  launch_pe_form(ctx->st, nocc, nl, a, deps, c, alpha, Hm);
  // Frobenius forms: node i: (M(i w_i) - f(w_i) M(0)) . K_i; then M(0) . Hp and M(0) . Hm
  std::vector<int> ia(nf + 2), ib(nf + 2, 0), ic(nf + 2);
  std::vector<double> fa(nf + 2, 0.0);
  for (int i = 0; i < nf; ++i) {
    ia[i] = 1 + i;
    ic[i] = i;
    fa[i] = alpha * alpha / (wall[1 + i] * wall[1 + i] + alpha * alpha);
  }
  int *dia, *dib, *dic;
  double* dfa;
  TRY(upload_table(ctx, "sc_ia", ia, &dia));
  TRY(upload_table(ctx, "sc_ib", ib, &dib));
  TRY(upload_table(ctx, "sc_ic", ic, &dic));
  TRY(upload_table(ctx, "sc_fa", fa, &dfa));
  TRY(getbuf(ctx, "sc_forms", (size_t)nf + 2, &forms));
  launch_frob_forms(ctx->st, nf, (int)nn, M, dia, dfa, M, dib, K, dic, forms);
  launch_frob_forms(ctx->st, 1, (int)nn, M, dib, dfa + nf, M, dib, Hp, dib, forms + nf);
  launch_frob_forms(ctx->st, 1, (int)nn, M, dib, dfa + nf, M, dib, Hm, dib, forms + nf + 1);
  std::vector<double> hf(nf + 2);
  std::vector<int> hsw(nf + 2);
  CK(cudaMemcpyAsync(hf.data(), forms, (nf + 2) * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(hsw.data(), sw, (nf + 2) * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  TRY(sync(ctx, "sigma_c"));
  for (int x : hsw)
    if (x > 40) return fail(ctx, GW_E_NOCONV, "Jacobi eigensolver did not converge in the self-energy");
  double integral = 0.0;
  for (int i = 0; i < nf; ++i) integral += Wt[i] * hf[i];
  const double SA = 0.5 * (hf[nf] + hf[nf + 1]);
  // Sigma^P: occupied states at or above c (w_ve >= 0); e_HOMO <= c leaves only e_v = c
  const std::vector<int> ho(nocc, 1);
  double SP = 0.0;
  std::vector<double> terms;
  TRY(sigma_p_core(ctx, ctx->P64.C + (size_t)e * npw, ctx->eps[e], delta, nocc, ctx->P64.C, ctx->eps, ho, kp, prec,
                   &SP, &terms));
  out[0] = integral + SA + SP;
  out[1] = integral;
  out[2] = SA;
  out[3] = SP;
  (void)kept;
  return GW_OK;
}

extern "C" {

gw_status gw_setup(gw_ctx** out, double L, int n_grid, double ecut, const double* vloc, int coulomb,
                   void* cuda_stream) {
  if (!out) return GW_E_ARG;
  *out = nullptr;
  if (!(L > 0) || n_grid < 4 || n_grid > kMaxN || !(ecut > 0) || !vloc || (coulomb != 0 && coulomb != 1))
    return GW_E_ARG;
  gw_ctx* ctx = new gw_ctx();
  ctx->L = L;
  ctx->N = n_grid;
  ctx->N3 = n_grid * n_grid * n_grid;
  ctx->ecut = ecut;
  ctx->vol = L * L * L;
  ctx->coulomb = coulomb;
  ctx->user = reinterpret_cast<cudaStream_t>(cuda_stream);
  auto bail = [&](gw_status s) { gw_destroy(ctx); return s; };
  if (!make_plan(n_grid, &ctx->plan)) return bail(GW_E_ARG);
  for (int r = 0; r < ctx->N3; ++r)
    if (!std::isfinite(vloc[r])) return bail(GW_E_NONFINITE);
  // run on the caller's stream when one is given, else on a private stream
  if (ctx->user) {
    ctx->st = ctx->user;
    ctx->own_stream = false;
  } else if (cudaStreamCreateWithFlags(&ctx->st, cudaStreamDefault) != cudaSuccess) {
    // a blocking stream: ordered with the legacy default stream, where callers
    // without a stream of their own (e.g. torch's default stream) put their work
    return bail(GW_E_CUDA);
  }
  if (cudaEventCreateWithFlags(&ctx->ev, cudaEventDisableTiming) != cudaSuccess) return bail(GW_E_CUDA);
  if (cudaMallocHost(&ctx->host_pin, 64) != cudaSuccess) return bail(GW_E_CUDA);
  if (fft_set_smem_limits<double>() != cudaSuccess || fft_set_smem_limits<float>() != cudaSuccess)
    return bail(GW_E_CUDA);
  gw_status s = build_geometry(ctx);
  if (s != GW_OK) return bail(s);
  // sqrt of the Coulomb kernel on the full grid (FFT order)
  const int N = n_grid;
  const double gg = 2.0 * M_PI / L, Rc = 0.5 * L;
  std::vector<double> v(vloc, vloc + ctx->N3), sqv(ctx->N3);
  for (double x : v) ctx->vmax = std::max(ctx->vmax, std::fabs(x));
  for (int i0 = 0; i0 < N; ++i0)
    for (int i1 = 0; i1 < N; ++i1)
      for (int i2 = 0; i2 < N; ++i2) {
        const int n0 = (2 * i0 < N) ? i0 : i0 - N;
        const int n1 = (2 * i1 < N) ? i1 : i1 - N;
        const int n2 = (2 * i2 < N) ? i2 : i2 - N;
        const double G2 = gg * gg * (double)((long)n0 * n0 + (long)n1 * n1 + (long)n2 * n2);
        double vc;
        if (G2 == 0.0) vc = (coulomb == 0) ? 2.0 * M_PI * Rc * Rc : 0.0;
        else if (coulomb == 0) vc = 4.0 * M_PI * (1.0 - std::cos(std::sqrt(G2) * Rc)) / G2;
        else vc = 4.0 * M_PI / G2;
        sqv[(i0 * N + i1) * N + i2] = std::sqrt(vc);
      }
  s = upload_prec<double>(ctx, v, sqv);
  if (s == GW_OK) s = upload_prec<float>(ctx, v, sqv);
  if (s == GW_OK) s = finish(ctx, GW_OK);
  if (s != GW_OK) return bail(s);
  *out = ctx;
  return GW_OK;
}

int gw_npw(const gw_ctx* ctx) { return ctx ? ctx->npw : 0; }

gw_status gw_sphere(const gw_ctx* ctx, int* miller) {
  if (!ctx || !miller) return GW_E_ARG;
  std::memcpy(miller, ctx->miller.data(), ctx->miller.size() * sizeof(int));
  return GW_OK;
}

gw_status gw_set_occupied(gw_ctx* ctx, int n_occ, const double* psi, const double* eps) {
  if (!ctx) return GW_E_ARG;
  if (n_occ < 1 || n_occ > kMaxOcc || !psi || !eps) return fail(ctx, GW_E_ARG, "bad n_occ / pointers");
  TRY(begin(ctx));
  const int npw = ctx->npw;
  for (int v = 0; v < n_occ; ++v) {
    if (!std::isfinite(eps[v])) return fail(ctx, GW_E_NONFINITE, "non-finite energy");
    if (v > 0 && eps[v] < eps[v - 1]) return fail(ctx, GW_E_ARG, "energies must be ascending");
  }
  std::vector<zc> R;
  std::vector<double> e;
  TRY(realify_block(ctx, n_occ, psi, eps, nullptr, 0, &R, &e, "occupied"));
  ctx->nocc = n_occ;
  ctx->eps = e;
  ctx->tkin.assign(n_occ, 0.0);
  for (int v = 0; v < n_occ; ++v) {     // T_v = sum_G |G|^2/2 |c_G|^2
    double t = 0.0;
    for (int s2 = 0; s2 < npw; ++s2) t += ctx->kin[s2] * std::norm(R[(size_t)v * npw + s2]);
    ctx->tkin[v] = std::max(t, 1e-3);
  }
  {
    double kmax = 0.0, emax = 0.0;
    for (double k : ctx->kin) kmax = std::max(kmax, k);
    for (double x : e) emax = std::max(emax, std::fabs(x));
    ctx->anorm = kmax + ctx->vmax + emax;
  }
  ctx->work_cols = 0;
  ctx->c_occ = R;
  ctx->ndef = 0;                      // a new occupied block drops any deflation block
  ctx->eps_def.clear();
  TRY(upload_projector(ctx, {}));
  // u_v(r) = sum_G c_G e^{iGr}: scatter, inverse transforms (FP64), then FP32 copy
  double2* U;
  float2* U32;
  TRY(getbuf(ctx, "occ_U64", (size_t)n_occ * ctx->N3, &U));
  TRY(getbuf(ctx, "occ_U32", (size_t)n_occ * ctx->N3, &U32));
  const Geometry& g = ctx->geo;
  launch_zpass<double>(ctx->st, Z_SCATTER_INV, g, ctx->P64, ctx->plan, U, ctx->P64.C, nullptr, nullptr, nullptr,
                       nullptr, nullptr, nullptr, nullptr, n_occ);
  launch_ypass<double>(ctx->st, 1, 1, 0, g, ctx->P64, ctx->plan, U, nullptr, n_occ, 0);
  launch_xpass_mul<double>(ctx->st, 1, 1, 0, g, ctx->P64, ctx->plan, U, nullptr, nullptr, n_occ);
  conv_real<double, float>(ctx->st, (size_t)2 * n_occ * ctx->N3, reinterpret_cast<double*>(U),
                           reinterpret_cast<float*>(U32));
  ctx->P64.U = U;
  ctx->P32.U = U32;
  TRY(launch_check(ctx, "set_occupied"));
  return finish(ctx, GW_OK);
}

gw_status gw_set_deflation(gw_ctx* ctx, int n_def, const double* psi, const double* eps) {
  if (!ctx) return GW_E_ARG;
  TRY(begin(ctx));
  if (ctx->nocc <= 0) return fail(ctx, GW_E_ARG, "gw_set_occupied has not been called");
  if (n_def < 0 || ctx->nocc + n_def > kMaxOcc || (n_def > 0 && (!psi || !eps)))
    return fail(ctx, GW_E_ARG, "bad n_def / pointers");
  for (int d = 0; d < n_def; ++d) {
    if (!std::isfinite(eps[d])) return fail(ctx, GW_E_NONFINITE, "non-finite energy");
    if ((d > 0 && eps[d] < eps[d - 1]) || eps[d] < ctx->eps.back())
      return fail(ctx, GW_E_ARG, "deflation energies must be ascending and above the occupied ones");
  }
  std::vector<zc> R;
  std::vector<double> e;
  if (n_def > 0) TRY(realify_block(ctx, n_def, psi, eps, &ctx->c_occ, ctx->nocc, &R, &e, "deflation"));
  ctx->work_cols = 0;
  ctx->ndef = n_def;
  ctx->eps_def = e;
  TRY(upload_projector(ctx, R));
  return finish(ctx, GW_OK);
}

gw_status gw_apply_h(gw_ctx* ctx, const double* x, int nb, double* y, gw_prec prec, int dev) {
  TRY(begin(ctx));
  if (nb < 0 || (nb > 0 && (!x || !y))) return fail(ctx, GW_E_ARG, "bad arguments");
  if (nb == 0) return GW_OK;
  const size_t bytes = (size_t)nb * ctx->npw * sizeof(double2);
  const void* xin;
  void* yout;
  TRY(stage_in(ctx, "io_in", x, bytes, dev, &xin));
  TRY(stage_out(ctx, "io_out", y, bytes, dev, &yout));
  std::vector<double2> E(nb, make_double2(0, 0));
  double2* dE;
  TRY(upload(ctx, "ah_E", E, &dE));
  if (prec == GW_FP64) {
    double2* xc;
    TRY(getbuf(ctx, "ah_x", (size_t)nb * ctx->npw, &xc));
    CK(cudaMemcpyAsync(xc, xin, bytes, cudaMemcpyDeviceToDevice, ctx->st));
    TRY(h_apply<double>(ctx, xc, nb, dE, nullptr, reinterpret_cast<double2*>(yout)));
  } else {
    float2 *xc, *yc;
    TRY(getbuf(ctx, "ah_x32", (size_t)nb * ctx->npw, &xc));
    TRY(getbuf(ctx, "ah_y32", (size_t)nb * ctx->npw, &yc));
    launch_gather_rows<float, double>(ctx->st, ctx->npw, nb, reinterpret_cast<const double2*>(xin), nullptr, xc);
    TRY(h_apply<float>(ctx, xc, nb, dE, nullptr, yc));
    launch_gather_rows<double, float>(ctx->st, ctx->npw, nb, yc, nullptr, reinterpret_cast<double2*>(yout));
  }
  TRY(copy_back(ctx, y, yout, bytes, dev));
  return finish(ctx, launch_check(ctx, "apply_h"));
}

static gw_status apply_common(gw_ctx* ctx, const double* x, int nb, const double* omega, int n_omega,
                              double* out, gw_prec prec, int dev, bool chi0_only, bool x_cplx) {
  TRY(begin(ctx));
  TRY(need_occ(ctx));
  if (nb < 0 || n_omega < 1 || !omega || (nb > 0 && (!x || !out))) return fail(ctx, GW_E_ARG, "bad arguments");
  if (prec != GW_FP64 && prec != GW_MIXED) return fail(ctx, GW_E_ARG, "bad precision");
  std::vector<double2> om;
  TRY(check_omega(ctx, omega, n_omega, &om));
  if (nb == 0) return GW_OK;
  bool out_cplx = x_cplx;
  for (auto& o : om) out_cplx |= (o.y != 0.0);
  for (int i = 0; i < 6; ++i) ctx->stats[i] = 0;
  ctx->pcg_iters = 0;
  const size_t ib = (size_t)nb * ctx->N3 * (x_cplx ? sizeof(double2) : sizeof(double));
  const size_t ob = (size_t)nb * ctx->N3 * n_omega * (out_cplx ? sizeof(double2) : sizeof(double));
  const void* xin;
  void* o;
  TRY(stage_in(ctx, "io_in", x, ib, dev, &xin));
  TRY(stage_out(ctx, "io_out", out, ob, dev, &o));
  gw_status sv = GW_OK;
  if (prec == GW_FP64) SOFT(sv, (eps_core<double>(ctx, xin, x_cplx, nb, om, o, chi0_only)));
  else SOFT(sv, (eps_core<float>(ctx, xin, x_cplx, nb, om, o, chi0_only)));
  TRY(copy_back(ctx, out, o, ob, dev));
  if (ctx->stats[0] > 0) ctx->stats[2] /= ctx->stats[0];
  return finish(ctx, sv);
}

gw_status gw_apply_chi0(gw_ctx* ctx, const double* dV, int nb, const double* omega, int n_omega, double* dn,
                        gw_prec prec, int dev) {
  return apply_common(ctx, dV, nb, omega, n_omega, dn, prec, dev, true, false);
}

gw_status gw_apply_eps(gw_ctx* ctx, const double* x, int nb, const double* omega, int n_omega, double* out,
                       gw_prec prec, int dev) {
  return apply_common(ctx, x, nb, omega, n_omega, out, prec, dev, false, false);
}

gw_status gw_apply_chi0_c(gw_ctx* ctx, const double* dV, int nb, const double* omega, int n_omega, double* dn,
                          gw_prec prec, int dev) {
  return apply_common(ctx, dV, nb, omega, n_omega, dn, prec, dev, true, true);
}

gw_status gw_apply_eps_c(gw_ctx* ctx, const double* x, int nb, const double* omega, int n_omega, double* out,
                         gw_prec prec, int dev) {
  return apply_common(ctx, x, nb, omega, n_omega, out, prec, dev, false, true);
}

gw_status gw_lanczos(gw_ctx* ctx, const double* start, int blk, int k, const double* omega, double* alpha,
                     double* beta, double* basis, gw_prec prec, int dev) {
  TRY(begin(ctx));
  TRY(need_occ(ctx));
  if (!start || !alpha || k < 1 || (k > 1 && !beta) || !omega) return fail(ctx, GW_E_ARG, "bad arguments");
  if (blk != 1) return fail(ctx, GW_E_UNSUPPORTED, "gw_lanczos takes blk = 1; blocks go through gw_block_lanczos");
  std::vector<double2> om;
  TRY(check_omega(ctx, omega, 1, &om));
  if (om[0].y != 0.0)
    return fail(ctx, GW_E_UNSUPPORTED, "gw_lanczos is the real-frequency recursion; use gw_block_lanczos");
  for (int i = 0; i < 6; ++i) ctx->stats[i] = 0;
  ctx->pcg_iters = 0;
  const size_t fb = (size_t)ctx->N3 * sizeof(double);
  const void* x0;
  TRY(stage_in(ctx, "lz_x0", start, fb, dev, &x0));
  double *a, *b, *Q;
  TRY(getbuf(ctx, "lz_alpha", k, &a));
  TRY(getbuf(ctx, "lz_beta", std::max(k - 1, 1), &b));
  if (dev && basis) Q = basis;
  else TRY(getbuf(ctx, "lz_Q", (size_t)k * ctx->N3, &Q));
  // the start vector may alias nothing we write; copy it (lanczos_core normalises from it)
  double* x0c;
  TRY(getbuf(ctx, "lz_x0c", ctx->N3, &x0c));
  CK(cudaMemcpyAsync(x0c, x0, fb, cudaMemcpyDeviceToDevice, ctx->st));
  gw_status s = (prec == GW_FP64) ? lanczos_core<double>(ctx, x0c, k, om, a, b, Q)
                                  : lanczos_core<float>(ctx, x0c, k, om, a, b, Q);
  if (s != GW_OK && s != GW_E_BREAKDOWN) return s;
  if (dev) {
    CK(cudaMemcpyAsync(alpha, a, k * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
    if (k > 1) CK(cudaMemcpyAsync(beta, b, (k - 1) * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
  } else {
    CK(cudaMemcpyAsync(alpha, a, k * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    if (k > 1) CK(cudaMemcpyAsync(beta, b, (k - 1) * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    if (basis) CK(cudaMemcpyAsync(basis, Q, (size_t)k * fb, cudaMemcpyDeviceToHost, ctx->st));
  }
  if (ctx->stats[0] > 0) ctx->stats[2] /= ctx->stats[0];
  return finish(ctx, s);
}

gw_status gw_lanczos_resume(gw_ctx* ctx, const double* basis_in, const double* alpha_in, const double* beta_in,
                            int k0, int k, const double* omega, double* alpha, double* beta, double* basis,
                            gw_prec prec, int dev) {
  TRY(begin(ctx));
  TRY(need_occ(ctx));
  if (!basis_in || !omega || !alpha || !beta || k0 < 1 || k <= k0) return fail(ctx, GW_E_ARG, "bad arguments");
  std::vector<double2> om;
  TRY(check_omega(ctx, omega, 1, &om));
  if (om[0].y != 0.0)
    return fail(ctx, GW_E_UNSUPPORTED, "gw_lanczos_resume is the real-frequency recursion");
  for (int i = 0; i < 6; ++i) ctx->stats[i] = 0;
  ctx->pcg_iters = 0;
  const size_t fb = (size_t)ctx->N3 * sizeof(double);
  // the saved coefficients: finite, beta > 0
  std::vector<double> ha(k0), hbv(k0);
  if (dev) {
    CK(cudaMemcpyAsync(ha.data(), alpha_in, k0 * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(hbv.data(), beta_in, k0 * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    TRY(sync(ctx, "resume"));
  } else {
    std::memcpy(ha.data(), alpha_in, k0 * sizeof(double));
    std::memcpy(hbv.data(), beta_in, k0 * sizeof(double));
  }
  for (int i = 0; i < k0; ++i)
    if (!std::isfinite(ha[i]) || !std::isfinite(hbv[i]) || !(hbv[i] > 0.0))
      return fail(ctx, GW_E_ARG, "Lanczos state rejected: non-finite or non-positive coefficient");
  double *a, *b, *Q;
  TRY(getbuf(ctx, "lz_alpha", k, &a));
  TRY(getbuf(ctx, "lz_beta", std::max(k - 1, 1), &b));
  if (dev && basis && basis != basis_in) Q = basis;
  else TRY(getbuf(ctx, "lz_Q", (size_t)k * ctx->N3, &Q));
  CK(cudaMemcpyAsync(Q, basis_in, (size_t)(k0 + 1) * fb, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     ctx->st));
  CK(cudaMemcpyAsync(a, ha.data(), k0 * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(b, hbv.data(), k0 * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
  // the saved vectors: orthonormal in <.|.> to 1e-8 (a damaged state fails here)
  {
    const double wgt = ctx->vol / ctx->N3;
    double* h;
    TRY(getbuf(ctx, "lz_h", k + 1, &h));
    TRY(ensure_work(ctx, (size_t)k + 1));
    std::vector<double> hh(k0 + 1);
    double worst = 0.0;
    for (int j = 0; j <= k0; ++j) {
      launch_gemv_t(ctx->st, Q, ctx->N3, ctx->N3, Q + (size_t)j * ctx->N3, wgt, k0 + 1, ctx->work, h);
      CK(cudaMemcpyAsync(hh.data(), h, (k0 + 1) * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
      TRY(sync(ctx, "resume check"));
      for (int i = 0; i <= k0; ++i) {
        const double d = std::fabs(hh[i] - (i == j ? 1.0 : 0.0));
        worst = std::isfinite(d) ? std::max(worst, d) : 1e300;
      }
    }
    if (!(worst <= 1e-8)) {
      char m[128];
      std::snprintf(m, sizeof(m), "Lanczos state rejected: vectors not orthonormal (max |Q^T Q - I| = %.3g)", worst);
      return fail(ctx, GW_E_ARG, m);
    }
  }
  gw_status s = (prec == GW_FP64) ? lanczos_core<double>(ctx, nullptr, k, om, a, b, Q, 1, nullptr, k0)
                                  : lanczos_core<float>(ctx, nullptr, k, om, a, b, Q, 1, nullptr, k0);
  if (s != GW_OK && s != GW_E_BREAKDOWN) return s;
  if (dev) {
    CK(cudaMemcpyAsync(alpha, a, k * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaMemcpyAsync(beta, b, (k - 1) * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
    if (basis && basis != Q) CK(cudaMemcpyAsync(basis, Q, (size_t)k * fb, cudaMemcpyDeviceToDevice, ctx->st));
  } else {
    CK(cudaMemcpyAsync(alpha, a, k * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(beta, b, (k - 1) * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    if (basis) CK(cudaMemcpyAsync(basis, Q, (size_t)k * fb, cudaMemcpyDeviceToHost, ctx->st));
  }
  if (ctx->stats[0] > 0) ctx->stats[2] /= ctx->stats[0];
  return finish(ctx, s);
}

gw_status gw_block_lanczos(gw_ctx* ctx, const double* start, int blk, int k, const double* omega, double* A,
                           double* B, double* basis, gw_prec prec, int dev) {
  TRY(begin(ctx));
  TRY(need_occ(ctx));
  if (!start || !A || !omega || k < 1 || (k > 1 && !B) || blk < 1 || blk > 16)
    return fail(ctx, GW_E_ARG, "bad arguments (1 <= blk <= 16)");
  std::vector<double2> om;
  TRY(check_omega(ctx, omega, 1, &om));
  for (int i = 0; i < 6; ++i) ctx->stats[i] = 0;
  ctx->pcg_iters = 0;
  const size_t N3 = ctx->N3;
  const void* x0;
  TRY(stage_in(ctx, "bl_start", start, (size_t)blk * N3 * sizeof(double), dev, &x0));
  double2* Q;
  if (dev && basis) Q = reinterpret_cast<double2*>(basis);
  else TRY(getbuf(ctx, "bl_Q", (size_t)k * blk * N3, &Q));
  std::vector<zcd> Ah, Bh;
  gw_status s = (prec == GW_FP64)
                    ? block_lanczos_core<double>(ctx, reinterpret_cast<const double*>(x0), blk, k, om[0], &Ah, &Bh, Q)
                    : block_lanczos_core<float>(ctx, reinterpret_cast<const double*>(x0), blk, k, om[0], &Ah, &Bh, Q);
  if (s != GW_OK && s != GW_E_BREAKDOWN) return s;
  const size_t na = (size_t)k * blk * blk, nbb = (size_t)(k - 1) * blk * blk;
  if (dev) {
    CK(cudaMemcpyAsync(A, Ah.data(), na * sizeof(zcd), cudaMemcpyHostToDevice, ctx->st));
    if (k > 1) CK(cudaMemcpyAsync(B, Bh.data(), nbb * sizeof(zcd), cudaMemcpyHostToDevice, ctx->st));
  } else {
    std::memcpy(A, Ah.data(), na * sizeof(zcd));
    if (k > 1) std::memcpy(B, Bh.data(), nbb * sizeof(zcd));
    if (basis) CK(cudaMemcpyAsync(basis, Q, (size_t)k * blk * N3 * sizeof(double2), cudaMemcpyDeviceToHost, ctx->st));
  }
  if (ctx->stats[0] > 0) ctx->stats[2] /= ctx->stats[0];
  return finish(ctx, s);
}

gw_status gw_epsinv_block(gw_ctx* ctx, const double* A, const double* B, int k, int blk, int bilinear, double* out,
                          int dev) {
  TRY(begin(ctx));
  if (!A || !out || k < 1 || blk < 1 || (k > 1 && !B)) return fail(ctx, GW_E_ARG, "bad arguments");
  const int n = k * blk;
  if (n > 2048) return fail(ctx, GW_E_ARG, "block Lanczos matrix larger than 2048");
  const size_t na = (size_t)k * blk * blk * sizeof(double2), nbb = (size_t)std::max(k - 1, 1) * blk * blk * sizeof(double2);
  const void *a, *b = nullptr;
  TRY(stage_in(ctx, "eb_a", A, na, dev, &a));
  if (k > 1) TRY(stage_in(ctx, "eb_b", B, nbb, dev, &b));
  else {
    double2* z;
    TRY(getbuf(ctx, "eb_bz", (size_t)blk * blk, &z));
    b = z;
  }
  double2* T;
  int* stat;
  TRY(getbuf(ctx, "eb_T", (size_t)n * n, &T));
  TRY(getbuf(ctx, "eb_stat", 1, &stat));
  void* o;
  TRY(stage_out(ctx, "eb_o", out, (size_t)n * n * sizeof(double2), dev, &o));
  launch_block_tridiag(ctx->st, k, blk, reinterpret_cast<const double2*>(a), reinterpret_cast<const double2*>(b),
                       bilinear ? 1 : 0, T);
  launch_cinv(ctx->st, n, T, reinterpret_cast<double2*>(o), stat);
  TRY(launch_check(ctx, "epsinv_block"));
  CK(cudaMemcpyAsync(ctx->host_pin, stat, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  TRY(copy_back(ctx, out, o, (size_t)n * n * sizeof(double2), dev));
  TRY(sync(ctx, "epsinv_block"));
  if (ctx->host_pin[0]) return fail(ctx, GW_E_BREAKDOWN, "singular block-tridiagonal matrix");
  return GW_OK;
}

gw_status gw_epsinv_elements(gw_ctx* ctx, const double* alpha, const double* beta, int k, int blk, double* out,
                             int dev) {
  TRY(begin(ctx));
  if (!alpha || !out || k < 1 || (k > 1 && !beta)) return fail(ctx, GW_E_ARG, "bad arguments");
  if (blk != 1) return fail(ctx, GW_E_UNSUPPORTED, "gw_epsinv_elements takes blk = 1; blocks go through gw_epsinv_block");
  const void *a, *b = nullptr;
  TRY(stage_in(ctx, "ei_a", alpha, k * sizeof(double), dev, &a));
  if (k > 1) TRY(stage_in(ctx, "ei_b", beta, (k - 1) * sizeof(double), dev, &b));
  double *d, *l, *o;
  int* stat;
  TRY(getbuf(ctx, "ei_d", k, &d));
  TRY(getbuf(ctx, "ei_l", k, &l));
  TRY(getbuf(ctx, "ei_stat", 1, &stat));
  void* op;
  TRY(stage_out(ctx, "ei_o", out, (size_t)k * k * sizeof(double), dev, &op));
  o = reinterpret_cast<double*>(op);
  launch_tridiag_inv(ctx->st, k, reinterpret_cast<const double*>(a), reinterpret_cast<const double*>(b), d, l, o,
                     stat);
  TRY(launch_check(ctx, "epsinv"));
  CK(cudaMemcpyAsync(ctx->host_pin, stat, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  TRY(copy_back(ctx, out, o, (size_t)k * k * sizeof(double), dev));
  TRY(sync(ctx, "epsinv"));
  if (ctx->host_pin[0]) return fail(ctx, GW_E_BREAKDOWN, "zero pivot in the tridiagonal inverse");
  return GW_OK;
}

gw_status gw_grad_vloc(gw_ctx* ctx, const double* phi, int k, double* s, double* grad, gw_prec prec, int dev) {
  TRY(begin(ctx));
  TRY(need_occ(ctx));
  if (ctx->op != GW_OP_STERNHEIMER)
    return fail(ctx, GW_E_UNSUPPORTED, "the gradient is of the Sternheimer operator; set GW_OP_STERNHEIMER");
  if (!phi || !s || !grad || k < 1) return fail(ctx, GW_E_ARG, "bad arguments");
  if (prec != GW_FP64 && prec != GW_MIXED) return fail(ctx, GW_E_ARG, "bad precision");
  for (int i = 0; i < 6; ++i) ctx->stats[i] = 0;
  const size_t fb = (size_t)ctx->N3 * sizeof(double);
  const void* ph;
  void* go;
  TRY(stage_in(ctx, "gr_phi", phi, fb, dev, &ph));
  TRY(stage_out(ctx, "gr_out", grad, fb, dev, &go));
  double sv = 0.0;
  gw_status st = (prec == GW_FP64)
                     ? grad_core<double>(ctx, reinterpret_cast<const double*>(ph), k, &sv, reinterpret_cast<double*>(go))
                     : grad_core<float>(ctx, reinterpret_cast<const double*>(ph), k, &sv, reinterpret_cast<double*>(go));
  if (st != GW_OK) return st;
  TRY(copy_back(ctx, grad, go, fb, dev));
  TRY(sync(ctx, "grad"));
  if (dev) CK(cudaMemcpy(s, &sv, sizeof(double), cudaMemcpyHostToDevice));
  else *s = sv;
  if (ctx->stats[0] > 0) ctx->stats[2] /= ctx->stats[0];
  return GW_OK;
}

gw_status gw_grad_vloc_basis(gw_ctx* ctx, const double* phi, const double* basis, const double* alpha,
                             const double* beta, int k, double* s, double* grad, gw_prec prec, int dev) {
  TRY(begin(ctx));
  TRY(need_occ(ctx));
  if (ctx->op != GW_OP_STERNHEIMER)
    return fail(ctx, GW_E_UNSUPPORTED, "the gradient is of the Sternheimer operator; set GW_OP_STERNHEIMER");
  if (!phi || !basis || !alpha || (k > 1 && !beta) || !s || !grad || k < 1) return fail(ctx, GW_E_ARG, "bad arguments");
  if (prec != GW_FP64 && prec != GW_MIXED) return fail(ctx, GW_E_ARG, "bad precision");
  for (int i = 0; i < 6; ++i) ctx->stats[i] = 0;
  const size_t fb = (size_t)ctx->N3 * sizeof(double);
  const void *ph, *qb, *ab, *bb;
  void* go;
  TRY(stage_in(ctx, "gr_phi", phi, fb, dev, &ph));
  TRY(stage_in(ctx, "grb_Q", basis, fb * k, dev, &qb));
  TRY(stage_in(ctx, "grb_a", alpha, (size_t)k * sizeof(double), dev, &ab));
  if (k > 1) TRY(stage_in(ctx, "grb_b", beta, (size_t)(k - 1) * sizeof(double), dev, &bb));
  else bb = ab;
  TRY(stage_out(ctx, "gr_out", grad, fb, dev, &go));
  double sv = 0.0;
  const double* P = reinterpret_cast<const double*>(ph);
  const double* Q = reinterpret_cast<const double*>(qb);
  const double* A = reinterpret_cast<const double*>(ab);
  const double* B = reinterpret_cast<const double*>(bb);
  gw_status st = (prec == GW_FP64) ? grad_from_basis<double>(ctx, P, Q, A, B, k, &sv, reinterpret_cast<double*>(go))
                                   : grad_from_basis<float>(ctx, P, Q, A, B, k, &sv, reinterpret_cast<double*>(go));
  if (st != GW_OK) return st;
  TRY(copy_back(ctx, grad, go, fb, dev));
  TRY(sync(ctx, "grad"));
  if (dev) CK(cudaMemcpy(s, &sv, sizeof(double), cudaMemcpyHostToDevice));
  else *s = sv;
  if (ctx->stats[0] > 0) ctx->stats[2] /= ctx->stats[0];
  return GW_OK;
}

gw_status gw_stats(const gw_ctx* ctx, double* out, int n) {
  if (!ctx || !out || n < 0) return GW_E_ARG;
  for (int i = 0; i < n && i < 6; ++i) out[i] = ctx->stats[i];
  if (n > 6) out[6] = (double)g_launches.load();
  if (n > 7) out[7] = (double)ctx->pcg_iters;
  if (n > 8) out[8] = (double)ctx->pcg_launch_blocks;
  if (n > 9) out[9] = (double)ctx->pcg_cluster;
  if (n > 10) out[10] = (double)ctx->graph_replays;
  if (n > 11) out[11] = (double)ctx->pcg_tpb;
  return GW_OK;
}

gw_status gw_set_autotune(gw_ctx* ctx, int on) {
  if (!ctx) return GW_E_ARG;
  ctx->tune = (on != 0);
  return GW_OK;
}

gw_status gw_set_tensor_cores(gw_ctx* ctx, int on) {
  if (!ctx) return GW_E_ARG;
  ctx->use_tc = (on != 0);
  return GW_OK;
}

gw_status gw_proj_coef(gw_ctx* ctx, const float* y, int ncol, double* coef, int kernel) {
  TRY(begin(ctx));
  TRY(need_occ(ctx));
  if (!y || !coef || ncol < 1 || (kernel != 0 && kernel != 1)) return fail(ctx, GW_E_ARG, "bad arguments");
  const int npw = ctx->npw, np = nproj(ctx);
  const float2* Y = reinterpret_cast<const float2*>(y);
  double2* out = reinterpret_cast<double2*>(coef);
  TRY(ensure_work(ctx, ncol));
  if (kernel == 0) {
    launch_gram<float>(ctx->st, ctx->P32.C, np, npw, Y, ncol, ctx->work, out);
  } else {
    if (!ctx->tc_ok) return fail(ctx, GW_E_UNSUPPORTED, "tensor-core projector unavailable (more than 64 rows?)");
    float* part;
    int* err;
    TRY(getbuf(ctx, "tc_part", tc_part_elems(npw, ncol), &part));
    TRY(getbuf(ctx, "tc_err", 1, &err));
    CK(cudaMemsetAsync(err, 0, sizeof(int), ctx->st));
    CK(launch_tc_dots(ctx->st, ctx->tc_maps, Y, npw, ncol, np, part, out, err,
                      std::max<unsigned long long>(ctx->wait_limit / 16, 1024)));
    int herr = 0;
    CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    TRY(sync(ctx, "proj_coef"));
    if (herr) return fail(ctx, GW_E_TIMEOUT, "tensor-core projector: a bounded device wait gave up");
  }
  TRY(launch_check(ctx, "proj_coef"));
  return finish(ctx, GW_OK);
}

gw_status gw_set_recycle_augment(gw_ctx* ctx, double w0) {
  if (!ctx) return GW_E_ARG;
  if (!(w0 >= 0.0) || !std::isfinite(w0)) return fail(ctx, GW_E_ARG, "w0 must be finite and >= 0");
  ctx->recycle_w0 = w0;
  return GW_OK;
}

gw_status gw_set_imaginary_route(gw_ctx* ctx, int route) {
  if (!ctx) return GW_E_ARG;
  if (route != GW_IMAG_SQMR && route != GW_IMAG_SQUARED) return fail(ctx, GW_E_ARG, "unknown imaginary-frequency route");
  ctx->imag_route = route;
  return GW_OK;
}

gw_status gw_set_graphs(gw_ctx* ctx, int on) {
  if (!ctx) return GW_E_ARG;
  ctx->use_graphs = (on != 0);
  return GW_OK;
}

gw_status gw_set_solver(gw_ctx* ctx, double tol, double tol_inner, int max_iter, int max_outer) {
  if (!ctx) return GW_E_ARG;
  if (tol > 0) { ctx->tol = tol; ctx->tol_mixed = std::max(tol, 1e-13); }
  if (tol_inner > 0) ctx->tol_inner = tol_inner;
  if (max_iter > 0) ctx->max_iter = max_iter;
  if (max_outer > 0) ctx->max_outer = max_outer;
  return GW_OK;
}

gw_status gw_set_cg_kernel(gw_ctx* ctx, int kind, long long wait_limit) {
  if (!ctx) return GW_E_ARG;
  if (kind < GW_CG_PERSISTENT || kind > GW_CG_CLUSTER) return fail(ctx, GW_E_ARG, "unknown CG kernel");
  if (wait_limit < 0) return fail(ctx, GW_E_ARG, "wait_limit must be >= 0");
  ctx->cg_kernel = kind;
  if (wait_limit > 0) ctx->wait_limit = (unsigned long long)wait_limit;
  return GW_OK;
}

gw_status gw_set_operator(gw_ctx* ctx, int op) {
  if (!ctx) return GW_E_ARG;
  if (op != GW_OP_STERNHEIMER && op != GW_OP_MODEL)
    return fail(ctx, GW_E_ARG, "operator must be GW_OP_STERNHEIMER (0) or GW_OP_MODEL (1)");
  ctx->op = op;
  return GW_OK;
}

// Eq. subs_epsilon: <phi_i|eps~^-1 - 1|phi_j> = a_i^T (T^-1 - M^-1) a_j + am_i^T (Tm^-1 - 1) am_j
// with a = <Q|phi>, am = <Qm|phi>, M = <Q|eps~_model Q> (model applied to the
// exact basis), T and Tm the tridiagonal Lanczos matrices of the two bases.
gw_status gw_epsinv_split(gw_ctx* ctx, const double* phi, int m, const double* basis, const double* alpha,
                          const double* beta, int k, const double* basis_m, const double* alpha_m,
                          const double* beta_m, int k_m, double omega, double* out, int dev) {
  TRY(begin(ctx));
  TRY(need_occ(ctx));
  if (!phi || !basis || !alpha || !basis_m || !alpha_m || !out || m < 1 || m > 64 || k < 1 || k_m < 1 ||
      k > 2048 || k_m > 4096 || (k > 1 && !beta) || (k_m > 1 && !beta_m))
    return fail(ctx, GW_E_ARG, "bad arguments");
  if (!std::isfinite(omega)) return fail(ctx, GW_E_NONFINITE, "non-finite omega");
  for (int i = 0; i < 6; ++i) ctx->stats[i] = 0;
  const int N3 = ctx->N3;
  const double wgt = ctx->vol / N3;
  const size_t fb = (size_t)N3 * sizeof(double);
  const void *ph, *Qv, *Qmv, *al, *alm, *be = nullptr, *bem = nullptr;
  TRY(stage_in(ctx, "sp_phi", phi, m * fb, dev, &ph));
  TRY(stage_in(ctx, "sp_Q", basis, k * fb, dev, &Qv));
  TRY(stage_in(ctx, "sp_Qm", basis_m, k_m * fb, dev, &Qmv));
  TRY(stage_in(ctx, "sp_al", alpha, k * sizeof(double), dev, &al));
  TRY(stage_in(ctx, "sp_alm", alpha_m, k_m * sizeof(double), dev, &alm));
  if (k > 1) TRY(stage_in(ctx, "sp_be", beta, (k - 1) * sizeof(double), dev, &be));
  if (k_m > 1) TRY(stage_in(ctx, "sp_bem", beta_m, (k_m - 1) * sizeof(double), dev, &bem));
  const double* Q = reinterpret_cast<const double*>(Qv);
  const double* Qm = reinterpret_cast<const double*>(Qmv);
  const double* P = reinterpret_cast<const double*>(ph);
  double *a, *am, *EQ, *Mt, *Ti, *Tmi, *d, *l;
  double2 *Mc, *Mi;
  int* stat;
  const int nbc = std::min(k, 16);
  TRY(getbuf(ctx, "sp_a", (size_t)m * k, &a));
  TRY(getbuf(ctx, "sp_am", (size_t)m * k_m, &am));
  TRY(getbuf(ctx, "sp_EQ", (size_t)nbc * N3, &EQ));
  TRY(getbuf(ctx, "sp_Mt", (size_t)k * k, &Mt));
  TRY(getbuf(ctx, "sp_Ti", (size_t)k * k, &Ti));
  TRY(getbuf(ctx, "sp_Tmi", (size_t)k_m * k_m, &Tmi));
  TRY(getbuf(ctx, "sp_d", std::max(k, k_m), &d));
  TRY(getbuf(ctx, "sp_l", std::max(k, k_m), &l));
  TRY(getbuf(ctx, "sp_Mc", (size_t)k * k, &Mc));
  TRY(getbuf(ctx, "sp_Mi", (size_t)k * k, &Mi));
  TRY(getbuf(ctx, "sp_stat", 3, &stat));
  // the model operator in the exact basis: Mt[j][i] = <q_i|eps~_model q_j>
  const int op0 = ctx->op;
  ctx->op = GW_OP_MODEL;
  const std::vector<double2> om{make_double2(omega, 0.0)};
  for (int j0 = 0; j0 < k; j0 += nbc) {
    const int nb = std::min(nbc, k - j0);
    gw_status st = eps_core<double>(ctx, Q + (size_t)j0 * N3, false, nb, om, EQ, false);
    if (st != GW_OK) { ctx->op = op0; return st; }
    TRY(ensure_work(ctx, std::max(k, k_m) + 1));
    for (int j = 0; j < nb; ++j)
      launch_gemv_t(ctx->st, Q, N3, N3, EQ + (size_t)j * N3, wgt, k, ctx->work, Mt + (size_t)(j0 + j) * k);
  }
  ctx->op = op0;
  // coefficients of the fields in both bases
  TRY(ensure_work(ctx, std::max(k, k_m) + 1));
  for (int i = 0; i < m; ++i) {
    launch_gemv_t(ctx->st, Q, N3, N3, P + (size_t)i * N3, wgt, k, ctx->work, a + (size_t)i * k);
    launch_gemv_t(ctx->st, Qm, N3, N3, P + (size_t)i * N3, wgt, k_m, ctx->work, am + (size_t)i * k_m);
  }
  // the three inverses and the two quadratic forms
  launch_tridiag_inv(ctx->st, k, reinterpret_cast<const double*>(al), reinterpret_cast<const double*>(be), d, l,
                     Ti, stat);
  launch_tridiag_inv(ctx->st, k_m, reinterpret_cast<const double*>(alm), reinterpret_cast<const double*>(bem), d,
                     l, Tmi, stat + 1);
  launch_to_cplx(ctx->st, (size_t)k * k, Mt, Mc);
  launch_cinv(ctx->st, k, Mc, Mi, stat + 2);
  void* op;
  TRY(stage_out(ctx, "sp_out", out, (size_t)m * m * sizeof(double), dev, &op));
  launch_split_form(ctx->st, m, k, k_m, a, Ti, Mi, am, Tmi, reinterpret_cast<double*>(op));
  TRY(launch_check(ctx, "epsinv_split"));
  CK(cudaMemcpyAsync(ctx->host_pin, stat, 3 * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  TRY(copy_back(ctx, out, op, (size_t)m * m * sizeof(double), dev));
  TRY(sync(ctx, "epsinv_split"));
  if (ctx->host_pin[0] || ctx->host_pin[1] || ctx->host_pin[2])
    return fail(ctx, GW_E_BREAKDOWN, "singular matrix in the split (tridiagonal or model Gram)");
  return GW_OK;
}

// Eq. pe: Sigma^P_e(delta) = - sum_v <e v*|v^1/2 (eps^-1(w_ve) - 1) v^1/2|v* e> Theta(w_ve)
//                             + sum_c <e c*|...(w_ce)...|c* e> Theta(-w_ce),  w_ne = e_n - e_e - delta,
// each element from k Lanczos steps on eps~(w_pe) seeded with phi = v^1/2 |p* e>:
// <phi|eps~^-1 - 1|phi> ~ |phi|^2 ((T^-1)_11 - 1).
gw_status gw_sigma_p(gw_ctx* ctx, const double* psi_e, double eps_e, double delta, int n, const double* psi,
                     const double* eps, const int* occ, int k, double* sigma, double* terms, gw_prec prec,
                     int dev) {
  TRY(begin(ctx));
  TRY(need_occ(ctx));
  if (!psi_e || !sigma || n < 0 || (n > 0 && (!psi || !eps || !occ)) || k < 1 || k > 256)
    return fail(ctx, GW_E_ARG, "bad arguments");
  if (prec != GW_FP64 && prec != GW_MIXED) return fail(ctx, GW_E_ARG, "bad precision");
  if (!std::isfinite(eps_e) || !std::isfinite(delta)) return fail(ctx, GW_E_NONFINITE, "non-finite energy");
  for (int i = 0; i < 6; ++i) ctx->stats[i] = 0;
  const int npw = ctx->npw;
  // host copies of the small per-state inputs
  std::vector<double> he(n);
  std::vector<int> ho(n);
  if (n > 0) {
    if (dev) {
      CK(cudaMemcpyAsync(he.data(), eps, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
      CK(cudaMemcpyAsync(ho.data(), occ, n * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
      TRY(sync(ctx, "sigma_p inputs"));
    } else {
      std::copy(eps, eps + n, he.begin());
      std::copy(occ, occ + n, ho.begin());
    }
  }
  std::vector<double> hterms;
  double total = 0.0;
  {
    const void *pe, *pp = nullptr;
    TRY(stage_in(ctx, "sgp_psie", psi_e, (size_t)npw * sizeof(double2), dev, &pe));
    if (n > 0) TRY(stage_in(ctx, "sgp_psi", psi, (size_t)n * npw * sizeof(double2), dev, &pp));
    TRY(sigma_p_core(ctx, reinterpret_cast<const double2*>(pe), eps_e, delta, n,
                     reinterpret_cast<const double2*>(pp), he, ho, k, prec, &total, &hterms));
  }
  if (dev) {
    CK(cudaMemcpyAsync(sigma, &total, sizeof(double), cudaMemcpyHostToDevice, ctx->st));
    if (terms && n > 0) CK(cudaMemcpyAsync(terms, hterms.data(), n * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
    TRY(sync(ctx, "sigma_p out"));
  } else {
    *sigma = total;
    if (terms) std::copy(hterms.begin(), hterms.end(), terms);
  }
  return launch_check(ctx, "sigma_p");
}

gw_status gw_recycle_eps(gw_ctx* ctx, const double* fields, int nl, const double* w, int nw, double rtol,
                         double* out, int* kept, gw_prec prec, int dev) {
  TRY(begin(ctx));
  TRY(need_occ(ctx));
  if (!fields || !w || !out || nl < 1 || nl > 256 || nw < 1 || nw > 4096 || rtol < 0.0 || rtol >= 1.0)
    return fail(ctx, GW_E_ARG, "bad arguments");
  if (prec != GW_FP64 && prec != GW_MIXED) return fail(ctx, GW_E_ARG, "bad precision");
  if (ctx->op != GW_OP_STERNHEIMER)
    return fail(ctx, GW_E_UNSUPPORTED, "the recycled basis is built from Sternheimer solutions");
  if ((size_t)ctx->nocc * (ctx->recycle_w0 > 0.0 ? 3 : 2) * nl > 65535)
    return fail(ctx, GW_E_ARG, "the recycled vectors (2 or 3 nl n_occ) exceed one launch (65535)");
  if (rtol == 0.0) rtol = 1e-6;
  for (int i = 0; i < 6; ++i) ctx->stats[i] = 0;
  const void *F, *W;
  TRY(stage_in(ctx, "rce_F", fields, (size_t)nl * ctx->N3 * sizeof(double), dev, &F));
  TRY(stage_in(ctx, "rce_w", w, (size_t)nw * sizeof(double), dev, &W));
  std::vector<double> hw(nw);
  CK(cudaMemcpyAsync(hw.data(), W, nw * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  TRY(sync(ctx, "recycle inputs"));
  for (double x : hw)
    if (!std::isfinite(x)) return fail(ctx, GW_E_NONFINITE, "non-finite frequency");
  void* o;
  TRY(stage_out(ctx, "rce_out", out, (size_t)nw * nl * nl * sizeof(double), dev, &o));
  int km = 0;
  gw_status st = (prec == GW_FP64)
                     ? recycle_core<double>(ctx, reinterpret_cast<const double*>(F), nl,
                                            reinterpret_cast<const double*>(W), nw, rtol, reinterpret_cast<double*>(o), &km)
                     : recycle_core<float>(ctx, reinterpret_cast<const double*>(F), nl,
                                           reinterpret_cast<const double*>(W), nw, rtol, reinterpret_cast<double*>(o), &km);
  if (st != GW_OK) return st;
  TRY(copy_back(ctx, out, o, (size_t)nw * nl * nl * sizeof(double), dev));
  if (kept) *kept = km;
  if (ctx->stats[0] > 0) ctx->stats[2] /= ctx->stats[0];
  return finish(ctx, GW_OK);
}

gw_status gw_sigma_c(gw_ctx* ctx, int e, double delta, double alpha, int n_freq, const double* fields, int nl,
                     int k_h, int k_p, double* out, gw_prec prec, int dev) {
  TRY(begin(ctx));
  TRY(need_occ(ctx));
  if (!fields || !out || e < 0 || e >= ctx->nocc || !(alpha > 0.0) || n_freq < 1 || n_freq > 64 || nl < 1 ||
      nl > 16 || k_h < 1 || k_h * nl > 512 || k_p < 1 || k_p > 256)
    return fail(ctx, GW_E_ARG, "bad arguments");
  if (prec != GW_FP64 && prec != GW_MIXED) return fail(ctx, GW_E_ARG, "bad precision");
  if (!std::isfinite(delta) || !std::isfinite(alpha)) return fail(ctx, GW_E_NONFINITE, "non-finite argument");
  if (ctx->op != GW_OP_STERNHEIMER) return fail(ctx, GW_E_UNSUPPORTED, "the self-energy uses the Sternheimer operator");
  const double ehomo = *std::max_element(ctx->eps.begin(), ctx->eps.end());
  if (ctx->eps[e] + delta < ehomo)
    return fail(ctx, GW_E_UNSUPPORTED, "e_e + delta below the highest occupied energy (Q_e is not P_c)");
  for (int i = 0; i < 6; ++i) ctx->stats[i] = 0;
  const void* F;
  TRY(stage_in(ctx, "sce_F", fields, (size_t)nl * ctx->N3 * sizeof(double), dev, &F));
  double res[4];
  gw_status st = (prec == GW_FP64)
                     ? sigma_c_core<double>(ctx, e, delta, alpha, n_freq, reinterpret_cast<const double*>(F), nl, k_h,
                                            k_p, prec, res)
                     : sigma_c_core<float>(ctx, e, delta, alpha, n_freq, reinterpret_cast<const double*>(F), nl, k_h,
                                           k_p, prec, res);
  if (st != GW_OK) return st;
  for (double x : res)
    if (!std::isfinite(x)) return fail(ctx, GW_E_NONFINITE, "non-finite self-energy");
  if (dev) {
    CK(cudaMemcpyAsync(out, res, sizeof(res), cudaMemcpyHostToDevice, ctx->st));
  } else {
    std::copy(res, res + 4, out);
  }
  return finish(ctx, GW_OK);
}

gw_status gw_set_precond(gw_ctx* ctx, int kind) {
  if (!ctx) return GW_E_ARG;
  if (kind != 0 && kind != 1) return fail(ctx, GW_E_ARG, "preconditioner kind must be 0 (none) or 1 (kinetic)");
  ctx->precond = kind;
  return GW_OK;
}

gw_status gw_profile(gw_ctx* ctx, unsigned mask) {
  if (!ctx) return GW_E_ARG;
  ctx->prof_mask = mask & ((1u << PC_N) - 1u);
  ctx->ev_used.clear();
  ctx->ev_next = 0;
  return GW_OK;
}

gw_status gw_profile_read(gw_ctx* ctx, double* ms, long long* count, int n) {
  if (!ctx || !ms || !count || n < 0) return GW_E_ARG;
  CK(cudaStreamSynchronize(ctx->st));
  for (int i = 0; i < n; ++i) { ms[i] = 0.0; count[i] = 0; }
  for (auto& u : ctx->ev_used) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, ctx->ev_pool[u.second.first], ctx->ev_pool[u.second.second]));
    if (u.first < n) { ms[u.first] += t; count[u.first] += 1; }
  }
  ctx->ev_used.clear();
  ctx->ev_next = 0;
  if (ctx->ptask && n > PC_TASKS + 6) {
    unsigned long long h[36];
    CK(cudaMemcpy(h, ctx->ptask, sizeof(h), cudaMemcpyDeviceToHost));
    CK(cudaMemset(ctx->ptask, 0, sizeof(h)));
    for (int k = 0; k < 3; ++k) {
      ms[PC_TASKS + 1 + 2 * k] = 1e-6 * (double)h[12 * k + 1];      // busy
      count[PC_TASKS + 1 + 2 * k] = (long long)h[12 * k + 0];
      ms[PC_TASKS + 2 + 2 * k] = 1e-6 * (double)h[12 * k + 2];      // waiting
      count[PC_TASKS + 2 + 2 * k] = (long long)h[12 * k + 3];
      for (int j = 0; j < 4; ++j)                                      // sub-phases
        if (n > PC_TASKS + 7 + 4 * k + j) ms[PC_TASKS + 7 + 4 * k + j] = 1e-6 * (double)h[12 * k + 4 + j];
    }
  }
  return GW_OK;
}

const char* gw_last_error(const gw_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void gw_destroy(gw_ctx* ctx) {
  if (!ctx) return;
  if (ctx->st) cudaStreamSynchronize(ctx->st);
  for (auto& kv : ctx->bufs)
    if (kv.second.first) cudaFree(kv.second.first);
  if (ctx->host_pin) cudaFreeHost(ctx->host_pin);
  if (ctx->stage) cudaFreeHost(ctx->stage);
  if (ctx->pcg_pin) cudaFreeHost(ctx->pcg_pin);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  for (cudaEvent_t e : ctx->tune_ev)
    if (e) cudaEventDestroy(e);
  if (ctx->ev) cudaEventDestroy(ctx->ev);
  if (ctx->st && ctx->own_stream) cudaStreamDestroy(ctx->st);
  delete ctx;
}

}  // extern "C"

namespace gw {
bool make_plan(int N, FftPlan* p) {
  if (N < 2 || N > kMaxN) return false;
  p->N = N;
  p->nst = 0;
  int m = N;
  const int order[4] = {4, 2, 3, 5};
  for (int r : order) {
    while (m % r == 0) {
      if (p->nst >= kMaxStages) return false;
      p->rad[p->nst++] = r;
      m /= r;
    }
  }
  if (m != 1) return false;
  p->dN.set(N);
  int span = 1;
  for (int s = 0; s < p->nst; ++s) {
    p->nb[s] = N / p->rad[s];
    p->ns[s] = span;
    p->dnb[s].set(p->nb[s]);
    p->dns[s].set(span);
    span *= p->rad[s];
  }
  return true;
}
}  // namespace gw

// Batch mode: contexts that share the GPU concurrently cap their persistent
// grids at 1/n of the resident slots (see launch_cg_persistent).
void gw_internal_set_cta_div(gw_ctx* ctx, int n) {
  if (ctx) ctx->cta_div = n < 1 ? 1 : n;
}
