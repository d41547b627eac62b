// Projector coefficients on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// The conduction projector of the Sternheimer solvers (Sec. Avoiding
// summations: orthogonalise to the valence space at every step) needs, for
// every solver column y_j, the coefficients coef[v][j] = <C_v|y_j> =
// sum_G conj(C_v(G)) y_j(G).  With many columns (the block, complex-frequency
// workload: 64 occupied states x 2 signs x 8 fields = 1024 columns) this is a
// dense contraction over the sphere, written here as one real GEMM
//   D[m][n] = sum_k A[m][k] B[n][k],   k = 2 G + {0: Re, 1: Im}
//   A[v][k]      = (Re C_v(G), Im C_v(G))      -> Re coef
//   A[64 + v][k] = (-Im C_v(G), Re C_v(G))     -> Im coef
//   B[j][k]      = (Re y_j(G), Im y_j(G))       (the FP32 column as stored)
// with M = 128 rows (up to 64 occupied states), N = 128 columns per CTA, K
// split over CTAs so that one wave covers the SMs.
//
// Precision: kind::tf32 MMAs with FP32 accumulation in tensor memory, and the
// operands split as x = hi + lo, hi = x rounded to the nearest TF32 value (10
// explicit mantissa bits), lo = x - hi (|lo| <= 2^-11 |x|) rounded to TF32 in
// turn, so that hi + lo meets x to 2^-22 relative; the MMA reads only the TF32
// bits of its operands, and a truncated split (hi with the low bits cleared)
// would leave a lo of up to 2^-10 |x| truncated again, 2^-20 relative.
// D = A_hi B_hi + A_hi B_lo + A_lo B_hi (the dropped A_lo B_lo term is 2^-22
// relative).  A (static: the occupied rows) is split once on the host; each B
// tile is split in shared memory after it is loaded.  Measured against the
// CUDA-core FP32 dots the coefficients still differ by about 2e-6 of the
// largest (1e-7 would be FP32 rounding): the accumulation in tensor memory
// over the CTA's K blocks dominates, not the split (rounding instead of
// truncating it changed 2.6e-6 to 2.2e-6).
//
// Data movement: the A tiles (128 rows x 32 FP32 = one 128-byte swizzle row
// per row) arrive by TMA (cp.async.bulk.tensor, 128-byte swizzle) on an
// mbarrier; the B rows start at an 8-byte boundary only (odd sphere sizes), so
// the CTA loads them with ordinary 8-byte loads and stores hi and lo into the
// same swizzled layout; one elected thread issues the MMAs (12 per 32-element
// K block: 4 K=8 steps x 3 products) and commits them to the stage's
// mbarrier, which frees the stage for the next loads.  Every wait is bounded:
// a wait that runs out sets the error flag, the CTA stops issuing work, waits
// (bounded) for its issued MMAs, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "gw_common.cuh"
#include "linalg.cuh"

namespace gw {

namespace {

constexpr int kTcM = 128;          // rows of A (Re and Im rows of up to 64 occupied states)
constexpr int kTcN = 128;          // solver columns per CTA
constexpr int kTcK = 32;           // FP32 elements of K per stage: one 128-byte swizzle row
constexpr int kTcStages = 3;
constexpr int kTcThreads = 128;
constexpr int kTileBytes = kTcM * kTcK * 4;            // 16 KB (A and B tiles alike: 128 rows)
constexpr int kStageBytes = 4 * kTileBytes;            // A_hi, A_lo, B_hi, B_lo
constexpr size_t kTcSmem = (size_t)kTcStages * kStageBytes + 1024 + 256;
constexpr uint32_t kTmemCols = 128;

// Instruction descriptor of tcgen05.mma kind::tf32: D in FP32 (bits 4-5 = 1),
// A and B TF32 (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                            ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of a K-major tile in the 128-byte swizzle
// layout: rows of 128 bytes, 8-row groups 1024 bytes apart (stride byte
// offset), leading byte offset unused within one swizzle row (1), version 1,
// layout type 2 (128-byte swizzle).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t a) {
  uint64_t d = 0;
  d |= (uint64_t)((a & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
}

// Bounded wait for the phase of the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned long long limit) {
  for (unsigned long long i = 0; i < limit; ++i) {
    uint32_t ok = 0;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          saddr(dst)),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(saddr(bar))
      : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          dtmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// The TF32 value nearest to x (ties away from zero): the magnitude bits
// rounded at the 13th mantissa bit, which stays within the exponent field's
// carry for finite x.
__device__ __forceinline__ float tf32_round(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// Byte offset of the 8-byte element q (0..15) of row n in a 128-byte-swizzled tile.
__device__ __forceinline__ uint32_t sw_off(int n, int q) {
  const uint32_t ob = (uint32_t)q * 8u;
  return (uint32_t)n * 128u + ((((ob >> 4) ^ (uint32_t)(n & 7)) << 4) | (ob & 15u));
}

}  // namespace

// part[ks][m][j] (FP32) = sum over this CTA's K blocks of D[m][j]; grid
// (ceil(ncol / 128), nks); K blocks [ks kb_per, min(nkb, (ks + 1) kb_per)).
__global__ void __launch_bounds__(kTcThreads, 1)
k_tc_dots(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
          const float2* __restrict__ Y, int npw, int ncol, int nkb, int kb_per, float* __restrict__ part,
          int* __restrict__ err, unsigned long long limit) {
  extern __shared__ unsigned char sm_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(sm_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + (size_t)kTcStages * kStageBytes);
  uint64_t* empty = full + kTcStages;
  uint64_t* done = empty + kTcStages;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int n0 = blockIdx.x * kTcN;
  const int kb0 = blockIdx.y * kb_per, kb1 = min(nkb, kb0 + kb_per);
  if (tid == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  int issued = 0;
  for (int kb = kb0, it = 0; kb < kb1; ++kb, ++it) {
    const int s = it % kTcStages;
    const uint32_t ph = (uint32_t)((it / kTcStages) & 1);
    unsigned char* Ahi = sm + (size_t)s * kStageBytes;
    unsigned char* Alo = Ahi + kTileBytes;
    unsigned char* Bhi = Alo + kTileBytes;
    unsigned char* Blo = Bhi + kTileBytes;
    if (it >= kTcStages) {                // the MMAs that read this stage have finished
      if (!mbar_wait(&empty[s], ph ^ 1u, limit)) atomicExch(&abort_flag, 1);
    }
    __syncthreads();
    if (abort_flag) break;
    if (tid == 0) {
      mbar_expect_tx(&full[s], 2 * kTileBytes);
      tma_load_2d(Ahi, &mAhi, kb * kTcK, 0, &full[s]);
      tma_load_2d(Alo, &mAlo, kb * kTcK, 0, &full[s]);
    }
    // B: rows n (solver columns n0 + n), 16 complex entries G = 16 kb + q each
    const int g0 = kb * (kTcK / 2);
#pragma unroll 4
    for (int e = tid; e < kTcN * (kTcK / 2); e += kTcThreads) {
      const int n = e >> 4, q = e & 15;
      const int j = n0 + n, G = g0 + q;
      float2 v = make_float2(0.f, 0.f);
      if (j < ncol && G < npw) v = Y[(size_t)j * npw + G];
      const float2 hi = make_float2(tf32_round(v.x), tf32_round(v.y));
      const float2 lo = make_float2(tf32_round(v.x - hi.x), tf32_round(v.y - hi.y));
      const uint32_t off = sw_off(n, q);
      *reinterpret_cast<float2*>(Bhi + off) = hi;
      *reinterpret_cast<float2*>(Blo + off) = lo;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      if (!mbar_wait(&full[s], ph, limit)) {
        atomicExch(&abort_flag, 1);
      } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ah = saddr(Ahi), al = saddr(Alo), bh = saddr(Bhi), bl = saddr(Blo);
#pragma unroll
        for (int kk = 0; kk < kTcK / 8; ++kk) {
          const uint32_t o = (uint32_t)kk * 32u;        // K = 8 TF32 = 32 bytes per MMA
          mma_tf32(tmem, sw128_desc(ah + o), sw128_desc(bh + o), (it > 0 || kk > 0) ? 1u : 0u);
          mma_tf32(tmem, sw128_desc(ah + o), sw128_desc(bl + o), 1u);
          mma_tf32(tmem, sw128_desc(al + o), sw128_desc(bh + o), 1u);
        }
        mma_commit(&empty[s]);
        issued = 1;
      }
    }
  }
  // all issued MMAs complete (bounded), then the accumulator leaves tensor memory
  __syncthreads();
  if (tid == 0) {
    mma_commit(done);       // arrives once every earlier MMA of this thread has completed
    if (!mbar_wait(done, 0, limit)) atomicExch(&abort_flag, 1);
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  (void)issued;
  if (!abort_flag && kb1 > kb0) {
    const int m = warp * 32 + (tid & 31);         // tensor-memory lane = row of D
    float* prow = part + ((size_t)blockIdx.y * kTcM + m) * ncol;
#pragma unroll 1
    for (int c0 = 0; c0 < kTcN; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int j = n0 + c0 + i;
        if (j < ncol) prow[j] = v[i];
      }
    }
  }
  if (abort_flag && tid == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// coef[v * ncol + j] = (sum_ks part[ks][v][j], sum_ks part[ks][64 + v][j]) in FP64, ks in order
__global__ void k_tc_reduce(const float* __restrict__ part, int nks, int nocc, int ncol, double2* __restrict__ coef) {
  const size_t n = (size_t)nocc * ncol;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int v = (int)(i / ncol), j = (int)(i - (size_t)v * ncol);
    double re = 0.0, im = 0.0;
    for (int ks = 0; ks < nks; ++ks) {
      const float* p = part + (size_t)ks * kTcM * ncol;
      re += (double)p[(size_t)v * ncol + j];
      im += (double)p[(size_t)(64 + v) * ncol + j];
    }
    coef[i] = make_double2(re, im);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

bool make_map(CUtensorMap* map, const float* base, int kpad) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)kTcM};
  const cuuint64_t strides[1] = {(cuuint64_t)kpad * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kTcK, (cuuint32_t)kTcM};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int tc_kpad(int npw) { return (2 * npw + kTcK - 1) / kTcK * kTcK; }

// A_hi, A_lo [128][kpad] from the occupied rows C [nocc][npw] (FP64), nocc <= 64.
void tc_split_rows(const std::vector<double2>& C, int nocc, int npw, std::vector<float>* hi, std::vector<float>* lo) {
  const int kpad = tc_kpad(npw);
  hi->assign((size_t)kTcM * kpad, 0.f);
  lo->assign((size_t)kTcM * kpad, 0.f);
  auto round_tf32 = [](float f) {   // as tf32_round on the device
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;
    std::memcpy(&f, &u, 4);
    return f;
  };
  auto put = [&](int m, int k, double x) {
    const float h = round_tf32((float)x);
    (*hi)[(size_t)m * kpad + k] = h;
    (*lo)[(size_t)m * kpad + k] = round_tf32((float)(x - (double)h));
  };
  for (int v = 0; v < nocc; ++v)
    for (int G = 0; G < npw; ++G) {
      const double2 c = C[(size_t)v * npw + G];
      put(v, 2 * G, c.x);
      put(v, 2 * G + 1, c.y);
      put(64 + v, 2 * G, -c.y);
      put(64 + v, 2 * G + 1, c.x);
    }
}

cudaError_t tc_maps(const float* Ahi, const float* Alo, int npw, TcMaps* maps) {
  const int kpad = tc_kpad(npw);
  static_assert(sizeof(CUtensorMap) <= sizeof(maps->hi), "tensor map storage");
  if (!make_map(reinterpret_cast<CUtensorMap*>(maps->hi), Ahi, kpad) ||
      !make_map(reinterpret_cast<CUtensorMap*>(maps->lo), Alo, kpad))
    return cudaErrorNotSupported;
  maps->kpad = kpad;
  return cudaSuccess;
}

namespace {
// K splits for one wave over the SMs: (number of splits, K blocks per split)
void tc_split(int npw, int ncol, int* nks, int* kb_per) {
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int nkb = tc_kpad(npw) / kTcK;
  const int ntile = (ncol + kTcN - 1) / kTcN;
  int k = std::max(1, std::min(nkb, (nsm + ntile - 1) / ntile));
  *kb_per = (nkb + k - 1) / k;
  *nks = (nkb + *kb_per - 1) / *kb_per;      // every split gets at least one K block
}
}  // namespace

size_t tc_part_elems(int npw, int ncol) {
  int nks = 1, kb_per = 1;
  tc_split(npw, ncol, &nks, &kb_per);
  return (size_t)nks * kTcM * ncol;
}

cudaError_t tc_prepare() {
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(k_tc_dots, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
  });
  return attr;
}

cudaError_t launch_tc_dots(cudaStream_t s, const TcMaps& maps, const float2* Y, int npw, int ncol, int nocc,
                           float* part, double2* coef, int* err, unsigned long long limit) {
  if (nocc > 64 || ncol < 1) return cudaErrorInvalidValue;
  const int nkb = maps.kpad / kTcK;
  const int ntile = (ncol + kTcN - 1) / kTcN;
  int nks = 1, kb_per = 1;
  tc_split(npw, ncol, &nks, &kb_per);
  ++g_launches;
  k_tc_dots<<<dim3(ntile, nks), kTcThreads, kTcSmem, s>>>(*reinterpret_cast<const CUtensorMap*>(maps.hi),
                                                         *reinterpret_cast<const CUtensorMap*>(maps.lo), Y, npw,
                                                         ncol, nkb, kb_per, part, err, limit);
  ++g_launches;
  const size_t n = (size_t)nocc * ncol;
  k_tc_reduce<<<(int)std::min<size_t>((n + 255) / 256, 152 * 8), 256, 0, s>>>(part, nks, nocc, ncol, coef);
  return cudaGetLastError();
}

}  // namespace gw
