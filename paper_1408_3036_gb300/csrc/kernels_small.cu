// Small dense FP64 algebra for the recycled per-state bases of the dielectric
// matrix at imaginary frequencies (Sec. "Calculating the dielectric matrix and
// the integrand at different frequencies", Eq. recy_eq): row normalisation of
// the recycled vectors, a batched symmetric eigensolver (parallel two-sided
// Jacobi), batched products of small matrices, the orthonormalising transform
// and the final quadratic forms.  One CTA per matrix; matrices row-major.
#include <algorithm>
#include <cmath>

#include "gw_common.cuh"
#include "linalg.cuh"

namespace gw {

namespace {
constexpr int kST = 256;   // threads per CTA

__device__ __forceinline__ double sum_block_all(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];   // every thread, same order
  __syncthreads();
  return r;
}
}  // namespace

// rows[j] /= |rows[j]| (complex sphere vectors of length n); a zero row stays zero
__global__ void __launch_bounds__(kST) k_normalize_rows(double2* __restrict__ rows, size_t n) {
  __shared__ double sh[32];
  double2* r = rows + (size_t)blockIdx.x * n;
  double acc = 0.0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) acc += r[i].x * r[i].x + r[i].y * r[i].y;
  const double nrm = sqrt(sum_block_all(acc, sh));
  if (!(nrm > 0.0)) return;
  const double s = 1.0 / nrm;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) r[i] = make_double2(r[i].x * s, r[i].y * s);
}

void launch_normalize_rows(cudaStream_t s, double2* rows, int nrows, size_t n) {
  if (nrows == 0) return;
  ++g_launches;
  k_normalize_rows<<<nrows, kST, 0, s>>>(rows, n);
}

// dst[b][i][j] = Re src[b][i][j]
__global__ void k_real_part(size_t n, const double2* __restrict__ src, double* __restrict__ dst) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[i].x;
}

void launch_real_part(cudaStream_t s, size_t n, const double2* src, double* dst) {
  ++g_launches;
  k_real_part<<<(int)std::min<size_t>((n + kST - 1) / kST, 152 * 8), kST, 0, s>>>(n, src, dst);
}

// A[b] = (A[b] + A[b]^T) / 2 (Gram and Hamiltonian matrices symmetric up to rounding)
__global__ void k_symmetrize(int m, double* __restrict__ Ab) {
  double* A = Ab + (size_t)blockIdx.x * m * m;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e - i * m;
    if (i < j) {
      const double a = 0.5 * (A[(size_t)i * m + j] + A[(size_t)j * m + i]);
      A[(size_t)i * m + j] = a;
      A[(size_t)j * m + i] = a;
    }
  }
}

void launch_symmetrize(cudaStream_t s, int nb, int m, double* A) {
  if (nb == 0) return;
  ++g_launches;
  k_symmetrize<<<nb, kST, 0, s>>>(m, A);
}

// Parallel two-sided Jacobi for symmetric m x m matrices (one CTA per matrix,
// blockIdx.x = batch index): A <- J^T A J with m/2 disjoint rotations per
// step in round-robin order (m - 1 steps per sweep, m padded to even), each
// rotation chosen to zero a_pq (Golub and Van Loan, Sec. 8.5, symmetric
// Schur decomposition), V <- V J.  Sweeps until the off-diagonal Frobenius
// norm is below tol times the Frobenius norm, at most max_sweeps.  On return
// A holds the eigenvalues on its diagonal, V the eigenvectors in its columns;
// sweeps[b] receives the sweeps run (max_sweeps + 1 when not converged).
__global__ void __launch_bounds__(kST)
k_jacobi_sym(int m, double* __restrict__ Ab, double* __restrict__ Vb, double tol, int max_sweeps,
             int* __restrict__ sweeps) {
  extern __shared__ double smj[];
  const int me = m + (m & 1);                 // even number of players (m odd: one bye)
  double* cs = smj;                           // [me/2] cos
  double* sn = cs + me / 2;                   // [me/2] sin
  int* pp = reinterpret_cast<int*>(sn + me / 2);   // [me/2] p of each pair
  int* qq = pp + me / 2;                      // [me/2] q
  __shared__ double sh[32];
  double* A = Ab + (size_t)blockIdx.x * m * m;
  double* V = Vb + (size_t)blockIdx.x * m * m;
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) V[i] = (i / m == i % m) ? 1.0 : 0.0;
  __syncthreads();
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = threadIdx.x; i < m * m; i += blockDim.x) {
      const double a = A[i];
      tot += a * a;
      if (i / m != i % m) off += a * a;
    }
    off = sum_block_all(off, sh);
    tot = sum_block_all(tot, sh);
    if (off <= tol * tol * tot || off == 0.0) break;
    for (int step = 0; step < me - 1; ++step) {
      // round-robin pairing: player 0 fixed, the others rotate
      for (int k = threadIdx.x; k < me / 2; k += blockDim.x) {
        auto pos = [&](int x) { return x == 0 ? 0 : 1 + ((x - 1 + step) % (me - 1)); };
        int p = pos(k), q = pos(me - 1 - k);
        if (p > q) { const int t = p; p = q; q = t; }
        pp[k] = p;
        qq[k] = q;
        double c = 1.0, s = 0.0;
        if (q < m) {
          const double apq = A[(size_t)p * m + q];
          if (apq != 0.0) {
            const double tau = (A[(size_t)q * m + q] - A[(size_t)p * m + p]) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        }
        cs[k] = c;
        sn[k] = s;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int e = threadIdx.x; e < (me / 2) * m; e += blockDim.x) {
        const int k = e / m, r = e - k * m;
        const int p = pp[k], q = qq[k];
        if (q >= m || sn[k] == 0.0) continue;
        const double c = cs[k], s = sn[k];
        double* ar = A + (size_t)r * m;
        const double ap = ar[p], aq = ar[q];
        ar[p] = c * ap - s * aq;
        ar[q] = s * ap + c * aq;
        double* vr = V + (size_t)r * m;
        const double vp = vr[p], vq = vr[q];
        vr[p] = c * vp - s * vq;
        vr[q] = s * vp + c * vq;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int e = threadIdx.x; e < (me / 2) * m; e += blockDim.x) {
        const int k = e / m, r = e - k * m;
        const int p = pp[k], q = qq[k];
        if (q >= m || sn[k] == 0.0) continue;
        const double c = cs[k], s = sn[k];
        const double ap = A[(size_t)p * m + r], aq = A[(size_t)q * m + r];
        A[(size_t)p * m + r] = c * ap - s * aq;
        A[(size_t)q * m + r] = s * ap + c * aq;
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) sweeps[blockIdx.x] = sweep < max_sweeps ? sweep : max_sweeps + 1;
}

cudaError_t launch_jacobi_sym(cudaStream_t s, int nb, int m, double* A, double* V, double tol, int max_sweeps,
                              int* sweeps) {
  if (nb == 0 || m == 0) return cudaSuccess;
  const int me = m + (m & 1);
  const size_t sm = (size_t)me * sizeof(double) + (size_t)me * sizeof(int);
  if (sm > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k_jacobi_sym, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  ++g_launches;
  k_jacobi_sym<<<nb, kST, sm, s>>>(m, A, V, tol, max_sweeps, sweeps);
  return cudaGetLastError();
}

// C[b] = op(A[b]) op(B[b]); op(A) is r x k (A stored r x k, or k x r when ta),
// op(B) is k x c (B stored k x c, or c x k when tb); 16 x 16 output tiles,
// grid (ceil(c / 16), ceil(r / 16), nb)
__global__ void k_gemm_small(int r, int k, int c, const double* __restrict__ Ab, int ta, const double* __restrict__ Bb,
                             int tb, double* __restrict__ Cb) {
  const int b = blockIdx.z;
  const double* A = Ab + (size_t)b * r * k;
  const double* B = Bb + (size_t)b * k * c;
  double* C = Cb + (size_t)b * r * c;
  const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
  __shared__ double As[16][17], Bs[16][17];
  double acc = 0.0;
  for (int k0 = 0; k0 < k; k0 += 16) {
    const int ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
    As[threadIdx.y][threadIdx.x] = (i < r && ka < k) ? (ta ? A[(size_t)ka * r + i] : A[(size_t)i * k + ka]) : 0.0;
    Bs[threadIdx.y][threadIdx.x] = (kb < k && j < c) ? (tb ? B[(size_t)j * k + kb] : B[(size_t)kb * c + j]) : 0.0;
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 16; ++t) acc += As[threadIdx.y][t] * Bs[t][threadIdx.x];
    __syncthreads();
  }
  if (i < r && j < c) C[(size_t)i * c + j] = acc;
}

void launch_gemm_small(cudaStream_t s, int nb, int r, int k, int c, const double* A, int ta, const double* B, int tb,
                       double* C) {
  if (nb == 0 || r == 0 || c == 0) return;
  ++g_launches;
  k_gemm_small<<<dim3((c + 15) / 16, (r + 15) / 16, nb), dim3(16, 16), 0, s>>>(r, k, c, A, ta, B, tb, C);
}

// T[b] = W[b] diag(t), t_j = s_j^-1/2 for s_j > rel * max_j s_j, else 0 (the
// eigenvalues s of the Gram matrix on the diagonal of S[b]); kept[b] counts them
__global__ void __launch_bounds__(kST)
k_orth_transform(int m, const double* __restrict__ Sb, const double* __restrict__ Wb, double rel,
                 double* __restrict__ Tb, int* __restrict__ kept) {
  __shared__ double smax;
  const double* S = Sb + (size_t)blockIdx.x * m * m;
  const double* W = Wb + (size_t)blockIdx.x * m * m;
  double* T = Tb + (size_t)blockIdx.x * m * m;
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int j = 0; j < m; ++j) mx = fmax(mx, S[(size_t)j * m + j]);
    smax = mx;
    int n = 0;
    for (int j = 0; j < m; ++j) n += (S[(size_t)j * m + j] > rel * mx) ? 1 : 0;
    kept[blockIdx.x] = n;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int j = e % m;
    const double sj = S[(size_t)j * m + j];
    T[e] = (sj > rel * smax) ? W[e] / sqrt(sj) : 0.0;
  }
}

void launch_orth_transform(cudaStream_t s, int nb, int m, const double* S, const double* W, double rel, double* T,
                           int* kept) {
  if (nb == 0) return;
  ++g_launches;
  k_orth_transform<<<nb, kST, 0, s>>>(m, S, W, rel, T, kept);
}

// out[o][l][l'] = 4 sum_b sum_i c[b][i][l] g(lambda[b][i], w_o) c[b][i][l'],
// g = lambda / (lambda^2 + w^2) (0 for lambda = 0: a dropped direction);
// lambda on the diagonal of L[b] (m x m), c[b] m x nl; grid (nl, nl, nw)
__global__ void __launch_bounds__(kST)
k_recycled_form(int nbat, int m, int nl, const double* __restrict__ Lb, const double* __restrict__ cb,
                const double* __restrict__ w, double* __restrict__ out) {
  __shared__ double sh[32];
  const int l = blockIdx.x, lp = blockIdx.y, o = blockIdx.z;
  const double w2 = w[o] * w[o];
  double acc = 0.0;
  for (int e = threadIdx.x; e < nbat * m; e += blockDim.x) {
    const int b = e / m, i = e - b * m;
    const double lam = Lb[(size_t)b * m * m + (size_t)i * m + i];
    const double den = lam * lam + w2;
    if (den == 0.0) continue;
    const double* c = cb + (size_t)b * m * nl + (size_t)i * nl;
    acc += c[l] * (lam / den) * c[lp];
  }
  acc = sum_block_all(acc, sh);
  if (threadIdx.x == 0) out[((size_t)o * nl + l) * nl + lp] = 4.0 * acc;
}

void launch_recycled_form(cudaStream_t s, int nbat, int m, int nl, int nw, const double* L, const double* c,
                          const double* w, double* out) {
  if (nl == 0 || nw == 0) return;
  ++g_launches;
  k_recycled_form<<<dim3(nl, nl, nw), kST, 0, s>>>(nbat, m, nl, L, c, w, out);
}

// out[b] = V[b] f(L[b]) V[b]^T for symmetric matrices diagonalised by
// k_jacobi_sym (eigenvalues on the diagonal of L[b], eigenvectors in the
// columns of V[b]); f(x) = 1/x - 1 (mode 0: eps^-1 - 1 from eps)
__global__ void k_eig_function(int m, const double* __restrict__ Lb, const double* __restrict__ Vb, int mode,
                               double* __restrict__ out) {
  const double* L = Lb + (size_t)blockIdx.x * m * m;
  const double* V = Vb + (size_t)blockIdx.x * m * m;
  double* O = out + (size_t)blockIdx.x * m * m;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e - i * m;
    double acc = 0.0;
    for (int k = 0; k < m; ++k) {
      const double lam = L[(size_t)k * m + k];
      const double f = (mode == 0) ? 1.0 / lam - 1.0 : lam;
      acc += V[(size_t)i * m + k] * f * V[(size_t)j * m + k];
    }
    O[e] = acc;
  }
}

void launch_eig_function(cudaStream_t s, int nb, int m, const double* L, const double* V, int mode, double* out) {
  if (nb == 0) return;
  ++g_launches;
  k_eig_function<<<nb, kST, 0, s>>>(m, L, V, mode, out);
}

// A[b] += diag(1)
__global__ void k_add_identity(int m, double* __restrict__ Ab) {
  double* A = Ab + (size_t)blockIdx.x * m * m;
  for (int i = threadIdx.x; i < m; i += blockDim.x) A[(size_t)i * m + i] += 1.0;
}

void launch_add_identity(cudaStream_t s, int nb, int m, double* A) {
  if (nb == 0) return;
  ++g_launches;
  k_add_identity<<<nb, kST, 0, s>>>(m, A);
}

// Shift-Lanczos quadrature of <z_l| g(H - c, w) |z_l'>, g(h) = h / (w^2 + h^2):
// out[o] = R^T U1 g(Theta, w_o) U1^T R with Theta on the diagonal of L (m x m,
// from k_jacobi_sym), U1 the first b rows of U, R (b x b); grid nw, one CTA
// per frequency; scratch G [nw][b][b]
__global__ void __launch_bounds__(kST)
k_shift_quadrature(int m, int b, const double* __restrict__ L, const double* __restrict__ U,
                   const double* __restrict__ R, const double* __restrict__ w, double* __restrict__ G,
                   double* __restrict__ out) {
  const int o = blockIdx.x;
  const double w2 = w[o] * w[o];
  double* Go = G + (size_t)o * b * b;
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e - i * b;
    double acc = 0.0;
    for (int k = 0; k < m; ++k) {
      const double th = L[(size_t)k * m + k];
      const double den = w2 + th * th;
      if (den == 0.0) continue;
      acc += U[(size_t)i * m + k] * (th / den) * U[(size_t)j * m + k];
    }
    Go[e] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e - i * b;
    double acc = 0.0;
    for (int p = 0; p < b; ++p)
      for (int q = 0; q < b; ++q) acc += R[(size_t)p * b + i] * Go[(size_t)p * b + q] * R[(size_t)q * b + j];
    out[(size_t)o * b * b + e] = acc;
  }
}

void launch_shift_quadrature(cudaStream_t s, int m, int b, const double* L, const double* U, const double* R,
                             const double* w, int nw, double* G, double* out) {
  if (nw == 0) return;
  ++g_launches;
  k_shift_quadrature<<<nw, kST, 0, s>>>(m, b, L, U, R, w, G, out);
}

// P_e part of Eq. khe in closed form on the occupied states below c:
// out[l][l'] = sum_{v: e_v < c} Re(conj(a[v][l]) a[v][l']) alpha / (e_v - c - alpha)
__global__ void k_pe_form(int nocc, int nl, const double2* __restrict__ a, const double* __restrict__ eps, double c,
                          double alpha, double* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nl * nl; e += gridDim.x * blockDim.x) {
    const int l = e / nl, lp = e - l * nl;
    double acc = 0.0;
    for (int v = 0; v < nocc; ++v) {
      if (!(eps[v] < c)) continue;
      const double2 x = a[(size_t)v * nl + l], y = a[(size_t)v * nl + lp];
      acc += (x.x * y.x + x.y * y.y) * alpha / (eps[v] - c - alpha);
    }
    out[e] = acc;
  }
}

void launch_pe_form(cudaStream_t s, int nocc, int nl, const double2* a, const double* eps, double c, double alpha,
                    double* out) {
  ++g_launches;
  k_pe_form<<<1, kST, 0, s>>>(nocc, nl, a, eps, c, alpha, out);
}

// out[j] = sum_e (A[ia[j]] - fa[j] B[ib[j]])[e] C[ic[j]][e] over n entries (Frobenius forms)
__global__ void __launch_bounds__(kST)
k_frob_forms(int n, const double* __restrict__ A, const int* __restrict__ ia, const double* __restrict__ fa,
             const double* __restrict__ B, const int* __restrict__ ib, const double* __restrict__ C,
             const int* __restrict__ ic, double* __restrict__ out) {
  __shared__ double sh[32];
  const int j = blockIdx.x;
  const double* a = A + (size_t)ia[j] * n;
  const double* bb = B + (size_t)ib[j] * n;
  const double* cc = C + (size_t)ic[j] * n;
  const double f = fa[j];
  double acc = 0.0;
  for (int e = threadIdx.x; e < n; e += blockDim.x) acc += (a[e] - f * bb[e]) * cc[e];
  acc = sum_block_all(acc, sh);
  if (threadIdx.x == 0) out[j] = acc;
}

void launch_frob_forms(cudaStream_t s, int nj, int n, const double* A, const int* ia, const double* fa,
                       const double* B, const int* ib, const double* C, const int* ic, double* out) {
  if (nj == 0) return;
  ++g_launches;
  k_frob_forms<<<nj, kST, 0, s>>>(n, A, ia, fa, B, ib, C, ic, out);
}

}  // namespace gw
