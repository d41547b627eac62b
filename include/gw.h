/*
 * libgw: the data-parallel hot path of the Lanczos-basis dielectric matrix
 * method for Sternheimer G0W0 (arXiv:1408.3036) on one NVIDIA GB300 (sm_103a).
 *
 * The library applies the independent-particle polarizability chi0(omega)
 * (Eq. P, computed through the Sternheimer equations Eqs. P1, fvpm, P2) and the
 * symmetric dielectric operator eps~(omega) = 1 - v^1/2 chi0(omega) v^1/2
 * (Eq. epsilon and its footnote) to batches of grid fields, runs the Lanczos
 * recursion with full Gram-Schmidt re-orthogonalisation that expresses eps~ in
 * a small basis (Sec. Lanczos, Eq. krylov), inverts the tridiagonal Lanczos
 * matrix (Sec. Lanczos, "inverted at a cost ~N^2"), and differentiates
 * s = <phi|eps~^-1(0)|phi> with respect to the local potential (not in the
 * paper; third-order perturbation theory).
 *
 * Units: Hartree atomic units.  Cell: cubic, edge L (bohr), volume Omega = L^3.
 * Grid: N^3 points r = L (i0, i1, i2) / N, C order [i0][i1][i2], N_g = N^3.
 * Plane waves: G = 2 pi n / L, n in FFT order; the basis is the sphere
 * |G|^2/2 <= ecut, ordered by ascending linear grid index of n mod N (see
 * gw_sphere).  A wavefunction with sphere coefficients c is
 * psi(r) = Omega^-1/2 sum_G c_G exp(i G r).  Grid inner product:
 * <f|g> = (Omega / N_g) sum_r conj(f) g.
 *
 * Ownership: the caller owns every buffer it passes; the library copies what
 * it keeps.  The library owns the context and its device workspaces.
 * Pointers: `device_ptrs = 0` means host memory; `device_ptrs = 1` means CUDA
 * device memory of the current device.  Complex numbers are interleaved
 * (re, im) doubles.  All calls are synchronous with respect to the host; the
 * work runs on the stream given at gw_setup (or a private one).
 *
 * Errors: every call returns a gw_status; nothing aborts.  gw_last_error()
 * returns a text for the last failure on a context.  On GW_E_NOCONV the
 * outputs are written (best iterate) and gw_stats reports the residuals.
 */
#ifndef GW_H
#define GW_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gw_ctx gw_ctx;

typedef enum {
  GW_OK = 0,
  GW_E_ARG = 1,          /* invalid argument (sizes, grid too small for the sphere, ...) */
  GW_E_CUDA = 2,         /* CUDA runtime error */
  GW_E_NOMEM = 3,        /* device allocation failed */
  GW_E_NOCONV = 4,       /* a Sternheimer solve did not reach its tolerance */
  GW_E_BREAKDOWN = 5,    /* Lanczos or CG breakdown (beta ~ 0, indefinite operator) */
  GW_E_TIMEOUT = 6,      /* a bounded device wait gave up (see gw_set_cg_kernel) */
  GW_E_NONFINITE = 7,    /* NaN or Inf in an input or a result */
  GW_E_UNSUPPORTED = 8   /* configuration the library does not handle */
} gw_status;

typedef enum {
  GW_FP64 = 0,   /* every step in FP64 */
  GW_MIXED = 1   /* FFTs, H and projector in FP32; FP64 outer Sternheimer residual,
                    FP64 Lanczos inner products and tridiagonal inverse */
} gw_prec;

typedef enum { GW_COULOMB_TRUNCATED = 0, GW_COULOMB_BARE = 1 } gw_coulomb;

/* Operator applied by the chi0 / eps~ / Lanczos entries (gw_set_operator). */
typedef enum {
  GW_OP_STERNHEIMER = 0,   /* chi0 through the Sternheimer equations (Eqs. P1, P2) */
  GW_OP_MODEL = 1          /* the model polarizability of Sec. Dielectric model (Eq. model_eq) */
} gw_operator;

/*
 * gw_setup -- create a context for one cell (Sec. Scaling: N_PW sphere
 * coefficients, N_FFT grid points; Sec. Results: spherical Coulomb truncation
 * with radius L/2).
 *   L        cell edge (bohr), > 0
 *   n_grid   FFT points per edge N, 4 <= N <= 128, factors 2, 3, 5 only
 *   ecut     plane-wave cutoff (Ha); the sphere must fit: 2 max|n| < N
 *   vloc     [N^3] local potential V(r) (Ha) on the grid, C order
 *   coulomb  GW_COULOMB_TRUNCATED: v(G) = 4 pi (1 - cos(|G| L/2)) / |G|^2,
 *            v(0) = pi L^2 / 2;  GW_COULOMB_BARE: 4 pi / |G|^2, v(0) = 0
 *   cuda_stream  caller stream (cudaStream_t): when non-NULL every kernel of the
 *            context runs on it (a stream that can be captured); when NULL the
 *            context creates a private blocking stream, ordered with the
 *            legacy default stream
 * Returns GW_E_ARG for bad sizes; *out is NULL on failure.
 */
gw_status gw_setup(gw_ctx** out, double L, int n_grid, double ecut, const double* vloc,
                   int coulomb, void* cuda_stream);

/* number of plane waves N_PW in the sphere (0 for a NULL context) */
int gw_npw(const gw_ctx* ctx);

/* miller[N_PW][3]: integer n (FFT order, signed) of each sphere coefficient */
gw_status gw_sphere(const gw_ctx* ctx, int* miller);

/*
 * gw_set_occupied -- the DFT input of the method (Eqs. P1, P2: occupied
 * states psi_v with energies e_v; each state holds two electrons).
 *   n_occ   1 <= n_occ <= 256
 *   psi     [n_occ][N_PW] complex sphere coefficients, orthonormal eigenvectors
 *           of H = |G|^2/2 + V_loc (the caller's ground state)
 *   eps     [n_occ] energies, ascending
 * The occupied space must be closed under complex conjugation (true when the
 * highest occupied state is separated from the next one).  The library
 * rotates each state to be real in real space (phase per state, real basis per
 * degenerate shell); results depend only on the occupied projector.
 * Host pointers only.  Returns GW_E_ARG if a state is not conjugation-closed.
 */
gw_status gw_set_occupied(gw_ctx* ctx, int n_occ, const double* psi, const double* eps);

/*
 * gw_set_deflation -- optional: the lowest n_def conduction states of the
 * same Hamiltonian (eigenpairs above the occupied ones, sphere order as in
 * gw_set_occupied, complete degenerate shells).  The Sternheimer solvers then
 * iterate on the complement of the occupied and these states and add the
 * latter's components exactly, x += sum_d D_d <D_d|b> / (e_d - e_v -/+ w), so
 * that the columns of the states nearest the gap need far fewer iterations;
 * the equations solved and the stopping test are unchanged (the FP64 residual
 * uses the occupied projector only).  Not in the paper, which uses no
 * conduction state at all.  n_def = 0 removes the block; gw_set_occupied
 * removes it too.  Host pointers.  GW_E_ARG without occupied states, for
 * energies below the highest occupied one, n_occ + n_def > 256, or a block
 * not closed under conjugation.
 */
gw_status gw_set_deflation(gw_ctx* ctx, int n_def, const double* psi, const double* eps);

/*
 * gw_apply_h -- y = H x for nb sphere vectors (the operator of Eq. P2:
 * kinetic |G|^2/2 plus V_loc applied on the grid through FFTs, Sec. Scaling).
 *   x, y  [nb][N_PW] complex
 */
gw_status gw_apply_h(gw_ctx* ctx, const double* x, int nb, double* y, gw_prec prec, int device_ptrs);

/*
 * gw_apply_chi0 -- dn = chi0(omega) dV for nb real fields and n_omega
 * frequencies (Eq. P through Eqs. P1 and P2: per occupied state one
 * Sternheimer solve at omega = 0, two (H - e_v -/+ omega) otherwise, projected
 * on the conduction space at every iteration).  omega = 0 uses conjugate
 * gradients; any other frequency, real (also above the excitation gap, where
 * H - e_v - omega is indefinite) or complex, uses simplified QMR with the
 * bilinear form sum_r x(r) y(r) (Sec. "Avoiding summations", SQMR footnote).
 *   dV     [nb][N^3] real
 *   omega  [n_omega] complex (interleaved re, im)
 *   dn     [n_omega][nb][N^3]: real when every omega is real, complex
 *          (interleaved) when one of them has a non-zero imaginary part
 */
gw_status gw_apply_chi0(gw_ctx* ctx, const double* dV, int nb, const double* omega, int n_omega,
                        double* dn, gw_prec prec, int device_ptrs);

/* gw_apply_eps -- out = eps~(omega) x = x - v^1/2 chi0(omega) v^1/2 x (Eq. epsilon);
   shapes and output type as gw_apply_chi0 (x: [nb][N^3] real). */
gw_status gw_apply_eps(gw_ctx* ctx, const double* x, int nb, const double* omega, int n_omega,
                       double* out, gw_prec prec, int device_ptrs);

/* gw_apply_chi0_c / gw_apply_eps_c -- the same on complex fields: input
   [nb][N^3] complex, output [n_omega][nb][N^3] complex (interleaved). */
gw_status gw_apply_chi0_c(gw_ctx* ctx, const double* dV, int nb, const double* omega, int n_omega,
                          double* dn, gw_prec prec, int device_ptrs);
gw_status gw_apply_eps_c(gw_ctx* ctx, const double* x, int nb, const double* omega, int n_omega,
                         double* out, gw_prec prec, int device_ptrs);

/*
 * gw_lanczos -- k steps of the Lanczos recursion on eps~(omega) (Sec. Lanczos,
 * Eq. krylov) from one real start field, with classical Gram-Schmidt applied
 * twice against all previous vectors at every step:
 *   q_1 = x0/|x0|;  w = eps~ q_k - beta_{k-1} q_{k-1};  alpha_k = <q_k|w>;
 *   w -= alpha_k q_k;  w -= Q (Q^T w) twice;  beta_k = |w|;  q_{k+1} = w / beta_k
 *   start   [N^3] real
 *   blk     block size, 1 (blocks: gw_block_lanczos)
 *   omega   real (imaginary part 0); complex frequencies: gw_block_lanczos
 *   alpha   [k] real;  beta [k-1] real
 *   basis   [k][N^3] real Lanczos vectors (orthonormal in <.|.>), or NULL
 * Returns GW_E_BREAKDOWN if beta_k underflows (invariant subspace reached).
 */
gw_status gw_lanczos(gw_ctx* ctx, const double* start, int blk, int k, const double* omega,
                     double* alpha, double* beta, double* basis, gw_prec prec, int device_ptrs);

/*
 * gw_lanczos_resume -- continue a real-frequency recursion of gw_lanczos from
 * a saved state (checkpoint/resume; not in the paper): the first k0 + 1
 * vectors and the coefficients of its first k0 steps, e.g. the output of a
 * gw_lanczos call with k0 + 1 steps.  Steps k0 .. k-1 then run as in
 * gw_lanczos (step k0 is recomputed from the saved vectors), so alpha and beta
 * equal those of an uninterrupted k-step run to rounding.
 *   basis_in  [k0 + 1][N^3] real: q_1 .. q_{k0+1}
 *   alpha_in  [k0] real;  beta_in [k0] real (beta_1 .. beta_k0)
 *   k0 >= 1, k > k0;  omega real (imaginary part 0)
 *   alpha     [k] real;  beta [k-1] real;  basis [k][N^3] or NULL
 * The saved state is checked before any step: coefficients finite, beta > 0,
 * vectors orthonormal in <.|.> to 1e-8; a state that fails returns GW_E_ARG
 * (a damaged checkpoint) and nothing is written.  With device_ptrs, basis may
 * equal basis_in (resumed in place; it must then hold k rows).
 */
gw_status gw_lanczos_resume(gw_ctx* ctx, const double* basis_in, const double* alpha_in, const double* beta_in,
                            int k0, int k, const double* omega, double* alpha, double* beta, double* basis,
                            gw_prec prec, int device_ptrs);

/*
 * gw_block_lanczos -- k block steps of the Lanczos recursion on eps~(omega)
 * from a block of blk real start fields (Sec. Lanczos; block form, with
 * classical Gram-Schmidt applied twice against all previous blocks):
 *   W = eps~ Q_k - Q_{k-1} B_{k-1}^(H/T);  A_k = <Q_k|W>;  W -= Q_k A_k
 *   W -= Q (Q^(H/T) W) twice;  W = Q_{k+1} B_k  (Cholesky of the Gram matrix)
 * At real omega the inner product is Hermitian and A_k is Hermitian; at complex
 * omega eps~ is complex symmetric and the recursion uses the bilinear form
 * sum_r x(r) y(r) (A_k symmetric), with principal square roots in the
 * factorisation.  Blocks are rows: vector j of block k is basis row k blk + j.
 *   start  [blk][N^3] real, linearly independent; 1 <= blk <= 16
 *   omega  complex (interleaved)
 *   A      [k][blk][blk] complex, A[k][i][j] = <q_i|eps~ q_j>
 *   B      [k-1][blk][blk] complex, upper triangular (B[k][i][j] = 0 for i > j)
 *   basis  [k blk][N^3] complex Lanczos vectors, or NULL
 * Returns GW_E_BREAKDOWN on rank loss (the outputs up to that step are valid).
 */
gw_status gw_block_lanczos(gw_ctx* ctx, const double* start, int blk, int k, const double* omega,
                           double* A, double* B, double* basis, gw_prec prec, int device_ptrs);

/*
 * gw_epsinv_block -- inverse of the block-tridiagonal Lanczos matrix T with
 * diagonal blocks A_k, B_k below and B_k^H (bilinear: B_k^T) above, i.e.
 * eps~^-1 in the block Lanczos basis, by Gauss-Jordan elimination with partial
 * pivoting on the GPU in FP64.
 *   A [k][blk][blk], B [k-1][blk][blk] complex (as from gw_block_lanczos)
 *   bilinear  1 for a complex-frequency (complex-symmetric) recursion
 *   out [k blk][k blk] complex;  k blk <= 2048
 */
gw_status gw_epsinv_block(gw_ctx* ctx, const double* A, const double* B, int k, int blk, int bilinear,
                          double* out, int device_ptrs);

/*
 * gw_epsinv_elements -- T_K^-1, the inverse dielectric matrix in the Lanczos
 * basis (Sec. Lanczos: tridiagonal inversion at cost ~K^2), in FP64.
 *   alpha [k], beta [k-1] real; out [k][k] real (symmetric)
 * Returns GW_E_BREAKDOWN for a zero pivot.
 */
gw_status gw_epsinv_elements(gw_ctx* ctx, const double* alpha, const double* beta, int k, int blk,
                             double* out, int device_ptrs);

/*
 * gw_epsinv_elements_noalloc -- the same T_K^-1 as gw_epsinv_elements, for
 * callers that cannot allocate device memory when they need it (their memory
 * is held by another allocator, or a cudaMalloc/cudaFree and its implicit
 * device synchronisation is not acceptable at that point).  The paper has no
 * counterpart: this is a deployment variant of the tridiagonal inverse.
 *   alpha [k], beta [k-1], out [k][k]: DEVICE pointers owned by the caller
 *   k         1 <= k <= 4096; larger k returns GW_E_ARG (use gw_epsinv_elements)
 *   cuda_stream  stream the work is ordered on (may be 0); the call returns
 *             after that stream has finished it
 * It needs no context and calls no cudaMalloc/cudaFree: its pivots,
 * multipliers and zero-pivot flag live in one fixed 64 KB __device__ array in
 * the library, which every GPU that loads the library keeps until the process
 * exits.  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress with the device current).  All calls on a device share the array:
 * calls that overlap on the GPU (other streams, other host threads) race and
 * must be serialised by the caller.  Returns GW_E_BREAKDOWN for a zero pivot.
 */
gw_status gw_epsinv_elements_noalloc(const double* alpha, const double* beta, int k, double* out,
                                     void* cuda_stream);

/*
 * gw_grad_vloc -- s = <phi|eps~^-1(0)|phi> and grad[i] = ds/dV_loc(r_i) (not in
 * the paper).  s and u = eps~^-1 phi come from k Lanczos steps started at phi;
 * the gradient follows third-order perturbation theory:
 *   w = v^1/2 u;  dpsi_v = -G_v P_c (w psi_v);  G_v = P_c (H - e_v)^-1 P_c
 *   g1 = sum_v |dpsi_v|^2 - sum_vv' <dpsi_v|dpsi_v'> psi_v'* psi_v
 *   lambda_v = G_v P_c [w dpsi_v - sum_v' <psi_v'|w|psi_v> dpsi_v']
 *   g2 = -sum_v lambda_v* psi_v;   grad = (Omega/N_g) (4 g1 + 8 Re g2)
 * i.e. one set of Sternheimer solves and one set of adjoint solves.
 *   phi [N^3] real; s scalar (host or device per device_ptrs); grad [N^3] real
 */
gw_status gw_grad_vloc(gw_ctx* ctx, const double* phi, int k, double* s, double* grad, gw_prec prec,
                       int device_ptrs);

/*
 * gw_grad_vloc_basis -- the same s and ds/dV_loc as gw_grad_vloc, from a
 * Lanczos basis the caller kept: basis [k][N^3], alpha [k], beta [k-1] as
 * returned by gw_lanczos(ctx, phi, 1, k, omega = 0, ...) on this context (the
 * checkpoint of a forward pass).  T^-1, s = |phi|^2 (T^-1)_11 and
 * u = |phi| sum_k q_k (T^-1)_k1 come from it; the first-order orbitals dpsi_v
 * and the adjoint solutions lambda_v are computed here and not kept, so a
 * caller that stores only the basis between a forward and a backward pass
 * holds k N^3 doubles, not the 2 n_occ N_PW complex orbitals as well.
 * Pointers all host or all device (device_ptrs).  GW_E_BREAKDOWN for a zero
 * pivot of T.
 */
gw_status gw_grad_vloc_basis(gw_ctx* ctx, const double* phi, const double* basis, const double* alpha,
                             const double* beta, int k, double* s, double* grad, gw_prec prec, int device_ptrs);

/*
 * gw_stats -- counters of the last solve on the context:
 *   out[0] Sternheimer columns solved, out[1] max inner iterations,
 *   out[2] mean inner iterations, out[3] outer (FP64 residual) passes,
 *   out[4] max final relative FP64 residual, out[5] H applications (columns),
 *   out[6] CUDA kernels launched by the library since it was loaded,
 *   out[7] iterations run by persistent CG launches (each launch counts the
 *          iterations of its slowest column)
 *   out[8] CTAs of the last persistent CG launch, out[9] its cluster size
 *          (0: the grid-wide cooperative kernel)
 *   out[10] CUDA-graph replays of SQMR iterations in the last SQMR solve
 *   out[11] threads per CTA of the last persistent CG launch (256 or 512)
 *   n: entries wanted (<= 12)
 */
gw_status gw_stats(const gw_ctx* ctx, double* out, int n);

/*
 * gw_set_autotune -- 1 (default): launch shapes that change speed only (the
 * persistent CG's CTA width: 256 threads, two CTAs per SM, or 512, one CTA per
 * SM) are chosen per problem shape by timing the first launches of each
 * candidate; the choice is kept for the process and written to a JSON cache
 * ($LIBGW_TUNE_CACHE, else $XDG_CACHE_HOME/libgw/tune.json, else
 * ~/.cache/libgw/tune.json) that later processes read.  The candidates
 * compute the same sums in different reduction orders (results agree to
 * rounding).  0: always 256 threads.
 */
gw_status gw_set_autotune(gw_ctx* ctx, int on);

/*
 * gw_proj_coef -- coef[v][j] = <C_v|y_j> = sum_G conj(C_v(G)) y_j(G), the
 * coefficients of the conduction projector P_c y = y - sum_v C_v <C_v|y>
 * (Sec. "Avoiding summations": orthogonalisation to the valence space at
 * every solver step; C_v: the occupied rows, then any deflation rows) for
 * ncol FP32 solver columns.
 *   kernel 0  CUDA cores (FP32 products, FP32 partial sums)
 *   kernel 1  tensor cores: tcgen05.mma kind::tf32 with both operands split
 *             into TF32 hi and lo parts (three products, FP32 accumulation in
 *             tensor memory), partial sums over K blocks added in FP64; up to
 *             64 projector rows
 *   y     [ncol][N_PW] complex FP32 (interleaved), DEVICE pointer
 *   coef  [n_proj][ncol] complex FP64 (interleaved), DEVICE pointer
 * GW_E_UNSUPPORTED for kernel 1 with more than 64 rows (or without a
 * tensor-map encoder in the driver).  The mixed simplified-QMR solver uses
 * kernel 1 from 256 columns on (gw_set_tensor_cores).
 */
gw_status gw_proj_coef(gw_ctx* ctx, const float* y, int ncol, double* coef, int kernel);

/* gw_set_tensor_cores -- 1: the mixed simplified-QMR solver takes its
   projector coefficients from the tensor cores (gw_proj_coef kernel 1) when
   it has at least 256 columns and at most 64 projector rows; 0 (default):
   CUDA cores always.  Off by default: the tensor-core coefficients carry
   about 2e-6 relative error (the FP32 accumulation in tensor memory) against
   about 1e-7 for the CUDA-core FP32 dots, and on the 64^3 cell with 64
   occupied states the solver then needs about four times as many
   iterations. */
gw_status gw_set_tensor_cores(gw_ctx* ctx, int on);

/*
 * gw_set_recycle_augment -- w0 > 0 adds to every recycled basis of
 * gw_recycle_eps (and gw_sigma_c, which uses it) the solutions at one more
 * imaginary frequency, x_{l,v}(i w0) = ((H - e_v)^2 + w0^2)^-1 (H - e_v) b_{l,v}
 * (Eq. P2+, CG on the squared operator): the accuracy control of the
 * recycling section (the paper takes w0 = 1 Ha).  3 nl vectors per state
 * then enter the decomposition, and 3 nl n_occ <= 65535.  0 (default) builds
 * the basis from x(0) and x(i inf) alone.  GW_E_ARG for w0 < 0 or non-finite.
 */
gw_status gw_set_recycle_augment(gw_ctx* ctx, double w0);

/* Solver of purely imaginary frequencies omega = i w (gw_set_imaginary_route). */
typedef enum {
  GW_IMAG_SQMR = 0,      /* the pair (H - e_v -/+ i w) x = b by simplified QMR (default) */
  GW_IMAG_SQUARED = 1    /* Eq. P2+: ((H - e_v)^2 + w^2) y = 2 (H - e_v) b by CG */
} gw_imag_route;

/*
 * gw_set_imaginary_route -- how gw_apply_chi0(_c), gw_apply_eps(_c) and the
 * Lanczos entries solve at a purely imaginary frequency i w.  GW_IMAG_SQUARED
 * solves the squared Hermitian positive definite system of Eq. P2+ (Sec.
 * "Avoiding summations"), whose solution is x^- + x^+ directly (Eq. fv): one
 * solve per occupied state instead of two, two H applications per CG
 * iteration, the kinetic preconditioner squared; P_c between the two
 * applications, and the FP64 refinement residual of the squared system.
 * Frequencies with a real part keep Eq. P2.  GW_E_ARG for another value.
 */
gw_status gw_set_imaginary_route(gw_ctx* ctx, int route);

/*
 * gw_set_graphs -- on (default 1): the ten launches of one simplified-QMR
 * iteration (the transform passes of H, the projector, the four update
 * steps) are captured once per solve into a CUDA graph and replayed every
 * iteration; 0: launched one by one.  Same arithmetic either way; a stream
 * that cannot be captured falls back to direct launches.
 */
gw_status gw_set_graphs(gw_ctx* ctx, int on);

/*
 * gw_set_solver -- Sternheimer solver controls (0 or negative keeps a value):
 *   tol        normwise backward error |b - A x| / (|A| |x| + |b|) that every
 *              column must reach, measured in FP64 (default 1e-13 for GW_FP64;
 *              the mixed path uses max(tol, 1e-13), default 1e-10); a pass
 *              that does not halve the error ends the refinement when the error
 *              is already within 10 tol (round-off and input-accuracy floor)
 *   tol_inner  relative residual at which each FP32 inner CG pass of the mixed
 *              path stops before the next FP64 residual (default 1e-5)
 *   max_iter   inner CG iterations per pass;  max_outer  FP64 residual passes
 * The paper solves Eq. P2 until |A x - b|^2 < 1e-20 Ha^2 (Sec. Results).
 */
gw_status gw_set_solver(gw_ctx* ctx, double tol, double tol_inner, int max_iter, int max_outer);

/* Kernel of the CG passes at omega = 0 (gw_set_cg_kernel). */
typedef enum {
  GW_CG_PERSISTENT = 0,    /* one cooperative persistent launch per pass (default) */
  GW_CG_MULTI_LAUNCH = 1,  /* one launch per transform pass, projector and update, per iteration */
  GW_CG_CLUSTER = 2        /* one thread-block cluster per column (falls back to the persistent
                              kernel when a column's planes do not fit in a cluster) */
} gw_cg_kernel;

/*
 * gw_set_cg_kernel -- which kernel runs the conjugate-gradient passes of the
 * Sternheimer solves at omega = 0 (Eq. P2; all three solve the same equations
 * to the same tolerance), and the bound on the device waits of the persistent
 * kernel.
 *   kind        a gw_cg_kernel value
 *   wait_limit  polls (each one memory round trip, with a short sleep after
 *               the first eight) that one CTA of the persistent kernel makes at
 *               one wait for other CTAs before it gives up; the kernel then
 *               returns early on every CTA and the call reports GW_E_TIMEOUT
 *               (the context stays usable).  0 keeps the current value
 *               (default 2^24, seconds); negative is GW_E_ARG.
 * GW_E_ARG for an unknown kind.
 */
gw_status gw_set_cg_kernel(gw_ctx* ctx, int kind, long long wait_limit);

/*
 * gw_set_precond -- preconditioner of the Sternheimer solvers (CG and SQMR):
 *   1 (default)  kinetic preconditioner of Teter, Payne and Allan, diagonal in
 *                G, with the kinetic energy of the column's occupied state as
 *                reference (symmetric, also in the bilinear form)
 *   0            none, as in the paper (Sec. Avoiding summations: SQMR without
 *                preconditioning)
 * Both solve the same equations to the same tolerance; the preconditioner
 * only changes the iteration count.  GW_E_ARG for any other kind.
 */
gw_status gw_set_precond(gw_ctx* ctx, int kind);

/*
 * gw_set_operator -- which polarizability gw_apply_chi0(_c), gw_apply_eps(_c),
 * gw_lanczos, gw_block_lanczos and gw_batch_lanczos apply (default
 * GW_OP_STERNHEIMER).  GW_OP_MODEL is the model operator of Sec. Dielectric
 * model (Eq. model_eq): H is replaced by the kinetic operator T in Eq. P2a,
 * so each Sternheimer solve becomes one division in the plane-wave sphere,
 *   f~_v(-/+) = P_c [ (|G|^2/2 - e_v -/+ omega)^-1 P_c (psi_v* dV) ],
 * summed over both signs and reduced as in Eq. P1.  The energies are the
 * absolute e_v given to gw_set_occupied; a denominator that is exactly zero
 * contributes zero (pseudo-inverse).  Under GW_OP_MODEL both precisions run
 * every step in FP64: the model has no Sternheimer solve whose FP64 residual
 * could recover what FP32 transforms lose (about 1e-5 on the Lanczos
 * coefficients after 20 steps), so GW_MIXED gives the FP64 result.  No solver
 * statistics are produced, and gw_grad_vloc returns GW_E_UNSUPPORTED.
 * GW_E_ARG for any other value.
 */
gw_status gw_set_operator(gw_ctx* ctx, int op);

/*
 * gw_epsinv_split -- matrix elements of eps~^-1 - 1 at a real frequency from
 * two Lanczos bases (Sec. Dielectric model, Eq. subs_epsilon):
 *   eps~^-1 - 1 = (eps~^-1 - eps~_m^-1) + (eps~_m^-1 - 1),
 * the first part in the basis {l} of the Sternheimer operator, the second in
 * the basis {l~} of the model operator:
 *   out[i][j] = a_i^T (T^-1 - M^-1) a_j + a~_i^T (T~^-1 - 1) a~_j,
 *   a = <l|phi>, a~ = <l~|phi>, M = <l|eps~_m l'> (the model operator applied
 *   to every vector of {l}: k model applications), T, T~ the tridiagonal
 *   Lanczos matrices (alpha, beta) of the two recursions.
 * The model operator in the exact basis is compressed to that basis and then
 * inverted, the way T^-1 stands for eps~^-1 there.  Runs on the GPU in FP64
 * whatever operator gw_set_operator selected.
 *   phi      [m][N^3] real fields, 1 <= m <= 64
 *   basis    [k][N^3], alpha [k], beta [k-1]: gw_lanczos with GW_OP_STERNHEIMER;
 *            1 <= k <= 2048
 *   basis_m  [k_m][N^3], alpha_m [k_m], beta_m [k_m-1]: gw_lanczos with
 *            GW_OP_MODEL at the same omega; 1 <= k_m <= 4096
 *   omega    the real frequency of both recursions
 *   out      [m][m] real
 * Returns GW_E_BREAKDOWN when T, T~ or M is singular.
 */
gw_status gw_epsinv_split(gw_ctx* ctx, const double* phi, int m, const double* basis, const double* alpha,
                          const double* beta, int k, const double* basis_m, const double* alpha_m,
                          const double* beta_m, int k_m, double omega, double* out, int device_ptrs);

/*
 * gw_sigma_p -- the residue term of the correlation self-energy (Eq. pe):
 *   Sigma^P_e(delta) = - sum_v <e v*|v^1/2 (eps^-1(w_ve) - 1) v^1/2|v* e> Theta(w_ve)
 *                      + sum_c <e c*|v^1/2 (eps^-1(w_ce) - 1) v^1/2|c* e> Theta(-w_ce),
 *   w_ne = e_n - e_e - delta, <r|n* e> = psi_n(r)* psi_e(r), Theta(0) = 1/2,
 * each element from a separate Lanczos recursion of k steps on eps~(w) at its
 * real frequency, seeded with phi = v^1/2 |p* e> (Sec. "Calculating the
 * dielectric matrix and the integrand at different frequencies": four steps
 * converge the term to 1 meV): <phi|eps~^-1 - 1|phi> ~ |phi|^2 ((T^-1)_11 - 1).
 * A seed that is complex in real space runs as the stacked real pair (real
 * part, imaginary part), which is the recursion of the complex vector in the
 * Hermitian inner product; the recursion stops early at an invariant subspace.
 * Uses the operator chosen by gw_set_operator and the solvers of gw_lanczos
 * (CG at w = 0, SQMR otherwise).
 *   psi_e   [N_PW] complex sphere coefficients of the state e
 *   eps_e, delta  energies (Ha)
 *   n       candidate pole states; psi [n][N_PW] complex, eps [n], occ [n]
 *           (1 occupied: enters when w_ve >= 0; 0 conduction: when w_ce <= 0)
 *   k       Lanczos steps per pole, 1 <= k <= 256
 *   sigma   scalar out; terms [n] out (signed term of each state, 0 where
 *           Theta excludes it), or NULL
 * Pointers are all host or all device (device_ptrs).  Errors of a recursion
 * (GW_E_NOCONV, GW_E_NONFINITE, ...) are returned as they are; a singular
 * Lanczos matrix gives GW_E_BREAKDOWN.
 */
gw_status gw_sigma_p(gw_ctx* ctx, const double* psi_e, double eps_e, double delta, int n, const double* psi,
                     const double* eps, const int* occ, int k, double* sigma, double* terms, gw_prec prec,
                     int device_ptrs);

/*
 * gw_recycle_eps -- the dielectric matrix in a basis of fields at any number of
 * imaginary frequencies from one recycled basis per occupied state (Sec.
 * "Calculating the dielectric matrix and the integrand at different
 * frequencies", Eq. recy_eq):
 *   out[o][l][l'] = <l| eps~(i w_o) - 1 |l'> = 4 sum_v <b_{l,v}| A_v^-1 |b_{l',v}>,
 *   b_{l,v} = P_c <G| psi_v* v^1/2 l>,  A_v(i w) = ((H - e_v)^2 + w^2) (H - e_v)^-1,
 * with A_v^-1 applied in the basis gamma_v spanned by the static Sternheimer
 * solutions x_{l,v}(0) = (H - e_v)^-1 b_{l,v} (solved here, mixed or FP64 as
 * prec says) and the high-frequency directions P_c (H - e_v) b_{l,v}: each of
 * the 2 nl vectors is normalised, their Gram matrix is diagonalised (Jacobi,
 * FP64) and directions with singular value below rtol times the largest are
 * dropped; then H_v = gamma^H (H - e_v) gamma is diagonalised and every
 * frequency costs only small dense algebra.  Exact at w = 0 and whenever the
 * recycled vectors span the conduction space.  Uses the Sternheimer operator
 * (GW_E_UNSUPPORTED under GW_OP_MODEL).
 *   fields  [nl][N^3] real (e.g. the Lanczos basis of eps~(0)), 1 <= nl <= 256 and
 *           2 nl n_occ <= 65535
 *   w       [nw] imaginary frequencies w (the frequency is i w), 1 <= nw <= 4096
 *   rtol    relative singular-value cut-off (0: 1e-6)
 *   out     [nw][nl][nl] real;  kept (optional, host int): the smallest number
 *           of recycled directions kept over the occupied states
 * Returns GW_E_NOCONV if a Jacobi eigensolver does not converge in 40 sweeps.
 */
gw_status gw_recycle_eps(gw_ctx* ctx, const double* fields, int nl, const double* w, int nw, double rtol,
                         double* out, int* kept, gw_prec prec, int device_ptrs);

/*
 * gw_sigma_c -- the correlation self-energy of an occupied state e (Eq. e_c):
 *   Sigma^c_e(delta) = (1/pi) int_0^inf dw (sigma^N_e(i w) - sigma^N0_e(i w)) + Sigma^A_e + Sigma^P_e,
 * evaluated in a basis {l} of fields as Eqs. ge, g0e, he and khe write it:
 *   sigma^N(i w) = sum_ll' M_ll'(i w) <z_l| g(H - c, w) |z_l'>,  g(h) = h / (w^2 + h^2),
 *   sigma^N0(i w) = f(w) sum_ll' M_ll'(0) <z_l| g(H - c, w) |z_l'>,  f(w) = alpha^2 / (w^2 + alpha^2),
 *   Sigma^A = 1/2 sum_ll' M_ll'(0) (<z_l|Q_e|h+_l'> + <z_l|P_e|h-_l'>)   (Eq. khe for h+-),
 * with c = e_e + delta, z_l = Phi_e v^1/2 |l*> (psi_e(r) (v^1/2 l)(r) in the
 * plane-wave sphere), M = eps~^-1 - 1 in the basis from the recycled
 * eps~(i w) (gw_recycle_eps) as (1 + E)^-1 - 1, <z|g(H - c)|z'> for every
 * frequency from one block Lanczos recursion of k_h steps on H - c started
 * with the z block (shift-Lanczos), h+ by the Sternheimer solver at the shift
 * c - alpha, the P_e part in closed form on the occupied states below c, and
 * Sigma^P from gw_sigma_p (k_p steps per pole).  The frequency integral uses
 * w = (1 + t)/(1 - t) at n_freq Gauss-Legendre nodes in t.
 * Written for e_HOMO <= e_e + delta < e_LUMO, where Q_e(delta) is the
 * conduction projector; e_e + delta below the highest occupied energy returns
 * GW_E_UNSUPPORTED, and staying below the lowest conduction energy is the
 * caller's part (the library holds no conduction states).
 *   e        occupied state (0 <= e < n_occ, in the order of gw_set_occupied)
 *   alpha    Lorentzian width (Ha), > 0 (the paper takes 1 Ha)
 *   n_freq   1 .. 64 (the paper: about 8 to 10 converge to 1 meV)
 *   fields   [nl][N^3] real, orthonormal in <.|.> (e.g. the Lanczos basis of
 *            eps~(0)); 1 <= nl <= 16
 *   k_h      block Lanczos steps on H, k_h nl <= 512;  k_p as in gw_sigma_p
 *   out      [4]: Sigma^c, the frequency integral, Sigma^A, Sigma^P (Ha)
 */
gw_status gw_sigma_c(gw_ctx* ctx, int e, double delta, double alpha, int n_freq, const double* fields, int nl,
                     int k_h, int k_p, double* out, gw_prec prec, int device_ptrs);

/*
 * gw_profile -- time selected kernel classes with CUDA events on the work
 * stream (one event pair around each launch; mask 0 turns timing off).
 * Classes (multi-launch CG): 0 scatter + inverse z pass (with the CG p update),
 * 1 inverse y pass, 2 x pass with V_loc (H), 3 forward y pass, 4 forward z pass
 * + gather + kinetic and shift, 5 projector P_c, 6 CG update; 7 FP64
 * refinement residual (H apply + P_c); 8 persistent CG launch (all phases);
 * 9 the persistent CG's tasks, timed inside the kernel (global timer): read
 * back as entries 10..15 = task kind A busy, A waiting, B busy, B waiting,
 * C busy, C waiting (milliseconds summed over tasks; counts: tasks run for
 * "busy", tasks skipped for "waiting"), then 16..27 the busy time of four
 * sub-phases per kind: A loads (records, partials, column state), A sums and
 * decisions, A update and scatter, A transforms; B slab load, B transforms and
 * V, B store, (unused); C plane and u loads, C transforms and gather, C
 * projector dots, C scalar sums and record (the remainder of a task's busy
 * time is its stores and signalling).
 * gw_profile_read -- per class: total milliseconds and launches since the last
 * read (synchronises the stream; resets the totals); n >= 16 for the task
 * entries, n >= 28 for the sub-phases.
 */
gw_status gw_profile(gw_ctx* ctx, unsigned mask);
gw_status gw_profile_read(gw_ctx* ctx, double* ms, long long* count, int n);

const char* gw_last_error(const gw_ctx* ctx);
void gw_destroy(gw_ctx* ctx);

/*
 * Batches of independent cells (the many-system workload: cells of different
 * size, cutoff and occupation, each with its own Lanczos recursions).  The
 * batch owns one context and one non-blocking CUDA stream per cell; a pool of
 * host threads runs the cells concurrently on the current device.
 */
typedef struct gw_batch gw_batch;

/*
 * gw_batch_setup -- one context per cell, as gw_setup (per-cell L, n_grid,
 * ecut, vloc[i] of n_grid[i]^3 doubles; coulomb shared).  n_workers <= 0 picks
 * min(n_cells, 8).  Occupied states are set per cell through gw_batch_cell and
 * gw_set_occupied.  On error nothing is allocated and *out is NULL.
 */
gw_status gw_batch_setup(gw_batch** out, int n_cells, const double* L, const int* n_grid, const double* ecut,
                         const double* const* vloc, int coulomb, int n_workers);

/* Number of cells; the context of cell i (owned by the batch; NULL if out of range).
 * A cell's context works on the batch's own non-blocking stream for that cell:
 * device-pointer arguments passed to it must be complete before the call
 * (synchronise the stream that produced them). */
int gw_batch_size(const gw_batch* b);
gw_ctx* gw_batch_cell(gw_batch* b, int i);

/*
 * gw_batch_lanczos -- for every cell i and frequency w, k Lanczos steps on
 * eps~(omega_w) of cell i from start[i] (host, n_grid[i]^3 doubles): the
 * recursion of gw_lanczos at real omega, of gw_block_lanczos with block size
 * 1 (bilinear form) at complex omega.
 *   omega  [n_cells][n_omega] complex (interleaved): each cell its own
 *          frequencies (a real frequency must keep clear of the cell's
 *          transition energies, where eps~ has poles)
 *   alpha  [n_cells][n_omega][k] complex (host);  beta [n_cells][n_omega][k-1]
 *   cell_status  [n_cells] per-cell gw_status, or NULL
 * Cells run concurrently; a failing cell stops its own remaining frequencies
 * only.  Returns the status of the lowest-numbered failing cell (its message
 * in gw_batch_last_error), else GW_OK.
 */
gw_status gw_batch_lanczos(gw_batch* b, const double* const* start, int k, int n_omega, const double* omega,
                           double* alpha, double* beta, gw_prec prec, int* cell_status);

const char* gw_batch_last_error(const gw_batch* b);
void gw_batch_destroy(gw_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* GW_H */
