/*
 * gw.h -- C ABI of libgw.so, the GB300 (sm_103a) hot path of the cubic-scaling
 * space-time GW method (Liu, Kaltak, Klimes, Kresse, arXiv:1607.02859).
 *
 * Conventions shared by every call
 * --------------------------------
 *  Grid      n[3] = (n1,n2,n3), N_r = n1*n2*n3, r index = (i1*n2+i2)*n3+i3,
 *            fractional position (i1/n1, i2/n2, i3/n3).  lattice[9] holds the
 *            three lattice vectors as rows (bohr); Omega = |det|, dV = Omega/N_r.
 *  G set     gvec[j] = integer triple g with G = sum_d g_d b_d; fft_index[j] =
 *            ((g1 mod n1)*n2 + g2 mod n2)*n3 + g3 mod n3 (see gw_g_set).
 *  Complex   interleaved (re, im).  Element type is given by gw_prec:
 *            GW_FP64 -> complex double (16 B); every other precision -> complex
 *            float (8 B).  Layouts are row-major.
 *  Orbitals  psi [N_b][N_r], band-major, normalised to dV sum_r |psi|^2 = 1.
 *            eps_h [N_b] ascending on the host; eps[n_occ-1] < mu < eps[n_occ].
 *  Pointers  without _h are DEVICE pointers owned by the caller; _h are host
 *            pointers.  The library never frees caller memory.  Scratch comes
 *            from the context: a grow-only device arena (cudaMalloc) that lives
 *            until gw_ctx_destroy.
 *  Streams   `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *            stream).  Calls are asynchronous on it unless documented as
 *            synchronous (those returning results in host memory).
 *  Errors    every call returns gw_status; nothing aborts or exits.  The message
 *            of the last failure is gw_last_error(ctx).  A GW_ERR_CUDA from a
 *            kernel fault leaves the CUDA context unusable (a CUDA property).
 *  Threads   a context may be used by one host thread at a time.
 */
#ifndef GW_H_
#define GW_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gw_status {
  GW_OK = 0,
  GW_ERR_ARG = 1,         /* bad pointer, sign, ordering or enum value        */
  GW_ERR_SHAPE = 2,       /* unsupported or inconsistent size                 */
  GW_ERR_OOM = 3,         /* device scratch allocation failed                 */
  GW_ERR_CUDA = 4,        /* a CUDA runtime call or kernel launch failed      */
  GW_ERR_NUMERIC = 5,     /* non-positive pivot, vanishing Thiele denominator */
  GW_ERR_TIMEOUT = 6,     /* a bounded device wait gave up                    */
  GW_ERR_UNSUPPORTED = 7  /* valid request this build does not implement      */
} gw_status;

typedef enum gw_prec {
  GW_FP64 = 0,   /* every step in double precision, CUDA cores                    */
  GW_FP32 = 1,   /* every step in single precision, CUDA cores                    */
  GW_F16X3 = 2,  /* G and Sigma contractions as 3 fp16 split products on tcgen05  */
                 /* tensor cores with FP32 accumulation; everything else as FP32  */
  GW_BF16X3 = 3  /* same with bf16 splits                                         */
} gw_prec;

typedef enum gw_transform {
  GW_CT = 0,     /* out[k] = sum_j M[k][j] in[j]        (Eqs. CT_FFT, CTX, CT_W) */
  GW_ST = 1,     /* out[k] = i * sum_j M[k][j] in[j]    (Eq. ST_FFT)             */
  GW_IST = 2     /* out[j] = -i * sum_k M[j][k] in[k]   (Eq. INV_ST_FFT)         */
} gw_transform;

typedef struct gw_grid {
  int n[3];
  double lattice[9];
} gw_grid;

typedef struct gw_ctx gw_ctx;

/* ---------------------------------------------------------------- context */

/* Create a context bound to CUDA device `device`. *out receives it. */
gw_status gw_ctx_create(int device, gw_ctx** out);
/* Free the scratch arena and the context (synchronises the device). */
gw_status gw_ctx_destroy(gw_ctx* ctx);
/* Message of the last failure on ctx ("" if none); ctx may be NULL for failures
 * of gw_ctx_create or of the host setup calls.  Valid until the next call. */
const char* gw_last_error(const gw_ctx* ctx);
/* Number of kernels this library launched through ctx since creation. */
unsigned long long gw_ctx_launches(const gw_ctx* ctx);
/* Current size of the context's device scratch arena in bytes. */
size_t gw_ctx_scratch_bytes(const gw_ctx* ctx);
/* Grow the scratch arena to at least `bytes` now (e.g. the largest
 * gw_workspace_size of the problems a server will run), so that later calls
 * do not reallocate it.  Growing frees and reallocates the arena, which
 * synchronises the device; a smaller request does nothing.  GW_ERR_OOM if the
 * allocation fails (the arena is then empty). */
gw_status gw_ctx_reserve(gw_ctx* ctx, size_t bytes);
/* Per-kernel timing for benchmarks.  While enabled, the library brackets every
 * launch of its main kernels with CUDA events on the launch stream and records,
 * per kernel family, the number of launches, their summed device time and their
 * summed algorithmic work (flops of the method for the contractions, bytes of
 * the minimal HBM traffic for the transforms).  Enabling or disabling clears
 * the totals.  Families: "green_tc", "cgemm_tc", "cgemm_simt", "row_fft",
 * "col_fft", "col_line_ct", "sigma_contract", "ct" (the standalone transform
 * over tau/omega), "cgemm_exact" (the refinement's sliced product),
 * "row_pw" (the plane-wave row passes of gw_chi0_omega_pw and gw_sigma_diag_pw;
 * work = their transforms' 5 N log2 N flops and the products).
 * gw_ctx_kernel_stats synchronises on the recorded events; any output pointer
 * may be NULL. */
gw_status gw_ctx_set_timing(gw_ctx* ctx, int enabled);
gw_status gw_ctx_kernel_stats(gw_ctx* ctx, const char* family, unsigned long long* launches,
                              double* ms, double* work, int* work_is_bytes);
/* ABI version (major*100 + minor). */
int gw_version(void);

/* ---------------------------------------------------------------- host setup
 * Negligible host work (Sec. II.A.2-3); no GPU is touched. */

/* The G set of chi and W (the cutoff sphere of Eq. FFTX1): the n_chi lowest
 * integer triples g_d in [-n_d/2, n_d/2) ordered by (g1^2+g2^2+g3^2, g1, g2, g3).
 * gvec_h [n_chi][3], fft_index_h [n_chi] (may be NULL).  1 <= n_chi <= N_r. */
gw_status gw_g_set(const gw_grid* grid, int n_chi, int32_t* gvec_h, int32_t* fft_index_h);

/* v^{1/2}(G) = sqrt(4 pi)/|G| of the symmetric Coulomb kernel (Eq. bareV,
 * e = 1), with the G = 0 entry set to 0 (head and wings of W~ dropped). */
gw_status gw_coulomb_sqrt(const gw_grid* grid, const int32_t* gvec_h, int n_chi,
                          double* vhalf_h);

/* Nonuniform cosine/sine transform matrices (Eqs. CT_FFT, cos_error_function,
 * ST_FFT, sin_error_function, INV_CT_FFT) for given grids tau_h[n], omega_h[n]:
 *   C[k][j] = gamma_kj cos(omega_k tau_j),  S[k][j] = lambda_kj sin(omega_k tau_j),
 *   Cinv = C^{-1} (Eq. INV_CT_FFT).
 * gamma_k (lambda_k) minimises, per omega_k, the relative error of the fitted
 * Lorentzian 2x/(x^2+w^2) (2w/(x^2+w^2)) at n_x log-spaced x in [x_min, x_max]
 * plus ridge^2 * n_x * |gamma_k|^2 (Householder QR, FP64).  fit_err_h[2]
 * receives the largest relative error of the cosine and sine fits.  Any of the
 * outputs may be NULL.  GW_ERR_NUMERIC if C is singular. */
gw_status gw_fit_transform(int n, const double* tau_h, const double* omega_h,
                           double x_min, double x_max, int n_x, double ridge,
                           double* C_h, double* S_h, double* Cinv_h, double* fit_err_h);

/* Optimised n-point imaginary-time and imaginary-frequency grids (Sec. II.A.2:
 * the grids minimise the discretisation error of the direct MP2 energy in each
 * domain) for transition energies x in [x_min, x_max] (Ha):
 *   tau_j   minimise max_x |1 - x sum_j alpha_j exp(-2 x tau_j)|
 *           (1/x = int dtau exp(-x|tau|)^2),
 *   omega_k minimise max_x |1 - x sum_k sigma_k (2x/(x^2 + omega_k^2))^2|
 *           (1/x = int dw/(2 pi) (2x/(x^2+w^2))^2),
 * each a Chebyshev (minimax) approximation computed in FP64 by the Remez
 * exchange with continuation in the number of terms.  Outputs ascending:
 * tau_h [n] (1/Ha), omega_h [n] (Ha); alpha_h, sigma_h [n] (may be NULL);
 * err_h [2] (may be NULL) receives the two largest relative errors.  Use the
 * grids with gw_fit_transform (ridge 0).  1 <= n <= 40, 0 < x_min < x_max,
 * x_max/x_min <= 1e7.  Host only, milliseconds. */
gw_status gw_mp2_grids(int n, double x_min, double x_max, double* tau_h, double* omega_h,
                       double* alpha_h, double* sigma_h, double* err_h);

/* Inverse of an n x n transform matrix (Eqs. INV_CT_FFT, INV_ST_FFT: the
 * matrices xi cos and zeta sin are the inverses of gamma cos and lambda sin) by
 * Gauss-Jordan elimination with partial pivoting in FP64.  Host only.
 * GW_ERR_NUMERIC if M is singular. */
gw_status gw_invert_transform(int n, const double* M_h, double* Minv_h);

/* Device scratch in bytes that the context arena needs for gw_chi0_omega
 * (r_block <= 0: the default), gw_screen_W (n frequencies) and gw_sigma_diag
 * (n_n bands, up to 64 real frequencies) on this problem.  The arena is shared
 * by the calls of one context, so a context needs the largest of the three.
 * gw_sigma_matrix needs at most 16 n (3 n_n^2 - 2 n_n) + 32 n_n min(N_r, 2048) bytes
 * more than the gw_sigma_diag figure, within 256-byte rounding;
 * gw_qp_energies and gw_sigma_to_tau need only a few arrays of n_n x n.
 * Host only; any output may be NULL.  Used for admission by memory footprint. */
gw_status gw_workspace_size(const gw_grid* grid, int n_b, int n_occ, int n, int n_chi, int n_n, gw_prec prec,
                            int r_block, size_t* chi0_bytes, size_t* screen_bytes, size_t* sigma_bytes);

/* ---------------------------------------------------------------- hot path */

/* Imaginary-time Green's functions for the rows r0 .. r0+n_rows-1 (Eqs.
 * Green_occ, Green_unocc with energies measured from mu, tau > 0):
 *   g_occ  [n_rows][N_r]:  sum_{i<n_occ}  psi_i(r) psi_i^*(r') exp(+(eps_i-mu) tau)
 *   g_unocc[n_rows][N_r]:  sum_{a>=n_occ} psi_a(r) psi_a^*(r') exp(-(eps_a-mu) tau)
 * Either output may be NULL.  The exponentials are formed in FP64 on the host
 * and pre-scaled by their largest value, which is restored in FP64 afterwards.
 * prec: GW_FP64/GW_FP32 SIMT GEMM; GW_F16X3/GW_BF16X3 tcgen05 split GEMM. */
gw_status gw_green_tau(gw_ctx* ctx, const gw_grid* grid, int n_b, int n_occ,
                       const void* psi, const double* eps_h, double mu, double tau,
                       int r0, int n_rows, gw_prec prec, void* g_occ, void* g_unocc,
                       void* stream);

/* Polarizability in real space and imaginary time (Eqs. chi_GG, chi_rr), spin
 * factor 2, index order of G_occ(r,r') G_unocc(r',r):
 *   chi[r][r'] = -2 g_occ[r][r'] * conj(g_unocc[r][r'])     (n_rows x n_cols)
 * chi may alias g_unocc or g_occ. */
gw_status gw_chi0_rtau(gw_ctx* ctx, int n_rows, int n_cols, gw_prec prec,
                       const void* g_occ, const void* g_unocc, void* chi, void* stream);

/* Fused G formation + Hadamard (Eqs. Green_occ/unocc and chi_rr in one pass;
 * G_occ and G_unocc tiles never leave the chip when prec is a tensor-core
 * precision).  chi [n_rows][N_r] as in gw_chi0_rtau. */
gw_status gw_chi0_rtau_fused(gw_ctx* ctx, const gw_grid* grid, int n_b, int n_occ,
                             const void* psi, const double* eps_h, double mu, double tau,
                             int r0, int n_rows, gw_prec prec, void* chi, void* stream);

/* Two-step spatial transform within the cell (Eqs. FFTX1, FFTX2 forward; Eq.
 * FFTW backward), 3-D mixed-radix FFTs on the n1 x n2 x n3 grid (radices 2, 3,
 * 5; each n_d in {4,6,8,10,12,16,18,20,24,30,32,36,40,48}):
 *  direction=+1 stage=1  in [n_rows][N_r] x(r,R')  -> out [n_rows][n_chi]
 *                        X(r,G') = sum_R' x(r,R') exp(+i G'.R')           (FFTX1)
 *  direction=+1 stage=2  in [N_r][n_chi] X(r,G')   -> out [n_chi][n_chi]
 *                        (dV^2/Omega) sum_r exp(-i G.r) X(r,G')          (FFTX2)
 *                        `in` is overwritten (used as the work buffer).
 *  direction=-1 stage=2  in [n_chi][n_chi] W(G,G') -> out [N_r][n_chi]
 *                        W(r,G') = sum_G exp(+i G.r) W(G,G')             (FFTW 1)
 *  direction=-1 stage=1  in [n_rows][n_chi] W(r,G') -> out [n_rows][N_r]
 *                        (1/Omega) sum_G' W(r,G') exp(-i G'.R')           (FFTW 2)
 * r0 is only checked against N_r (rows are independent).  fft_index_h as
 * returned by gw_g_set. */
gw_status gw_rr_to_GG_fft(gw_ctx* ctx, const gw_grid* grid, int direction, int stage,
                          int n_chi, const int32_t* fft_index_h, gw_prec prec, int r0,
                          int n_rows, const void* in, void* out, void* stream);

/* gw_rr_to_GG_fft without any device allocation and without a context.
 * The paper has no counterpart: this exists for callers that must not call
 * cudaMalloc at all -- for example a program whose memory pool owns the whole
 * GPU and forbids allocations outside it, or a latency-bound loop that cannot
 * take the device-wide synchronisation an allocation may cause.
 * Arguments, layouts and results are exactly those of gw_rr_to_GG_fft.  The
 * two index maps the transform needs live in one fixed array inside the
 * library's device image (n_chi + N_r <= 27648 entries, i.e. up to the 24^3
 * grid); larger requests return GW_ERR_SHAPE.  That array exists on every GPU
 * that loads the library until the process exits.  Its device address is
 * looked up once per device, on the first call made with that device current.
 * Every call rewrites both maps in full, so nothing carries over between
 * calls, but all calls share the array: calls whose work overlaps on the GPU
 * (different streams, or different host threads) race on it.  Calls on one
 * stream are ordered and safe.  The maps are uploaded on every call by a copy
 * from pageable host memory, which waits for the stream's earlier work before
 * it starts.  Because that copy's host source lives only for the call, a call
 * made while `stream` is being captured into a CUDA graph is refused with
 * GW_ERR_UNSUPPORTED and does nothing.  Errors are reported through
 * gw_last_error(NULL). */
gw_status gw_rr_to_GG_fft_noalloc(const gw_grid* grid, int direction, int stage, int n_chi,
                                  const int32_t* fft_index_h, gw_prec prec, int r0, int n_rows,
                                  const void* in, void* out, void* stream);

/* Nonuniform time <-> frequency transform of `elems` complex elements per slice
 * (Eqs. CTX, CT_W, ST_FFT, INV_ST_FFT):
 *   out[k][e] = f sum_j M_h[k][j] in[j][e],  f = 1 (GW_CT), i (GW_ST), -i (GW_IST)
 * for k, j < n.  M_h is FP64 on the host; the FP64 path sums in FP64, the
 * others in FP32 with M split into two FP32 parts.  Use C for chi(tau)->chi(i
 * omega), Cinv for W~(i omega)->W~(i tau), S for the odd part of Sigma, and Sinv
 * (gw_invert_transform of S) with GW_IST to take it back to imaginary time.
 * in and out must not overlap. */
gw_status gw_tau_to_omega(gw_ctx* ctx, int kind, int n, const double* M_h, size_t elems,
                          gw_prec prec, const void* in, void* out, void* stream);

/* Screened interaction at n_omega frequencies (Eqs. W_tot, bareV, die,
 * W_correlated):  chi~ = v^{1/2} chi v^{1/2},  eps~ = 1 - chi~,
 *   W~ = v^{1/2} (eps~^{-1} - 1) v^{1/2}
 * by a blocked Cholesky factorisation eps~ = L L^H, L^{-1}, and
 * eps~^{-1} = L^{-H} L^{-1} on CUDA cores (FP64 or FP32 by prec; the tensor-core
 * precisions run this step in FP32).  chi_w, w_w [n_omega][n_chi][n_chi];
 * chi_w must be Hermitian (only its lower triangle is read); w_w may equal
 * chi_w (in place).  resid_h[n_omega] (may be NULL) receives the relative
 * residual |eps~ X - chi~| / |chi~| of X = eps~^{-1} - 1 estimated in FP64 on
 * 4 seeded probe vectors.  Synchronous (it reads back the pivot check).
 * GW_ERR_NUMERIC if a pivot is not positive (eps~ not positive definite). */
gw_status gw_screen_W(gw_ctx* ctx, const gw_grid* grid, int n_chi, const int32_t* gvec_h,
                      int n_omega, gw_prec prec, const void* chi_w, void* w_w,
                      double* resid_h, void* stream);
/* gw_screen_W followed by refine_iters (0..8) FP64 refinement steps per
 * frequency of X = eps~^{-1} - 1 before W~ is formed: with the residual
 * R = chi~ - eps~ X = chi~ - X + chi~ X (chi~ = v^1/2 chi v^1/2), X <- X + (1 + X) R,
 * which squares the relative error of X each step (Newton-Schulz for the
 * inverse of eps~; the same solve of Eq. W_correlated).  GW_FP64 and GW_FP32:
 * two N^3 FP64 complex GEMMs per step and frequency on CUDA cores, 64 n_chi^2
 * bytes more scratch.  GW_F16X3 / GW_BF16X3: the product chi~ X on tcgen05 as
 * exact fp16 slice products (gw_zgemm_sliced, 4 levels: 30 bits of the row and
 * column maxima) and X R as split fp16 products (R is small), about 160
 * n_chi^2 bytes more scratch.  The result is then limited by the
 * working precision of w_w.  refine_iters = 0 is gw_screen_W. */
gw_status gw_screen_W_refine(gw_ctx* ctx, const gw_grid* grid, int n_chi, const int32_t* gvec_h,
                             int n_omega, gw_prec prec, int refine_iters, const void* chi_w,
                             void* w_w, double* resid_h, void* stream);

/* Complex FP64 matrix product C = A B with FP64-class accuracy on the fp16
 * tensor cores (the product chi~ X of the refinement residual above; the paper
 * has no counterpart).  Each row of A and column of B is scaled by a power of
 * two and cut into 6-bit integer slices (exact in fp16); the products of
 * slice pairs of one level a + b, summed over 4096 real K elements, are
 * integers whose bounds add up to at most 2^24 in groups of up to four pairs,
 * and so exact in one FP32 accumulator; the slice pairs with a + b <= levels
 * (largest first) are scaled back group by group and added up in pairs of
 * FP32 numbers (~48 bits), converted to FP64 at the end.  The error is below about
 * 2^(-6(levels+1)) * K * max|A_i.| max|B_.j| per element (levels 5: 2^-36).
 * A [M][K] (lda), B [K][N] (ldb), C [M][N] (ldc) complex double, device,
 * 16-byte aligned, row-major; C is overwritten and must not overlap A or B.
 * 1 <= levels <= 7; scratch (context arena): about 2 (levels+1) K (2M + 4N)
 * bytes.  Synchronous (reports GW_ERR_TIMEOUT from the bounded pipeline
 * waits). */
gw_status gw_zgemm_sliced(gw_ctx* ctx, int M, int N, int K, const void* A, long lda, const void* B, long ldb,
                          void* C, long ldc, int levels, void* stream);

/* Diagonal correlation self-energy (Eqs. Sigma_occ, Sigma_rr and the first term
 * of Sigma_occ_reduce; even/odd split Eqs. cos_sin_sigma_matrix1/2; CT+ST Eqs.
 * sigma_r_w, cos_sin_sigma1/2; Thiele continuation Eqs. pade1, pade2):
 * for every tau_j, W~(r,R',tau_j) is formed from w_tau [n][n_chi][n_chi]
 * (Eq. FFTW), G_occ/G_unocc are recomputed, and
 *   Sigma_unocc_nn(tau) = +dV^2 sum_{r,R'} psi_n^*(r) G_unocc(r,R') W~(r,R') psi_n(R')
 *   Sigma_occ_nn(-tau)  = -dV^2 sum_{r,R'} psi_n^*(r) G_occ(r,R')   W~(r,R') psi_n(R')
 * (real parts), then Sigma^c = (Su+So)/2, Sigma^s = (Su-So)/2 and
 *   Sigma_nn(i omega_k) = sum_j C_kj Sigma^c(tau_j) + i sum_j S_kj Sigma^s(tau_j).
 * Thiele coefficients through z_k = i omega_k, evaluated at the real
 * frequencies w_real_h (measured from mu).
 * bands_h [n_n]; tau_h, omega_h [n]; C_h, S_h [n][n].  psi (device, [n_b][N_r])
 * must be 16-byte aligned (GW_ERR_ARG otherwise).
 * Outputs (host, FP64): sigma_tau_h [2][n_n][n] = (Su, So) (may be NULL);
 * sigma_iw_h [n_n][n] complex; sigma_real_h [n_n][n_real] complex (may be NULL).
 * Synchronous.  GW_ERR_NUMERIC if a Thiele denominator vanishes (|.| < 1e-300);
 * the other bands are still returned. */
gw_status gw_sigma_diag(gw_ctx* ctx, const gw_grid* grid, int n_b, int n_occ,
                        const void* psi, const double* eps_h, double mu, const int32_t* bands_h,
                        int n_n, int n, const double* tau_h, const double* omega_h,
                        const double* C_h, const double* S_h, const void* w_tau, int n_chi,
                        const int32_t* fft_index_h, gw_prec prec, double* sigma_tau_h,
                        double* sigma_iw_h, const double* w_real_h, int n_real,
                        double* sigma_real_h, void* stream);

/* Full correlation self-energy matrix Sigma_nm = <psi_n|Sigma|psi_m> over the
 * listed bands (Eq. Sigma_occ_reduce, first term, for a pair of bands; Eqs.
 * cos_sin_sigma, sigma_r_w, cos_sin_sigma1/2 element by element):
 *   Sigma_unocc_nm(tau) = +dV^2 sum_{r,R'} psi_n^*(r) G_unocc(r,R') W~(r,R') psi_m(R')
 *   Sigma_occ_nm(-tau)  = -dV^2 sum_{r,R'} psi_n^*(r) G_occ(r,R')   W~(r,R') psi_m(R')
 * (complex; Hermitian in (n, m); the diagonal is gw_sigma_diag's), then
 *   Sigma_nm(i omega_k) = sum_j C_kj Sigma^c_nm(tau_j) + i sum_j S_kj Sigma^s_nm(tau_j)
 * with Sigma^c = (Su+So)/2, Sigma^s = (Su-So)/2.  The contraction of
 * gw_sigma_diag keeps V_m(r) = sum_R' G(r,R') W~(r,R') psi_m(R') per row and
 * band; an FP64 kernel then adds conj(psi_n(r)) V_m(r) over the rows.
 * Arguments as for gw_sigma_diag, 1 <= n_n <= 256.  Outputs (host, FP64
 * complex): sigma_tau_h [2][n_n][n_n][n] = (Su, So) (may be NULL);
 * sigma_iw_h [n_n][n_n][n].  No continuation (the QP equation needs the
 * diagonal only).  Synchronous. */
gw_status gw_sigma_matrix(gw_ctx* ctx, const gw_grid* grid, int n_b, int n_occ,
                          const void* psi, const double* eps_h, double mu, const int32_t* bands_h,
                          int n_n, int n, const double* tau_h, const double* omega_h,
                          const double* C_h, const double* S_h, const void* w_tau, int n_chi,
                          const int32_t* fft_index_h, gw_prec prec, double* sigma_tau_h,
                          double* sigma_iw_h, void* stream);

/* The self-energy back on the imaginary time axis (Eqs. INV_CT_FFT,
 * INV_ST_FFT), the inverse of the CT + ST of gw_sigma_diag / gw_sigma_matrix:
 * Sigma(i omega) = C Sigma^c(tau) + i S Sigma^s(tau) with Sigma^c, Sigma^s
 * Hermitian in the band indices, so the Hermitian part of Sigma(i omega)
 * (the real part for diagonal elements) is the cosine part and the
 * anti-Hermitian part the sine part; then
 *   Sigma^c(tau_j) = sum_k Cinv_jk Herm(i omega_k),  Sigma^s(tau_j) = -i sum_k Sinv_jk Anti(i omega_k)
 *   Sigma_unocc(tau_j) = Sigma^c + Sigma^s,  Sigma_occ(-tau_j) = Sigma^c - Sigma^s.
 * matrix = 0: sigma_iw_h [n_n][n] complex -> sigma_tau_h [2][n_n][n] real
 * (gw_sigma_diag's layout); matrix = 1: sigma_iw_h [n_n][n_n][n] complex ->
 * sigma_tau_h [2][n_n][n_n][n] complex (gw_sigma_matrix's).  Cinv_h, Sinv_h
 * [n][n] (gw_fit_transform, gw_invert_transform).  FP64 throughout: the sine
 * matrix of the fitted grids is ill-conditioned (cond(S) ~ 2e6 at 16 points),
 * so the inverse amplifies input errors by up to that factor.  Synchronous. */
gw_status gw_sigma_to_tau(gw_ctx* ctx, int n_n, int n, int matrix, const double* Cinv_h,
                          const double* Sinv_h, const double* sigma_iw_h, double* sigma_tau_h,
                          void* stream);

/* Quasiparticle energies and spectral functions from the continued
 * self-energy (Sec. II.E.2, Eqs. QP, GWQP, Z, A).  For every entry b (a band,
 * or a band and k point) with Sigma_b(i omega_k) at the nodes omega_h [n]
 * (sigma_iw_h [n_n][n] complex, as gw_sigma_diag returns it), the Thiele
 * approximant of Eqs. pade1, pade2 is built again and, with real frequencies
 * measured from mu as in gw_sigma_diag,
 *   Z_b = 1 / (1 - d Re Sigma_b(w - mu) / dw at w = eps_b)
 *   E_b = eps_b + Z_b Re(v_b + Sigma_b(eps_b - mu) - eps_b)
 *   A_b(w) = |Im D| / pi / ((w - eps_b - Re D)^2 + (Im D)^2),  D = v_b + Sigma_b(w - mu) - eps_b.
 * eps_h [n_n]: the entries' Kohn-Sham energies (Ha); vstat_h [n_n]: the
 * frequency-independent rest of the paper's Sigma plus <T + V_ne + V_H>
 * (e.g. bare exchange + core-valence exchange + eps_b - <V_xc>_b).  The
 * derivative is the continued fraction's own (quotient rule on the backward
 * recursion), not a finite difference.  w_h [n_w] absolute real energies.
 * Outputs (host): e_qp_h [n_n]; z_h [n_n], sigma_eps_h [n_n] complex
 * Sigma_b(eps_b - mu), dsigma_h [n_n] complex derivative (each may be NULL);
 * spectral_h [n_n][n_w] (1/Ha; needed when n_w > 0).  1 <= n <= 32, distinct
 * omega > 0.  Synchronous.  GW_ERR_NUMERIC (naming the entry) if a reciprocal
 * difference or a denominator vanishes or Z is not finite; the other entries
 * are still returned. */
gw_status gw_qp_energies(gw_ctx* ctx, int n_n, int n, const double* omega_h, const double* sigma_iw_h,
                         const double* eps_h, double mu, const double* vstat_h, int n_w,
                         const double* w_h, double* e_qp_h, double* z_h, double* sigma_eps_h,
                         double* dsigma_h, double* spectral_h, void* stream);

/* The chi0 chain of Fig. 1 steps (1)-(3) in one call: for every tau_j and every
 * r-block of r_block rows, fused G formation + Hadamard + row transform into the
 * chi(r,G',tau_j) slab (Eqs. chi_rr, FFTX1; chi(r,R') is never stored whole, as
 * in Sec. II.C step (i)), then the column transform (Eq. FFTX2) and the cosine
 * transform (Eq. CTX) fused into one pass:
 *   chi_w [n][n_chi][n_chi] = chi0(G,G',i omega_k),  k < n.
 * C_h [n][n] as from gw_fit_transform.  r_block <= 0 picks a default. */
gw_status gw_chi0_omega(gw_ctx* ctx, const gw_grid* grid, int n_b, int n_occ,
                        const void* psi, const double* eps_h, double mu, int n,
                        const double* tau_h, const double* C_h, int n_chi,
                        const int32_t* fft_index_h, gw_prec prec, int r_block, void* chi_w,
                        void* stream);

/* chi0(G,G',i omega_k) as gw_chi0_omega, with G taken through its plane-wave
 * form (the paper evaluates G in a plane-wave representation and Fourier
 * transforms it to real space when needed, Sec. II.B; at one k point Eqs.
 * FFT_G1, FFT_G2 are two ordinary transforms).  The orbitals must lie in the
 * span of the n_pw plane waves e^{+i g.r} whose g sit at the FFT positions
 * pw_index_h[n_pw] (the formula of fft_index_h); each band's coefficients
 * D_a(g) = sum_r psi_a(r) e^{-i g.r} must hold its whole norm (Parseval,
 * relative 1e-5; 1e-10 for GW_FP64), else GW_ERR_ARG names the band.  Per tau_j:
 *   M(g,g') = sum_a f_a D_a(g) conj(D_a(g')) / N_r^2     (occupied, unoccupied)
 * over the set, a contraction of n_pw^2 N_b instead of N_r^2 N_b (tcgen05 for
 * GW_F16X3 / GW_BF16X3), its column transform over the grid, and one row pass
 * that expands both rows over R', forms chi(r,R') = -2 G_occ conj(G_unocc)
 * (Eq. chi_rr) and transforms it onto the G set (Eq. FFTX1); then Eqs. FFTX2
 * and CTX as in gw_chi0_omega.  Scratch (context arena): the slabs
 * (N_r n_chi n elements) plus 2 N_r n_pw + 2 n_pw^2 + N_b n_pw elements (8 or 16
 * bytes each) and the tensor-core operands.  GW_ERR_UNSUPPORTED where two
 * expanded rows of the grid do not fit a thread-block cluster's shared memory
 * (GW_FP64 at 36^3, every precision at 48^3).  Synchronises the stream once
 * (the norm check). */
gw_status gw_chi0_omega_pw(gw_ctx* ctx, const gw_grid* grid, int n_b, int n_occ, const void* psi,
                           const double* eps_h, double mu, int n, const double* tau_h, const double* C_h,
                           int n_chi, const int32_t* fft_index_h, int n_pw, const int32_t* pw_index_h,
                           gw_prec prec, void* chi_w, void* stream);

/* gw_sigma_diag with G through its plane-wave form (as gw_chi0_omega_pw; same
 * pw_index_h convention and span check).  Per tau_j: the plane-wave G
 * formation and its column transform, W~(r, G') from the column transform of
 * w_tau (Eq. FFTW, first step), then per row r one pass that expands W~(r,.),
 * G_unocc(r,.) and G_occ(r,.) over R', forms H = W~ G and transforms it back
 * onto the plane waves, h(r, g) = sum_R' H(r,R') e^{+i g.R'}; with the Sigma
 * bands' coefficients c_n (psi_n = sum_g c_n(g) e^{+i g.r})
 *   sum_R' H(r,R') psi_n(R') = sum_g h(r,g) c_n(g)
 * (a GEMM), and Sigma_nn(+-tau_j) as in gw_sigma_diag (first term of Eq.
 * Sigma_occ_reduce), then the same transforms and continuation.  Scratch
 * (context arena): N_r (n_chi + 4 n_pw + 2 n_n) + 2 n_pw^2 + (N_b + n_n) n_pw
 * elements (8 or 16 bytes) and the tensor-core operands.  GW_ERR_UNSUPPORTED
 * where the expanded rows do not fit a thread-block cluster (GW_FP64 at 36^3,
 * every precision at 48^3).  Synchronous. */
gw_status gw_sigma_diag_pw(gw_ctx* ctx, const gw_grid* grid, int n_b, int n_occ, const void* psi,
                           const double* eps_h, double mu, const int32_t* bands_h, int n_n, int n,
                           const double* tau_h, const double* omega_h, const double* C_h, const double* S_h,
                           const void* w_tau, int n_chi, const int32_t* fft_index_h, int n_pw,
                           const int32_t* pw_index_h, gw_prec prec, double* sigma_tau_h, double* sigma_iw_h,
                           const double* w_real_h, int n_real, double* sigma_real_h, void* stream);

/* chi0(q+G, q+G', i omega_k) for every q of a Gamma-centred nk[0] x nk[1] x nk[2]
 * k mesh, through the supercell stripe of Sec. II.A (spatial transform within
 * a supercell, Eqs. FFT_G1, FFT_G2): for every tau_j and block of cell rows r,
 * G_occ,k / G_unocc,k (Eqs. Green_occ/unocc over the orbitals of k), the stripe
 *   G(r, r'+L) = (1/N_k) sum_k exp(-i k.L) G_k(r, r')     (L: cell lattice vectors of the supercell)
 * and chi(r, R') = -2 G_occ(r, R') conj(G_unocc(r, R')) on the supercell grid,
 * the transform over R' to the supercell G set {q + g'}, then per q the factor
 * exp(-i q.r), the transform over r with dV^2/Omega (Eq. FFTX2) and the cosine
 * transform (Eq. CTX):
 *   chi_w [N_k][n][n_chi][n_chi] = chi_q(g, g', i omega_k),  q in k order.
 * psi_k: device [N_k][n_b][N_r], the Bloch orbitals exp(i k.r) u_nk(r) of each k
 * on the cell grid, normalised as at Gamma; k index (k1 nk[1] + k2) nk[2] + k3
 * for k = sum_d (k_d / nk[d]) b_d, k_d in [0, nk[d]).  eps_k_h [N_k][n_b]
 * ascending per k with mu in every gap.  gvec_h [n_chi][3]: the cell G set as
 * integer triples with g_d in [-n_d/2, n_d/2).  At most 64 k points; the
 * supercell grid nk[d] n_d must be one the library compiles.  r_block <= 0
 * picks a default.  The result is the q-diagonal block of the Gamma-point
 * chi0 of the supercell holding the N_k cells. */
gw_status gw_chi0_omega_kmesh(gw_ctx* ctx, const gw_grid* grid, const int* nk, int n_b, int n_occ,
                              const void* psi_k, const double* eps_k_h, double mu, int n,
                              const double* tau_h, const double* C_h, int n_chi, const int32_t* gvec_h,
                              gw_prec prec, int r_block, void* chi_w, void* stream);

/* chi_w as gw_chi0_omega_kmesh, with every G_k taken through its plane-wave
 * form (Sec. II.B, Eqs. G1_unocc_k, G1_occ_k; the stripe by Eqs. FFT_G1,
 * FFT_G2).  The cell-periodic parts u_nk = exp(-i k.r) psi_nk of every orbital
 * must lie in the span of the n_pw plane waves e^{+i g.r} at the cell FFT
 * positions pw_index_h[n_pw] (one set for all k; checked per band and k by
 * Parseval as in gw_chi0_omega_pw, else GW_ERR_ARG).  Per tau_j and k: the
 * matrix over the set from the coefficients of u_nk (tcgen05 for GW_F16X3 /
 * GW_BF16X3) and its column transform T_k(r, g') over the cell grid; the stripe
 * row r is exp(-i k.r) T_k(r, g') / N_k at the supercell plane waves k + nk g'
 * of every k, and one row pass over the supercell grid expands both Green's
 * functions over R', forms -2 G_occ conj(G_unocc) and transforms it onto the
 * supercell G set {q + g}; the rest as gw_chi0_omega_kmesh.  Scratch (context
 * arena): the slabs (N_r N_k n_chi n elements) plus 2 N_r N_k n_pw + 2 n_pw^2 +
 * N_k N_b n_pw + N_b N_r elements and the tensor-core operands.
 * GW_ERR_UNSUPPORTED where two expanded supercell rows do not fit a
 * thread-block cluster (supercells beyond 36^3, GW_FP64 at 36^3).  Synchronises
 * the stream once per k (the norm check). */
gw_status gw_chi0_omega_kmesh_pw(gw_ctx* ctx, const gw_grid* grid, const int* nk, int n_b, int n_occ,
                                 const void* psi_k, const double* eps_k_h, double mu, int n,
                                 const double* tau_h, const double* C_h, int n_chi, const int32_t* gvec_h,
                                 int n_pw, const int32_t* pw_index_h, gw_prec prec, void* chi_w, void* stream);

/* Diagonal self-energy of Bloch states on the k mesh of gw_chi0_omega_kmesh:
 * the space-time route of gw_sigma_diag on the supercell stripe.  For every
 * tau_j, W~(r, R') = (1/Omega_S) sum_q sum_{g,g'} exp(i(q+g).r) W~_q(g,g') exp(-i(q+g').R')
 * (Eq. FFTW on the supercell, whose W~ is block-diagonal in q), G_occ / G_unocc
 * on the stripe as for chi0, and
 *   Sigma_unocc_nk(tau) = +dV^2 sum_{r in C} sum_{R' in S} psi*_nk(r) G_unocc(r,R') W~(r,R') psi_nk(R')
 *   Sigma_occ_nk(-tau)  = -dV^2 ... G_occ ...,   psi_nk(r'+L) = exp(i k.L) psi_nk(r'),
 * then the even/odd split, CT + ST and Thiele continuation of gw_sigma_diag.
 * bk_h [n_n][2]: (band, k index) pairs; w_tau [N_k][n][n_chi][n_chi]:
 * W~_q(g, g', tau_j) for every q (e.g. gw_screen_W per q with the supercell G
 * triples q + nk g, then gw_tau_to_omega); the other arguments and outputs as
 * for gw_chi0_omega_kmesh and gw_sigma_diag (outputs per pair).  Synchronous. */
gw_status gw_sigma_diag_kmesh(gw_ctx* ctx, const gw_grid* grid, const int* nk, int n_b, int n_occ,
                              const void* psi_k, const double* eps_k_h, double mu, const int32_t* bk_h, int n_n,
                              int n, const double* tau_h, const double* omega_h, const double* C_h,
                              const double* S_h, const void* w_tau, int n_chi, const int32_t* gvec_h,
                              gw_prec prec, double* sigma_tau_h, double* sigma_iw_h, const double* w_real_h,
                              int n_real, double* sigma_real_h, void* stream);

/* ---------------------------------------------------------------- plans
 * gw_chi0_omega split into a set-up and a launch, for callers that replay the
 * same chi0 evaluation (serving) or capture it in a CUDA graph: the launch
 * issues kernels and device-side memsets only, with no host-device copy and no
 * synchronisation.  The paper has no counterpart. */
typedef struct gw_chi0_plan gw_chi0_plan;
/* Everything of gw_chi0_omega but psi and chi_w: validates, computes the
 * tables on the host, copies them to a device buffer the plan owns
 * (synchronous) and grows ctx's arena to what a launch needs.  Plans made from
 * one context share its arena: launch them in order (one stream or one graph),
 * and do not interleave other calls on that context between a launch and its
 * gw_chi0_plan_status. */
gw_status gw_chi0_plan_create(gw_ctx* ctx, const gw_grid* grid, int n_b, int n_occ, const double* eps_h,
                              double mu, int n, const double* tau_h, const double* C_h, int n_chi,
                              const int32_t* fft_index_h, gw_prec prec, int r_block, gw_chi0_plan** out);
/* The kernels of gw_chi0_omega for this plan on `stream`: psi [n_b][N_r] and
 * chi_w [n][n_chi][n_chi] on the device, as for gw_chi0_omega.  Asynchronous;
 * pointers are read at launch (a captured graph keeps those of the capture). */
gw_status gw_chi0_plan_launch(gw_chi0_plan* plan, const void* psi, void* chi_w, void* stream);
/* Waits for `stream` and reports a time-out recorded by the tensor-core
 * kernels of the last launch (GW_ERR_TIMEOUT). */
gw_status gw_chi0_plan_status(gw_chi0_plan* plan, void* stream);
/* Frees the plan's tables (synchronises the device). */
gw_status gw_chi0_plan_destroy(gw_chi0_plan* plan);

/* ---------------------------------------------------------------- batches
 * Many uneven systems through the whole hot path in one CUDA-graph launch (the
 * batched form of the serving layer; the paper has no counterpart).  Per
 * system: chi0(i omega) (as gw_chi0_omega), W~(i omega) (gw_screen_W_refine
 * with refine_iters), W~(i tau) (gw_tau_to_omega with Cinv) and the diagonal
 * self-energy Sigma_nn(i omega) with its Thiele coefficients (gw_sigma_diag
 * without real-axis points).  gw_batch_plan does all host work once
 * (validation, tables, weights, uploads, the context arena grown to the
 * largest need) and records the kernels of every system, in order, into one
 * CUDA graph; gw_batch_launch replays it with no host work and no
 * host-device copy; gw_batch_wait waits (bounded) and reads the results.
 * The systems share the context's arena and run one after the other inside
 * the graph.  A plan is invalidated if the context's arena is reallocated
 * afterwards (a later call on the context that needs more scratch):
 * gw_batch_launch then returns GW_ERR_ARG. */
typedef struct gw_batch gw_batch;
typedef struct gw_batch_system {
  gw_grid grid;
  int n_b, n_occ;
  const double* eps_h;          /* host [n_b], ascending, mu in the gap          */
  double mu;
  int n;                        /* tau / omega points (<= 32)                   */
  const double* tau_h;          /* host [n]                                     */
  const double* omega_h;        /* host [n]                                     */
  const double* C_h;            /* host [n][n] cosine transform (gw_fit_transform) */
  const double* S_h;            /* host [n][n] sine transform                   */
  const double* Cinv_h;         /* host [n][n] inverse cosine transform          */
  int n_chi;
  const int32_t* gvec_h;        /* host [n_chi][3] G set (gw_g_set)              */
  const int32_t* fft_index_h;   /* host [n_chi]                                  */
  int n_n;                      /* self-energy bands                            */
  const int32_t* bands_h;       /* host [n_n]                                   */
  int r_block;                  /* rows per r-block of the chi0 pass (e.g. from an autotuner); <= 0: default */
  int refine_iters;             /* 0..8 refinement steps of the screening        */
  const void* psi;              /* device [n_b][N_r], 16-byte aligned            */
  void* chi_w;                  /* device [n][n_chi][n_chi] work: chi0(i omega), then W~(i omega) */
  void* w_tau;                  /* device [n][n_chi][n_chi]: W~(i tau) (not overlapping chi_w) */
} gw_batch_system;
/* Host pointers are read during the call only; device pointers are recorded
 * in the graph and must stay valid while the plan is used. */
gw_status gw_batch_plan(gw_ctx* ctx, int n_sys, const gw_batch_system* systems, gw_prec prec, gw_batch** out);
/* Replays the graph on `stream` (asynchronous). */
gw_status gw_batch_launch(gw_batch* batch, void* stream);
/* Waits at most timeout_ms (< 0: no limit) for the last launch; GW_ERR_TIMEOUT
 * if it has not finished (the work continues; call again).  Then
 * sigma_iw_h (host, may be NULL) receives every system's Sigma_nn(i omega)
 * [n_n][n] complex, one system after the other, and status_h [n_sys] (may be
 * NULL) each system's gw_status (GW_ERR_NUMERIC for a non-positive-definite
 * eps~ or a vanishing Thiele denominator, GW_ERR_TIMEOUT for a tensor-core
 * wait that gave up); the call returns the first failure. */
gw_status gw_batch_wait(gw_batch* batch, int timeout_ms, double* sigma_iw_h, int* status_h);
/* Frees the plan (synchronises its stream). */
gw_status gw_batch_destroy(gw_batch* batch);

#ifdef __cplusplus
}
#endif
#endif /* GW_H_ */
