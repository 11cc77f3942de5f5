// Launchers shared between the libgw translation units (internal).
#pragma once

#include "gw_common.cuh"

namespace gw {

// gw_fft.cu
// Rows whose shared-memory copy exceeds kRowSmemMax go through two passes
// (row_two_pass(g, prec)); those need inv (grid position -> G index or -1) and,
// forward, a [n_rows][N_r] workspace tmp (which may be a itself for mode 0).
constexpr size_t kRowSmemMax = 227 * 1024;
gw_status launch_row_fft(gw_ctx* ctx, const GridInfo& g, gw_prec prec, int mode, const void* a, const void* b,
                         long lda, void* out, long ldo, const int* map, int n_chi, int n_rows, double scale,
                         cudaStream_t st, const int* inv = nullptr, void* tmp = nullptr);
bool row_two_pass(const GridInfo& g, gw_prec prec);
// chi rows from the plane-wave form of G: a = T_unocc, b = T_occ rows [n_rows][lda]
// over the orbitals' plane-wave set (inv_pw: grid position -> set index or -1),
// out [n_rows][ldo] = FFT+(scale a conj(b)) on chi's G set (inv_chi).
gw_status launch_row_pw_chi(gw_ctx* ctx, const GridInfo& g, gw_prec prec, const void* a, const void* b, long lda,
                            void* out, long ldo, const int* inv_pw, int n_pw, const int* inv_chi, int n_chi,
                            int n_rows, double scale, cudaStream_t st);
// GW_OK if launch_row_pw_chi supports the grid, precision and set sizes.
gw_status check_row_pw(gw_ctx* ctx, const GridInfo& g, gw_prec prec, int n_pw, int n_chi);
// Sigma rows in the plane-wave form: tu, to [n_rows][ldt] (T rows over the negated
// plane-wave set), wg [n_rows][ldw] (W~ over chi's G set) -> hu, ho [n_rows][ldh] =
// FFT+(W~ conj(G')) gathered on the plane-wave set (inv_nat).
gw_status launch_row_pw_sigma(gw_ctx* ctx, const GridInfo& g, gw_prec prec, const void* tu, const void* to, long ldt,
                              const void* wg, long ldw, void* hu, void* ho, long ldh, const int* inv_neg,
                              const int* inv_nat, int n_pw, const int* inv_chi, int n_chi, int n_rows,
                              cudaStream_t st);
gw_status check_row_pw_sigma(gw_ctx* ctx, const GridInfo& g, gw_prec prec, int n_pw, int n_chi);

// gw_pipeline.cu: the plane-wave form of G.  pw_negate turns the FFT positions
// of the orbitals' plane waves e^{+i g.r} into those of -g (where the forward
// coefficients sit) and rebuilds inv; pw_coefficients writes
// dc [n_b][n_pw] = conj(D)/N_r, D_a = sum_r psi_a(r) e^{+i g'.r} at the negated set,
// after checking (one synchronisation) that every band lies in the set's span;
// pw_grid is the GridInfo of the G formation over the set.
void pw_negate(const GridInfo& g, std::vector<int>& map, std::vector<int>& inv);
gw_status pw_coefficients(gw_ctx* ctx, const GridInfo& g, gw_prec prec, const void* psi, int n_b, int n_pw,
                          const int* dmap_neg, const int* dinv_neg, void* dc, double* dnorm, void* tmp,
                          cudaStream_t s);
GridInfo pw_grid(const GridInfo& g, int n_pw);

// gw_sigma.cu: the Sigma contraction over rows of G_occ, G_unocc, W~ (length
// nr, leading dimension ld) against psi_n (rows of length nr; the row's own
// value read from psi_row [.][ld_row] if given, else from psi), and the finish
// (even/odd split, CT + ST, Thiele, results to the host).  With vout, the
// contraction stores V_m(r) in vout [2][n_n][vstride] instead of reducing the
// diagonal (the matrix Sigma_nm).
gw_status launch_sigma_contract(gw_ctx* ctx, gw_prec prec, const void* wrr, const void* go, const void* gu, long ld,
                                int nr, int rows, const void* psi, const int* bands, int n_n, int r0, double coef,
                                double* acc_u, double* acc_o, int acc_stride, cudaStream_t st,
                                const void* psi_row = nullptr, long ld_row = 0, double2* vout = nullptr,
                                int vstride = 0);
gw_status sigma_finish(gw_ctx* ctx, double* acc, int n_n, int n, const double* tab, int n_real, double2* out,
                       int* stat, const int32_t* labels, double* sigma_tau_h, double* sigma_iw_h,
                       double* sigma_real_h, cudaStream_t s);
gw_status launch_col_plane(gw_ctx* ctx, const GridInfo& g, gw_prec prec, int dir, void* buf, long ld, int ncols,
                           double scale, cudaStream_t st);
gw_status launch_col_line(gw_ctx* ctx, const GridInfo& g, gw_prec prec, int dir, int variant, const void* in,
                          long ldi, void* out, long ldo, int ncols, const int* inv, double scale, cudaStream_t st);
gw_status launch_col_line_ct(gw_ctx* ctx, const GridInfo& g, gw_prec prec, const void* slabs, long slab_stride,
                             long ld, int ntau, const void* cw, int nw, void* out, long out_slice, long ldo,
                             const int* inv, int ncols, cudaStream_t st, const float* cw_h = nullptr);
gw_status launch_ct(gw_ctx* ctx, gw_prec prec, bool st_kind, int n, const void* dM, size_t elems, const void* in,
                    void* out, cudaStream_t st, const float* w_h = nullptr);
gw_status launch_hadamard(gw_ctx* ctx, gw_prec prec, size_t count, const void* a, const void* b, double scale,
                          void* out, cudaStream_t st);
gw_status upload(gw_ctx* ctx, void* dst, const void* src, size_t bytes, cudaStream_t st);
// FP32 weights of a transform as hi[count] then lo[count], hi + lo = fac * w to ~2^-48.
std::vector<float> split_weights(const double* w, int count, double fac);
gw_status index_maps(gw_ctx* ctx, const GridInfo& g, const int32_t* fft_index_h, int n_chi, std::vector<int>& map,
                     std::vector<int>& inv);

// gw_gemm.cu: C = alpha * op(A) op(B) + beta * C on CUDA cores (complex).
//  a(m,k) = A[m*lda+k] (a_km = 0) or A[k*lda+m] (a_km = 1), conjugated if a_conj;
//  b(k,n) = B[k*ldb+n] (b_nk = 0) or B[n*ldb+k] (b_nk = 1), conjugated if b_conj;
//  kscale (real, length K) multiplies a(m,k) if not NULL;
//  tri = 1 computes only the lower triangle (m >= n); tri = 2 additionally
//  starts the k loop at the first row of each tile (for L^H L with L lower).
struct GemmArgs {
  int M, N, K;
  double alpha_re, alpha_im, beta;
  const void* A; long lda; int a_km; bool a_conj;
  const void* B; long ldb; int b_nk; bool b_conj;
  void* C; long ldc;
  const void* kscale;
  int tri;
  int batch = 1;              // grid z: independent problems sA/sB/sC elements apart
  long sA = 0, sB = 0, sC = 0;
};
gw_status launch_gemm(gw_ctx* ctx, gw_prec prec, const GemmArgs& a, cudaStream_t st);

// gw_green.cu: pre-scaled exponentials of Eqs. Green_occ/unocc for one tau.
struct GreenScales {
  std::vector<double> s;   // [N_b], s_i / max over the occupied set and s_a / max over the unoccupied set
  double amax_occ, amax_unocc;
};
GreenScales green_scales(const double* eps, int n_b, int n_occ, double mu, double tau);
gw_status green_rows(gw_ctx* ctx, const GridInfo& g, int n_b, int n_occ, const void* psi, const void* dscale,
                     const GreenScales& gs, int r0, int n_rows, gw_prec prec, void* g_occ, void* g_unocc,
                     cudaStream_t st);

}  // namespace gw

namespace gw {
// scratch each composite call reserves in the context arena
size_t chi0_omega_scratch(const GridInfo& g, int n_b, int n_occ, int n, int n_chi, gw_prec prec, int rb);
size_t screen_scratch(int n_chi, int n_omega, gw_prec prec, int* bsz_out, int* nbatch_out, bool refine = false);
size_t sigma_scratch(const GridInfo& g, int n_b, int n_occ, int n, int n_chi, int n_n, int n_real, gw_prec prec,
                     bool full = false);
gw_status upload_scales(gw_ctx* ctx, void* dst, const GreenScales& gs, gw_prec prec, cudaStream_t st);

// ---- chi0 plans (gw_pipeline.cu), as used by the batch plans
int* chi0_plan_status_words(gw_chi0_plan* p);
size_t chi0_plan_work(const gw_chi0_plan* p);

// ---- the screening without host work (gw_dyson.cu); see its definition
gw_status screen_launch(gw_ctx* ctx, int n_chi, int n_omega, gw_prec prec, int refine_iters, const double* dvh,
                        const void* chi_w, void* w_w, Carver& cv, double* resid_h, int* first_bad, cudaStream_t s);

// ---- the self-energy pass split for plans (gw_sigma.cu)
// Device tables of one evaluation: G-set maps, bands, per-tau band factors
// (n_b 8-byte slots per tau, packed in the working precision), C, S, omega and
// real frequencies, the accumulators, the results and the Thiele status.
struct SigmaTables {
  int* map;
  int* inv;
  int* bands;
  char* scale;
  double* tab;
  double2* acc2;
  double2* out;
  int* stat;
};
// Work buffers of one evaluation (r-block rows of G and W~, the W~(r,G') plane
// stack, tensor-core scratch).
struct SigmaWork {
  bool fused;
  double2* vout;
  char* wrg;
  char* gob;
  char* gub;
  char* wrr;
  void* tcs;
};
void sigma_carve_tables(Carver& cv, const GridInfo& g, int n_b, int n, int n_chi, int n_n, int n_real, bool full,
                        SigmaTables& t);
void sigma_carve_work(Carver& cv, const GridInfo& g, int n_b, int n_occ, int n_chi, int n_n, gw_prec prec, bool full,
                      SigmaWork& w);
gw_status sigma_check(gw_ctx* ctx, const gw_grid* grid, GridInfo* g, int n_b, int n_occ, const void* psi,
                      const double* eps_h, double mu, const int32_t* bands_h, int n_n, int n, const double* tau_h,
                      const double* omega_h, const double* C_h, const double* S_h, const void* w_tau, int n_chi,
                      const int32_t* fft_index_h, gw_prec prec, bool full, const double* w_real_h, int n_real,
                      std::vector<int>& map, std::vector<int>& inv, std::vector<GreenScales>& scales);
gw_status sigma_upload_tables(gw_ctx* ctx, const SigmaTables& t, const GridInfo& g, int n_b, int n, int n_chi,
                              const std::vector<int>& map, const std::vector<int>& inv, const int32_t* bands_h, int n_n,
                              const std::vector<GreenScales>& scales, const double* C_h, const double* S_h,
                              const double* omega_h, const double* w_real_h, int n_real, gw_prec prec, cudaStream_t s);
gw_status sigma_kernels(gw_ctx* ctx, const GridInfo& g, gw_prec prec, bool full, int n_b, int n_occ, const void* psi,
                        int n_n, int n, int n_chi, int n_real, const std::vector<GreenScales>& scales,
                        const SigmaTables& t, const SigmaWork& w, const void* w_tau, cudaStream_t s);
gw_status sigma_finish_launch(gw_ctx* ctx, const double* acc, int n_n, int n, const double* tab, int n_real,
                              double2* out, int* stat, cudaStream_t s);
}  // namespace gw
