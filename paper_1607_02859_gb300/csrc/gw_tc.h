// Tensor-core (tcgen05) split-precision contractions (internal).
#pragma once

#include <cuda.h>

#include "gw_kernels.h"

namespace gw {

// Scratch the two calls below need for n_rows rows (with_tmp: room for an
// output the caller did not supply).
size_t tc_scratch_bytes(const GridInfo& g, int n_b, int n_occ, int n_rows, bool with_tmp, int n_sig = 0);
// G_occ / G_unocc rows as 3 fp16 (or bf16) split products on tcgen05 with FP32
// accumulation in tensor memory.  Either output may be NULL.  prep_b = false
// reuses the psi-only operand an earlier call left in the same scratch.
gw_status tc_green_rows(gw_ctx* ctx, const GridInfo& g, int n_b, int n_occ, const void* psi,
                        const GreenScales& gs, int r0, int n_rows, gw_prec prec, void* g_occ, void* g_unocc,
                        void* scratch, bool prep_b, cudaStream_t st, const float* sk_dev = nullptr);
// chi rows = -2 G_occ o conj(G_unocc) with both tiles accumulated in tensor memory.
// sk_dev: the per-band factors gs.s already on the device as FP32 (then the
// call copies nothing from the host).
// lower: only R' <= r (grid rows r0 ..): the diagonal halved and zeros above it, whose
// transform X gives chi(G,G') = X + X^H (chi is Hermitian in (r, R')).
gw_status tc_chi_rows(gw_ctx* ctx, const GridInfo& g, int n_b, int n_occ, const void* psi, const GreenScales& gs,
                      int r0, int n_rows, gw_prec prec, void* chi, void* scratch, bool prep_b, cudaStream_t st,
                      const float* sk_dev = nullptr, int* status_dev = nullptr, bool lower = false);
// The self-energy contraction fused into the G formation of rows r0 .. r0+n_rows-1
// (first term of Eq. Sigma_occ_reduce): for every 128 x 128 tile with R' <= r
// (G o W~ is Hermitian in (r, R'), so the real quadratic form is twice its
// strictly lower part plus its diagonal), H = w G o W~ on CUDA cores (w = 2, 1),
// V_n = H psi_n on tcgen05, and
//   acc_u[n * acc_stride] += coef sum_r Re(conj(psi_n(r)) V_n^unocc(r)),  acc_o likewise with -coef.
// G never leaves the chip.  wrr: W~(r,R') rows of the block [n_rows][ldw] (FP32
// complex); bands: device [n_n], 1 <= n_n <= 32.  The scratch must come from
// tc_scratch_bytes(..., n_sig >= n_n); prep_b as for tc_green_rows (also
// prepares the psi_n operand).
struct TcSigma {
  const float2* wrr;
  long ldw;
  const int* bands;
  int n_n;
  double coef;
  double* acc_u;
  double* acc_o;
  int acc_stride;
  const float* sk = nullptr;   // the per-band factors gs.s on the device as FP32 (else copied per call)
};
gw_status tc_sigma_rows(gw_ctx* ctx, const GridInfo& g, int n_b, int n_occ, const void* psi, const GreenScales& gs,
                        int r0, int n_rows, gw_prec prec, const TcSigma& sig, void* scratch, bool prep_b,
                        cudaStream_t st);
// As tc_check for a status word the caller owns (status_dev of tc_chi_rows).
gw_status tc_check_status(gw_ctx* ctx, const int* status_dev, cudaStream_t st);
// Synchronises and reports a time-out of the tensor-core pipeline waits
// (GW_ERR_TIMEOUT) recorded in `scratch` since its last prep_b call.
gw_status tc_check(gw_ctx* ctx, void* scratch, cudaStream_t st);

// 2-D TMA map over a [rows][kpad] row-major 16-bit array (fmt 0: fp16, 1: bf16),
// box 64 x box_rows, 128-byte swizzle.
gw_status tc_make_map(gw_ctx* ctx, CUtensorMap* m, const void* base, int kpad, long rows, int box_rows,
                      uint32_t fmt);
// Same over a [batch][rows][kpad] array (3-D map, box depth 1), with a box of
// box_k elements along K and the matching swizzle (64 -> 128 B, 32 -> 64 B).
gw_status tc_make_map3(gw_ctx* ctx, CUtensorMap* m, const void* base, int kpad, long rows, int batch, int box_rows,
                       uint32_t fmt, int box_k);

// C = alpha * opA(A) opB(B) (+ C if accumulate) on tcgen05 tensor cores with
// split 16-bit products; opA(m,k) = A[m][k] or A[k][m] (a_trans), conjugated if
// a_conj; opB(k,n) = B[k][n] or B[n][k] (b_trans), conjugated if b_conj.
// tri = 1: only m >= n; tri = 2: also start each tile's k loop at its first row.
// The operands are converted to split copies first, so C may alias A or B.
struct TcGemm {
  int M, N, K;
  const float2* A;
  long lda;
  bool a_trans, a_conj;
  const float2* B;
  long ldb;
  bool b_trans, b_conj;
  float2* C;
  long ldc;
  float alpha;
  bool accumulate;
  int tri;
  int* status;          // device: 2 ints, set on a pipeline time-out
  int batch = 1;        // independent products sA/sB/sC elements apart (grid z)
  long sA = 0, sB = 0, sC = 0;
};
size_t tc_gemm_scratch(int M, int N, int K, int batch);
gw_status tc_gemm(gw_ctx* ctx, gw_prec prec, const TcGemm& g, void* scratch, cudaStream_t st);

// C = A B for complex FP64 A [M][K] (lda), B [K][N] (ldb), C [M][N] (ldc, written)
// with FP64-class accuracy from exact fp16 slice products on tcgen05 (slice pairs
// a + b <= levels, 6 bits per slice; error below 2^(-6(levels+1)) of the row and
// column maxima).  status: device words set on a pipeline time-out.
size_t tc_zgemm_sliced_scratch(int M, int N, int K, int levels);
gw_status tc_zgemm_sliced(gw_ctx* ctx, int M, int N, int K, const double2* A, long lda, const double2* B, long ldb,
                          double2* C, long ldc, int levels, int* status, void* scratch, cudaStream_t st);

}  // namespace gw
