// Complex GEMM on CUDA cores (FP32 or FP64), used by the SIMT precisions of
// the Green's-function contraction and by the blocked Cholesky / triangular
// inverse of the screening step.  64x64 output tile per 256-thread CTA, 4x4
// complex outputs per thread on an interleaved (stride-16) pattern so that the
// shared-memory reads of a warp are broadcasts or consecutive.
#include "gw_kernels.h"

namespace gw {

template <typename T>
struct GemmP {
  using C = typename cpx<T>::t;
  int M, N, K;
  C alpha;
  T beta;
  const C* A;
  long lda;
  const C* B;
  long ldb;
  C* Cm;
  long ldc;
  const T* kscale;
  long sA, sB, sC;
};

template <typename T, int AKM, bool AC, int BNK, bool BC, bool SCALE, int TRI>
__global__ void __launch_bounds__(256) cgemm_kernel(GemmP<T> p) {
  using C = typename cpx<T>::t;
  constexpr int BM = 64, BN = 64, BK = 8, PAD = 1;
  __shared__ C As[BK][BM + PAD];
  __shared__ C Bs[BK][BN + PAD];
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  if (TRI && n0 > m0 + BM - 1) return;
  p.A += blockIdx.z * p.sA;
  p.B += blockIdx.z * p.sB;
  p.Cm += blockIdx.z * p.sC;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  // FP32 sums are blocked: acc collects KBLK terms of k, then is added to tot.
  // A sequential FP32 sum over K terms has a relative rounding error growing
  // like u sqrt(K/2); blocking by ~sqrt(K) brings it to ~u K^(1/4) (4x less at
  // K = 1024) for one extra add per KBLK terms.
  constexpr int KBLK = sizeof(T) == 4 ? 32 : 0;
  C acc[4][4], tot[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = tot[i][j] = mk(T(0), T(0));
  const int kbeg = TRI == 2 ? m0 : 0;
  for (int k0 = kbeg; k0 < p.K; k0 += BK) {
    if (KBLK && k0 != kbeg && (k0 - kbeg) % KBLK == 0) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          tot[i][j] = cadd(tot[i][j], acc[i][j]);
          acc[i][j] = mk(T(0), T(0));
        }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int e = tid + 256 * q;
      int ml, kl;
      if (AKM) { kl = e / BM; ml = e % BM; } else { ml = e / BK; kl = e % BK; }
      const int m = m0 + ml, k = k0 + kl;
      C v = mk(T(0), T(0));
      if (m < p.M && k < p.K) {
        v = AKM ? p.A[(long)k * p.lda + m] : p.A[(long)m * p.lda + k];
        if (AC) v = cconj(v);
        if (SCALE) v = cscale(v, p.kscale[k]);
      }
      As[kl][ml] = v;
      int nl, kb;
      if (BNK) { nl = e / BK; kb = e % BK; } else { kb = e / BN; nl = e % BN; }
      const int n = n0 + nl, kk = k0 + kb;
      C w = mk(T(0), T(0));
      if (n < p.N && kk < p.K) {
        w = BNK ? p.B[(long)n * p.ldb + kk] : p.B[(long)kk * p.ldb + n];
        if (BC) w = cconj(w);
      }
      Bs[kb][nl] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      C a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fma(a[i].x, b[j].x, fma(-a[i].y, b[j].y, acc[i][j].x));
          acc[i][j].y = fma(a[i].x, b[j].y, fma(a[i].y, b[j].x, acc[i][j].y));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m >= p.M || n >= p.N) continue;
      if (TRI && m < n) continue;
      C v = cmul(p.alpha, cadd(tot[i][j], acc[i][j]));
      C* dst = p.Cm + (long)m * p.ldc + n;
      if (p.beta != T(0)) v = cadd(v, cscale(*dst, p.beta));
      *dst = v;
    }
}

template <typename T>
static gw_status run_gemm(gw_ctx* ctx, const GemmArgs& a, cudaStream_t st) {
  using C = typename cpx<T>::t;
  GemmP<T> p;
  p.M = a.M;
  p.N = a.N;
  p.K = a.K;
  p.alpha = mk(T(a.alpha_re), T(a.alpha_im));
  p.beta = T(a.beta);
  p.A = (const C*)a.A;
  p.lda = a.lda;
  p.B = (const C*)a.B;
  p.ldb = a.ldb;
  p.Cm = (C*)a.C;
  p.ldc = a.ldc;
  p.kscale = (const T*)a.kscale;
  p.sA = a.sA;
  p.sB = a.sB;
  p.sC = a.sC;
  dim3 grid((a.N + 63) / 64, (a.M + 63) / 64, a.batch > 0 ? a.batch : 1);
  if (grid.y > 65535) return fail(ctx, GW_ERR_SHAPE, "GEMM M too large");
#define GW_GEMM_CASE(AKM, AC, BNK, BC, SC, TRI)                                                   \
  if (a.a_km == AKM && a.a_conj == AC && a.b_nk == BNK && a.b_conj == BC && (a.kscale != nullptr) == SC && \
      a.tri == TRI) {                                                                               \
    KTimer kt(ctx, KF_CGEMM_SIMT, grid.z * gemm_flops(a.M, a.N, a.K, TRI), st);                   \
    cgemm_kernel<T, AKM, AC, BNK, BC, SC, TRI><<<grid, 256, 0, st>>>(p);                           \
    return launch_check(ctx, "cgemm_kernel");                                                       \
  }
  GW_GEMM_CASE(1, false, 0, true, true, 0)    // Green's functions: psi^T diag(s) conj(psi)
  GW_GEMM_CASE(0, false, 1, true, false, 1)   // Hermitian rank-k update: C -= L21 L21^H (lower)
  GW_GEMM_CASE(0, false, 0, false, false, 0)  // triangular-inverse update: C -= L_below X_i
  GW_GEMM_CASE(1, true, 0, false, false, 2)   // L^{-H} L^{-1}, lower triangle
  GW_GEMM_CASE(0, false, 0, false, false, 1)
  GW_GEMM_CASE(0, false, 1, true, false, 0)   // A B^H (plane-wave self-energy: h c^H)
#undef GW_GEMM_CASE
  return fail(ctx, GW_ERR_UNSUPPORTED, "GEMM layout combination not compiled");
}

gw_status launch_gemm(gw_ctx* ctx, gw_prec prec, const GemmArgs& a, cudaStream_t st) {
  if (a.M <= 0 || a.N <= 0) return GW_OK;
  return is_fp64(prec) ? run_gemm<double>(ctx, a, st) : run_gemm<float>(ctx, a, st);
}

}  // namespace gw
