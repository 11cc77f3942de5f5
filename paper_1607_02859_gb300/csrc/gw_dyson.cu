// Screened interaction W~ (Eqs. W_tot, bareV, die, W_correlated).
//
// With chi~ = v^{1/2} chi v^{1/2} Hermitian negative semidefinite, the matrix
// eps~ = 1 - chi~ is Hermitian positive definite with eps~ >= 1, so
//   W~ = v^{1/2} (eps~^{-1} - 1) v^{1/2}
// follows from a Cholesky factorisation without pivoting.  The identity is
// carried implicitly so that nothing is ever formed as "1 + small" and then
// subtracted again (at large omega chi~ is tiny and such a round trip would
// lose its low digits):
//   B = eps~ - 1 = -chi~,  eps~ = L L^H with L = 1 + K on the diagonal,
//   L_jj - 1 = B'_jj / (1 + sqrt(1 + B'_jj))  (B' = B after the updates),
//   L^{-1} = 1 + P,
//   eps~^{-1} - 1 = P + P^H + P^H P.
// N^3/2 complex multiply-adds in all (Cholesky, L^{-1}, P^H P: N^3/6 each),
// instead of the N^3 + N^3/6 of a solve against chi~ with N right-hand sides.
//
// The frequencies are independent, so every launch works on a batch of them
// (grid z): the chain of small sequential launches on the diagonal blocks is
// paid once per batch instead of once per frequency, and the GEMMs grow.
//  * CUDA-core precisions: 64-column panels; the trailing updates are CUDA-core
//    complex GEMMs.
//  * tensor-core precisions: 512-column panels whose 512 x 512 diagonal blocks
//    are factored and inverted on CUDA cores; everything with a 512-wide inner
//    dimension is a tcgen05 GEMM with split 16-bit products:
//      L21 = A21 (1 + P11)^H,  A22 -= L21 L21^H,
//      P_i[:, <k0] += P_ii P_i[:, <k0],  rows below -= L_li (1 + P_i),
//      X = P^H P (one frequency per launch: the largest GEMM of the step).
#include <cmath>
#include <type_traits>

#include "gw_kernels.h"
#include "gw_tc.h"

namespace gw {

constexpr int kNB = 64;     // CUDA-core panel width
constexpr int kTB = 512;    // tensor-core panel width

// One CTA per row a (and batch entry): the lower part b <= a of the row.
template <typename T>
__global__ void __launch_bounds__(256) build_eps_kernel(const typename cpx<T>::t* __restrict__ chi, long s_chi,
                                                        const double* __restrict__ vh,
                                                        typename cpx<T>::t* __restrict__ E, long s_e, int n) {
  const int a = blockIdx.x;
  const double va = vh[a];
  const auto* src = chi + blockIdx.y * s_chi + (long)a * n;
  auto* dst = E + blockIdx.y * s_e + (long)a * n;
  for (int b = threadIdx.x; b <= a; b += blockDim.x) {
    const T vv = T(va * vh[b]);
    const auto x = src[b];
    dst[b] = mk(-vv * x.x, -vv * x.y);
  }
}

// Unblocked Cholesky (K form) of the kb x kb diagonal block, in shared memory.
template <typename T>
__global__ void __launch_bounds__(256) potrf_diag_kernel(typename cpx<T>::t* A, long lda, long s_a, int kb, int* flag,
                                                         int col0) {
  using C = typename cpx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C (*S)[kNB + 1] = reinterpret_cast<C (*)[kNB + 1]>(smem_raw);    // [kNB][kNB+1]
  A += blockIdx.z * s_a;
  for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
    const int i = e / kb, c = e % kb;
    S[i][c] = c <= i ? A[(long)i * lda + c] : mk(T(0), T(0));
  }
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    if (threadIdx.x == 0) {
      T b = S[j][j].x;                       // eps~_jj - 1 after the updates
      if (!(T(1) + b > T(0))) {
        if (atomicCAS(flag, 0, 1) == 0) {
          flag[1] = col0 + j;
          flag[2] = blockIdx.z;
        }
        b = T(0);
      }
      S[j][j] = mk(b / (T(1) + sqrt(T(1) + b)), T(0));   // L_jj - 1
    }
    __syncthreads();
    const T piv = T(1) + S[j][j].x;
    for (int i = j + 1 + threadIdx.x; i < kb; i += blockDim.x) S[i][j] = cscale(S[i][j], T(1) / piv);
    __syncthreads();
    const int m = kb - j - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = j + 1 + e / m, c = j + 1 + e % m;
      if (c <= i) S[i][c] = csub(S[i][c], cmulc(S[i][j], S[c][j]));
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
    const int i = e / kb, c = e % kb;
    if (c <= i) A[(long)i * lda + c] = S[i][c];
  }
}

// Rows below the diagonal block: x L11^H = a  ->  x (row of L21).  64 rows per CTA.
template <typename T>
__global__ void __launch_bounds__(64) trsm_panel_kernel(typename cpx<T>::t* A, long lda, long s_a, int k0, int kb,
                                                        int rows) {
  using C = typename cpx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* L = reinterpret_cast<C*>(smem_raw);          // [kb][kb+1]
  C* X = L + kNB * (kNB + 1);                       // [kb][64]  (column c of thread t at X[c*64+t])
  A += blockIdx.z * s_a;
  const int t = threadIdx.x;
  for (int e = t; e < kb * kb; e += blockDim.x) {
    const int i = e / kb, c = e % kb;
    L[i * (kNB + 1) + c] = c <= i ? A[(long)(k0 + i) * lda + k0 + c] : mk(T(0), T(0));
  }
  const long row = (long)k0 + kb + (long)blockIdx.x * 64 + t;
  const bool active = blockIdx.x * 64 + t < rows;
  if (active)
    for (int c = 0; c < kb; ++c) X[c * 64 + t] = A[row * lda + k0 + c];
  __syncthreads();
  if (!active) return;
  for (int c = 0; c < kb; ++c) {
    C s = X[c * 64 + t];
    for (int p = 0; p < c; ++p) s = csub(s, cmulc(X[p * 64 + t], L[c * (kNB + 1) + p]));
    X[c * 64 + t] = cscale(s, T(1) / (T(1) + L[c * (kNB + 1) + c].x));
  }
  for (int c = 0; c < kb; ++c) A[row * lda + k0 + c] = X[c * 64 + t];
}

// P[rows below][col0 .. col0+kb) = -L[rows below][col0 .. col0+kb): the identity
// part of (1 + P) contributes L_li * 1 to the update of the rows below block row i.
template <typename T>
__global__ void neg_copy_kernel(const typename cpx<T>::t* __restrict__ Lm, long ldl, long s_l,
                                typename cpx<T>::t* __restrict__ P, long ldp, long s_p, int row0, int rows, int col0,
                                int kb) {
  const long r = row0 + (long)blockIdx.x;
  if ((int)blockIdx.x >= rows) return;
  Lm += blockIdx.z * s_l;
  P += blockIdx.z * s_p;
  for (int c = threadIdx.x; c < kb; c += blockDim.x) {
    const auto v = Lm[r * ldl + col0 + c];
    P[r * ldp + col0 + c] = mk(-v.x, -v.y);
  }
}

// Y = L_ii^{-1} Y for the block rows k0..k0+kb-1 and columns 0..ncols-1 of Y,
// with the identity as right-hand side in the diagonal-block columns (their
// stored values are ignored) and P = L^{-1} - 1 stored on the diagonal.
template <typename T>
__global__ void __launch_bounds__(64) trsm_left_kernel(const typename cpx<T>::t* Lm, long ldl, long s_l,
                                                      typename cpx<T>::t* Y, long ldy, long s_y, int k0, int kb,
                                                      int ncols) {
  using C = typename cpx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* L = reinterpret_cast<C*>(smem_raw);
  C* X = L + kNB * (kNB + 1);
  Lm += blockIdx.z * s_l;
  Y += blockIdx.z * s_y;
  const int t = threadIdx.x;
  for (int e = t; e < kb * kb; e += blockDim.x) {
    const int i = e / kb, c = e % kb;
    L[i * (kNB + 1) + c] = c <= i ? Lm[(long)(k0 + i) * ldl + k0 + c] : mk(T(0), T(0));
  }
  const int col = blockIdx.x * 64 + t;
  const bool active = col < ncols;
  const int dc = col - k0;                   // column inside the diagonal block, or < 0
  if (active)
    for (int r = 0; r < kb; ++r)
      X[r * 64 + t] = dc >= 0 ? mk(T(r == dc ? 1 : 0), T(0)) : Y[(long)(k0 + r) * ldy + col];
  __syncthreads();
  if (!active) return;
  for (int r = 0; r < kb; ++r) {
    C s = X[r * 64 + t];
    for (int p = 0; p < r; ++p) s = csub(s, cmul(L[r * (kNB + 1) + p], X[p * 64 + t]));
    X[r * 64 + t] = cscale(s, T(1) / (T(1) + L[r * (kNB + 1) + r].x));
  }
  for (int r = 0; r < kb; ++r) {
    C y = X[r * 64 + t];
    if (r == dc) {                           // (1 + K)^{-1} - 1 = -K / (1 + K)
      const T k = L[r * (kNB + 1) + r].x;
      y = mk(-k / (T(1) + k), T(0));
    }
    Y[(long)(k0 + r) * ldy + col] = y;
  }
}

// Zero `cols` columns of `rows` rows (leading dimension ld) per batch entry.
template <typename T>
__global__ void zero_block_kernel(typename cpx<T>::t* __restrict__ P, long ld, long s_p, int cols) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= cols) return;
  P[blockIdx.z * s_p + (long)blockIdx.y * ld + b] = mk(T(0), T(0));
}

// X = P^H P + P + P^H (lower triangle, in place over P^H P); one CTA per row.
template <typename T>
__global__ void __launch_bounds__(256) assemble_kernel(typename cpx<T>::t* __restrict__ X, long s_x,
                                                       const typename cpx<T>::t* __restrict__ P, long s_p, int n) {
  const int a = blockIdx.x;
  auto* xr = X + blockIdx.y * s_x + (long)a * n;
  const auto* pr = P + blockIdx.y * s_p + (long)a * n;
  for (int b = threadIdx.x; b <= a; b += blockDim.x) {
    auto x = xr[b];
    const auto p = pr[b];
    x.x += a == b ? T(2) * p.x : p.x;
    x.y += a == b ? T(0) : p.y;
    xr[b] = x;
  }
}

// W~[a][b] = v_a X[a][b] v_b, both triangles from the lower one.  One 32 x 32
// tile pair (ta >= tb) per CTA through shared memory, so that the mirrored
// (conjugate-transposed) writes are row segments too.
template <typename T>
__global__ void __launch_bounds__(256) finalize_kernel(const typename cpx<T>::t* __restrict__ Xl, long s_x,
                                                       const double* __restrict__ vh, typename cpx<T>::t* __restrict__ W,
                                                       long s_w, int n) {
  using C = typename cpx<T>::t;
  const int ta = blockIdx.y, tb = blockIdx.x;
  if (tb > ta) return;
  __shared__ C t[32][33];
  Xl += blockIdx.z * s_x;
  W += blockIdx.z * s_w;
  const int a0 = ta * 32, b0 = tb * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int a = a0 + y, b = b0 + threadIdx.x;
    C v = mk(T(0), T(0));
    if (a < n && b < n) {
      // lower element, or the mirror of one inside a diagonal tile
      v = b <= a ? Xl[(long)a * n + b] : cconj(Xl[(long)b * n + a]);
      v = cscale(v, T(vh[a] * vh[b]));
      W[(long)a * n + b] = v;
    }
    t[y][threadIdx.x] = v;
  }
  if (ta == tb) return;
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int b = b0 + y, a = a0 + threadIdx.x;
    if (a < n && b < n) W[(long)b * n + a] = cconj(t[threadIdx.x][y]);
  }
}

// y = F z in FP64 for the Hermitian F given by its lower triangle Mlow:
// F[a][b] = s_a s_b (Mlow or conj of the mirrored entry) - sub * delta_ab.
template <typename T>
__global__ void __launch_bounds__(256) hemv_probe_kernel(const typename cpx<T>::t* __restrict__ Mlow,
                                                         const double* __restrict__ sv, double sub,
                                                         const double2* __restrict__ z, double2* __restrict__ y,
                                                         int n) {
  const int a = blockIdx.x;
  double re = 0, im = 0;
  for (int b = threadIdx.x; b < n; b += blockDim.x) {
    double2 m;
    if (b <= a) {
      auto v = Mlow[(long)a * n + b];
      m = make_double2(v.x, v.y);
    } else {
      auto v = Mlow[(long)b * n + a];
      m = make_double2(v.x, -v.y);
    }
    const double s = sv ? sv[a] * sv[b] : 1.0;
    m.x *= s;
    m.y *= s;
    if (a == b) m.x -= sub;
    re += m.x * z[b].x - m.y * z[b].y;
    im += m.x * z[b].y + m.y * z[b].x;
  }
  __shared__ double sr[256], si[256];
  sr[threadIdx.x] = re;
  si[threadIdx.x] = im;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sr[threadIdx.x] += sr[threadIdx.x + w];
      si[threadIdx.x] += si[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) y[a] = make_double2(sr[0], si[0]);
}

// A batch of B frequencies whose matrices are `ms` elements apart.
struct Batch {
  int B;
  long ms;
};

template <typename T>
static gw_status set_attrs(gw_ctx* ctx) {
  using C = typename cpx<T>::t;
  const size_t tsm = sizeof(C) * (kNB * (kNB + 1) + kNB * 64);
  const size_t psm = sizeof(C) * kNB * (kNB + 1);
  gw_status rc = GW_OK;
  if (tsm > 48 * 1024) {
    rc = cuda_check(ctx, cudaFuncSetAttribute(trsm_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm),
                    "cudaFuncSetAttribute");
    if (!rc)
      rc = cuda_check(ctx, cudaFuncSetAttribute(trsm_left_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm),
                      "cudaFuncSetAttribute");
  }
  if (!rc && psm > 48 * 1024)
    rc = cuda_check(ctx, cudaFuncSetAttribute(potrf_diag_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm),
                    "cudaFuncSetAttribute");
  return rc;
}

// Cholesky (lower, K form on the diagonal) of the n x n block at a (leading
// dimension lda) of every batch entry, on CUDA cores, 64-column panels.
template <typename T>
static gw_status chol_simt(gw_ctx* ctx, gw_prec prec, typename cpx<T>::t* a, long lda, int n, int col0, Batch bt,
                           cudaStream_t st) {
  using C = typename cpx<T>::t;
  gw_status rc;
  const size_t tsm = sizeof(C) * (kNB * (kNB + 1) + kNB * 64);
  const size_t psm = sizeof(C) * kNB * (kNB + 1);
  for (int k0 = 0; k0 < n; k0 += kNB) {
    const int kb = std::min(kNB, n - k0);
    potrf_diag_kernel<T><<<dim3(1, 1, bt.B), 256, psm, st>>>(a + (long)k0 * lda + k0, lda, bt.ms, kb, ctx->dflag,
                                                             col0 + k0);
    if ((rc = launch_check(ctx, "potrf_diag_kernel"))) return rc;
    const int rows = n - k0 - kb;
    if (rows <= 0) break;
    trsm_panel_kernel<T><<<dim3((rows + 63) / 64, 1, bt.B), 64, tsm, st>>>(a, lda, bt.ms, k0, kb, rows);
    if ((rc = launch_check(ctx, "trsm_panel_kernel"))) return rc;
    GemmArgs g{};
    g.M = rows;
    g.N = rows;
    g.K = kb;
    g.alpha_re = -1;
    g.beta = 1;
    g.A = a + (long)(k0 + kb) * lda + k0;
    g.lda = lda;
    g.a_km = 0;
    g.B = a + (long)(k0 + kb) * lda + k0;
    g.ldb = lda;
    g.b_nk = 1;
    g.b_conj = true;
    g.C = a + (long)(k0 + kb) * lda + k0 + kb;
    g.ldc = lda;
    g.tri = 1;
    g.batch = bt.B;
    g.sA = g.sB = g.sC = bt.ms;
    if ((rc = launch_gemm(ctx, prec, g, st))) return rc;
  }
  return GW_OK;
}

// P = L^{-1} - 1 for the n x n lower factor L (K form diagonal) at Lm, written
// to the n x n block at p, for every batch entry (CUDA cores).
template <typename T>
static gw_status inv_simt(gw_ctx* ctx, gw_prec prec, const typename cpx<T>::t* Lm, long ldl,
                          typename cpx<T>::t* p, long ldp, int n, Batch bt, cudaStream_t st) {
  using C = typename cpx<T>::t;
  gw_status rc;
  const size_t tsm = sizeof(C) * (kNB * (kNB + 1) + kNB * 64);
  zero_block_kernel<T><<<dim3((n + 127) / 128, n, bt.B), 128, 0, st>>>(p, ldp, bt.ms, n);
  if ((rc = launch_check(ctx, "zero_block_kernel"))) return rc;
  for (int k0 = 0; k0 < n; k0 += kNB) {
    const int kb = std::min(kNB, n - k0);
    const int ncols = k0 + kb;
    trsm_left_kernel<T><<<dim3((ncols + 63) / 64, 1, bt.B), 64, tsm, st>>>(Lm, ldl, bt.ms, p, ldp, bt.ms, k0, kb,
                                                                          ncols);
    if ((rc = launch_check(ctx, "trsm_left_kernel"))) return rc;
    const int rows = n - k0 - kb;
    if (rows <= 0) break;
    neg_copy_kernel<T><<<dim3(rows, 1, bt.B), kNB, 0, st>>>(Lm, ldl, bt.ms, p, ldp, bt.ms, k0 + kb, rows, k0, kb);
    if ((rc = launch_check(ctx, "neg_copy_kernel"))) return rc;
    GemmArgs g{};
    g.M = rows;
    g.N = ncols;
    g.K = kb;
    g.alpha_re = -1;
    g.beta = 1;
    g.A = Lm + (long)(k0 + kb) * ldl + k0;
    g.lda = ldl;
    g.B = p + (long)k0 * ldp;
    g.ldb = ldp;
    g.C = p + (long)(k0 + kb) * ldp;
    g.ldc = ldp;
    g.batch = bt.B;
    g.sA = g.sB = g.sC = bt.ms;
    if ((rc = launch_gemm(ctx, prec, g, st))) return rc;
  }
  return GW_OK;
}

// |eps~ X z - chi~ z| / |chi~ z| over 4 seeded probes z, in FP64, with X the
// assembled lower triangle of eps~^{-1} - 1 (one frequency) and chi intact.
template <typename T>
static gw_status residual_probe(gw_ctx* ctx, int n, const typename cpx<T>::t* chi, const double* dvh,
                                const typename cpx<T>::t* e, double2* probe, double* resid_h, cudaStream_t st) {
  gw_status rc;
  double num = 0, den = 0;
  std::vector<double2> hz(n), hu(n), hw(n), hc(n);
  for (int q = 0; q < 4; ++q) {
    uint64_t sd = 0x9E3779B97F4A7C15ull * (q + 1);
    for (int i = 0; i < n; ++i) {
      sd = sd * 6364136223846793005ull + 1442695040888963407ull;
      const double u1 = ((sd >> 11) & ((1ull << 53) - 1)) / 9007199254740992.0;
      sd = sd * 6364136223846793005ull + 1442695040888963407ull;
      const double u2 = ((sd >> 11) & ((1ull << 53) - 1)) / 9007199254740992.0;
      hz[i] = make_double2(u1 - 0.5, u2 - 0.5);
    }
    double2 *z = probe, *u = probe + n, *w = probe + 2 * n, *c = probe + 3 * n;
    if ((rc = upload(ctx, z, hz.data(), sizeof(double2) * n, st))) return rc;
    hemv_probe_kernel<T><<<n, 256, 0, st>>>(e, nullptr, 0.0, z, u, n);       // u = X z
    hemv_probe_kernel<T><<<n, 256, 0, st>>>(chi, dvh, 0.0, u, w, n);         // w = chi~ u
    hemv_probe_kernel<T><<<n, 256, 0, st>>>(chi, dvh, 0.0, z, c, n);         // c = chi~ z
    if ((rc = launch_check(ctx, "hemv_probe_kernel"))) return rc;
    ctx->launches += 2;
    cudaMemcpyAsync(hu.data(), u, sizeof(double2) * n, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(hw.data(), w, sizeof(double2) * n, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(hc.data(), c, sizeof(double2) * n, cudaMemcpyDeviceToHost, st);
    if ((rc = cuda_check(ctx, cudaStreamSynchronize(st), "probe sync"))) return rc;
    for (int i = 0; i < n; ++i) {
      const double rr = hu[i].x - hw[i].x - hc[i].x, ri = hu[i].y - hw[i].y - hc[i].y;
      num += rr * rr + ri * ri;
      den += hc[i].x * hc[i].x + hc[i].y * hc[i].y;
    }
  }
  *resid_h = den > 0 ? std::sqrt(num / den) : 0.0;
  return GW_OK;
}

// Refinement of X = eps~^{-1} - 1 in FP64 after the working-precision solve.
// With chi~ = v^1/2 chi v^1/2 and eps~ = 1 - chi~, X = eps~^{-1} chi~ solves
// eps~ X = chi~.  For an approximate X with error E, the residual
//   R = chi~ - eps~ X = chi~ - X + chi~ X
// and the update X <- X + (1 + X) R (the current 1 + X standing in for
// eps~^{-1}) leave the error -E eps~ E: Newton-Schulz, quadratic convergence,
// two N^3 FP64 GEMMs per step.
template <typename T>
__global__ void refine_expand_kernel(const typename cpx<T>::t* __restrict__ Xl, const typename cpx<T>::t* __restrict__ chi,
                                     const double* __restrict__ vh, double2* __restrict__ X, double2* __restrict__ Ct,
                                     int n) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int a = blockIdx.y;
  if (b >= n) return;
  const long e = (long)a * n + b;
  const auto x = b <= a ? Xl[e] : Xl[(long)b * n + a];
  X[e] = b <= a ? make_double2(x.x, x.y) : make_double2(x.x, -x.y);
  const auto c = chi[e];
  const double sc = vh[a] * vh[b];
  Ct[e] = make_double2(sc * c.x, sc * c.y);
}

__global__ void refine_resid_kernel(const double2* __restrict__ Ct, const double2* __restrict__ X, double2* R, long nn) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < nn; e += (long)gridDim.x * blockDim.x)
    R[e] = make_double2(Ct[e].x - X[e].x + R[e].x, Ct[e].y - X[e].y + R[e].y);
}

__global__ void refine_update_kernel(double2* X, const double2* __restrict__ R, const double2* __restrict__ XR, long nn) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < nn; e += (long)gridDim.x * blockDim.x)
    X[e] = make_double2(X[e].x + R[e].x + XR[e].x, X[e].y + R[e].y + XR[e].y);
}

// Lower triangle back in the working precision, Hermitian part of X.
template <typename T>
__global__ void refine_store_kernel(const double2* __restrict__ X, typename cpx<T>::t* __restrict__ Xl, int n) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int a = blockIdx.y;
  if (b > a || b >= n) return;
  const double2 u = X[(long)a * n + b], w = X[(long)b * n + a];
  Xl[(long)a * n + b] = mk(T(0.5 * (u.x + w.x)), T(0.5 * (u.y - w.y)));
}

template <typename T>
static gw_status refine_one(gw_ctx* ctx, int n, const typename cpx<T>::t* chi, const double* dvh,
                            typename cpx<T>::t* xl, double2* ws, int iters, cudaStream_t st) {
  const long nn = (long)n * n;
  double2* X = ws;
  double2* Ct = ws + nn;
  double2* R = ws + 2 * nn;
  double2* XR = ws + 3 * nn;
  const dim3 tb(128), gb((n + 127) / 128, n);
  const int eb = (int)std::min<long>((nn + 255) / 256, (long)ctx->num_sms * 8);
  gw_status rc;
  refine_expand_kernel<T><<<gb, tb, 0, st>>>(xl, chi, dvh, X, Ct, n);
  if ((rc = launch_check(ctx, "refine_expand_kernel"))) return rc;
  for (int it = 0; it < iters; ++it) {
    GemmArgs g{};
    g.M = g.N = g.K = n;
    g.alpha_re = 1.0;
    g.lda = g.ldb = g.ldc = n;
    g.A = Ct;                 // R = chi~ X
    g.B = X;
    g.C = R;
    if ((rc = launch_gemm(ctx, GW_FP64, g, st))) return rc;
    refine_resid_kernel<<<eb, 256, 0, st>>>(Ct, X, R, nn);
    if ((rc = launch_check(ctx, "refine_resid_kernel"))) return rc;
    g.A = X;                  // XR = X R
    g.B = R;
    g.C = XR;
    if ((rc = launch_gemm(ctx, GW_FP64, g, st))) return rc;
    refine_update_kernel<<<eb, 256, 0, st>>>(X, R, XR, nn);
    if ((rc = launch_check(ctx, "refine_update_kernel"))) return rc;
  }
  refine_store_kernel<T><<<gb, tb, 0, st>>>(X, xl, n);
  return launch_check(ctx, "refine_store_kernel");
}

// The same refinement for the tensor-core precisions, with the product chi~ X
// of the residual on the tensor cores as exact fp16 slice products (slice pairs
// up to kRefineLevels, i.e. 30 bits of the row and column maxima: the residual
// then bounds X to ~1e-9, below the FP32 storage of W~), and the correction
// X R as three fp16 split products (R is small: the correction needs only the
// working precision).  Work: X, chi~, R in FP64 and R, X R in FP32 (the last
// slot of ws); X in FP32 goes to the upper part of xl, which the final store
// overwrites with the lower triangle.
constexpr int kRefineLevels = 4;

__global__ void to_f32_kernel(const double2* __restrict__ X, float2* __restrict__ Y, long nn) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < nn; e += (long)gridDim.x * blockDim.x)
    Y[e] = make_float2((float)X[e].x, (float)X[e].y);
}

__global__ void refine_update_f32_kernel(double2* X, const double2* __restrict__ R, const float2* __restrict__ XR,
                                         long nn) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < nn; e += (long)gridDim.x * blockDim.x)
    X[e] = make_double2(X[e].x + R[e].x + (double)XR[e].x, X[e].y + R[e].y + (double)XR[e].y);
}

static gw_status refine_one_tc(gw_ctx* ctx, gw_prec prec, int n, const float2* chi, const double* dvh, float2* xl,
                               double2* ws, void* tcs, void* sls, int iters, cudaStream_t st) {
  const long nn = (long)n * n;
  double2* X = ws;
  double2* Ct = ws + nn;
  double2* R = ws + 2 * nn;
  float2* R32 = reinterpret_cast<float2*>(ws + 3 * nn);
  float2* XR32 = R32 + nn;
  const dim3 tb(128), gb((n + 127) / 128, n);
  const int eb = (int)std::min<long>((nn + 255) / 256, (long)ctx->num_sms * 8);
  int* tstat = ctx->dflag + 4;
  gw_status rc;
  refine_expand_kernel<float><<<gb, tb, 0, st>>>(xl, chi, dvh, X, Ct, n);
  if ((rc = launch_check(ctx, "refine_expand_kernel"))) return rc;
  for (int it = 0; it < iters; ++it) {
    // R = chi~ X (FP64-class), then R = chi~ - X + R
    if ((rc = tc_zgemm_sliced(ctx, n, n, n, Ct, n, X, n, R, n, kRefineLevels, tstat, sls, st))) return rc;
    refine_resid_kernel<<<eb, 256, 0, st>>>(Ct, X, R, nn);
    if ((rc = launch_check(ctx, "refine_resid_kernel"))) return rc;
    to_f32_kernel<<<eb, 256, 0, st>>>(X, xl, nn);
    to_f32_kernel<<<eb, 256, 0, st>>>(R, R32, nn);
    if ((rc = launch_check(ctx, "to_f32_kernel"))) return rc;
    ctx->launches++;
    TcGemm g;
    g.M = g.N = g.K = n;
    g.A = xl;
    g.lda = n;
    g.a_trans = g.a_conj = false;
    g.B = R32;
    g.ldb = n;
    g.b_trans = g.b_conj = false;
    g.C = XR32;
    g.ldc = n;
    g.alpha = 1.0f;
    g.accumulate = false;
    g.tri = 0;
    g.status = tstat;
    if ((rc = tc_gemm(ctx, prec, g, tcs, st))) return rc;
    refine_update_f32_kernel<<<eb, 256, 0, st>>>(X, R, XR32, nn);
    if ((rc = launch_check(ctx, "refine_update_f32_kernel"))) return rc;
  }
  refine_store_kernel<float><<<gb, tb, 0, st>>>(X, xl, n);
  return launch_check(ctx, "refine_store_kernel");
}

// One batch of frequencies: chi[B][n][n] -> W[B][n][n] (may alias chi), with
// work buffers E and P of the same shape.  tcs: tensor-core scratch (NULL for
// the CUDA-core precisions).
template <typename T>
static gw_status screen_batch(gw_ctx* ctx, gw_prec prec, int n, int B, const void* chi, const double* dvh, void* E,
                              void* Pm, void* W, double2* probe, double* resid_h, void* tcs, int refine,
                              double2* rws, void* sls, cudaStream_t st) {
  using C = typename cpx<T>::t;
  gw_status rc;
  C* e = static_cast<C*>(E);
  C* p = static_cast<C*>(Pm);
  const long nn = (long)n * n;
  const Batch bt{B, nn};
  if ((rc = set_attrs<T>(ctx))) return rc;
  build_eps_kernel<T><<<dim3(n, B), 256, 0, st>>>(static_cast<const C*>(chi), nn, dvh, e, nn, n);
  if ((rc = launch_check(ctx, "build_eps_kernel"))) return rc;
  if (!tcs) {
    // CUDA cores, 64-column panels over the whole matrix
    if ((rc = chol_simt<T>(ctx, prec, e, n, n, 0, bt, st))) return rc;
    if ((rc = inv_simt<T>(ctx, prec, e, n, p, n, n, bt, st))) return rc;
    GemmArgs g{};
    g.M = n;
    g.N = n;
    g.K = n;
    g.alpha_re = 1;
    g.beta = 0;
    g.A = p;
    g.lda = n;
    g.a_km = 1;
    g.a_conj = true;
    g.B = p;
    g.ldb = n;
    g.C = e;
    g.ldc = n;
    g.tri = 2;
    g.batch = B;
    g.sA = g.sB = g.sC = nn;
    if ((rc = launch_gemm(ctx, prec, g, st))) return rc;
  } else {
    if constexpr (std::is_same<T, float>::value) {
      int* tstat = ctx->dflag + 4;
      auto gemm = [&](int M, int N, int K, const C* A, bool at, bool ac, const C* Bm, bool btr, bool bc, C* Cm,
                      float alpha, bool acc, int tri, int batch) {
        TcGemm g;
        g.M = M;
        g.N = N;
        g.K = K;
        g.A = A;
        g.lda = n;
        g.a_trans = at;
        g.a_conj = ac;
        g.B = Bm;
        g.ldb = n;
        g.b_trans = btr;
        g.b_conj = bc;
        g.C = Cm;
        g.ldc = n;
        g.alpha = alpha;
        g.accumulate = acc;
        g.tri = tri;
        g.status = tstat;
        g.batch = batch;
        g.sA = g.sB = g.sC = nn;
        return tc_gemm(ctx, prec, g, tcs, st);
      };
      // 1. Cholesky and the inverted diagonal blocks P_kk
      for (int k0 = 0; k0 < n; k0 += kTB) {
        const int kb = std::min(kTB, n - k0);
        C* akk = e + (long)k0 * n + k0;
        C* pkk = p + (long)k0 * n + k0;
        if ((rc = chol_simt<float>(ctx, GW_FP32, akk, n, kb, k0, bt, st))) return rc;
        if ((rc = inv_simt<float>(ctx, GW_FP32, akk, n, pkk, n, kb, bt, st))) return rc;
        const int rows = n - k0 - kb;
        if (rows <= 0) break;
        C* a21 = e + (long)(k0 + kb) * n + k0;
        // L21 = A21 + A21 P_kk^H   (opB(k, j) = conj(P_kk[j][k]))
        if ((rc = gemm(rows, kb, kb, a21, false, false, pkk, true, true, a21, 1.0f, true, 0, B))) return rc;
        // A22 -= L21 L21^H
        if ((rc = gemm(rows, rows, kb, a21, false, false, a21, true, true, a21 + kb, -1.0f, true, 1, B))) return rc;
      }
      // 2. off-diagonal blocks of P = L^{-1} - 1, block row by block row, and
      //    the zero upper part
      for (int k0 = 0; k0 < n; k0 += kTB) {
        const int kb = std::min(kTB, n - k0);
        C* pi = p + (long)k0 * n;
        C* pkk = pi + k0;
        if (k0 > 0 && (rc = gemm(kb, k0, kb, pkk, false, false, pi, false, false, pi, 1.0f, true, 0, B))) return rc;
        const int rows = n - k0 - kb;
        if (rows <= 0) break;
        zero_block_kernel<float><<<dim3((rows + 127) / 128, kb, B), 128, 0, st>>>(pi + k0 + kb, n, nn, rows);
        if ((rc = launch_check(ctx, "zero_block_kernel"))) return rc;
        neg_copy_kernel<float><<<dim3(rows, 1, B), 256, 0, st>>>(e, n, nn, p, n, nn, k0 + kb, rows, k0, kb);
        if ((rc = launch_check(ctx, "neg_copy_kernel"))) return rc;
        if ((rc = gemm(rows, k0 + kb, kb, e + (long)(k0 + kb) * n + k0, false, false, pi, false, false,
                       p + (long)(k0 + kb) * n, -1.0f, true, 0, B)))
          return rc;
      }
      // 3. P^H P (lower) in K blocks of kTB rows of P.  P is lower triangular,
      //    so block [k1, k2) touches only the leading k2 x k2 part; going from
      //    the last block (which writes the whole lower triangle) to the first,
      //    each block is added to C by the epilogue in round-to-nearest FP32.
      //    One accumulation over all N rows would take ~3N/8 truncating
      //    tensor-core adds per element (5000 at N = 13824) and lose ~1e-4.
      for (int k1 = (n - 1) / kTB * kTB; k1 >= 0; k1 -= kTB) {
        const int k2 = std::min(n, k1 + kTB);
        if ((rc = gemm(k2, k2, k2 - k1, p + (long)k1 * n, true, true, p + (long)k1 * n, false, false, e, 1.0f,
                       k2 < n, 1, B)))
          return rc;
      }
    }
  }
  assemble_kernel<T><<<dim3(n, B), 256, 0, st>>>(e, nn, p, nn, n);
  if ((rc = launch_check(ctx, "assemble_kernel"))) return rc;
  if (refine > 0)
    for (int b = 0; b < B; ++b) {
      if constexpr (std::is_same<T, float>::value) {
        if (tcs) {
          if ((rc = refine_one_tc(ctx, prec, n, static_cast<const C*>(chi) + b * nn, dvh, e + b * nn, rws, tcs, sls,
                                  refine, st)))
            return rc;
          continue;
        }
      }
      if ((rc = refine_one<T>(ctx, n, static_cast<const C*>(chi) + b * nn, dvh, e + b * nn, rws, refine, st)))
        return rc;
    }
  if (resid_h)
    for (int b = 0; b < B; ++b)
      if ((rc = residual_probe<T>(ctx, n, static_cast<const C*>(chi) + b * nn, dvh, e + b * nn, probe, resid_h + b,
                                  st)))
        return rc;
  const int nt = (n + 31) / 32;
  finalize_kernel<T><<<dim3(nt, nt, B), dim3(32, 8), 0, st>>>(e, nn, dvh, static_cast<C*>(W), nn, n);
  return launch_check(ctx, "finalize_kernel");
}

// Tensor-core GEMM scratch of the screening: panels of kTB over a batch, and
// with refinement the full n x n x n correction product.
static size_t screen_tc_scratch(int n_chi, int bsz, bool refine) {
  const size_t a = tc_gemm_scratch(n_chi, n_chi, kTB, bsz);
  return refine ? std::max(a, tc_gemm_scratch(n_chi, n_chi, n_chi, 1)) : a;
}

// Frequencies per batch (the two work matrices of a batch within 64 GB) and
// the scratch gw_screen_W needs.
size_t screen_scratch(int n_chi, int n_omega, gw_prec prec, int* bsz_out, int* nbatch_out, bool refine) {
  const size_t es = csize(prec);
  const size_t nn = (size_t)n_chi * n_chi;
  const bool tc = prec == GW_F16X3 || prec == GW_BF16X3;
  const size_t budget = size_t(64) << 30;
  const int no = std::max(n_omega, 1);
  const int bmax = (int)std::max<size_t>(1, std::min<size_t>(no, budget / (2 * nn * es)));
  const int nbatch = (no + bmax - 1) / bmax;
  const int bsz = (no + nbatch - 1) / nbatch;
  Carver probe(nullptr);
  probe.take<double>(n_chi);
  probe.take<char>(bsz * nn * es);
  probe.take<char>(bsz * nn * es);
  probe.take<double2>(4 * (size_t)n_chi);
  if (tc) probe.take<char>(screen_tc_scratch(n_chi, bsz, refine));
  if (refine) probe.take<double2>(4 * nn);
  if (refine && tc) probe.take<char>(tc_zgemm_sliced_scratch(n_chi, n_chi, n_chi, kRefineLevels));
  if (bsz_out) *bsz_out = bsz;
  if (nbatch_out) *nbatch_out = nbatch;
  return probe.off;
}

// The screening of n_omega frequencies with v^1/2 already on the device (dvh)
// and the arena carved by cv after it: device-side memsets and kernels only
// when resid_h and first_bad are NULL (then a plan can capture it in a CUDA
// graph).  Pivot and time-out flags are left in ctx->dflag (zeroed here first).
// resid_h: the FP64 probe residuals (synchronous); first_bad: with several
// batches of frequencies, the first frequency whose factorisation failed
// (synchronises between batches).
gw_status screen_launch(gw_ctx* ctx, int n_chi, int n_omega, gw_prec prec, int refine_iters, const double* dvh,
                        const void* chi_w, void* w_w, Carver& cv, double* resid_h, int* first_bad, cudaStream_t s) {
  gw_status st;
  const size_t es = csize(prec);
  const size_t nn = (size_t)n_chi * n_chi;
  const bool tc = prec == GW_F16X3 || prec == GW_BF16X3;
  int bsz = 0, nbatch = 0;
  screen_scratch(n_chi, n_omega, prec, &bsz, &nbatch, refine_iters > 0);
  const size_t tcs_bytes = tc ? screen_tc_scratch(n_chi, bsz, refine_iters > 0) : 0;
  void* E = cv.take<char>(bsz * nn * es);
  void* M = cv.take<char>(bsz * nn * es);
  double2* pr = cv.take<double2>(4 * (size_t)n_chi);
  void* tcs = tc ? cv.take<char>(tcs_bytes) : nullptr;
  double2* rws = refine_iters > 0 ? cv.take<double2>(4 * nn) : nullptr;
  void* sls = refine_iters > 0 && tc ? cv.take<char>(tc_zgemm_sliced_scratch(n_chi, n_chi, n_chi, kRefineLevels))
                                     : nullptr;
  if ((st = cuda_check(ctx, cudaMemsetAsync(ctx->dflag, 0, 8 * sizeof(int), s), "memset flag"))) return st;
  for (int k0 = 0; k0 < n_omega; k0 += bsz) {
    const int B = std::min(bsz, n_omega - k0);
    const char* in = static_cast<const char*>(chi_w) + k0 * nn * es;
    char* out = static_cast<char*>(w_w) + k0 * nn * es;
    double* rk = resid_h ? resid_h + k0 : nullptr;
    if (is_fp64(prec))
      st = screen_batch<double>(ctx, prec, n_chi, B, in, dvh, E, M, out, pr, rk, nullptr, refine_iters, rws, nullptr, s);
    else st = screen_batch<float>(ctx, prec, n_chi, B, in, dvh, E, M, out, pr, rk, tcs, refine_iters, rws, sls, s);
    if (st) return st;
    if (first_bad && nbatch > 1 && *first_bad < 0) {
      int f[3] = {0, 0, 0};
      cudaMemcpyAsync(f, ctx->dflag, sizeof(f), cudaMemcpyDeviceToHost, s);
      if ((st = cuda_check(ctx, cudaStreamSynchronize(s), "sync"))) return st;
      if (f[0]) *first_bad = k0 + f[2];
    }
  }
  return GW_OK;
}

}  // namespace gw

using namespace gw;

extern "C" gw_status gw_workspace_size(const gw_grid* grid, int n_b, int n_occ, int n, int n_chi, int n_n,
                                       gw_prec prec, int r_block, size_t* chi0_bytes, size_t* screen_bytes,
                                       size_t* sigma_bytes) {
  GridInfo g;
  gw_status st = grid_info(nullptr, grid, &g);
  if (st) return st;
  if (!valid_prec(prec)) return fail(nullptr, GW_ERR_ARG, "bad precision");
  if (n_b < 2 || n_occ < 1 || n_occ >= n_b || n < 1 || n_chi < 1 || n_chi > g.nr || n_n < 1)
    return fail(nullptr, GW_ERR_SHAPE, "bad sizes");
  const int rb = r_block > 0 ? std::min(r_block, g.nr) : std::min(g.nr, 2048);
  if (chi0_bytes) *chi0_bytes = chi0_omega_scratch(g, n_b, n_occ, n, n_chi, prec, rb);
  if (screen_bytes) *screen_bytes = screen_scratch(n_chi, n, prec, nullptr, nullptr);
  if (sigma_bytes) *sigma_bytes = sigma_scratch(g, n_b, n_occ, n, n_chi, n_n, 64, prec);
  return GW_OK;
}

extern "C" gw_status gw_screen_W(gw_ctx* ctx, const gw_grid* grid, int n_chi, const int32_t* gvec_h, int n_omega,
                                 gw_prec prec, const void* chi_w, void* w_w, double* resid_h, void* stream) {
  return gw_screen_W_refine(ctx, grid, n_chi, gvec_h, n_omega, prec, 0, chi_w, w_w, resid_h, stream);
}

extern "C" gw_status gw_screen_W_refine(gw_ctx* ctx, const gw_grid* grid, int n_chi, const int32_t* gvec_h,
                                        int n_omega, gw_prec prec, int refine_iters, const void* chi_w, void* w_w,
                                        double* resid_h, void* stream) {
  if (!ctx) return fail(nullptr, GW_ERR_ARG, "ctx is NULL");
  GridInfo g;
  gw_status st = grid_info(ctx, grid, &g);
  if (st) return st;
  if (!valid_prec(prec)) return fail(ctx, GW_ERR_ARG, "bad precision");
  if (n_chi < 1 || n_chi > g.nr || n_chi > 65535) return fail(ctx, GW_ERR_SHAPE, "need 1 <= n_chi <= min(N_r, 65535)");
  if (n_omega < 0) return fail(ctx, GW_ERR_SHAPE, "n_omega < 0");
  if (n_omega == 0) return GW_OK;
  if (!gvec_h || !chi_w || !w_w) return fail(ctx, GW_ERR_ARG, "NULL pointer");
  if (refine_iters < 0 || refine_iters > 8) return fail(ctx, GW_ERR_ARG, "need 0 <= refine_iters <= 8");
  cudaStream_t s = as_stream(stream);
  std::vector<double> vh(n_chi);
  if ((st = gw_coulomb_sqrt(grid, gvec_h, n_chi, vh.data()))) return fail(ctx, st, gw_last_error(nullptr));
  if ((st = reserve(ctx, screen_scratch(n_chi, n_omega, prec, nullptr, nullptr, refine_iters > 0)))) return st;
  Carver cv(ctx->arena);
  double* dvh = cv.take<double>(n_chi);
  if ((st = upload(ctx, dvh, vh.data(), sizeof(double) * n_chi, s))) return st;
  int first_bad = -1;
  if ((st = screen_launch(ctx, n_chi, n_omega, prec, refine_iters, dvh, chi_w, w_w, cv, resid_h, &first_bad, s)))
    return st;
  int flag[8] = {0};
  if ((st = cuda_check(ctx, cudaMemcpyAsync(flag, ctx->dflag, sizeof(flag), cudaMemcpyDeviceToHost, s), "flag")))
    return st;
  if ((st = cuda_check(ctx, cudaStreamSynchronize(s), "sync"))) return st;
  if (flag[4]) return fail(ctx, GW_ERR_TIMEOUT, "tensor-core GEMM wait timed out (role " + std::to_string(flag[5]) + ")");
  if (flag[0])
    return fail(ctx, GW_ERR_NUMERIC, "eps~ not positive definite at column " + std::to_string(flag[1]) +
                                         " of frequency " + std::to_string(first_bad >= 0 ? first_bad : flag[2]));
  return GW_OK;
}
