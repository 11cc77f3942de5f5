// The chi0 chain of Fig. 1 steps (1)-(3) in one call (Sec. II.C steps (i)-(ii)).
//
// for tau_j:
//   for each block of r rows:  G_occ, G_unocc rows -> chi(r,R') = -2 G_occ o
//       conj(G_unocc) -> FFT over R' -> rows of the chi(r,G',tau_j) slab.
//       chi(r,R') only ever exists for one r-block (Eq. FFTX1 and the text
//       after it: the second transform waits until every r is done).
//   (i2,i3) column planes of the slab (first part of Eq. FFTX2).
// i1 column pass of every slab fused with the cosine transform (Eqs. FFTX2,
// CTX): chi0(G,G',i omega_k) = sum_j (dV^2/Omega) C_kj FFT_i1(slab_j).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "gw_kernels.h"
#include "gw_tc.h"

namespace gw {

size_t chi0_omega_scratch(const GridInfo& g, int n_b, int n_occ, int n, int n_chi, gw_prec prec, int rb) {
  const size_t es = csize(prec);
  const size_t slab = (size_t)g.nr * n_chi;
  Carver probe(nullptr);
  probe.take<int>(n_chi);
  probe.take<int>(g.nr);
  probe.take<double>((size_t)n * n_b);
  probe.take<double>((size_t)n * n);
  probe.take<char>(slab * n * es);
  probe.take<char>((size_t)rb * g.nr * es);
  probe.take<char>((size_t)rb * g.nr * es);
  if (prec == GW_F16X3 || prec == GW_BF16X3) probe.take<char>(tc_scratch_bytes(g, n_b, n_occ, rb, false));
  return probe.off;
}

// chi(G,G') = X(G,G') + conj(X(G',G)) in place, for every frequency.  The
// tensor-core chi pass forms only the lower triangle T of chi(r,R') (R' <= r)
// with its diagonal halved; chi(r,R') is Hermitian, so chi = T + T^H, and the
// transforms of Eqs. FFTX1, FFTX2 and the cosine transform (Eq. CTX, real
// weights) carry that over: chi(G,G',i omega) = X + X^H with X the result for T.
// One CTA per pair of 32 x 32 tiles (I, J), I <= J, through shared memory.
__global__ void __launch_bounds__(256) hermitize_kernel(float2* __restrict__ X, long sx, int n) {
  __shared__ float2 a[32][33], b[32][33];
  const int I = blockIdx.x, J = blockIdx.y;
  if (I > J) return;
  float2* x = X + blockIdx.z * sx;
  const int tx = threadIdx.x;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int r = I * 32 + y, c = J * 32 + tx;
    a[y][tx] = (r < n && c < n) ? x[(long)r * n + c] : make_float2(0.f, 0.f);
    const int r2 = J * 32 + y, c2 = I * 32 + tx;
    b[y][tx] = (r2 < n && c2 < n) ? x[(long)r2 * n + c2] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int r = I * 32 + y, c = J * 32 + tx;
    if (r < n && c < n) x[(long)r * n + c] = make_float2(a[y][tx].x + b[tx][y].x, a[y][tx].y - b[tx][y].y);
    const int r2 = J * 32 + y, c2 = I * 32 + tx;
    if (I != J && r2 < n && c2 < n) x[(long)r2 * n + c2] = make_float2(b[y][tx].x + a[tx][y].x, b[y][tx].y - a[tx][y].y);
  }
}

// Device tables of one chi0 evaluation.
struct Chi0Dev {
  const int* map = nullptr;      // [n_chi] FFT positions of the G set
  const int* inv = nullptr;      // [N_r] position -> G index or -1
  const char* scale = nullptr;   // CUDA-core path: [n][n_b] per-band factors in 8-byte slots
  const float* sk = nullptr;     // tensor path: [n][n_b] FP32 factors, or NULL to copy them per call
  const void* cw = nullptr;      // transform weights, dV^2/Omega folded in (FP32 hi/lo or FP64)
  int* status = nullptr;         // tensor path: time-out status words owned by the caller, or NULL (in the scratch)
};

static gw_status chi0_check(gw_ctx* ctx, const gw_grid* grid, GridInfo* g, int n_b, int n_occ, const double* eps_h,
                            double mu, int n, const double* tau_h, const double* C_h, gw_prec prec) {
  gw_status st = grid_info(ctx, grid, g);
  if (st) return st;
  if (!grid_supported(g->n1, g->n2, g->n3)) return fail(ctx, GW_ERR_UNSUPPORTED, "no kernels compiled for this grid");
  if (!valid_prec(prec)) return fail(ctx, GW_ERR_ARG, "bad precision");
  if (!tau_h || !C_h) return fail(ctx, GW_ERR_ARG, "NULL pointer");
  if (n_b < 2 || n_b > g->nr) return fail(ctx, GW_ERR_SHAPE, "need 2 <= n_b <= N_r");
  if ((st = check_energies(ctx, eps_h, n_b, n_occ, mu))) return st;
  if (n < 1 || n > 32) return fail(ctx, GW_ERR_SHAPE, "need 1 <= n <= 32");
  for (int j = 0; j < n; ++j)
    if (!(tau_h[j] > 0)) return fail(ctx, GW_ERR_ARG, "tau must be > 0");
  return GW_OK;
}

// Host-side tables: per-tau band factors, FP32 weights.
static void chi0_tables(const GridInfo& g, int n_b, int n_occ, const double* eps_h, double mu, int n,
                        const double* tau_h, const double* C_h, gw_prec prec, std::vector<GreenScales>& scales,
                        std::vector<double>& cw64, std::vector<float>& cw32) {
  scales.resize(n);
  for (int j = 0; j < n; ++j) scales[j] = green_scales(eps_h, n_b, n_occ, mu, tau_h[j]);
  const double fac = g.dv * g.dv / g.volume;   // Eq. FFTX2 normalisation
  if (is_fp64(prec)) {
    cw64.assign(C_h, C_h + n * n);
    for (auto& v : cw64) v *= fac;
  } else {
    cw32 = split_weights(C_h, n * n, fac);
  }
}

// The kernels of the chain, launched on s with no host-device copy when t.sk
// (tensor path) is given; scratch carved from cv.  *tcs_out: the tensor-core
// status region for tc_check.
static gw_status chi0_launch(gw_ctx* ctx, const GridInfo& g, int n_b, int n_occ, const void* psi, int n,
                             const std::vector<GreenScales>& scales, int n_chi, gw_prec prec, int rb,
                             const Chi0Dev& t, const std::vector<float>& cw32, Carver& cv, void* chi_w,
                             cudaStream_t s, void** tcs_out) {
  gw_status st;
  const size_t es = csize(prec);
  const bool tc = prec == GW_F16X3 || prec == GW_BF16X3;
  const size_t slab = (size_t)g.nr * n_chi;
  char* slabs = cv.take<char>(slab * n * es);
  char* ga = cv.take<char>((size_t)rb * g.nr * es);
  char* gb = cv.take<char>((size_t)rb * g.nr * es);
  void* tcs = tc ? cv.take<char>(tc_scratch_bytes(g, n_b, n_occ, rb, false)) : nullptr;
  if (tcs_out) *tcs_out = tcs;
  bool first = true;
  for (int j = 0; j < n; ++j) {
    const GreenScales& gs = scales[j];
    const char* sj = t.scale + (size_t)j * n_b * 8;
    char* slab_j = slabs + (size_t)j * slab * es;
    for (int r0 = 0; r0 < g.nr; r0 += rb) {
      const int rows = std::min(rb, g.nr - r0);
      if (tc) {
        if ((st = tc_chi_rows(ctx, g, n_b, n_occ, psi, gs, r0, rows, prec, ga, tcs, first, s,
                              t.sk ? t.sk + (size_t)j * n_b : nullptr, t.status, true)))
          return st;
        first = false;
        st = launch_row_fft(ctx, g, prec, 1, ga, nullptr, g.nr, slab_j + (size_t)r0 * n_chi * es, n_chi, t.map, n_chi,
                            rows, 1.0, s, t.inv, gb);
      } else {
        if ((st = green_rows(ctx, g, n_b, n_occ, psi, sj, gs, r0, rows, prec, ga, gb, s))) return st;
        st = launch_row_fft(ctx, g, prec, 0, ga, gb, g.nr, slab_j + (size_t)r0 * n_chi * es, n_chi, t.map, n_chi,
                            rows, -2.0, s, t.inv, ga);
      }
      if (st) return st;
    }
    if ((st = launch_col_plane(ctx, g, prec, -1, slab_j, n_chi, n_chi, 1.0, s))) return st;
  }
  if ((st = launch_col_line_ct(ctx, g, prec, slabs, (long)slab, n_chi, n, t.cw, n, chi_w, (long)n_chi * n_chi, n_chi,
                               t.inv, n_chi, s, cw32.empty() ? nullptr : cw32.data())))
    return st;
  if (!tc) return GW_OK;
  const int nt = (n_chi + 31) / 32;
  hermitize_kernel<<<dim3(nt, nt, n), dim3(32, 8), 0, s>>>(static_cast<float2*>(chi_w), (long)n_chi * n_chi, n_chi);
  return launch_check(ctx, "hermitize_kernel");
}

}  // namespace gw

using namespace gw;

extern "C" gw_status gw_chi0_omega(gw_ctx* ctx, const gw_grid* grid, int n_b, int n_occ, const void* psi,
                                   const double* eps_h, double mu, int n, const double* tau_h, const double* C_h,
                                   int n_chi, const int32_t* fft_index_h, gw_prec prec, int r_block, void* chi_w,
                                   void* stream) {
  if (!ctx) return fail(nullptr, GW_ERR_ARG, "ctx is NULL");
  GridInfo g;
  gw_status st = chi0_check(ctx, grid, &g, n_b, n_occ, eps_h, mu, n, tau_h, C_h, prec);
  if (st) return st;
  if (!psi || !chi_w) return fail(ctx, GW_ERR_ARG, "NULL pointer");
  std::vector<int> map, inv;
  if ((st = index_maps(ctx, g, fft_index_h, n_chi, map, inv))) return st;
  cudaStream_t s = as_stream(stream);
  const int rb = r_block > 0 ? std::min(r_block, g.nr) : std::min(g.nr, 2048);
  const bool tc = prec == GW_F16X3 || prec == GW_BF16X3;
  if ((st = reserve(ctx, chi0_omega_scratch(g, n_b, n_occ, n, n_chi, prec, rb)))) return st;
  std::vector<GreenScales> scales;
  std::vector<double> cw64;
  std::vector<float> cw32;
  chi0_tables(g, n_b, n_occ, eps_h, mu, n, tau_h, C_h, prec, scales, cw64, cw32);
  Carver cv(ctx->arena);
  int* dmap = cv.take<int>(n_chi);
  int* dinv = cv.take<int>(g.nr);
  char* dscale = cv.take<char>((size_t)n * n_b * 8);
  char* dcw = cv.take<char>((size_t)n * n * 8);
  if ((st = upload(ctx, dmap, map.data(), sizeof(int) * n_chi, s))) return st;
  if ((st = upload(ctx, dinv, inv.data(), sizeof(int) * g.nr, s))) return st;
  if (is_fp64(prec)) st = upload(ctx, dcw, cw64.data(), sizeof(double) * n * n, s);
  else st = upload(ctx, dcw, cw32.data(), sizeof(float) * 2 * n * n, s);
  if (st) return st;
  if (!tc)
    for (int j = 0; j < n; ++j)
      if ((st = upload_scales(ctx, dscale + (size_t)j * n_b * 8, scales[j], prec, s))) return st;
  Chi0Dev t;
  t.map = dmap;
  t.inv = dinv;
  t.scale = dscale;
  t.cw = dcw;
  void* tcs = nullptr;
  if ((st = chi0_launch(ctx, g, n_b, n_occ, psi, n, scales, n_chi, prec, rb, t, cw32, cv, chi_w, s, &tcs))) return st;
  return tc ? tc_check(ctx, tcs, s) : GW_OK;
}

namespace gw {

// ------------------------------------------------------------------ plane-wave form of G
//
// The paper keeps G in a plane-wave representation and transforms it to real
// space when needed (Sec. II.B; at one k point Eqs. FFT_G1, FFT_G2).  With the
// orbitals in the span of n_pw plane waves e^{+i g.r} (pw_index), their
// coefficients D_a(g) = sum_r psi_a(r) e^{+i g.r}, nonzero on the negated set,
// give
//   G(r,R') = (1/N_r^2) sum_{g,g'} e^{-i g.r} [sum_a f_a D_a(g) conj(D_a(g'))] e^{+i g'.R'},
// so with Dc = conj(D)/N_r and Mc = Dc F Dc^H (a G formation over n_pw points)
//   conj(G(r,R')) = sum_{g,g'} e^{+i g.r} Mc(g,g') e^{-i g'.R'}:
// a column transform T(r,g') = sum_g e^{+i g.r} Mc(g,g') over the grid, then per
// row a backward transform over g', and Eq. chi_rr becomes
//   chi(r,R') = -2 G_occ conj(G_unocc) = -2 conj(G'_occ) G'_unocc     (G' = conj G).
// The contraction shrinks from N_r^2 N_b to n_pw^2 N_b per tau and occupation;
// the row kernel expands both rows, multiplies and transforms onto chi's G set.

template <typename C, typename R>
__global__ void conj_scale_kernel(C* __restrict__ x, size_t n, R s) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    x[e] = mk(x[e].x * s, -x[e].y * s);
}

// out[2b] = sum_r |psi_b(r)|^2, out[2b+1] = sum_g |D_b(g)|^2 (FP64), one CTA per band.
template <typename C>
__global__ void __launch_bounds__(256) band_norms_kernel(const C* __restrict__ psi, long nr, const C* __restrict__ d,
                                                         long npw, double* __restrict__ out) {
  __shared__ double red[2][8];
  const long b = blockIdx.x;
  double s0 = 0, s1 = 0;
  for (long i = threadIdx.x; i < nr; i += blockDim.x) {
    const C v = psi[b * nr + i];
    s0 += (double)v.x * v.x + (double)v.y * v.y;
  }
  for (long i = threadIdx.x; i < npw; i += blockDim.x) {
    const C v = d[b * npw + i];
    s1 += (double)v.x * v.x + (double)v.y * v.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s0;
    red[1][threadIdx.x >> 5] = s1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, c = 0;
    for (int w = 0; w < 8; ++w) {
      a += red[0][w];
      c += red[1][w];
    }
    out[2 * b] = a;
    out[2 * b + 1] = c;
  }
}

GridInfo pw_grid(const GridInfo& g, int n_pw) {
  GridInfo q = g;                 // the G formation over the plane-wave set: n_pw "points"
  q.nr = n_pw;
  return q;
}

void pw_negate(const GridInfo& g, std::vector<int>& map, std::vector<int>& inv) {
  // psi = sum_g c(g) e^{+i g.r}: D(g') = sum_r psi e^{+i g'.r} is nonzero at g' = -g
  for (auto& q : map) {
    const int i1 = q / (g.n2 * g.n3), i2 = (q / g.n3) % g.n2, i3 = q % g.n3;
    q = (((g.n1 - i1) % g.n1) * g.n2 + (g.n2 - i2) % g.n2) * g.n3 + (g.n3 - i3) % g.n3;
  }
  std::fill(inv.begin(), inv.end(), -1);
  for (size_t j = 0; j < map.size(); ++j) inv[map[j]] = (int)j;
}

gw_status pw_coefficients(gw_ctx* ctx, const GridInfo& g, gw_prec prec, const void* psi, int n_b, int n_pw,
                          const int* dmap_neg, const int* dinv_neg, void* dc, double* dnorm, void* tmp,
                          cudaStream_t s) {
  gw_status st;
  if ((st = launch_row_fft(ctx, g, prec, 1, psi, nullptr, g.nr, dc, n_pw, dmap_neg, n_pw, n_b, 1.0, s, dinv_neg, tmp)))
    return st;
  if (is_fp64(prec))
    band_norms_kernel<double2><<<n_b, 256, 0, s>>>((const double2*)psi, g.nr, (const double2*)dc, n_pw, dnorm);
  else
    band_norms_kernel<float2><<<n_b, 256, 0, s>>>((const float2*)psi, g.nr, (const float2*)dc, n_pw, dnorm);
  if ((st = launch_check(ctx, "band_norms_kernel"))) return st;
  std::vector<double> nh(2 * (size_t)n_b);
  if ((st = cuda_check(ctx, cudaMemcpyAsync(nh.data(), dnorm, sizeof(double) * 2 * n_b, cudaMemcpyDeviceToHost, s),
                       "norms")))
    return st;
  if ((st = cuda_check(ctx, cudaStreamSynchronize(s), "sync"))) return st;
  // Parseval: sum_g |D(g)|^2 = N_r sum_r |psi(r)|^2 when psi lies in the set's span
  const double tol = is_fp64(prec) ? 1e-10 : 1e-5;
  for (int b = 0; b < n_b; ++b) {
    const double full = nh[2 * b] * g.nr, part = nh[2 * b + 1];
    if (!(std::fabs(full - part) <= tol * full))
      return fail(ctx, GW_ERR_ARG, "band " + std::to_string(b) + " is not in the span of the plane waves of pw_index "
                                   "(fraction " + std::to_string(full > 0 ? part / full : 0.0) + ")");
  }
  const size_t nel = (size_t)n_b * n_pw;
  const int blocks = (int)std::min<size_t>((nel + 255) / 256, (size_t)ctx->num_sms * 8);
  if (is_fp64(prec)) conj_scale_kernel<<<blocks, 256, 0, s>>>((double2*)dc, nel, 1.0 / g.nr);
  else conj_scale_kernel<<<blocks, 256, 0, s>>>((float2*)dc, nel, (float)(1.0 / g.nr));
  return launch_check(ctx, "conj_scale_kernel");
}

size_t chi0_pw_scratch(const GridInfo& g, int n_b, int n_occ, int n, int n_chi, int n_pw, gw_prec prec) {
  const size_t es = csize(prec);
  const bool tc = prec == GW_F16X3 || prec == GW_BF16X3;
  Carver probe(nullptr);
  probe.take<int>(n_chi);
  probe.take<int>(g.nr);
  probe.take<int>(n_pw);
  probe.take<int>(g.nr);
  probe.take<double>((size_t)n * n_b);
  probe.take<double>((size_t)n * n);
  probe.take<double>(2 * (size_t)n_b);
  probe.take<char>((size_t)g.nr * n_chi * n * es);       // slabs
  probe.take<char>((size_t)n_b * n_pw * es);             // Dc
  probe.take<char>((size_t)n_pw * n_pw * es);            // Mc occ
  probe.take<char>((size_t)n_pw * n_pw * es);            // Mc unocc
  probe.take<char>((size_t)g.nr * n_pw * es);            // T occ
  probe.take<char>((size_t)g.nr * n_pw * es);            // T unocc
  if (row_two_pass(g, prec) && is_fp64(prec)) probe.take<char>((size_t)n_b * g.nr * es);
  if (tc) probe.take<char>(tc_scratch_bytes(pw_grid(g, n_pw), n_b, n_occ, n_pw, false));
  return probe.off;
}

}  // namespace gw

using namespace gw;

extern "C" gw_status gw_chi0_omega_pw(gw_ctx* ctx, const gw_grid* grid, int n_b, int n_occ, const void* psi,
                                      const double* eps_h, double mu, int n, const double* tau_h, const double* C_h,
                                      int n_chi, const int32_t* fft_index_h, int n_pw, const int32_t* pw_index_h,
                                      gw_prec prec, void* chi_w, void* stream) {
  if (!ctx) return fail(nullptr, GW_ERR_ARG, "ctx is NULL");
  GridInfo g;
  gw_status st = chi0_check(ctx, grid, &g, n_b, n_occ, eps_h, mu, n, tau_h, C_h, prec);
  if (st) return st;
  if (!psi || !chi_w) return fail(ctx, GW_ERR_ARG, "NULL pointer");
  std::vector<int> map, inv, map_pw, inv_pw;
  if ((st = index_maps(ctx, g, fft_index_h, n_chi, map, inv))) return st;
  if ((st = index_maps(ctx, g, pw_index_h, n_pw, map_pw, inv_pw))) return st;
  pw_negate(g, map_pw, inv_pw);
  if ((st = check_row_pw(ctx, g, prec, n_pw, n_chi))) return st;
  cudaStream_t s = as_stream(stream);
  const bool tc = prec == GW_F16X3 || prec == GW_BF16X3;
  const size_t es = csize(prec);
  if ((st = reserve(ctx, chi0_pw_scratch(g, n_b, n_occ, n, n_chi, n_pw, prec)))) return st;
  std::vector<GreenScales> scales;
  std::vector<double> cw64;
  std::vector<float> cw32;
  chi0_tables(g, n_b, n_occ, eps_h, mu, n, tau_h, C_h, prec, scales, cw64, cw32);
  Carver cv(ctx->arena);
  int* dmap = cv.take<int>(n_chi);
  int* dinv = cv.take<int>(g.nr);
  int* dmap_pw = cv.take<int>(n_pw);
  int* dinv_pw = cv.take<int>(g.nr);
  char* dscale = cv.take<char>((size_t)n * n_b * 8);
  char* dcw = cv.take<char>((size_t)n * n * 8);
  double* dnorm = cv.take<double>(2 * (size_t)n_b);
  const size_t slab = (size_t)g.nr * n_chi;
  char* slabs = cv.take<char>(slab * n * es);
  char* dc = cv.take<char>((size_t)n_b * n_pw * es);
  char* mo = cv.take<char>((size_t)n_pw * n_pw * es);
  char* mu_ = cv.take<char>((size_t)n_pw * n_pw * es);
  char* to = cv.take<char>((size_t)g.nr * n_pw * es);
  char* tu = cv.take<char>((size_t)g.nr * n_pw * es);
  char* tmp = row_two_pass(g, prec) && is_fp64(prec) ? cv.take<char>((size_t)n_b * g.nr * es) : nullptr;
  const GridInfo gp = pw_grid(g, n_pw);
  void* tcs = tc ? cv.take<char>(tc_scratch_bytes(gp, n_b, n_occ, n_pw, false)) : nullptr;
  if ((st = upload(ctx, dmap, map.data(), sizeof(int) * n_chi, s))) return st;
  if ((st = upload(ctx, dinv, inv.data(), sizeof(int) * g.nr, s))) return st;
  if ((st = upload(ctx, dmap_pw, map_pw.data(), sizeof(int) * n_pw, s))) return st;
  if ((st = upload(ctx, dinv_pw, inv_pw.data(), sizeof(int) * g.nr, s))) return st;
  if (is_fp64(prec)) st = upload(ctx, dcw, cw64.data(), sizeof(double) * n * n, s);
  else st = upload(ctx, dcw, cw32.data(), sizeof(float) * 2 * n * n, s);
  if (st) return st;
  if (!tc)
    for (int j = 0; j < n; ++j)
      if ((st = upload_scales(ctx, dscale + (size_t)j * n_b * 8, scales[j], prec, s))) return st;
  if ((st = pw_coefficients(ctx, g, prec, psi, n_b, n_pw, dmap_pw, dinv_pw, dc, dnorm, tmp, s))) return st;
  bool first = true;
  for (int j = 0; j < n; ++j) {
    // Mc_occ, Mc_unocc over the plane-wave set, then their column transforms T(r, g')
    if (tc) {
      st = tc_green_rows(ctx, gp, n_b, n_occ, dc, scales[j], 0, n_pw, prec, mo, mu_, tcs, first, s);
      first = false;
    } else {
      st = green_rows(ctx, gp, n_b, n_occ, dc, dscale + (size_t)j * n_b * 8, scales[j], 0, n_pw, prec, mo, mu_, s);
    }
    if (st) return st;
    for (int part = 0; part < 2; ++part) {
      char* m = part ? mu_ : mo;
      char* t = part ? tu : to;
      if ((st = launch_col_line(ctx, g, prec, +1, 1, m, n_pw, t, n_pw, n_pw, dinv_pw, 1.0, s))) return st;
      if ((st = launch_col_plane(ctx, g, prec, +1, t, n_pw, n_pw, 1.0, s))) return st;
    }
    // chi(r, G', tau_j) for every row r: expand, multiply (Eq. chi_rr), transform (Eq. FFTX1)
    char* slab_j = slabs + (size_t)j * slab * es;
    if ((st = launch_row_pw_chi(ctx, g, prec, tu, to, n_pw, slab_j, n_chi, dinv_pw, n_pw, dinv, n_chi, g.nr, -2.0, s)))
      return st;
    if ((st = launch_col_plane(ctx, g, prec, -1, slab_j, n_chi, n_chi, 1.0, s))) return st;
  }
  if ((st = launch_col_line_ct(ctx, g, prec, slabs, (long)slab, n_chi, n, dcw, n, chi_w, (long)n_chi * n_chi, n_chi,
                               dinv, n_chi, s, cw32.empty() ? nullptr : cw32.data())))
    return st;
  return tc ? tc_check(ctx, tcs, s) : GW_OK;
}

// ------------------------------------------------------------------ plan

struct gw_chi0_plan {
  gw_ctx* ctx = nullptr;
  GridInfo g{};
  int n_b = 0, n_occ = 0, n = 0, n_chi = 0, rb = 0;
  gw_prec prec = GW_FP32;
  std::vector<GreenScales> scales;
  std::vector<float> cw32;
  void* dev = nullptr;           // the tables, owned by the plan
  Chi0Dev t;
  size_t work = 0;               // context arena bytes a launch uses
};

extern "C" gw_status gw_chi0_plan_create(gw_ctx* ctx, const gw_grid* grid, int n_b, int n_occ, const double* eps_h,
                                         double mu, int n, const double* tau_h, const double* C_h, int n_chi,
                                         const int32_t* fft_index_h, gw_prec prec, int r_block, gw_chi0_plan** out) {
  if (!ctx) return fail(nullptr, GW_ERR_ARG, "ctx is NULL");
  if (!out) return fail(ctx, GW_ERR_ARG, "out is NULL");
  *out = nullptr;
  GridInfo g;
  gw_status st = chi0_check(ctx, grid, &g, n_b, n_occ, eps_h, mu, n, tau_h, C_h, prec);
  if (st) return st;
  std::vector<int> map, inv;
  if ((st = index_maps(ctx, g, fft_index_h, n_chi, map, inv))) return st;
  auto* p = new gw_chi0_plan;
  p->ctx = ctx;
  p->g = g;
  p->n_b = n_b;
  p->n_occ = n_occ;
  p->n = n;
  p->n_chi = n_chi;
  p->prec = prec;
  p->rb = r_block > 0 ? std::min(r_block, g.nr) : std::min(g.nr, 2048);
  std::vector<double> cw64;
  chi0_tables(g, n_b, n_occ, eps_h, mu, n, tau_h, C_h, prec, p->scales, cw64, p->cw32);
  // table layout
  Carver probe(nullptr);
  const size_t o_map = probe.off;
  probe.take<int>(n_chi);
  const size_t o_inv = probe.off;
  probe.take<int>(g.nr);
  const size_t o_scale = probe.off;
  probe.take<char>((size_t)n * n_b * 8);
  const size_t o_sk = probe.off;
  probe.take<float>((size_t)n * n_b);
  const size_t o_cw = probe.off;
  probe.take<char>((size_t)n * n * 8);
  const size_t o_status = probe.off;
  probe.take<int>(2);
  std::vector<char> host(probe.off, 0);
  std::memcpy(host.data() + o_map, map.data(), sizeof(int) * n_chi);
  std::memcpy(host.data() + o_inv, inv.data(), sizeof(int) * g.nr);
  for (int j = 0; j < n; ++j)
    for (int b = 0; b < n_b; ++b) {
      const double v = p->scales[j].s[b];
      // per-tau regions of n_b 8-byte slots, factors packed in the working precision (as upload_scales)
      char* slot = host.data() + o_scale + (size_t)j * n_b * 8 + (size_t)b * (is_fp64(prec) ? 8 : 4);
      if (is_fp64(prec)) std::memcpy(slot, &v, 8);
      else {
        const float f = (float)v;
        std::memcpy(slot, &f, 4);
      }
      const float f = (float)v;
      std::memcpy(host.data() + o_sk + ((size_t)j * n_b + b) * 4, &f, 4);
    }
  if (is_fp64(prec)) std::memcpy(host.data() + o_cw, cw64.data(), sizeof(double) * n * n);
  else std::memcpy(host.data() + o_cw, p->cw32.data(), sizeof(float) * 2 * n * n);
  cudaError_t e = cudaMalloc(&p->dev, host.size());
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return fail(ctx, GW_ERR_OOM, "cannot allocate the plan's tables");
  }
  if ((e = cudaMemcpy(p->dev, host.data(), host.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
    cudaFree(p->dev);
    delete p;
    return cuda_check(ctx, e, "plan tables");
  }
  char* d = static_cast<char*>(p->dev);
  p->t.map = reinterpret_cast<const int*>(d + o_map);
  p->t.inv = reinterpret_cast<const int*>(d + o_inv);
  p->t.scale = d + o_scale;
  p->t.sk = reinterpret_cast<const float*>(d + o_sk);
  p->t.cw = d + o_cw;
  p->t.status = reinterpret_cast<int*>(d + o_status);
  p->work = chi0_omega_scratch(g, n_b, n_occ, n, n_chi, prec, p->rb);
  if ((st = reserve(ctx, p->work))) {
    cudaFree(p->dev);
    delete p;
    return st;
  }
  *out = p;
  return GW_OK;
}

extern "C" gw_status gw_chi0_plan_launch(gw_chi0_plan* p, const void* psi, void* chi_w, void* stream) {
  if (!p) return fail(nullptr, GW_ERR_ARG, "plan is NULL");
  gw_ctx* ctx = p->ctx;
  if (!psi || !chi_w) return fail(ctx, GW_ERR_ARG, "NULL pointer");
  if (ctx->arena_bytes < p->work) return fail(ctx, GW_ERR_ARG, "the context arena is smaller than the plan's");
  Carver cv(ctx->arena);
  return chi0_launch(ctx, p->g, p->n_b, p->n_occ, psi, p->n, p->scales, p->n_chi, p->prec, p->rb, p->t, p->cw32, cv,
                     chi_w, as_stream(stream), nullptr);
}

extern "C" gw_status gw_chi0_plan_status(gw_chi0_plan* p, void* stream) {
  if (!p) return fail(nullptr, GW_ERR_ARG, "plan is NULL");
  gw_status st = cuda_check(p->ctx, cudaStreamSynchronize(as_stream(stream)), "plan sync");
  if (st) return st;
  const bool tc = p->prec == GW_F16X3 || p->prec == GW_BF16X3;
  return tc ? tc_check_status(p->ctx, p->t.status, as_stream(stream)) : GW_OK;
}

namespace gw {
// For the batch plans: the device time-out words of a chi0 plan (2 ints) and
// the arena bytes a launch uses.
int* chi0_plan_status_words(gw_chi0_plan* p) { return p->t.status; }
size_t chi0_plan_work(const gw_chi0_plan* p) { return p->work; }
}  // namespace gw

extern "C" gw_status gw_chi0_plan_destroy(gw_chi0_plan* p) {
  if (!p) return GW_OK;
  cudaFree(p->dev);
  delete p;
  return GW_OK;
}
