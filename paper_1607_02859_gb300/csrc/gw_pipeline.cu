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
