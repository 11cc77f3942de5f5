// Imaginary-time Green's functions (Eqs. Green_occ, Green_unocc) and the fused
// G formation + real-space product of Eq. chi_rr.
//
// G_occ(r,R') = A_occ sum_{i<n_occ} psi_i(r) s_i psi_i^*(R'),
// s_i = exp((eps_i-mu) tau) / A_occ,  A_occ = max_i exp((eps_i-mu) tau)
// (likewise for the unoccupied set with exp(-(eps_a-mu) tau)).  The
// exponentials are formed in FP64 on the host; dividing by the largest one
// keeps every pre-scaled factor in (0, 1] whatever tau is, and the FP64 factor
// A is applied once to the accumulated tile.
#include <algorithm>
#include <cmath>

#include "gw_kernels.h"
#include "gw_tc.h"

namespace gw {

GreenScales green_scales(const double* eps, int n_b, int n_occ, double mu, double tau) {
  GreenScales gs;
  gs.s.resize(n_b);
  double lo = -1e300, hi = -1e300;
  for (int i = 0; i < n_occ; ++i) lo = std::max(lo, (eps[i] - mu) * tau);
  for (int a = n_occ; a < n_b; ++a) hi = std::max(hi, -(eps[a] - mu) * tau);
  for (int i = 0; i < n_occ; ++i) gs.s[i] = std::exp((eps[i] - mu) * tau - lo);
  for (int a = n_occ; a < n_b; ++a) gs.s[a] = std::exp(-(eps[a] - mu) * tau - hi);
  gs.amax_occ = std::exp(lo);
  gs.amax_unocc = std::exp(hi);
  return gs;
}

gw_status green_rows(gw_ctx* ctx, const GridInfo& g, int n_b, int n_occ, const void* psi, const void* dscale,
                     const GreenScales& gs, int r0, int n_rows, gw_prec prec, void* g_occ, void* g_unocc,
                     cudaStream_t st) {
  const size_t es = csize(prec);
  const size_t ss = is_fp64(prec) ? 8 : 4;
  const char* p = static_cast<const char*>(psi);
  const char* sc = static_cast<const char*>(dscale);
  gw_status rc;
  for (int part = 0; part < 2; ++part) {
    void* out = part == 0 ? g_occ : g_unocc;
    if (!out) continue;
    const int k0 = part == 0 ? 0 : n_occ;
    const int kn = part == 0 ? n_occ : n_b - n_occ;
    GemmArgs a{};
    a.M = n_rows;
    a.N = g.nr;
    a.K = kn;
    a.alpha_re = part == 0 ? gs.amax_occ : gs.amax_unocc;
    a.alpha_im = 0;
    a.beta = 0;
    a.A = p + ((size_t)k0 * g.nr + r0) * es;
    a.lda = g.nr;
    a.a_km = 1;
    a.a_conj = false;
    a.B = p + (size_t)k0 * g.nr * es;
    a.ldb = g.nr;
    a.b_nk = 0;
    a.b_conj = true;
    a.C = out;
    a.ldc = g.nr;
    a.kscale = sc + (size_t)k0 * ss;
    a.tri = 0;
    if ((rc = launch_gemm(ctx, prec, a, st))) return rc;
  }
  return GW_OK;
}

// Validation shared by the two entry points below.
static gw_status check_green(gw_ctx* ctx, const gw_grid* grid, GridInfo* g, int n_b, int n_occ, const void* psi,
                             const double* eps_h, double mu, double tau, int r0, int n_rows, gw_prec prec) {
  if (!ctx) return fail(nullptr, GW_ERR_ARG, "ctx is NULL");
  gw_status st = grid_info(ctx, grid, g);
  if (st) return st;
  if (!valid_prec(prec)) return fail(ctx, GW_ERR_ARG, "bad precision");
  if (!psi) return fail(ctx, GW_ERR_ARG, "psi is NULL");
  if (n_b < 2 || n_b > g->nr) return fail(ctx, GW_ERR_SHAPE, "need 2 <= n_b <= N_r");
  if ((st = check_energies(ctx, eps_h, n_b, n_occ, mu))) return st;
  if (!(tau > 0) || !std::isfinite(tau)) return fail(ctx, GW_ERR_ARG, "tau must be > 0");
  if (n_rows < 0 || r0 < 0 || r0 + n_rows > g->nr) return fail(ctx, GW_ERR_SHAPE, "rows out of range");
  return GW_OK;
}

gw_status upload_scales(gw_ctx* ctx, void* dst, const GreenScales& gs, gw_prec prec, cudaStream_t st) {
  if (is_fp64(prec)) return upload(ctx, dst, gs.s.data(), sizeof(double) * gs.s.size(), st);
  std::vector<float> f(gs.s.begin(), gs.s.end());
  return upload(ctx, dst, f.data(), sizeof(float) * f.size(), st);
}

}  // namespace gw

using namespace gw;

extern "C" gw_status gw_green_tau(gw_ctx* ctx, const gw_grid* grid, int n_b, int n_occ, const void* psi,
                                  const double* eps_h, double mu, double tau, int r0, int n_rows, gw_prec prec,
                                  void* g_occ, void* g_unocc, void* stream) {
  GridInfo g;
  gw_status st = check_green(ctx, grid, &g, n_b, n_occ, psi, eps_h, mu, tau, r0, n_rows, prec);
  if (st) return st;
  if (n_rows == 0 || (!g_occ && !g_unocc)) return GW_OK;
  cudaStream_t s = as_stream(stream);
  GreenScales gs = green_scales(eps_h, n_b, n_occ, mu, tau);
  if (prec == GW_F16X3 || prec == GW_BF16X3) {
    if ((st = reserve(ctx, tc_scratch_bytes(g, n_b, n_occ, n_rows, !g_occ || !g_unocc)))) return st;
    if ((st = tc_green_rows(ctx, g, n_b, n_occ, psi, gs, r0, n_rows, prec, g_occ, g_unocc, ctx->arena, true, s)))
      return st;
    return tc_check(ctx, ctx->arena, s);
  }
  if ((st = reserve(ctx, Carver::round(sizeof(double) * n_b)))) return st;
  if ((st = upload_scales(ctx, ctx->arena, gs, prec, s))) return st;
  return green_rows(ctx, g, n_b, n_occ, psi, ctx->arena, gs, r0, n_rows, prec, g_occ, g_unocc, s);
}

extern "C" gw_status gw_chi0_rtau_fused(gw_ctx* ctx, const gw_grid* grid, int n_b, int n_occ, const void* psi,
                                        const double* eps_h, double mu, double tau, int r0, int n_rows,
                                        gw_prec prec, void* chi, void* stream) {
  GridInfo g;
  gw_status st = check_green(ctx, grid, &g, n_b, n_occ, psi, eps_h, mu, tau, r0, n_rows, prec);
  if (st) return st;
  if (!chi) return fail(ctx, GW_ERR_ARG, "chi is NULL");
  if (n_rows == 0) return GW_OK;
  cudaStream_t s = as_stream(stream);
  GreenScales gs = green_scales(eps_h, n_b, n_occ, mu, tau);
  if (prec == GW_F16X3 || prec == GW_BF16X3) {
    if ((st = reserve(ctx, tc_scratch_bytes(g, n_b, n_occ, n_rows, false)))) return st;
    if ((st = tc_chi_rows(ctx, g, n_b, n_occ, psi, gs, r0, n_rows, prec, chi, ctx->arena, true, s))) return st;
    return tc_check(ctx, ctx->arena, s);
  }
  // CUDA-core precisions: G_occ goes through scratch, G_unocc is formed in
  // place in chi and the product overwrites it.
  const size_t es = csize(prec);
  Carver probe(nullptr);
  probe.take<double>(n_b);
  probe.take<char>((size_t)n_rows * g.nr * es);
  if ((st = reserve(ctx, probe.off))) return st;
  Carver cv(ctx->arena);
  void* dscale = cv.take<double>(n_b);
  void* gocc = cv.take<char>((size_t)n_rows * g.nr * es);
  if ((st = upload_scales(ctx, dscale, gs, prec, s))) return st;
  if ((st = green_rows(ctx, g, n_b, n_occ, psi, dscale, gs, r0, n_rows, prec, gocc, chi, s))) return st;
  return launch_hadamard(ctx, prec, (size_t)n_rows * g.nr, gocc, chi, -2.0, chi, s);
}
