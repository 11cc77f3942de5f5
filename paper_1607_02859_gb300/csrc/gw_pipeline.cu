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

}  // namespace gw

using namespace gw;

extern "C" gw_status gw_chi0_omega(gw_ctx* ctx, const gw_grid* grid, int n_b, int n_occ, const void* psi,
                                   const double* eps_h, double mu, int n, const double* tau_h, const double* C_h,
                                   int n_chi, const int32_t* fft_index_h, gw_prec prec, int r_block, void* chi_w,
                                   void* stream) {
  if (!ctx) return fail(nullptr, GW_ERR_ARG, "ctx is NULL");
  GridInfo g;
  gw_status st = grid_info(ctx, grid, &g);
  if (st) return st;
  if (!grid_supported(g.n1, g.n2, g.n3)) return fail(ctx, GW_ERR_UNSUPPORTED, "no kernels compiled for this grid");
  if (!valid_prec(prec)) return fail(ctx, GW_ERR_ARG, "bad precision");
  if (!psi || !tau_h || !C_h || !chi_w) return fail(ctx, GW_ERR_ARG, "NULL pointer");
  if (n_b < 2 || n_b > g.nr) return fail(ctx, GW_ERR_SHAPE, "need 2 <= n_b <= N_r");
  if ((st = check_energies(ctx, eps_h, n_b, n_occ, mu))) return st;
  if (n < 1 || n > 32) return fail(ctx, GW_ERR_SHAPE, "need 1 <= n <= 32");
  for (int j = 0; j < n; ++j)
    if (!(tau_h[j] > 0)) return fail(ctx, GW_ERR_ARG, "tau must be > 0");
  std::vector<int> map, inv;
  if ((st = index_maps(ctx, g, fft_index_h, n_chi, map, inv))) return st;
  cudaStream_t s = as_stream(stream);
  const size_t es = csize(prec);
  const int rb = r_block > 0 ? std::min(r_block, g.nr) : std::min(g.nr, 2048);
  const bool tc = prec == GW_F16X3 || prec == GW_BF16X3;
  const size_t slab = (size_t)g.nr * n_chi;
  if ((st = reserve(ctx, chi0_omega_scratch(g, n_b, n_occ, n, n_chi, prec, rb)))) return st;
  Carver cv(ctx->arena);
  int* dmap = cv.take<int>(n_chi);
  int* dinv = cv.take<int>(g.nr);
  char* dscale = cv.take<char>((size_t)n * n_b * 8);
  char* dcw = cv.take<char>((size_t)n * n * 8);
  char* slabs = cv.take<char>(slab * n * es);
  char* ga = cv.take<char>((size_t)rb * g.nr * es);
  char* gb = cv.take<char>((size_t)rb * g.nr * es);
  void* tcs = tc ? cv.take<char>(tc_scratch_bytes(g, n_b, n_occ, rb, false)) : nullptr;
  bool first = true;
  if ((st = upload(ctx, dmap, map.data(), sizeof(int) * n_chi, s))) return st;
  if ((st = upload(ctx, dinv, inv.data(), sizeof(int) * g.nr, s))) return st;
  const double fac = g.dv * g.dv / g.volume;   // Eq. FFTX2 normalisation
  std::vector<float> cw32;                     // FP32 weights (hi, lo) for the register variant of the last pass
  if (is_fp64(prec)) {
    std::vector<double> cw(C_h, C_h + n * n);
    for (auto& v : cw) v *= fac;
    if ((st = upload(ctx, dcw, cw.data(), sizeof(double) * n * n, s))) return st;
  } else {
    cw32 = split_weights(C_h, n * n, fac);
    if ((st = upload(ctx, dcw, cw32.data(), sizeof(float) * 2 * n * n, s))) return st;
  }
  for (int j = 0; j < n; ++j) {
    GreenScales gs = green_scales(eps_h, n_b, n_occ, mu, tau_h[j]);
    char* sj = dscale + (size_t)j * n_b * 8;
    if (!tc && (st = upload_scales(ctx, sj, gs, prec, s))) return st;
    char* slab_j = slabs + (size_t)j * slab * es;
    for (int r0 = 0; r0 < g.nr; r0 += rb) {
      const int rows = std::min(rb, g.nr - r0);
      if (tc) {
        if ((st = tc_chi_rows(ctx, g, n_b, n_occ, psi, gs, r0, rows, prec, ga, tcs, first, s))) return st;
        first = false;
        st = launch_row_fft(ctx, g, prec, 1, ga, nullptr, g.nr, slab_j + (size_t)r0 * n_chi * es, n_chi, dmap, n_chi,
                            rows, 1.0, s, dinv, gb);
      } else {
        if ((st = green_rows(ctx, g, n_b, n_occ, psi, sj, gs, r0, rows, prec, ga, gb, s))) return st;
        st = launch_row_fft(ctx, g, prec, 0, ga, gb, g.nr, slab_j + (size_t)r0 * n_chi * es, n_chi, dmap, n_chi, rows,
                            -2.0, s, dinv, ga);
      }
      if (st) return st;
    }
    if ((st = launch_col_plane(ctx, g, prec, -1, slab_j, n_chi, n_chi, 1.0, s))) return st;
  }
  if ((st = launch_col_line_ct(ctx, g, prec, slabs, (long)slab, n_chi, n, dcw, n, chi_w, (long)n_chi * n_chi, n_chi,
                               dinv, n_chi, s, cw32.empty() ? nullptr : cw32.data())))
    return st;
  return tc ? tc_check(ctx, tcs, s) : GW_OK;
}
