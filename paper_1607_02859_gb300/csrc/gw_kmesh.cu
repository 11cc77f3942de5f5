// chi0 on a Gamma-centred k mesh through the supercell stripe (Sec. II.A,
// "Spatial fast Fourier transformation", Eqs. FFT_G1, FFT_G2).
//
// With Bloch orbitals psi_nk(r + L) = exp(i k.L) psi_nk(r), the Green's
// function on the stripe r in the cell C, R' = r' + L in the supercell S is
//   G(r, r'+L, tau) = (1/N_k) sum_k exp(-i k.L) G_k(r, r', tau),
// where G_k is the Gamma-point band sum of Eqs. Green_occ/unocc over the
// orbitals of k (the 1/N_k normalises them over S).  Then, as at Gamma,
//   chi(r, R') = -2 G_occ(r, R') conj(G_unocc(r, R'))            (reading R2)
// and for every q of the mesh
//   chi_q(g, g') = (dV^2/Omega) sum_{r in C} exp(-i(q+g).r)
//                                sum_{R' in S} chi(r, R') exp(+i(q+g').R'),
// the q-diagonal block of the supercell's Gamma-point chi.
//
// For tau_j and each block of r rows:
//   G_occ,k / G_unocc,k rows for every k (the Gamma-point kernels, orbitals of k),
//   stripe_chi_kernel: the k -> L transform of both and their product, written
//       as rows over the supercell grid,
//   the row transform over the supercell grid, gathered to the supercell G set
//       {q + g'} (q outer, g' inner) -> rows of the chi(r, q+g', tau_j) slab.
// Then per slab: exp(-i q.r) on the block of each q, the (i2, i3) column planes;
// last, per q, the i1 column pass fused with the cosine transform.
#include <cmath>

#include "gw_kernels.h"
#include "gw_tc.h"

namespace gw {

constexpr int kMaxK = 64;   // k points per mesh (4 x 4 x 4)

// One row r of the block and 32 consecutive r' per CTA: the N_k values of
// G_occ,k and G_unocc,k are staged in shared memory, then every (L, r') output
// takes its k sum with the phase table ph[k][L] = exp(-i k.L) / N_k.
template <typename T>
__global__ void __launch_bounds__(256) stripe_chi_kernel(const typename cpx<T>::t* __restrict__ go,
                                                         const typename cpx<T>::t* __restrict__ gu, long k_stride,
                                                         int nr, const typename cpx<T>::t* __restrict__ ph, int n_k,
                                                         int n1, int n2, int n3, int nk1, int nk2, int nk3,
                                                         typename cpx<T>::t* __restrict__ out, long ldo) {
  using C = typename cpx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* so = reinterpret_cast<C*>(smem_raw);            // [n_k][32]
  C* su = so + n_k * 32;                             // [n_k][32]
  C* sp = su + n_k * 32;                             // [n_k][n_k]
  const long row = blockIdx.y;
  const int c0 = blockIdx.x * 32;
  for (int e = threadIdx.x; e < n_k * n_k; e += blockDim.x) sp[e] = ph[e];
  for (int e = threadIdx.x; e < n_k * 32; e += blockDim.x) {
    const int k = e >> 5, c = e & 31;
    const long src = (long)k * k_stride + row * nr + c0 + c;
    const bool ok = c0 + c < nr;
    so[e] = ok ? go[src] : mk(T(0), T(0));
    su[e] = ok ? gu[src] : mk(T(0), T(0));
  }
  __syncthreads();
  const int ns2 = n2 * nk2, ns3 = n3 * nk3;
  for (int w = threadIdx.x; w < n_k * 32; w += blockDim.x) {
    const int l = w >> 5, c = w & 31;
    const int rp = c0 + c;
    if (rp >= nr) continue;
    C a = mk(T(0), T(0)), b = a;
    for (int k = 0; k < n_k; ++k) {
      const C p = sp[k * n_k + l];
      a = cadd(a, cmul(p, so[k * 32 + c]));
      b = cadd(b, cmul(p, su[k * 32 + c]));
    }
    const int i1 = rp / (n2 * n3), rem = rp - i1 * n2 * n3, i2 = rem / n3, i3 = rem - i2 * n3;
    const int l1 = l / (nk2 * nk3), lr = l - l1 * nk2 * nk3, l2 = lr / nk3, l3 = lr - l2 * nk3;
    const long pos = ((long)(i1 + n1 * l1) * ns2 + (i2 + n2 * l2)) * ns3 + (i3 + n3 * l3);
    out[row * ldo + pos] = cscale(cmulc(a, b), T(-2));
  }
}

// slab[r][q*n_chi + j] *= exp(-i q.r) for every q of the mesh (r on the cell grid).
template <typename T>
__global__ void __launch_bounds__(256) q_phase_kernel(typename cpx<T>::t* slab, long ld, int n_chi, int n1, int n2,
                                                      int n3, int nk1, int nk2, int nk3) {
  const long r = blockIdx.x;
  const int i1 = (int)(r / (n2 * n3)), rem = (int)(r - (long)i1 * n2 * n3), i2 = rem / n3, i3 = rem - i2 * n3;
  const int n_k = nk1 * nk2 * nk3;
  for (int q = blockIdx.y; q < n_k; q += gridDim.y) {
    const int q1 = q / (nk2 * nk3), qr = q - q1 * nk2 * nk3, q2 = qr / nk3, q3 = qr - q2 * nk3;
    // q.r / 2 pi = sum_d q_d i_d / (nk_d n_d), reduced mod 1 before the trigonometry
    double f = (double)q1 * i1 / (nk1 * n1) + (double)q2 * i2 / (nk2 * n2) + (double)q3 * i3 / (nk3 * n3);
    f -= floor(f);
    double s, c;
    sincospi(-2.0 * f, &s, &c);
    const T cr = T(c), ci = T(s);
    auto* p = slab + r * ld + (long)q * n_chi;
    for (int j = threadIdx.x; j < n_chi; j += blockDim.x) {
      const auto v = p[j];
      p[j] = mk(v.x * cr - v.y * ci, v.x * ci + v.y * cr);
    }
  }
}

}  // namespace gw

using namespace gw;

extern "C" gw_status gw_chi0_omega_kmesh(gw_ctx* ctx, const gw_grid* grid, const int* nk, int n_b, int n_occ,
                                         const void* psi_k, const double* eps_k_h, double mu, int n,
                                         const double* tau_h, const double* C_h, int n_chi, const int32_t* gvec_h,
                                         gw_prec prec, int r_block, void* chi_w, void* stream) {
  if (!ctx) return fail(nullptr, GW_ERR_ARG, "ctx is NULL");
  GridInfo g;
  gw_status st = grid_info(ctx, grid, &g);
  if (st) return st;
  if (!nk || !psi_k || !eps_k_h || !tau_h || !C_h || !gvec_h || !chi_w) return fail(ctx, GW_ERR_ARG, "NULL pointer");
  if (!valid_prec(prec)) return fail(ctx, GW_ERR_ARG, "bad precision");
  for (int d = 0; d < 3; ++d)
    if (nk[d] < 1) return fail(ctx, GW_ERR_SHAPE, "k mesh dimensions must be >= 1");
  const int n_k = nk[0] * nk[1] * nk[2];
  if (n_k > kMaxK) return fail(ctx, GW_ERR_SHAPE, "at most 64 k points");
  gw_grid sgrid;
  for (int d = 0; d < 3; ++d) {
    sgrid.n[d] = grid->n[d] * nk[d];
    for (int e = 0; e < 3; ++e) sgrid.lattice[3 * d + e] = grid->lattice[3 * d + e] * nk[d];
  }
  GridInfo gs;
  if ((st = grid_info(ctx, &sgrid, &gs))) return st;
  if (!grid_supported(g.n1, g.n2, g.n3) || !grid_supported(gs.n1, gs.n2, gs.n3))
    return fail(ctx, GW_ERR_UNSUPPORTED, "no kernels compiled for the cell or the supercell grid");
  if (n_b < 2 || n_b > g.nr) return fail(ctx, GW_ERR_SHAPE, "need 2 <= n_b <= N_r");
  for (int k = 0; k < n_k; ++k)
    if ((st = check_energies(ctx, eps_k_h + (size_t)k * n_b, n_b, n_occ, mu))) return st;
  if (n < 1 || n > 32) return fail(ctx, GW_ERR_SHAPE, "need 1 <= n <= 32");
  for (int j = 0; j < n; ++j)
    if (!(tau_h[j] > 0)) return fail(ctx, GW_ERR_ARG, "tau must be > 0");
  if (n_chi < 1 || n_chi > g.nr) return fail(ctx, GW_ERR_SHAPE, "need 1 <= n_chi <= N_r");
  // cell G set -> cell grid positions, supercell G set {q + g} -> supercell grid positions
  const int cn[3] = {g.n1, g.n2, g.n3}, sn[3] = {gs.n1, gs.n2, gs.n3};
  std::vector<int32_t> fidx(n_chi), sidx((size_t)n_k * n_chi);
  for (int j = 0; j < n_chi; ++j) {
    int p = 0;
    for (int d = 0; d < 3; ++d) {
      const int v = gvec_h[3 * j + d];
      if (v < -(cn[d] / 2) || v >= cn[d] - cn[d] / 2) return fail(ctx, GW_ERR_ARG, "G vector outside the cell grid");
      p = p * cn[d] + ((v % cn[d]) + cn[d]) % cn[d];
    }
    fidx[j] = p;
  }
  for (int q = 0; q < n_k; ++q) {
    const int qv[3] = {q / (nk[1] * nk[2]), (q / nk[2]) % nk[1], q % nk[2]};
    for (int j = 0; j < n_chi; ++j) {
      int p = 0;
      for (int d = 0; d < 3; ++d) {
        const int m = qv[d] + nk[d] * gvec_h[3 * j + d];
        p = p * sn[d] + ((m % sn[d]) + sn[d]) % sn[d];
      }
      sidx[(size_t)q * n_chi + j] = p;
    }
  }
  std::vector<int> map, inv, smap, sinv;
  if ((st = index_maps(ctx, g, fidx.data(), n_chi, map, inv))) return st;
  if ((st = index_maps(ctx, gs, sidx.data(), n_k * n_chi, smap, sinv))) return st;
  cudaStream_t s = as_stream(stream);
  const size_t es = csize(prec);
  const int rb = r_block > 0 ? std::min(r_block, g.nr) : std::min(g.nr, 1024);
  const bool tc = prec == GW_F16X3 || prec == GW_BF16X3;
  const bool two_pass = row_two_pass(gs, prec);
  const long ld = (long)n_k * n_chi;                   // slab row: all q blocks
  const size_t slab = (size_t)g.nr * ld;
  // scratch
  Carver probe(nullptr);
  probe.take<int>(n_chi);
  probe.take<int>(g.nr);
  probe.take<int>((size_t)n_k * n_chi);
  probe.take<int>(gs.nr);
  probe.take<double>((size_t)n_k * n_b);
  probe.take<double>((size_t)n * n);
  probe.take<double2>((size_t)n_k * n_k);
  probe.take<char>(slab * n * es);
  probe.take<char>((size_t)n_k * rb * g.nr * es);
  probe.take<char>((size_t)n_k * rb * g.nr * es);
  probe.take<char>((size_t)rb * gs.nr * es);
  if (two_pass) probe.take<char>((size_t)rb * gs.nr * es);
  if (tc) probe.take<char>(tc_scratch_bytes(g, n_b, n_occ, rb, false));
  if ((st = reserve(ctx, probe.off))) return st;
  Carver cv(ctx->arena);
  int* dmap = cv.take<int>(n_chi);
  int* dinv = cv.take<int>(g.nr);
  int* dsmap = cv.take<int>((size_t)n_k * n_chi);
  int* dsinv = cv.take<int>(gs.nr);
  char* dscale = cv.take<char>((size_t)n_k * n_b * 8);
  char* dcw = cv.take<char>((size_t)n * n * 8);
  char* dph = cv.take<char>((size_t)n_k * n_k * 16);
  char* slabs = cv.take<char>(slab * n * es);
  char* gok = cv.take<char>((size_t)n_k * rb * g.nr * es);
  char* guk = cv.take<char>((size_t)n_k * rb * g.nr * es);
  char* rows_s = cv.take<char>((size_t)rb * gs.nr * es);
  char* tmp_s = two_pass ? cv.take<char>((size_t)rb * gs.nr * es) : nullptr;
  void* tcs = tc ? cv.take<char>(tc_scratch_bytes(g, n_b, n_occ, rb, false)) : nullptr;
  if ((st = upload(ctx, dmap, map.data(), sizeof(int) * n_chi, s))) return st;
  if ((st = upload(ctx, dinv, inv.data(), sizeof(int) * g.nr, s))) return st;
  if ((st = upload(ctx, dsmap, smap.data(), sizeof(int) * n_k * n_chi, s))) return st;
  if ((st = upload(ctx, dsinv, sinv.data(), sizeof(int) * gs.nr, s))) return st;
  // phase table exp(-i k.L) / N_k, k.L / 2 pi = sum_d k_d l_d / nk_d
  {
    std::vector<double> ph(2 * (size_t)n_k * n_k);
    for (int k = 0; k < n_k; ++k)
      for (int l = 0; l < n_k; ++l) {
        const int kv[3] = {k / (nk[1] * nk[2]), (k / nk[2]) % nk[1], k % nk[2]};
        const int lv[3] = {l / (nk[1] * nk[2]), (l / nk[2]) % nk[1], l % nk[2]};
        long num = 0;   // sum_d k_d l_d / nk_d over a common denominator
        const long den = (long)nk[0] * nk[1] * nk[2];
        for (int d = 0; d < 3; ++d) num += (long)kv[d] * lv[d] * (den / nk[d]);
        const double a = -2.0 * M_PI * (double)(num % den) / (double)den;
        ph[2 * ((size_t)k * n_k + l)] = std::cos(a) / n_k;
        ph[2 * ((size_t)k * n_k + l) + 1] = std::sin(a) / n_k;
      }
    if (is_fp64(prec)) {
      if ((st = upload(ctx, dph, ph.data(), sizeof(double) * ph.size(), s))) return st;
    } else {
      std::vector<float> f(ph.begin(), ph.end());
      if ((st = upload(ctx, dph, f.data(), sizeof(float) * f.size(), s))) return st;
    }
  }
  const double fac = g.dv * g.dv / g.volume;   // Eq. FFTX2 normalisation
  std::vector<float> cw32;
  if (is_fp64(prec)) {
    std::vector<double> cw(C_h, C_h + n * n);
    for (auto& v : cw) v *= fac;
    if ((st = upload(ctx, dcw, cw.data(), sizeof(double) * n * n, s))) return st;
  } else {
    cw32 = split_weights(C_h, n * n, fac);
    if ((st = upload(ctx, dcw, cw32.data(), sizeof(float) * 2 * n * n, s))) return st;
  }
  const size_t smem = (size_t)(2 * n_k * 32 + n_k * n_k) * es;
  const long kstr = (long)rb * g.nr;
  for (int j = 0; j < n; ++j) {
    std::vector<GreenScales> scales(n_k);
    for (int k = 0; k < n_k; ++k) {
      scales[k] = green_scales(eps_k_h + (size_t)k * n_b, n_b, n_occ, mu, tau_h[j]);
      if (!tc && (st = upload_scales(ctx, dscale + (size_t)k * n_b * 8, scales[k], prec, s))) return st;
    }
    char* slab_j = slabs + (size_t)j * slab * es;
    for (int r0 = 0; r0 < g.nr; r0 += rb) {
      const int rows = std::min(rb, g.nr - r0);
      for (int k = 0; k < n_k; ++k) {
        const char* pk = static_cast<const char*>(psi_k) + (size_t)k * n_b * g.nr * es;
        char* ok = gok + (size_t)k * kstr * es;
        char* uk = guk + (size_t)k * kstr * es;
        if (tc) st = tc_green_rows(ctx, g, n_b, n_occ, pk, scales[k], r0, rows, prec, ok, uk, tcs, true, s);
        else st = green_rows(ctx, g, n_b, n_occ, pk, dscale + (size_t)k * n_b * 8, scales[k], r0, rows, prec, ok,
                             uk, s);
        if (st) return st;
      }
      const dim3 grd((g.nr + 31) / 32, rows);
      if (is_fp64(prec)) {
        auto kern = stripe_chi_kernel<double>;
        if (smem > 48 * 1024 && (st = cuda_check(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                                          (int)smem), "cudaFuncSetAttribute")))
          return st;
        kern<<<grd, 256, smem, s>>>((const double2*)gok, (const double2*)guk, kstr, g.nr, (const double2*)dph, n_k,
                                    g.n1, g.n2, g.n3, nk[0], nk[1], nk[2], (double2*)rows_s, gs.nr);
      } else {
        auto kern = stripe_chi_kernel<float>;
        if (smem > 48 * 1024 && (st = cuda_check(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                                          (int)smem), "cudaFuncSetAttribute")))
          return st;
        kern<<<grd, 256, smem, s>>>((const float2*)gok, (const float2*)guk, kstr, g.nr, (const float2*)dph, n_k,
                                    g.n1, g.n2, g.n3, nk[0], nk[1], nk[2], (float2*)rows_s, gs.nr);
      }
      if ((st = launch_check(ctx, "stripe_chi_kernel"))) return st;
      if ((st = launch_row_fft(ctx, gs, prec, 1, rows_s, nullptr, gs.nr, slab_j + (size_t)r0 * ld * es, ld, dsmap,
                               n_k * n_chi, rows, 1.0, s, dsinv, tmp_s)))
        return st;
    }
    const dim3 gq(g.nr, std::min(n_k, 8));
    if (is_fp64(prec))
      q_phase_kernel<double><<<gq, 256, 0, s>>>((double2*)slab_j, ld, n_chi, g.n1, g.n2, g.n3, nk[0], nk[1], nk[2]);
    else
      q_phase_kernel<float><<<gq, 256, 0, s>>>((float2*)slab_j, ld, n_chi, g.n1, g.n2, g.n3, nk[0], nk[1], nk[2]);
    if ((st = launch_check(ctx, "q_phase_kernel"))) return st;
    if ((st = launch_col_plane(ctx, g, prec, -1, slab_j, ld, (int)ld, 1.0, s))) return st;
  }
  for (int q = 0; q < n_k; ++q) {
    char* out_q = static_cast<char*>(chi_w) + (size_t)q * n * n_chi * n_chi * es;
    if ((st = launch_col_line_ct(ctx, g, prec, slabs + (size_t)q * n_chi * es, (long)slab, ld, n, dcw, n, out_q,
                                 (long)n_chi * n_chi, n_chi, dinv, n_chi, s, cw32.empty() ? nullptr : cw32.data())))
      return st;
  }
  return tc ? tc_check(ctx, tcs, s) : GW_OK;
}
