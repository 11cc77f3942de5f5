// chi0 on a Gamma-centred k mesh through the supercell stripe (Sec. II.A,
// "Spatial fast Fourier transformation", Eqs. FFT_G1, FFT_G2).
//
// With Bloch orbitals psi_nk(r + L) = exp(i k.L) psi_nk(r), the Green's
// function on the stripe r in the cell C, R' = r' + L in the supercell S is
//   G(r, r'+L, tau) = (1/N_k) sum_k exp(-i k.L) G_k(r, r', tau),
// where G_k is the Gamma-point band sum of Eqs. Green_occ/unocc over the
// orbitals of k (the 1/N_k normalises them over S).  Then, as at Gamma,
//   chi(r, R') = -2 G_occ(r, R') conj(G_unocc(r, R'))
// (spin-degenerate, index order G_occ(r,r') G_unocc(r',r), i.e. the conjugate
// of the printed tau > 0 slice of Eq. chi_rr for complex orbitals)
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
#include <cstring>
#include <type_traits>

#include "gw_kernels.h"
#include "gw_tc.h"

namespace gw {

constexpr int kMaxK = 64;   // k points per mesh (4 x 4 x 4)

// One row r of the block and 32 consecutive r' per CTA: the N_k values of
// G_occ,k and G_unocc,k are staged in shared memory, then every (L, r') output
// takes its k sum with the phase table ph[k][L] = exp(-i k.L) / N_k.
// PRODUCT: out = -2 G_occ conj(G_unocc) on the stripe; else out = G_occ and out2 = G_unocc.
template <typename T, bool PRODUCT>
__global__ void __launch_bounds__(256) stripe_chi_kernel(const typename cpx<T>::t* __restrict__ go,
                                                         const typename cpx<T>::t* __restrict__ gu, long k_stride,
                                                         int nr, const typename cpx<T>::t* __restrict__ ph, int n_k,
                                                         int n1, int n2, int n3, int nk1, int nk2, int nk3,
                                                         typename cpx<T>::t* __restrict__ out,
                                                         typename cpx<T>::t* __restrict__ out2, long ldo) {
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
    if (PRODUCT) {
      out[row * ldo + pos] = cscale(cmulc(a, b), T(-2));
    } else {
      out[row * ldo + pos] = a;
      out2[row * ldo + pos] = b;
    }
  }
}

// slab[r][q*n_chi + j] *= exp(sgn i q.r)
template <typename T>
__global__ void __launch_bounds__(256) q_phase_kernel(typename cpx<T>::t* slab, long ld, int n_chi, int n1, int n2,
                                                      int n3, int nk1, int nk2, int nk3, double sgn) {
  const long r = blockIdx.x;
  const int i1 = (int)(r / (n2 * n3)), rem = (int)(r - (long)i1 * n2 * n3), i2 = rem / n3, i3 = rem - i2 * n3;
  const int n_k = nk1 * nk2 * nk3;
  for (int q = blockIdx.y; q < n_k; q += gridDim.y) {
    const int q1 = q / (nk2 * nk3), qr = q - q1 * nk2 * nk3, q2 = qr / nk3, q3 = qr - q2 * nk3;
    // q.r / 2 pi = sum_d q_d i_d / (nk_d n_d), reduced mod 1 before the trigonometry
    double f = (double)q1 * i1 / (nk1 * n1) + (double)q2 * i2 / (nk2 * n2) + (double)q3 * i3 / (nk3 * n3);
    f -= floor(f);
    double s, c;
    sincospi(2.0 * sgn * f, &s, &c);
    const T cr = T(c), ci = T(s);
    auto* p = slab + r * ld + (long)q * n_chi;
    for (int j = threadIdx.x; j < n_chi; j += blockDim.x) {
      const auto v = p[j];
      p[j] = mk(v.x * cr - v.y * ci, v.x * ci + v.y * cr);
    }
  }
}

// Orbitals of the requested (band, k) pairs: ext[i][pos(r', L)] = exp(i k.L) psi_bk(r')
// over the supercell grid, and row[i][r'] = psi_bk(r') on the cell grid.
template <typename T>
__global__ void __launch_bounds__(256) bloch_extend_kernel(const typename cpx<T>::t* __restrict__ psi_k, long k_stride,
                                                           int nr, const int* __restrict__ bk, int n1, int n2, int n3,
                                                           int nk1, int nk2, int nk3, typename cpx<T>::t* __restrict__ ext,
                                                           typename cpx<T>::t* __restrict__ row) {
  const int rp = blockIdx.x * blockDim.x + threadIdx.x;
  const int l = blockIdx.y, i = blockIdx.z;
  if (rp >= nr) return;
  const int b = bk[2 * i], k = bk[2 * i + 1];
  const auto v = psi_k[(long)k * k_stride + (long)b * nr + rp];
  const int k1 = k / (nk2 * nk3), kr = k - k1 * nk2 * nk3, k2 = kr / nk3, k3 = kr - k2 * nk3;
  const int l1 = l / (nk2 * nk3), lr = l - l1 * nk2 * nk3, l2 = lr / nk3, l3 = lr - l2 * nk3;
  double f = (double)k1 * l1 / nk1 + (double)k2 * l2 / nk2 + (double)k3 * l3 / nk3;   // k.L / 2 pi
  f -= floor(f);
  double sn, cs;
  sincospi(2.0 * f, &sn, &cs);
  const T c = T(cs), s = T(sn);
  const int i1 = rp / (n2 * n3), rem = rp - i1 * n2 * n3, i2 = rem / n3, i3 = rem - i2 * n3;
  const long ns = (long)n1 * nk1 * n2 * nk2 * n3 * nk3;
  const long pos = ((long)(i1 + n1 * l1) * (n2 * nk2) + (i2 + n2 * l2)) * (n3 * nk3) + (i3 + n3 * l3);
  ext[(long)i * ns + pos] = mk(v.x * c - v.y * s, v.x * s + v.y * c);
  if (l == 0) row[(long)i * nr + rp] = v;
}

// The orbitals of one k with the Bloch phase taken off: u[b][r] = exp(-i k.r) psi_bk(r),
// the cell-periodic parts whose plane-wave coefficients the plane-wave form of
// G_k is built from (k.r / 2 pi = sum_d k_d i_d / (nk_d n_d), reduced mod 1).
template <typename T>
__global__ void __launch_bounds__(256) bloch_unphase_kernel(const typename cpx<T>::t* __restrict__ psi, int nr,
                                                            int n1, int n2, int n3, int k1, int k2, int k3, int nk1,
                                                            int nk2, int nk3, typename cpx<T>::t* __restrict__ u) {
  const int rp = blockIdx.x * blockDim.x + threadIdx.x;
  if (rp >= nr) return;
  const long b = blockIdx.y;
  const int i1 = rp / (n2 * n3), rem = rp - i1 * n2 * n3, i2 = rem / n3, i3 = rem - i2 * n3;
  double f = (double)k1 * i1 / (nk1 * n1) + (double)k2 * i2 / (nk2 * n2) + (double)k3 * i3 / (nk3 * n3);
  f -= floor(f);
  double sn, cs;
  sincospi(-2.0 * f, &sn, &cs);
  const T c = T(cs), s = T(sn);
  const auto v = psi[b * nr + rp];
  u[b * nr + rp] = mk(v.x * c - v.y * s, v.x * s + v.y * c);
}

// The supercell grid of a k mesh, and the index maps of the cell G set (cell
// grid) and of the supercell G set {q + g} (q outer, g inner) on the supercell grid.
static gw_status kmesh_grids(gw_ctx* ctx, const gw_grid* grid, const int* nk, int n_chi, const int32_t* gvec_h,
                             GridInfo* g, GridInfo* gs, std::vector<int>& map, std::vector<int>& inv,
                             std::vector<int>& smap, std::vector<int>& sinv) {
  gw_status st = grid_info(ctx, grid, g);
  if (st) return st;
  if (!nk || !gvec_h) return fail(ctx, GW_ERR_ARG, "NULL pointer");
  for (int d = 0; d < 3; ++d)
    if (nk[d] < 1) return fail(ctx, GW_ERR_SHAPE, "k mesh dimensions must be >= 1");
  const int n_k = nk[0] * nk[1] * nk[2];
  if (n_k > kMaxK) return fail(ctx, GW_ERR_SHAPE, "at most 64 k points");
  gw_grid sgrid;
  for (int d = 0; d < 3; ++d) {
    sgrid.n[d] = grid->n[d] * nk[d];
    for (int e = 0; e < 3; ++e) sgrid.lattice[3 * d + e] = grid->lattice[3 * d + e] * nk[d];
  }
  if ((st = grid_info(ctx, &sgrid, gs))) return st;
  if (!grid_supported(g->n1, g->n2, g->n3) || !grid_supported(gs->n1, gs->n2, gs->n3))
    return fail(ctx, GW_ERR_UNSUPPORTED, "no kernels compiled for the cell or the supercell grid");
  if (n_chi < 1 || n_chi > g->nr) return fail(ctx, GW_ERR_SHAPE, "need 1 <= n_chi <= N_r");
  const int cn[3] = {g->n1, g->n2, g->n3}, sn[3] = {gs->n1, gs->n2, gs->n3};
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
  if ((st = index_maps(ctx, *g, fidx.data(), n_chi, map, inv))) return st;
  return index_maps(ctx, *gs, sidx.data(), n_k * n_chi, smap, sinv);
}

// exp(-i k.L) / N_k for every k (rows) and L (columns), k.L / 2 pi = sum_d k_d l_d / nk_d.
static std::vector<double> kl_phases(const int* nk) {
  const int n_k = nk[0] * nk[1] * nk[2];
  std::vector<double> ph(2 * (size_t)n_k * n_k);
  const long den = (long)nk[0] * nk[1] * nk[2];
  for (int k = 0; k < n_k; ++k)
    for (int l = 0; l < n_k; ++l) {
      const int kv[3] = {k / (nk[1] * nk[2]), (k / nk[2]) % nk[1], k % nk[2]};
      const int lv[3] = {l / (nk[1] * nk[2]), (l / nk[2]) % nk[1], l % nk[2]};
      long num = 0;
      for (int d = 0; d < 3; ++d) num += (long)kv[d] * lv[d] * (den / nk[d]);
      const double a = -2.0 * M_PI * (double)(num % den) / (double)den;
      ph[2 * ((size_t)k * n_k + l)] = std::cos(a) / n_k;
      ph[2 * ((size_t)k * n_k + l) + 1] = std::sin(a) / n_k;
    }
  return ph;
}

static gw_status upload_phases(gw_ctx* ctx, void* dst, const std::vector<double>& ph, gw_prec prec, cudaStream_t s) {
  if (is_fp64(prec)) return upload(ctx, dst, ph.data(), sizeof(double) * ph.size(), s);
  std::vector<float> f(ph.begin(), ph.end());
  return upload(ctx, dst, f.data(), sizeof(float) * f.size(), s);
}

template <bool PRODUCT>
static gw_status launch_stripe(gw_ctx* ctx, gw_prec prec, const GridInfo& g, const int* nk, const void* gok,
                               const void* guk, long kstr, const void* dph, int rows, void* out, void* out2, long ldo,
                               cudaStream_t s) {
  const int n_k = nk[0] * nk[1] * nk[2];
  const size_t smem = (size_t)(2 * n_k * 32 + n_k * n_k) * csize(prec);
  const dim3 grd((g.nr + 31) / 32, rows);
  gw_status st;
  auto go = [&](auto kern, auto* tag) -> gw_status {
    using C = std::remove_pointer_t<decltype(tag)>;
    if (smem > 48 * 1024 &&
        (st = cuda_check(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                         "cudaFuncSetAttribute")))
      return st;
    kern<<<grd, 256, smem, s>>>((const C*)gok, (const C*)guk, kstr, g.nr, (const C*)dph, n_k, g.n1, g.n2, g.n3, nk[0],
                                nk[1], nk[2], (C*)out, (C*)out2, ldo);
    return launch_check(ctx, "stripe_chi_kernel");
  };
  if (is_fp64(prec)) return go(stripe_chi_kernel<double, PRODUCT>, (double2*)nullptr);
  return go(stripe_chi_kernel<float, PRODUCT>, (float2*)nullptr);
}

static gw_status launch_q_phase(gw_ctx* ctx, gw_prec prec, const GridInfo& g, const int* nk, void* slab, long ld,
                                int n_chi, double sgn, cudaStream_t s) {
  const int n_k = nk[0] * nk[1] * nk[2];
  const dim3 gq(g.nr, std::min(n_k, 8));
  if (is_fp64(prec))
    q_phase_kernel<double><<<gq, 256, 0, s>>>((double2*)slab, ld, n_chi, g.n1, g.n2, g.n3, nk[0], nk[1], nk[2], sgn);
  else
    q_phase_kernel<float><<<gq, 256, 0, s>>>((float2*)slab, ld, n_chi, g.n1, g.n2, g.n3, nk[0], nk[1], nk[2], sgn);
  return launch_check(ctx, "q_phase_kernel");
}

}  // namespace gw

using namespace gw;

extern "C" gw_status gw_chi0_omega_kmesh(gw_ctx* ctx, const gw_grid* grid, const int* nk, int n_b, int n_occ,
                                         const void* psi_k, const double* eps_k_h, double mu, int n,
                                         const double* tau_h, const double* C_h, int n_chi, const int32_t* gvec_h,
                                         gw_prec prec, int r_block, void* chi_w, void* stream) {
  if (!ctx) return fail(nullptr, GW_ERR_ARG, "ctx is NULL");
  if (!psi_k || !eps_k_h || !tau_h || !C_h || !chi_w) return fail(ctx, GW_ERR_ARG, "NULL pointer");
  if (!valid_prec(prec)) return fail(ctx, GW_ERR_ARG, "bad precision");
  GridInfo g, gs;
  std::vector<int> map, inv, smap, sinv;
  gw_status st = kmesh_grids(ctx, grid, nk, n_chi, gvec_h, &g, &gs, map, inv, smap, sinv);
  if (st) return st;
  const int n_k = nk[0] * nk[1] * nk[2];
  if (n_b < 2 || n_b > g.nr) return fail(ctx, GW_ERR_SHAPE, "need 2 <= n_b <= N_r");
  for (int k = 0; k < n_k; ++k)
    if ((st = check_energies(ctx, eps_k_h + (size_t)k * n_b, n_b, n_occ, mu))) return st;
  if (n < 1 || n > 32) return fail(ctx, GW_ERR_SHAPE, "need 1 <= n <= 32");
  for (int j = 0; j < n; ++j)
    if (!(tau_h[j] > 0)) return fail(ctx, GW_ERR_ARG, "tau must be > 0");
  cudaStream_t s = as_stream(stream);
  const size_t es = csize(prec);
  const int rb = r_block > 0 ? std::min(r_block, g.nr) : std::min(g.nr, 1024);
  const bool tc = prec == GW_F16X3 || prec == GW_BF16X3;
  const bool two_pass = row_two_pass(gs, prec);
  const long ld = (long)n_k * n_chi;                   // slab row: all q blocks
  const size_t slab = (size_t)g.nr * ld;
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
  if ((st = upload_phases(ctx, dph, kl_phases(nk), prec, s))) return st;
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
      if ((st = launch_stripe<true>(ctx, prec, g, nk, gok, guk, kstr, dph, rows, rows_s, nullptr, gs.nr, s)))
        return st;
      if ((st = launch_row_fft(ctx, gs, prec, 1, rows_s, nullptr, gs.nr, slab_j + (size_t)r0 * ld * es, ld, dsmap,
                               n_k * n_chi, rows, 1.0, s, dsinv, tmp_s)))
        return st;
    }
    if ((st = launch_q_phase(ctx, prec, g, nk, slab_j, ld, n_chi, -1.0, s))) return st;
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

// chi0 on a k mesh with G_k in its plane-wave form (Sec. II.B, Eqs. G1_unocc_k,
// G1_occ_k, then Eqs. FFT_G1 and FFT_G2 on the stripe).  With u_ak = exp(-i k.r)
// psi_ak (cell-periodic) and its coefficients over the plane-wave set, the G
// formation of the Gamma-point plane-wave chain gives per k the matrix over the
// set and its column transform T_k(r, g') over the cell grid (Eq. FFT_G1 without
// the Bloch factor).  The stripe row r of the supercell's plane-wave chain is
// then exp(-i k.r) T_k(r, g') / N_k at the (negated) supercell positions k + nk g'
// for every k: the same rows the Gamma-point chain would form for the orbitals
// extended over the supercell, whose plane waves of different k never meet.
// The plane-wave row pass expands both Green's functions over R' (Eq. FFT_G2),
// multiplies them and transforms onto the supercell G set {q + g} (the two
// factors 1/N_k go into its scale); the q phases, column passes and cosine
// transform are those of gw_chi0_omega_kmesh.
extern "C" gw_status gw_chi0_omega_kmesh_pw(gw_ctx* ctx, const gw_grid* grid, const int* nk, int n_b, int n_occ,
                                            const void* psi_k, const double* eps_k_h, double mu, int n,
                                            const double* tau_h, const double* C_h, int n_chi, const int32_t* gvec_h,
                                            int n_pw, const int32_t* pw_index_h, gw_prec prec, void* chi_w,
                                            void* stream) {
  if (!ctx) return fail(nullptr, GW_ERR_ARG, "ctx is NULL");
  if (!psi_k || !eps_k_h || !tau_h || !C_h || !chi_w || !pw_index_h) return fail(ctx, GW_ERR_ARG, "NULL pointer");
  if (!valid_prec(prec)) return fail(ctx, GW_ERR_ARG, "bad precision");
  GridInfo g, gs;
  std::vector<int> map, inv, smap, sinv;
  gw_status st = kmesh_grids(ctx, grid, nk, n_chi, gvec_h, &g, &gs, map, inv, smap, sinv);
  if (st) return st;
  const int n_k = nk[0] * nk[1] * nk[2];
  if (n_b < 2 || n_b > g.nr) return fail(ctx, GW_ERR_SHAPE, "need 2 <= n_b <= N_r");
  for (int k = 0; k < n_k; ++k)
    if ((st = check_energies(ctx, eps_k_h + (size_t)k * n_b, n_b, n_occ, mu))) return st;
  if (n < 1 || n > 32) return fail(ctx, GW_ERR_SHAPE, "need 1 <= n <= 32");
  for (int j = 0; j < n; ++j)
    if (!(tau_h[j] > 0)) return fail(ctx, GW_ERR_ARG, "tau must be > 0");
  std::vector<int> map_pw, inv_pw;
  if ((st = index_maps(ctx, g, pw_index_h, n_pw, map_pw, inv_pw))) return st;
  // supercell positions of the plane waves k + nk g' of every k, negated as on the cell grid;
  // (k, g') -> k + nk g' is one-to-one onto the supercell grid, so no two entries meet
  const int sn[3] = {gs.n1, gs.n2, gs.n3};
  std::vector<int> inv_pws(gs.nr, -1);
  for (int k = 0; k < n_k; ++k) {
    const int kv[3] = {k / (nk[1] * nk[2]), (k / nk[2]) % nk[1], k % nk[2]};
    for (int j = 0; j < n_pw; ++j) {
      const int p = map_pw[j];
      const int pv[3] = {p / (g.n2 * g.n3), (p / g.n3) % g.n2, p % g.n3};
      int pos = 0;
      for (int d = 0; d < 3; ++d) {
        const int m = (kv[d] + nk[d] * pv[d]) % sn[d];
        pos = pos * sn[d] + (sn[d] - m) % sn[d];
      }
      inv_pws[pos] = k * n_pw + j;
    }
  }
  pw_negate(g, map_pw, inv_pw);
  const int n_pws = n_k * n_pw, n_chis = n_k * n_chi;
  if ((st = check_row_pw(ctx, gs, prec, n_pws, n_chis))) return st;
  cudaStream_t s = as_stream(stream);
  const size_t es = csize(prec);
  const bool tc = prec == GW_F16X3 || prec == GW_BF16X3;
  const long ld = (long)n_chis;                        // slab row: all q blocks
  const long ldt = (long)n_pws;                        // T row: all k blocks
  const size_t slab = (size_t)g.nr * ld;
  const GridInfo gp = pw_grid(g, n_pw);
  const bool tmp_needed = row_two_pass(g, prec) && is_fp64(prec);
  Carver probe(nullptr);
  probe.take<int>(g.nr);
  probe.take<int>(gs.nr);
  probe.take<int>(n_pw);
  probe.take<int>(g.nr);
  probe.take<int>(gs.nr);
  probe.take<char>((size_t)n_k * n_b * 8);
  probe.take<char>((size_t)n * n * 8);
  probe.take<double>(2 * (size_t)n_b);
  probe.take<char>(slab * n * es);
  probe.take<char>((size_t)n_b * g.nr * es);
  probe.take<char>((size_t)n_k * n_b * n_pw * es);
  probe.take<char>((size_t)n_pw * n_pw * es);
  probe.take<char>((size_t)n_pw * n_pw * es);
  probe.take<char>((size_t)g.nr * ldt * es);
  probe.take<char>((size_t)g.nr * ldt * es);
  if (tmp_needed) probe.take<char>((size_t)n_b * g.nr * es);
  if (tc) probe.take<char>(tc_scratch_bytes(gp, n_b, n_occ, n_pw, false));
  if ((st = reserve(ctx, probe.off))) return st;
  Carver cv(ctx->arena);
  int* dinv = cv.take<int>(g.nr);
  int* dsinv = cv.take<int>(gs.nr);
  int* dmap_pw = cv.take<int>(n_pw);
  int* dinv_pw = cv.take<int>(g.nr);
  int* dinv_pws = cv.take<int>(gs.nr);
  char* dscale = cv.take<char>((size_t)n_k * n_b * 8);
  char* dcw = cv.take<char>((size_t)n * n * 8);
  double* dnorm = cv.take<double>(2 * (size_t)n_b);
  char* slabs = cv.take<char>(slab * n * es);
  char* u = cv.take<char>((size_t)n_b * g.nr * es);
  char* dc = cv.take<char>((size_t)n_k * n_b * n_pw * es);
  char* mo = cv.take<char>((size_t)n_pw * n_pw * es);
  char* mu_ = cv.take<char>((size_t)n_pw * n_pw * es);
  char* to = cv.take<char>((size_t)g.nr * ldt * es);
  char* tu = cv.take<char>((size_t)g.nr * ldt * es);
  char* tmp = tmp_needed ? cv.take<char>((size_t)n_b * g.nr * es) : nullptr;
  void* tcs = tc ? cv.take<char>(tc_scratch_bytes(gp, n_b, n_occ, n_pw, false)) : nullptr;
  if ((st = upload(ctx, dinv, inv.data(), sizeof(int) * g.nr, s))) return st;
  if ((st = upload(ctx, dsinv, sinv.data(), sizeof(int) * gs.nr, s))) return st;
  if ((st = upload(ctx, dmap_pw, map_pw.data(), sizeof(int) * n_pw, s))) return st;
  if ((st = upload(ctx, dinv_pw, inv_pw.data(), sizeof(int) * g.nr, s))) return st;
  if ((st = upload(ctx, dinv_pws, inv_pws.data(), sizeof(int) * gs.nr, s))) return st;
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
  // the coefficients of u_ak over the set for every k (checked to span every band)
  for (int k = 0; k < n_k; ++k) {
    const int kv[3] = {k / (nk[1] * nk[2]), (k / nk[2]) % nk[1], k % nk[2]};
    const char* pk = static_cast<const char*>(psi_k) + (size_t)k * n_b * g.nr * es;
    const dim3 grd((g.nr + 255) / 256, n_b);
    if (is_fp64(prec))
      bloch_unphase_kernel<double><<<grd, 256, 0, s>>>((const double2*)pk, g.nr, g.n1, g.n2, g.n3, kv[0], kv[1],
                                                       kv[2], nk[0], nk[1], nk[2], (double2*)u);
    else
      bloch_unphase_kernel<float><<<grd, 256, 0, s>>>((const float2*)pk, g.nr, g.n1, g.n2, g.n3, kv[0], kv[1], kv[2],
                                                      nk[0], nk[1], nk[2], (float2*)u);
    if ((st = launch_check(ctx, "bloch_unphase_kernel"))) return st;
    if ((st = pw_coefficients(ctx, g, prec, u, n_b, n_pw, dmap_pw, dinv_pw, dc + (size_t)k * n_b * n_pw * es, dnorm,
                              tmp, s)))
      return st;
  }
  const double row_scale = -2.0 / ((double)n_k * n_k);
  for (int j = 0; j < n; ++j) {
    for (int k = 0; k < n_k; ++k) {
      const GreenScales sc = green_scales(eps_k_h + (size_t)k * n_b, n_b, n_occ, mu, tau_h[j]);
      const char* dck = dc + (size_t)k * n_b * n_pw * es;
      if (tc) {
        st = tc_green_rows(ctx, gp, n_b, n_occ, dck, sc, 0, n_pw, prec, mo, mu_, tcs, true, s);
      } else {
        if ((st = upload_scales(ctx, dscale + (size_t)k * n_b * 8, sc, prec, s))) return st;
        st = green_rows(ctx, gp, n_b, n_occ, dck, dscale + (size_t)k * n_b * 8, sc, 0, n_pw, prec, mo, mu_, s);
      }
      if (st) return st;
      for (int part = 0; part < 2; ++part) {
        const char* m = part ? mu_ : mo;
        char* t = (part ? tu : to) + (size_t)k * n_pw * es;
        if ((st = launch_col_line(ctx, g, prec, +1, 1, m, n_pw, t, ldt, n_pw, dinv_pw, 1.0, s))) return st;
        if ((st = launch_col_plane(ctx, g, prec, +1, t, ldt, n_pw, 1.0, s))) return st;
      }
    }
    // exp(-i k.r) on the block of each k, then per row: expand, multiply, transform onto {q + g}
    if ((st = launch_q_phase(ctx, prec, g, nk, to, ldt, n_pw, -1.0, s))) return st;
    if ((st = launch_q_phase(ctx, prec, g, nk, tu, ldt, n_pw, -1.0, s))) return st;
    char* slab_j = slabs + (size_t)j * slab * es;
    if ((st = launch_row_pw_chi(ctx, gs, prec, tu, to, ldt, slab_j, ld, dinv_pws, n_pws, dsinv, n_chis, g.nr,
                                row_scale, s)))
      return st;
    if ((st = launch_q_phase(ctx, prec, g, nk, slab_j, ld, n_chi, -1.0, s))) return st;
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

// Diagonal self-energy of Bloch states on a k mesh: the space-time route of
// gw_sigma_diag on the supercell stripe.  For tau_j:
//   W~(r, q+g') = exp(+i q.r) sum_g exp(+i g.r) W~_q(g, g', tau_j) for every q
//       (the column passes of Eq. FFTW on each q block, then the factor),
//   per block of cell rows: G_occ / G_unocc on the stripe (k -> L transform of
//       the G_k rows), W~(r, R') by the row transform over the supercell grid
//       from the G set {q + g'}, and the contraction
//   Sigma_unocc_nk(tau) = +dV^2 sum_{r in C} sum_{R' in S} psi*_nk(r) G_unocc(r,R') W~(r,R') psi_nk(R')
//       with psi_nk(r' + L) = exp(i k.L) psi_nk(r') and the 1/Omega_S of Eq. FFTW,
//       likewise occupied with a minus sign.
// Then the same even/odd split, CT + ST and Thiele continuation as at Gamma.
extern "C" gw_status gw_sigma_diag_kmesh(gw_ctx* ctx, const gw_grid* grid, const int* nk, int n_b, int n_occ,
                                         const void* psi_k, const double* eps_k_h, double mu, const int32_t* bk_h,
                                         int n_n, int n, const double* tau_h, const double* omega_h,
                                         const double* C_h, const double* S_h, const void* w_tau, int n_chi,
                                         const int32_t* gvec_h, gw_prec prec, double* sigma_tau_h, double* sigma_iw_h,
                                         const double* w_real_h, int n_real, double* sigma_real_h, void* stream) {
  if (!ctx) return fail(nullptr, GW_ERR_ARG, "ctx is NULL");
  if (!psi_k || !eps_k_h || !bk_h || !tau_h || !omega_h || !C_h || !S_h || !w_tau || !sigma_iw_h)
    return fail(ctx, GW_ERR_ARG, "NULL pointer");
  if (!valid_prec(prec)) return fail(ctx, GW_ERR_ARG, "bad precision");
  if (reinterpret_cast<uintptr_t>(psi_k) % 16) return fail(ctx, GW_ERR_ARG, "psi_k must be 16-byte aligned");
  GridInfo g, gs;
  std::vector<int> map, inv, smap, sinv;
  gw_status st = kmesh_grids(ctx, grid, nk, n_chi, gvec_h, &g, &gs, map, inv, smap, sinv);
  if (st) return st;
  const int n_k = nk[0] * nk[1] * nk[2];
  if (n_b < 2 || n_b > g.nr) return fail(ctx, GW_ERR_SHAPE, "need 2 <= n_b <= N_r");
  for (int k = 0; k < n_k; ++k)
    if ((st = check_energies(ctx, eps_k_h + (size_t)k * n_b, n_b, n_occ, mu))) return st;
  if (n < 1 || n > 32) return fail(ctx, GW_ERR_SHAPE, "need 1 <= n <= 32");
  if (n_n < 1 || n_n > 1024) return fail(ctx, GW_ERR_SHAPE, "need 1 <= n_n <= 1024");
  if (n_real < 0 || (n_real > 0 && (!w_real_h || !sigma_real_h))) return fail(ctx, GW_ERR_ARG, "bad real-axis request");
  for (int i = 0; i < n_n; ++i)
    if (bk_h[2 * i] < 0 || bk_h[2 * i] >= n_b || bk_h[2 * i + 1] < 0 || bk_h[2 * i + 1] >= n_k)
      return fail(ctx, GW_ERR_ARG, "(band, k) pair out of range");
  for (int j = 0; j < n; ++j)
    if (!(tau_h[j] > 0)) return fail(ctx, GW_ERR_ARG, "tau must be > 0");
  cudaStream_t s = as_stream(stream);
  const size_t es = csize(prec);
  const int rb = std::min(g.nr, 1024);
  const bool tc = prec == GW_F16X3 || prec == GW_BF16X3;
  const long ld = (long)n_k * n_chi;
  const int nreal1 = std::max(n_real, 1);
  Carver probe(nullptr);
  probe.take<int>(n_chi);
  probe.take<int>(g.nr);
  probe.take<int>((size_t)n_k * n_chi);
  probe.take<int>(gs.nr);
  probe.take<int>(3 * (size_t)n_n);
  probe.take<double>((size_t)n_k * n_b);
  probe.take<double2>((size_t)n_k * n_k);
  probe.take<double>(2 * (size_t)n * n + n + nreal1);
  probe.take<double>(2 * (size_t)n_n * n);
  probe.take<double2>((size_t)n_n * (n + nreal1));
  probe.take<int>(n_n);
  probe.take<char>((size_t)g.nr * ld * es);
  probe.take<char>((size_t)n_k * rb * g.nr * es);
  probe.take<char>((size_t)n_k * rb * g.nr * es);
  probe.take<char>(3 * (size_t)rb * gs.nr * es);
  probe.take<char>((size_t)n_n * (gs.nr + g.nr) * es);
  if (tc) probe.take<char>(tc_scratch_bytes(g, n_b, n_occ, rb, false));
  if ((st = reserve(ctx, probe.off))) return st;
  Carver cv(ctx->arena);
  int* dmap = cv.take<int>(n_chi);
  int* dinv = cv.take<int>(g.nr);
  int* dsmap = cv.take<int>((size_t)n_k * n_chi);
  int* dsinv = cv.take<int>(gs.nr);
  int* dbk = cv.take<int>(3 * (size_t)n_n);           // (band, k) pairs, then 0 .. n_n-1
  int* dbid = dbk + 2 * n_n;
  char* dscale = cv.take<char>((size_t)n_k * n_b * 8);
  char* dph = cv.take<char>((size_t)n_k * n_k * 16);
  double* tab = cv.take<double>(2 * (size_t)n * n + n + nreal1);
  double* acc = cv.take<double>(2 * (size_t)n_n * n);
  double2* out = cv.take<double2>((size_t)n_n * (n + nreal1));
  int* dstat = cv.take<int>(n_n);
  char* wrg = cv.take<char>((size_t)g.nr * ld * es);
  char* gok = cv.take<char>((size_t)n_k * rb * g.nr * es);
  char* guk = cv.take<char>((size_t)n_k * rb * g.nr * es);
  char* go_s = cv.take<char>(3 * (size_t)rb * gs.nr * es);   // G_occ, G_unocc and W~ stripes of a block
  char* gu_s = go_s + (size_t)rb * gs.nr * es;
  char* w_s = gu_s + (size_t)rb * gs.nr * es;
  char* ext = cv.take<char>((size_t)n_n * (gs.nr + g.nr) * es);
  char* prow = ext + (size_t)n_n * gs.nr * es;
  void* tcs = tc ? cv.take<char>(tc_scratch_bytes(g, n_b, n_occ, rb, false)) : nullptr;
  if ((st = upload(ctx, dmap, map.data(), sizeof(int) * n_chi, s))) return st;
  if ((st = upload(ctx, dinv, inv.data(), sizeof(int) * g.nr, s))) return st;
  if ((st = upload(ctx, dsmap, smap.data(), sizeof(int) * n_k * n_chi, s))) return st;
  if ((st = upload(ctx, dsinv, sinv.data(), sizeof(int) * gs.nr, s))) return st;
  std::vector<int> bk(3 * (size_t)n_n);
  for (int i = 0; i < 2 * n_n; ++i) bk[i] = bk_h[i];
  for (int i = 0; i < n_n; ++i) bk[2 * n_n + i] = i;
  if ((st = upload(ctx, dbk, bk.data(), sizeof(int) * 3 * n_n, s))) return st;
  if ((st = upload_phases(ctx, dph, kl_phases(nk), prec, s))) return st;
  if ((st = upload(ctx, tab, C_h, sizeof(double) * n * n, s))) return st;
  if ((st = upload(ctx, tab + (size_t)n * n, S_h, sizeof(double) * n * n, s))) return st;
  if ((st = upload(ctx, tab + 2 * (size_t)n * n, omega_h, sizeof(double) * n, s))) return st;
  if (n_real > 0 && (st = upload(ctx, tab + 2 * (size_t)n * n + n, w_real_h, sizeof(double) * n_real, s))) return st;
  if ((st = cuda_check(ctx, cudaMemsetAsync(acc, 0, sizeof(double) * 2 * n_n * n, s), "memset"))) return st;
  // the requested orbitals over the supercell (Bloch phase) and on the cell
  {
    const dim3 grd((g.nr + 255) / 256, n_k, n_n);
    if (is_fp64(prec))
      bloch_extend_kernel<double><<<grd, 256, 0, s>>>((const double2*)psi_k, (long)n_b * g.nr, g.nr, dbk, g.n1, g.n2,
                                                      g.n3, nk[0], nk[1], nk[2], (double2*)ext, (double2*)prow);
    else
      bloch_extend_kernel<float><<<grd, 256, 0, s>>>((const float2*)psi_k, (long)n_b * g.nr, g.nr, dbk, g.n1, g.n2,
                                                     g.n3, nk[0], nk[1], nk[2], (float2*)ext, (float2*)prow);
    if ((st = launch_check(ctx, "bloch_extend_kernel"))) return st;
  }
  double* acc_u = acc;
  double* acc_o = acc + (size_t)n_n * n;
  const double coef = g.dv * g.dv / (g.volume * n_k);   // dV^2 and the 1/Omega_S of Eq. FFTW
  const long kstr = (long)rb * g.nr;
  for (int j = 0; j < n; ++j) {
    std::vector<GreenScales> scales(n_k);
    for (int k = 0; k < n_k; ++k) {
      scales[k] = green_scales(eps_k_h + (size_t)k * n_b, n_b, n_occ, mu, tau_h[j]);
      if (!tc && (st = upload_scales(ctx, dscale + (size_t)k * n_b * 8, scales[k], prec, s))) return st;
    }
    for (int q = 0; q < n_k; ++q) {
      const char* wq = static_cast<const char*>(w_tau) + ((size_t)q * n + j) * n_chi * n_chi * es;
      char* blk = wrg + (size_t)q * n_chi * es;
      if ((st = launch_col_line(ctx, g, prec, +1, 1, wq, n_chi, blk, ld, n_chi, dinv, 1.0, s))) return st;
      if ((st = launch_col_plane(ctx, g, prec, +1, blk, ld, n_chi, 1.0, s))) return st;
    }
    if ((st = launch_q_phase(ctx, prec, g, nk, wrg, ld, n_chi, +1.0, s))) return st;
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
      if ((st = launch_stripe<false>(ctx, prec, g, nk, gok, guk, kstr, dph, rows, go_s, gu_s, gs.nr, s))) return st;
      if ((st = launch_row_fft(ctx, gs, prec, 2, wrg + (size_t)r0 * ld * es, nullptr, ld, w_s, gs.nr, dsmap,
                               n_k * n_chi, rows, 1.0, s, dsinv)))
        return st;
      if ((st = launch_sigma_contract(ctx, prec, w_s, go_s, gu_s, gs.nr, gs.nr, rows, ext, dbid, n_n, r0, coef,
                                      acc_u + j, acc_o + j, n, s, prow, g.nr)))
        return st;
    }
  }
  if (tc && (st = tc_check(ctx, tcs, s))) return st;
  std::vector<int32_t> labels(n_n);
  for (int i = 0; i < n_n; ++i) labels[i] = bk_h[2 * i];
  return sigma_finish(ctx, acc, n_n, n, tab, n_real, out, dstat, labels.data(), sigma_tau_h, sigma_iw_h, sigma_real_h,
                      s);
}
