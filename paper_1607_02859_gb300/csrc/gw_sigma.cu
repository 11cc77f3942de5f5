// Diagonal correlation self-energy (Sec. II.D and II.E.1).
//
// For each tau_j:
//   W~(G,G',tau_j) -> W~(r,G')  (i1 pass gathering the G rows, then (i2,i3)
//                                planes; first step of Eq. FFTW)
//   per r-block: G_occ / G_unocc rows recomputed (Eqs. Green_occ/unocc), and
//   one CTA per row r forms W~(r,R') in shared memory (second step of Eq. FFTW)
//   and contracts (first term of Eq. Sigma_occ_reduce)
//      V_n(r) = sum_R' G(r,R') W~(r,R') psi_n(R'),
//      Sigma_nn += -/+ dV^2 Re( psi_n^*(r) V_n(r) )
//   with FP64 atomics into Sigma_unocc_nn(tau_j), Sigma_occ_nn(-tau_j).
// Then one FP64 thread per band: even/odd split (Eqs.
// cos_sin_sigma_matrix1/2), CT + ST (Eqs. sigma_r_w, cos_sin_sigma1/2) and the
// Thiele continued fraction (Eqs. pade1, pade2).
#include <cmath>
#include <cstring>

#include "gw_fft.cuh"
#include "gw_kernels.h"
#include "gw_tc.h"

namespace gw {

constexpr int kSigBands = 8;   // bands accumulated per pass over a row

constexpr int kSigThreads = 512;   // one CTA per row; its W~ row (up to 115 KB) leaves room for one CTA per SM

// Two consecutive complex elements (16-byte aligned) in one 16-byte load for FP32.
__device__ __forceinline__ void ld_pair(const float2* p, float2& a, float2& b) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void ld_pair(const double2* p, double2& a, double2& b) {
  a = __ldg(p);
  b = __ldg(p + 1);
}

// One row r per CTA: W~(r,G') is scattered into the FFT grid in shared memory
// and transformed to W~(r,R'); then, streaming G_occ(r,.), G_unocc(r,.) and
// psi_n(.) two R' at a time (16-byte loads, two pairs in flight per thread),
// V_n = sum_R' G(r,R') W~(r,R') psi_n(R') for kSigBands bands per pass.
template <typename T, int N1, int N2, int N3>
__global__ void __launch_bounds__(kSigThreads) sigma_row_kernel(
    const typename cpx<T>::t* __restrict__ wrg, long ldw, const int* __restrict__ map, int n_chi,
    const typename cpx<T>::t* __restrict__ go, const typename cpx<T>::t* __restrict__ gu, long ldg,
    const typename cpx<T>::t* __restrict__ psi, const int* __restrict__ bands, int n_n, int r0, double coef,
    double* __restrict__ acc_u, double* __restrict__ acc_o, int acc_stride) {
  using C = typename cpx<T>::t;
  using L = RowLayout<N1, N2, N3>;
  static_assert(N3 % 2 == 0 && L::NR % 2 == 0, "pairs along i3");
  constexpr int NW = kSigThreads / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  __shared__ T red[NW][kSigBands * 4];
  const long row = blockIdx.x;
  const int r = r0 + (int)row;
  for (int e = threadIdx.x; e < L::TOT; e += blockDim.x) s[e] = mk(T(0), T(0));
  __syncthreads();
  const C* src = wrg + (long)r * ldw;
  for (int j0 = threadIdx.x; j0 < n_chi; j0 += 4 * kSigThreads) {
    C v[4];
    int m[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = j0 + u * kSigThreads;
      if (j < n_chi) {
        v[u] = src[j];
        m[u] = map[j];
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (j0 + u * kSigThreads < n_chi) s[L::pos(m[u])] = v[u];
  }
  __syncthreads();
  fft3_smem<N1, N2, N3, -1>(s);
  const C* pgo = go + row * ldg;
  const C* pgu = gu + row * ldg;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NP = L::NR / 2;
  for (int b0 = 0; b0 < n_n; b0 += kSigBands) {
    const int nb = min(kSigBands, n_n - b0);
    const C* pb[kSigBands];
#pragma unroll
    for (int b = 0; b < kSigBands; ++b) pb[b] = psi + (long)bands[b0 + (b < nb ? b : 0)] * L::NR;
    T vo[kSigBands][2], vu[kSigBands][2];
#pragma unroll
    for (int b = 0; b < kSigBands; ++b) vo[b][0] = vo[b][1] = vu[b][0] = vu[b][1] = T(0);
    for (int q0 = threadIdx.x; q0 < NP; q0 += 2 * kSigThreads) {
      C xo[2][2], xu[2][2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int q = q0 + u * kSigThreads;
        if (q < NP) {
          ld_pair(pgo + 2 * q, xo[u][0], xo[u][1]);
          ld_pair(pgu + 2 * q, xu[u][0], xu[u][1]);
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int q = q0 + u * kSigThreads;
        if (q >= NP) continue;
        const int p0 = L::pos(2 * q);            // 2q and 2q+1 share an i3 pencil
        const C w0 = s[p0], w1 = s[p0 + 1];
        const C ho0 = cmul(xo[u][0], w0), ho1 = cmul(xo[u][1], w1);
        const C hu0 = cmul(xu[u][0], w0), hu1 = cmul(xu[u][1], w1);
#pragma unroll
        for (int b = 0; b < kSigBands; ++b) {
          if (b < nb) {
            C a0, a1;
            ld_pair(pb[b] + 2 * q, a0, a1);
            vo[b][0] += ho0.x * a0.x - ho0.y * a0.y + ho1.x * a1.x - ho1.y * a1.y;
            vo[b][1] += ho0.x * a0.y + ho0.y * a0.x + ho1.x * a1.y + ho1.y * a1.x;
            vu[b][0] += hu0.x * a0.x - hu0.y * a0.y + hu1.x * a1.x - hu1.y * a1.y;
            vu[b][1] += hu0.x * a0.y + hu0.y * a0.x + hu1.x * a1.y + hu1.y * a1.x;
          }
        }
      }
    }
#pragma unroll
    for (int b = 0; b < kSigBands; ++b)
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          vo[b][q] += __shfl_xor_sync(0xffffffffu, vo[b][q], off);
          vu[b][q] += __shfl_xor_sync(0xffffffffu, vu[b][q], off);
        }
    if (lane == 0)
#pragma unroll
      for (int b = 0; b < kSigBands; ++b) {
        red[warp][4 * b + 0] = vo[b][0];
        red[warp][4 * b + 1] = vo[b][1];
        red[warp][4 * b + 2] = vu[b][0];
        red[warp][4 * b + 3] = vu[b][1];
      }
    __syncthreads();
    if (threadIdx.x < nb) {
      const int b = threadIdx.x;
      double o_re = 0, o_im = 0, u_re = 0, u_im = 0;
      for (int w = 0; w < NW; ++w) {
        o_re += red[w][4 * b + 0];
        o_im += red[w][4 * b + 1];
        u_re += red[w][4 * b + 2];
        u_im += red[w][4 * b + 3];
      }
      const C pn = psi[(long)bands[b0 + b] * L::NR + r];
      // Re(conj(pn) * V)
      const double so = -coef * ((double)pn.x * o_re + (double)pn.y * o_im);
      const double su = coef * ((double)pn.x * u_re + (double)pn.y * u_im);
      atomicAdd(acc_o + (long)(b0 + b) * acc_stride, so);
      atomicAdd(acc_u + (long)(b0 + b) * acc_stride, su);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
  // a / b with the larger component of b factored out (Smith's method)
  if (fabs(b.x) >= fabs(b.y)) {
    const double r = b.y / b.x, d = b.x + b.y * r;
    return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  }
  const double r = b.x / b.y, d = b.x * r + b.y;
  return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
}
__device__ __forceinline__ double zabs2(double2 a) { return a.x * a.x + a.y * a.y; }

constexpr int kMaxN = 32;

__global__ void sigma_finish_kernel(const double* __restrict__ acc_u, const double* __restrict__ acc_o, int n_n, int n,
                                    const double* __restrict__ Cm, const double* __restrict__ Sm,
                                    const double* __restrict__ omega, const double* __restrict__ wreal, int n_real,
                                    double2* __restrict__ out_iw, double2* __restrict__ out_real,
                                    int* __restrict__ status) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_n) return;
  double2 f[kMaxN], g[kMaxN], a[kMaxN], z[kMaxN];
  for (int k = 0; k < n; ++k) {
    double re = 0, im = 0;
    for (int j = 0; j < n; ++j) {
      const double sc = 0.5 * (acc_u[b * n + j] + acc_o[b * n + j]);
      const double ss = 0.5 * (acc_u[b * n + j] - acc_o[b * n + j]);
      re += Cm[k * n + j] * sc;
      im += Sm[k * n + j] * ss;
    }
    f[k] = make_double2(re, im);
    out_iw[b * n + k] = f[k];
    z[k] = make_double2(0.0, omega[k]);
    g[k] = f[k];
  }
  int bad = 0;
  a[0] = g[0];
  for (int p = 1; p < n && !bad; ++p) {
    const double2 prev = g[p - 1];
    for (int m = p; m < n; ++m) {
      const double2 dz = make_double2(z[m].x - z[p - 1].x, z[m].y - z[p - 1].y);
      const double2 den = make_double2(dz.x * g[m].x - dz.y * g[m].y, dz.x * g[m].y + dz.y * g[m].x);
      if (!(sqrt(zabs2(den)) >= 1e-300)) {
        bad = 1;
        break;
      }
      g[m] = zdiv(make_double2(prev.x - g[m].x, prev.y - g[m].y), den);
    }
    a[p] = g[p];
  }
  for (int q = 0; q < n_real; ++q) {
    double2 res = make_double2(NAN, NAN);
    if (!bad) {
      const double2 x = make_double2(wreal[q], 0.0);
      double2 t = make_double2(1.0, 0.0);
      for (int p = n - 1; p >= 1 && !bad; --p) {
        if (!(sqrt(zabs2(t)) >= 1e-300)) { bad = 1; break; }
        const double2 dx = make_double2(x.x - z[p - 1].x, x.y - z[p - 1].y);
        const double2 num = make_double2(a[p].x * dx.x - a[p].y * dx.y, a[p].x * dx.y + a[p].y * dx.x);
        const double2 qv = zdiv(num, t);
        t = make_double2(1.0 + qv.x, qv.y);
      }
      if (!bad && sqrt(zabs2(t)) >= 1e-300) res = zdiv(a[0], t);
      else bad = 1;
    }
    if (out_real) out_real[b * n_real + q] = res;
  }
  status[b] = bad;
}

template <typename T, int N1, int N2, int N3>
struct SigmaOps {
  static gw_status row(gw_ctx* ctx, const void* wrg, long ldw, const int* map, int n_chi, const void* go,
                       const void* gu, long ldg, const void* psi, const int* bands, int n_n, int r0, int n_rows,
                       double coef, double* acc_u, double* acc_o, int acc_stride, cudaStream_t st) {
    using C = typename cpx<T>::t;
    const size_t bytes = RowLayout<N1, N2, N3>::TOT * sizeof(C);
    auto kernel = sigma_row_kernel<T, N1, N2, N3>;
    if (bytes > 200 * 1024) return fail(ctx, GW_ERR_UNSUPPORTED, "grid row too large for shared memory");
    if (bytes > 48 * 1024) {
      gw_status rc = cuda_check(ctx, cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes),
                                "cudaFuncSetAttribute");
      if (rc) return rc;
    }
    KTimer kt(ctx, KF_SIGMA_ROW, (double)n_rows * (n_chi + 2.0 * RowLayout<N1, N2, N3>::NR) * sizeof(C), st);
    kernel<<<n_rows, kSigThreads, bytes, st>>>((const C*)wrg, ldw, map, n_chi, (const C*)go, (const C*)gu, ldg,
                                       (const C*)psi, bands, n_n, r0, coef, acc_u, acc_o, acc_stride);
    return launch_check(ctx, "sigma_row_kernel");
  }
};

static gw_status launch_sigma_rows(gw_ctx* ctx, const GridInfo& g, gw_prec prec, const void* wrg, long ldw,
                                   const int* map, int n_chi, const void* go, const void* gu, long ldg,
                                   const void* psi, const int* bands, int n_n, int r0, int n_rows, double coef,
                                   double* acc_u, double* acc_o, int acc_stride, cudaStream_t st) {
#define X(a, b, c)                                                                                               \
  if (g.n1 == a && g.n2 == b && g.n3 == c)                                                                       \
    return is_fp64(prec) ? SigmaOps<double, a, b, c>::row(ctx, wrg, ldw, map, n_chi, go, gu, ldg, psi, bands,   \
                                                          n_n, r0, n_rows, coef, acc_u, acc_o, acc_stride, st) \
                         : SigmaOps<float, a, b, c>::row(ctx, wrg, ldw, map, n_chi, go, gu, ldg, psi, bands,    \
                                                         n_n, r0, n_rows, coef, acc_u, acc_o, acc_stride, st);
  GW_GRIDS(X)
#undef X
  return fail(ctx, GW_ERR_UNSUPPORTED, "no kernels compiled for this grid");
}

size_t sigma_scratch(const GridInfo& g, int n_b, int n_occ, int n, int n_chi, int n_n, int n_real, gw_prec prec) {
  const size_t es = csize(prec);
  const int rb = std::min(g.nr, 2048);
  Carver probe(nullptr);
  probe.take<int>(n_chi);
  probe.take<int>(g.nr);
  probe.take<int>(n_n);
  probe.take<double>((size_t)n * n_b);
  probe.take<double>(4 * (size_t)n * n + 2 * n + std::max(n_real, 1));
  probe.take<double>(2 * (size_t)n_n * n);
  probe.take<double2>((size_t)n_n * n + (size_t)n_n * std::max(n_real, 1));
  probe.take<int>(n_n);
  probe.take<char>((size_t)g.nr * n_chi * es);
  probe.take<char>((size_t)rb * g.nr * es);
  probe.take<char>((size_t)rb * g.nr * es);
  if (prec == GW_F16X3 || prec == GW_BF16X3) probe.take<char>(tc_scratch_bytes(g, n_b, n_occ, rb, false));
  return probe.off;
}

}  // namespace gw

using namespace gw;

extern "C" gw_status gw_sigma_diag(gw_ctx* ctx, const gw_grid* grid, int n_b, int n_occ, const void* psi,
                                   const double* eps_h, double mu, const int32_t* bands_h, int n_n, int n,
                                   const double* tau_h, const double* omega_h, const double* C_h, const double* S_h,
                                   const void* w_tau, int n_chi, const int32_t* fft_index_h, gw_prec prec,
                                   double* sigma_tau_h, double* sigma_iw_h, const double* w_real_h, int n_real,
                                   double* sigma_real_h, void* stream) {
  if (!ctx) return fail(nullptr, GW_ERR_ARG, "ctx is NULL");
  GridInfo g;
  gw_status st = grid_info(ctx, grid, &g);
  if (st) return st;
  if (!grid_supported(g.n1, g.n2, g.n3)) return fail(ctx, GW_ERR_UNSUPPORTED, "no kernels compiled for this grid");
  if (!valid_prec(prec)) return fail(ctx, GW_ERR_ARG, "bad precision");
  if (!psi || !w_tau || !bands_h || !tau_h || !omega_h || !C_h || !S_h || !sigma_iw_h)
    return fail(ctx, GW_ERR_ARG, "NULL pointer");
  if (n_b < 2 || n_b > g.nr) return fail(ctx, GW_ERR_SHAPE, "need 2 <= n_b <= N_r");
  if (reinterpret_cast<uintptr_t>(psi) % 16) return fail(ctx, GW_ERR_ARG, "psi must be 16-byte aligned");
  if ((st = check_energies(ctx, eps_h, n_b, n_occ, mu))) return st;
  if (n < 1 || n > kMaxN) return fail(ctx, GW_ERR_SHAPE, "need 1 <= n <= 32");
  if (n_n < 1 || n_n > 1024) return fail(ctx, GW_ERR_SHAPE, "need 1 <= n_n <= 1024");
  if (n_real < 0 || (n_real > 0 && (!w_real_h || !sigma_real_h))) return fail(ctx, GW_ERR_ARG, "bad real-axis request");
  for (int b = 0; b < n_n; ++b)
    if (bands_h[b] < 0 || bands_h[b] >= n_b) return fail(ctx, GW_ERR_ARG, "band index out of range");
  for (int j = 0; j < n; ++j)
    if (!(tau_h[j] > 0)) return fail(ctx, GW_ERR_ARG, "tau must be > 0");
  std::vector<int> map, inv;
  if ((st = index_maps(ctx, g, fft_index_h, n_chi, map, inv))) return st;
  cudaStream_t s = as_stream(stream);
  const size_t es = csize(prec);
  const int rb = std::min(g.nr, 2048);
  const bool tc = prec == GW_F16X3 || prec == GW_BF16X3;
  if ((st = reserve(ctx, sigma_scratch(g, n_b, n_occ, n, n_chi, n_n, n_real, prec)))) return st;
  Carver cv(ctx->arena);
  int* dmap = cv.take<int>(n_chi);
  int* dinv = cv.take<int>(g.nr);
  int* dbands = cv.take<int>(n_n);
  char* dscale = cv.take<char>((size_t)n * n_b * 8);
  double* dC = cv.take<double>(4 * (size_t)n * n + 2 * n + std::max(n_real, 1));
  double* dS = dC + (size_t)n * n;
  double* dom = dS + (size_t)n * n;
  double* dwr = dom + n;
  double* acc = cv.take<double>(2 * (size_t)n_n * n);
  double2* out_iw = cv.take<double2>((size_t)n_n * n + (size_t)n_n * std::max(n_real, 1));
  double2* out_re = out_iw + (size_t)n_n * n;
  int* dstat = cv.take<int>(n_n);
  char* wrg = cv.take<char>((size_t)g.nr * n_chi * es);
  char* gob = cv.take<char>((size_t)rb * g.nr * es);
  char* gub = cv.take<char>((size_t)rb * g.nr * es);
  void* tcs = tc ? cv.take<char>(tc_scratch_bytes(g, n_b, n_occ, rb, false)) : nullptr;
  if ((st = upload(ctx, dmap, map.data(), sizeof(int) * n_chi, s))) return st;
  if ((st = upload(ctx, dinv, inv.data(), sizeof(int) * g.nr, s))) return st;
  std::vector<int> bv(bands_h, bands_h + n_n);
  if ((st = upload(ctx, dbands, bv.data(), sizeof(int) * n_n, s))) return st;
  std::vector<GreenScales> scales(n);
  for (int j = 0; j < n; ++j) {
    scales[j] = green_scales(eps_h, n_b, n_occ, mu, tau_h[j]);
    if ((st = upload_scales(ctx, dscale + (size_t)j * n_b * 8, scales[j], prec, s))) return st;
  }
  if ((st = upload(ctx, dC, C_h, sizeof(double) * n * n, s))) return st;
  if ((st = upload(ctx, dS, S_h, sizeof(double) * n * n, s))) return st;
  if ((st = upload(ctx, dom, omega_h, sizeof(double) * n, s))) return st;
  if (n_real > 0 && (st = upload(ctx, dwr, w_real_h, sizeof(double) * n_real, s))) return st;
  if ((st = cuda_check(ctx, cudaMemsetAsync(acc, 0, sizeof(double) * 2 * n_n * n, s), "memset"))) return st;
  double* acc_u = acc;
  double* acc_o = acc + (size_t)n_n * n;
  const double coef = g.dv * g.dv / g.volume;   // dV^2 and the 1/Omega of Eq. FFTW
  bool first = true;
  for (int j = 0; j < n; ++j) {
    const char* wj = static_cast<const char*>(w_tau) + (size_t)j * n_chi * n_chi * es;
    if ((st = launch_col_line(ctx, g, prec, +1, 1, wj, n_chi, wrg, n_chi, n_chi, dinv, 1.0, s))) return st;
    if ((st = launch_col_plane(ctx, g, prec, +1, wrg, n_chi, n_chi, 1.0, s))) return st;
    for (int r0 = 0; r0 < g.nr; r0 += rb) {
      const int rows = std::min(rb, g.nr - r0);
      if (tc) {
        st = tc_green_rows(ctx, g, n_b, n_occ, psi, scales[j], r0, rows, prec, gob, gub, tcs, first, s);
        first = false;
      }
      else st = green_rows(ctx, g, n_b, n_occ, psi, dscale + (size_t)j * n_b * 8, scales[j], r0, rows, prec, gob, gub, s);
      if (st) return st;
      if ((st = launch_sigma_rows(ctx, g, prec, wrg, n_chi, dmap, n_chi, gob, gub, g.nr, psi, dbands, n_n, r0, rows,
                                  coef, acc_u + j, acc_o + j, n, s)))
        return st;
    }
  }
  if (tc && (st = tc_check(ctx, tcs, s))) return st;
  sigma_finish_kernel<<<(n_n + 63) / 64, 64, 0, s>>>(acc_u, acc_o, n_n, n, dC, dS, dom, dwr, n_real, out_iw,
                                                      n_real > 0 ? out_re : nullptr, dstat);
  if ((st = launch_check(ctx, "sigma_finish_kernel"))) return st;
  std::vector<double2> h_iw((size_t)n_n * n), h_re((size_t)n_n * std::max(n_real, 1));
  std::vector<int> h_stat(n_n);
  std::vector<double> h_acc(2 * (size_t)n_n * n);
  cudaMemcpyAsync(h_iw.data(), out_iw, sizeof(double2) * n_n * n, cudaMemcpyDeviceToHost, s);
  if (n_real > 0) cudaMemcpyAsync(h_re.data(), out_re, sizeof(double2) * n_n * n_real, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(h_stat.data(), dstat, sizeof(int) * n_n, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(h_acc.data(), acc, sizeof(double) * 2 * n_n * n, cudaMemcpyDeviceToHost, s);
  if ((st = cuda_check(ctx, cudaStreamSynchronize(s), "sigma sync"))) return st;
  std::memcpy(sigma_iw_h, h_iw.data(), sizeof(double2) * n_n * n);
  if (n_real > 0) std::memcpy(sigma_real_h, h_re.data(), sizeof(double2) * n_n * n_real);
  if (sigma_tau_h) std::memcpy(sigma_tau_h, h_acc.data(), sizeof(double) * 2 * n_n * n);
  for (int b = 0; b < n_n; ++b)
    if (h_stat[b]) return fail(ctx, GW_ERR_NUMERIC, "Thiele continuation broke down for band " + std::to_string(bands_h[b]));
  return GW_OK;
}
