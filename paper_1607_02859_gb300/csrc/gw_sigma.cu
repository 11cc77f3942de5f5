// Diagonal correlation self-energy (Sec. II.D and II.E.1).
//
// For each tau_j:
//   W~(G,G',tau_j) -> W~(r,G')  (i1 pass gathering the G rows, then (i2,i3)
//                                planes; first step of Eq. FFTW)
//   per r-block: G_occ / G_unocc rows recomputed (Eqs. Green_occ/unocc),
//   W~(r,R') by the row transform (second step of Eq. FFTW), and the
//   contraction (first term of Eq. Sigma_occ_reduce)
//      V_n(r) = sum_R' G(r,R') W~(r,R') psi_n(R'),
//      Sigma_nn += -/+ dV^2 Re( psi_n^*(r) V_n(r) )
//   with FP64 atomics into Sigma_unocc_nn(tau_j), Sigma_occ_nn(-tau_j).
// Then one FP64 thread per band: even/odd split (Eqs.
// cos_sin_sigma_matrix1/2), CT + ST (Eqs. sigma_r_w, cos_sin_sigma1/2) and the
// Thiele continued fraction (Eqs. pade1, pade2).
#include <cmath>
#include <cstring>
#include <type_traits>

#include "gw_fft.cuh"
#include "gw_kernels.h"
#include "gw_tc.h"

namespace gw {

constexpr int kSigBands = 8;   // bands accumulated per pass over a row

// Sigma contraction for a block of rows r (first term of Eq. Sigma_occ_reduce):
//   V_n(r) = sum_R' G(r,R') W~(r,R') psi_n(R')   for G_occ and G_unocc,
//   Sigma_occ_nn += -coef Re(conj(psi_n(r)) V_n^occ),  Sigma_unocc_nn += coef Re(...)
// with W~(r,R') already in real space.  One row per warp, kSigRows rows per
// CTA; R' runs in chunks whose psi_n values are copied asynchronously
// (cp.async, double-buffered) into shared memory once for all the CTA's rows.
// Lanes take pairs of consecutive R' (16-byte loads), four pairs of each of the
// three streams in flight.
constexpr int kSigRows = 8;
constexpr int kSigThreads = 32 * kSigRows;
constexpr int kSigUnroll = 4;

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

template <typename T>
__global__ void __launch_bounds__(kSigThreads) sigma_contract_kernel(
    const typename cpx<T>::t* __restrict__ wrr, const typename cpx<T>::t* __restrict__ go,
    const typename cpx<T>::t* __restrict__ gu, long ld, int nr, int rows,
    const typename cpx<T>::t* __restrict__ psi, const int* __restrict__ bands, int n_n, int r0, double coef,
    double* __restrict__ acc_u, double* __restrict__ acc_o, int acc_stride,
    const typename cpx<T>::t* __restrict__ psi_row, long ld_row) {
  using C = typename cpx<T>::t;
  constexpr int CHUNK = sizeof(T) == 4 ? 512 : 256;          // R' per chunk: 32 KB of psi per buffer
  constexpr int PAIRS = CHUNK / 2;
  constexpr int EPP = sizeof(C) == 8 ? 2 : 1;                 // elements per 16-byte copy
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sp = reinterpret_cast<C*>(smem_raw);                      // [2][kSigBands][CHUNK]
  __shared__ double red[kSigRows][kSigBands][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rl = warp, r = blockIdx.x * kSigRows + rl;
  const bool active = r < rows;
  const long off = (long)r * ld;
  const int nchunks = (nr + CHUNK - 1) / CHUNK;
  for (int b0 = 0; b0 < n_n; b0 += kSigBands) {
    const int nb = min(kSigBands, n_n - b0);
    auto stage = [&](int buf, int k0) {
      const int kn = min(CHUNK, nr - k0);
      C* dst = sp + buf * kSigBands * CHUNK;
      for (int e = threadIdx.x; e < kSigBands * CHUNK / EPP; e += kSigThreads) {
        const int b = e / (CHUNK / EPP), k = (e - b * (CHUNK / EPP)) * EPP;
        const bool ok = b < nb && k < kn;
        cp_async16(dst + b * CHUNK + k, ok ? psi + (long)bands[b0 + b] * nr + k0 + k : psi, ok);
      }
    };
    T vo[kSigBands][2], vu[kSigBands][2];
#pragma unroll
    for (int b = 0; b < kSigBands; ++b) vo[b][0] = vo[b][1] = vu[b][0] = vu[b][1] = T(0);
    __syncthreads();                       // the previous band pass is done with both buffers
    stage(0, 0);
    cp_async_commit();
    for (int c = 0; c < nchunks; ++c) {
      if (c + 1 < nchunks) stage((c + 1) & 1, (c + 1) * CHUNK);
      cp_async_commit();
      cp_async_wait1();
      __syncthreads();
      const C* ps = sp + (c & 1) * kSigBands * CHUNK;
      const int k0 = c * CHUNK, kp = min(CHUNK, nr - k0) / 2;
      if (active) {
        for (int q0 = lane; q0 < PAIRS; q0 += 32 * kSigUnroll) {
          C o[kSigUnroll][2], u[kSigUnroll][2], w[kSigUnroll][2];
#pragma unroll
          for (int v = 0; v < kSigUnroll; ++v) {
            const int q = q0 + 32 * v;
            if (q < kp) {
              ld_pair(go + off + k0 + 2 * q, o[v][0], o[v][1]);
              ld_pair(gu + off + k0 + 2 * q, u[v][0], u[v][1]);
              ld_pair(wrr + off + k0 + 2 * q, w[v][0], w[v][1]);
            }
          }
#pragma unroll
          for (int v = 0; v < kSigUnroll; ++v) {
            const int q = q0 + 32 * v;
            if (q >= kp) continue;
            const C ho0 = cmul(o[v][0], w[v][0]), ho1 = cmul(o[v][1], w[v][1]);
            const C hu0 = cmul(u[v][0], w[v][0]), hu1 = cmul(u[v][1], w[v][1]);
#pragma unroll
            for (int b = 0; b < kSigBands; ++b) {
              const C a0 = ps[b * CHUNK + 2 * q], a1 = ps[b * CHUNK + 2 * q + 1];
              vo[b][0] += ho0.x * a0.x - ho0.y * a0.y + ho1.x * a1.x - ho1.y * a1.y;
              vo[b][1] += ho0.x * a0.y + ho0.y * a0.x + ho1.x * a1.y + ho1.y * a1.x;
              vu[b][0] += hu0.x * a0.x - hu0.y * a0.y + hu1.x * a1.x - hu1.y * a1.y;
              vu[b][1] += hu0.x * a0.y + hu0.y * a0.x + hu1.x * a1.y + hu1.y * a1.x;
            }
          }
        }
      }
      __syncthreads();                     // buffer c & 1 is staged again at chunk c + 2
    }
    // warp sums, then Re(conj(psi_n(r)) V_n), then one atomic per band and CTA
#pragma unroll
    for (int b = 0; b < kSigBands; ++b) {
#pragma unroll
      for (int o2 = 16; o2 > 0; o2 >>= 1) {
        vo[b][0] += __shfl_xor_sync(0xffffffffu, vo[b][0], o2);
        vo[b][1] += __shfl_xor_sync(0xffffffffu, vo[b][1], o2);
        vu[b][0] += __shfl_xor_sync(0xffffffffu, vu[b][0], o2);
        vu[b][1] += __shfl_xor_sync(0xffffffffu, vu[b][1], o2);
      }
      if (lane == b) {
        double so = 0, su = 0;
        if (b < nb && active) {
          const C pn = psi_row[(long)bands[b0 + b] * ld_row + r0 + r];
          so = -coef * ((double)pn.x * vo[b][0] + (double)pn.y * vo[b][1]);
          su = coef * ((double)pn.x * vu[b][0] + (double)pn.y * vu[b][1]);
        }
        red[rl][b][0] = so;
        red[rl][b][1] = su;
      }
    }
    __syncthreads();
    if (threadIdx.x < 2 * nb) {
      const int b = threadIdx.x >> 1, which = threadIdx.x & 1;
      double t = 0;
      for (int i = 0; i < kSigRows; ++i) t += red[i][b][which];
      atomicAdd((which ? acc_u : acc_o) + (long)(b0 + b) * acc_stride, t);
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
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

gw_status launch_sigma_contract(gw_ctx* ctx, gw_prec prec, const void* wrr, const void* go, const void* gu, long ld,
                                int nr, int rows, const void* psi, const int* bands, int n_n, int r0, double coef,
                                double* acc_u, double* acc_o, int acc_stride, cudaStream_t st, const void* psi_row,
                                long ld_row) {
  if (rows <= 0) return GW_OK;
  if (!psi_row) {
    psi_row = psi;
    ld_row = nr;
  }
  const dim3 grid((rows + kSigRows - 1) / kSigRows);
  auto go_ = [&](auto kernel, size_t esz, int chunk, auto* tag) -> gw_status {
    using C = std::remove_pointer_t<decltype(tag)>;
    const size_t bytes = (size_t)kSigBands * chunk * esz;
    gw_status rc = cuda_check(ctx, cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes),
                              "cudaFuncSetAttribute");
    if (rc) return rc;
    KTimer kt(ctx, KF_SIGMA, 3.0 * rows * (double)nr * esz, st);
    kernel<<<grid, kSigThreads, bytes, st>>>((const C*)wrr, (const C*)go, (const C*)gu, ld, nr, rows, (const C*)psi,
                                             bands, n_n, r0, coef, acc_u, acc_o, acc_stride, (const C*)psi_row,
                                             ld_row);
    return launch_check(ctx, "sigma_contract_kernel");
  };
  if (is_fp64(prec)) return go_(sigma_contract_kernel<double>, sizeof(double2), 2 * 256, (double2*)nullptr);
  return go_(sigma_contract_kernel<float>, sizeof(float2), 2 * 512, (float2*)nullptr);
}

// Even/odd split, CT + ST and Thiele continuation of the accumulated
// Sigma(tau) (acc [2][n_n][n]: unoccupied, occupied), then the results to the
// host.  tab: C [n][n], S [n][n], omega [n], real frequencies [n_real] in one
// device block; out [n_n][n] + [n_n][n_real] complex; stat [n_n].
gw_status sigma_finish(gw_ctx* ctx, double* acc, int n_n, int n, const double* tab, int n_real, double2* out,
                       int* stat, const int32_t* labels, double* sigma_tau_h, double* sigma_iw_h,
                       double* sigma_real_h, cudaStream_t s) {
  gw_status st;
  const double* dC = tab;
  const double* dS = dC + (size_t)n * n;
  const double* dom = dS + (size_t)n * n;
  const double* dwr = dom + n;
  double2* out_re = out + (size_t)n_n * n;
  sigma_finish_kernel<<<(n_n + 63) / 64, 64, 0, s>>>(acc, acc + (size_t)n_n * n, n_n, n, dC, dS, dom, dwr, n_real,
                                                      out, n_real > 0 ? out_re : nullptr, stat);
  if ((st = launch_check(ctx, "sigma_finish_kernel"))) return st;
  std::vector<double2> h_iw((size_t)n_n * n), h_re((size_t)n_n * std::max(n_real, 1));
  std::vector<int> h_stat(n_n);
  std::vector<double> h_acc(2 * (size_t)n_n * n);
  cudaMemcpyAsync(h_iw.data(), out, sizeof(double2) * n_n * n, cudaMemcpyDeviceToHost, s);
  if (n_real > 0) cudaMemcpyAsync(h_re.data(), out_re, sizeof(double2) * n_n * n_real, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(h_stat.data(), stat, sizeof(int) * n_n, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(h_acc.data(), acc, sizeof(double) * 2 * n_n * n, cudaMemcpyDeviceToHost, s);
  if ((st = cuda_check(ctx, cudaStreamSynchronize(s), "sigma sync"))) return st;
  std::memcpy(sigma_iw_h, h_iw.data(), sizeof(double2) * n_n * n);
  if (n_real > 0) std::memcpy(sigma_real_h, h_re.data(), sizeof(double2) * n_n * n_real);
  if (sigma_tau_h) std::memcpy(sigma_tau_h, h_acc.data(), sizeof(double) * 2 * n_n * n);
  for (int b = 0; b < n_n; ++b)
    if (h_stat[b])
      return fail(ctx, GW_ERR_NUMERIC, "Thiele continuation broke down for band " + std::to_string(labels[b]));
  return GW_OK;
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
  char* wrr = cv.take<char>((size_t)rb * g.nr * es);
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
      // W~(r,R') of the block (second step of Eq. FFTW), then the contraction
      if ((st = launch_row_fft(ctx, g, prec, 2, wrg + (size_t)r0 * n_chi * es, nullptr, n_chi, wrr, g.nr, dmap, n_chi,
                               rows, 1.0, s, dinv)))
        return st;
      if ((st = launch_sigma_contract(ctx, prec, wrr, gob, gub, g.nr, g.nr, rows, psi, dbands, n_n, r0, coef,
                                      acc_u + j, acc_o + j, n, s)))
        return st;
    }
  }
  if (tc && (st = tc_check(ctx, tcs, s))) return st;
  return sigma_finish(ctx, acc, n_n, n, dC, n_real, out_iw, dstat, bands_h, sigma_tau_h, sigma_iw_h, sigma_real_h, s);
}
