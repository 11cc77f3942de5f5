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

// Two consecutive complex values from shared memory, one 16-byte access for
// FP32 (four wavefronts per warp instead of eight; measured time unchanged, so
// shared memory is not what limits the contraction).
__device__ __forceinline__ void ld_smem_pair(const float2* p, float2& a, float2& b) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void ld_smem_pair(const double2* p, double2& a, double2& b) {
  a = p[0];
  b = p[1];
}

// FULL: instead of the diagonal reduction, V_m(r) itself goes to vout
// [2][n_n][vstride] (occupied, then unoccupied) for the matrix Sigma_nm.
template <typename T, bool FULL>
__global__ void __launch_bounds__(kSigThreads) sigma_contract_kernel(
    const typename cpx<T>::t* __restrict__ wrr, const typename cpx<T>::t* __restrict__ go,
    const typename cpx<T>::t* __restrict__ gu, long ld, int nr, int rows,
    const typename cpx<T>::t* __restrict__ psi, const int* __restrict__ bands, int n_n, int r0, double coef,
    double* __restrict__ acc_u, double* __restrict__ acc_o, int acc_stride,
    const typename cpx<T>::t* __restrict__ psi_row, long ld_row, double2* __restrict__ vout, int vstride) {
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
              C a0, a1;
              ld_smem_pair(ps + b * CHUNK + 2 * q, a0, a1);
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
      if constexpr (FULL) {
        if (lane == b && b < nb && active) {
          vout[(long)(b0 + b) * vstride + r] = make_double2(vo[b][0], vo[b][1]);
          vout[(long)(n_n + b0 + b) * vstride + r] = make_double2(vu[b][0], vu[b][1]);
        }
      } else if (lane == b) {
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
    if constexpr (FULL) continue;
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

__device__ __forceinline__ bool tiny(double2 a) { return !(sqrt(zabs2(a)) >= 1e-300); }

// Thiele coefficients a_p = g_p(z_p) by reciprocal differences (Eq. pade2).
// g holds f(z_k) on entry and is overwritten.  False if a difference vanishes.
__device__ bool thiele_coeffs(double2* g, const double2* z, int n, double2* a) {
  a[0] = g[0];
  for (int p = 1; p < n; ++p) {
    const double2 prev = g[p - 1];
    for (int m = p; m < n; ++m) {
      const double2 den = cmul(csub(z[m], z[p - 1]), g[m]);
      if (tiny(den)) return false;
      g[m] = zdiv(csub(prev, g[m]), den);
    }
    a[p] = g[p];
  }
  return true;
}

// The continued fraction of Eq. pade1 (tail set to zero) at x by backward
// evaluation, t <- 1 + a_p (x - z_{p-1}) / t from t = 1, value a_1 / t; with
// dval, also its derivative: each step differentiated by the quotient rule,
// t' <- a_p / t - a_p (x - z_{p-1}) t' / t^2, and the value's -a_1 t' / t^2.
// a and z are read through their index (registers or global memory).
template <typename A, typename Z>
__device__ bool thiele_eval(const A& a, const Z& z, int n, double2 x, double2* val, double2* dval) {
  double2 t = make_double2(1.0, 0.0), dt = make_double2(0.0, 0.0);
  for (int p = n - 1; p >= 1; --p) {
    if (tiny(t)) return false;
    const double2 ap = a(p);
    const double2 u = cmul(ap, csub(x, z(p - 1)));
    if (dval) dt = csub(zdiv(ap, t), zdiv(cmul(u, dt), cmul(t, t)));
    const double2 q = zdiv(u, t);
    t = make_double2(1.0 + q.x, q.y);
  }
  if (tiny(t)) return false;
  *val = zdiv(a(0), t);
  if (dval) {
    const double2 d = zdiv(cmul(a(0), dt), cmul(t, t));
    *dval = make_double2(-d.x, -d.y);
  }
  return true;
}

__global__ void sigma_finish_kernel(const double* __restrict__ acc_u, const double* __restrict__ acc_o, int n_n, int n,
                                    const double* __restrict__ Cm, const double* __restrict__ Sm,
                                    const double* __restrict__ omega, const double* __restrict__ wreal, int n_real,
                                    double2* __restrict__ out_iw, double2* __restrict__ out_real,
                                    int* __restrict__ status) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_n) return;
  double2 g[kMaxN], a[kMaxN], z[kMaxN];
  for (int k = 0; k < n; ++k) {
    double re = 0, im = 0;
    for (int j = 0; j < n; ++j) {
      const double sc = 0.5 * (acc_u[b * n + j] + acc_o[b * n + j]);
      const double ss = 0.5 * (acc_u[b * n + j] - acc_o[b * n + j]);
      re += Cm[k * n + j] * sc;
      im += Sm[k * n + j] * ss;
    }
    g[k] = make_double2(re, im);
    out_iw[b * n + k] = g[k];
    z[k] = make_double2(0.0, omega[k]);
  }
  bool ok = thiele_coeffs(g, z, n, a);
  auto av = [&](int p) { return a[p]; };
  auto zv = [&](int p) { return z[p]; };
  for (int q = 0; q < n_real; ++q) {
    double2 res = make_double2(NAN, NAN);
    if (ok) ok = thiele_eval(av, zv, n, make_double2(wreal[q], 0.0), &res, nullptr);
    if (!ok) res = make_double2(NAN, NAN);
    if (out_real) out_real[b * n_real + q] = res;
  }
  status[b] = ok ? 0 : 1;
}

// ---------------------------------------------------------------- full matrix
// Sigma_nm(tau_j) += coef conj(psi_n(r0 + r)) V_m(r) summed over rows for the
// unoccupied V (plus) and the occupied V (minus); one thread per (n, m) of a
// 16 x 16 tile (blockIdx.x, blockIdx.y) and rows_per_cta rows per CTA
// (blockIdx.z), staged 32 at a time in shared memory; the CTAs' partial sums
// meet in FP64 atomics.  acc_u / acc_o are [n_n][n_n][acc_stride] complex,
// already offset to tau_j.  Spreading the rows over CTAs matters: the sums are
// FP64, whose per-SM rate is low.
template <typename T>
__global__ void __launch_bounds__(256) sigma_outer_kernel(const double2* __restrict__ vout, int vstride, int rows,
                                                          int rows_per_cta,
                                                          const typename cpx<T>::t* __restrict__ psi_row, long ld_row,
                                                          const int* __restrict__ bands, int n_n, int r0, double coef,
                                                          double2* __restrict__ acc_u, double2* __restrict__ acc_o,
                                                          int acc_stride) {
  __shared__ double2 sp[16][33], svo[16][33], svu[16][33];
  const int n0 = blockIdx.y * 16, m0 = blockIdx.x * 16;
  const int tn = threadIdx.x >> 4, tm = threadIdx.x & 15;
  const int c0 = blockIdx.z * rows_per_cta, c1 = min(rows, c0 + rows_per_cta);
  const double2* vo = vout;
  const double2* vu = vout + (long)n_n * vstride;
  double2 ao = make_double2(0.0, 0.0), au = make_double2(0.0, 0.0);
  for (int c = c0; c < c1; c += 32) {
    for (int e = threadIdx.x; e < 16 * 32; e += 256) {
      const int i = e >> 5, r = e & 31;
      const bool in = c + r < c1;
      double2 pv = make_double2(0.0, 0.0), o = pv, u = pv;
      if (in && n0 + i < n_n) {
        const auto v = psi_row[(long)bands[n0 + i] * ld_row + r0 + c + r];
        pv = make_double2((double)v.x, (double)v.y);
      }
      if (in && m0 + i < n_n) {
        o = vo[(long)(m0 + i) * vstride + c + r];
        u = vu[(long)(m0 + i) * vstride + c + r];
      }
      sp[i][r] = pv;
      svo[i][r] = o;
      svu[i][r] = u;
    }
    __syncthreads();
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
      const double2 pv = sp[tn][r];
      ao = cadd(ao, cmul(cconj(pv), svo[tm][r]));
      au = cadd(au, cmul(cconj(pv), svu[tm][r]));
    }
    __syncthreads();
  }
  if (n0 + tn < n_n && m0 + tm < n_n) {
    const long idx = ((long)(n0 + tn) * n_n + (m0 + tm)) * acc_stride;
    double* po = reinterpret_cast<double*>(acc_o + idx);
    double* pu = reinterpret_cast<double*>(acc_u + idx);
    atomicAdd(po, -coef * ao.x);
    atomicAdd(po + 1, -coef * ao.y);
    atomicAdd(pu, coef * au.x);
    atomicAdd(pu + 1, coef * au.y);
  }
}

// Sigma_nm(i omega_k) = sum_j C_kj Sigma^c_nm(tau_j) + i sum_j S_kj Sigma^s_nm(tau_j)
// on the complex matrices (Eqs. cos_sin_sigma, sigma_r_w, cos_sin_sigma1/2);
// one thread per (n, m, k).
__global__ void sigma_matrix_finish_kernel(const double2* __restrict__ acc_u, const double2* __restrict__ acc_o,
                                           int nnm, int n, const double* __restrict__ Cm,
                                           const double* __restrict__ Sm, double2* __restrict__ out_iw) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)nnm * n) return;
  const long e = t / n;
  const int k = (int)(t - e * n);
  double2 c = make_double2(0.0, 0.0), sn = c;
  for (int j = 0; j < n; ++j) {
    const double2 u = acc_u[e * n + j], o = acc_o[e * n + j];
    c = cadd(c, cscale(cscale(cadd(u, o), 0.5), Cm[k * n + j]));
    sn = cadd(sn, cscale(cscale(csub(u, o), 0.5), Sm[k * n + j]));
  }
  out_iw[t] = cadd(c, cmuli(sn));
}

// ---------------------------------------------------------------- back to imaginary time
// Sigma(i omega) = C Sigma^c(tau) + i S Sigma^s(tau), with Sigma^c, Sigma^s
// Hermitian in the band indices and C, S real: the Hermitian part of Sigma(i
// omega) is the cosine part, the anti-Hermitian part the sine part.  One thread
// per element e of [n_n][n_n] (matrix) or [n_n] (diagonal: real and imaginary
// parts), writing both parts frequency-major, [n][E], for the transform.
__global__ void sigma_split_kernel(const double2* __restrict__ sig, int n_n, int n, int matrix,
                                   double2* __restrict__ herm, double2* __restrict__ anti) {
  const long E = matrix ? (long)n_n * n_n : n_n;
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  long et = e;                                     // the transposed element
  if (matrix) {
    const long a = e / n_n, b = e - a * n_n;
    et = b * n_n + a;
  }
  for (int k = 0; k < n; ++k) {
    const double2 v = sig[e * n + k];
    if (matrix) {
      const double2 t = cconj(sig[et * n + k]);
      herm[(long)k * E + e] = cscale(cadd(v, t), 0.5);
      anti[(long)k * E + e] = cscale(csub(v, t), 0.5);
    } else {
      herm[(long)k * E + e] = make_double2(v.x, 0.0);
      anti[(long)k * E + e] = make_double2(0.0, v.y);
    }
  }
}

// Sigma_unocc(tau_j) = Sigma^c + Sigma^s, Sigma_occ(-tau_j) = Sigma^c - Sigma^s
// from the transformed parts [n][E], written [2][E][n] (real parts only for the
// diagonal form, as gw_sigma_diag returns them).
__global__ void sigma_combine_kernel(const double2* __restrict__ sc, const double2* __restrict__ ss, long E, int n,
                                     int matrix, double* __restrict__ out) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= E * n) return;
  const long e = t / n;
  const int j = (int)(t - e * n);
  const double2 c = sc[(long)j * E + e], d = ss[(long)j * E + e];
  const double2 u = cadd(c, d), o = csub(c, d);
  if (matrix) {
    double2* o2 = reinterpret_cast<double2*>(out);
    o2[e * n + j] = u;
    o2[E * n + e * n + j] = o;
  } else {
    out[e * n + j] = u.x;
    out[E * n + e * n + j] = o.x;
  }
}

// ---------------------------------------------------------------- QP energies
// Thiele coefficients of every band's Sigma_n through z_k = i omega_k.
__global__ void qp_coeff_kernel(const double2* __restrict__ sig, const double* __restrict__ omega, int n_n, int n,
                                double2* __restrict__ coef, int* __restrict__ status) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_n) return;
  double2 g[kMaxN], a[kMaxN], z[kMaxN];
  for (int k = 0; k < n; ++k) {
    g[k] = sig[(long)b * n + k];
    z[k] = make_double2(0.0, omega[k]);
  }
  const bool ok = thiele_coeffs(g, z, n, a);
  for (int k = 0; k < n; ++k) coef[(long)b * n + k] = ok ? a[k] : make_double2(NAN, NAN);
  status[b] = ok ? 0 : 1;
}

// One thread per (band, point).  Point 0: the linearised QP equation at eps_n
// (Eqs. QP, GWQP, Z) with Sigma_n(eps_n - mu) and its derivative; points
// 1..n_w: the spectral function of Eq. A at w_q, with
// DeltaSigma = v_n + Sigma_n(w - mu) - eps_n.
__global__ void qp_eval_kernel(const double2* __restrict__ coef, const double* __restrict__ omega, int n_n, int n,
                               const double* __restrict__ eps, const double* __restrict__ vstat, double mu,
                               const double* __restrict__ w, int n_w, double* __restrict__ e_qp,
                               double* __restrict__ zf, double2* __restrict__ s_eps, double2* __restrict__ ds,
                               double* __restrict__ spec, int* __restrict__ status) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)n_n * (n_w + 1)) return;
  const int b = (int)(t / (n_w + 1));
  const int q = (int)(t - (long)b * (n_w + 1));
  const double2* ab = coef + (long)b * n;
  auto av = [&](int p) { return ab[p]; };
  auto zv = [&](int p) { return make_double2(0.0, omega[p]); };
  const double e = eps[b];
  double2 val = make_double2(NAN, NAN), dval = val;
  if (q == 0) {
    const bool ok = (status[b] & 1) == 0 && thiele_eval(av, zv, n, make_double2(e - mu, 0.0), &val, &dval);
    const double z = ok ? 1.0 / (1.0 - dval.x) : NAN;
    s_eps[b] = ok ? val : make_double2(NAN, NAN);
    ds[b] = ok ? dval : make_double2(NAN, NAN);
    zf[b] = z;
    e_qp[b] = e + z * (vstat[b] + val.x - e);
    if (!ok || !isfinite(z)) atomicOr(status + b, 2);
  } else {
    const double x = w[q - 1];
    const bool ok = (status[b] & 1) == 0 && thiele_eval(av, zv, n, make_double2(x - mu, 0.0), &val, nullptr);
    const double dre = vstat[b] + val.x - e, dim = val.y;
    const double d = x - e - dre;
    spec[(long)b * n_w + q - 1] = ok ? fabs(dim) / kPi / (d * d + dim * dim) : NAN;
    if (!ok) atomicOr(status + b, 4);
  }
}

gw_status launch_sigma_contract(gw_ctx* ctx, gw_prec prec, const void* wrr, const void* go, const void* gu, long ld,
                                int nr, int rows, const void* psi, const int* bands, int n_n, int r0, double coef,
                                double* acc_u, double* acc_o, int acc_stride, cudaStream_t st, const void* psi_row,
                                long ld_row, double2* vout, int vstride) {
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
                                             ld_row, vout, vstride);
    return launch_check(ctx, "sigma_contract_kernel");
  };
  if (vout) {
    if (is_fp64(prec)) return go_(sigma_contract_kernel<double, true>, sizeof(double2), 2 * 256, (double2*)nullptr);
    return go_(sigma_contract_kernel<float, true>, sizeof(float2), 2 * 512, (float2*)nullptr);
  }
  if (is_fp64(prec)) return go_(sigma_contract_kernel<double, false>, sizeof(double2), 2 * 256, (double2*)nullptr);
  return go_(sigma_contract_kernel<float, false>, sizeof(float2), 2 * 512, (float2*)nullptr);
}

// The matrix update of one block of rows from the V_m(r) of the contraction.
static gw_status launch_sigma_outer(gw_ctx* ctx, gw_prec prec, const double2* vout, int vstride, int rows,
                                    const void* psi, long ld, const int* bands, int n_n, int r0, double coef,
                                    double2* acc_u, double2* acc_o, int acc_stride, cudaStream_t st) {
  if (rows <= 0) return GW_OK;
  // about two CTAs per SM in all, rows split in multiples of 32
  const long tiles = (long)((n_n + 15) / 16) * ((n_n + 15) / 16);
  const long splits = std::max(1L, 2L * ctx->num_sms / tiles);
  const int rpc = (int)std::max(32L, ((rows + splits - 1) / splits + 31) / 32 * 32);
  const dim3 grid((n_n + 15) / 16, (n_n + 15) / 16, (rows + rpc - 1) / rpc);
  if (is_fp64(prec))
    sigma_outer_kernel<double><<<grid, 256, 0, st>>>(vout, vstride, rows, rpc, (const double2*)psi, ld, bands, n_n, r0,
                                                     coef, acc_u, acc_o, acc_stride);
  else
    sigma_outer_kernel<float><<<grid, 256, 0, st>>>(vout, vstride, rows, rpc, (const float2*)psi, ld, bands, n_n, r0,
                                                    coef, acc_u, acc_o, acc_stride);
  return launch_check(ctx, "sigma_outer_kernel");
}

// The kernel of sigma_finish alone (device results, no synchronisation).
gw_status sigma_finish_launch(gw_ctx* ctx, const double* acc, int n_n, int n, const double* tab, int n_real,
                              double2* out, int* stat, cudaStream_t s) {
  const double* dC = tab;
  const double* dS = dC + (size_t)n * n;
  const double* dom = dS + (size_t)n * n;
  const double* dwr = dom + n;
  double2* out_re = out + (size_t)n_n * n;
  sigma_finish_kernel<<<(n_n + 63) / 64, 64, 0, s>>>(acc, acc + (size_t)n_n * n, n_n, n, dC, dS, dom, dwr, n_real,
                                                      out, n_real > 0 ? out_re : nullptr, stat);
  return launch_check(ctx, "sigma_finish_kernel");
}

// Results of sigma_finish_launch to the host (synchronises s).
static gw_status sigma_fetch(gw_ctx* ctx, const double* acc, int n_n, int n, int n_real, const double2* out,
                             const int* stat, const int32_t* labels, double* sigma_tau_h, double* sigma_iw_h,
                             double* sigma_real_h, cudaStream_t s) {
  gw_status st;
  const double2* out_re = out + (size_t)n_n * n;
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

// Even/odd split, CT + ST and Thiele continuation of the accumulated
// Sigma(tau) (acc [2][n_n][n]: unoccupied, occupied), then the results to the
// host.  tab: C [n][n], S [n][n], omega [n], real frequencies [n_real] in one
// device block; out [n_n][n] + [n_n][n_real] complex; stat [n_n].
gw_status sigma_finish(gw_ctx* ctx, double* acc, int n_n, int n, const double* tab, int n_real, double2* out,
                       int* stat, const int32_t* labels, double* sigma_tau_h, double* sigma_iw_h,
                       double* sigma_real_h, cudaStream_t s) {
  gw_status st = sigma_finish_launch(ctx, acc, n_n, n, tab, n_real, out, stat, s);
  if (st) return st;
  return sigma_fetch(ctx, acc, n_n, n, n_real, out, stat, labels, sigma_tau_h, sigma_iw_h, sigma_real_h, s);
}

// Up to this many bands, the tensor-core precisions fuse the contraction into
// the G formation (tc_sigma_rows): G never goes to memory.
constexpr int kFusedBands = 32;

void sigma_carve_tables(Carver& cv, const GridInfo& g, int n_b, int n, int n_chi, int n_n, int n_real, bool full,
                        SigmaTables& t) {
  const size_t nnm = full ? (size_t)n_n * n_n : (size_t)n_n;
  t.map = cv.take<int>(n_chi);
  t.inv = cv.take<int>(g.nr);
  t.bands = cv.take<int>(n_n);
  t.scale = cv.take<char>((size_t)n * n_b * 8);
  t.tab = cv.take<double>(4 * (size_t)n * n + 2 * n + std::max(n_real, 1));
  t.acc2 = cv.take<double2>((full ? 2 : 1) * nnm * n);   // [2][n_n][n] real, or [2][n_n][n_n][n] complex
  t.out = cv.take<double2>(nnm * n + (size_t)n_n * std::max(n_real, 1));
  t.stat = cv.take<int>(n_n);
}

void sigma_carve_work(Carver& cv, const GridInfo& g, int n_b, int n_occ, int n_chi, int n_n, gw_prec prec, bool full,
                      SigmaWork& w) {
  const size_t es = csize(prec);
  const int rb = std::min(g.nr, 2048);
  w.fused = (prec == GW_F16X3 || prec == GW_BF16X3) && !full && n_n <= kFusedBands;
  w.vout = full ? cv.take<double2>(2 * (size_t)n_n * rb) : nullptr;
  w.wrg = cv.take<char>((size_t)g.nr * n_chi * es);
  w.gob = cv.take<char>((size_t)rb * g.nr * es);
  w.gub = cv.take<char>((size_t)rb * g.nr * es);
  w.wrr = cv.take<char>((size_t)rb * g.nr * es);
  w.tcs = (prec == GW_F16X3 || prec == GW_BF16X3)
              ? cv.take<char>(tc_scratch_bytes(g, n_b, n_occ, rb, false, w.fused ? n_n : 0))
              : nullptr;
}

size_t sigma_scratch(const GridInfo& g, int n_b, int n_occ, int n, int n_chi, int n_n, int n_real, gw_prec prec,
                     bool full) {
  Carver probe(nullptr);
  SigmaTables t;
  SigmaWork w;
  sigma_carve_tables(probe, g, n_b, n, n_chi, n_n, n_real, full, t);
  sigma_carve_work(probe, g, n_b, n_occ, n_chi, n_n, prec, full, w);
  return probe.off;
}

gw_status sigma_upload_tables(gw_ctx* ctx, const SigmaTables& t, const GridInfo& g, int n_b, int n, int n_chi,
                              const std::vector<int>& map, const std::vector<int>& inv, const int32_t* bands_h, int n_n,
                              const std::vector<GreenScales>& scales, const double* C_h, const double* S_h,
                              const double* omega_h, const double* w_real_h, int n_real, gw_prec prec, cudaStream_t s) {
  gw_status st;
  if ((st = upload(ctx, t.map, map.data(), sizeof(int) * n_chi, s))) return st;
  if ((st = upload(ctx, t.inv, inv.data(), sizeof(int) * g.nr, s))) return st;
  if ((st = upload(ctx, t.bands, bands_h, sizeof(int) * n_n, s))) return st;
  for (int j = 0; j < n; ++j)
    if ((st = upload_scales(ctx, t.scale + (size_t)j * n_b * 8, scales[j], prec, s))) return st;
  double* dC = t.tab;
  double* dS = dC + (size_t)n * n;
  double* dom = dS + (size_t)n * n;
  double* dwr = dom + n;
  if ((st = upload(ctx, dC, C_h, sizeof(double) * n * n, s))) return st;
  if ((st = upload(ctx, dS, S_h, sizeof(double) * n * n, s))) return st;
  if ((st = upload(ctx, dom, omega_h, sizeof(double) * n, s))) return st;
  if (n_real > 0 && (st = upload(ctx, dwr, w_real_h, sizeof(double) * n_real, s))) return st;
  return GW_OK;
}

// The kernels of one self-energy evaluation on s, with the tables already on the
// device: device-side memsets and launches only (no host copy, no
// synchronisation), so that a plan can capture them in a CUDA graph.  Results
// stay in t.out / t.stat (diagonal) or t.out (matrix); the tensor-core time-out
// words in the scratch w.tcs.
gw_status sigma_kernels(gw_ctx* ctx, const GridInfo& g, gw_prec prec, bool full, int n_b, int n_occ, const void* psi,
                        int n_n, int n, int n_chi, int n_real, const std::vector<GreenScales>& scales,
                        const SigmaTables& t, const SigmaWork& w, const void* w_tau, cudaStream_t s) {
  gw_status st;
  const size_t es = csize(prec);
  const int rb = std::min(g.nr, 2048);
  const bool tc = prec == GW_F16X3 || prec == GW_BF16X3;
  const size_t nnm = full ? (size_t)n_n * n_n : (size_t)n_n;
  const size_t acc_elems = (full ? 2 : 1) * nnm * n;
  if ((st = cuda_check(ctx, cudaMemsetAsync(t.acc2, 0, sizeof(double2) * acc_elems, s), "memset"))) return st;
  double* acc = reinterpret_cast<double*>(t.acc2);
  double* acc_u = acc;
  double* acc_o = acc + (size_t)n_n * n;
  double2* accm_u = t.acc2;
  double2* accm_o = t.acc2 + nnm * n;
  const double coef = g.dv * g.dv / g.volume;   // dV^2 and the 1/Omega of Eq. FFTW
  bool first = true;
  for (int j = 0; j < n; ++j) {
    const char* wj = static_cast<const char*>(w_tau) + (size_t)j * n_chi * n_chi * es;
    const char* sj = t.scale + (size_t)j * n_b * 8;
    if ((st = launch_col_line(ctx, g, prec, +1, 1, wj, n_chi, w.wrg, n_chi, n_chi, t.inv, 1.0, s))) return st;
    if ((st = launch_col_plane(ctx, g, prec, +1, w.wrg, n_chi, n_chi, 1.0, s))) return st;
    for (int r0 = 0; r0 < g.nr; r0 += rb) {
      const int rows = std::min(rb, g.nr - r0);
      if (w.fused) {
        // W~(r,R') of the block, then G formation with the contraction in its epilogue
        if ((st = launch_row_fft(ctx, g, prec, 2, w.wrg + (size_t)r0 * n_chi * es, nullptr, n_chi, w.wrr, g.nr, t.map,
                                 n_chi, rows, 1.0, s, t.inv)))
          return st;
        TcSigma sg;
        sg.wrr = reinterpret_cast<const float2*>(w.wrr);
        sg.ldw = g.nr;
        sg.bands = t.bands;
        sg.n_n = n_n;
        sg.coef = coef;
        sg.acc_u = acc_u + j;
        sg.acc_o = acc_o + j;
        sg.acc_stride = n;
        sg.sk = reinterpret_cast<const float*>(sj);     // FP32 factors of tau_j (no host copy)
        if ((st = tc_sigma_rows(ctx, g, n_b, n_occ, psi, scales[j], r0, rows, prec, sg, w.tcs, first, s))) return st;
        first = false;
        continue;
      }
      if (tc) {
        st = tc_green_rows(ctx, g, n_b, n_occ, psi, scales[j], r0, rows, prec, w.gob, w.gub, w.tcs, first, s,
                           reinterpret_cast<const float*>(sj));
        first = false;
      }
      else st = green_rows(ctx, g, n_b, n_occ, psi, sj, scales[j], r0, rows, prec, w.gob, w.gub, s);
      if (st) return st;
      // W~(r,R') of the block (second step of Eq. FFTW), then the contraction
      if ((st = launch_row_fft(ctx, g, prec, 2, w.wrg + (size_t)r0 * n_chi * es, nullptr, n_chi, w.wrr, g.nr, t.map,
                               n_chi, rows, 1.0, s, t.inv)))
        return st;
      if (!full) {
        if ((st = launch_sigma_contract(ctx, prec, w.wrr, w.gob, w.gub, g.nr, g.nr, rows, psi, t.bands, n_n, r0, coef,
                                        acc_u + j, acc_o + j, n, s)))
          return st;
      } else {
        if ((st = launch_sigma_contract(ctx, prec, w.wrr, w.gob, w.gub, g.nr, g.nr, rows, psi, t.bands, n_n, r0, coef,
                                        nullptr, nullptr, n, s, nullptr, 0, w.vout, rb)))
          return st;
        if ((st = launch_sigma_outer(ctx, prec, w.vout, rb, rows, psi, g.nr, t.bands, n_n, r0, coef, accm_u + j,
                                     accm_o + j, n, s)))
          return st;
      }
    }
  }
  if (!full) return sigma_finish_launch(ctx, acc, n_n, n, t.tab, n_real, t.out, t.stat, s);
  const long tot = (long)nnm * n;
  const double* dS = t.tab + (size_t)n * n;
  sigma_matrix_finish_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(accm_u, accm_o, (int)nnm, n, t.tab, dS,
                                                                             t.out);
  return launch_check(ctx, "sigma_matrix_finish_kernel");
}

// Validation and host tables shared by the self-energy entry points and plans.
gw_status sigma_check(gw_ctx* ctx, const gw_grid* grid, GridInfo* g, int n_b, int n_occ, const void* psi,
                      const double* eps_h, double mu, const int32_t* bands_h, int n_n, int n, const double* tau_h,
                      const double* omega_h, const double* C_h, const double* S_h, const void* w_tau, int n_chi,
                      const int32_t* fft_index_h, gw_prec prec, bool full, const double* w_real_h, int n_real,
                      std::vector<int>& map, std::vector<int>& inv, std::vector<GreenScales>& scales) {
  if (!ctx) return fail(nullptr, GW_ERR_ARG, "ctx is NULL");
  gw_status st = grid_info(ctx, grid, g);
  if (st) return st;
  if (!grid_supported(g->n1, g->n2, g->n3)) return fail(ctx, GW_ERR_UNSUPPORTED, "no kernels compiled for this grid");
  if (!valid_prec(prec)) return fail(ctx, GW_ERR_ARG, "bad precision");
  if (!psi || !w_tau || !bands_h || !tau_h || !omega_h || !C_h || !S_h) return fail(ctx, GW_ERR_ARG, "NULL pointer");
  if (n_b < 2 || n_b > g->nr) return fail(ctx, GW_ERR_SHAPE, "need 2 <= n_b <= N_r");
  if (reinterpret_cast<uintptr_t>(psi) % 16) return fail(ctx, GW_ERR_ARG, "psi must be 16-byte aligned");
  if ((st = check_energies(ctx, eps_h, n_b, n_occ, mu))) return st;
  if (n < 1 || n > kMaxN) return fail(ctx, GW_ERR_SHAPE, "need 1 <= n <= 32");
  if (n_n < 1 || n_n > (full ? 256 : 1024))
    return fail(ctx, GW_ERR_SHAPE, full ? "need 1 <= n_n <= 256" : "need 1 <= n_n <= 1024");
  if (n_real < 0 || (n_real > 0 && !w_real_h)) return fail(ctx, GW_ERR_ARG, "bad real-axis request");
  for (int b = 0; b < n_n; ++b)
    if (bands_h[b] < 0 || bands_h[b] >= n_b) return fail(ctx, GW_ERR_ARG, "band index out of range");
  for (int j = 0; j < n; ++j)
    if (!(tau_h[j] > 0)) return fail(ctx, GW_ERR_ARG, "tau must be > 0");
  if ((st = index_maps(ctx, *g, fft_index_h, n_chi, map, inv))) return st;
  scales.resize(n);
  for (int j = 0; j < n; ++j) scales[j] = green_scales(eps_h, n_b, n_occ, mu, tau_h[j]);
  return GW_OK;
}

}  // namespace gw

using namespace gw;

// Shared body of gw_sigma_diag (full = false: acc real [2][n_n][n], Thiele
// continuation) and gw_sigma_matrix (full = true: acc complex [2][n_n][n_n][n]).
static gw_status sigma_impl(gw_ctx* ctx, const gw_grid* grid, int n_b, int n_occ, const void* psi,
                            const double* eps_h, double mu, const int32_t* bands_h, int n_n, int n,
                            const double* tau_h, const double* omega_h, const double* C_h, const double* S_h,
                            const void* w_tau, int n_chi, const int32_t* fft_index_h, gw_prec prec, bool full,
                            double* sigma_tau_h, double* sigma_iw_h, const double* w_real_h, int n_real,
                            double* sigma_real_h, cudaStream_t s) {
  GridInfo g;
  std::vector<int> map, inv;
  std::vector<GreenScales> scales;
  gw_status st = sigma_check(ctx, grid, &g, n_b, n_occ, psi, eps_h, mu, bands_h, n_n, n, tau_h, omega_h, C_h, S_h,
                             w_tau, n_chi, fft_index_h, prec, full, w_real_h, n_real, map, inv, scales);
  if (st) return st;
  if (!sigma_iw_h || (n_real > 0 && !sigma_real_h)) return fail(ctx, GW_ERR_ARG, "NULL output pointer");
  const bool tc = prec == GW_F16X3 || prec == GW_BF16X3;
  const size_t nnm = full ? (size_t)n_n * n_n : (size_t)n_n;
  if ((st = reserve(ctx, sigma_scratch(g, n_b, n_occ, n, n_chi, n_n, n_real, prec, full)))) return st;
  Carver cv(ctx->arena);
  SigmaTables t;
  SigmaWork w;
  sigma_carve_tables(cv, g, n_b, n, n_chi, n_n, n_real, full, t);
  sigma_carve_work(cv, g, n_b, n_occ, n_chi, n_n, prec, full, w);
  if ((st = sigma_upload_tables(ctx, t, g, n_b, n, n_chi, map, inv, bands_h, n_n, scales, C_h, S_h, omega_h, w_real_h,
                                n_real, prec, s)))
    return st;
  if ((st = sigma_kernels(ctx, g, prec, full, n_b, n_occ, psi, n_n, n, n_chi, n_real, scales, t, w, w_tau, s))) return st;
  if (tc && (st = tc_check(ctx, w.tcs, s))) return st;
  if (!full)
    return sigma_fetch(ctx, reinterpret_cast<const double*>(t.acc2), n_n, n, n_real, t.out, t.stat, bands_h,
                       sigma_tau_h, sigma_iw_h, sigma_real_h, s);
  std::vector<double2> h_iw(nnm * n), h_acc(2 * nnm * n);
  if ((st = cuda_check(ctx, cudaMemcpyAsync(h_iw.data(), t.out, sizeof(double2) * nnm * n, cudaMemcpyDeviceToHost, s),
                       "copy sigma")))
    return st;
  if (sigma_tau_h && (st = cuda_check(ctx, cudaMemcpyAsync(h_acc.data(), t.acc2, sizeof(double2) * 2 * nnm * n,
                                                           cudaMemcpyDeviceToHost, s), "copy sigma")))
    return st;
  if ((st = cuda_check(ctx, cudaStreamSynchronize(s), "sigma sync"))) return st;
  std::memcpy(sigma_iw_h, h_iw.data(), sizeof(double2) * nnm * n);
  if (sigma_tau_h) std::memcpy(sigma_tau_h, h_acc.data(), sizeof(double2) * 2 * nnm * n);
  return GW_OK;
}

extern "C" gw_status gw_sigma_diag(gw_ctx* ctx, const gw_grid* grid, int n_b, int n_occ, const void* psi,
                                   const double* eps_h, double mu, const int32_t* bands_h, int n_n, int n,
                                   const double* tau_h, const double* omega_h, const double* C_h, const double* S_h,
                                   const void* w_tau, int n_chi, const int32_t* fft_index_h, gw_prec prec,
                                   double* sigma_tau_h, double* sigma_iw_h, const double* w_real_h, int n_real,
                                   double* sigma_real_h, void* stream) {
  return sigma_impl(ctx, grid, n_b, n_occ, psi, eps_h, mu, bands_h, n_n, n, tau_h, omega_h, C_h, S_h, w_tau, n_chi,
                    fft_index_h, prec, false, sigma_tau_h, sigma_iw_h, w_real_h, n_real, sigma_real_h,
                    as_stream(stream));
}

extern "C" gw_status gw_sigma_matrix(gw_ctx* ctx, const gw_grid* grid, int n_b, int n_occ, const void* psi,
                                     const double* eps_h, double mu, const int32_t* bands_h, int n_n, int n,
                                     const double* tau_h, const double* omega_h, const double* C_h, const double* S_h,
                                     const void* w_tau, int n_chi, const int32_t* fft_index_h, gw_prec prec,
                                     double* sigma_tau_h, double* sigma_iw_h, void* stream) {
  return sigma_impl(ctx, grid, n_b, n_occ, psi, eps_h, mu, bands_h, n_n, n, tau_h, omega_h, C_h, S_h, w_tau, n_chi,
                    fft_index_h, prec, true, sigma_tau_h, sigma_iw_h, nullptr, 0, nullptr, as_stream(stream));
}

// ------------------------------------------------------------------ plane-wave form of G
//
// Sigma_nn(tau) with G through its plane-wave form (as gw_chi0_omega_pw): per
// tau, M = Dc F Dc^H over the orbitals' plane waves and its column transform
// T(r, g'), W~(r, G') by the column transform of W~(G, G') (Eq. FFTW, first
// step), then per row the kernel that expands W~, G_unocc and G_occ over R',
// forms H = W~ G and transforms H back onto the plane waves (hu, ho);
//   V_n(r) = sum_R' H(r,R') psi_n(R') = sum_g h(r,g) c_n(g)          (c_n = conj(Dc) rows)
// is a GEMM against the Sigma bands' coefficients, and
//   Sigma_unocc_nn(tau) += coef sum_r Re(conj(psi_n(r)) V^unocc_n(r)),  Sigma_occ_nn(-tau) -= ... V^occ,
// as the fused tensor-core pass does (first term of Eq. Sigma_occ_reduce).

namespace gw {

template <typename C>
__global__ void gather_rows_kernel(const C* __restrict__ src, long ld, const int* __restrict__ rows, int len,
                                   C* __restrict__ dst) {
  const long r = blockIdx.y;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < len; j += gridDim.x * blockDim.x)
    dst[r * len + j] = src[(long)rows[r] * ld + j];
}

// acc[n * stride] += coef sum_r Re(conj(psi_{bands[n]}(r)) V[r][n]); CTAs split the rows, FP64 sums.
template <typename C>
__global__ void __launch_bounds__(256) sigma_pw_reduce_kernel(const C* __restrict__ V, int n_n,
                                                              const C* __restrict__ psi, long nr,
                                                              const int* __restrict__ bands, double coef,
                                                              double* __restrict__ acc, int stride) {
  __shared__ double red[8];
  const int n = blockIdx.y;
  const C* pn = psi + (long)bands[n] * nr;
  double s = 0;
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < nr; r += (long)gridDim.x * blockDim.x) {
    const C p = pn[r], v = V[r * n_n + n];
    s += (double)p.x * v.x + (double)p.y * v.y;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < 8; ++w) t += red[w];
    atomicAdd(acc + (long)n * stride, coef * t);
  }
}

}  // namespace gw

extern "C" gw_status gw_sigma_diag_pw(gw_ctx* ctx, const gw_grid* grid, int n_b, int n_occ, const void* psi,
                                      const double* eps_h, double mu, const int32_t* bands_h, int n_n, int n,
                                      const double* tau_h, const double* omega_h, const double* C_h, const double* S_h,
                                      const void* w_tau, int n_chi, const int32_t* fft_index_h, int n_pw,
                                      const int32_t* pw_index_h, gw_prec prec, double* sigma_tau_h,
                                      double* sigma_iw_h, const double* w_real_h, int n_real, double* sigma_real_h,
                                      void* stream) {
  GridInfo g;
  std::vector<int> map, inv;
  std::vector<GreenScales> scales;
  gw_status st = sigma_check(ctx, grid, &g, n_b, n_occ, psi, eps_h, mu, bands_h, n_n, n, tau_h, omega_h, C_h, S_h,
                             w_tau, n_chi, fft_index_h, prec, false, w_real_h, n_real, map, inv, scales);
  if (st) return st;
  if (!sigma_iw_h || (n_real > 0 && !sigma_real_h)) return fail(ctx, GW_ERR_ARG, "NULL output pointer");
  std::vector<int> map_nat, inv_nat;
  if ((st = index_maps(ctx, g, pw_index_h, n_pw, map_nat, inv_nat))) return st;
  std::vector<int> map_neg = map_nat, inv_neg = inv_nat;
  pw_negate(g, map_neg, inv_neg);
  if ((st = check_row_pw_sigma(ctx, g, prec, n_pw, n_chi))) return st;
  cudaStream_t s = as_stream(stream);
  const bool tc = prec == GW_F16X3 || prec == GW_BF16X3;
  const size_t es = csize(prec);
  const GridInfo gp = pw_grid(g, n_pw);
  SigmaTables t;
  int *dmap_neg = nullptr, *dinv_neg = nullptr, *dinv_nat = nullptr;
  double* dnorm = nullptr;
  char *dc = nullptr, *cn = nullptr, *mo = nullptr, *mu_ = nullptr, *to = nullptr, *tu = nullptr, *wg = nullptr;
  char *hu = nullptr, *ho = nullptr, *vu = nullptr, *vo = nullptr, *tmp = nullptr;
  void* tcs = nullptr;
  auto carve = [&](Carver& cv) {
    sigma_carve_tables(cv, g, n_b, n, n_chi, n_n, n_real, false, t);
    dmap_neg = cv.take<int>(n_pw);
    dinv_neg = cv.take<int>(g.nr);
    dinv_nat = cv.take<int>(g.nr);
    dnorm = cv.take<double>(2 * (size_t)n_b);
    dc = cv.take<char>((size_t)n_b * n_pw * es);
    cn = cv.take<char>((size_t)n_n * n_pw * es);
    mo = cv.take<char>((size_t)n_pw * n_pw * es);
    mu_ = cv.take<char>((size_t)n_pw * n_pw * es);
    to = cv.take<char>((size_t)g.nr * n_pw * es);
    tu = cv.take<char>((size_t)g.nr * n_pw * es);
    wg = cv.take<char>((size_t)g.nr * n_chi * es);
    hu = cv.take<char>((size_t)g.nr * n_pw * es);
    ho = cv.take<char>((size_t)g.nr * n_pw * es);
    vu = cv.take<char>((size_t)g.nr * n_n * es);
    vo = cv.take<char>((size_t)g.nr * n_n * es);
    tmp = row_two_pass(g, prec) && is_fp64(prec) ? cv.take<char>((size_t)n_b * g.nr * es) : nullptr;
    tcs = tc ? cv.take<char>(tc_scratch_bytes(gp, n_b, n_occ, n_pw, false)) : nullptr;
  };
  {
    Carver probe(nullptr);
    carve(probe);
    if ((st = reserve(ctx, probe.off))) return st;
  }
  Carver cv(ctx->arena);
  carve(cv);
  if ((st = sigma_upload_tables(ctx, t, g, n_b, n, n_chi, map, inv, bands_h, n_n, scales, C_h, S_h, omega_h, w_real_h,
                                n_real, prec, s)))
    return st;
  if ((st = upload(ctx, dmap_neg, map_neg.data(), sizeof(int) * n_pw, s))) return st;
  if ((st = upload(ctx, dinv_neg, inv_neg.data(), sizeof(int) * g.nr, s))) return st;
  if ((st = upload(ctx, dinv_nat, inv_nat.data(), sizeof(int) * g.nr, s))) return st;
  if ((st = pw_coefficients(ctx, g, prec, psi, n_b, n_pw, dmap_neg, dinv_neg, dc, dnorm, tmp, s))) return st;
  {
    const dim3 gg((n_pw + 255) / 256, n_n);
    if (is_fp64(prec)) gather_rows_kernel<<<gg, 256, 0, s>>>((const double2*)dc, n_pw, t.bands, n_pw, (double2*)cn);
    else gather_rows_kernel<<<gg, 256, 0, s>>>((const float2*)dc, n_pw, t.bands, n_pw, (float2*)cn);
    if ((st = launch_check(ctx, "gather_rows_kernel"))) return st;
  }
  const size_t acc_elems = (size_t)n_n * n;
  if ((st = cuda_check(ctx, cudaMemsetAsync(t.acc2, 0, sizeof(double2) * acc_elems, s), "memset"))) return st;
  double* acc_u = reinterpret_cast<double*>(t.acc2);
  double* acc_o = acc_u + (size_t)n_n * n;
  const double coef = g.dv * g.dv / g.volume;   // dV^2 and the 1/Omega of Eq. FFTW
  bool first = true;
  for (int j = 0; j < n; ++j) {
    const char* sj = t.scale + (size_t)j * n_b * 8;
    if (tc) {
      st = tc_green_rows(ctx, gp, n_b, n_occ, dc, scales[j], 0, n_pw, prec, mo, mu_, tcs, first, s,
                         reinterpret_cast<const float*>(sj));
      first = false;
    } else {
      st = green_rows(ctx, gp, n_b, n_occ, dc, sj, scales[j], 0, n_pw, prec, mo, mu_, s);
    }
    if (st) return st;
    for (int part = 0; part < 2; ++part) {
      char* m = part ? mu_ : mo;
      char* tt = part ? tu : to;
      if ((st = launch_col_line(ctx, g, prec, +1, 1, m, n_pw, tt, n_pw, n_pw, dinv_neg, 1.0, s))) return st;
      if ((st = launch_col_plane(ctx, g, prec, +1, tt, n_pw, n_pw, 1.0, s))) return st;
    }
    const char* wj = static_cast<const char*>(w_tau) + (size_t)j * n_chi * n_chi * es;
    if ((st = launch_col_line(ctx, g, prec, +1, 1, wj, n_chi, wg, n_chi, n_chi, t.inv, 1.0, s))) return st;
    if ((st = launch_col_plane(ctx, g, prec, +1, wg, n_chi, n_chi, 1.0, s))) return st;
    if ((st = launch_row_pw_sigma(ctx, g, prec, tu, to, n_pw, wg, n_chi, hu, ho, n_pw, dinv_neg, dinv_nat, n_pw, t.inv,
                                  n_chi, g.nr, s)))
      return st;
    for (int part = 0; part < 2; ++part) {
      GemmArgs a{};
      a.M = g.nr;
      a.N = n_n;
      a.K = n_pw;
      a.alpha_re = 1.0;
      a.A = part ? ho : hu;
      a.lda = n_pw;
      a.a_km = 0;
      a.B = cn;
      a.ldb = n_pw;
      a.b_nk = 1;
      a.b_conj = true;                 // c_n(g) = conj(Dc[band][g])
      a.C = part ? vo : vu;
      a.ldc = n_n;
      if ((st = launch_gemm(ctx, prec, a, s))) return st;
      const dim3 gr((unsigned)std::min<long>((g.nr + 255) / 256, 64), n_n);
      double* acc = (part ? acc_o : acc_u) + j;
      const double cf = part ? -coef : coef;
      if (is_fp64(prec))
        sigma_pw_reduce_kernel<<<gr, 256, 0, s>>>((const double2*)a.C, n_n, (const double2*)psi, g.nr, t.bands, cf,
                                                  acc, n);
      else
        sigma_pw_reduce_kernel<<<gr, 256, 0, s>>>((const float2*)a.C, n_n, (const float2*)psi, g.nr, t.bands, cf,
                                                  acc, n);
      if ((st = launch_check(ctx, "sigma_pw_reduce_kernel"))) return st;
    }
  }
  if ((st = sigma_finish_launch(ctx, acc_u, n_n, n, t.tab, n_real, t.out, t.stat, s))) return st;
  if (tc && (st = tc_check(ctx, tcs, s))) return st;
  return sigma_fetch(ctx, acc_u, n_n, n, n_real, t.out, t.stat, bands_h, sigma_tau_h, sigma_iw_h, sigma_real_h, s);
}

extern "C" gw_status gw_qp_energies(gw_ctx* ctx, int n_n, int n, const double* omega_h, const double* sigma_iw_h,
                                    const double* eps_h, double mu, const double* vstat_h, int n_w, const double* w_h,
                                    double* e_qp_h, double* z_h, double* sigma_eps_h, double* dsigma_h,
                                    double* spectral_h, void* stream) {
  if (!ctx) return fail(nullptr, GW_ERR_ARG, "ctx is NULL");
  if (n < 1 || n > kMaxN) return fail(ctx, GW_ERR_SHAPE, "need 1 <= n <= 32");
  if (n_n < 1 || n_n > (1 << 20)) return fail(ctx, GW_ERR_SHAPE, "need 1 <= n_n <= 2^20");
  if (n_w < 0 || n_w > (1 << 24)) return fail(ctx, GW_ERR_SHAPE, "need 0 <= n_w <= 2^24");
  if (!omega_h || !sigma_iw_h || !eps_h || !vstat_h || !e_qp_h) return fail(ctx, GW_ERR_ARG, "NULL pointer");
  if (n_w > 0 && (!w_h || !spectral_h)) return fail(ctx, GW_ERR_ARG, "n_w > 0 needs w_h and spectral_h");
  for (int k = 0; k < n; ++k)
    if (!(omega_h[k] > 0)) return fail(ctx, GW_ERR_ARG, "omega must be > 0");
  for (int k = 1; k < n; ++k)
    if (!(omega_h[k] != omega_h[k - 1])) return fail(ctx, GW_ERR_ARG, "omega nodes must be distinct");
  cudaStream_t s = as_stream(stream);
  const size_t nw1 = std::max(n_w, 1);
  // layout: Sigma(i omega), coefficients, omega, eps, v, w, E, Z, Sigma(eps), dSigma, A, status
  auto carve = [&](Carver& c, double2** sig, double2** cf, double** om, double** ep, double** vs, double** w,
                   double** e, double** z, double2** se, double2** ds, double** sp, int** stat) {
    *sig = c.take<double2>((size_t)n_n * n);
    *cf = c.take<double2>((size_t)n_n * n);
    *om = c.take<double>(n);
    *ep = c.take<double>(n_n);
    *vs = c.take<double>(n_n);
    *w = c.take<double>(nw1);
    *e = c.take<double>(n_n);
    *z = c.take<double>(n_n);
    *se = c.take<double2>(n_n);
    *ds = c.take<double2>(n_n);
    *sp = c.take<double>((size_t)n_n * nw1);
    *stat = c.take<int>(n_n);
  };
  double2 *dsig, *dcf, *dse, *dds;
  double *dom, *deps, *dvs, *dw, *de, *dz, *dsp;
  int* dstat;
  Carver probe(nullptr);
  carve(probe, &dsig, &dcf, &dom, &deps, &dvs, &dw, &de, &dz, &dse, &dds, &dsp, &dstat);
  gw_status st;
  if ((st = reserve(ctx, probe.off))) return st;
  Carver cv(ctx->arena);
  carve(cv, &dsig, &dcf, &dom, &deps, &dvs, &dw, &de, &dz, &dse, &dds, &dsp, &dstat);
  if ((st = upload(ctx, dsig, sigma_iw_h, sizeof(double2) * n_n * n, s))) return st;
  if ((st = upload(ctx, dom, omega_h, sizeof(double) * n, s))) return st;
  if ((st = upload(ctx, deps, eps_h, sizeof(double) * n_n, s))) return st;
  if ((st = upload(ctx, dvs, vstat_h, sizeof(double) * n_n, s))) return st;
  if (n_w > 0 && (st = upload(ctx, dw, w_h, sizeof(double) * n_w, s))) return st;
  qp_coeff_kernel<<<(n_n + 63) / 64, 64, 0, s>>>(dsig, dom, n_n, n, dcf, dstat);
  if ((st = launch_check(ctx, "qp_coeff_kernel"))) return st;
  const long pts = (long)n_n * (n_w + 1);
  qp_eval_kernel<<<(unsigned)((pts + 127) / 128), 128, 0, s>>>(dcf, dom, n_n, n, deps, dvs, mu, dw, n_w, de, dz, dse,
                                                              dds, dsp, dstat);
  if ((st = launch_check(ctx, "qp_eval_kernel"))) return st;
  std::vector<double> h_e(n_n), h_z(n_n), h_sp(n_w > 0 ? (size_t)n_n * n_w : 0);
  std::vector<double2> h_se(n_n), h_ds(n_n);
  std::vector<int> h_stat(n_n);
  auto d2h = [&](void* dst, const void* src, size_t bytes) {
    return cuda_check(ctx, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s), "copy qp");
  };
  if ((st = d2h(h_e.data(), de, sizeof(double) * n_n))) return st;
  if ((st = d2h(h_z.data(), dz, sizeof(double) * n_n))) return st;
  if ((st = d2h(h_se.data(), dse, sizeof(double2) * n_n))) return st;
  if ((st = d2h(h_ds.data(), dds, sizeof(double2) * n_n))) return st;
  if (n_w > 0 && (st = d2h(h_sp.data(), dsp, sizeof(double) * n_n * n_w))) return st;
  if ((st = d2h(h_stat.data(), dstat, sizeof(int) * n_n))) return st;
  if ((st = cuda_check(ctx, cudaStreamSynchronize(s), "qp sync"))) return st;
  std::memcpy(e_qp_h, h_e.data(), sizeof(double) * n_n);
  if (z_h) std::memcpy(z_h, h_z.data(), sizeof(double) * n_n);
  if (sigma_eps_h) std::memcpy(sigma_eps_h, h_se.data(), sizeof(double2) * n_n);
  if (dsigma_h) std::memcpy(dsigma_h, h_ds.data(), sizeof(double2) * n_n);
  if (n_w > 0) std::memcpy(spectral_h, h_sp.data(), sizeof(double) * n_n * n_w);
  for (int b = 0; b < n_n; ++b)
    if (h_stat[b])
      return fail(ctx, GW_ERR_NUMERIC, std::string(h_stat[b] & 1 ? "Thiele coefficients broke down" :
                                                    h_stat[b] & 2 ? "QP equation not finite" :
                                                                    "Thiele evaluation broke down") +
                                            " for entry " + std::to_string(b));
  return GW_OK;
}

extern "C" gw_status gw_sigma_to_tau(gw_ctx* ctx, int n_n, int n, int matrix, const double* Cinv_h,
                                     const double* Sinv_h, const double* sigma_iw_h, double* sigma_tau_h,
                                     void* stream) {
  if (!ctx) return fail(nullptr, GW_ERR_ARG, "ctx is NULL");
  if (n < 1 || n > kMaxN) return fail(ctx, GW_ERR_SHAPE, "need 1 <= n <= 32");
  if (n_n < 1 || n_n > (matrix ? 4096 : (1 << 22))) return fail(ctx, GW_ERR_SHAPE, "n_n out of range");
  if (matrix != 0 && matrix != 1) return fail(ctx, GW_ERR_ARG, "matrix must be 0 or 1");
  if (!Cinv_h || !Sinv_h || !sigma_iw_h || !sigma_tau_h) return fail(ctx, GW_ERR_ARG, "NULL pointer");
  cudaStream_t s = as_stream(stream);
  const long E = matrix ? (long)n_n * n_n : n_n;
  const size_t cplx = (size_t)E * n;
  auto carve = [&](Carver& c, double** M, double2** sig, double2** herm, double2** anti, double2** sc, double2** ss,
                   double2** out) {
    *M = c.take<double>(2 * (size_t)n * n);      // Cinv, then -Sinv (the sine kernel multiplies by +i)
    *sig = c.take<double2>(cplx);
    *herm = c.take<double2>(cplx);
    *anti = c.take<double2>(cplx);
    *sc = c.take<double2>(cplx);
    *ss = c.take<double2>(cplx);
    *out = c.take<double2>(2 * cplx);           // [2][E][n], complex or (diagonal) real
  };
  double* dM;
  double2 *dsig, *herm, *anti, *sc, *ss, *dout;
  Carver probe(nullptr);
  carve(probe, &dM, &dsig, &herm, &anti, &sc, &ss, &dout);
  gw_status st;
  if ((st = reserve(ctx, probe.off))) return st;
  Carver cv(ctx->arena);
  carve(cv, &dM, &dsig, &herm, &anti, &sc, &ss, &dout);
  std::vector<double> m(2 * (size_t)n * n);
  for (size_t i = 0; i < (size_t)n * n; ++i) {
    m[i] = Cinv_h[i];
    m[(size_t)n * n + i] = -Sinv_h[i];
  }
  if ((st = upload(ctx, dM, m.data(), sizeof(double) * m.size(), s))) return st;
  if ((st = upload(ctx, dsig, sigma_iw_h, sizeof(double2) * cplx, s))) return st;
  sigma_split_kernel<<<(unsigned)((E + 127) / 128), 128, 0, s>>>(dsig, n_n, n, matrix, herm, anti);
  if ((st = launch_check(ctx, "sigma_split_kernel"))) return st;
  // Eq. INV_CT_FFT on the cosine part, Eq. INV_ST_FFT (-i zeta sin) on the sine part, in FP64
  if ((st = launch_ct(ctx, GW_FP64, false, n, dM, (size_t)E, herm, sc, s, nullptr))) return st;
  if ((st = launch_ct(ctx, GW_FP64, true, n, dM + (size_t)n * n, (size_t)E, anti, ss, s, nullptr))) return st;
  sigma_combine_kernel<<<(unsigned)((cplx + 255) / 256), 256, 0, s>>>(sc, ss, E, n, matrix,
                                                                      reinterpret_cast<double*>(dout));
  if ((st = launch_check(ctx, "sigma_combine_kernel"))) return st;
  const size_t out_bytes = 2 * cplx * (matrix ? sizeof(double2) : sizeof(double));
  std::vector<char> h(out_bytes);
  if ((st = cuda_check(ctx, cudaMemcpyAsync(h.data(), dout, out_bytes, cudaMemcpyDeviceToHost, s), "copy sigma")))
    return st;
  if ((st = cuda_check(ctx, cudaStreamSynchronize(s), "sigma sync"))) return st;
  std::memcpy(sigma_tau_h, h.data(), out_bytes);
  return GW_OK;
}
