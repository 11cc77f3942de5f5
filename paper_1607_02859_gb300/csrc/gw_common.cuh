// Internal declarations shared by the libgw translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/gw.h"

// Kernel families whose launches can be timed individually (gw_ctx_set_timing).
enum gw_kfam { KF_GREEN_TC = 0, KF_CGEMM_TC, KF_CGEMM_SIMT, KF_ROW_FFT, KF_COL_FFT, KF_COL_LINE_CT, KF_SIGMA, KF_CT,
               KF_CGEMM_EXACT, KF_ROW_PW,
               KF_COUNT };

struct gw_krec {
  int fam;
  cudaEvent_t a, b;
  double work;
};

struct gw_ctx {
  int device = 0;
  std::string err;
  void* arena = nullptr;       // grow-only device scratch
  size_t arena_bytes = 0;
  unsigned long long launches = 0;
  int* dflag = nullptr;        // device status word written by kernels
  int num_sms = 0;
  // opt-in per-launch timing of the main kernels
  bool timing = false;
  std::vector<gw_krec> pending;
  std::vector<cudaEvent_t> pool;
  double tot_ms[KF_COUNT] = {0};
  double tot_work[KF_COUNT] = {0};
  unsigned long long tot_n[KF_COUNT] = {0};
};

namespace gw {

// ------------------------------------------------------------------ errors
gw_status fail(gw_ctx* ctx, gw_status st, const std::string& msg);
gw_status cuda_check(gw_ctx* ctx, cudaError_t e, const char* what);
gw_status launch_check(gw_ctx* ctx, const char* what);
gw_status reserve(gw_ctx* ctx, size_t bytes);   // ensure arena >= bytes (syncs if it grows)

// Carves aligned pieces out of the context arena.
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + off);
    off += count * sizeof(T);
    return p;
  }
  static size_t round(size_t b) { return (b + 255) & ~size_t(255); }
};

inline cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

// Brackets one kernel launch with CUDA events on its stream when the context's
// timing is on; `work` is the launch's algorithmic flops (GEMMs) or bytes.
struct KTimer {
  gw_ctx* ctx;
  int fam;
  double work;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  KTimer(gw_ctx* c, int f, double w, cudaStream_t s);
  ~KTimer();
};

// Algorithmic flops of a complex GEMM (8 per complex multiply-add), counting
// only the computed lower triangle for tri = 1 and, for tri = 2 (X^H X with X
// lower, K = N), only the nonzero terms.
inline double gemm_flops(int M, int N, int K, int tri) {
  if (tri == 0) return 8.0 * M * (double)N * K;
  double s = 0;
  for (int m = 0; m < M; ++m) {
    const double cols = m + 1 < N ? m + 1 : N;
    s += tri == 1 ? cols * K : cols * (double)(K - m > 0 ? K - m : 0);
  }
  return 8.0 * s;
}
inline bool is_fp64(gw_prec p) { return p == GW_FP64; }
inline size_t csize(gw_prec p) { return is_fp64(p) ? 16 : 8; }
inline bool valid_prec(int p) { return p >= GW_FP64 && p <= GW_BF16X3; }

// ------------------------------------------------------------------ grid facts
struct GridInfo {
  int n1, n2, n3, nr;
  double volume, dv;
};
gw_status grid_info(gw_ctx* ctx, const gw_grid* g, GridInfo* out);
bool fft_len_ok(int n);
gw_status check_energies(gw_ctx* ctx, const double* eps, int n_b, int n_occ, double mu);

// ------------------------------------------------------------------ complex math
template <typename T> struct cpx;
template <> struct cpx<float> { using t = float2; };
template <> struct cpx<double> { using t = double2; };

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {  // a * conj(b)
  return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { return mk(a.x, -a.y); }
template <typename C> __host__ __device__ __forceinline__ C cmuli(C a) { return mk(-a.y, a.x); }  // i*a
template <typename C, typename R> __host__ __device__ __forceinline__ C cscale(C a, R s) {
  return mk(a.x * s, a.y * s);
}

// ------------------------------------------------------------------ compile-time trig
// sin/cos of 2 pi m / n from their Taylor series (argument reduced to [-pi, pi]);
// 40 terms put the truncation far below double rounding.  Only used for FFT
// twiddle constants that the compiler folds into immediates.
constexpr double kPi = 3.14159265358979323846264338327950288;
__host__ __device__ constexpr double taylor_sin(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 40; ++k) {
    term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 40; ++k) {
    term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double cos2pi(int m, int n) {
  int mm = ((m % n) + n) % n;
  double x = 2.0 * kPi * mm / n;
  if (x > kPi) x -= 2.0 * kPi;
  return taylor_cos(x);
}
__host__ __device__ constexpr double sin2pi(int m, int n) {
  int mm = ((m % n) + n) % n;
  double x = 2.0 * kPi * mm / n;
  if (x > kPi) x -= 2.0 * kPi;
  return taylor_sin(x);
}

template <int N, int DIR>
struct Twiddle {
  double c[N], s[N];
  constexpr Twiddle() : c(), s() {
    for (int m = 0; m < N; ++m) {
      c[m] = cos2pi(m, N);
      s[m] = DIR * sin2pi(m, N);
    }
  }
};

// ------------------------------------------------------------------ register FFTs
// X[k] = sum_j x[j] exp(DIR * 2 pi i j k / N), in place on a register array.
__host__ __device__ constexpr int first_factor(int n) {
  return n % 4 == 0 ? 4 : (n % 2 == 0 ? 2 : (n % 3 == 0 ? 3 : 5));
}

template <int P, int DIR>
struct Butterfly;

template <int DIR>
struct Butterfly<2, DIR> {
  template <typename C> __device__ __forceinline__ static void run(C* x) {
    C a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
  }
};

template <int DIR>
struct Butterfly<3, DIR> {
  template <typename C> __device__ __forceinline__ static void run(C* x) {
    using R = decltype(x[0].x);
    constexpr double s3 = 0.86602540378443864676372317075293618;
    C a = x[0], b = x[1], c = x[2];
    C t = cadd(b, c);
    C m = csub(a, cscale(t, R(0.5)));
    C d = cscale(csub(b, c), R(DIR * s3));
    x[0] = cadd(a, t);
    x[1] = cadd(m, cmuli(d));
    x[2] = csub(m, cmuli(d));
  }
};

template <int DIR>
struct Butterfly<4, DIR> {
  template <typename C> __device__ __forceinline__ static void run(C* x) {
    C a = x[0], b = x[1], c = x[2], d = x[3];
    C s0 = cadd(a, c), d0 = csub(a, c);
    C s1 = cadd(b, d), d1 = csub(b, d);
    C rot = DIR > 0 ? cmuli(d1) : cconj(cmuli(cconj(d1)));   // DIR * i * d1
    x[0] = cadd(s0, s1);
    x[2] = csub(s0, s1);
    x[1] = cadd(d0, rot);
    x[3] = csub(d0, rot);
  }
};

template <int DIR>
struct Butterfly<5, DIR> {
  template <typename C> __device__ __forceinline__ static void run(C* x) {
    using R = decltype(x[0].x);
    constexpr double c1 = cos2pi(1, 5), c2 = cos2pi(2, 5);
    constexpr double s1 = sin2pi(1, 5), s2 = sin2pi(2, 5);
    C a = x[0];
    C t1 = cadd(x[1], x[4]), t2 = cadd(x[2], x[3]);
    C t3 = csub(x[1], x[4]), t4 = csub(x[2], x[3]);
    C r1 = cadd(a, cadd(cscale(t1, R(c1)), cscale(t2, R(c2))));
    C r2 = cadd(a, cadd(cscale(t1, R(c2)), cscale(t2, R(c1))));
    C i1 = cscale(cadd(cscale(t3, R(s1)), cscale(t4, R(s2))), R(DIR));
    C i2 = cscale(csub(cscale(t3, R(s2)), cscale(t4, R(s1))), R(DIR));
    x[0] = cadd(a, cadd(t1, t2));
    x[1] = cadd(r1, cmuli(i1));
    x[4] = csub(r1, cmuli(i1));
    x[2] = cadd(r2, cmuli(i2));
    x[3] = csub(r2, cmuli(i2));
  }
};

template <int N, int DIR>
struct RegFFT {
  template <typename C> __device__ __forceinline__ static void run(C* x) {
    using R = decltype(x[0].x);
    constexpr int P = first_factor(N);
    constexpr int Q = N / P;
    if constexpr (Q == 1) {
      Butterfly<P, DIR>::run(x);
    } else {
      constexpr Twiddle<N, DIR> tw{};
      C y[N];
#pragma unroll
      for (int j1 = 0; j1 < P; ++j1)
#pragma unroll
        for (int j2 = 0; j2 < Q; ++j2) y[j1 * Q + j2] = x[P * j2 + j1];
#pragma unroll
      for (int j1 = 0; j1 < P; ++j1) RegFFT<Q, DIR>::run(y + j1 * Q);
#pragma unroll
      for (int j1 = 1; j1 < P; ++j1)
#pragma unroll
        for (int k1 = 1; k1 < Q; ++k1) {
          const int m = (j1 * k1) % N;
          y[j1 * Q + k1] = cmul(y[j1 * Q + k1], mk(R(tw.c[m]), R(tw.s[m])));
        }
#pragma unroll
      for (int k1 = 0; k1 < Q; ++k1) {
        C z[P];
#pragma unroll
        for (int j1 = 0; j1 < P; ++j1) z[j1] = y[j1 * Q + k1];
        Butterfly<P, DIR>::run(z);
#pragma unroll
        for (int k2 = 0; k2 < P; ++k2) x[k1 + Q * k2] = z[k2];
      }
    }
  }
};

// Grids with compiled FFT kernels (each kernel is specialised on its lengths so
// that the register FFTs are fully unrolled).  Other grids get GW_ERR_UNSUPPORTED.
#define GW_GRIDS(X) \
  X(4, 4, 4) X(6, 6, 6) X(6, 4, 6) X(8, 8, 8) X(8, 6, 10) X(12, 12, 12) X(16, 16, 16) X(20, 20, 20) X(24, 24, 24) X(36, 36, 36) X(48, 48, 48)
bool grid_supported(int n1, int n2, int n3);

}  // namespace gw
