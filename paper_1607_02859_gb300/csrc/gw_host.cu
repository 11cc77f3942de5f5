// Context, error handling and the host-side setup of the hot path:
// the G set (Eq. FFTX1 cutoff sphere), the Coulomb kernel (Eq. bareV) and the
// nonuniform cosine/sine transform matrices (Eqs. CT_FFT, cos_error_function,
// ST_FFT, sin_error_function, INV_CT_FFT).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <tuple>

#include "gw_common.cuh"

namespace {
thread_local std::string g_orphan_err;
}

namespace gw {

gw_status fail(gw_ctx* ctx, gw_status st, const std::string& msg) {
  if (ctx) ctx->err = msg; else g_orphan_err = msg;
  return st;
}

gw_status cuda_check(gw_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return GW_OK;
  return fail(ctx, e == cudaErrorMemoryAllocation ? GW_ERR_OOM : GW_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

gw_status launch_check(gw_ctx* ctx, const char* what) {
  ctx->launches++;
  return cuda_check(ctx, cudaGetLastError(), what);
}

gw_status reserve(gw_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->arena_bytes) return GW_OK;
  if (ctx->arena) {
    cudaError_t e = cudaFree(ctx->arena);   // implicit device synchronisation
    ctx->arena = nullptr;
    ctx->arena_bytes = 0;
    if (e != cudaSuccess) return cuda_check(ctx, e, "cudaFree(arena)");
  }
  size_t want = (bytes + (size_t(1) << 21) - 1) & ~((size_t(1) << 21) - 1);
  cudaError_t e = cudaMalloc(&ctx->arena, want);
  if (e != cudaSuccess) {
    ctx->arena = nullptr;
    cudaGetLastError();
    return fail(ctx, GW_ERR_OOM, "cannot allocate " + std::to_string(want) + " bytes of scratch");
  }
  ctx->arena_bytes = want;
  return GW_OK;
}

bool fft_len_ok(int n) {
  static const int ok[] = {4, 6, 8, 10, 12, 16, 18, 20, 24, 30, 32, 36, 40, 48};
  for (int v : ok)
    if (v == n) return true;
  return false;
}

gw_status grid_info(gw_ctx* ctx, const gw_grid* g, GridInfo* out) {
  if (!g) return fail(ctx, GW_ERR_ARG, "grid is NULL");
  for (int d = 0; d < 3; ++d)
    if (!fft_len_ok(g->n[d]))
      return fail(ctx, GW_ERR_SHAPE, "grid length " + std::to_string(g->n[d]) +
                                         " not in {4,6,8,10,12,16,18,20,24,30,32,36,40,48}");
  const double* a = g->lattice;
  double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
               a[2] * (a[3] * a[7] - a[4] * a[6]);
  if (!(std::fabs(det) > 0)) return fail(ctx, GW_ERR_ARG, "lattice is singular");
  out->n1 = g->n[0];
  out->n2 = g->n[1];
  out->n3 = g->n[2];
  out->nr = g->n[0] * g->n[1] * g->n[2];
  out->volume = std::fabs(det);
  out->dv = out->volume / out->nr;
  return GW_OK;
}

gw_status check_energies(gw_ctx* ctx, const double* eps, int n_b, int n_occ, double mu) {
  if (!eps) return fail(ctx, GW_ERR_ARG, "eps_h is NULL");
  if (n_occ < 1 || n_occ >= n_b) return fail(ctx, GW_ERR_SHAPE, "need 1 <= n_occ < n_b");
  for (int i = 1; i < n_b; ++i)
    if (!(eps[i] >= eps[i - 1])) return fail(ctx, GW_ERR_ARG, "eps_h not ascending");
  if (!(eps[n_occ - 1] < mu && mu < eps[n_occ]))
    return fail(ctx, GW_ERR_ARG, "mu must lie in the gap: eps[n_occ-1] < mu < eps[n_occ]");
  return GW_OK;
}

static cudaEvent_t take_event(gw_ctx* ctx) {
  if (!ctx->pool.empty()) {
    cudaEvent_t e = ctx->pool.back();
    ctx->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

KTimer::KTimer(gw_ctx* c, int f, double w, cudaStream_t s) : ctx(c), fam(f), work(w), st(s) {
  if (ctx && ctx->timing) {
    a = take_event(ctx);
    if (a) cudaEventRecord(a, st);
  }
}

KTimer::~KTimer() {
  if (!a) return;
  cudaEvent_t b = take_event(ctx);
  if (!b) {
    ctx->pool.push_back(a);
    return;
  }
  cudaEventRecord(b, st);
  ctx->pending.push_back({fam, a, b, work});
}

static void drain_timers(gw_ctx* ctx) {
  for (auto& r : ctx->pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      ctx->tot_ms[r.fam] += ms;
      ctx->tot_work[r.fam] += r.work;
      ctx->tot_n[r.fam] += 1;
    }
    ctx->pool.push_back(r.a);
    ctx->pool.push_back(r.b);
  }
  ctx->pending.clear();
  cudaGetLastError();
}

}  // namespace gw

using namespace gw;

static const char* kFamNames[KF_COUNT] = {"green_tc", "cgemm_tc", "cgemm_simt", "row_fft", "col_fft",
                                          "col_line_ct", "sigma_contract", "ct", "cgemm_exact", "row_pw"};

extern "C" gw_status gw_ctx_set_timing(gw_ctx* ctx, int enabled) {
  if (!ctx) return fail(nullptr, GW_ERR_ARG, "ctx is NULL");
  drain_timers(ctx);
  for (int f = 0; f < KF_COUNT; ++f) {
    ctx->tot_ms[f] = 0;
    ctx->tot_work[f] = 0;
    ctx->tot_n[f] = 0;
  }
  ctx->timing = enabled != 0;
  return GW_OK;
}

extern "C" gw_status gw_ctx_kernel_stats(gw_ctx* ctx, const char* family, unsigned long long* launches, double* ms,
                                         double* work, int* work_is_bytes) {
  if (!ctx || !family) return fail(ctx, GW_ERR_ARG, "NULL argument");
  int f = -1;
  for (int i = 0; i < KF_COUNT; ++i)
    if (std::strcmp(family, kFamNames[i]) == 0) f = i;
  if (f < 0) return fail(ctx, GW_ERR_ARG, std::string("unknown kernel family ") + family);
  drain_timers(ctx);
  if (launches) *launches = ctx->tot_n[f];
  if (ms) *ms = ctx->tot_ms[f];
  if (work) *work = ctx->tot_work[f];
  if (work_is_bytes) *work_is_bytes = (f == KF_GREEN_TC || f == KF_CGEMM_TC || f == KF_CGEMM_SIMT || f == KF_CGEMM_EXACT ||
                                    f == KF_ROW_PW) ? 0 : 1;
  return GW_OK;
}

// ---------------------------------------------------------------------- context

extern "C" gw_status gw_ctx_create(int device, gw_ctx** out) {
  if (!out) return fail(nullptr, GW_ERR_ARG, "out is NULL");
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || device < 0 || device >= count)
    return fail(nullptr, GW_ERR_CUDA, std::string("no CUDA device ") + std::to_string(device) +
                                          (e != cudaSuccess ? std::string(": ") + cudaGetErrorString(e) : ""));
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return fail(nullptr, GW_ERR_CUDA, cudaGetErrorString(e));
  gw_ctx* c = new gw_ctx();
  c->device = device;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  e = cudaMalloc(&c->dflag, 64);
  if (e != cudaSuccess) {
    delete c;
    return fail(nullptr, GW_ERR_OOM, "cannot allocate the status word");
  }
  cudaMemset(c->dflag, 0, 64);
  *out = c;
  return GW_OK;
}

extern "C" gw_status gw_ctx_destroy(gw_ctx* ctx) {
  if (!ctx) return GW_OK;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  drain_timers(ctx);
  for (cudaEvent_t e : ctx->pool) cudaEventDestroy(e);
  if (ctx->arena) cudaFree(ctx->arena);
  if (ctx->dflag) cudaFree(ctx->dflag);
  delete ctx;
  return GW_OK;
}

extern "C" const char* gw_last_error(const gw_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_orphan_err.c_str();
}

extern "C" unsigned long long gw_ctx_launches(const gw_ctx* ctx) { return ctx ? ctx->launches : 0ull; }
extern "C" size_t gw_ctx_scratch_bytes(const gw_ctx* ctx) { return ctx ? ctx->arena_bytes : 0; }

extern "C" gw_status gw_ctx_reserve(gw_ctx* ctx, size_t bytes) {
  if (!ctx) return fail(nullptr, GW_ERR_ARG, "ctx is NULL");
  return reserve(ctx, bytes);
}
extern "C" int gw_version(void) { return 101; }

// ---------------------------------------------------------------------- G set

extern "C" gw_status gw_g_set(const gw_grid* grid, int n_chi, int32_t* gvec_h, int32_t* fft_index_h) {
  GridInfo gi;
  gw_status st = grid_info(nullptr, grid, &gi);
  if (st) return st;
  if (n_chi < 1 || n_chi > gi.nr) return fail(nullptr, GW_ERR_SHAPE, "need 1 <= n_chi <= N_r");
  if (!gvec_h) return fail(nullptr, GW_ERR_ARG, "gvec_h is NULL");
  std::vector<std::tuple<int, int, int, int>> pts;
  pts.reserve(gi.nr);
  const int n[3] = {gi.n1, gi.n2, gi.n3};
  for (int a = -(n[0] / 2); a < n[0] - n[0] / 2; ++a)
    for (int b = -(n[1] / 2); b < n[1] - n[1] / 2; ++b)
      for (int c = -(n[2] / 2); c < n[2] - n[2] / 2; ++c) pts.emplace_back(a * a + b * b + c * c, a, b, c);
  std::sort(pts.begin(), pts.end());
  for (int j = 0; j < n_chi; ++j) {
    int g[3] = {std::get<1>(pts[j]), std::get<2>(pts[j]), std::get<3>(pts[j])};
    for (int d = 0; d < 3; ++d) gvec_h[3 * j + d] = g[d];
    if (fft_index_h) {
      int m[3];
      for (int d = 0; d < 3; ++d) m[d] = ((g[d] % n[d]) + n[d]) % n[d];
      fft_index_h[j] = (m[0] * n[1] + m[1]) * n[2] + m[2];
    }
  }
  return GW_OK;
}

extern "C" gw_status gw_coulomb_sqrt(const gw_grid* grid, const int32_t* gvec_h, int n_chi, double* vhalf_h) {
  GridInfo gi;
  gw_status st = grid_info(nullptr, grid, &gi);
  if (st) return st;
  if (!gvec_h || !vhalf_h) return fail(nullptr, GW_ERR_ARG, "NULL pointer");
  // reciprocal vectors b_d = 2 pi (a_e x a_f) / (a_d . (a_e x a_f))
  const double* a = grid->lattice;
  double b[3][3];
  const double vol = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                     a[2] * (a[3] * a[7] - a[4] * a[6]);
  for (int d = 0; d < 3; ++d) {
    const double* u = a + 3 * ((d + 1) % 3);
    const double* v = a + 3 * ((d + 2) % 3);
    b[d][0] = 2 * kPi * (u[1] * v[2] - u[2] * v[1]) / vol;
    b[d][1] = 2 * kPi * (u[2] * v[0] - u[0] * v[2]) / vol;
    b[d][2] = 2 * kPi * (u[0] * v[1] - u[1] * v[0]) / vol;
  }
  for (int j = 0; j < n_chi; ++j) {
    double gc[3] = {0, 0, 0};
    for (int d = 0; d < 3; ++d)
      for (int e = 0; e < 3; ++e) gc[e] += gvec_h[3 * j + d] * b[d][e];
    double g2 = gc[0] * gc[0] + gc[1] * gc[1] + gc[2] * gc[2];
    vhalf_h[j] = g2 > 0 ? std::sqrt(4 * kPi) / std::sqrt(g2) : 0.0;
  }
  return GW_OK;
}

// ---------------------------------------------------------------------- CT/ST fit

namespace {

// Least squares min |A x - b|^2 for A [m][n] (row-major, m >= n) by Householder QR.
bool householder_lstsq(std::vector<double>& A, std::vector<double>& b, int m, int n, std::vector<double>& x) {
  for (int j = 0; j < n; ++j) {
    double norm = 0;
    for (int i = j; i < m; ++i) norm += A[(size_t)i * n + j] * A[(size_t)i * n + j];
    norm = std::sqrt(norm);
    if (norm == 0) return false;
    double alpha = A[(size_t)j * n + j] > 0 ? -norm : norm;
    // v = a_j - alpha e_j, stored in place below the diagonal
    A[(size_t)j * n + j] -= alpha;
    double vnorm2 = 0;
    for (int i = j; i < m; ++i) vnorm2 += A[(size_t)i * n + j] * A[(size_t)i * n + j];
    if (vnorm2 > 0) {
      for (int c = j + 1; c < n; ++c) {
        double dot = 0;
        for (int i = j; i < m; ++i) dot += A[(size_t)i * n + j] * A[(size_t)i * n + c];
        double f = 2 * dot / vnorm2;
        for (int i = j; i < m; ++i) A[(size_t)i * n + c] -= f * A[(size_t)i * n + j];
      }
      double dot = 0;
      for (int i = j; i < m; ++i) dot += A[(size_t)i * n + j] * b[i];
      double f = 2 * dot / vnorm2;
      for (int i = j; i < m; ++i) b[i] -= f * A[(size_t)i * n + j];
    }
    A[(size_t)j * n + j] = alpha;   // R diagonal
  }
  x.assign(n, 0.0);
  for (int j = n - 1; j >= 0; --j) {
    double s = b[j];
    for (int c = j + 1; c < n; ++c) s -= A[(size_t)j * n + c] * x[c];
    x[j] = s / A[(size_t)j * n + j];
  }
  return true;
}

// Fit rows of gamma (kind 0) or lambda (kind 1); returns the largest relative error.
bool fit_rows(int n, const double* tau, const double* omega, double x_min, double x_max, int n_x,
              double ridge, int kind, std::vector<double>& W, double* worst) {
  std::vector<double> xs(n_x);
  const double lmin = std::log(x_min), lmax = std::log(x_max);
  for (int i = 0; i < n_x; ++i) xs[i] = n_x == 1 ? x_min : std::exp(lmin + (lmax - lmin) * i / (n_x - 1));
  W.assign((size_t)n * n, 0.0);
  *worst = 0;
  const int m = n_x + n;
  std::vector<double> A((size_t)m * n), b(m), A0((size_t)n_x * n), x;
  for (int k = 0; k < n; ++k) {
    const double w = omega[k];
    for (int i = 0; i < n_x; ++i) {
      const double xv = xs[i];
      const double target = (kind == 0 ? 2 * xv : 2 * w) / (xv * xv + w * w);
      for (int j = 0; j < n; ++j) {
        const double trig = kind == 0 ? std::cos(w * tau[j]) : std::sin(w * tau[j]);
        A0[(size_t)i * n + j] = trig * std::exp(-xv * tau[j]) / target;
      }
    }
    std::copy(A0.begin(), A0.end(), A.begin());
    std::fill(A.begin() + (size_t)n_x * n, A.end(), 0.0);
    for (int j = 0; j < n; ++j) A[(size_t)(n_x + j) * n + j] = ridge * std::sqrt((double)n_x);
    for (int i = 0; i < m; ++i) b[i] = i < n_x ? 1.0 : 0.0;
    if (!householder_lstsq(A, b, m, n, x)) return false;
    for (int j = 0; j < n; ++j) W[(size_t)k * n + j] = x[j];
    for (int i = 0; i < n_x; ++i) {
      double r = -1.0;
      for (int j = 0; j < n; ++j) r += A0[(size_t)i * n + j] * x[j];
      *worst = std::max(*worst, std::fabs(r));
    }
  }
  return true;
}

// Gauss-Jordan inverse with partial pivoting.
bool invert(int n, const double* M, double* out) {
  std::vector<double> a(M, M + (size_t)n * n), inv((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[(size_t)r * n + c]) > std::fabs(a[(size_t)p * n + c])) p = r;
    if (a[(size_t)p * n + c] == 0) return false;
    if (p != c)
      for (int k = 0; k < n; ++k) {
        std::swap(a[(size_t)p * n + k], a[(size_t)c * n + k]);
        std::swap(inv[(size_t)p * n + k], inv[(size_t)c * n + k]);
      }
    const double d = a[(size_t)c * n + c];
    for (int k = 0; k < n; ++k) {
      a[(size_t)c * n + k] /= d;
      inv[(size_t)c * n + k] /= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = a[(size_t)r * n + c];
      if (f == 0) continue;
      for (int k = 0; k < n; ++k) {
        a[(size_t)r * n + k] -= f * a[(size_t)c * n + k];
        inv[(size_t)r * n + k] -= f * inv[(size_t)c * n + k];
      }
    }
  }
  std::copy(inv.begin(), inv.end(), out);
  return true;
}

}  // namespace

extern "C" gw_status gw_invert_transform(int n, const double* M_h, double* Minv_h) {
  if (n < 1 || n > 64) return fail(nullptr, GW_ERR_SHAPE, "need 1 <= n <= 64");
  if (!M_h || !Minv_h) return fail(nullptr, GW_ERR_ARG, "NULL pointer");
  if (!invert(n, M_h, Minv_h)) return fail(nullptr, GW_ERR_NUMERIC, "matrix is singular");
  return GW_OK;
}

extern "C" gw_status gw_fit_transform(int n, const double* tau_h, const double* omega_h, double x_min,
                                      double x_max, int n_x, double ridge, double* C_h, double* S_h,
                                      double* Cinv_h, double* fit_err_h) {
  if (n < 1 || n > 64) return fail(nullptr, GW_ERR_SHAPE, "need 1 <= n <= 64 time points");
  if (!tau_h || !omega_h) return fail(nullptr, GW_ERR_ARG, "tau_h/omega_h NULL");
  if (!(x_min > 0 && x_max > x_min) || n_x < n || !(ridge >= 0))
    return fail(nullptr, GW_ERR_ARG, "need 0 < x_min < x_max, n_x >= n, ridge >= 0");
  for (int j = 0; j < n; ++j)
    if (!(tau_h[j] > 0) || !(omega_h[j] > 0)) return fail(nullptr, GW_ERR_ARG, "tau and omega must be > 0");
  std::vector<double> gam, lam;
  double ec = 0, es = 0;
  if (!fit_rows(n, tau_h, omega_h, x_min, x_max, n_x, ridge, 0, gam, &ec) ||
      !fit_rows(n, tau_h, omega_h, x_min, x_max, n_x, ridge, 1, lam, &es))
    return fail(nullptr, GW_ERR_NUMERIC, "rank-deficient weight fit");
  std::vector<double> C((size_t)n * n), S((size_t)n * n);
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j) {
      C[(size_t)k * n + j] = gam[(size_t)k * n + j] * std::cos(omega_h[k] * tau_h[j]);
      S[(size_t)k * n + j] = lam[(size_t)k * n + j] * std::sin(omega_h[k] * tau_h[j]);
    }
  if (C_h) std::copy(C.begin(), C.end(), C_h);
  if (S_h) std::copy(S.begin(), S.end(), S_h);
  if (Cinv_h && !invert(n, C.data(), Cinv_h)) return fail(nullptr, GW_ERR_NUMERIC, "C is singular");
  if (fit_err_h) {
    fit_err_h[0] = ec;
    fit_err_h[1] = es;
  }
  return GW_OK;
}
