// Batched evaluation of many uneven systems as one CUDA-graph launch (the
// systems layer of the serving and batching forms; the paper has no
// counterpart).  For every system the whole hot path of Fig. 1 runs:
//   chi0(i omega)  (Eqs. Green_occ/unocc, chi_rr, FFTX1, FFTX2, CTX)
//   W~(i omega)    (Eqs. die, W_correlated; optional refinement)
//   W~(i tau)      (Eq. CT_W)
//   Sigma_nn(i omega) and its Thiele coefficients (Eqs. Sigma_rr, Sigma_occ_reduce,
//                  cos_sin_sigma1/2, pade1, pade2)
// gw_batch_plan does every piece of host work once -- validation, tables,
// weights, uploads, the context arena at its largest need -- and then records
// the kernels of all systems, in order, on a private stream into one CUDA
// graph; gw_batch_launch replays that graph (no host work, no host-device
// copy), gw_batch_wait reads the results and the per-system status words.
// The systems share the context arena, so they run one after the other inside
// the graph; each keeps its own tables, results and status.
#include <chrono>
#include <cstring>
#include <thread>

#include "gw_kernels.h"
#include "gw_tc.h"

using namespace gw;

namespace {

constexpr int kStatusInts = 16;   // per system: ctx flags [0..8), chi0 tensor words [8..10), sigma tensor words [10..12)

struct BatchSys {
  gw_batch_system in;            // the caller's description (pointers into its memory)
  GridInfo g{};
  gw_chi0_plan* chi0 = nullptr;
  std::vector<GreenScales> scales;
  std::vector<float> ict32;      // inverse CT weights as FP32 hi/lo (kernel parameters)
  double* dvh = nullptr;         // v^1/2 on the device
  double* dict = nullptr;        // inverse CT weights on the device (general path)
  SigmaTables st{};
  int* status = nullptr;         // [kStatusInts]
};

}  // namespace

struct gw_batch {
  gw_ctx* ctx = nullptr;
  gw_prec prec = GW_FP32;
  std::vector<BatchSys> sys;
  void* dev = nullptr;           // every system's tables, results and status words
  cudaStream_t cs = nullptr;     // capture stream
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t done = nullptr;
  bool launched = false;
  void* arena = nullptr;         // the context arena the graph was recorded with
  size_t arena_bytes = 0;
};

static size_t sigma_work_bytes(const GridInfo& g, const gw_batch_system& s, gw_prec prec) {
  Carver probe(nullptr);
  SigmaWork w;
  sigma_carve_work(probe, g, s.n_b, s.n_occ, s.n_chi, s.n_n, prec, false, w);
  return probe.off;
}

static void batch_free(gw_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->done) cudaEventDestroy(b->done);
  if (b->cs) cudaStreamDestroy(b->cs);
  for (auto& s : b->sys)
    if (s.chi0) gw_chi0_plan_destroy(s.chi0);
  if (b->dev) cudaFree(b->dev);
  delete b;
}

// The kernels of one system on s (recorded into the graph).
static gw_status record_system(gw_batch* b, BatchSys& y, cudaStream_t s) {
  gw_ctx* ctx = b->ctx;
  const gw_batch_system& in = y.in;
  const GridInfo& g = y.g;
  const gw_prec prec = b->prec;
  const size_t es = csize(prec);
  const size_t slice = (size_t)in.n_chi * in.n_chi;
  gw_status st;
  if ((st = gw_chi0_plan_launch(y.chi0, in.psi, in.chi_w, s))) return st;
  {
    Carver cv(ctx->arena);
    cv.take<double>(in.n_chi);                     // the slot gw_screen_W gives v^1/2 (here in the tables)
    if ((st = screen_launch(ctx, in.n_chi, in.n, prec, in.refine_iters, y.dvh, in.chi_w, in.chi_w, cv, nullptr,
                            nullptr, s)))
      return st;
  }
  if ((st = launch_ct(ctx, prec, false, in.n, y.dict, slice, in.chi_w, in.w_tau, s,
                      y.ict32.empty() ? nullptr : y.ict32.data())))
    return st;
  {
    Carver cv(ctx->arena);
    SigmaWork w;
    sigma_carve_work(cv, g, in.n_b, in.n_occ, in.n_chi, in.n_n, prec, false, w);
    if ((st = sigma_kernels(ctx, g, prec, false, in.n_b, in.n_occ, in.psi, in.n_n, in.n, in.n_chi, 0, y.scales, y.st, w,
                            in.w_tau, s)))
      return st;
    // status words of this system, then clear them for the next one
    if ((st = cuda_check(ctx, cudaMemcpyAsync(y.status, ctx->dflag, 8 * sizeof(int), cudaMemcpyDeviceToDevice, s),
                         "status")))
      return st;
    if (prec == GW_F16X3 || prec == GW_BF16X3) {
      if ((st = cuda_check(ctx, cudaMemcpyAsync(y.status + 8, chi0_plan_status_words(y.chi0), 2 * sizeof(int),
                                                cudaMemcpyDeviceToDevice, s), "status")))
        return st;
      // the self-energy pass keeps its tensor-core time-out words at ints 2, 3 of its scratch
      if ((st = cuda_check(ctx, cudaMemcpyAsync(y.status + 10, static_cast<int*>(w.tcs) + 2, 2 * sizeof(int),
                                                cudaMemcpyDeviceToDevice, s), "status")))
        return st;
    }
    if ((st = cuda_check(ctx, cudaMemsetAsync(ctx->dflag, 0, 8 * sizeof(int), s), "memset"))) return st;
  }
  (void)es;
  return GW_OK;
}

extern "C" gw_status gw_batch_plan(gw_ctx* ctx, int n_sys, const gw_batch_system* systems, gw_prec prec,
                                   gw_batch** out) {
  if (!ctx) return fail(nullptr, GW_ERR_ARG, "ctx is NULL");
  if (!out || !systems) return fail(ctx, GW_ERR_ARG, "NULL pointer");
  *out = nullptr;
  if (n_sys < 1 || n_sys > 4096) return fail(ctx, GW_ERR_SHAPE, "need 1 <= n_sys <= 4096");
  if (!valid_prec(prec)) return fail(ctx, GW_ERR_ARG, "bad precision");
  auto* b = new gw_batch;
  b->ctx = ctx;
  b->prec = prec;
  b->sys.resize(n_sys);
  gw_status st = GW_OK;
  auto bail = [&](gw_status e) {
    batch_free(b);
    return e;
  };
  // ---- host work: validation, chi0 plans, sizes
  size_t arena = 0;
  std::vector<std::vector<int>> maps(n_sys), invs(n_sys);
  for (int i = 0; i < n_sys; ++i) {
    BatchSys& y = b->sys[i];
    y.in = systems[i];
    const gw_batch_system& in = y.in;
    if (!in.psi || !in.chi_w || !in.w_tau || !in.Cinv_h || !in.gvec_h)
      return bail(fail(ctx, GW_ERR_ARG, "NULL pointer in system " + std::to_string(i)));
    if (in.w_tau == in.chi_w) return bail(fail(ctx, GW_ERR_ARG, "w_tau must not overlap chi_w"));
    if (in.refine_iters < 0 || in.refine_iters > 8) return bail(fail(ctx, GW_ERR_ARG, "need 0 <= refine_iters <= 8"));
    // the self-energy checks cover the grid, energies, bands, tau and the G-set maps, and give the band factors
    if ((st = sigma_check(ctx, &in.grid, &y.g, in.n_b, in.n_occ, in.psi, in.eps_h, in.mu, in.bands_h, in.n_n, in.n,
                          in.tau_h, in.omega_h, in.C_h, in.S_h, in.w_tau, in.n_chi, in.fft_index_h, prec, false,
                          nullptr, 0, maps[i], invs[i], y.scales)))
      return bail(st);
    if (in.n_chi > 65535) return bail(fail(ctx, GW_ERR_SHAPE, "need n_chi <= 65535"));
    if ((st = gw_chi0_plan_create(ctx, &in.grid, in.n_b, in.n_occ, in.eps_h, in.mu, in.n, in.tau_h, in.C_h, in.n_chi,
                                  in.fft_index_h, prec, in.r_block, &y.chi0)))
      return bail(st);
    arena = std::max(arena, chi0_plan_work(y.chi0));
    arena = std::max(arena, screen_scratch(in.n_chi, in.n, prec, nullptr, nullptr, in.refine_iters > 0));
    arena = std::max(arena, sigma_work_bytes(y.g, in, prec));
  }
  // ---- the batch's own block: per system v^1/2, inverse CT weights, self-energy tables, status words
  auto carve = [&](Carver& cv) {
    for (auto& y : b->sys) {
      y.dvh = cv.take<double>(y.in.n_chi);
      y.dict = cv.take<double>((size_t)2 * y.in.n * y.in.n);
      sigma_carve_tables(cv, y.g, y.in.n_b, y.in.n, y.in.n_chi, y.in.n_n, 0, false, y.st);
      y.status = cv.take<int>(kStatusInts);
    }
  };
  Carver probe(nullptr);
  carve(probe);
  if ((st = reserve(ctx, arena))) return bail(st);
  cudaError_t e = cudaMalloc(&b->dev, std::max<size_t>(probe.off, 256));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(ctx, GW_ERR_OOM, "cannot allocate the batch tables"));
  }
  Carver cv(b->dev);
  carve(cv);
  if ((st = cuda_check(ctx, cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking), "cudaStreamCreate"))) return bail(st);
  if ((st = cuda_check(ctx, cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming), "cudaEventCreate"))) return bail(st);
  for (int i = 0; i < n_sys; ++i) {
    BatchSys& y = b->sys[i];
    const gw_batch_system& in = y.in;
    std::vector<double> vh(in.n_chi);
    if ((st = gw_coulomb_sqrt(&in.grid, in.gvec_h, in.n_chi, vh.data()))) return bail(fail(ctx, st, gw_last_error(nullptr)));
    if ((st = upload(ctx, y.dvh, vh.data(), sizeof(double) * in.n_chi, b->cs))) return bail(st);
    if (is_fp64(prec)) {
      if ((st = upload(ctx, y.dict, in.Cinv_h, sizeof(double) * in.n * in.n, b->cs))) return bail(st);
    } else {
      y.ict32 = split_weights(in.Cinv_h, in.n * in.n, 1.0);
      if ((st = upload(ctx, y.dict, y.ict32.data(), sizeof(float) * 2 * in.n * in.n, b->cs))) return bail(st);
    }
    if ((st = sigma_upload_tables(ctx, y.st, y.g, in.n_b, in.n, in.n_chi, maps[i], invs[i], in.bands_h, in.n_n,
                                  y.scales, in.C_h, in.S_h, in.omega_h, nullptr, 0, prec, b->cs)))
      return bail(st);
    if ((st = cuda_check(ctx, cudaMemsetAsync(y.status, 0, kStatusInts * sizeof(int), b->cs), "memset"))) return bail(st);
  }
  if ((st = cuda_check(ctx, cudaMemsetAsync(ctx->dflag, 0, 8 * sizeof(int), b->cs), "memset"))) return bail(st);
  if ((st = cuda_check(ctx, cudaStreamSynchronize(b->cs), "batch tables"))) return bail(st);
  // ---- record every system's kernels into one graph (per-kernel timing off while recording)
  const bool timing = ctx->timing;
  ctx->timing = false;
  e = cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    ctx->timing = timing;
    return bail(cuda_check(ctx, e, "cudaStreamBeginCapture"));
  }
  gw_status rec = GW_OK;
  for (int i = 0; i < n_sys && !rec; ++i) rec = record_system(b, b->sys[i], b->cs);
  e = cudaStreamEndCapture(b->cs, &b->graph);
  ctx->timing = timing;
  if (rec) return bail(rec);
  if (e != cudaSuccess) return bail(cuda_check(ctx, e, "cudaStreamEndCapture"));
  if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess) return bail(cuda_check(ctx, e, "cudaGraphInstantiate"));
  b->arena = ctx->arena;
  b->arena_bytes = ctx->arena_bytes;
  *out = b;
  return GW_OK;
}

extern "C" gw_status gw_batch_launch(gw_batch* b, void* stream) {
  if (!b) return fail(nullptr, GW_ERR_ARG, "batch is NULL");
  gw_ctx* ctx = b->ctx;
  if (ctx->arena != b->arena || ctx->arena_bytes != b->arena_bytes)
    return fail(ctx, GW_ERR_ARG, "the context arena was reallocated after gw_batch_plan (a call needed more scratch): "
                                 "plan again, or reserve the arena before planning");
  cudaStream_t s = as_stream(stream);
  gw_status st;
  if ((st = cuda_check(ctx, cudaGraphLaunch(b->exec, s), "cudaGraphLaunch"))) return st;
  if ((st = cuda_check(ctx, cudaEventRecord(b->done, s), "cudaEventRecord"))) return st;
  ctx->launches += 1;
  b->launched = true;
  return GW_OK;
}

extern "C" gw_status gw_batch_wait(gw_batch* b, int timeout_ms, double* sigma_iw_h, int* status_h) {
  if (!b) return fail(nullptr, GW_ERR_ARG, "batch is NULL");
  gw_ctx* ctx = b->ctx;
  if (!b->launched) return fail(ctx, GW_ERR_ARG, "gw_batch_wait before gw_batch_launch");
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t q = cudaEventQuery(b->done);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) return cuda_check(ctx, q, "batch");
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (timeout_ms >= 0 && ms > timeout_ms) return fail(ctx, GW_ERR_TIMEOUT, "batch not finished within the time limit");
    std::this_thread::sleep_for(std::chrono::microseconds(200));
  }
  gw_status worst = GW_OK;
  std::string msg;
  size_t o = 0;
  for (size_t i = 0; i < b->sys.size(); ++i) {
    BatchSys& y = b->sys[i];
    const int n_n = y.in.n_n, n = y.in.n;
    int words[kStatusInts];
    std::vector<int> stat(n_n);
    gw_status st;
    if ((st = cuda_check(ctx, cudaMemcpy(words, y.status, sizeof(words), cudaMemcpyDeviceToHost), "status"))) return st;
    if ((st = cuda_check(ctx, cudaMemcpy(stat.data(), y.st.stat, sizeof(int) * n_n, cudaMemcpyDeviceToHost), "status")))
      return st;
    if (sigma_iw_h &&
        (st = cuda_check(ctx, cudaMemcpy(sigma_iw_h + 2 * o, y.st.out, sizeof(double2) * n_n * n, cudaMemcpyDeviceToHost),
                         "sigma")))
      return st;
    o += (size_t)n_n * n;
    gw_status si = GW_OK;
    if (words[4] || words[8] || words[10]) si = GW_ERR_TIMEOUT;
    else if (words[0]) si = GW_ERR_NUMERIC;
    else
      for (int k = 0; k < n_n; ++k)
        if (stat[k]) si = GW_ERR_NUMERIC;
    if (status_h) status_h[i] = si;
    if (si && !worst) {
      worst = si;
      msg = "system " + std::to_string(i) + (si == GW_ERR_TIMEOUT ? ": tensor-core wait timed out"
                                                                 : ": eps~ not positive definite or Thiele breakdown");
    }
  }
  if (worst) return fail(ctx, worst, msg);
  return GW_OK;
}

extern "C" gw_status gw_batch_destroy(gw_batch* b) {
  if (!b) return GW_OK;
  cudaStreamSynchronize(b->cs);
  batch_free(b);
  return GW_OK;
}
