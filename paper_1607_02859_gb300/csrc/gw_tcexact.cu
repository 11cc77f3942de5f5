// Complex FP64 matrix product with FP64-class accuracy on tcgen05 fp16 tensor
// cores, for the residual of the refinement of the screening solve (Eq.
// W_correlated: R = chi~ - eps~ X needs the product chi~ X to more digits than
// the FP32-class solve it corrects).
//
// Error-free splitting (the approach of Ozaki, Ogita, Oishi and Rump for
// accurate matrix products).  Row i of A gets the power of two 2^e_i above its
// largest component and column j of B the power 2^f_j; each element is then
// cut into S slices of beta = 6 bits,
//   A_ik = sum_a s_a(i,k) 2^(e_i - (a+1) beta) + rest,   |s_0| <= 64, |s_a>0| <= 32,
// all small integers, exact in fp16.  Over a K block of 4096 real elements
// the sum of slice products of a pair (a, b) is an integer of at most 2^24
// (a = b = 0), 2^23 (one of them 0) or 2^22 (neither); pairs of the same level
// a + b carry the same scale 2^(e_i + f_j - (a+b+2) beta), so a group of them
// whose bounds add up to at most 2^24 is summed in one FP32 accumulator in
// tensor memory exactly, whatever the order or rounding of the additions.
// Levels 0..L (largest terms first) are packed into such groups (L = 4: 15
// pairs in 8 groups), and for every group and K block one tcgen05 pass forms
// the exact sum, which the epilogue adds, times its scale, into the output.
// Dropped pairs and the rest are below 2^(-6(L+1)) of the row and column maxima.

// GB300's FP64 rate is a few operations per clock and SM, too slow for an
// FP64 update per pass.  A block sum times 2^-(a+b+2) beta is exact in FP32, so
// the passes add it into an unevaluated pair hi + lo of FP32 numbers (the
// error-free sum of Knuth, then a renormalisation: ~48 bits) kept in the
// output's own 16 bytes per complex element; the last pass converts the pair to
// FP64 and applies 2^(e_i + f_j).  Tiles are taken in groups of kGroupM row
// tiles so that the CTAs running together share their operand rows in L2.
//
// Complex-to-real mapping as in the other tensor-core GEMMs: A is a real
// [M][2K] operand with (re, im) interleaved along K, B holds two real rows per
// complex column, (br, -bi) and (bi, br).  Tile 128 rows x 128 complex columns
// (MMA 128 x 256 x 16), one slice of A and one of B per 32-wide K stage, six
// stages in flight; two 256-column accumulators in tensor memory so that one
// pass's epilogue overlaps the next pass's MMAs; the FP64 output tile (256 KB)
// stays in L2 across a tile's passes.  Persistent CTAs, bounded waits.
#include <algorithm>
#include <climits>

#include "gw_tc.h"
#include "gw_tcgen05.cuh"

namespace gw {
namespace tx {

using namespace tcx;

constexpr int BM = 128, BNC = 128, BK = 32, STAGES = 6;
constexpr int BETA = 6;                          // bits per slice
constexpr int KB_REAL = 1 << (24 - 2 * BETA);    // real K per exact block: 4096
constexpr int KB_STEPS = KB_REAL / BK;
constexpr int MAX_LEVELS = 7;
constexpr int MAX_PAIRS = (MAX_LEVELS + 1) * (MAX_LEVELS + 2) / 2;
constexpr int MAX_GROUPS = MAX_PAIRS;
constexpr int A_BYTES = BM * BK * 2;             // 8 KB
constexpr int B_BYTES = 2 * BNC * BK * 2;        // 16 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int EPI_CPX = 16;                      // complex columns per epilogue round
constexpr int EPI_WARPS = 8;                     // two per tensor-memory lane quarter, one per column half
constexpr int EPI_BYTES = EPI_WARPS * 32 * EPI_CPX * 8;   // per epilogue warp: 32 rows x 16 complex (FP32)
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + EPI_BYTES + 1024 + 256;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr int kGroupM = 8;                       // row tiles per group of the tile order
static_assert(SMEM_BYTES <= 232448, "shared memory per CTA");

// tile t of the persistent order -> (row tile, column tile): kGroupM row tiles are
// walked down each column before moving on, so ~152 consecutive tiles span
// kGroupM row tiles and ~19 column tiles of operands
__device__ __forceinline__ void tile_of(long t, int tm, int tn, int& bm, int& bn) {
  const long per_group = (long)kGroupM * tn;
  const int g = (int)(t / per_group);
  const int first = g * kGroupM;
  const int rows = min(kGroupM, tm - first);
  const long r = t - (long)g * per_group;
  bm = first + (int)(r % rows);
  bn = (int)(r / rows);
}

// hi + lo += v exactly (Knuth's two-sum), then renormalised
__device__ __forceinline__ void dd_add(float& hi, float& lo, float v) {
  const float s = hi + v;
  const float bb = s - hi;
  const float e = (hi - (s - bb)) + (v - bb);
  const float t = lo + e;
  hi = s + t;
  lo = t - (hi - s);
}

struct XParams {
  int M, N;               // complex output size
  int k_steps;            // BK stages over the padded real K
  int n_kb;               // K blocks (KB_STEPS stages each, the last one shorter)
  int n_groups;           // groups of pairs summed in one accumulator
  int tm, tn;
  int gstart[MAX_GROUPS + 1];          // pairs gstart[g] .. gstart[g+1]-1 form group g
  int glevel[MAX_GROUPS];              // a + b of the group's pairs
  int pa[MAX_PAIRS], pb[MAX_PAIRS];    // slice indices of each pair
  const int* rexp;        // [M] e_i
  const int* cexp;        // [N] f_j
  double2* C;
  long ldc;
  int* status;
};

template <int DUMMY>
__global__ void __launch_bounds__(THREADS, 1) cgemm_sliced_kernel(const __grid_constant__ CUtensorMap mA,
                                                                  const __grid_constant__ CUtensorMap mB, XParams p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float2* epi = reinterpret_cast<float2*>(smem + STAGES * STAGE_BYTES);     // [EPI_WARPS][32 rows][16]
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES + EPI_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* done = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long ntiles = (long)p.tm * p.tn;
  const int passes = p.n_groups * p.n_kb;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], EPI_WARPS);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  auto timed_out = [&](int where) {
    *abort_flag = 1;
    if (atomicCAS(p.status, 0, 1) == 0) p.status[1] = where;
  };
  auto k_first = [&](int kb) { return kb * KB_STEPS; };
  auto k_last = [&](int kb) { return min((kb + 1) * KB_STEPS, p.k_steps); };

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------- TMA producer
    long kit = 0;
    for (long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
      int bm, bn;
      tile_of(t, p.tm, p.tn, bm, bn);
      for (int q = 0; q < passes && !*abort_flag; ++q) {
        const int g = q / p.n_kb, kb = q - g * p.n_kb;
        for (int pr = p.gstart[g]; pr < p.gstart[g + 1] && !*abort_flag; ++pr)
          for (int ks = k_first(kb); ks < k_last(kb); ++ks, ++kit) {
            const int s = (int)(kit % STAGES);
            if (kit >= STAGES && !mbar_wait(&empty[s], (uint32_t)(((kit / STAGES) & 1) ^ 1))) {
              timed_out(31);
              break;
            }
            uint8_t* st = smem + s * STAGE_BYTES;
            mbar_expect_tx(&full[s], STAGE_BYTES);
            tma_load_3d(st, &mA, &full[s], ks * BK, bm * BM, p.pa[pr]);
            tma_load_3d(st + A_BYTES, &mB, &full[s], ks * BK, 2 * bn * BNC, p.pb[pr]);
          }
      }
    }
    if (*abort_flag)
      for (long it = kit - STAGES < 0 ? 0 : kit - STAGES; it < kit; ++it)
        mbar_wait(&full[it % STAGES], (uint32_t)((it / STAGES) & 1));
  } else if (warp == 1 && lane == 0) {
    // ---------------------------------------------------------- MMA issuer
    constexpr uint32_t idesc = make_idesc(0u, 2 * BNC, BM);
    long kit = 0;
    long pc = 0;                                   // passes issued by this CTA
    bool ok = true;
    for (long t = blockIdx.x; t < ntiles && ok && !*abort_flag; t += gridDim.x) {
      for (int q = 0; q < passes && ok; ++q, ++pc) {
        const int g = q / p.n_kb, kb = q - g * p.n_kb;
        const int b = (int)(pc & 1);
        if (pc >= 2 && !mbar_wait(&tempty[b], (uint32_t)(((pc >> 1) & 1) ^ 1))) {
          timed_out(32);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(b * 256);
        const int f = k_first(kb);
        for (int pr = p.gstart[g]; pr < p.gstart[g + 1] && ok; ++pr)
          for (int ks = f; ks < k_last(kb); ++ks, ++kit) {
            const int s = (int)(kit % STAGES);
            if (!mbar_wait(&full[s], (uint32_t)((kit / STAGES) & 1))) {
              timed_out(33);
              ok = false;
              break;
            }
            tc_fence_after();
            uint8_t* st = smem + s * STAGE_BYTES;
            const uint64_t ad = sw64_desc(st), bd = sw64_desc(st + A_BYTES);
            const bool fresh = pr == p.gstart[g] && ks == f;      // first stage of the group's sum
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              const uint64_t off = (uint64_t)(kk * 32) >> 4;
              umma(d, ad + off, bd + off, idesc, (fresh && kk == 0) ? 0u : 1u);
            }
            umma_commit(&empty[s]);
          }
        umma_commit(&tfull[b]);
      }
    }
    umma_commit(done);
    mbar_wait(done, 0);
  } else if (warp >= 2) {
    // ---------------------------------------------------------- epilogue
    const int ew = warp - 2;
    const int qw = warp & 3;                     // tensor-memory lane quarter
    const int hh = ew >> 2;                      // column half: complex columns hh*64 .. hh*64+63
    const uint32_t lane_addr = (uint32_t)(qw * 32) << 16;
    float2* stg = epi + ew * 32 * EPI_CPX;
    long pc = 0;
    bool go = true;
    for (long t = blockIdx.x; t < ntiles && go; t += gridDim.x) {
      int bm, bn;
      tile_of(t, p.tm, p.tn, bm, bn);
      const int r0 = bm * BM + qw * 32;
      const int n0 = bn * BNC;
      for (int q = 0; q < passes; ++q, ++pc) {
        const int g = q / p.n_kb;
        const int b = (int)(pc & 1);
        const bool ok = mbar_wait(&tfull[b], (uint32_t)((pc >> 1) & 1));
        if (!ok) timed_out(34);
        tc_fence_after();
        if (!__all_sync(0xffffffffu, ok && !*abort_flag)) {
          go = false;
          break;
        }
        const int shift = (p.glevel[g] + 2) * BETA;
        const float scl = __int_as_float((127 - shift) << 23);    // 2^-shift, exact
        const bool first = q == 0, last = q == passes - 1;
#pragma unroll 1
        for (int c = hh * BNC; c < (hh + 1) * BNC; c += 2 * EPI_CPX) {
          uint32_t r[2][16];
          tmem_ld16(tmem + lane_addr + (uint32_t)(b * 256 + c), r[0]);
          tmem_ld16(tmem + lane_addr + (uint32_t)(b * 256 + c + 16), r[1]);
          tmem_wait_ld();
#pragma unroll
          for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int j = 0; j < 8; ++j)
              stg[lane * EPI_CPX + ((u * 8 + j + lane) & (EPI_CPX - 1))] =
                  make_float2(__uint_as_float(r[u][2 * j]), __uint_as_float(r[u][2 * j + 1]));
          __syncwarp();
          const int nc0 = n0 + c / 2;
          // two rows of 16 complex (256 B each) per warp instruction; the sixteen loads of the
          // running sums are all issued before the first is used
          const int cc = lane & 15, gn = nc0 + cc;
          float4 acc[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int gm = r0 + 2 * i + (lane >> 4);
            acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (!first && gm < p.M && gn < p.N)
              acc[i] = *reinterpret_cast<const float4*>(p.C + (long)gm * p.ldc + gn);
          }
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int rr = 2 * i + (lane >> 4);
            const int gm = r0 + rr;
            if (gm < p.M && gn < p.N) {
              const float2 v = stg[rr * EPI_CPX + ((cc + rr) & (EPI_CPX - 1))];
              double2* o = p.C + (long)gm * p.ldc + gn;
              dd_add(acc[i].x, acc[i].y, v.x * scl);           // (re hi, re lo, im hi, im lo) until the last pass
              dd_add(acc[i].z, acc[i].w, v.y * scl);
              if (last) {
                const int sc = max(p.rexp[gm] + p.cexp[gn], -1000);
                *o = make_double2(ldexp((double)acc[i].x + (double)acc[i].y, sc),
                                  ldexp((double)acc[i].z + (double)acc[i].w, sc));
              } else {
                *reinterpret_cast<float4*>(o) = acc[i];
              }
            }
          }
          __syncwarp();
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[b]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

__device__ __forceinline__ int exp_above(double m) {
  int e = 0;
  frexp(m, &e);            // m = f 2^e, f in [0.5, 1): |x| <= m < 2^e
  return e;
}

// e_i of each row of A [M][K] (one warp per row).
__global__ void __launch_bounds__(256) row_exp_kernel(const double2* __restrict__ A, long lda, int M, int K,
                                                      int* __restrict__ rexp) {
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i >= M) return;
  double m = 0.0;
  for (int k = lane; k < K; k += 32) {
    const double2 v = A[(long)i * lda + k];
    m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) rexp[i] = m > 0.0 ? exp_above(m) : 0;
}

// f_j of each column of B [K][N]: threads along j, blocks of rows along y; max
// of the per-block exponents (exponents order as the values they bound).
__global__ void __launch_bounds__(256) col_exp_kernel(const double2* __restrict__ B, long ldb, int K, int N, int rows,
                                                      int* __restrict__ cexp) {
  const int j = blockIdx.x * 256 + threadIdx.x;
  if (j >= N) return;
  const int k0 = blockIdx.y * rows, k1 = min(K, k0 + rows);
  double m = 0.0;
  for (int k = k0; k < k1; ++k) {
    const double2 v = B[(long)k * ldb + j];
    m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
  }
  if (m > 0.0) atomicMax(&cexp[j], exp_above(m));
}

__global__ void col_exp_fix_kernel(int* cexp, int N) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < N && cexp[j] < -1100) cexp[j] = 0;     // all-zero column
}

__device__ __forceinline__ uint16_t ihalf(long long s) { return __half_as_ushort(__int2half_rn((int)s)); }

// The S slices of x 2^(beta - e) (|.| < 2^beta): the integer V = rint(x 2^(beta S - e))
// (one FP64 multiply and conversion; V < 2^(6S) fits 64 bits) written in balanced
// base 2^beta, V = sum_a s_a 2^(beta (S-1-a)), lower digits s_a in [-32, 32), the top
// one |s_0| <= 64, all exact in fp16.  Integer digit extraction keeps FP64 work to two
// operations.
template <int S>
__device__ __forceinline__ void cut(double x, int e, uint16_t (&out)[S]) {
  constexpr int beta = BETA;
  long long v = __double2ll_rn(ldexp(x, beta * S - e));
  constexpr long long half = 1LL << (beta - 1), mask = (1LL << beta) - 1;
#pragma unroll
  for (int a = S - 1; a > 0; --a) {
    const long long d = ((v + half) & mask) - half;
    out[a] = ihalf(d);
    v = (v - d) >> beta;          // exact: v - d is a multiple of 2^beta
  }
  out[0] = ihalf(v);
}

// A [M][K] -> As [S][M][kp]: (re, im) slices at real columns 2k, 2k+1; zero padding.
template <int S>
__global__ void __launch_bounds__(256) slice_a_kernel(const double2* __restrict__ A, long lda, int M, int K, int kp,
                                                      const int* __restrict__ rexp, uint16_t* __restrict__ As) {
  const int i = blockIdx.y;
  const int k = blockIdx.x * 256 + threadIdx.x;
  if (2 * k >= kp) return;
  uint16_t re[S], im[S];
  if (k < K) {
    const double2 v = A[(long)i * lda + k];
    const int e = rexp[i];
    cut<S>(v.x, e, re);
    cut<S>(v.y, e, im);
  } else {
#pragma unroll
    for (int a = 0; a < S; ++a) re[a] = im[a] = 0;
  }
  const size_t plane = (size_t)M * kp;
#pragma unroll
  for (int a = 0; a < S; ++a)
    reinterpret_cast<uint32_t*>(As + a * plane + (size_t)i * kp + 2 * k)[0] = (uint32_t)re[a] | ((uint32_t)im[a] << 16);
}

// B [K][N] -> Bs [S][2N][kp]: row 2j = (br, -bi), row 2j+1 = (bi, br) along K,
// through a 32 x 32 shared tile so that reads (along j) and writes (along k)
// are both coalesced.
template <int S>
__global__ void __launch_bounds__(256) slice_b_kernel(const double2* __restrict__ B, long ldb, int K, int N, int kp,
                                                      const int* __restrict__ cexp, uint16_t* __restrict__ Bs) {
  __shared__ double2 t[32][33];                   // t[j][k]
  const int j0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int k = k0 + y, j = j0 + threadIdx.x;
    t[threadIdx.x][y] = (k < K && j < N) ? B[(long)k * ldb + j] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const size_t plane = (size_t)2 * N * kp;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int j = j0 + y, k = k0 + threadIdx.x;
    if (j >= N || 2 * k >= kp) continue;
    const double2 v = t[y][threadIdx.x];
    uint16_t br[S], bi[S];
    const int e = cexp[j];
    cut<S>(v.x, e, br);
    cut<S>(v.y, e, bi);
    const size_t o0 = (size_t)(2 * j) * kp + 2 * k, o1 = o0 + kp;
#pragma unroll
    for (int a = 0; a < S; ++a) {
      const uint16_t nbi = bi[a] ^ 0x8000u;                  // -bi (exact for integers; -0 is harmless)
      reinterpret_cast<uint32_t*>(Bs + a * plane + o0)[0] = (uint32_t)br[a] | ((uint32_t)nbi << 16);
      reinterpret_cast<uint32_t*>(Bs + a * plane + o1)[0] = (uint32_t)bi[a] | ((uint32_t)br[a] << 16);
    }
  }
}

template <int S>
static gw_status slice_ops(gw_ctx* ctx, int M, int N, int K, int kp, const double2* A, long lda, const double2* B,
                           long ldb, const int* rexp, const int* cexp, uint16_t* As, uint16_t* Bs, cudaStream_t st) {
  slice_a_kernel<S><<<dim3((kp / 2 + 255) / 256, M), 256, 0, st>>>(A, lda, M, K, kp, rexp, As);
  gw_status rc = launch_check(ctx, "slice_a_kernel");
  if (rc) return rc;
  slice_b_kernel<S><<<dim3((N + 31) / 32, (kp / 2 + 31) / 32), dim3(32, 8), 0, st>>>(B, ldb, K, N, kp, cexp, Bs);
  return launch_check(ctx, "slice_b_kernel");
}

}  // namespace tx

size_t tc_zgemm_sliced_scratch(int M, int N, int K, int levels) {
  const size_t kp = (size_t)(2 * std::max(K, 1) + tx::BK - 1) / tx::BK * tx::BK;
  const int S = levels + 1;
  Carver probe(nullptr);
  probe.take<int>(M);
  probe.take<int>(N);
  probe.take<uint16_t>((size_t)S * M * kp);
  probe.take<uint16_t>((size_t)S * 2 * N * kp);
  return Carver::round(probe.off);
}

gw_status tc_zgemm_sliced(gw_ctx* ctx, int M, int N, int K, const double2* A, long lda, const double2* B, long ldb,
                          double2* C, long ldc, int levels, int* status, void* scratch, cudaStream_t st) {
  using namespace tx;
  if (M <= 0 || N <= 0) return GW_OK;
  if (K <= 0) return fail(ctx, GW_ERR_SHAPE, "sliced GEMM needs K >= 1");
  if (levels < 1 || levels > MAX_LEVELS) return fail(ctx, GW_ERR_ARG, "sliced GEMM: levels must be 1..7");
  const int S = levels + 1;
  const int kp = (2 * K + BK - 1) / BK * BK;
  Carver cv(scratch);
  int* rexp = cv.take<int>(M);
  int* cexp = cv.take<int>(N);
  uint16_t* As = cv.take<uint16_t>((size_t)S * M * kp);
  uint16_t* Bs = cv.take<uint16_t>((size_t)S * 2 * N * kp);
  gw_status rc;
  row_exp_kernel<<<(M + 7) / 8, 256, 0, st>>>(A, lda, M, K, rexp);
  if ((rc = launch_check(ctx, "row_exp_kernel"))) return rc;
  if ((rc = cuda_check(ctx, cudaMemsetAsync(cexp, 0x80, sizeof(int) * N, st), "memset exponents"))) return rc;
  const int rows = 256;
  col_exp_kernel<<<dim3((N + 255) / 256, (K + rows - 1) / rows), 256, 0, st>>>(B, ldb, K, N, rows, cexp);
  if ((rc = launch_check(ctx, "col_exp_kernel"))) return rc;
  col_exp_fix_kernel<<<(N + 255) / 256, 256, 0, st>>>(cexp, N);
  if ((rc = launch_check(ctx, "col_exp_fix_kernel"))) return rc;
  switch (S) {
    case 2: rc = slice_ops<2>(ctx, M, N, K, kp, A, lda, B, ldb, rexp, cexp, As, Bs, st); break;
    case 3: rc = slice_ops<3>(ctx, M, N, K, kp, A, lda, B, ldb, rexp, cexp, As, Bs, st); break;
    case 4: rc = slice_ops<4>(ctx, M, N, K, kp, A, lda, B, ldb, rexp, cexp, As, Bs, st); break;
    case 5: rc = slice_ops<5>(ctx, M, N, K, kp, A, lda, B, ldb, rexp, cexp, As, Bs, st); break;
    case 6: rc = slice_ops<6>(ctx, M, N, K, kp, A, lda, B, ldb, rexp, cexp, As, Bs, st); break;
    case 7: rc = slice_ops<7>(ctx, M, N, K, kp, A, lda, B, ldb, rexp, cexp, As, Bs, st); break;
    default: rc = slice_ops<8>(ctx, M, N, K, kp, A, lda, B, ldb, rexp, cexp, As, Bs, st); break;
  }
  if (rc) return rc;
  CUtensorMap ma, mb;
  if ((rc = tc_make_map3(ctx, &ma, As, kp, M, S, BM, 0, BK))) return rc;
  if ((rc = tc_make_map3(ctx, &mb, Bs, kp, 2L * N, S, 2 * BNC, 0, BK))) return rc;
  XParams P;
  P.M = M;
  P.N = N;
  P.k_steps = kp / BK;
  P.n_kb = (P.k_steps + KB_STEPS - 1) / KB_STEPS;
  // pairs level by level (largest terms first), packed into groups whose block sums are
  // bounded by 2^24 together: log2 bound 24 for (0,0), 23 with one top slice, 22 without
  int n_pairs = 0;
  P.n_groups = 0;
  for (int lv = 0; lv <= levels; ++lv) {
    long room = 0;                                 // units of 2^22 left in the open group
    for (int a = 0; a <= lv; ++a) {
      const int b = lv - a;
      const long need = (a == 0 && b == 0) ? 4 : (a == 0 || b == 0) ? 2 : 1;
      if (need > room) {                           // open a new group at this pair
        P.gstart[P.n_groups] = n_pairs;
        P.glevel[P.n_groups] = lv;
        ++P.n_groups;
        room = 4;
      }
      room -= need;
      P.pa[n_pairs] = a;
      P.pb[n_pairs] = b;
      ++n_pairs;
    }
  }
  P.gstart[P.n_groups] = n_pairs;
  P.tm = (M + BM - 1) / BM;
  P.tn = (N + BNC - 1) / BNC;
  P.rexp = rexp;
  P.cexp = cexp;
  P.C = C;
  P.ldc = ldc;
  P.status = status;
  const long tiles = (long)P.tm * P.tn;
  const dim3 grid((unsigned)std::max<long>(1, std::min<long>(tiles, ctx->num_sms)));
  auto kernel = cgemm_sliced_kernel<0>;
  if ((rc = cuda_check(ctx, cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES),
                       "cudaFuncSetAttribute")))
    return rc;
  KTimer kt(ctx, KF_CGEMM_EXACT, 8.0 * M * (double)N * K, st);
  kernel<<<grid, THREADS, SMEM_BYTES, st>>>(ma, mb, P);
  return launch_check(ctx, "cgemm_sliced_kernel");
}

}  // namespace gw

using namespace gw;

extern "C" gw_status gw_zgemm_sliced(gw_ctx* ctx, int M, int N, int K, const void* A, long lda, const void* B,
                                     long ldb, void* C, long ldc, int levels, void* stream) {
  if (!ctx) return fail(nullptr, GW_ERR_ARG, "ctx is NULL");
  if (M < 1 || N < 1 || K < 1 || M > 65535 || N > 65535 || K > 65535)
    return fail(ctx, GW_ERR_SHAPE, "need 1 <= M, N, K <= 65535");
  if (lda < K || ldb < N || ldc < N) return fail(ctx, GW_ERR_SHAPE, "leading dimension below the row length");
  if (!A || !B || !C) return fail(ctx, GW_ERR_ARG, "NULL pointer");
  if (((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B) | reinterpret_cast<uintptr_t>(C)) & 15) != 0)
    return fail(ctx, GW_ERR_ARG, "A, B and C must be 16-byte aligned");
  if (levels < 1 || levels > tx::MAX_LEVELS) return fail(ctx, GW_ERR_ARG, "need 1 <= levels <= 7");
  cudaStream_t s = as_stream(stream);
  gw_status st;
  if ((st = reserve(ctx, tc_zgemm_sliced_scratch(M, N, K, levels)))) return st;
  int* tstat = ctx->dflag + 4;
  if ((st = cuda_check(ctx, cudaMemsetAsync(tstat, 0, 2 * sizeof(int), s), "memset status"))) return st;
  if ((st = tc_zgemm_sliced(ctx, M, N, K, static_cast<const double2*>(A), lda, static_cast<const double2*>(B), ldb,
                            static_cast<double2*>(C), ldc, levels, tstat, ctx->arena, s)))
    return st;
  int f[2] = {0, 0};
  if ((st = cuda_check(ctx, cudaMemcpyAsync(f, tstat, sizeof(f), cudaMemcpyDeviceToHost, s), "status"))) return st;
  if ((st = cuda_check(ctx, cudaStreamSynchronize(s), "sync"))) return st;
  if (f[0]) return fail(ctx, GW_ERR_TIMEOUT, "tensor-core pipeline wait timed out (role " + std::to_string(f[1]) + ")");
  return GW_OK;
}
