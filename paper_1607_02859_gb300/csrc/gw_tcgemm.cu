// General complex GEMM on tcgen05 tensor cores with split 16-bit products,
// used by the screening step (Eqs. die, W_correlated) for the tensor-core
// precisions:
//   C[m][n] = alpha * sum_k opA(m,k) opB(k,n)   (+ C[m][n] if accumulate)
// opA(m,k) = A[m][k] or A[k][m] (a_trans), conjugated if a_conj; opB likewise.
// The complex-to-real mapping, the hi/lo split and the TMA/mbarrier/TMEM
// pipeline are those of the Green's-function kernel (gw_tc.cu): A becomes a
// real [M][2K] operand with (re, im) interleaved along K, B two real rows per
// complex column, (br, -bi) and (bi, br), so the FP32 accumulator holds
// (re, im) pairs.  tri = 1 writes only m >= n (and skips tiles above the
// diagonal); tri = 2 also starts each tile's k loop at its first row, for
// products X^H X with X lower triangular.
#include <algorithm>

#include "gw_tc.h"
#include "gw_tcgen05.cuh"

namespace gw {
namespace tg {

using namespace tcx;

constexpr int BM = 128, BNC = 128, BK = 32, STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;            // 8 KB
constexpr int B_BYTES = 2 * BNC * BK * 2;       // 16 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int EPI_COLS = 32;                     // complex columns per epilogue round
constexpr int EPI_BYTES = 4 * 32 * EPI_COLS * 8; // per epilogue warp: 32 rows x 32 complex
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + EPI_BYTES + 1024 + 256;
constexpr int THREADS = 192;

struct KParams {
  int M, N;               // complex output size
  int k_steps;            // BK stages over the padded real K
  int batch, tm, tn;      // batch entries, row tiles, column tiles
  float2* C;
  long ldc;
  long sC;
  float alpha;
  int accumulate;
  const unsigned int* maxbits;   // [b] A, [batch + b] B: max |component| (float bits)
  int* status;
};

__device__ __forceinline__ int scale_exp(unsigned int bits) {
  const float m = __uint_as_float(bits);
  int ex = 0;
  if (!(m > 0.f)) return 0;
  frexpf(m, &ex);
  return min(15 - ex, 126);      // 2^e stays a finite FP32 number for the tiniest operands
}

// Persistent: CTA c takes tiles c, c + gridDim.x, ... (row tiles ascending, so
// the longest tiles of a triangular product go first).  Two 256-column
// accumulators in tensor memory let the epilogue of one tile run while the
// MMAs of the next one issue.  Stages are 32 real K (64-byte swizzled rows),
// four in flight.
template <uint32_t FMT, int TRI>
__global__ void __launch_bounds__(THREADS, 1) cgemm_tc_kernel(const __grid_constant__ CUtensorMap mA_hi,
                                                              const __grid_constant__ CUtensorMap mA_lo,
                                                              const __grid_constant__ CUtensorMap mB_hi,
                                                              const __grid_constant__ CUtensorMap mB_lo, KParams p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float2* epi = reinterpret_cast<float2*>(smem + STAGES * STAGE_BYTES);     // [4 warps][32 rows][32]
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES + EPI_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;       // [2] accumulator ready for the epilogue
  uint64_t* tempty = tfull + 2;           // [2] accumulator drained by the epilogue
  uint64_t* done = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long per_b = (long)p.tm * p.tn;
  const long ntiles = per_b * p.batch;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
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
  // tile t -> (batch entry, row tile, column tile); false if above the diagonal
  auto tile = [&](long t, int& bz, int& bm, int& bn) {
    bz = (int)(t / per_b);
    const long r = t - (long)bz * per_b;
    bm = (int)(r / p.tn);
    bn = (int)(r - (long)bm * p.tn);
    return !TRI || bn <= bm;
  };
  auto first_k = [&](int bm) { return TRI == 2 ? min(2 * bm * BM / BK, p.k_steps) : 0; };

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------- TMA producer
    long kit = 0;
    for (long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
      int bz, bm, bn;
      if (!tile(t, bz, bm, bn)) continue;
      for (int ks = first_k(bm); ks < p.k_steps; ++ks, ++kit) {
        const int s = (int)(kit % STAGES);
        if (kit >= STAGES && !mbar_wait(&empty[s], (uint32_t)(((kit / STAGES) & 1) ^ 1))) {
          timed_out(21);
          break;
        }
        uint8_t* st = smem + s * STAGE_BYTES;
        const int x = ks * BK;
        mbar_expect_tx(&full[s], STAGE_BYTES);
        tma_load_3d(st, &mA_hi, &full[s], x, bm * BM, bz);
        tma_load_3d(st + A_BYTES, &mA_lo, &full[s], x, bm * BM, bz);
        tma_load_3d(st + 2 * A_BYTES, &mB_hi, &full[s], x, 2 * bn * BNC, bz);
        tma_load_3d(st + 2 * A_BYTES + B_BYTES, &mB_lo, &full[s], x, 2 * bn * BNC, bz);
      }
    }
    if (*abort_flag)
      for (long it = kit - STAGES < 0 ? 0 : kit - STAGES; it < kit; ++it)
        mbar_wait(&full[it % STAGES], (uint32_t)((it / STAGES) & 1));
  } else if (warp == 1 && lane == 0) {
    // ---------------------------------------------------------- MMA issuer
    constexpr uint32_t idesc = make_idesc(FMT, 2 * BNC, BM);
    long kit = 0;
    int tl = 0;
    for (long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
      int bz, bm, bn;
      if (!tile(t, bz, bm, bn)) continue;
      const int b = tl & 1;
      if (tl >= 2 && !mbar_wait(&tempty[b], (uint32_t)(((tl >> 1) & 1) ^ 1))) {
        timed_out(22);
        break;
      }
      tc_fence_after();
      const uint32_t d = tmem + (uint32_t)(b * 256);
      const int f = first_k(bm);
      for (int ks = f; ks < p.k_steps; ++ks, ++kit) {
        const int s = (int)(kit % STAGES);
        if (!mbar_wait(&full[s], (uint32_t)((kit / STAGES) & 1))) {
          timed_out(23);
          break;
        }
        tc_fence_after();
        uint8_t* st = smem + s * STAGE_BYTES;
        const uint64_t ah = sw64_desc(st), al = sw64_desc(st + A_BYTES);
        const uint64_t bh = sw64_desc(st + 2 * A_BYTES), bl = sw64_desc(st + 2 * A_BYTES + B_BYTES);
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint64_t off = (uint64_t)(kk * 32) >> 4;    // 16 elements = 32 bytes along K
          umma(d, ah + off, bh + off, idesc, (ks > f || kk > 0) ? 1u : 0u);
          umma(d, ah + off, bl + off, idesc, 1u);
          umma(d, al + off, bh + off, idesc, 1u);
        }
        umma_commit(&empty[s]);
      }
      umma_commit(&tfull[b]);
      ++tl;
    }
    umma_commit(done);
    mbar_wait(done, 0);      // every MMA of this CTA has completed before tensor memory is freed
  } else if (warp >= 2) {
    // ---------------------------------------------------------- epilogue
    const int q = warp & 3;                         // tensor-memory lane quarter of this warp
    const int row = q * 32 + lane;
    const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
    int tl = 0;
    for (long t = blockIdx.x; t < ntiles; t += gridDim.x) {
      int bz, bm, bn;
      if (!tile(t, bz, bm, bn)) continue;
      const int b = tl & 1;
      const bool ok = mbar_wait(&tfull[b], (uint32_t)((tl >> 1) & 1));
      if (!ok) timed_out(24);
      tc_fence_after();
      if (!__all_sync(0xffffffffu, ok && !*abort_flag)) break;
      const int n0 = bn * BNC;
      const int r0 = bm * BM + q * 32;                // first output row of this warp
      const float sc = p.alpha * ldexpf(1.0f, -(scale_exp(p.maxbits[bz]) + scale_exp(p.maxbits[p.batch + bz])));
      const bool have = first_k(bm) < p.k_steps;
      float2* stg = epi + q * 32 * EPI_COLS;          // this warp's 32 x 32 staging tile
      float2* cb = p.C + bz * p.sC;
#pragma unroll 1
      for (int c = 0; c < 2 * BNC; c += 2 * EPI_COLS) {
        // four 16-column loads from tensor memory: row `lane`, complex columns c/2 .. c/2+31
        uint32_t r[4][16];
        if (have) {
#pragma unroll
          for (int u = 0; u < 4; ++u) tmem_ld16(tmem + lane_addr + (uint32_t)(b * 256 + c + 16 * u), r[u]);
          tmem_wait_ld();
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int j = 0; j < 16; ++j) r[u][j] = 0u;
        }
        // row-rotated staging so that both the writes here and the row reads below are spread over banks
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int j = 0; j < 8; ++j)
            stg[lane * EPI_COLS + ((u * 8 + j + lane) & (EPI_COLS - 1))] =
                make_float2(__uint_as_float(r[u][2 * j]) * sc, __uint_as_float(r[u][2 * j + 1]) * sc);
        __syncwarp();
        const int nc0 = n0 + c / 2;
        // 16 pairs of complex values per lane: two 256-byte row segments per warp instruction
        float4 old[16];
        if (p.accumulate) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int idx = i * 32 + lane;
            const int rr = idx >> 4, pc = (idx & 15) * 2;
            const int gm = r0 + rr, gn = nc0 + pc;
            const float2* o = cb + (long)gm * p.ldc + gn;
            const bool full2 = gm < p.M && gn + 1 < p.N && ((reinterpret_cast<uintptr_t>(o) & 15) == 0);
            old[i] = full2 ? *reinterpret_cast<const float4*>(o) : make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int idx = i * 32 + lane;
          const int rr = idx >> 4, pc = (idx & 15) * 2;
          const int gm = r0 + rr, gn = nc0 + pc;
          if (gm >= p.M) continue;
          float2 v0 = stg[rr * EPI_COLS + ((pc + rr) & (EPI_COLS - 1))];
          float2 v1 = stg[rr * EPI_COLS + ((pc + 1 + rr) & (EPI_COLS - 1))];
          float2* o = cb + (long)gm * p.ldc + gn;
          const bool ok0 = gn < p.N && (!TRI || gn <= gm);
          const bool ok1 = gn + 1 < p.N && (!TRI || gn + 1 <= gm);
          if (gn + 1 < p.N && ((reinterpret_cast<uintptr_t>(o) & 15) == 0) && ok0 && ok1) {
            if (p.accumulate) {
              v0.x += old[i].x;
              v0.y += old[i].y;
              v1.x += old[i].z;
              v1.y += old[i].w;
            }
            *reinterpret_cast<float4*>(o) = make_float4(v0.x, v0.y, v1.x, v1.y);
          } else {
            if (ok0) {
              if (p.accumulate) {
                v0.x += o[0].x;
                v0.y += o[0].y;
              }
              o[0] = v0;
            }
            if (ok1) {
              if (p.accumulate) {
                v1.x += o[1].x;
                v1.y += o[1].y;
              }
              o[1] = v1;
            }
          }
        }
        __syncwarp();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[b]);
      ++tl;
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

// max |component| of an outer x inner block of a strided matrix (batch entry
// blockIdx.y): one warp per row, lanes along the row, four loads in flight.
__global__ void __launch_bounds__(256) maxabs2d_kernel(const float2* __restrict__ X, long ld, int outer, int inner,
                                                       long sx, unsigned int* __restrict__ out) {
  X += blockIdx.y * sx;
  out += blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  float m = 0.f;
  for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < outer; i += gridDim.x * wpb) {
    const float2* row = X + (long)i * ld;
    for (int j0 = lane; j0 < inner; j0 += 128) {
      float2 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = j0 + 32 * u < inner ? __ldg(row + j0 + 32 * u) : make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 4; ++u) m = fmaxf(m, fmaxf(fabsf(v[u].x), fabsf(v[u].y)));
    }
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) atomicMax(out, __float_as_uint(m));   // non-negative floats order as uints
}

// Split operand rows.  Element (i, k) of op(X) (i < rows, k < K; padding
// columns up to kp/2 are zero) goes to real columns 2k, 2k+1 of row i (A form)
// or of rows 2i and 2i+1 as (br, -bi), (bi, br) (B form).  A 32 x 32 shared
// tile makes both the read and the write coalesced for either layout.
template <bool IS_B, uint32_t FMT>
__global__ void __launch_bounds__(256) prep_op_kernel(const float2* __restrict__ X, long ld, long sx, int trans,
                                                      int conj, int rows, int K, int kp,
                                                      const unsigned int* __restrict__ maxbits,
                                                      uint16_t* __restrict__ hi, uint16_t* __restrict__ lo) {
  __shared__ float2 t[32][33];                  // t[i][k]
  const int i0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  X += blockIdx.z * sx;
  const long ob = (long)blockIdx.z * (IS_B ? 2 : 1) * rows * kp;
  hi += ob;
  lo += ob;
  const float sc = ldexpf(1.0f, scale_exp(maxbits[blockIdx.z]));
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    // trans: X[k][i] is contiguous in i -> thread x walks i; else walks k
    const int i = trans ? i0 + threadIdx.x : i0 + y;
    const int k = trans ? k0 + y : k0 + threadIdx.x;
    float2 v = make_float2(0.f, 0.f);
    if (i < rows && k < K) {
      v = trans ? X[(long)k * ld + i] : X[(long)i * ld + k];
      if (conj) v.y = -v.y;
      v.x *= sc;
      v.y *= sc;
    }
    if (trans) t[threadIdx.x][y] = v;
    else t[y][threadIdx.x] = v;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int i = i0 + y, k = k0 + threadIdx.x;
    if (i >= rows || 2 * k >= kp) continue;
    const float2 v = t[y][threadIdx.x];
    uint16_t h0, l0, h1, l1;
    split<FMT>(v.x, h0, l0);
    split<FMT>(v.y, h1, l1);
    if (!IS_B) {
      const long o = (long)i * kp + 2 * k;
      reinterpret_cast<uint32_t*>(hi + o)[0] = (uint32_t)h0 | ((uint32_t)h1 << 16);
      reinterpret_cast<uint32_t*>(lo + o)[0] = (uint32_t)l0 | ((uint32_t)l1 << 16);
    } else {
      // rows 2i: (br, -bi); 2i+1: (bi, br)
      uint16_t h2, l2;
      split<FMT>(-v.y, h2, l2);
      const long o0 = (long)(2 * i) * kp + 2 * k, o1 = o0 + kp;
      reinterpret_cast<uint32_t*>(hi + o0)[0] = (uint32_t)h0 | ((uint32_t)h2 << 16);
      reinterpret_cast<uint32_t*>(lo + o0)[0] = (uint32_t)l0 | ((uint32_t)l2 << 16);
      reinterpret_cast<uint32_t*>(hi + o1)[0] = (uint32_t)h1 | ((uint32_t)h0 << 16);
      reinterpret_cast<uint32_t*>(lo + o1)[0] = (uint32_t)l1 | ((uint32_t)l0 << 16);
    }
  }
}

}  // namespace tg

size_t tc_gemm_scratch(int M, int N, int K, int batch) {
  const size_t kp = (size_t)(2 * std::max(K, 1) + tg::BK - 1) / tg::BK * tg::BK;
  Carver probe(nullptr);
  probe.take<unsigned int>(256);
  probe.take<uint16_t>((size_t)batch * M * kp);
  probe.take<uint16_t>((size_t)batch * M * kp);
  probe.take<uint16_t>((size_t)batch * 2 * N * kp);
  probe.take<uint16_t>((size_t)batch * 2 * N * kp);
  return Carver::round(probe.off);
}

gw_status tc_gemm(gw_ctx* ctx, gw_prec prec, const TcGemm& g, void* scratch, cudaStream_t st) {
  using namespace tg;
  if (g.M <= 0 || g.N <= 0) return GW_OK;
  const int batch = std::max(g.batch, 1);
  if (batch > 128) return fail(ctx, GW_ERR_SHAPE, "tensor-core GEMM batch above 128");
  const uint32_t fmt = prec == GW_BF16X3 ? 1u : 0u;
  const int K = std::max(g.K, 1);
  const int kp = (2 * K + BK - 1) / BK * BK;
  Carver cv(scratch);
  unsigned int* words = cv.take<unsigned int>(256);    // [b] max A, [batch + b] max B
  uint16_t* ahi = cv.take<uint16_t>((size_t)batch * g.M * kp);
  uint16_t* alo = cv.take<uint16_t>((size_t)batch * g.M * kp);
  uint16_t* bhi = cv.take<uint16_t>((size_t)batch * 2 * g.N * kp);
  uint16_t* blo = cv.take<uint16_t>((size_t)batch * 2 * g.N * kp);
  gw_status rc;
  if ((rc = cuda_check(ctx, cudaMemsetAsync(words, 0, 2 * batch * sizeof(unsigned int), st), "memset"))) return rc;
  // A is [M][K] (or [K][M] if transposed); B's op is [K][N]: stored [K][N], or [N][K] if transposed
  const int a_out = g.a_trans ? g.K : g.M, a_in = g.a_trans ? g.M : g.K;
  const int b_out = g.b_trans ? g.N : g.K, b_in = g.b_trans ? g.K : g.N;
  // the same stored elements (A A^H-type products) share one scan
  const bool same = g.A == g.B && g.lda == g.ldb && g.sA == g.sB && a_out == b_out && a_in == b_in;
  auto blocks_for = [&](int outer) {
    return (int)std::max(1L, std::min<long>((outer + 7) / 8, (long)ctx->num_sms * 8 / batch));
  };
  maxabs2d_kernel<<<dim3(blocks_for(a_out), batch), 256, 0, st>>>(g.A, g.lda, a_out, a_in, g.sA, words);
  if (!same)
    maxabs2d_kernel<<<dim3(blocks_for(b_out), batch), 256, 0, st>>>(g.B, g.ldb, b_out, b_in, g.sB, words + batch);
  else if ((rc = cuda_check(ctx, cudaMemcpyAsync(words + batch, words, batch * sizeof(unsigned int),
                                                  cudaMemcpyDeviceToDevice, st), "copy max")))
    return rc;
  if ((rc = launch_check(ctx, "maxabs2d_kernel"))) return rc;
  if (!same) ctx->launches++;            // launch_check counted one
  const dim3 tb(32, 8);
  const dim3 ga((g.M + 31) / 32, (kp / 2 + 31) / 32, batch), gb((g.N + 31) / 32, (kp / 2 + 31) / 32, batch);
  // B operand rows are indexed by n with k along the row: element (n, k) = opB(k, n), i.e.
  // B[k][n] (stored [K][N]: read transposed) or B[n][k] (b_trans: read as is).
  if (fmt == 0) {
    prep_op_kernel<false, 0><<<ga, tb, 0, st>>>(g.A, g.lda, g.sA, g.a_trans, g.a_conj, g.M, g.K, kp, words, ahi, alo);
    prep_op_kernel<true, 0><<<gb, tb, 0, st>>>(g.B, g.ldb, g.sB, !g.b_trans, g.b_conj, g.N, g.K, kp, words + batch,
                                                bhi, blo);
  } else {
    prep_op_kernel<false, 1><<<ga, tb, 0, st>>>(g.A, g.lda, g.sA, g.a_trans, g.a_conj, g.M, g.K, kp, words, ahi, alo);
    prep_op_kernel<true, 1><<<gb, tb, 0, st>>>(g.B, g.ldb, g.sB, !g.b_trans, g.b_conj, g.N, g.K, kp, words + batch,
                                                bhi, blo);
  }
  if ((rc = launch_check(ctx, "prep_op_kernel"))) return rc;
  ctx->launches++;
  CUtensorMap mah, mal, mbh, mbl;
  if ((rc = tc_make_map3(ctx, &mah, ahi, kp, g.M, batch, BM, fmt, BK))) return rc;
  if ((rc = tc_make_map3(ctx, &mal, alo, kp, g.M, batch, BM, fmt, BK))) return rc;
  if ((rc = tc_make_map3(ctx, &mbh, bhi, kp, 2L * g.N, batch, 2 * BNC, fmt, BK))) return rc;
  if ((rc = tc_make_map3(ctx, &mbl, blo, kp, 2L * g.N, batch, 2 * BNC, fmt, BK))) return rc;
  KParams P;
  P.M = g.M;
  P.N = g.N;
  P.k_steps = kp / BK;
  P.batch = batch;
  P.tm = (g.M + BM - 1) / BM;
  P.tn = (g.N + BNC - 1) / BNC;
  P.C = g.C;
  P.ldc = g.ldc;
  P.sC = g.sC;
  P.alpha = g.alpha;
  P.accumulate = g.accumulate ? 1 : 0;
  P.maxbits = words;
  P.status = g.status;
  long tiles = 0;                                       // tiles with work (lower ones only for tri)
  for (int bm = 0; bm < P.tm; ++bm) tiles += g.tri ? std::min(bm + 1, P.tn) : P.tn;
  tiles *= batch;
  const dim3 grid((unsigned)std::max<long>(1, std::min<long>(tiles, ctx->num_sms)));
  auto go = [&](auto kernel) -> gw_status {
    gw_status r = cuda_check(ctx, cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES),
                             "cudaFuncSetAttribute");
    if (r) return r;
    KTimer kt(ctx, KF_CGEMM_TC, batch * gemm_flops(g.M, g.N, g.K, g.tri), st);
    kernel<<<grid, THREADS, SMEM_BYTES, st>>>(mah, mal, mbh, mbl, P);
    return launch_check(ctx, "cgemm_tc_kernel");
  };
  if (fmt == 0) rc = g.tri == 0 ? go(cgemm_tc_kernel<0, 0>) : g.tri == 1 ? go(cgemm_tc_kernel<0, 1>) : go(cgemm_tc_kernel<0, 2>);
  else rc = g.tri == 0 ? go(cgemm_tc_kernel<1, 0>) : g.tri == 1 ? go(cgemm_tc_kernel<1, 1>) : go(cgemm_tc_kernel<1, 2>);
  return rc;
}

}  // namespace gw
