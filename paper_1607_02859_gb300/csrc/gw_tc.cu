// Tensor-core (tcgen05) formation of the imaginary-time Green's functions
// (Eqs. Green_occ, Green_unocc) and of the real-space product of Eq. chi_rr.
//
// Complex products on real tensor cores.  With a(r,k) = psi_k(r) s_k and
// b(R',k) = conj(psi_k(R')), G(r,R') = sum_k a(r,k) b(R',k) is one real GEMM
//   D[r][2R'+c] = sum_k' A[r][k'] B[2R'+c][k']     (k' = 2k, 2k+1)
// where A is the complex array viewed as real (re, im interleaved along k) and B
// holds two real rows per complex column:
//   B[2R'  ] = ( br_k, -bi_k )   ->  D[r][2R'  ] = Re G(r,R')
//   B[2R'+1] = ( bi_k,  br_k )   ->  D[r][2R'+1] = Im G(r,R')
// so the FP32 accumulator in tensor memory already holds (re, im) pairs.
//
// FP32-level accuracy from 16-bit tensor cores: every operand is split as
// x = hi + lo (hi = fp16(x), lo = fp16(x - hi)) after a power-of-two scaling
// that puts max|x| near 2^15, and D = A_hi B_hi + A_hi B_lo + A_lo B_hi
// (dropping A_lo B_lo ~ 2^-22 |A||B|), accumulated in FP32.  bf16 splits are
// the same code with a coarser 2 x 8-bit representation.
//
// Tile: 128 rows r x 128 complex columns R' (MMA 128 x 256 x 16), K staged 32
// real elements (64 B, SWIZZLE_64B) at a time through a 4-stage TMA/mbarrier
// pipeline; the epilogue stages rows in shared memory and writes 128-byte row
// segments.  G_unocc is summed blockwise through the two 256-column halves of
// tensor memory into registers, G_occ accumulates last in one half; the
// epilogue either writes both (gw_green_tau) or their product
// chi = -2 G_occ conj(G_unocc) (gw_chi0_rtau_fused), so for chi neither G tile
// ever reaches HBM.  Warp roles: 0 = TMA producer, 1 = MMA issuer (and tensor
// memory owner), 2..9 = epilogue.  Every wait is bounded; on time-out the
// kernel records it in the status word, drains its own copies and MMAs, frees
// its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>
#include <mutex>

#include "gw_tc.h"
#include "gw_tcgen05.cuh"

namespace gw {
namespace tc {

using namespace tcx;

constexpr int BM = 128;                 // rows per tile
constexpr int BNC = 128;                // complex columns per tile (MMA N = 256)
constexpr int BK = 32;                  // real K per stage (one 64-byte swizzle row)
constexpr int STAGES = 4;
constexpr int CH = 4;                   // stages per accumulation block (128 real K)
constexpr int EPI_WARPS = 8;            // two per tensor-memory lane quarter, one per column half
constexpr int A_BYTES = BM * BK * 2;            // 8 KB
constexpr int B_BYTES = 2 * BNC * BK * 2;       // 16 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int EPI_COLS = 16;                    // complex columns per epilogue round
constexpr int EPI_BYTES = EPI_WARPS * 32 * EPI_COLS * 8;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + EPI_BYTES + 1024 + 256;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
static_assert(SMEM_BYTES <= 232448, "shared memory per CTA");

struct Params {
  int m_rows;             // valid output rows
  int n_cols;             // valid complex output columns (N_r)
  int k_occ_steps;        // BK stages of the occupied region
  int k_un_steps;         // BK stages of the unoccupied region
  int k_un_x;             // first real K index of the unoccupied region
  float2* out0;           // chi, or G_occ
  float2* out1;           // G_unocc (green mode)
  long ldo;
  float alpha_occ;        // A_occ (FP64 max exponential, rounded) times 2^{-2e}
  float alpha_un;
  const int* dexp;        // device: e of the 2^e operand scaling
  int* status;            // device: [0] time-out flag, [1] where
  // MODE 2 (self-energy): contraction of G o W~ with psi_n on the tensor cores
  const float2* wrr;      // W~(r, R') rows of the block, [m_rows][ldw]
  long ldw;
  const float2* psi;      // psi [N_b][ldpsi]: psi_n(r) for the final sum over r
  long ldpsi;
  const int* bands;       // [n_n] device
  int n_n, np;            // bands; MMA N = 2 n_n rounded up to 16
  int r0;                 // grid row of the block's first row
  double coef;            // dV^2 / Omega
  double* acc_u;          // Sigma_unocc_nn(tau_j) at acc_u[n * acc_stride], Sigma_occ likewise
  double* acc_o;
  int acc_stride;
  // MODE 0 and 2: only tiles with R' <= r (the grid row of the tile's rows is r0 + local row).
  // chi(r,R') and G(r,R') W~(r,R') are Hermitian in (r, R'): MODE 0 writes the lower triangle with
  // the diagonal halved (T, so that the transform of chi is X + X^H with X that of T) and zeros
  // above; MODE 2 weights the strictly lower part 2 and the diagonal 1 (the real quadratic form).
  int lower;
};

// Blocked accumulation.  The tensor cores add each MMA's products into the FP32
// accumulator without rounding to nearest, so the relative error of a long
// accumulation grows about linearly with the number of MMAs (3 per 16 real K
// here): ~1e-5 for a thousand bands.  G_unocc is therefore summed in blocks of
// CH stages: each block accumulates from zero in one of the two 256-column
// halves of tensor memory while the epilogue warps add the other half's
// finished block into FP32 registers (round to nearest), which keeps the
// error at the level of one block.  G_occ (the short sum over the occupied
// bands) follows as the last block and stays in tensor memory for the
// epilogue.
//
// MODE 0: out0 = -2 G_occ conj(G_unocc);  MODE 1: out0 = G_occ, out1 = G_unocc.
// MODE 2: the self-energy contraction of the tile (first term of Eq.
// Sigma_occ_reduce, Eq. Sigma_rr), with nothing written but the band sums:
//   H(r,R') = G(r,R') W~(r,R')                        (CUDA cores, FP32)
//   V_n(r)  = sum_{R' in tile} H(r,R') psi_n(R')      (tcgen05, 3 fp16 split products)
//   Sigma_unocc_nn += coef Re(conj(psi_n(r)) V_n^unocc(r)),  Sigma_occ_nn -= ... V_n^occ
// Once the tile's G is complete the pipeline stages are free: the epilogue
// writes H row by row (its own power-of-two scale per row and column half) as
// split fp16 in the 64-byte-swizzled K-major layout TMA would produce, the
// producer loads the tile's psi_n operand behind it, and the MMA warp
// accumulates V for each half of the tile's columns in the free half of
// tensor memory; unoccupied first, then occupied in the same shared memory.
template <int MODE, uint32_t FMT>
__global__ void __launch_bounds__(THREADS, 1) green_tc_kernel(const __grid_constant__ CUtensorMap mA_hi,
                                                              const __grid_constant__ CUtensorMap mA_lo,
                                                              const __grid_constant__ CUtensorMap mB_hi,
                                                              const __grid_constant__ CUtensorMap mB_lo,
                                                              const __grid_constant__ CUtensorMap mP_hi,
                                                              const __grid_constant__ CUtensorMap mP_lo, Params p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float2* epi = reinterpret_cast<float2*>(smem + STAGES * STAGE_BYTES);     // [8 warps][32 rows][16]
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES + EPI_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;      // [2] block finished in tensor-memory half b
  uint64_t* tempty = tfull + 2;          // [2] half b drained by the epilogue
  uint64_t* done = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  // MODE 2
  uint64_t* hready = done + 2;           // [2] H operand of column half h written (4 warps)
  uint64_t* hfree = hready + 2;          // [2] unoccupied MMAs of half h done: its H may be overwritten
  uint64_t* vready = hfree + 2;          // [2] every V MMA of half h done
  uint64_t* psi_full = vready + 2;       // psi_n operand of the tile landed
  uint64_t* redbar = psi_full + 1;       // the epilogue warps' band sums are in shared memory
  uint64_t* done2 = redbar + 1;          // every MMA of the self-energy phase done
  double* red = reinterpret_cast<double*>(epi);   // [2][32] band sums of the CTA (MODE 2 only)

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // tiles in groups of kGroupRows row tiles: the CTAs that run together walk a group's rows for
  // each column tile, so they share B (and A) tiles in L2 instead of each reading its B from DRAM
  int m0, n0;
  {
    constexpr int kGroupRows = 8;
    const int gx = gridDim.x, gy = gridDim.y;
    const int id = blockIdx.y * gx + blockIdx.x;
    const int per = kGroupRows * gx, grp = id / per, first = grp * kGroupRows;
    const int rows = min(kGroupRows, gy - first), r = id - grp * per;
    m0 = (first + r % rows) * BM;
    n0 = (r / rows) * BNC;
  }
  const long grow0 = (long)p.r0 + m0;                 // grid row of the tile's first row
  if (MODE != 1 && p.lower && n0 >= grow0 + BM) {
    // every R' of the tile is above every r: zeros (chi), or nothing (self-energy)
    if (MODE == 0) {
      for (int idx = threadIdx.x; idx < BM * (BNC / 2); idx += blockDim.x) {
        const int row = idx / (BNC / 2), pc = 2 * (idx % (BNC / 2));
        const int gm = m0 + row, gn = n0 + pc;
        if (gm >= p.m_rows || gn >= p.n_cols) continue;
        float2* o = p.out0 + (long)gm * p.ldo + gn;
        if (gn + 1 < p.n_cols && ((reinterpret_cast<uintptr_t>(o) & 15) == 0)) {
          *reinterpret_cast<float4*>(o) = make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
          o[0] = make_float2(0.f, 0.f);
          if (gn + 1 < p.n_cols) o[1] = make_float2(0.f, 0.f);
        }
      }
    }
    return;
  }
  const bool diag_tile = MODE != 1 && p.lower && n0 + BNC > grow0;   // the tile meets the diagonal
  const int total = p.k_occ_steps + p.k_un_steps;
  const int n_un_blocks = (p.k_un_steps + CH - 1) / CH;
  const bool have_occ = p.k_occ_steps > 0;

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
    if (MODE == 2) {
      for (int b = 0; b < 2; ++b) {
        mbar_init(&hready[b], 4);
        mbar_init(&hfree[b], 1);
        mbar_init(&vready[b], 1);
      }
      mbar_init(psi_full, 1);
      mbar_init(redbar, EPI_WARPS);
      mbar_init(done2, 1);
      for (int i = 0; i < 64; ++i) red[i] = 0.0;
    }
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
  // MODE 2 operands in the freed pipeline stages: H hi [0, 64 KB), H lo [64, 128 KB) as eight
  // 32-wide K chunks of 128 rows; psi_n hi and lo from 128 KB, chunks of np rows.
  uint8_t* const h_hi = smem;
  uint8_t* const h_lo = smem + 8 * A_BYTES;
  uint8_t* const p_hi = smem + 16 * A_BYTES;
  const int p_chunk = MODE == 2 ? p.np * BK * 2 : 0;
  uint8_t* const p_lo = p_hi + 8 * p_chunk;

  auto timed_out = [&](int where) {
    *abort_flag = 1;
    if (atomicCAS(p.status, 0, 1) == 0) p.status[1] = where;
  };
  // bounded wait that also gives up once another role has aborted
  auto wait_or_abort = [&](uint64_t* bar, uint32_t parity) -> bool {
    const unsigned long long t0 = gtimer();
    while (!mbar_test(bar, parity)) {
      if (*abort_flag) return false;
      if (gtimer() - t0 > kWaitNs) return false;
    }
    return true;
  };

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------- TMA producer (unoccupied K first)
    int issued = 0;
    for (int it = 0; it < total && !*abort_flag; ++it) {
      const int s = it % STAGES;
      if (it >= STAGES && !mbar_wait(&empty[s], ((it / STAGES) & 1) ^ 1)) {
        timed_out(1);
        break;
      }
      uint8_t* st = smem + s * STAGE_BYTES;
      const int x = it < p.k_un_steps ? p.k_un_x + it * BK : (it - p.k_un_steps) * BK;
      mbar_expect_tx(&full[s], STAGE_BYTES);
      tma_load_3d(st, &mA_hi, &full[s], x, m0, 0);
      tma_load_3d(st + A_BYTES, &mA_lo, &full[s], x, m0, 0);
      tma_load_3d(st + 2 * A_BYTES, &mB_hi, &full[s], x, 2 * n0, 0);
      tma_load_3d(st + 2 * A_BYTES + B_BYTES, &mB_lo, &full[s], x, 2 * n0, 0);
      issued = it + 1;
    }
    if (*abort_flag) {
      // let our own copies land before the CTA exits
      for (int it = issued - STAGES < 0 ? 0 : issued - STAGES; it < issued; ++it)
        mbar_wait(&full[it % STAGES], (it / STAGES) & 1);
    } else if constexpr (MODE == 2) {
      // the tile's psi_n operand, once every MMA of the G formation has read its stages
      if (wait_or_abort(done, 0)) {
        mbar_expect_tx(psi_full, (uint32_t)(16 * p_chunk));
        for (int cc = 0; cc < 8; ++cc) {
          tma_load_3d(p_hi + cc * p_chunk, &mP_hi, psi_full, 2 * n0 + cc * BK, 0, 0);
          tma_load_3d(p_lo + cc * p_chunk, &mP_lo, psi_full, 2 * n0 + cc * BK, 0, 0);
        }
        mbar_wait(psi_full, 0);    // our copies land before the CTA can exit
      } else if (!*abort_flag) {
        timed_out(6);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------------------------------------------------- MMA issuer
    constexpr uint32_t idesc = make_idesc(FMT, 2 * BNC, BM);
    const int n_blocks = n_un_blocks + (have_occ ? 1 : 0);
    int it = 0;
    bool ok = true;
    for (int c = 0; c < n_blocks && ok; ++c) {
      const int b = c & 1, use = c >> 1;
      const int first = c < n_un_blocks ? c * CH : p.k_un_steps;
      const int last = c < n_un_blocks ? min(p.k_un_steps, (c + 1) * CH) : total;
      if (use > 0 && !wait_or_abort(&tempty[b], (use - 1) & 1)) {
        if (!*abort_flag) timed_out(4);
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d = tmem + (uint32_t)(b * 256);
      for (; it < last; ++it) {
        const int s = it % STAGES;
        if (!wait_or_abort(&full[s], (it / STAGES) & 1)) {
          if (!*abort_flag) timed_out(2);
          ok = false;
          break;
        }
        tc_fence_after();
        uint8_t* st = smem + s * STAGE_BYTES;
        const uint64_t ah = sw64_desc(st), al = sw64_desc(st + A_BYTES);
        const uint64_t bh = sw64_desc(st + 2 * A_BYTES), bl = sw64_desc(st + 2 * A_BYTES + B_BYTES);
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint64_t off = (uint64_t)(kk * 32) >> 4;    // 16 elements = 32 bytes along K
          umma(d, ah + off, bh + off, idesc, (it > first || kk > 0) ? 1u : 0u);
          umma(d, ah + off, bl + off, idesc, 1u);
          umma(d, al + off, bh + off, idesc, 1u);
        }
        umma_commit(&empty[s]);
      }
      if (ok) umma_commit(&tfull[b]);
    }
    umma_commit(done);     // arrives once every MMA issued above has completed
    if (!mbar_wait(done, 0)) timed_out(5);
    if constexpr (MODE == 2) {
      // V accumulators [occ][half] of np columns each in the tensor-memory half the
      // last G_unocc block used (drained before the epilogue signals hready)
      const uint32_t vbase = tmem + (uint32_t)((1 - (n_un_blocks & 1)) * 256);
      const uint32_t idesc2 = make_idesc(FMT, p.np, BM);
      bool go = ok && wait_or_abort(psi_full, 0);
      if (!go && !*abort_flag) timed_out(7);
      for (int o = 0; o < 2 && go; ++o) {
        for (int h = 0; h < 2 && go; ++h) {
          if (!wait_or_abort(&hready[h], (uint32_t)o)) {
            if (!*abort_flag) timed_out(8);
            go = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = vbase + (uint32_t)((2 * o + h) * p.np);
#pragma unroll 1
          for (int cc = 4 * h; cc < 4 * h + 4; ++cc) {
            const uint64_t ah = sw64_desc(h_hi + cc * A_BYTES), al = sw64_desc(h_lo + cc * A_BYTES);
            const uint64_t bh = sw64_desc(p_hi + cc * p_chunk), bl = sw64_desc(p_lo + cc * p_chunk);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              const uint64_t off = (uint64_t)(kk * 32) >> 4;
              umma(d, ah + off, bh + off, idesc2, (cc > 4 * h || kk > 0) ? 1u : 0u);
              umma(d, ah + off, bl + off, idesc2, 1u);
              umma(d, al + off, bh + off, idesc2, 1u);
            }
          }
          umma_commit(o == 0 ? &hfree[h] : &vready[h]);
        }
      }
      umma_commit(done2);
      if (!mbar_wait(done2, 0)) timed_out(9);
    }
  } else if (warp >= 2) {
    // ---------------------------------------------------------- epilogue
    const int ew = warp - 2;
    const int q = warp & 3;                       // tensor-memory lane quarter of this warp
    const int h = ew >> 2;                        // column half: real columns h*128 .. h*128+127
    const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
    float tot[128];                               // this thread's row of G_unocc, FP32 round-to-nearest sums
#pragma unroll
    for (int i = 0; i < 128; ++i) tot[i] = 0.f;
    bool ok = true;
    for (int c = 0; c < n_un_blocks; ++c) {
      const int b = c & 1;
      const bool got = wait_or_abort(&tfull[b], (c >> 1) & 1);
      if (!__all_sync(0xffffffffu, got)) {
        if (lane == 0 && !*abort_flag) timed_out(3);
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t base = tmem + lane_addr + (uint32_t)(b * 256 + h * 128);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        uint32_t x[16];
        tmem_ld16(base + 16 * u, x);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 16; ++i) tot[16 * u + i] += __uint_as_float(x[i]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[b]);
    }
    const int bo = n_un_blocks & 1;
    if (ok && have_occ) {
      const bool got = wait_or_abort(&tfull[bo], (n_un_blocks >> 1) & 1);
      if (!__all_sync(0xffffffffu, got)) {
        if (lane == 0 && !*abort_flag) timed_out(3);
        ok = false;
      }
      tc_fence_after();
    }
    // tcgen05.ld is warp-collective: the whole warp takes the same branch
    if (__all_sync(0xffffffffu, ok && !*abort_flag)) {
      const int r0 = m0 + q * 32;                   // first output row of this warp
      const float sc = ldexpf(1.0f, -2 * (*p.dexp));
      const float ao = p.alpha_occ * sc, au = p.alpha_un * sc;
      if constexpr (MODE == 2) {
        // ---------------------------------------------- self-energy contraction of the tile
        const int row = q * 32 + lane;               // tensor-memory lane = tile row
        const int gm = m0 + row;
        const bool rvalid = gm < p.m_rows;
        const float2* wrow = p.wrr + (long)(rvalid ? gm : 0) * p.ldw;
        const int c0 = n0 + h * 64;                   // first complex column of this warp's half
        const bool vec = (p.ldw % 2 == 0) && ((reinterpret_cast<uintptr_t>(p.wrr) & 15) == 0);
        // H = g tot o W~ in place; returns the power of two that puts the row's max below 2^15
        const long grow = grow0 + row;             // grid row r of this thread
        auto times_w = [&](float g) -> int {
          float m = 0.f;
#pragma unroll
          for (int c = 0; c < 64; c += 2) {
            const int gn = c0 + c;
            float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
            // weight of (r, R'): 2 below the diagonal, 1 on it, 0 above (lower-triangle mode)
            float wa = 1.f, wb = 1.f;
            if (p.lower) {
              wa = gn < grow ? 2.f : (gn == grow ? 1.f : 0.f);
              wb = gn + 1 < grow ? 2.f : (gn + 1 == grow ? 1.f : 0.f);
            }
            if (rvalid) {
              if (vec && gn + 1 < p.n_cols) {
                w = __ldg(reinterpret_cast<const float4*>(wrow + gn));
              } else {
                if (gn < p.n_cols) {
                  const float2 a = wrow[gn];
                  w.x = a.x;
                  w.y = a.y;
                }
                if (gn + 1 < p.n_cols) {
                  const float2 b = wrow[gn + 1];
                  w.z = b.x;
                  w.w = b.y;
                }
              }
            }
            const float ar = tot[2 * c] * g * wa, ai = tot[2 * c + 1] * g * wa;
            const float br = tot[2 * c + 2] * g * wb, bi = tot[2 * c + 3] * g * wb;
            tot[2 * c] = ar * w.x - ai * w.y;
            tot[2 * c + 1] = ar * w.y + ai * w.x;
            tot[2 * c + 2] = br * w.z - bi * w.w;
            tot[2 * c + 3] = br * w.w + bi * w.z;
            m = fmaxf(m, fmaxf(fmaxf(fabsf(tot[2 * c]), fabsf(tot[2 * c + 1])),
                               fmaxf(fabsf(tot[2 * c + 2]), fabsf(tot[2 * c + 3]))));
          }
          int ex = 0;
          if (m > 0.f) frexpf(m, &ex);
          return m > 0.f ? 14 - ex : 0;
        };
        // this row of H, scaled by 2^sh and split in two 16-bit parts, into K chunks
        // 4h..4h+3: row `row` of a chunk is 64 bytes at (row/8)*512 + (row%8)*64, its
        // 16-byte segment s stored at s ^ ((row/2) % 4) (the 64-byte swizzle of TMA)
        auto store_h = [&](int sh) {
          // 2^sh in two factors: a row of tiny H (W~ of a large tau decays like exp(-omega tau))
          // can need sh above 127, where one FP32 power of two would overflow
          const float s1 = ldexpf(1.0f, sh >> 1), s2 = ldexpf(1.0f, sh - (sh >> 1));
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int base = (4 * h + j) * A_BYTES + (row >> 3) * 512 + (row & 7) * 64;
#pragma unroll
            for (int sg = 0; sg < 4; ++sg) {
              uint32_t hw[4], lw[4];
#pragma unroll
              for (int t = 0; t < 4; ++t) {
                const int c = 16 * j + 4 * sg + t;
                uint16_t h0, l0, h1, l1;
                split<FMT>(tot[2 * c] * s1 * s2, h0, l0);
                split<FMT>(tot[2 * c + 1] * s1 * s2, h1, l1);
                hw[t] = (uint32_t)h0 | ((uint32_t)h1 << 16);
                lw[t] = (uint32_t)l0 | ((uint32_t)l1 << 16);
              }
              const int off = base + ((sg ^ ((row >> 1) & 3)) << 4);
              *reinterpret_cast<uint4*>(h_hi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
              *reinterpret_cast<uint4*>(h_lo + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the tensor cores
          __syncwarp();
        };
        const int shu = times_w(au);
        store_h(shu);
        if (lane == 0) mbar_arrive(&hready[h]);
        // G_occ of this row and half from tensor memory
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          uint32_t x[16];
          tmem_ld16(tmem + lane_addr + (uint32_t)(bo * 256 + h * 128 + 16 * u), x);
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < 16; ++i) tot[16 * u + i] = __uint_as_float(x[i]);
        }
        const int sho = times_w(ao);
        bool fine = wait_or_abort(&hfree[h], 0);     // the unoccupied MMAs have read this half
        if (__all_sync(0xffffffffu, fine)) {
          tc_fence_after();
          store_h(sho);
          if (lane == 0) mbar_arrive(&hready[h]);
          fine = wait_or_abort(&vready[h], 0);
        }
        if (__all_sync(0xffffffffu, fine)) {
          tc_fence_after();
          const uint32_t vb = tmem + lane_addr + (uint32_t)((1 - bo) * 256);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (16 * u < p.np) {                      // np is the same for the whole warp
              uint32_t x[16], y[16];
              tmem_ld16(vb + (uint32_t)(h * p.np + 16 * u), x);
              tmem_ld16(vb + (uint32_t)((2 + h) * p.np + 16 * u), y);
              tmem_wait_ld();
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                tot[16 * u + i] = __uint_as_float(x[i]);
                tot[64 + 16 * u + i] = __uint_as_float(y[i]);
              }
            }
          }
          // 2^-(sh + e) in two factors as well, applied one after the other, so that the
          // tiny rows come back as normal FP32 numbers where they are representable
          const int e = *p.dexp, ku = shu + e, ko = sho + e;
          const float fu1 = ldexpf(1.0f, -(ku >> 1)), fu2 = ldexpf(1.0f, -(ku - (ku >> 1)));
          const float fo1 = ldexpf(1.0f, -(ko >> 1)), fo2 = ldexpf(1.0f, -(ko - (ko >> 1)));
#pragma unroll
          for (int n = 0; n < 32; ++n) {
            if (n < p.n_n) {
              float2 ps = make_float2(0.f, 0.f);
              if (rvalid) ps = __ldg(p.psi + (long)p.bands[n] * p.ldpsi + grow);
              float su = (ps.x * tot[2 * n] + ps.y * tot[2 * n + 1]) * fu1 * fu2;    // Re(conj(psi_n) V_n)
              float so = (ps.x * tot[64 + 2 * n] + ps.y * tot[64 + 2 * n + 1]) * fo1 * fo2;
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) {
                su += __shfl_xor_sync(0xffffffffu, su, o);
                so += __shfl_xor_sync(0xffffffffu, so, o);
              }
              if (lane == 0) {
                atomicAdd(&red[n], (double)su);
                atomicAdd(&red[32 + n], (double)so);
              }
            }
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(redbar);
        } else if (lane == 0 && !*abort_flag) {
          timed_out(10);
        }
        // one warp adds the CTA's band sums into Sigma_unocc_nn(tau_j), Sigma_occ_nn(-tau_j)
        if (ew == 0) {
          const bool got = wait_or_abort(redbar, 0);
          if (got && lane < p.n_n) {
            atomicAdd(&p.acc_u[(long)lane * p.acc_stride], p.coef * red[lane]);
            atomicAdd(&p.acc_o[(long)lane * p.acc_stride], -p.coef * red[32 + lane]);
          } else if (!got && lane == 0 && !*abort_flag) {
            timed_out(11);
          }
        }
      } else {
        float2* stg = epi + ew * 32 * EPI_COLS;
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const int nc0 = n0 + h * 64 + cc * 16;
#pragma unroll
          for (int pass = 0; pass < (MODE == 0 ? 1 : 2); ++pass) {
            // row `lane` of the chunk to shared memory (rotated), then 128-byte row segments out
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              uint32_t ro[16];
              const bool need_occ = MODE == 0 || pass == 0;
              if (need_occ && have_occ) {
                tmem_ld16(tmem + lane_addr + (uint32_t)(bo * 256 + h * 128 + 32 * cc + 16 * u), ro);
                tmem_wait_ld();
              } else {
#pragma unroll
                for (int i = 0; i < 16; ++i) ro[i] = 0u;
              }
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const float gor = __uint_as_float(ro[2 * j]) * ao, goi = __uint_as_float(ro[2 * j + 1]) * ao;
                const float gur = tot[32 * cc + 16 * u + 2 * j] * au, gui = tot[32 * cc + 16 * u + 2 * j + 1] * au;
                float2 v;
                if (MODE == 0) {
                  v = make_float2(-2.0f * (gor * gur + goi * gui), -2.0f * (goi * gur - gor * gui));
                  if (diag_tile) {
                    const long rr = grow0 + q * 32 + lane, cn = nc0 + u * 8 + j;
                    const float f = cn < rr ? 1.f : (cn == rr ? 0.5f : 0.f);
                    v.x *= f;
                    v.y *= f;
                  }
                } else {
                  v = pass == 0 ? make_float2(gor, goi) : make_float2(gur, gui);
                }
                stg[lane * EPI_COLS + ((u * 8 + j + lane) & (EPI_COLS - 1))] = v;
              }
            }
            __syncwarp();
            float2* outp = (MODE == 0 || pass == 0) ? p.out0 : p.out1;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int idx = i * 32 + lane;
              const int rr = idx >> 3, pc = (idx & 7) * 2;
              const int gm = r0 + rr, gn = nc0 + pc;
              if (gm >= p.m_rows || gn >= p.n_cols) continue;
              const float2 v0 = stg[rr * EPI_COLS + ((pc + rr) & (EPI_COLS - 1))];
              const float2 v1 = stg[rr * EPI_COLS + ((pc + 1 + rr) & (EPI_COLS - 1))];
              float2* o = outp + (long)gm * p.ldo + gn;
              if (gn + 1 < p.n_cols && ((reinterpret_cast<uintptr_t>(o) & 15) == 0)) {
                *reinterpret_cast<float4*>(o) = make_float4(v0.x, v0.y, v1.x, v1.y);
              } else {
                o[0] = v0;
                if (gn + 1 < p.n_cols) o[1] = v1;
              }
            }
            __syncwarp();
          }
        }
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

// ---------------------------------------------------------------------- operand preparation

__global__ void maxabs_kernel(const float2* __restrict__ x, size_t n, unsigned int* __restrict__ out) {
  float m = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fmaxf(fabsf(x[i].x), fabsf(x[i].y)));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));   // non-negative floats order as uints
}

// e such that max|x| * 2^e lies in [2^14, 2^15)
__global__ void exponent_kernel(const unsigned int* __restrict__ maxbits, int* __restrict__ e) {
  const float m = __uint_as_float(*maxbits);
  int ex = 0;
  if (m > 0.f) {
    frexpf(m, &ex);        // m = f * 2^ex, f in [0.5, 1)
    *e = 15 - ex;
  } else {
    *e = 0;
  }
}

// Operand rows from psi [N_b][N_r] (band-major), transposed to K-major through a
// 32 x 32 shared tile.  Band k goes to real column kcol(k) = 2k (occupied) or
// k_un_x + 2(k - n_occ) (unoccupied); padding columns are written as zero.
//  A: row r (rows r0..r0+rows-1):  (ar, ai) * s_k * 2^e
//  B: rows 2R', 2R'+1:             (br, -bi) and (bi, br) of conj(psi) * 2^e
template <bool IS_B, uint32_t FMT>
__global__ void __launch_bounds__(256) prep_kernel(const float2* __restrict__ psi, int n_b, int n_occ, int nr, int r0,
                                                   int rows, const float* __restrict__ sk,
                                                   const int* __restrict__ dexp, int k_occ_pad, int k_un_x,
                                                   int kpad, uint16_t* __restrict__ hi, uint16_t* __restrict__ lo) {
  __shared__ float2 t[32][33];
  const int kb = blockIdx.y * 32;       // band tile (covers padded band slots)
  const int rb = blockIdx.x * 32;       // row tile
  const float sc = ldexpf(1.0f, *dexp);
  // band slot -> band index (or -1 for padding)
  const int occ_slots = k_occ_pad / 2, un_slots = (kpad - k_un_x) / 2;
  auto band_of = [&](int slot) -> int {
    if (slot < occ_slots) return slot < n_occ ? slot : -1;
    const int u = slot - occ_slots;
    return (u < un_slots && n_occ + u < n_b) ? n_occ + u : -1;
  };
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int band = band_of(kb + i);
    const int r = r0 + rb + threadIdx.x;
    float2 v = make_float2(0.f, 0.f);
    if (band >= 0 && rb + threadIdx.x < rows) {
      v = psi[(long)band * nr + r];
      const float s = IS_B ? sc : sc * sk[band];
      v.x *= s;
      v.y *= s;
    }
    t[i][threadIdx.x] = v;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int rr = rb + i;
    if (rr >= rows) continue;
    const int slot = kb + threadIdx.x;
    const int col = slot < occ_slots ? 2 * slot : k_un_x + 2 * (slot - occ_slots);
    if (col >= kpad) continue;
    const float2 v = t[threadIdx.x][i];
    uint16_t h0, l0, h1, l1;
    if (!IS_B) {
      split<FMT>(v.x, h0, l0);
      split<FMT>(v.y, h1, l1);
      const long o = (long)rr * kpad + col;
      reinterpret_cast<uint32_t*>(hi + o)[0] = (uint32_t)h0 | ((uint32_t)h1 << 16);
      reinterpret_cast<uint32_t*>(lo + o)[0] = (uint32_t)l0 | ((uint32_t)l1 << 16);
    } else {
      // b = conj(psi): br = v.x, bi = -v.y;  row 2R': (br, -bi) = (v.x, v.y); row 2R'+1: (bi, br) = (-v.y, v.x)
      split<FMT>(v.x, h0, l0);
      split<FMT>(v.y, h1, l1);
      const long o0 = (long)(2 * rr) * kpad + col;
      reinterpret_cast<uint32_t*>(hi + o0)[0] = (uint32_t)h0 | ((uint32_t)h1 << 16);
      reinterpret_cast<uint32_t*>(lo + o0)[0] = (uint32_t)l0 | ((uint32_t)l1 << 16);
      uint16_t h2, l2;
      split<FMT>(-v.y, h2, l2);
      const long o1 = o0 + kpad;
      reinterpret_cast<uint32_t*>(hi + o1)[0] = (uint32_t)h2 | ((uint32_t)h0 << 16);
      reinterpret_cast<uint32_t*>(lo + o1)[0] = (uint32_t)l2 | ((uint32_t)l0 << 16);
    }
  }
}

// The psi_n operand of the self-energy contraction (MODE 2): B rows 2n and 2n+1
// hold (br, -bi) and (bi, br) of b = psi_{bands[n]}(R') * 2^e along real K =
// 2R', 2R'+1, so that D[r][2n + c] = (Re, Im) sum_R' H(r,R') psi_n(R').  Rows of
// band slots n >= n_n (up to np/2) are zero.  One thread per (R', n).
template <uint32_t FMT>
__global__ void __launch_bounds__(256) prep_psin_kernel(const float2* __restrict__ psi, int nr,
                                                        const int* __restrict__ bands, int n_n, int kp,
                                                        const int* __restrict__ dexp, uint16_t* __restrict__ hi,
                                                        uint16_t* __restrict__ lo) {
  const int rp = blockIdx.x * 256 + threadIdx.x;
  const int n = blockIdx.y;
  if (2 * rp >= kp) return;
  float2 v = make_float2(0.f, 0.f);
  if (n < n_n && rp < nr) {
    v = psi[(long)bands[n] * nr + rp];
    const float sc = ldexpf(1.0f, *dexp);
    v.x *= sc;
    v.y *= sc;
  }
  uint16_t h0, l0, h1, l1, h2, l2;
  split<FMT>(v.x, h0, l0);
  split<FMT>(-v.y, h1, l1);
  split<FMT>(v.y, h2, l2);
  const long o0 = (long)(2 * n) * kp + 2 * rp, o1 = o0 + kp;
  reinterpret_cast<uint32_t*>(hi + o0)[0] = (uint32_t)h0 | ((uint32_t)h1 << 16);
  reinterpret_cast<uint32_t*>(lo + o0)[0] = (uint32_t)l0 | ((uint32_t)l1 << 16);
  reinterpret_cast<uint32_t*>(hi + o1)[0] = (uint32_t)h2 | ((uint32_t)h0 << 16);
  reinterpret_cast<uint32_t*>(lo + o1)[0] = (uint32_t)l2 | ((uint32_t)l0 << 16);
}

// ---------------------------------------------------------------------- host side

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeFn encoder(gw_ctx* ctx, gw_status* st) {
  static std::mutex mu;
  static EncodeFn fn = nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
      *st = fail(ctx, GW_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
      return nullptr;
    }
    fn = reinterpret_cast<EncodeFn>(p);
  }
  *st = GW_OK;
  return fn;
}

// 2-D map over a [rows][kpad] 16-bit row-major array, box = 64 x box_rows, 128-byte swizzle.
}  // namespace tc

gw_status tc_make_map(gw_ctx* ctx, CUtensorMap* m, const void* base, int kpad, long rows, int box_rows,
                      uint32_t fmt) {
  using namespace tc;
  gw_status st;
  EncodeFn enc = encoder(ctx, &st);
  if (!enc) return st;
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, fmt == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                   const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, GW_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return GW_OK;
}

gw_status tc_make_map3(gw_ctx* ctx, CUtensorMap* m, const void* base, int kpad, long rows, int batch, int box_rows,
                       uint32_t fmt, int box_k) {
  using namespace tc;
  gw_status st;
  EncodeFn enc = encoder(ctx, &st);
  if (!enc) return st;
  cuuint64_t dims[3] = {(cuuint64_t)kpad, (cuuint64_t)rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)kpad * 2, (cuuint64_t)kpad * 2 * (cuuint64_t)rows};
  cuuint32_t box[3] = {(cuuint32_t)box_k, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  if (box_k != 64 && box_k != 32) return fail(ctx, GW_ERR_ARG, "TMA box along K must be 32 or 64 elements");
  CUresult r = enc(m, fmt == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                   const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   box_k == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, GW_ERR_CUDA, "cuTensorMapEncodeTiled (3-D) failed (" + std::to_string((int)r) + ")");
  return GW_OK;
}

namespace tc {

struct Layout {
  int k_occ_pad, k_un_pad, k_un_x, kpad;
};
static Layout layout(int n_b, int n_occ) {
  Layout L;
  L.k_occ_pad = (2 * n_occ + BK - 1) / BK * BK;
  L.k_un_pad = (2 * (n_b - n_occ) + BK - 1) / BK * BK;
  L.k_un_x = L.k_occ_pad;
  L.kpad = L.k_occ_pad + L.k_un_pad;
  return L;
}

// MMA N of the self-energy contraction for n_sig bands, and the padded real K of its operand
static int sig_np(int n_sig) { return (2 * n_sig + 15) / 16 * 16; }
static int sig_kp(const GridInfo& g) { return (2 * g.nr + BK - 1) / BK * BK; }

static size_t scratch_bytes(const GridInfo& g, int n_b, int n_occ, int n_rows, bool with_tmp, int n_sig = 0) {
  const Layout L = layout(n_b, n_occ);
  Carver probe(nullptr);
  probe.take<unsigned int>(64);
  probe.take<float>(n_b);
  probe.take<uint16_t>((size_t)2 * g.nr * L.kpad);
  probe.take<uint16_t>((size_t)2 * g.nr * L.kpad);
  if (n_sig > 0) {
    probe.take<uint16_t>((size_t)sig_np(n_sig) * sig_kp(g));
    probe.take<uint16_t>((size_t)sig_np(n_sig) * sig_kp(g));
  }
  probe.take<uint16_t>((size_t)n_rows * L.kpad);
  probe.take<uint16_t>((size_t)n_rows * L.kpad);
  if (with_tmp) probe.take<float2>((size_t)n_rows * g.nr);
  return Carver::round(probe.off);
}

// One G/chi formation for rows r0 .. r0+n_rows-1 using `scratch` (of at least
// scratch_bytes()).  mode 0: chi into out0; mode 1: G_occ into out0 and G_unocc
// into out1 (a NULL one goes to scratch).  prep_b = false reuses the B operand
// and the operand scaling left in the same scratch by an earlier call for the
// same psi.
static gw_status run(gw_ctx* ctx, const GridInfo& g, int n_b, int n_occ, const void* psi, const GreenScales& gs,
                     int r0, int n_rows, gw_prec prec, int mode, void* out0, void* out1, void* scratch, bool prep_b,
                     cudaStream_t st, const float* sk_dev = nullptr, int* status_dev = nullptr,
                     const TcSigma* sig = nullptr, bool lower = false) {
  const uint32_t fmt = prec == GW_BF16X3 ? 1u : 0u;
  const Layout L = layout(n_b, n_occ);
  gw_status rc;
  const bool need_tmp = mode == 1 && (!out0 || !out1);
  Carver cv(scratch);
  unsigned int* dmax = cv.take<unsigned int>(64);
  int* dexp = reinterpret_cast<int*>(dmax + 1);
  // time-out status: in the scratch, or in a word the caller owns (kept past later uses of the scratch)
  int* status = status_dev ? status_dev : reinterpret_cast<int*>(dmax + 2);
  float* dsk = cv.take<float>(n_b);
  uint16_t* bhi = cv.take<uint16_t>((size_t)2 * g.nr * L.kpad);
  uint16_t* blo = cv.take<uint16_t>((size_t)2 * g.nr * L.kpad);
  // the psi_n operand is prepared by the first call and read by later ones: its place must
  // not depend on this call's number of rows, so it comes before the A operand
  const int np = mode == 2 ? sig_np(sig->n_n) : 0, kps = sig_kp(g);
  uint16_t* phi = mode == 2 ? cv.take<uint16_t>((size_t)np * kps) : nullptr;
  uint16_t* plo = mode == 2 ? cv.take<uint16_t>((size_t)np * kps) : nullptr;
  uint16_t* ahi = cv.take<uint16_t>((size_t)n_rows * L.kpad);
  uint16_t* alo = cv.take<uint16_t>((size_t)n_rows * L.kpad);
  float2* tmp = need_tmp ? cv.take<float2>((size_t)n_rows * g.nr) : nullptr;
  if (mode == 1) {
    if (!out0) out0 = tmp;
    if (!out1) out1 = tmp;
  }
  // per-band factors: uploaded here, or already on the device (sk_dev: no host-to-device copy in this call)
  const float* sk = sk_dev;
  if (!sk) {
    std::vector<float> skf(gs.s.begin(), gs.s.end());
    if ((rc = upload(ctx, dsk, skf.data(), sizeof(float) * n_b, st))) return rc;
    sk = dsk;
  }
  const dim3 tb(32, 8);
  const int slots = L.kpad / 2;
  if (prep_b) {
    if ((rc = cuda_check(ctx, cudaMemsetAsync(dmax, 0, 64 * sizeof(unsigned int), st), "memset"))) return rc;
    if (status_dev && (rc = cuda_check(ctx, cudaMemsetAsync(status_dev, 0, 2 * sizeof(int), st), "memset")))
      return rc;
    const size_t nel = (size_t)n_b * g.nr;
    maxabs_kernel<<<std::min<size_t>((nel + 255) / 256, (size_t)ctx->num_sms * 8), 256, 0, st>>>(
        static_cast<const float2*>(psi), nel, dmax);
    if ((rc = launch_check(ctx, "maxabs_kernel"))) return rc;
    exponent_kernel<<<1, 1, 0, st>>>(dmax, dexp);
    if ((rc = launch_check(ctx, "exponent_kernel"))) return rc;
    const dim3 gbB((g.nr + 31) / 32, (slots + 31) / 32);
    if (fmt == 0)
      prep_kernel<true, 0><<<gbB, tb, 0, st>>>((const float2*)psi, n_b, n_occ, g.nr, 0, g.nr, sk, dexp,
                                                L.k_occ_pad, L.k_un_x, L.kpad, bhi, blo);
    else
      prep_kernel<true, 1><<<gbB, tb, 0, st>>>((const float2*)psi, n_b, n_occ, g.nr, 0, g.nr, sk, dexp,
                                                L.k_occ_pad, L.k_un_x, L.kpad, bhi, blo);
    if ((rc = launch_check(ctx, "prep_kernel(B)"))) return rc;
    if (mode == 2) {
      const dim3 gp((kps / 2 + 255) / 256, np / 2);
      if (fmt == 0)
        prep_psin_kernel<0><<<gp, 256, 0, st>>>((const float2*)psi, g.nr, sig->bands, sig->n_n, kps, dexp, phi, plo);
      else
        prep_psin_kernel<1><<<gp, 256, 0, st>>>((const float2*)psi, g.nr, sig->bands, sig->n_n, kps, dexp, phi, plo);
      if ((rc = launch_check(ctx, "prep_psin_kernel"))) return rc;
    }
  } else {
    if ((rc = cuda_check(ctx, cudaMemsetAsync(status, 0, 2 * sizeof(int), st), "memset"))) return rc;
  }
  const dim3 gbA((n_rows + 31) / 32, (slots + 31) / 32);
  if (fmt == 0)
    prep_kernel<false, 0><<<gbA, tb, 0, st>>>((const float2*)psi, n_b, n_occ, g.nr, r0, n_rows, sk, dexp,
                                               L.k_occ_pad, L.k_un_x, L.kpad, ahi, alo);
  else
    prep_kernel<false, 1><<<gbA, tb, 0, st>>>((const float2*)psi, n_b, n_occ, g.nr, r0, n_rows, sk, dexp,
                                               L.k_occ_pad, L.k_un_x, L.kpad, ahi, alo);
  if ((rc = launch_check(ctx, "prep_kernel(A)"))) return rc;
  CUtensorMap mah, mal, mbh, mbl, mph, mpl;
  if ((rc = tc_make_map3(ctx, &mah, ahi, L.kpad, n_rows, 1, BM, fmt, BK))) return rc;
  if ((rc = tc_make_map3(ctx, &mal, alo, L.kpad, n_rows, 1, BM, fmt, BK))) return rc;
  if ((rc = tc_make_map3(ctx, &mbh, bhi, L.kpad, 2L * g.nr, 1, 2 * BNC, fmt, BK))) return rc;
  if ((rc = tc_make_map3(ctx, &mbl, blo, L.kpad, 2L * g.nr, 1, 2 * BNC, fmt, BK))) return rc;
  if (mode == 2) {
    if ((rc = tc_make_map3(ctx, &mph, phi, kps, np, 1, np, fmt, BK))) return rc;
    if ((rc = tc_make_map3(ctx, &mpl, plo, kps, np, 1, np, fmt, BK))) return rc;
  } else {
    mph = mah;                                   // unused outside the self-energy mode
    mpl = mal;
  }
  Params P;
  P.m_rows = n_rows;
  P.n_cols = g.nr;
  P.k_occ_steps = L.k_occ_pad / BK;
  P.k_un_steps = L.k_un_pad / BK;
  P.k_un_x = L.k_un_x;
  P.out0 = static_cast<float2*>(out0);
  P.out1 = static_cast<float2*>(mode == 1 ? out1 : out0);
  P.ldo = g.nr;
  P.alpha_occ = (float)gs.amax_occ;
  P.alpha_un = (float)gs.amax_unocc;
  P.dexp = dexp;
  P.status = status;
  P.wrr = nullptr;
  P.ldw = 0;
  P.psi = static_cast<const float2*>(psi);
  P.ldpsi = g.nr;
  P.bands = nullptr;
  P.n_n = 0;
  P.np = np;
  P.r0 = r0;
  P.coef = 0.0;
  P.acc_u = P.acc_o = nullptr;
  P.acc_stride = 0;
  P.lower = (mode != 1 && lower) ? 1 : 0;
  if (mode == 2) {
    P.wrr = sig->wrr;
    P.ldw = sig->ldw;
    P.bands = sig->bands;
    P.n_n = sig->n_n;
    P.coef = sig->coef;
    P.acc_u = sig->acc_u;
    P.acc_o = sig->acc_o;
    P.acc_stride = sig->acc_stride;
  }
  // lower-triangle self-energy: the column tiles past the block's last row hold no R' <= r
  const int col_end = (mode == 2 && P.lower) ? std::min(g.nr, r0 + n_rows) : g.nr;
  const dim3 grid((col_end + BNC - 1) / BNC, (n_rows + BM - 1) / BM);
  // multiply-adds the launch performs: full tiles, or those meeting R' <= r
  double tiles = (double)grid.x * grid.y;
  if (P.lower) {
    tiles = 0;
    for (unsigned by = 0; by < grid.y; ++by) {
      const long last_row = (long)r0 + by * BM + BM - 1;
      tiles += std::min<double>(grid.x, (double)(last_row / BNC + 1));
    }
  }
  const double tile_frac = tiles / ((double)((g.nr + BNC - 1) / BNC) * grid.y);
  auto go = [&](auto kernel) -> gw_status {
    gw_status r = cuda_check(ctx, cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES),
                             "cudaFuncSetAttribute");
    if (r) return r;
    const double work =
        tile_frac * (8.0 * n_rows * (double)g.nr * n_b + (mode == 2 ? 16.0 * n_rows * (double)g.nr * P.n_n : 0.0));
    KTimer kt(ctx, KF_GREEN_TC, work, st);
    kernel<<<grid, THREADS, SMEM_BYTES, st>>>(mah, mal, mbh, mbl, mph, mpl, P);
    return launch_check(ctx, "green_tc_kernel");
  };
  if (mode == 0) rc = fmt == 0 ? go(green_tc_kernel<0, 0>) : go(green_tc_kernel<0, 1>);
  else if (mode == 1) rc = fmt == 0 ? go(green_tc_kernel<1, 0>) : go(green_tc_kernel<1, 1>);
  else rc = fmt == 0 ? go(green_tc_kernel<2, 0>) : go(green_tc_kernel<2, 1>);
  return rc;
}

// Reads the status word the kernels' bounded waits write (synchronises the stream).
static gw_status check_status(gw_ctx* ctx, void* scratch, cudaStream_t st) {
  int hs[2] = {0, 0};
  const int* status = reinterpret_cast<const int*>(static_cast<const unsigned int*>(scratch) + 2);
  gw_status rc;
  if ((rc = cuda_check(ctx, cudaMemcpyAsync(hs, status, sizeof(hs), cudaMemcpyDeviceToHost, st), "status"))) return rc;
  if ((rc = cuda_check(ctx, cudaStreamSynchronize(st), "tensor-core GEMM"))) return rc;
  if (hs[0]) return fail(ctx, GW_ERR_TIMEOUT, "tensor-core pipeline wait timed out (role " + std::to_string(hs[1]) + ")");
  return GW_OK;
}

}  // namespace tc

size_t tc_scratch_bytes(const GridInfo& g, int n_b, int n_occ, int n_rows, bool with_tmp, int n_sig) {
  return tc::scratch_bytes(g, n_b, n_occ, n_rows, with_tmp, n_sig);
}

gw_status tc_sigma_rows(gw_ctx* ctx, const GridInfo& g, int n_b, int n_occ, const void* psi, const GreenScales& gs,
                        int r0, int n_rows, gw_prec prec, const TcSigma& sig, void* scratch, bool prep_b,
                        cudaStream_t st) {
  if (sig.n_n < 1 || sig.n_n > 32) return fail(ctx, GW_ERR_SHAPE, "fused self-energy contraction takes 1..32 bands");
  return tc::run(ctx, g, n_b, n_occ, psi, gs, r0, n_rows, prec, 2, nullptr, nullptr, scratch, prep_b, st, sig.sk,
                 nullptr, &sig, true);
}

gw_status tc_green_rows(gw_ctx* ctx, const GridInfo& g, int n_b, int n_occ, const void* psi, const GreenScales& gs,
                        int r0, int n_rows, gw_prec prec, void* g_occ, void* g_unocc, void* scratch, bool prep_b,
                        cudaStream_t st, const float* sk_dev) {
  return tc::run(ctx, g, n_b, n_occ, psi, gs, r0, n_rows, prec, 1, g_occ, g_unocc, scratch, prep_b, st, sk_dev);
}

gw_status tc_chi_rows(gw_ctx* ctx, const GridInfo& g, int n_b, int n_occ, const void* psi, const GreenScales& gs,
                      int r0, int n_rows, gw_prec prec, void* chi, void* scratch, bool prep_b, cudaStream_t st,
                      const float* sk_dev, int* status_dev, bool lower) {
  return tc::run(ctx, g, n_b, n_occ, psi, gs, r0, n_rows, prec, 0, chi, nullptr, scratch, prep_b, st, sk_dev,
                 status_dev, nullptr, lower);
}

gw_status tc_check_status(gw_ctx* ctx, const int* status_dev, cudaStream_t st) {
  int hs[2] = {0, 0};
  gw_status rc;
  if ((rc = cuda_check(ctx, cudaMemcpyAsync(hs, status_dev, sizeof(hs), cudaMemcpyDeviceToHost, st), "status"))) return rc;
  if ((rc = cuda_check(ctx, cudaStreamSynchronize(st), "tensor-core GEMM"))) return rc;
  if (hs[0]) return fail(ctx, GW_ERR_TIMEOUT, "tensor-core pipeline wait timed out (role " + std::to_string(hs[1]) + ")");
  return GW_OK;
}

gw_status tc_check(gw_ctx* ctx, void* scratch, cudaStream_t st) { return tc::check_status(ctx, scratch, st); }

}  // namespace gw
