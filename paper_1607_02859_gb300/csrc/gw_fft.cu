// Spatial transforms within the cell (Eqs. FFTX1, FFTX2, FFTW), the
// real-space product of Eq. chi_rr fused into the row transform, and the
// nonuniform time/frequency transforms (Eqs. CTX, CT_W, ST_FFT).
//
// Data stay in HBM as row-major complex matrices whose row index is a grid
// point r = (i1*n2+i2)*n3+i3 or a G-set index, and whose column index is a grid
// point R' or a G' of the set.
//  * row kernels: one CTA per row; the N_r-point row is staged in shared memory
//    (odd-padded pencil stride, so every pencil pass is bank-conflict free) and
//    transformed by three passes of fully unrolled register FFTs.
//  * column kernels: the transform runs over the row index for a chunk of
//    contiguous columns, so every HBM access is a coalesced row segment:
//    a "plane" kernel does the (i2,i3) 2-D FFT through shared memory and a
//    "line" kernel the i1 1-D FFT in registers.  The last i1 pass of the chi
//    chain also applies the cosine transform over all tau (Eq. CTX) before
//    anything is written, saving a full read+write of chi(G,G',tau).
#include <cooperative_groups.h>
#include <mutex>
#include <type_traits>

#include "gw_common.cuh"
#include "gw_kernels.h"
#include "gw_fft.cuh"

namespace gw {

bool grid_supported(int a, int b, int c) {
#define X(x, y, z) \
  if (a == x && b == y && c == z) return true;
  GW_GRIDS(X)
#undef X
  return false;
}

// MODE 0: x = scale * a * conj(b) (Eq. chi_rr), forward (+i), gather the G' set.
// MODE 1: x = a, forward (+i), gather.            (Eq. FFTX1)
// MODE 2: scatter a[j] to fft positions, backward (-i), times scale.   (Eq. FFTW, 2nd step)
// VEC: rows 16-byte aligned with even lengths; contiguous rows move as pairs of
// elements, four pairs in flight per thread.
template <typename T, int N1, int N2, int N3, int MODE, int THREADS, bool VEC>
__global__ void __launch_bounds__(THREADS) row_fft_kernel(const typename cpx<T>::t* __restrict__ a,
                                                          const typename cpx<T>::t* __restrict__ b, long lda,
                                                          typename cpx<T>::t* __restrict__ out, long ldo,
                                                          const int* __restrict__ map, int n_chi, T scale) {
  using C = typename cpx<T>::t;
  using L = RowLayout<N1, N2, N3>;
  constexpr int NP = L::NR / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const long row = blockIdx.x;
  if (MODE == 2) {
    for (int e = threadIdx.x; e < L::TOT; e += THREADS) s[e] = mk(T(0), T(0));
    __syncthreads();
    const C* src = a + row * lda;
    for (int j0 = threadIdx.x; j0 < n_chi; j0 += 4 * THREADS) {
      C v[4];
      int m[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = j0 + u * THREADS;
        if (j < n_chi) {
          v[u] = src[j];
          m[u] = map[j];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (j0 + u * THREADS < n_chi) s[L::pos(m[u])] = v[u];
    }
  } else {
    const C* pa = a + row * lda;
    const C* pb = b + row * lda;
    if (VEC) {
      for (int q0 = threadIdx.x; q0 < NP; q0 += 4 * THREADS) {
        C v[4][2], w[4][2];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int q = q0 + u * THREADS;
          if (q < NP) {
            ld_pair(pa + 2 * q, v[u][0], v[u][1]);
            if (MODE == 0) ld_pair(pb + 2 * q, w[u][0], w[u][1]);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int q = q0 + u * THREADS;
          if (q >= NP) continue;
          const int p = L::pos(2 * q);           // 2q and 2q+1 share an i3 pencil (N3 even)
          s[p] = MODE == 0 ? cscale(cmulc(v[u][0], w[u][0]), scale) : v[u][0];
          s[p + 1] = MODE == 0 ? cscale(cmulc(v[u][1], w[u][1]), scale) : v[u][1];
        }
      }
    } else {
      for (int r = threadIdx.x; r < L::NR; r += THREADS) {
        C v = pa[r];
        if (MODE == 0) v = cscale(cmulc(v, pb[r]), scale);
        s[L::pos(r)] = v;
      }
    }
  }
  __syncthreads();
  fft3_smem<N1, N2, N3, MODE == 2 ? -1 : +1>(s);
  C* dst = out + row * ldo;
  if (MODE == 2) {
    if (VEC) {
      for (int q = threadIdx.x; q < NP; q += THREADS) {
        const int p = L::pos(2 * q);
        st_pair(dst + 2 * q, cscale(s[p], scale), cscale(s[p + 1], scale));
      }
    } else {
      for (int r = threadIdx.x; r < L::NR; r += THREADS) dst[r] = cscale(s[L::pos(r)], scale);
    }
  } else {
    if (VEC) {
      for (int q = threadIdx.x; q < n_chi / 2; q += THREADS)
        st_pair(dst + 2 * q, s[L::pos(map[2 * q])], s[L::pos(map[2 * q + 1])]);
    } else {
      for (int j = threadIdx.x; j < n_chi; j += THREADS) dst[j] = s[L::pos(map[j])];
    }
  }
}

// Rows too long for shared memory (36^3 = 46656 points, 373 KB) take two
// passes through HBM.  The plane pass does the (i2, i3) 2-D transform of
// kRowPlanes consecutive planes of one row per CTA; the line pass does the i1
// transforms of one row per CTA in registers, with the G-set side of the row
// (n_chi values) held in shared memory: forward, the results are scattered
// there through inv and the row is written out in order; backward, the input
// row is staged there and gathered through inv.
constexpr int kRowPlanes = 4;

// MODE 0: x = scale a conj(b) -> out;  MODE 1: x = a -> out;  MODE 2: out in place, times scale.
template <typename T, int N1, int N2, int N3, int MODE, int DIR>
__global__ void __launch_bounds__(256) row_plane_kernel(const typename cpx<T>::t* a,
                                                        const typename cpx<T>::t* b, long lda,
                                                        typename cpx<T>::t* out, long ldo, T scale) {
  using C = typename cpx<T>::t;
  constexpr int S2 = N3 % 2 == 0 ? N3 + 1 : N3;      // odd pencil stride
  constexpr int PL = N2 * N3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);               // [kRowPlanes][N2][S2]
  const long row = blockIdx.y;
  const int i10 = blockIdx.x * kRowPlanes;
  const int np = min(kRowPlanes, N1 - i10);
  const long base = (long)i10 * PL;
  for (int e = threadIdx.x; e < np * PL; e += blockDim.x) {
    const int p = e / PL, rem = e - p * PL, i2 = rem / N3, i3 = rem - i2 * N3;
    C v;
    if (MODE == 2) {
      v = out[row * ldo + base + e];
    } else {
      v = a[row * lda + base + e];
      if (MODE == 0) v = cscale(cmulc(v, b[row * lda + base + e]), scale);
    }
    s[(p * N2 + i2) * S2 + i3] = v;
  }
  __syncthreads();
  pencil_pass<N3, DIR>(s, np * N2, 1, [](int q) { return q * S2; });
  __syncthreads();
  pencil_pass<N2, DIR>(s, np * N3, S2, [](int q) { return (q / N3) * (N2 * S2) + (q % N3); });
  __syncthreads();
  for (int e = threadIdx.x; e < np * PL; e += blockDim.x) {
    const int p = e / PL, rem = e - p * PL, i2 = rem / N3, i3 = rem - i2 * N3;
    const C v = s[(p * N2 + i2) * S2 + i3];
    out[row * ldo + base + e] = MODE == 2 ? cscale(v, scale) : v;
  }
}

// Forward line pass: i1 transforms (+i) of tmp's row, the G set scattered into
// shared memory through inv, then out[row][j], j < n_chi, in order.
template <typename T, int N1, int N2, int N3>
__global__ void __launch_bounds__(256) row_line_fwd_kernel(const typename cpx<T>::t* __restrict__ tmp, long ldt,
                                                           typename cpx<T>::t* __restrict__ out, long ldo,
                                                           const int* __restrict__ inv, int n_chi) {
  using C = typename cpx<T>::t;
  constexpr int PL = N2 * N3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* so = reinterpret_cast<C*>(smem_raw);              // [n_chi]
  const long row = blockIdx.x;
  for (int i23 = threadIdx.x; i23 < PL; i23 += blockDim.x) {
    C x[N1];
#pragma unroll
    for (int i1 = 0; i1 < N1; ++i1) x[i1] = tmp[row * ldt + (long)i1 * PL + i23];
    RegFFT<N1, +1>::run(x);
#pragma unroll
    for (int i1 = 0; i1 < N1; ++i1) {
      const int j = inv[i1 * PL + i23];
      if (j >= 0) so[j] = x[i1];
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n_chi; j += blockDim.x) out[row * ldo + j] = so[j];
}

// Backward line pass: a's row (n_chi values of the G set) staged in shared
// memory, gathered through inv into the grid, i1 transforms (-i) into out.
template <typename T, int N1, int N2, int N3>
__global__ void __launch_bounds__(256) row_line_bwd_kernel(const typename cpx<T>::t* __restrict__ a, long lda,
                                                           typename cpx<T>::t* __restrict__ out, long ldo,
                                                           const int* __restrict__ inv, int n_chi) {
  using C = typename cpx<T>::t;
  constexpr int PL = N2 * N3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* si = reinterpret_cast<C*>(smem_raw);              // [n_chi]
  const long row = blockIdx.x;
  for (int j = threadIdx.x; j < n_chi; j += blockDim.x) si[j] = a[row * lda + j];
  __syncthreads();
  for (int i23 = threadIdx.x; i23 < PL; i23 += blockDim.x) {
    C x[N1];
#pragma unroll
    for (int i1 = 0; i1 < N1; ++i1) {
      const int j = inv[i1 * PL + i23];
      x[i1] = j >= 0 ? si[j] : mk(T(0), T(0));
    }
    RegFFT<N1, -1>::run(x);
#pragma unroll
    for (int i1 = 0; i1 < N1; ++i1) out[row * ldo + (long)i1 * PL + i23] = x[i1];
  }
}

// Rows too long for one CTA's shared memory, split over a thread-block cluster
// of CL CTAs: CTA c holds planes i1 in [c P, (c+1) P) (P = N1 / CL) of the row
// and the slice [c n_s, (c+1) n_s) of its G-set side (n_s = ceil(n_chi / CL)).
// The (i2, i3) transforms run on the CTA's own planes; for the i1 transforms
// each CTA takes N2 N3 / CL of the (i2, i3) columns and reads and writes the
// other CTAs' planes and G-set slices through distributed shared memory.  Each
// element crosses HBM once, as for the one-CTA rows.
template <typename T, int N1, int N2, int N3>
struct ClusterRow {
  using C = typename cpx<T>::t;
  static constexpr int S2 = N3 % 2 == 0 ? N3 + 1 : N3;
  static constexpr int PL = N2 * N3;
  static constexpr size_t plane_bytes(int cl) { return (size_t)(N1 / cl) * N2 * S2 * sizeof(C); }
  static constexpr bool fits(int cl) {
    return N1 % cl == 0 && PL % cl == 0 && plane_bytes(cl) + 32768 <= 200 * 1024;
  }
  // the smallest cluster whose planes leave room for two CTAs per SM, else the smallest that fits
  static constexpr int pick() {
    for (int cl : {2, 4, 8})
      if (fits(cl) && plane_bytes(cl) <= 96 * 1024) return cl;
    for (int cl : {2, 4, 8})
      if (fits(cl)) return cl;
    return 0;
  }
  static constexpr int CL = pick();
  static constexpr int P = CL ? N1 / CL : 1;
  static constexpr int COLS = CL ? PL / CL : 1;
  // one thread per pencil of the local planes (P N2 = COLS when N2 = N3), two CTAs per SM
  static constexpr int THREADS = CL ? ((P * N2 > COLS ? P * N2 : COLS) + 1) / 2 : 32;
  static size_t smem(int n_chi) { return plane_bytes(CL) + (size_t)((n_chi + CL - 1) / CL) * sizeof(C); }
};

// MODE 0 / 1 / 2 as for row_fft_kernel; grid (CL, rows), clusters of CL along x.
template <typename T, int N1, int N2, int N3, int MODE, bool VEC>
__global__ void __launch_bounds__(ClusterRow<T, N1, N2, N3>::THREADS, 2)
    row_cluster_kernel(const typename cpx<T>::t* __restrict__ a, const typename cpx<T>::t* __restrict__ b, long lda,
                       typename cpx<T>::t* __restrict__ out, long ldo, const int* __restrict__ inv, int n_chi,
                       T scale) {
  namespace cg = cooperative_groups;
  using C = typename cpx<T>::t;
  using R = ClusterRow<T, N1, N2, N3>;
  constexpr int P = R::P, PL = R::PL, S2 = R::S2, COLS = R::COLS;
  constexpr int TH = R::THREADS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);                         // [P][N2][S2] own planes
  C* gs = reinterpret_cast<C*>(smem_raw + R::plane_bytes(R::CL));  // [n_s] own G-set slice
  cg::cluster_group cluster = cg::this_cluster();
  const int c = (int)cluster.block_rank();
  const long row = blockIdx.y;
  const int n_s = (n_chi + R::CL - 1) / R::CL;
  const int j0 = c * n_s, j1 = min(n_chi, j0 + n_s);
  const long pbase = (long)c * P * PL;                           // the CTA's planes within the row
  auto plane_pos = [](int e) {
    const int p = e / PL, rem = e - p * PL, i2 = rem / N3;
    return (p * N2 + i2) * S2 + (rem - i2 * N3);
  };
  auto planes_2d = [&](auto dir) {
    constexpr int D = decltype(dir)::value;
    pencil_pass<N3, D>(s, P * N2, 1, [](int q) { return q * S2; });
    __syncthreads();
    pencil_pass<N2, D>(s, P * N3, S2, [](int q) { return (q / N3) * (N2 * S2) + (q % N3); });
    __syncthreads();
  };
  if (MODE == 2) {
    // the G-set slice, then i1 transforms of the CTA's columns into every CTA's planes
    for (int j = j0 + threadIdx.x; j < j1; j += TH) gs[j - j0] = a[row * lda + j];
    cluster.sync();
    for (int q = c * COLS + threadIdx.x; q < (c + 1) * COLS; q += TH) {
      const int i2 = q / N3, i3 = q - i2 * N3;
      C x[N1];
      bool any = false;
#pragma unroll
      for (int i1 = 0; i1 < N1; ++i1) {
        const int j = __ldg(inv + i1 * PL + q);
        x[i1] = mk(T(0), T(0));
        if (j >= 0) {
          const int o = j / n_s;
          x[i1] = cluster.map_shared_rank(gs, o)[j - o * n_s];
          any = true;
        }
      }
      // columns outside the G set's projection are zero and stay zero
      if (__any_sync(__activemask(), any)) RegFFT<N1, -1>::run(x);
#pragma unroll
      for (int i1 = 0; i1 < N1; ++i1) cluster.map_shared_rank(s, i1 / P)[((i1 % P) * N2 + i2) * S2 + i3] = x[i1];
    }
    cluster.sync();                                              // no remote access after this point
    planes_2d(std::integral_constant<int, -1>{});
    C* dst = out + row * ldo + pbase;
    if (VEC) {
      for (int q = threadIdx.x; q < P * PL / 2; q += TH) {
        const int ps = plane_pos(2 * q);
        st_pair(dst + 2 * q, cscale(s[ps], scale), cscale(s[ps + 1], scale));
      }
    } else {
      for (int e = threadIdx.x; e < P * PL; e += TH) dst[e] = cscale(s[plane_pos(e)], scale);
    }
    return;
  }
  // forward: the CTA's planes (with the product of Eq. chi_rr for MODE 0) ...
  const C* pa = a + row * lda + pbase;
  const C* pb = b + row * lda + pbase;
  if (VEC) {
    constexpr int NP = P * PL / 2;
    // the row's ~93 KB per CTA arrive in few round trips: LB 16-byte loads in flight per thread
    // (the FFT's registers are free here)
    constexpr int LB = MODE == 0 ? 6 : 12;
    for (int q0 = threadIdx.x; q0 < NP; q0 += LB * TH) {
      C v[LB][2], w[LB][2];
#pragma unroll
      for (int u = 0; u < LB; ++u) {
        const int q = q0 + u * TH;
        if (q < NP) {
          ld_pair(pa + 2 * q, v[u][0], v[u][1]);
          if (MODE == 0) ld_pair(pb + 2 * q, w[u][0], w[u][1]);
        }
      }
#pragma unroll
      for (int u = 0; u < LB; ++u) {
        const int q = q0 + u * TH;
        if (q >= NP) continue;
        const int ps = plane_pos(2 * q);
        s[ps] = MODE == 0 ? cscale(cmulc(v[u][0], w[u][0]), scale) : v[u][0];
        s[ps + 1] = MODE == 0 ? cscale(cmulc(v[u][1], w[u][1]), scale) : v[u][1];
      }
    }
  } else {
    for (int e = threadIdx.x; e < P * PL; e += TH) {
      C v = pa[e];
      if (MODE == 0) v = cscale(cmulc(v, pb[e]), scale);
      s[plane_pos(e)] = v;
    }
  }
  __syncthreads();
  planes_2d(std::integral_constant<int, +1>{});
  cluster.sync();
  // ... i1 transforms of the CTA's columns, each result scattered to the G-set slice that holds it
  for (int q = c * COLS + threadIdx.x; q < (c + 1) * COLS; q += TH) {
    const int i2 = q / N3, i3 = q - i2 * N3;
    // a column with no G-set point has nothing to deliver: skip it where the whole warp may
    bool any = false;
#pragma unroll
    for (int i1 = 0; i1 < N1; ++i1) any |= __ldg(inv + i1 * PL + q) >= 0;
    if (!__any_sync(__activemask(), any)) continue;
    C x[N1];
#pragma unroll
    for (int i1 = 0; i1 < N1; ++i1) x[i1] = cluster.map_shared_rank(s, i1 / P)[((i1 % P) * N2 + i2) * S2 + i3];
    RegFFT<N1, +1>::run(x);
#pragma unroll
    for (int i1 = 0; i1 < N1; ++i1) {
      const int j = __ldg(inv + i1 * PL + q);
      if (j >= 0) {
        const int o = j / n_s;
        cluster.map_shared_rank(gs, o)[j - o * n_s] = x[i1];
      }
    }
  }
  cluster.sync();                                                // no remote access after this point
  for (int j = j0 + threadIdx.x; j < j1; j += TH) out[row * ldo + j] = gs[j - j0];
}

// chi rows from the plane-wave form of G (the paper evaluates G in a plane-wave
// representation and transforms it to real space when needed, Sec. II.B; at one
// k point Eqs. FFT_G1, FFT_G2 are two ordinary transforms).  For each row r the
// rows a = T_unocc(r, .) and b = T_occ(r, .) over the orbitals' plane-wave set
// (the column-transformed plane-wave G, length n_pw) are expanded over the grid
// R' (backward transform), multiplied as
//   x(R') = scale a(R') conj(b(R'))            (Eq. chi_rr)
// and transformed forward onto the n_chi-long G set of chi (Eq. FFTX1).  Each
// element of a row crosses HBM once: n_pw + n_pw values in, n_chi out.  The CL
// CTAs of a cluster share a row as in row_cluster_kernel (CL = 1: one CTA), with
// two plane buffers; the slices of the input rows and of the output row share
// one region (the inputs are read before the first cluster barrier, the output
// written after the third).
template <typename T, int N1, int N2, int N3>
struct PwRow {
  using C = typename cpx<T>::t;
  static constexpr int S2 = N3 % 2 == 0 ? N3 + 1 : N3;
  static constexpr int PL = N2 * N3;
  static constexpr size_t plane_bytes(int cl) { return (size_t)(N1 / cl) * N2 * S2 * sizeof(C); }
  static constexpr int pick() {
    for (int cl : {1, 2, 3, 4, 6, 8})
      if (N1 % cl == 0 && PL % cl == 0 && 2 * plane_bytes(cl) <= 192 * 1024) return cl;
    return 0;
  }
  static constexpr int CL = pick();
  static constexpr int P = CL ? N1 / CL : 1;
  static constexpr int COLS = CL ? PL / CL : 1;
  static constexpr int WORK = P * N2 > COLS ? (P * N2 > P * N3 ? P * N2 : P * N3) : (COLS > P * N3 ? COLS : P * N3);
  static constexpr int THREADS = CL ? ((WORK + 31) / 32 * 32 > 1024 ? 1024 : (WORK + 31) / 32 * 32) : 32;
  static size_t slice_elems(int n_pw, int n_chi) {
    const size_t in = 2 * (size_t)((n_pw + CL - 1) / CL), out = (size_t)((n_chi + CL - 1) / CL);
    return in > out ? in : out;
  }
  static size_t smem(int n_pw, int n_chi) { return 2 * plane_bytes(CL) + slice_elems(n_pw, n_chi) * sizeof(C); }
  // row_pw_sigma_kernel: [T_occ | T_unocc | W~] slices in, hu and ho out over the last two
  static size_t sig_smem(int n_pw, int n_chi) {
    const size_t ps = (size_t)((n_pw + CL - 1) / CL), ws = (size_t)((n_chi + CL - 1) / CL);
    const size_t e = 2 * ps + ws > 3 * ps ? 2 * ps + ws : 3 * ps;
    return 2 * plane_bytes(CL) + e * sizeof(C);
  }
};

template <typename T, int N1, int N2, int N3>
__global__ void __launch_bounds__(PwRow<T, N1, N2, N3>::THREADS)
    row_pw_chi_kernel(const typename cpx<T>::t* __restrict__ a, const typename cpx<T>::t* __restrict__ b, long lda,
                      typename cpx<T>::t* __restrict__ out, long ldo, const int* __restrict__ inv_pw, int n_pw,
                      const int* __restrict__ inv_chi, int n_chi, T scale) {
  namespace cg = cooperative_groups;
  using C = typename cpx<T>::t;
  using R = PwRow<T, N1, N2, N3>;
  constexpr int P = R::P, PL = R::PL, S2 = R::S2, COLS = R::COLS, CL = R::CL;
  constexpr int TH = R::THREADS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sa = reinterpret_cast<C*>(smem_raw);                              // [P][N2][S2] a, then x
  C* sb = reinterpret_cast<C*>(smem_raw + R::plane_bytes(CL));         // [P][N2][S2] b
  C* sl = reinterpret_cast<C*>(smem_raw + 2 * R::plane_bytes(CL));     // slices
  cg::cluster_group cluster = cg::this_cluster();
  const int c = (int)cluster.block_rank();
  const long row = blockIdx.y;
  const int n_ps = (n_pw + CL - 1) / CL, n_cs = (n_chi + CL - 1) / CL;
  C* su = sl;                 // [n_ps] this CTA's part of a's row
  C* so = sl + n_ps;          // [n_ps] of b's row
  {
    const int j0 = c * n_ps, j1 = min(n_pw, j0 + n_ps);
    for (int j = j0 + threadIdx.x; j < j1; j += TH) {
      su[j - j0] = a[row * lda + j];
      so[j - j0] = b[row * lda + j];
    }
  }
  cluster.sync();
  // backward i1 transforms of the CTA's columns, for both rows, into every CTA's planes
  for (int q = c * COLS + threadIdx.x; q < (c + 1) * COLS; q += TH) {
    const int i2 = q / N3, i3 = q - i2 * N3;
#pragma unroll 1
    for (int which = 0; which < 2; ++which) {
      C* src = which ? so : su;
      C* dst = which ? sb : sa;
      C x[N1];
      bool any = false;
#pragma unroll
      for (int i1 = 0; i1 < N1; ++i1) {
        const int j = __ldg(inv_pw + i1 * PL + q);
        x[i1] = mk(T(0), T(0));
        if (j >= 0) {
          const int o = j / n_ps;
          x[i1] = cluster.map_shared_rank(src, o)[j - o * n_ps];
          any = true;
        }
      }
      if (__any_sync(__activemask(), any)) RegFFT<N1, -1>::run(x);   // empty columns stay zero
#pragma unroll
      for (int i1 = 0; i1 < N1; ++i1)
        cluster.map_shared_rank(dst, i1 / P)[((i1 % P) * N2 + i2) * S2 + i3] = x[i1];
    }
  }
  cluster.sync();                  // the planes are complete and the input slices free
  // (i2, i3) backward transforms of the CTA's planes, both rows
  pencil_pass<N3, -1>(sa, P * N2, 1, [](int q) { return q * S2; });
  pencil_pass<N3, -1>(sb, P * N2, 1, [](int q) { return q * S2; });
  __syncthreads();
  pencil_pass<N2, -1>(sa, P * N3, S2, [](int q) { return (q / N3) * (N2 * S2) + (q % N3); });
  pencil_pass<N2, -1>(sb, P * N3, S2, [](int q) { return (q / N3) * (N2 * S2) + (q % N3); });
  __syncthreads();
  // the product of Eq. chi_rr, then the forward (i2, i3) transforms
  for (int e = threadIdx.x; e < P * PL; e += TH) {
    const int p = e / PL, rem = e - p * PL, i2 = rem / N3;
    const int ps = (p * N2 + i2) * S2 + (rem - i2 * N3);
    sa[ps] = cscale(cmulc(sa[ps], sb[ps]), scale);
  }
  __syncthreads();
  pencil_pass<N2, +1>(sa, P * N3, S2, [](int q) { return (q / N3) * (N2 * S2) + (q % N3); });
  __syncthreads();
  pencil_pass<N3, +1>(sa, P * N2, 1, [](int q) { return q * S2; });
  cluster.sync();                  // every CTA's x planes are final
  // forward i1 transforms of the CTA's columns, each result into the slice of chi that holds it
  C* sx = sl;                      // [n_cs] this CTA's part of the chi row
  for (int q = c * COLS + threadIdx.x; q < (c + 1) * COLS; q += TH) {
    const int i2 = q / N3, i3 = q - i2 * N3;
    bool any = false;                // columns with no point of chi's G set deliver nothing
#pragma unroll
    for (int i1 = 0; i1 < N1; ++i1) any |= __ldg(inv_chi + i1 * PL + q) >= 0;
    if (!__any_sync(__activemask(), any)) continue;
    C x[N1];
#pragma unroll
    for (int i1 = 0; i1 < N1; ++i1) x[i1] = cluster.map_shared_rank(sa, i1 / P)[((i1 % P) * N2 + i2) * S2 + i3];
    RegFFT<N1, +1>::run(x);
#pragma unroll
    for (int i1 = 0; i1 < N1; ++i1) {
      const int j = __ldg(inv_chi + i1 * PL + q);
      if (j >= 0) {
        const int o = j / n_cs;
        cluster.map_shared_rank(sx, o)[j - o * n_cs] = x[i1];
      }
    }
  }
  cluster.sync();                  // no remote access after this point
  {
    const int j0 = c * n_cs, j1 = min(n_chi, j0 + n_cs);
    for (int j = j0 + threadIdx.x; j < j1; j += TH) out[row * ldo + j] = sx[j - j0];
  }
}

// The self-energy's rows in the same plane-wave form (first term of Eq.
// Sigma_occ_reduce with Eq. Sigma_rr): for each row r, the W~ row over chi's G
// set (wg, column-transformed, Eq. FFTW) and the rows T_unocc(r, .), T_occ(r, .)
// of the column-transformed plane-wave G are expanded over the grid R'; then
//   H(r,R') = W~(r,R') G(r,R') = W~ conj(G')            (G' the expanded T row)
// is transformed forward and gathered on the orbitals' plane waves,
//   hu / ho(r, g) = sum_R' H(r,R') e^{+i g.R'},
// so that sum_R' H(r,R') psi_n(R') = sum_g hu(r,g) c_n(g) needs only the
// plane-wave coefficients c_n of the Sigma bands.  Five transforms per row, W~
// kept expanded in the first plane buffer while the second takes G_unocc, then
// G_occ.  inv_neg: grid position -> index into the T rows (the negated set),
// inv_nat: grid position -> plane-wave index of the outputs, inv_chi: the G set.
template <typename T, int N1, int N2, int N3>
__global__ void __launch_bounds__(PwRow<T, N1, N2, N3>::THREADS)
    row_pw_sigma_kernel(const typename cpx<T>::t* __restrict__ tu, const typename cpx<T>::t* __restrict__ to,
                        long ldt, const typename cpx<T>::t* __restrict__ wg, long ldw,
                        typename cpx<T>::t* __restrict__ hu, typename cpx<T>::t* __restrict__ ho, long ldh,
                        const int* __restrict__ inv_neg, const int* __restrict__ inv_nat, int n_pw,
                        const int* __restrict__ inv_chi, int n_chi) {
  namespace cg = cooperative_groups;
  using C = typename cpx<T>::t;
  using R = PwRow<T, N1, N2, N3>;
  constexpr int P = R::P, PL = R::PL, S2 = R::S2, COLS = R::COLS, CL = R::CL;
  constexpr int TH = R::THREADS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sa = reinterpret_cast<C*>(smem_raw);                              // W~ planes
  C* sb = reinterpret_cast<C*>(smem_raw + R::plane_bytes(CL));         // G', then H planes
  C* sl = reinterpret_cast<C*>(smem_raw + 2 * R::plane_bytes(CL));
  cg::cluster_group cluster = cg::this_cluster();
  const int c = (int)cluster.block_rank();
  const long row = blockIdx.y;
  const int n_ps = (n_pw + CL - 1) / CL, n_ws = (n_chi + CL - 1) / CL;
  // slices: [T_occ | T_unocc | W~]; outputs hu over T_unocc's, ho from 2 n_ps (both read by then)
  C* so_in = sl;
  C* su_in = sl + n_ps;
  C* sw = sl + 2 * n_ps;
  C* hu_s = sl + n_ps;
  C* ho_s = sl + 2 * n_ps;
  {
    const int j0 = c * n_ps, j1 = min(n_pw, j0 + n_ps);
    for (int j = j0 + threadIdx.x; j < j1; j += TH) {
      su_in[j - j0] = tu[row * ldt + j];
      so_in[j - j0] = to[row * ldt + j];
    }
    const int w0 = c * n_ws, w1 = min(n_chi, w0 + n_ws);
    for (int j = w0 + threadIdx.x; j < w1; j += TH) sw[j - w0] = wg[row * ldw + j];
  }
  cluster.sync();
  // backward i1 transforms of a slice-held row into every CTA's planes
  auto line_bwd = [&](const C* src, int ns, const int* inv, C* dst) {
    for (int q = c * COLS + threadIdx.x; q < (c + 1) * COLS; q += TH) {
      const int i2 = q / N3, i3 = q - i2 * N3;
      C x[N1];
      bool any = false;
#pragma unroll
      for (int i1 = 0; i1 < N1; ++i1) {
        const int j = __ldg(inv + i1 * PL + q);
        x[i1] = mk(T(0), T(0));
        if (j >= 0) {
          const int o = j / ns;
          x[i1] = cluster.map_shared_rank(src, o)[j - o * ns];
          any = true;
        }
      }
      if (__any_sync(__activemask(), any)) RegFFT<N1, -1>::run(x);   // empty columns stay zero
#pragma unroll
      for (int i1 = 0; i1 < N1; ++i1)
        cluster.map_shared_rank(dst, i1 / P)[((i1 % P) * N2 + i2) * S2 + i3] = x[i1];
    }
  };
  // forward i1 transforms of every CTA's H planes, gathered on the plane-wave set
  auto line_fwd = [&](C* out) {
    for (int q = c * COLS + threadIdx.x; q < (c + 1) * COLS; q += TH) {
      const int i2 = q / N3, i3 = q - i2 * N3;
      bool any = false;              // columns with no plane wave of the set deliver nothing
#pragma unroll
      for (int i1 = 0; i1 < N1; ++i1) any |= __ldg(inv_nat + i1 * PL + q) >= 0;
      if (!__any_sync(__activemask(), any)) continue;
      C x[N1];
#pragma unroll
      for (int i1 = 0; i1 < N1; ++i1) x[i1] = cluster.map_shared_rank(sb, i1 / P)[((i1 % P) * N2 + i2) * S2 + i3];
      RegFFT<N1, +1>::run(x);
#pragma unroll
      for (int i1 = 0; i1 < N1; ++i1) {
        const int j = __ldg(inv_nat + i1 * PL + q);
        if (j >= 0) {
          const int o = j / n_ps;
          cluster.map_shared_rank(out, o)[j - o * n_ps] = x[i1];
        }
      }
    }
  };
  auto planes_bwd = [&](C* buf) {
    pencil_pass<N3, -1>(buf, P * N2, 1, [](int q) { return q * S2; });
    __syncthreads();
    pencil_pass<N2, -1>(buf, P * N3, S2, [](int q) { return (q / N3) * (N2 * S2) + (q % N3); });
    __syncthreads();
  };
  // H = W~ conj(G') on the CTA's planes, then the forward (i2, i3) transforms
  auto product_fwd = [&]() {
    for (int e = threadIdx.x; e < P * PL; e += TH) {
      const int p = e / PL, rem = e - p * PL, i2 = rem / N3;
      const int ps = (p * N2 + i2) * S2 + (rem - i2 * N3);
      sb[ps] = cmulc(sa[ps], sb[ps]);
    }
    __syncthreads();
    pencil_pass<N2, +1>(sb, P * N3, S2, [](int q) { return (q / N3) * (N2 * S2) + (q % N3); });
    __syncthreads();
    pencil_pass<N3, +1>(sb, P * N2, 1, [](int q) { return q * S2; });
  };
  line_bwd(sw, n_ws, inv_chi, sa);
  line_bwd(su_in, n_ps, inv_neg, sb);
  cluster.sync();                  // W~ and G'_unocc planes complete; W~ and T_unocc slices free
  planes_bwd(sa);
  planes_bwd(sb);
  product_fwd();
  cluster.sync();                  // H_unocc planes final
  line_fwd(hu_s);
  cluster.sync();                  // hu complete; the second buffer free
  line_bwd(so_in, n_ps, inv_neg, sb);
  cluster.sync();
  planes_bwd(sb);
  product_fwd();
  cluster.sync();
  line_fwd(ho_s);
  cluster.sync();                  // no remote access after this point
  {
    const int j0 = c * n_ps, j1 = min(n_pw, j0 + n_ps);
    for (int j = j0 + threadIdx.x; j < j1; j += TH) {
      hu[row * ldh + j] = hu_s[j - j0];
      ho[row * ldh + j] = ho_s[j - j0];
    }
  }
}

constexpr int kPlaneW = 16;

// In-place 2-D FFT over (i2, i3) of the rows of plane i1 = blockIdx.y, for 16
// contiguous columns per CTA.  PAIRS (FP32 only): rows move as 16-byte pairs
// of columns; the host takes it when ld and ncols are even (every pair then
// starts on a 16-byte boundary and lies wholly inside or outside the matrix).
template <typename T, int N2, int N3, int DIR, bool PAIRS>
__global__ void __launch_bounds__(256) col_plane_kernel(typename cpx<T>::t* __restrict__ buf, long ld, int ncols,
                                                        T scale) {
  using C = typename cpx<T>::t;
  constexpr int W = kPlaneW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const long i1 = blockIdx.y;
  const int c0 = blockIdx.x * W;
  C* base = buf + i1 * (N2 * N3) * ld + c0;
  if constexpr (PAIRS) {
    for (int e = threadIdx.x; e < N2 * N3 * W / 2; e += blockDim.x) {
      const int rr = e / (W / 2), w = 2 * (e - rr * (W / 2));
      C a = mk(T(0), T(0)), b = a;
      if (c0 + w < ncols) ld_pair(base + rr * ld + w, a, b);
      s[rr * W + w] = a;
      s[rr * W + w + 1] = b;
    }
  } else {
    for (int e = threadIdx.x; e < N2 * N3 * W; e += blockDim.x) {
      const int rr = e / W, w = e - rr * W;
      s[e] = (c0 + w < ncols) ? base[rr * ld + w] : mk(T(0), T(0));
    }
  }
  __syncthreads();
  pencil_pass<N3, DIR>(s, N2 * W, W, [](int p) { return (p / W) * (N3 * W) + (p % W); });
  __syncthreads();
  pencil_pass<N2, DIR>(s, N3 * W, N3 * W, [](int p) { return (p / W) * W + (p % W); });
  __syncthreads();
  if constexpr (PAIRS) {
    for (int e = threadIdx.x; e < N2 * N3 * W / 2; e += blockDim.x) {
      const int rr = e / (W / 2), w = 2 * (e - rr * (W / 2));
      if (c0 + w < ncols) st_pair(base + rr * ld + w, cscale(s[rr * W + w], scale), cscale(s[rr * W + w + 1], scale));
    }
  } else {
    for (int e = threadIdx.x; e < N2 * N3 * W; e += blockDim.x) {
      const int rr = e / W, w = e - rr * W;
      if (c0 + w < ncols) base[rr * ld + w] = cscale(s[e], scale);
    }
  }
}

// In-place 1-D FFT over i1 for the column c and the (i2,i3) pair blockIdx.y.
// GATHER_IN: read row inv[pos] of `in` (zero if -1) instead of buf[pos].
// SCATTER_OUT: write row inv[pos] of `out` (skip if -1) instead of buf[pos].
template <typename T, int N1, int DIR, bool GATHER_IN, bool SCATTER_OUT>
__global__ void __launch_bounds__(256) col_line_kernel(const typename cpx<T>::t* __restrict__ in, long ldi,
                                                       typename cpx<T>::t* __restrict__ out, long ldo, int ncols,
                                                       int plane, const int* __restrict__ inv, T scale) {
  using C = typename cpx<T>::t;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int i23 = blockIdx.y;
  if (c >= ncols) return;
  C x[N1];
#pragma unroll
  for (int i1 = 0; i1 < N1; ++i1) {
    const long pos = (long)i1 * plane + i23;
    if (GATHER_IN) {
      const int j = inv[pos];
      x[i1] = j >= 0 ? in[(long)j * ldi + c] : mk(T(0), T(0));
    } else {
      x[i1] = in[pos * ldi + c];
    }
  }
  RegFFT<N1, DIR>::run(x);
#pragma unroll
  for (int i1 = 0; i1 < N1; ++i1) {
    const long pos = (long)i1 * plane + i23;
    if (SCATTER_OUT) {
      const int j = inv[pos];
      if (j >= 0) out[(long)j * ldo + c] = cscale(x[i1], scale);
    } else {
      out[pos * ldo + c] = cscale(x[i1], scale);
    }
  }
}

// Weighted sums of the transforms in FP32.  The weights of the time/frequency
// transforms reach |c_kj| ~ 10^2 with both signs; rounded to FP32 they alone
// would perturb sum_j c_kj x_j by ~4e-7 relative.  The FP32 path keeps each
// weight as an unevaluated pair hi + lo (hi = fl32(c), lo = fl32(c - hi)) and
// accumulates c x as fma(hi, x, fma(lo, x, s)), which removes the weight
// rounding for one extra FMA per term; the remaining FP32 accumulation error
// is below the rounding already present in the x_j themselves.  FP64 keeps the
// plain sum.
template <typename T>
struct WSum {
  T s = 0;
  __device__ void add(T wh, T, T x) { s += wh * x; }
  __device__ T value() const { return s; }
};
template <>
struct WSum<float> {
  float s = 0.f;
  __device__ void add(float wh, float wl, float x) { s = __fmaf_rn(wh, x, __fmaf_rn(wl, x, s)); }
  __device__ float value() const { return s; }
};
// The weight arrays hold hi[n_k][n_j] and, for FP32, lo[n_k][n_j] right after.
template <typename T>
constexpr int kWParts = sizeof(T) == 4 ? 2 : 1;

// Last column pass of the chi chain: i1 FFT (-i) of every tau slab, then
// out[k][inv[pos]][c] = sum_j cw[k][j] * slab_j(pos, c)  (Eq. CTX with the
// dV^2/Omega of Eq. FFTX2 folded into cw).  32 columns x 8 warps per CTA.
template <typename T, int N1>
__global__ void __launch_bounds__(256) col_line_ct_kernel(const typename cpx<T>::t* __restrict__ slabs,
                                                          long slab_stride, long ld, int ntau,
                                                          const T* __restrict__ cw, int nw,
                                                          typename cpx<T>::t* __restrict__ out, long out_slice,
                                                          long ldo, const int* __restrict__ inv, int plane,
                                                          int ncols) {
  using C = typename cpx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);                       // [ntau][N1][32]
  T* w = reinterpret_cast<T*>(s + (size_t)ntau * N1 * 32);      // [parts][nw][ntau]
  const T* wl = w + (kWParts<T> - 1) * nw * ntau;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + lane;
  const int i23 = blockIdx.y;
  for (int e = threadIdx.x; e < kWParts<T> * nw * ntau; e += blockDim.x) w[e] = cw[e];
  for (int j = warp; j < ntau; j += 8) {
    C x[N1];
    const C* src = slabs + (long)j * slab_stride;
#pragma unroll
    for (int i1 = 0; i1 < N1; ++i1)
      x[i1] = c < ncols ? src[((long)i1 * plane + i23) * ld + c] : mk(T(0), T(0));
    RegFFT<N1, -1>::run(x);
#pragma unroll
    for (int i1 = 0; i1 < N1; ++i1) s[(j * N1 + i1) * 32 + lane] = x[i1];
  }
  __syncthreads();
  if (c >= ncols) return;
  for (int q = warp; q < nw * N1; q += 8) {
    const int k = q / N1, i1 = q - k * N1;
    const int row = inv[(long)i1 * plane + i23];
    if (row < 0) continue;
    WSum<T> re, im;
    for (int j = 0; j < ntau; ++j) {
      const C v = s[(j * N1 + i1) * 32 + lane];
      const T wh = w[k * ntau + j], wlo = wl[k * ntau + j];
      re.add(wh, wlo, v.x);
      im.add(wh, wlo, v.y);
    }
    out[(long)k * out_slice + (long)row * ldo + c] = mk(re.value(), im.value());
  }
}

// Same pass with a compile-time count of tau points (FP32): each lane keeps the
// NT values of its column and one i1 in registers and the weights come from a
// kernel-parameter block (constant bank), so the transform costs one
// shared-memory read per input instead of three per multiply-add.
template <int NT>
struct CtWeights {
  float hi[NT * NT];
  float lo[NT * NT];
};

template <int N1, int NT>
__global__ void __launch_bounds__(256, (NT * N1 * 32 * 8 <= 110 * 1024) ? 2 : 1) col_line_ct_reg_kernel(const float2* __restrict__ slabs, long slab_stride,
                                                              long ld, const __grid_constant__ CtWeights<NT> cw,
                                                              float2* __restrict__ out, long out_slice, long ldo,
                                                              const int* __restrict__ inv, int plane, int ncols) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* s = reinterpret_cast<float2*>(smem_raw);             // [NT][N1][32]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + lane;
  const int i23 = blockIdx.y;
  for (int j = warp; j < NT; j += 8) {
    float2 x[N1];
    const float2* src = slabs + (long)j * slab_stride;
#pragma unroll
    for (int i1 = 0; i1 < N1; ++i1)
      x[i1] = c < ncols ? src[((long)i1 * plane + i23) * ld + c] : make_float2(0.f, 0.f);
    RegFFT<N1, -1>::run(x);
#pragma unroll
    for (int i1 = 0; i1 < N1; ++i1) s[(j * N1 + i1) * 32 + lane] = x[i1];
  }
  __syncthreads();
  if (c >= ncols) return;
  for (int i1 = warp; i1 < N1; i1 += 8) {
    const int row = inv[(long)i1 * plane + i23];
    if (row < 0) continue;
    float2 x[NT];
#pragma unroll
    for (int j = 0; j < NT; ++j) x[j] = s[(j * N1 + i1) * 32 + lane];
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      WSum<float> re, im;
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        re.add(cw.hi[k * NT + j], cw.lo[k * NT + j], x[j].x);
        im.add(cw.hi[k * NT + j], cw.lo[k * NT + j], x[j].y);
      }
      out[(long)k * out_slice + (long)row * ldo + c] = make_float2(re.value(), im.value());
    }
  }
}

// Same map with a compile-time size (FP32, weights in a kernel-parameter
// block, constant bank): each thread keeps one element of all n slices in
// registers.  Capped at 80 registers for three CTAs (24 warps) per SM, which
// keeps enough loads in flight to approach the HBM rate.
template <int NT, bool ST>
__global__ void __launch_bounds__(256, 3) ct_reg1_kernel(const float2* __restrict__ in, float2* __restrict__ out,
                                                      size_t elems, const __grid_constant__ CtWeights<NT> w) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < elems; e += (size_t)gridDim.x * blockDim.x) {
    float2 x[NT];
#pragma unroll
    for (int j = 0; j < NT; ++j) x[j] = __ldg(in + (size_t)j * elems + e);
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      WSum<float> re, im;
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        re.add(w.hi[k * NT + j], w.lo[k * NT + j], x[j].x);
        im.add(w.hi[k * NT + j], w.lo[k * NT + j], x[j].y);
      }
      out[(size_t)k * elems + e] = ST ? make_float2(-im.value(), re.value()) : make_float2(re.value(), im.value());
    }
  }
}

// out[k][e] = (i if ST) sum_j M[k][j] in[j][e]
template <typename T, bool ST>
__global__ void __launch_bounds__(256) ct_kernel(const typename cpx<T>::t* __restrict__ in,
                                                 typename cpx<T>::t* __restrict__ out, size_t elems, int n,
                                                 const T* __restrict__ M) {
  using C = typename cpx<T>::t;
  __shared__ T w[kWParts<T> * 32 * 32];
  const T* wl = w + (kWParts<T> - 1) * n * n;
  for (int e = threadIdx.x; e < kWParts<T> * n * n; e += blockDim.x) w[e] = M[e];
  __syncthreads();
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < elems; e += (size_t)gridDim.x * blockDim.x) {
    C x[32];
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (j < n) x[j] = in[(size_t)j * elems + e];
    for (int k = 0; k < n; ++k) {
      WSum<T> re, im;
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j < n) {
          re.add(w[k * n + j], wl[k * n + j], x[j].x);
          im.add(w[k * n + j], wl[k * n + j], x[j].y);
        }
      out[(size_t)k * elems + e] = ST ? mk(-im.value(), re.value()) : mk(re.value(), im.value());
    }
  }
}

template <typename T>
__global__ void hadamard_kernel(const typename cpx<T>::t* __restrict__ a, const typename cpx<T>::t* __restrict__ b,
                                typename cpx<T>::t* out, size_t count, T scale) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
    out[e] = cscale(cmulc(a[e], b[e]), scale);
}

// ---------------------------------------------------------------------- launchers

template <typename K>
static gw_status set_smem(gw_ctx* ctx, K kernel, size_t bytes) {
  if (bytes > 227 * 1024) return fail(ctx, GW_ERR_UNSUPPORTED, "shared-memory tile too large for this grid/precision");
  if (bytes > 48 * 1024)
    return cuda_check(ctx, cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes),
                      "cudaFuncSetAttribute");
  return GW_OK;
}

template <typename T, int N1, int N2, int N3>
struct GridOps {
  using C = typename cpx<T>::t;
  static gw_status row_two_pass(gw_ctx* ctx, int mode, const void* a, const void* b, long lda, void* out, long ldo,
                                const int* inv, void* tmp, int n_chi, int n_rows, double scale, cudaStream_t st) {
    constexpr int NR = N1 * N2 * N3;
    constexpr int S2 = N3 % 2 == 0 ? N3 + 1 : N3;
    const size_t pbytes = (size_t)kRowPlanes * N2 * S2 * sizeof(C);
    const size_t lbytes = (size_t)n_chi * sizeof(C);
    if (!inv || (mode != 2 && !tmp))
      return fail(ctx, GW_ERR_UNSUPPORTED, "this grid's rows need the two-pass transform (index map and workspace)");
    if (lbytes > 200 * 1024) return fail(ctx, GW_ERR_UNSUPPORTED, "G set too large for the two-pass row transform");
    const dim3 pgrid((N1 + kRowPlanes - 1) / kRowPlanes, n_rows);
    const double rd = mode == 0 ? 2.0 * NR : (mode == 1 ? NR : n_chi);
    const double wr = mode == 2 ? NR : n_chi;
    gw_status rc;
    auto plane = [&](auto kernel, const void* pa, const void* pb, long pld, void* po, long pldo) -> gw_status {
      gw_status r = set_smem(ctx, kernel, pbytes);
      if (r) return r;
      KTimer kt(ctx, KF_ROW_FFT, 0.0, st);
      kernel<<<pgrid, 256, pbytes, st>>>((const C*)pa, (const C*)pb, pld, (C*)po, pldo, (T)scale);
      return launch_check(ctx, "row_plane_kernel");
    };
    if (mode == 2) {
      auto kl = row_line_bwd_kernel<T, N1, N2, N3>;
      if ((rc = set_smem(ctx, kl, lbytes))) return rc;
      {
        KTimer kt(ctx, KF_ROW_FFT, (double)n_rows * (rd + wr) * sizeof(C), st);
        kl<<<n_rows, 256, lbytes, st>>>((const C*)a, lda, (C*)out, ldo, inv, n_chi);
        if ((rc = launch_check(ctx, "row_line_bwd_kernel"))) return rc;
      }
      return plane(row_plane_kernel<T, N1, N2, N3, 2, -1>, nullptr, nullptr, 0, out, ldo);
    }
    if (mode == 0) rc = plane(row_plane_kernel<T, N1, N2, N3, 0, +1>, a, b, lda, tmp, NR);
    else rc = plane(row_plane_kernel<T, N1, N2, N3, 1, +1>, a, nullptr, lda, tmp, NR);
    if (rc) return rc;
    auto kl = row_line_fwd_kernel<T, N1, N2, N3>;
    if ((rc = set_smem(ctx, kl, lbytes))) return rc;
    KTimer kt(ctx, KF_ROW_FFT, (double)n_rows * (rd + wr) * sizeof(C), st);
    kl<<<n_rows, 256, lbytes, st>>>((const C*)tmp, NR, (C*)out, ldo, inv, n_chi);
    return launch_check(ctx, "row_line_fwd_kernel");
  }
  static gw_status row(gw_ctx* ctx, int mode, const void* a, const void* b, long lda, void* out, long ldo,
                       const int* map, int n_chi, int n_rows, double scale, cudaStream_t st, const int* inv,
                       void* tmp) {
    const size_t bytes = RowLayout<N1, N2, N3>::TOT * sizeof(C);
    const double rd = mode == 0 ? 2.0 * RowLayout<N1, N2, N3>::NR : (mode == 1 ? RowLayout<N1, N2, N3>::NR : n_chi);
    const double wr = mode == 2 ? RowLayout<N1, N2, N3>::NR : n_chi;
    auto al = [](const void* p) { return p == nullptr || reinterpret_cast<uintptr_t>(p) % 16 == 0; };
    const bool vec = al(a) && al(b) && al(out) && lda % 2 == 0 && ldo % 2 == 0 && n_chi % 2 == 0 && N3 % 2 == 0;
    if (bytes > kRowSmemMax) {
      using CR = ClusterRow<T, N1, N2, N3>;
      if constexpr (CR::CL > 0 && RowLayout<N1, N2, N3>::TOT * sizeof(C) > kRowSmemMax) {
        if (inv && CR::smem(n_chi) <= kRowSmemMax) {
          const size_t cbytes = CR::smem(n_chi);
          auto go = [&](auto kernel) -> gw_status {
            gw_status s = set_smem(ctx, kernel, cbytes);
            if (s) return s;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(CR::CL, (unsigned)n_rows);
            cfg.blockDim = dim3(CR::THREADS);
            cfg.dynamicSmemBytes = cbytes;
            cfg.stream = st;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = CR::CL;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            KTimer kt(ctx, KF_ROW_FFT, (double)n_rows * (rd + wr) * sizeof(C), st);
            gw_status r = cuda_check(ctx, cudaLaunchKernelEx(&cfg, kernel, (const C*)a, (const C*)b, lda, (C*)out, ldo,
                                                             inv, n_chi, (T)scale),
                                     "cudaLaunchKernelEx(row_cluster_kernel)");
            if (r) return r;
            return launch_check(ctx, "row_cluster_kernel");
          };
#define GW_ROWC_GO(M)                                                                        \
          if (mode == M) return vec ? go(row_cluster_kernel<T, N1, N2, N3, M, N3 % 2 == 0>)  \
                                    : go(row_cluster_kernel<T, N1, N2, N3, M, false>);
          GW_ROWC_GO(0)
          GW_ROWC_GO(1)
          GW_ROWC_GO(2)
#undef GW_ROWC_GO
          return fail(ctx, GW_ERR_ARG, "bad row transform mode");
        }
      }
      return row_two_pass(ctx, mode, a, b, lda, out, ldo, inv, tmp, n_chi, n_rows, scale, st);
    }
    auto go = [&](auto kernel, int threads) -> gw_status {
      gw_status s = set_smem(ctx, kernel, bytes);
      if (s) return s;
      KTimer kt(ctx, KF_ROW_FFT, (double)n_rows * (rd + wr) * sizeof(C), st);
      kernel<<<n_rows, threads, bytes, st>>>((const C*)a, (const C*)b, lda, (C*)out, ldo, map, n_chi, (T)scale);
      return launch_check(ctx, "row_fft_kernel");
    };
    constexpr bool big = N1 * N2 * N3 >= 4096;
    constexpr int TH = big ? 512 : 256;
#define GW_ROW_GO(M)                                                              \
    if (mode == M) return vec ? go(row_fft_kernel<T, N1, N2, N3, M, TH, N3 % 2 == 0>, TH) \
                              : go(row_fft_kernel<T, N1, N2, N3, M, TH, false>, TH);
    GW_ROW_GO(0)
    GW_ROW_GO(1)
    GW_ROW_GO(2)
#undef GW_ROW_GO
    return fail(ctx, GW_ERR_ARG, "bad row transform mode");
  }
  static bool row_pw_ok(int n_pw, int n_chi) {
    using PR = PwRow<T, N1, N2, N3>;
    if constexpr (PR::CL > 0) return PR::smem(n_pw, n_chi) <= kRowSmemMax;
    return false;
  }
  static gw_status row_pw(gw_ctx* ctx, const void* a, const void* b, long lda, void* out, long ldo,
                           const int* inv_pw, int n_pw, const int* inv_chi, int n_chi, int n_rows, double scale,
                           cudaStream_t st) {
    using PR = PwRow<T, N1, N2, N3>;
    if constexpr (PR::CL > 0) {
      const size_t bytes = PR::smem(n_pw, n_chi);
      if (bytes > kRowSmemMax) return fail(ctx, GW_ERR_UNSUPPORTED, "plane-wave chi rows: G sets too large for this grid");
      auto kernel = row_pw_chi_kernel<T, N1, N2, N3>;
      gw_status s = set_smem(ctx, kernel, bytes);
      if (s) return s;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(PR::CL, (unsigned)n_rows);
      cfg.blockDim = dim3(PR::THREADS);
      cfg.dynamicSmemBytes = bytes;
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = PR::CL;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      // FP32/FP64 ALU work: three transforms of N_r points (5 N log2 N each) and the product per row
      const double nr = (double)N1 * N2 * N3;
      KTimer kt(ctx, KF_ROW_PW, (double)n_rows * (3.0 * 5.0 * nr * std::log2(nr) + 6.0 * nr), st);
      s = cuda_check(ctx, cudaLaunchKernelEx(&cfg, kernel, (const C*)a, (const C*)b, lda, (C*)out, ldo, inv_pw, n_pw,
                                             inv_chi, n_chi, (T)scale),
                     "cudaLaunchKernelEx(row_pw_chi_kernel)");
      if (s) return s;
      return launch_check(ctx, "row_pw_chi_kernel");
    } else {
      return fail(ctx, GW_ERR_UNSUPPORTED, "plane-wave chi rows: no cluster split fits this grid and precision");
    }
  }
  static bool row_pw_sigma_ok(int n_pw, int n_chi) {
    using PR = PwRow<T, N1, N2, N3>;
    if constexpr (PR::CL > 0) return PR::sig_smem(n_pw, n_chi) <= kRowSmemMax;
    return false;
  }
  static gw_status row_pw_sigma(gw_ctx* ctx, const void* tu, const void* to, long ldt, const void* wg, long ldw,
                                void* hu, void* ho, long ldh, const int* inv_neg, const int* inv_nat, int n_pw,
                                const int* inv_chi, int n_chi, int n_rows, cudaStream_t st) {
    using PR = PwRow<T, N1, N2, N3>;
    if constexpr (PR::CL > 0) {
      const size_t bytes = PR::sig_smem(n_pw, n_chi);
      if (bytes > kRowSmemMax) return fail(ctx, GW_ERR_UNSUPPORTED, "plane-wave Sigma rows: G sets too large");
      auto kernel = row_pw_sigma_kernel<T, N1, N2, N3>;
      gw_status s = set_smem(ctx, kernel, bytes);
      if (s) return s;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(PR::CL, (unsigned)n_rows);
      cfg.blockDim = dim3(PR::THREADS);
      cfg.dynamicSmemBytes = bytes;
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = PR::CL;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      // five transforms of N_r points and two products per row
      const double nr = (double)N1 * N2 * N3;
      KTimer kt(ctx, KF_ROW_PW, (double)n_rows * (5.0 * 5.0 * nr * std::log2(nr) + 12.0 * nr), st);
      s = cuda_check(ctx, cudaLaunchKernelEx(&cfg, kernel, (const C*)tu, (const C*)to, ldt, (const C*)wg, ldw, (C*)hu,
                                             (C*)ho, ldh, inv_neg, inv_nat, n_pw, inv_chi, n_chi),
                     "cudaLaunchKernelEx(row_pw_sigma_kernel)");
      if (s) return s;
      return launch_check(ctx, "row_pw_sigma_kernel");
    } else {
      return fail(ctx, GW_ERR_UNSUPPORTED, "plane-wave Sigma rows: no cluster split fits this grid and precision");
    }
  }
  static gw_status plane(gw_ctx* ctx, int dir, void* buf, long ld, int ncols, double scale, cudaStream_t st) {
    const size_t bytes = (size_t)N2 * N3 * kPlaneW * sizeof(C);
    dim3 grid((ncols + kPlaneW - 1) / kPlaneW, N1);
    auto go = [&](auto kernel) -> gw_status {
      gw_status s = set_smem(ctx, kernel, bytes);
      if (s) return s;
      KTimer kt(ctx, KF_COL_FFT, 2.0 * N1 * N2 * N3 * (double)ncols * sizeof(C), st);
      kernel<<<grid, 256, bytes, st>>>((C*)buf, ld, ncols, (T)scale);
      return launch_check(ctx, "col_plane_kernel");
    };
    const bool pairs = sizeof(T) == 4 && ld % 2 == 0 && ncols % 2 == 0 && reinterpret_cast<uintptr_t>(buf) % 16 == 0;
    if (pairs) return dir > 0 ? go(col_plane_kernel<T, N2, N3, +1, true>) : go(col_plane_kernel<T, N2, N3, -1, true>);
    return dir > 0 ? go(col_plane_kernel<T, N2, N3, +1, false>) : go(col_plane_kernel<T, N2, N3, -1, false>);
  }
  static gw_status line(gw_ctx* ctx, int dir, int variant, const void* in, long ldi, void* out, long ldo, int ncols,
                        const int* inv, double scale, cudaStream_t st) {
    dim3 grid((ncols + 127) / 128, N2 * N3);
    auto go = [&](auto kernel) -> gw_status {
      KTimer kt(ctx, KF_COL_FFT, 2.0 * N1 * N2 * N3 * (double)ncols * sizeof(C), st);
      kernel<<<grid, 128, 0, st>>>((const C*)in, ldi, (C*)out, ldo, ncols, N2 * N3, inv, (T)scale);
      return launch_check(ctx, "col_line_kernel");
    };
    // variant 0: in place / plain; 1: gather rows of `in` through inv; 2: scatter rows of `out` through inv
    if (variant == 0) return dir > 0 ? go(col_line_kernel<T, N1, +1, false, false>)
                                     : go(col_line_kernel<T, N1, -1, false, false>);
    if (variant == 1) return dir > 0 ? go(col_line_kernel<T, N1, +1, true, false>)
                                     : go(col_line_kernel<T, N1, -1, true, false>);
    return dir > 0 ? go(col_line_kernel<T, N1, +1, false, true>) : go(col_line_kernel<T, N1, -1, false, true>);
  }
  template <int NT>
  static gw_status line_ct_reg(gw_ctx* ctx, const void* slabs, long slab_stride, long ld, const float* cw_h, void* out,
                               long out_slice, long ldo, const int* inv, int ncols, cudaStream_t st) {
    CtWeights<NT> w;
    for (int e = 0; e < NT * NT; ++e) {
      w.hi[e] = cw_h[e];
      w.lo[e] = cw_h[NT * NT + e];
    }
    const size_t bytes = (size_t)NT * N1 * 32 * sizeof(float2);
    auto kernel = col_line_ct_reg_kernel<N1, NT>;
    gw_status s = set_smem(ctx, kernel, bytes);
    if (s) return s;
    dim3 grid((ncols + 31) / 32, N2 * N3);
    KTimer kt(ctx, KF_COL_LINE_CT, ((double)NT * N1 * N2 * N3 + (double)NT * ncols) * ncols * sizeof(float2), st);
    kernel<<<grid, 256, bytes, st>>>((const float2*)slabs, slab_stride, ld, w, (float2*)out, out_slice, ldo, inv,
                                     N2 * N3, ncols);
    return launch_check(ctx, "col_line_ct_reg_kernel");
  }
  static gw_status line_ct(gw_ctx* ctx, const void* slabs, long slab_stride, long ld, int ntau, const void* cw, int nw,
                           void* out, long out_slice, long ldo, const int* inv, int ncols, cudaStream_t st,
                           const float* cw_h = nullptr) {
    if (std::is_same<T, float>::value && cw_h && nw == ntau) {
      switch (ntau) {
        case 6: return line_ct_reg<6>(ctx, slabs, slab_stride, ld, cw_h, out, out_slice, ldo, inv, ncols, st);
        case 8: return line_ct_reg<8>(ctx, slabs, slab_stride, ld, cw_h, out, out_slice, ldo, inv, ncols, st);
        case 12: return line_ct_reg<12>(ctx, slabs, slab_stride, ld, cw_h, out, out_slice, ldo, inv, ncols, st);
        case 16: return line_ct_reg<16>(ctx, slabs, slab_stride, ld, cw_h, out, out_slice, ldo, inv, ncols, st);
        case 20: return line_ct_reg<20>(ctx, slabs, slab_stride, ld, cw_h, out, out_slice, ldo, inv, ncols, st);
        default: break;
      }
    }
    const size_t bytes = (size_t)ntau * N1 * 32 * sizeof(C) + (size_t)kWParts<T> * nw * ntau * sizeof(T);
    auto kernel = col_line_ct_kernel<T, N1>;
    gw_status s = set_smem(ctx, kernel, bytes);
    if (s) return s;
    dim3 grid((ncols + 31) / 32, N2 * N3);
    KTimer kt(ctx, KF_COL_LINE_CT, ((double)ntau * N1 * N2 * N3 + (double)nw * ncols) * ncols * sizeof(C), st);
    kernel<<<grid, 256, bytes, st>>>((const C*)slabs, slab_stride, ld, ntau, (const T*)cw, nw, (C*)out, out_slice,
                                     ldo, inv, N2 * N3, ncols);
    return launch_check(ctx, "col_line_ct_kernel");
  }
};

template <typename T, typename F>
static bool with_grid(const GridInfo& g, F&& f) {
#define X(a, b, c)                                 \
  if (g.n1 == a && g.n2 == b && g.n3 == c) {       \
    f(GridOps<T, a, b, c>{});                      \
    return true;                                   \
  }
  GW_GRIDS(X)
#undef X
  return false;
}

#define GW_DISPATCH(prec, g, BODY)                                                              \
  gw_status rc = GW_OK;                                                                         \
  bool found = is_fp64(prec) ? with_grid<double>(g, [&](auto ops) { using O = decltype(ops); BODY; }) \
                             : with_grid<float>(g, [&](auto ops) { using O = decltype(ops); BODY; });  \
  if (!found) return fail(ctx, GW_ERR_UNSUPPORTED, "no FFT kernels compiled for this grid");     \
  return rc;

gw_status launch_row_fft(gw_ctx* ctx, const GridInfo& g, gw_prec prec, int mode, const void* a, const void* b,
                         long lda, void* out, long ldo, const int* map, int n_chi, int n_rows, double scale,
                         cudaStream_t st, const int* inv, void* tmp) {
  if (n_rows <= 0) return GW_OK;
  GW_DISPATCH(prec, g, rc = O::row(ctx, mode, a, b, lda, out, ldo, map, n_chi, n_rows, scale, st, inv, tmp))
}

gw_status launch_row_pw_chi(gw_ctx* ctx, const GridInfo& g, gw_prec prec, const void* a, const void* b, long lda,
                            void* out, long ldo, const int* inv_pw, int n_pw, const int* inv_chi, int n_chi,
                            int n_rows, double scale, cudaStream_t st) {
  if (n_rows <= 0) return GW_OK;
  GW_DISPATCH(prec, g, rc = O::row_pw(ctx, a, b, lda, out, ldo, inv_pw, n_pw, inv_chi, n_chi, n_rows, scale, st))
}

gw_status check_row_pw(gw_ctx* ctx, const GridInfo& g, gw_prec prec, int n_pw, int n_chi) {
  GW_DISPATCH(prec, g, rc = O::row_pw_ok(n_pw, n_chi) ? GW_OK : fail(ctx, GW_ERR_UNSUPPORTED,
                                                                     "plane-wave chi rows: this grid, precision and "
                                                                     "G sets do not fit a thread-block cluster"))
}

gw_status launch_row_pw_sigma(gw_ctx* ctx, const GridInfo& g, gw_prec prec, const void* tu, const void* to, long ldt,
                              const void* wg, long ldw, void* hu, void* ho, long ldh, const int* inv_neg,
                              const int* inv_nat, int n_pw, const int* inv_chi, int n_chi, int n_rows,
                              cudaStream_t st) {
  if (n_rows <= 0) return GW_OK;
  GW_DISPATCH(prec, g, rc = O::row_pw_sigma(ctx, tu, to, ldt, wg, ldw, hu, ho, ldh, inv_neg, inv_nat, n_pw, inv_chi,
                                            n_chi, n_rows, st))
}

gw_status check_row_pw_sigma(gw_ctx* ctx, const GridInfo& g, gw_prec prec, int n_pw, int n_chi) {
  GW_DISPATCH(prec, g, rc = O::row_pw_sigma_ok(n_pw, n_chi) ? GW_OK : fail(ctx, GW_ERR_UNSUPPORTED,
                                                                           "plane-wave Sigma rows: this grid, "
                                                                           "precision and G sets do not fit a "
                                                                           "thread-block cluster"))
}

bool row_two_pass(const GridInfo& g, gw_prec prec) {
  const size_t s2 = g.n3 % 2 == 0 ? g.n3 + 1 : g.n3;
  return (size_t)g.n1 * g.n2 * s2 * csize(prec) > kRowSmemMax;
}

gw_status launch_col_plane(gw_ctx* ctx, const GridInfo& g, gw_prec prec, int dir, void* buf, long ld, int ncols,
                           double scale, cudaStream_t st) {
  GW_DISPATCH(prec, g, rc = O::plane(ctx, dir, buf, ld, ncols, scale, st))
}

gw_status launch_col_line(gw_ctx* ctx, const GridInfo& g, gw_prec prec, int dir, int variant, const void* in,
                          long ldi, void* out, long ldo, int ncols, const int* inv, double scale, cudaStream_t st) {
  GW_DISPATCH(prec, g, rc = O::line(ctx, dir, variant, in, ldi, out, ldo, ncols, inv, scale, st))
}

gw_status launch_col_line_ct(gw_ctx* ctx, const GridInfo& g, gw_prec prec, const void* slabs, long slab_stride,
                             long ld, int ntau, const void* cw, int nw, void* out, long out_slice, long ldo,
                             const int* inv, int ncols, cudaStream_t st, const float* cw_h) {
  GW_DISPATCH(prec, g,
              rc = O::line_ct(ctx, slabs, slab_stride, ld, ntau, cw, nw, out, out_slice, ldo, inv, ncols, st, cw_h))
}

template <int NT>
static gw_status launch_ct_reg(gw_ctx* ctx, bool st_kind, const float* w_h, size_t elems, const void* in, void* out,
                               cudaStream_t st) {
  CtWeights<NT> w;
  for (int e = 0; e < NT * NT; ++e) {
    w.hi[e] = w_h[e];
    w.lo[e] = w_h[NT * NT + e];
  }
  KTimer kt(ctx, KF_CT, 2.0 * NT * (double)elems * sizeof(float2), st);
  const int blocks = (int)std::min<size_t>((elems + 255) / 256, (size_t)ctx->num_sms * 12);
  if (st_kind) ct_reg1_kernel<NT, true><<<blocks, 256, 0, st>>>((const float2*)in, (float2*)out, elems, w);
  else ct_reg1_kernel<NT, false><<<blocks, 256, 0, st>>>((const float2*)in, (float2*)out, elems, w);
  return launch_check(ctx, "ct_reg_kernel");
}

gw_status launch_ct(gw_ctx* ctx, gw_prec prec, bool st_kind, int n, const void* dM, size_t elems, const void* in,
                    void* out, cudaStream_t st, const float* w_h) {
  if (elems == 0) return GW_OK;
  if (!is_fp64(prec) && w_h) {
    switch (n) {
      case 6: return launch_ct_reg<6>(ctx, st_kind, w_h, elems, in, out, st);
      case 8: return launch_ct_reg<8>(ctx, st_kind, w_h, elems, in, out, st);
      case 12: return launch_ct_reg<12>(ctx, st_kind, w_h, elems, in, out, st);
      case 16: return launch_ct_reg<16>(ctx, st_kind, w_h, elems, in, out, st);
      case 20: return launch_ct_reg<20>(ctx, st_kind, w_h, elems, in, out, st);
      default: break;
    }
  }
  int blocks = (int)std::min<size_t>((elems + 255) / 256, (size_t)ctx->num_sms * 8);
  if (is_fp64(prec)) {
    if (st_kind) ct_kernel<double, true><<<blocks, 256, 0, st>>>((const double2*)in, (double2*)out, elems, n, (const double*)dM);
    else ct_kernel<double, false><<<blocks, 256, 0, st>>>((const double2*)in, (double2*)out, elems, n, (const double*)dM);
  } else {
    if (st_kind) ct_kernel<float, true><<<blocks, 256, 0, st>>>((const float2*)in, (float2*)out, elems, n, (const float*)dM);
    else ct_kernel<float, false><<<blocks, 256, 0, st>>>((const float2*)in, (float2*)out, elems, n, (const float*)dM);
  }
  return launch_check(ctx, "ct_kernel");
}

gw_status launch_hadamard(gw_ctx* ctx, gw_prec prec, size_t count, const void* a, const void* b, double scale,
                          void* out, cudaStream_t st) {
  if (count == 0) return GW_OK;
  int blocks = (int)std::min<size_t>((count + 255) / 256, (size_t)ctx->num_sms * 16);
  if (is_fp64(prec))
    hadamard_kernel<double><<<blocks, 256, 0, st>>>((const double2*)a, (const double2*)b, (double2*)out, count, scale);
  else
    hadamard_kernel<float><<<blocks, 256, 0, st>>>((const float2*)a, (const float2*)b, (float2*)out, count, (float)scale);
  return launch_check(ctx, "hadamard_kernel");
}

// Transform weights w * fac as FP32 pairs: hi = fl(w fac), lo = fl(w fac - hi);
// returns [hi_0 .. hi_{count-1}, lo_0 .. lo_{count-1}].
std::vector<float> split_weights(const double* w, int count, double fac) {
  std::vector<float> out(2 * (size_t)count);
  for (int e = 0; e < count; ++e) {
    const double v = w[e] * fac;
    out[e] = (float)v;
    out[count + e] = (float)(v - (double)out[e]);
  }
  return out;
}

// Upload a host array into arena memory (pageable copy; the host buffer may be
// released on return).
gw_status upload(gw_ctx* ctx, void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return GW_OK;
  return cuda_check(ctx, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st), "upload");
}

gw_status index_maps(gw_ctx* ctx, const GridInfo& g, const int32_t* fft_index_h, int n_chi, std::vector<int>& map,
                     std::vector<int>& inv) {
  if (!fft_index_h) return fail(ctx, GW_ERR_ARG, "fft_index_h is NULL");
  if (n_chi < 1 || n_chi > g.nr) return fail(ctx, GW_ERR_SHAPE, "need 1 <= n_chi <= N_r");
  map.assign(fft_index_h, fft_index_h + n_chi);
  inv.assign(g.nr, -1);
  for (int j = 0; j < n_chi; ++j) {
    if (map[j] < 0 || map[j] >= g.nr) return fail(ctx, GW_ERR_ARG, "fft_index out of range");
    if (inv[map[j]] >= 0) return fail(ctx, GW_ERR_ARG, "fft_index has duplicates");
    inv[map[j]] = j;
  }
  return GW_OK;
}

}  // namespace gw

using namespace gw;

extern "C" gw_status gw_chi0_rtau(gw_ctx* ctx, int n_rows, int n_cols, gw_prec prec, const void* g_occ,
                                  const void* g_unocc, void* chi, void* stream) {
  if (!ctx) return fail(nullptr, GW_ERR_ARG, "ctx is NULL");
  if (!valid_prec(prec)) return fail(ctx, GW_ERR_ARG, "bad precision");
  if (n_rows < 0 || n_cols < 0) return fail(ctx, GW_ERR_SHAPE, "negative size");
  if ((size_t)n_rows * n_cols == 0) return GW_OK;
  if (!g_occ || !g_unocc || !chi) return fail(ctx, GW_ERR_ARG, "NULL pointer");
  return launch_hadamard(ctx, prec, (size_t)n_rows * n_cols, g_occ, g_unocc, -2.0, chi, as_stream(stream));
}

extern "C" gw_status gw_rr_to_GG_fft(gw_ctx* ctx, const gw_grid* grid, int direction, int stage, int n_chi,
                                     const int32_t* fft_index_h, gw_prec prec, int r0, int n_rows, const void* in,
                                     void* out, void* stream) {
  if (!ctx) return fail(nullptr, GW_ERR_ARG, "ctx is NULL");
  GridInfo g;
  gw_status st = grid_info(ctx, grid, &g);
  if (st) return st;
  if (!grid_supported(g.n1, g.n2, g.n3)) return fail(ctx, GW_ERR_UNSUPPORTED, "no FFT kernels compiled for this grid");
  if (!valid_prec(prec)) return fail(ctx, GW_ERR_ARG, "bad precision");
  if (direction != 1 && direction != -1) return fail(ctx, GW_ERR_ARG, "direction must be +1 or -1");
  if (stage != 1 && stage != 2) return fail(ctx, GW_ERR_ARG, "stage must be 1 or 2");
  if (!in || !out) return fail(ctx, GW_ERR_ARG, "NULL pointer");
  std::vector<int> map, inv;
  if ((st = index_maps(ctx, g, fft_index_h, n_chi, map, inv))) return st;
  if (stage == 1 && (n_rows < 0 || r0 < 0 || r0 + n_rows > g.nr)) return fail(ctx, GW_ERR_SHAPE, "rows out of range");
  cudaStream_t s = as_stream(stream);
  // rows too long for shared memory need a [n_rows][N_r] workspace forward
  const bool work_rows = stage == 1 && direction > 0 && row_two_pass(g, prec);
  Carver probe(nullptr);
  probe.take<int>(n_chi);
  probe.take<int>(g.nr);
  if (work_rows) probe.take<char>((size_t)n_rows * g.nr * csize(prec));
  if ((st = reserve(ctx, probe.off))) return st;
  Carver cv(ctx->arena);
  int* dmap = cv.take<int>(n_chi);
  int* dinv = cv.take<int>(g.nr);
  void* tmp = work_rows ? cv.take<char>((size_t)n_rows * g.nr * csize(prec)) : nullptr;
  if ((st = upload(ctx, dmap, map.data(), sizeof(int) * n_chi, s))) return st;
  if ((st = upload(ctx, dinv, inv.data(), sizeof(int) * g.nr, s))) return st;
  if (stage == 1) {
    if (direction > 0)
      return launch_row_fft(ctx, g, prec, 1, in, nullptr, g.nr, out, n_chi, dmap, n_chi, n_rows, 1.0, s, dinv, tmp);
    return launch_row_fft(ctx, g, prec, 2, in, nullptr, n_chi, out, g.nr, dmap, n_chi, n_rows, 1.0 / g.volume, s,
                          dinv);
  }
  if (direction > 0) {
    // in [N_r][n_chi] is the work buffer: (i2,i3) planes in place, then the i1 pass writes the G rows of out.
    void* work = const_cast<void*>(in);
    if ((st = launch_col_plane(ctx, g, prec, -1, work, n_chi, n_chi, 1.0, s))) return st;
    return launch_col_line(ctx, g, prec, -1, 2, work, n_chi, out, n_chi, n_chi, dinv, g.dv * g.dv / g.volume, s);
  }
  // W(G,G') -> W(r,G'): i1 pass gathering the G rows, then the (i2,i3) planes in place in out.
  if ((st = launch_col_line(ctx, g, prec, +1, 1, in, n_chi, out, n_chi, n_chi, dinv, 1.0, s))) return st;
  return launch_col_plane(ctx, g, prec, +1, out, n_chi, n_chi, 1.0, s);
}

extern "C" gw_status gw_tau_to_omega(gw_ctx* ctx, int kind, int n, const double* M_h, size_t elems, gw_prec prec,
                                     const void* in, void* out, void* stream) {
  if (!ctx) return fail(nullptr, GW_ERR_ARG, "ctx is NULL");
  if (!valid_prec(prec)) return fail(ctx, GW_ERR_ARG, "bad precision");
  if (kind != GW_CT && kind != GW_ST && kind != GW_IST) return fail(ctx, GW_ERR_ARG, "kind must be GW_CT, GW_ST or GW_IST");
  if (n < 1 || n > 32) return fail(ctx, GW_ERR_SHAPE, "need 1 <= n <= 32");
  if (!M_h || !in || !out) return fail(ctx, GW_ERR_ARG, "NULL pointer");
  if (in == out) return fail(ctx, GW_ERR_ARG, "in and out must not overlap");
  cudaStream_t s = as_stream(stream);
  gw_status st = reserve(ctx, 8 * 32 * 32);
  if (st) return st;
  std::vector<double> neg;
  if (kind == GW_IST) {             // -i sum M x = i sum (-M) x: the sine kernel with M negated
    neg.assign(M_h, M_h + (size_t)n * n);
    for (double& v : neg) v = -v;
    M_h = neg.data();
  }
  std::vector<float> m32;
  if (is_fp64(prec)) {
    if ((st = upload(ctx, ctx->arena, M_h, sizeof(double) * n * n, s))) return st;
  } else {
    m32 = split_weights(M_h, n * n, 1.0);
    if ((st = upload(ctx, ctx->arena, m32.data(), sizeof(float) * 2 * n * n, s))) return st;
  }
  return launch_ct(ctx, prec, kind != GW_CT, n, ctx->arena, elems, in, out, s, m32.empty() ? nullptr : m32.data());
}

// ---------------------------------------------------------------------- no-allocation variant
//
// gw_rr_to_GG_fft needs two small index maps on the device (the G set's FFT
// positions and their inverse).  The regular entry point keeps them in the
// context's scratch arena, which is created with cudaMalloc.  This variant keeps
// them instead in one fixed array in the library's own device memory, so a
// caller that may not allocate device memory at all can still run the
// transform: for example a program whose memory pool has taken the whole GPU
// and forbids any other cudaMalloc, or a serving loop that cannot afford the
// device-wide synchronisation a cudaMalloc/cudaFree may bring.  The maps are
// still uploaded on every call, by cudaMemcpyAsync from pageable host memory:
// that copy waits for the stream's earlier work before it starts, so a call
// is not free of host-side waiting, only of allocation.

namespace {

constexpr int kNoAllocMaxInts = 2 * 13824;   // n_chi + N_r for the largest compiled grid (24^3)

// Holds fft_index followed by its inverse map.  Every GPU that loads the
// library keeps this array until the process exits; all calls share it.
static __device__ __align__(256) int g_noalloc_maps[kNoAllocMaxInts];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
int* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_maps on the current device (looked up once per
// device).  In host code the symbol itself is only a host-side stand-in.
gw_status noalloc_maps_ptr(gw_ctx* err_ctx, int** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_check(err_ctx, e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(err_ctx, GW_ERR_UNSUPPORTED, "device index too large");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_maps);
    if (e != cudaSuccess) return cuda_check(err_ctx, e, "cudaGetSymbolAddress(g_noalloc_maps)");
    g_noalloc_ptr[dev] = static_cast<int*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return GW_OK;
}

}  // namespace

extern "C" gw_status gw_rr_to_GG_fft_noalloc(const gw_grid* grid, int direction, int stage, int n_chi,
                                             const int32_t* fft_index_h, gw_prec prec, int r0, int n_rows,
                                             const void* in, void* out, void* stream) {
  gw_ctx local;                       // host-only bookkeeping: no device memory behind it
  local.num_sms = 1;
  auto done = [&](gw_status st) {
    if (st) fail(nullptr, st, local.err);
    return st;
  };
  GridInfo g;
  gw_status st = grid_info(&local, grid, &g);
  if (st) return done(st);
  if (!grid_supported(g.n1, g.n2, g.n3)) return done(fail(&local, GW_ERR_UNSUPPORTED, "no FFT kernels compiled for this grid"));
  if (!valid_prec(prec)) return done(fail(&local, GW_ERR_ARG, "bad precision"));
  if (direction != 1 && direction != -1) return done(fail(&local, GW_ERR_ARG, "direction must be +1 or -1"));
  if (stage != 1 && stage != 2) return done(fail(&local, GW_ERR_ARG, "stage must be 1 or 2"));
  if (!in || !out) return done(fail(&local, GW_ERR_ARG, "NULL pointer"));
  cudaStream_t s = as_stream(stream);
  // The maps are copied from host vectors that live only for this call: a
  // captured copy would replay from freed host memory, so refuse capture.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t ce = cudaStreamIsCapturing(s, &cap);
  if (ce != cudaSuccess) return done(cuda_check(&local, ce, "cudaStreamIsCapturing"));
  if (cap != cudaStreamCaptureStatusNone)
    return done(fail(&local, GW_ERR_UNSUPPORTED,
                     "gw_rr_to_GG_fft_noalloc cannot be called while its stream is being captured"));
  std::vector<int> map, inv;
  if ((st = index_maps(&local, g, fft_index_h, n_chi, map, inv))) return done(st);
  if ((long)n_chi + g.nr > kNoAllocMaxInts)
    return done(fail(&local, GW_ERR_SHAPE, "n_chi + N_r exceeds the fixed index-map capacity of " +
                                               std::to_string(kNoAllocMaxInts) + " entries"));
  if (stage == 1 && (n_rows < 0 || r0 < 0 || r0 + n_rows > g.nr))
    return done(fail(&local, GW_ERR_SHAPE, "rows out of range"));
  int* maps = nullptr;
  if ((st = noalloc_maps_ptr(&local, &maps))) return done(st);
  int* dmap = maps;
  int* dinv = maps + n_chi;
  // both maps are rewritten in full on every call, so nothing carries over
  if ((st = upload(&local, dmap, map.data(), sizeof(int) * n_chi, s))) return done(st);
  if ((st = upload(&local, dinv, inv.data(), sizeof(int) * g.nr, s))) return done(st);
  if (stage == 1) {
    if (direction > 0) st = launch_row_fft(&local, g, prec, 1, in, nullptr, g.nr, out, n_chi, dmap, n_chi, n_rows, 1.0, s);
    else st = launch_row_fft(&local, g, prec, 2, in, nullptr, n_chi, out, g.nr, dmap, n_chi, n_rows, 1.0 / g.volume, s);
    return done(st);
  }
  if (direction > 0) {
    void* work = const_cast<void*>(in);
    if ((st = launch_col_plane(&local, g, prec, -1, work, n_chi, n_chi, 1.0, s))) return done(st);
    return done(launch_col_line(&local, g, prec, -1, 2, work, n_chi, out, n_chi, n_chi, dinv, g.dv * g.dv / g.volume, s));
  }
  if ((st = launch_col_line(&local, g, prec, +1, 1, in, n_chi, out, n_chi, n_chi, dinv, 1.0, s))) return done(st);
  return done(launch_col_plane(&local, g, prec, +1, out, n_chi, n_chi, 1.0, s));
}
