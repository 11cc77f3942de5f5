// Shared-memory 3-D FFT of one grid row (internal).
#pragma once

#include "gw_common.cuh"

namespace gw {

template <int N1, int N2, int N3>
struct RowLayout {
  static constexpr int S2 = N3 % 2 == 0 ? N3 + 1 : N3;   // odd pencil stride
  static constexpr int S1 = N2 * S2;
  static constexpr int TOT = N1 * S1;
  static constexpr int NR = N1 * N2 * N3;
  __device__ __forceinline__ static int pos(int r) {
    const int i1 = r / (N2 * N3);
    const int rem = r - i1 * (N2 * N3);
    const int i2 = rem / N3;
    const int i3 = rem - i2 * N3;
    return i1 * S1 + i2 * S2 + i3;
  }
};

// Two consecutive complex elements in one 16-byte access (FP32), two for FP64.
__device__ __forceinline__ void ld_pair(const float2* p, float2& a, float2& b) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void ld_pair(const double2* p, double2& a, double2& b) {
  a = __ldg(p);
  b = __ldg(p + 1);
}
__device__ __forceinline__ void st_pair(float2* p, float2 a, float2 b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st_pair(double2* p, double2 a, double2 b) {
  p[0] = a;
  p[1] = b;
}

template <int N, int DIR, typename C, typename BaseF>
__device__ __forceinline__ void pencil_pass(C* s, int count, int stride, BaseF base) {
  for (int p = threadIdx.x; p < count; p += blockDim.x) {
    const int b = base(p);
    C x[N];
#pragma unroll
    for (int k = 0; k < N; ++k) x[k] = s[b + k * stride];
    RegFFT<N, DIR>::run(x);
#pragma unroll
    for (int k = 0; k < N; ++k) s[b + k * stride] = x[k];
  }
}

template <int N1, int N2, int N3, int DIR, typename C>
__device__ __forceinline__ void fft3_smem(C* s) {
  using L = RowLayout<N1, N2, N3>;
  pencil_pass<N3, DIR>(s, N1 * N2, 1, [](int p) { return p * L::S2; });
  __syncthreads();
  pencil_pass<N2, DIR>(s, N1 * N3, L::S2, [](int p) { return (p / N3) * L::S1 + (p % N3); });
  __syncthreads();
  pencil_pass<N1, DIR>(s, N2 * N3, L::S1, [](int p) { return (p / N3) * L::S2 + (p % N3); });
  __syncthreads();
}

}  // namespace gw
