// sg_frv.cuh -- device helpers of the Freivalds partial sums, shared by the
// stand-alone check (k_freivalds.cu) and the fused product (k_gemm_tc.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sgk {
namespace frv {

// Sum each of V values (V = 8 or 16) over the warp's 32 lanes.  While more
// than one value is left, partner lanes swap halves (each keeps one half and
// adds the partner's copy of it), then the last value is summed over the
// remaining lanes.  Lane l ends up with the total of value (l >> 1) & 15 when
// V = 16, of value (l >> 2) & 7 when V = 8.
template <int V>
__device__ __forceinline__ float warp_sum_spread(float (&o)[V], int lane) {
  int off = 16;
#pragma unroll
  for (int h = V / 2; h >= 1; h >>= 1, off >>= 1) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      const float send = up ? o[j] : o[j + h];
      const float keep = up ? o[j + h] : o[j];
      o[j] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  float v = o[0];
  for (; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// four consecutive entries of a row from column `col` (zeros past N); a
// 16-byte load when `vec` says rows are 16-byte aligned
__device__ __forceinline__ float4 ldv(const float* row, long long col, int N, bool vec) {
  if (vec && col + 3 < N) return __ldcs(reinterpret_cast<const float4*>(row + col));
  float v[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] = col + q < N ? __ldcs(row + col + q) : 0.0f;
  return make_float4(v[0], v[1], v[2], v[3]);
}

__device__ __forceinline__ float4 ldvec(const float4* p, long long j, int N) {
  return j < N ? p[j] : make_float4(0.f, 0.f, 0.f, 0.f);
}

}  // namespace frv
}  // namespace sgk
