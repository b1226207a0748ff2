// k_fprint.cu -- the `old` of Sec. 4's postconditions (Listing 3:
// `Current = old Current`) without a copy of the collection: a
// position-dependent fingerprint of a value's bytes, taken when the snapshot
// is queued and again when the postcondition is checked.
//
// The value is read as units of its element width (16-bit units for bf16 /
// fp16, 32-bit words otherwise; 64-bit elements are two words).  Unit i with
// bits w contributes h_i = mix64(i * 2^32 + w), mix64 being SplitMix64's
// output function (Steele, Lea, Flood 2014), a bijection of 64-bit words: so
// the pair (i, w) determines h_i and changing any one unit changes
// F1 = sum h_i.  F2 = sum hi32(h_i) * lo32(h_i) is a second, non-linear sum.
// Both are taken mod 2^64: integer sums are exact and independent of the
// order of the additions, so the fingerprint is deterministic.  One read of
// the value (its bytes), HBM-bound.
#include <stdint.h>

#include "sg_internal.h"

namespace sgk {
namespace {

__device__ __forceinline__ unsigned long long fp_mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ void fp_unit(unsigned long long i, unsigned w, unsigned long long& f1,
                                        unsigned long long& f2) {
  const unsigned long long h = fp_mix64((i << 32) | w);
  f1 += h;
  f2 += (unsigned long long)(unsigned)(h >> 32) * (unsigned)h;
}

// U: the unit type (uint16_t or uint32_t); units = bytes / sizeof(U)
template <typename U>
__global__ void __launch_bounds__(256) k_fprint(const U* __restrict__ x, long long units,
                                                unsigned long long* out) {
  constexpr int kPer = 16 / sizeof(U);   // units per 16-byte load
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  unsigned long long f1 = 0, f2 = 0;
  long long start = 0;
  if (((uintptr_t)x & 15) == 0) {
    const long long nv = units / kPer;
    start = nv * kPer;
    const uint4* x4 = reinterpret_cast<const uint4*>(x);
    for (long long v = tid; v < nv; v += stride) {
      const uint4 q = __ldcs(x4 + v);
      const unsigned wd[4] = {q.x, q.y, q.z, q.w};
      const long long i0 = v * kPer;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (sizeof(U) == 4) {
          fp_unit((unsigned long long)(i0 + k), wd[k], f1, f2);
        } else {
          fp_unit((unsigned long long)(i0 + 2 * k), wd[k] & 0xFFFFu, f1, f2);
          fp_unit((unsigned long long)(i0 + 2 * k + 1), wd[k] >> 16, f1, f2);
        }
      }
    }
  }
  for (long long i = start + tid; i < units; i += stride)
    fp_unit((unsigned long long)i, (unsigned)__ldcs(x + i), f1, f2);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    f1 += __shfl_xor_sync(0xffffffffu, f1, o);
    f2 += __shfl_xor_sync(0xffffffffu, f2, o);
  }
  if ((threadIdx.x & 31) == 0 && (f1 | f2)) {
    atomicAdd(out, f1);
    atomicAdd(out + 1, f2);
  }
}

}  // namespace

cudaError_t launch_fprint(const void* x, size_t bytes, int unit_bytes, unsigned long long* out,
                          cudaStream_t s, int num_sms, int64_t* kernels, Prof* prof) {
  cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(unsigned long long), s);
  if (e != cudaSuccess || bytes == 0) return e;
  const long long units = (long long)(bytes / (size_t)unit_bytes);
  long long grid = (units / (16 / unit_bytes) + 255) / 256;
  const long long cap = (long long)num_sms * 8;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  prof_begin(prof, "fingerprint_old", s);
  if (unit_bytes == 2)
    k_fprint<uint16_t><<<(int)grid, 256, 0, s>>>(static_cast<const uint16_t*>(x), units, out);
  else
    k_fprint<uint32_t><<<(int)grid, 256, 0, s>>>(static_cast<const uint32_t*>(x), units, out);
  prof_end(prof, s);
  *kernels += 1;
  return cudaGetLastError();
}

}  // namespace sgk
