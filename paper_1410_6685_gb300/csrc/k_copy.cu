// k_copy.cu -- contiguous copies (sm_103a): `concatenate` (Table 2) places
// its operands one after the other in a new vector, and a flush stores its
// pass results into the pinned host buffer (device-addressable) with it.
// 16-byte loads and stores when both ends are 16-byte aligned and the length
// is a multiple of 16, else 4-byte, else single bytes; grid-stride.
#include "sg_internal.h"

namespace sgk {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_copy(const T* __restrict__ src, T* __restrict__ dst,
                                              long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

}  // namespace

cudaError_t launch_copy(void* dst, const void* src, size_t bytes, int num_sms, cudaStream_t s) {
  if (bytes == 0) return cudaSuccess;
  const uintptr_t a = (uintptr_t)dst | (uintptr_t)src;
  auto grid = [&](long long units) {
    long long g = (units + 255) / 256;
    const long long cap = (long long)num_sms * 8;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
  };
  if ((a % 16) == 0 && bytes % 16 == 0) {
    const long long n = (long long)(bytes / 16);
    k_copy<uint4><<<grid(n), 256, 0, s>>>(static_cast<const uint4*>(src), static_cast<uint4*>(dst), n);
  } else if ((a % 4) == 0 && bytes % 4 == 0) {
    const long long n = (long long)(bytes / 4);
    k_copy<unsigned><<<grid(n), 256, 0, s>>>(static_cast<const unsigned*>(src),
                                            static_cast<unsigned*>(dst), n);
  } else {
    const long long n = (long long)bytes;
    k_copy<unsigned char><<<grid(n), 256, 0, s>>>(static_cast<const unsigned char*>(src),
                                                 static_cast<unsigned char*>(dst), n);
  }
  return cudaGetLastError();
}

}  // namespace sgk
