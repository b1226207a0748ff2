// k_freivalds.cu -- the postcondition of matrix `multiply` (Sec. 3.4):
// Freivalds' randomized check that C = A B, evaluated on the GPU.
//
// For each of `nvec` Rademacher vectors r (entries +-1 from the SplitMix64
// stream `seed`, draw t = v*N + j + 1 for entry j of vector v):
//   z = A (B r),  w = C r,  and row i is violated when |z_i - w_i| > tau_i,
//   tau_i = c * u_eff * sqrt( sum_k a_ik^2 ((B r)_k^2 + s_k) ),  s_k = sum_j b_kj^2,
// a c-sigma bound on the rounding noise of a product whose operand rounding
// and accumulation have unit roundoff u_eff.  Three streaming passes, one
// warp per row: r, then B (B r and s), then A and C together.
#include <math.h>

#include "sg_linalg_kernels.h"

namespace sgk {
namespace {

constexpr int kMaxVec = 8;

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_frv_r(float* r, int N, int nvec, unsigned long long seed) {
  const long long total = (long long)N * nvec;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const unsigned long long z = mix64(seed + (unsigned long long)(t + 1) * 0x9E3779B97F4A7C15ull);
    r[t] = (z >> 63) ? -1.0f : 1.0f;   // r[v*N + j]
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// br[v*N + k] = sum_j B[k][j] r[v][j];  s[k] = sum_j B[k][j]^2
template <int NV>
__global__ void __launch_bounds__(256) k_frv_b(const float* __restrict__ B, int N,
                                               const float* __restrict__ r, float* br, float* s) {
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long k = warp; k < N; k += nwarps) {
    const float* row = B + k * (long long)N;
    float acc[NV], sq = 0.0f;
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0.0f;
    for (int j = lane; j < N; j += 32) {
      const float b = __ldcs(row + j);
      sq = fmaf(b, b, sq);
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] = fmaf(b, __ldg(r + (long long)v * N + j), acc[v]);
    }
    sq = warp_sum(sq);
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = warp_sum(acc[v]);
    if (lane == 0) {
      s[k] = sq;
#pragma unroll
      for (int v = 0; v < NV; ++v) br[(long long)v * N + k] = acc[v];
    }
  }
}

template <int NV>
__global__ void __launch_bounds__(256) k_frv_ac(const float* __restrict__ A,
                                                const float* __restrict__ C, int N,
                                                const float* __restrict__ r,
                                                const float* __restrict__ br,
                                                const float* __restrict__ s, float c, float u_eff,
                                                FreivaldsResult* res) {
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long i = warp; i < N; i += nwarps) {
    const float* arow = A + i * (long long)N;
    const float* crow = C + i * (long long)N;
    float z[NV], q[NV], w[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) z[v] = q[v] = w[v] = 0.0f;
    for (int k = lane; k < N; k += 32) {
      const float a = __ldcs(arow + k);
      const float cc = __ldcs(crow + k);
      const float a2 = a * a;
      const float sk = __ldg(s + k);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float b = __ldg(br + (long long)v * N + k);
        z[v] = fmaf(a, b, z[v]);
        q[v] = fmaf(a2, fmaf(b, b, sk), q[v]);
        w[v] = fmaf(cc, __ldg(r + (long long)v * N + k), w[v]);
      }
    }
    float worst = 0.0f;
    bool bad = false;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const float zz = warp_sum(z[v]), qq = warp_sum(q[v]), ww = warp_sum(w[v]);
      const float tau = c * u_eff * sqrtf(qq);
      const float gap = fabsf(zz - ww);
      const float ratio = tau > 0.0f ? gap / tau : (gap > 0.0f ? INFINITY : 0.0f);
      worst = fmaxf(worst, ratio);
      bad |= !(gap <= tau);
    }
    if (lane == 0) {
      if (bad) atomicMax(&res->viol_enc, ~(unsigned long long)i);
      // ratios are non-negative: their float bits order like unsigned ints
      atomicMax(reinterpret_cast<unsigned*>(&res->max_ratio), __float_as_uint(worst));
    }
  }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

size_t freivalds_scratch_bytes(int N, int nvec) {
  return 2 * align256((size_t)N * nvec * sizeof(float)) + align256((size_t)N * sizeof(float));
}

cudaError_t launch_freivalds(const float* A, const float* B, const float* C, int N,
                             unsigned long long seed, int nvec, float c, float u_eff,
                             void* scratch, FreivaldsResult* res, cudaStream_t st, Prof* prof,
                             int64_t* kernels) {
  if (N <= 0) return cudaSuccess;
  if (nvec < 1 || nvec > kMaxVec) return cudaErrorInvalidValue;
  char* p = static_cast<char*>(scratch);
  float* r = reinterpret_cast<float*>(p);
  float* br = reinterpret_cast<float*>(p + align256((size_t)N * nvec * sizeof(float)));
  float* s = reinterpret_cast<float*>(p + 2 * align256((size_t)N * nvec * sizeof(float)));
  const int rows_grid = (N + 7) / 8;   // 8 warps per block, one row per warp
  prof_begin(prof, "freivalds", st);
  k_frv_r<<<(N * nvec + 255) / 256, 256, 0, st>>>(r, N, nvec, seed);
#define SG_FRV(NV)                                                                      \
  k_frv_b<NV><<<rows_grid, 256, 0, st>>>(B, N, r, br, s);                               \
  k_frv_ac<NV><<<rows_grid, 256, 0, st>>>(A, C, N, r, br, s, c, u_eff, res)
  switch (nvec) {
    case 1: SG_FRV(1); break;
    case 2: SG_FRV(2); break;
    case 3: SG_FRV(3); break;
    case 4: SG_FRV(4); break;
    case 5: SG_FRV(5); break;
    case 6: SG_FRV(6); break;
    case 7: SG_FRV(7); break;
    default: SG_FRV(8); break;
  }
#undef SG_FRV
  prof_end(prof, st);
  *kernels += 3;
  return cudaGetLastError();
}

}  // namespace sgk
