// k_gemm_simt.cu -- matrix `multiply` of Sec. 3.4 in binary32 on the CUDA
// cores (sm_103a): C = A B, row-major.  The plain form the tensor-core path
// is measured against.
//
// 128x128 CTA tile, 8-deep k slices, 256 threads each owning an 8x8 block of
// C in registers (two 4x4 quadrants per dimension, so shared-memory reads
// are 128-bit and conflict-free).  Shared memory is double-buffered: the
// next slice is fetched into registers while the current one is consumed.
#include "sg_linalg_kernels.h"

namespace sgk {
namespace {

constexpr int BM = 128, BN = 128, BK = 8;

template <bool VEC>
__global__ void __launch_bounds__(256) k_gemm_f32(const float* __restrict__ A, int lda,
                                                  const float* __restrict__ B, int ldb,
                                                  float* __restrict__ C, int ldc, int M, int N,
                                                  int K, int subtract) {
  __shared__ __align__(16) float As[2][BK][BM];
  __shared__ __align__(16) float Bs[2][BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  // global -> shared mapping: A slice 128x8 (one float4 of a row per thread),
  // B slice 8x128 (one float4 of a row per thread)
  const int a_row = tid >> 1, a_k = (tid & 1) * 4;
  const int b_k = tid >> 5, b_n = (tid & 31) * 4;

  float ra[4], rb[4];
  auto load = [&](int k0) {
    const int gm = m0 + a_row;
    const int gk = k0 + a_k;
    if (VEC && gm < M && gk + 3 < K) {
      const float4 t = *reinterpret_cast<const float4*>(A + (size_t)gm * lda + gk);
      ra[0] = t.x; ra[1] = t.y; ra[2] = t.z; ra[3] = t.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        ra[j] = (gm < M && gk + j < K) ? A[(size_t)gm * lda + gk + j] : 0.0f;
    }
    const int gkb = k0 + b_k;
    const int gn = n0 + b_n;
    if (VEC && gkb < K && gn + 3 < N) {
      const float4 t = *reinterpret_cast<const float4*>(B + (size_t)gkb * ldb + gn);
      rb[0] = t.x; rb[1] = t.y; rb[2] = t.z; rb[3] = t.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        rb[j] = (gkb < K && gn + j < N) ? B[(size_t)gkb * ldb + gn + j] : 0.0f;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int j = 0; j < 4; ++j) As[buf][a_k + j][a_row] = ra[j];
    *reinterpret_cast<float4*>(&Bs[buf][b_k][b_n]) = make_float4(rb[0], rb[1], rb[2], rb[3]);
  };

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

  const int nk = (K + BK - 1) / BK;
  load(0);
  store(0);
  __syncthreads();
  for (int kt = 0; kt < nk; ++kt) {
    const int cur = kt & 1;
    if (kt + 1 < nk) load((kt + 1) * BK);
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      float a[8], b[8];
      const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][k][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][k][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][k][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][k][64 + tx * 4]);
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
      a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
      b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
      b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (kt + 1 < nk) store(cur ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gm = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
    if (gm >= M) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int gn = n0 + h * 64 + tx * 4;
      float* c = C + (size_t)gm * ldc + gn;
      if (VEC && gn + 3 < N) {
        float4 v = make_float4(acc[i][h * 4], acc[i][h * 4 + 1], acc[i][h * 4 + 2],
                               acc[i][h * 4 + 3]);
        if (subtract) {
          const float4 o = *reinterpret_cast<const float4*>(c);
          v = make_float4(o.x - v.x, o.y - v.y, o.z - v.z, o.w - v.w);
        }
        *reinterpret_cast<float4*>(c) = v;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (gn + j < N) c[j] = subtract ? c[j] - acc[i][h * 4 + j] : acc[i][h * 4 + j];
      }
    }
  }
}

}  // namespace

cudaError_t launch_gemm_f32(const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                            int M, int N, int K, bool subtract, cudaStream_t s, Prof* prof) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const bool vec = (lda % 4 == 0) && (ldb % 4 == 0) && (ldc % 4 == 0) &&
                   ((uintptr_t)A % 16 == 0) && ((uintptr_t)B % 16 == 0) &&
                   ((uintptr_t)C % 16 == 0);
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
  prof_begin(prof, "gemm_f32_simt", s);
  if (vec)
    k_gemm_f32<true><<<grid, 256, 0, s>>>(A, lda, B, ldb, C, ldc, M, N, K, subtract ? 1 : 0);
  else
    k_gemm_f32<false><<<grid, 256, 0, s>>>(A, lda, B, ldb, C, ldc, M, N, K, subtract ? 1 : 0);
  prof_end(prof, s);
  return cudaGetLastError();
}

}  // namespace sgk
