// sg_linalg_kernels.h -- matrix product, Freivalds check and elimination
// kernels (k_gemm_*.cu, k_freivalds.cu, k_lu.cu).  Internal.
#pragma once
#include "sg_internal.h"

namespace sgk {

// binary32 SIMT product C = A B (or C = C - A B), row-major with leading
// dimensions (M x K, K x N, M x N).
cudaError_t launch_gemm_f32(const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                            int M, int N, int K, bool subtract, cudaStream_t s, Prof* prof);

// Tensor-core product: operands rounded (nearest even) to bf16 or fp16,
// binary32 accumulation in tensor memory.  beta = 0: C = A B; beta = 1:
// C = C - A B (the elimination update).  a16 / bt16 are scratch operand
// copies (M x Kp and N x Kp, K-major, Kp = K rounded up to 64).
size_t gemm_tc_scratch_bytes(int M, int N, int K);
cudaError_t launch_gemm_tc(const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                           int M, int N, int K, bool fp16, bool subtract, void* scratch,
                           cudaStream_t s, Prof* prof, int64_t* kernels);

// Freivalds' check of C = A B for square N x N matrices with `nvec`
// Rademacher vectors drawn from SplitMix64 (seed); tau_i = c u_eff sigma_i.
struct FreivaldsResult {
  unsigned long long viol_enc;   // ~row of the smallest violated row, 0 = none
  float max_ratio;               // largest |z_i - w_i| / tau_i seen
  int pad;
};
size_t freivalds_scratch_bytes(int N, int nvec);
cudaError_t launch_freivalds(const float* A, const float* B, const float* C, int N,
                             unsigned long long seed, int nvec, float c, float u_eff,
                             void* scratch, FreivaldsResult* res, cudaStream_t s,
                             Prof* prof, int64_t* kernels);

}  // namespace sgk
