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
// inj_row / inj_col >= 0: contract testing, inj_delta is added to that
// product element before it is stored.
size_t gemm_tc_scratch_bytes(int M, int N, int K);
// process-wide: use the portable kernel forms (one-CTA tensor-core product,
// 8-CTA elimination panel) even where the device schedules the fast ones
void set_portable_kernels(bool on);
bool portable_kernels();
// kernel attributes and the CTA-pair decision of the tensor-core product;
// called before a product is captured into a graph
void gemm_tc_prepare();
// form: 0 the CTA-pair kernel where the device schedules pairs, else the
// one-CTA kernel; 1 the one-CTA kernel; 2 the pair where available
cudaError_t launch_gemm_tc(const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                           int M, int N, int K, bool fp16, bool subtract, void* scratch,
                           cudaStream_t s, Prof* prof, int64_t* kernels, int inj_row = -1,
                           int inj_col = -1, float inj_delta = 0.0f, int form = 0);
bool gemm_pair_available();
// Casts the operands once, then times the product C = A B in each of `forms`
// (a warm-up, then the better of two runs, CUDA events on s, a product
// under 16 us repeated within a run; waits for s): us[f] microseconds.  C
// holds the last form's result.
cudaError_t time_gemm_forms(const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                            int M, int N, int K, bool fp16, void* scratch, cudaStream_t s,
                            const int* forms, int nforms, double* us, int64_t* kernels);

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

// Freivalds' check fused into the tensor-core product of square N x N
// matrices: the cast of B also forms the partial sums of B r and |B_k|^2,
// the cast of A those of A (B r) and (A.A) t, and the GEMM epilogue those of
// C r, so the check reads no matrix a second time.  Partial sums are over
// column stripes (kFrvStripeB of B, kFrvStripeA of A, kFrvTileC of C) and are
// added in a fixed order by the final per-row test.
constexpr int kFrvStripeB = 512;
constexpr int kFrvStripeA = 1024;
constexpr int kFrvTileC = 128;
struct FrvFused {
  float4* r4;      // [N] the nvec Rademacher vectors, entry j of each
  float4* br4;     // [N] B r
  float4* t4;      // [N] (B r)_k^2 + |B_k|^2
  float* pb;       // [nsb][N][5] partial B r and |B_k|^2
  float* pzq;      // [nsa][N][8] partial A (B r) and (A.A) t
  float4* pw;      // [nsc][N] partial C r
  int nsb, nsa, nsc;
  size_t bytes;
};
FrvFused frv_fused_layout(void* scratch, int N);
size_t frv_fused_scratch_bytes(int N);
cudaError_t launch_frv_vectors(const FrvFused& f, int N, int nvec, unsigned long long seed,
                               cudaStream_t st);
cudaError_t launch_frv_b_reduce(const FrvFused& f, int N, cudaStream_t st);
cudaError_t launch_frv_check_fused(const FrvFused& f, int N, int nvec, float c, float u_eff,
                                   FreivaldsResult* res, cudaStream_t st);
// C = A B on the tensor cores with the fused check (scratch: gemm_tc_scratch_bytes
// followed by frv_fused_scratch_bytes)
cudaError_t launch_gemm_tc_checked(const float* A, const float* B, float* C, int N, bool fp16,
                                   unsigned long long seed, int nvec, float c, float u_eff,
                                   void* scratch, FreivaldsResult* res, cudaStream_t s,
                                   Prof* prof, int64_t* kernels, int inj_row = -1,
                                   int inj_col = -1, float inj_delta = 0.0f, int form = 0);

// Sec. 3.4 `transpose`, `right_multiply`, `left_multiply` (binary32,
// row-major).  At: cols x rows.  matvec: y = A x (x: cols, y: rows); vecmat:
// y = x^T A (x: rows, y: cols), scratch of vecmat_scratch_bytes(rows, cols).
cudaError_t launch_transpose(const float* A, int rows, int cols, float* At, cudaStream_t s,
                             Prof* prof);
cudaError_t launch_matvec(const float* A, int rows, int cols, const float* x, float* y,
                          cudaStream_t s, Prof* prof);
size_t vecmat_scratch_bytes(int rows, int cols);
cudaError_t launch_vecmat(const float* x, const float* A, int rows, int cols, float* y,
                          void* scratch, cudaStream_t s, Prof* prof);

}  // namespace sgk
