// sg_mlp.h -- the 2x64 MLP cost model kernels (k_mlp.cu).  Internal.
#pragma once
#include "sg_internal.h"

namespace sgk {

constexpr int kMlpHidden = 64;

__host__ __device__ inline int mlp_nparams(int d_in) {
  return kMlpHidden * d_in + kMlpHidden + kMlpHidden * kMlpHidden + kMlpHidden + kMlpHidden + 1;
}

// work buffer of launch_mlp_loss_grad for a batch of B samples
size_t mlp_work_bytes(int B);
cudaError_t launch_mlp_forward(const float* P, int d_in, const float* X, int B, float* yhat,
                               cudaStream_t s);
cudaError_t launch_mlp_loss_grad(const float* P, int d_in, const float* X, const float* y, int B,
                                 float* G, float* loss, void* work, cudaStream_t s);
cudaError_t launch_mlp_adam(float* P, const float* G, float* m, float* v, int np, long long t,
                            float lr, float b1, float b2, float eps, cudaStream_t s);

}  // namespace sgk
