// sg_mlp_api.cpp -- the cost model's network kernels on caller buffers.
#include <cuda_runtime.h>

#include "sg_mlp.h"
#include "sg_runtime.h"

namespace {

sg_status done(sg_ctx* c, cudaError_t e) {
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->err = cudaGetErrorString(e);
    return SG_ERR_CUDA;
  }
  return SG_OK;
}

}  // namespace

extern "C" sg_status sg_mlp_forward(sg_ctx* c, const float* P, int32_t d_in, const float* X,
                                    int64_t B, float* yhat) {
  if (!c || c->planning_only || !P || !X || !yhat || d_in < 1 || d_in > 32 || B < 1 ||
      B > (1 << 24))
    return SG_ERR_INVALID_ARG;
  c->kernels += 1;
  return done(c, sgk::launch_mlp_forward(P, d_in, X, (int)B, yhat, c->stream));
}

extern "C" sg_status sg_mlp_loss_grad(sg_ctx* c, const float* P, int32_t d_in, const float* X,
                                      const float* y, int64_t B, float* G, float* loss) {
  if (!c || c->planning_only || !P || !X || !y || !G || d_in < 1 || d_in > 32 || B < 1 ||
      B > (1 << 20))
    return SG_ERR_INVALID_ARG;
  void* work = nullptr;
  cudaError_t e = cudaMallocAsync(&work, sgk::mlp_work_bytes((int)B), c->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SG_ERR_OOM;
  }
  e = sgk::launch_mlp_loss_grad(P, d_in, X, y, (int)B, G, loss, work, c->stream);
  cudaFreeAsync(work, c->stream);
  c->kernels += 4;
  return done(c, e);
}

extern "C" sg_status sg_mlp_adam(sg_ctx* c, float* P, const float* G, float* m, float* v,
                                 int64_t np, int64_t step, float lr, float b1, float b2,
                                 float eps) {
  if (!c || c->planning_only || !P || !G || !m || !v || np < 1 || step < 1) return SG_ERR_INVALID_ARG;
  c->kernels += 1;
  return done(c, sgk::launch_mlp_adam(P, G, m, v, (int)np, step, lr, b1, b2, eps, c->stream));
}
