// k_mlp.cu -- the 2x64 MLP cost model trained on the GPU (sm_103a).
//
// yhat = W3 relu(W2 relu(W1 x + b1) + b2) + b3, hidden width 64, binary32.
// Parameters are one flat vector [W1 (64 x d_in, row-major), b1, W2 (64 x 64),
// b2, W3 (64), b3].  Loss = mean over the batch of (yhat - y)^2; ReLU'(0) = 0;
// Adam (Kingma & Ba) with bias correction.
//   k_mlp_fwd   : one thread per sample; keeps z1, z2 (pre-activations) for
//                 the backward pass.
//   k_mlp_delta : one thread per sample; the output error and the hidden
//                 deltas d2, d1.
//   k_mlp_grad  : one thread per parameter, summing its gradient over the
//                 batch in sample order (deterministic), and the loss.
//   k_mlp_adam  : one thread per parameter.
#include "sg_mlp.h"

namespace sgk {
namespace {

constexpr int H = kMlpHidden;

__device__ __forceinline__ const float* w1(const float* P) { return P; }

__global__ void __launch_bounds__(128) k_mlp_fwd(const float* __restrict__ P, int d_in,
                                                 const float* __restrict__ X, int B, float* z1,
                                                 float* z2, float* yhat) {
  extern __shared__ float sp[];
  const int np = mlp_nparams(d_in);
  for (int i = threadIdx.x; i < np; i += blockDim.x) sp[i] = P[i];
  __syncthreads();
  const float* W1 = sp;
  const float* b1 = W1 + H * d_in;
  const float* W2 = b1 + H;
  const float* b2 = W2 + H * H;
  const float* W3 = b2 + H;
  const float b3 = W3[H];
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float* x = X + (size_t)b * d_in;
  float h1[H];
  for (int j = 0; j < H; ++j) {
    float a = b1[j];
    for (int k = 0; k < d_in; ++k) a = fmaf(W1[j * d_in + k], x[k], a);
    if (z1) z1[(size_t)b * H + j] = a;
    h1[j] = a > 0.0f ? a : 0.0f;
  }
  float o = b3;
  for (int j = 0; j < H; ++j) {
    float a = b2[j];
#pragma unroll 8
    for (int k = 0; k < H; ++k) a = fmaf(W2[j * H + k], h1[k], a);
    if (z2) z2[(size_t)b * H + j] = a;
    o = fmaf(W3[j], a > 0.0f ? a : 0.0f, o);
  }
  yhat[b] = o;
}

// per sample: e = 2 (yhat - y) / B, d2 = relu'(z2) e W3, d1 = relu'(z1) W2^T d2
__global__ void __launch_bounds__(128) k_mlp_delta(const float* __restrict__ P, int d_in,
                                                   const float* __restrict__ y,
                                                   const float* __restrict__ yhat, int B,
                                                   const float* __restrict__ z1,
                                                   const float* __restrict__ z2, float* e,
                                                   float* d1, float* d2) {
  extern __shared__ float sp[];
  const int np = mlp_nparams(d_in);
  for (int i = threadIdx.x; i < np; i += blockDim.x) sp[i] = P[i];
  __syncthreads();
  const float* W2 = sp + H * d_in + H;
  const float* W3 = W2 + H * H + H;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float eb = 2.0f * (yhat[b] - y[b]) / (float)B;
  e[b] = eb;
  float dd2[H];
  for (int j = 0; j < H; ++j) {
    dd2[j] = z2[(size_t)b * H + j] > 0.0f ? eb * W3[j] : 0.0f;
    d2[(size_t)b * H + j] = dd2[j];
  }
  for (int k = 0; k < H; ++k) {
    float a = 0.0f;
    for (int j = 0; j < H; ++j) a = fmaf(W2[j * H + k], dd2[j], a);
    d1[(size_t)b * H + k] = z1[(size_t)b * H + k] > 0.0f ? a : 0.0f;
  }
}

// one thread per parameter: gradient summed over the batch in sample order
__global__ void __launch_bounds__(256) k_mlp_grad(int d_in, const float* __restrict__ X, int B,
                                                  const float* __restrict__ z1,
                                                  const float* __restrict__ z2,
                                                  const float* __restrict__ e,
                                                  const float* __restrict__ d1,
                                                  const float* __restrict__ d2, float* G) {
  const int np = mlp_nparams(d_in);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const int oW1 = 0, ob1 = H * d_in, oW2 = ob1 + H, ob2 = oW2 + H * H, oW3 = ob2 + H, ob3 = oW3 + H;
  float g = 0.0f;
  if (i < ob1) {                       // W1[j][k]: sum_b d1[b][j] x[b][k]
    const int j = i / d_in, k = i % d_in;
    for (int b = 0; b < B; ++b) g = fmaf(d1[(size_t)b * H + j], X[(size_t)b * d_in + k], g);
  } else if (i < oW2) {                // b1[j]
    const int j = i - ob1;
    for (int b = 0; b < B; ++b) g += d1[(size_t)b * H + j];
  } else if (i < ob2) {                // W2[j][k]: sum_b d2[b][j] relu(z1[b][k])
    const int j = (i - oW2) / H, k = (i - oW2) % H;
    for (int b = 0; b < B; ++b) {
      const float h = z1[(size_t)b * H + k];
      g = fmaf(d2[(size_t)b * H + j], h > 0.0f ? h : 0.0f, g);
    }
  } else if (i < oW3) {                // b2[j]
    const int j = i - ob2;
    for (int b = 0; b < B; ++b) g += d2[(size_t)b * H + j];
  } else if (i < ob3) {                // W3[k]: sum_b e[b] relu(z2[b][k])
    const int k = i - oW3;
    for (int b = 0; b < B; ++b) {
      const float h = z2[(size_t)b * H + k];
      g = fmaf(e[b], h > 0.0f ? h : 0.0f, g);
    }
  } else {                             // b3
    for (int b = 0; b < B; ++b) g += e[b];
  }
  G[i] = g;
}

__global__ void k_mlp_loss(const float* __restrict__ y, const float* __restrict__ yhat, int B,
                           float* loss) {
  // one block, fixed order: per-thread strided partials, then a tree
  __shared__ double sh[256];
  double s = 0.0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const double d = (double)yhat[b] - (double)y[b];
    s += d * d;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = (float)(sh[0] / (double)B);
}

__global__ void k_mlp_adam(float* P, const float* __restrict__ G, float* m, float* v, int np,
                           float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const float g = G[i];
  const float mi = b1 * m[i] + (1.0f - b1) * g;
  const float vi = b2 * v[i] + (1.0f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

size_t mlp_work_bytes(int B) {
  return (size_t)B * (4 * H + 2) * sizeof(float) + 256;
}

cudaError_t launch_mlp_forward(const float* P, int d_in, const float* X, int B, float* yhat,
                               cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const size_t sm = (size_t)mlp_nparams(d_in) * sizeof(float);
  k_mlp_fwd<<<(B + 127) / 128, 128, sm, s>>>(P, d_in, X, B, nullptr, nullptr, yhat);
  return cudaGetLastError();
}

cudaError_t launch_mlp_loss_grad(const float* P, int d_in, const float* X, const float* y, int B,
                                 float* G, float* loss, void* work, cudaStream_t s) {
  if (B <= 0) return cudaErrorInvalidValue;
  float* z1 = static_cast<float*>(work);
  float* z2 = z1 + (size_t)B * H;
  float* d1 = z2 + (size_t)B * H;
  float* d2 = d1 + (size_t)B * H;
  float* yhat = d2 + (size_t)B * H;
  float* e = yhat + B;
  const size_t sm = (size_t)mlp_nparams(d_in) * sizeof(float);
  const int np = mlp_nparams(d_in);
  k_mlp_fwd<<<(B + 127) / 128, 128, sm, s>>>(P, d_in, X, B, z1, z2, yhat);
  k_mlp_delta<<<(B + 127) / 128, 128, sm, s>>>(P, d_in, y, yhat, B, z1, z2, e, d1, d2);
  k_mlp_grad<<<(np + 255) / 256, 256, 0, s>>>(d_in, X, B, z1, z2, e, d1, d2, G);
  if (loss) k_mlp_loss<<<1, 256, 0, s>>>(y, yhat, B, loss);
  return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* P, const float* G, float* m, float* v, int np, long long t,
                            float lr, float b1, float b2, float eps, cudaStream_t s) {
  const float c1 = 1.0f - powf(b1, (float)t);
  const float c2 = 1.0f - powf(b2, (float)t);
  k_mlp_adam<<<(np + 255) / 256, 256, 0, s>>>(P, G, m, v, np, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace sgk
