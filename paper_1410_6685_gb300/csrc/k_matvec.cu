// k_matvec.cu -- matrix `transpose` and the matrix-vector products
// `right_multiply` (y = A x) and `left_multiply` (y = x^T A) of Sec. 3.4 and
// Listing 1, binary32, row-major (sm_103a).  All three are bound by HBM.
//
//   k_transpose : 64 x 64 tiles staged in shared memory (one padding column
//                 against bank conflicts); 16-byte loads and stores when both
//                 extents are multiples of 4, else element by element.
//   k_matvec_cta: rows of 2048 or more aligned columns, one CTA per row,
//                 eight 16-byte loads in flight per thread, binary32 FMA per
//                 thread, a warp tree, the eight warp sums added in order.
//   k_matvec    : narrower or unaligned rows, one warp per row.
//   k_vecmat    : column strips of 1024 (4 columns per thread, eight rows'
//                 16-byte loads in flight), the rows split into row stripes; each CTA leaves one partial row per stripe,
//                 which k_vecmat_sum adds in a fixed order (deterministic).
#include "sg_linalg_kernels.h"

namespace sgk {
namespace {

constexpr int kT = 64;   // transpose tile

__global__ void __launch_bounds__(256) k_transpose(const float* __restrict__ A, int rows, int cols,
                                                   float* __restrict__ At, int vec) {
  __shared__ float t[kT][kT + 1];
  const int r0 = blockIdx.y * kT, c0 = blockIdx.x * kT;
  const int tid = threadIdx.x;
  if (vec) {
    // load: 16 float4 per tile row, 16 rows per step
    const int cq = (tid & 15) * 4, rr = tid >> 4;
#pragma unroll
    for (int k = 0; k < kT; k += 16) {
      const int r = r0 + rr + k, c = c0 + cq;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < rows && c < cols) v = __ldcs(reinterpret_cast<const float4*>(A + (size_t)r * cols + c));
      t[rr + k][cq] = v.x;
      t[rr + k][cq + 1] = v.y;
      t[rr + k][cq + 2] = v.z;
      t[rr + k][cq + 3] = v.w;
    }
    __syncthreads();
    // store: output row c (a tile column), 4 consecutive r per thread
#pragma unroll
    for (int k = 0; k < kT; k += 16) {
      const int cc = rr + k;
      const int c = c0 + cc, r = r0 + cq;
      if (c < cols && r < rows) {
        const float4 v = make_float4(t[cq][cc], t[cq + 1][cc], t[cq + 2][cc], t[cq + 3][cc]);
        __stcs(reinterpret_cast<float4*>(At + (size_t)c * rows + r), v);
      }
    }
  } else {
    const int cx = tid & 63, ry = tid >> 6;
    for (int k = 0; k < kT; k += 4) {
      const int r = r0 + ry + k, c = c0 + cx;
      t[ry + k][cx] = (r < rows && c < cols) ? A[(size_t)r * cols + c] : 0.0f;
    }
    __syncthreads();
    for (int k = 0; k < kT; k += 4) {
      const int cc = ry + k;
      const int c = c0 + cc, r = r0 + cx;
      if (c < cols && r < rows) At[(size_t)c * rows + r] = t[cx][cc];
    }
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// y[i] = sum_j A[i][j] x[j], one warp per row
__global__ void __launch_bounds__(256) k_matvec(const float* __restrict__ A, int rows, int cols,
                                                const float* __restrict__ x, float* __restrict__ y,
                                                int vec) {
  const int lane = threadIdx.x & 31;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long i = w0; i < rows; i += nw) {
    const float* a = A + i * (long long)cols;
    float acc0 = 0.0f, acc1 = 0.0f, acc2 = 0.0f, acc3 = 0.0f;
    if (vec) {
      const int nq = cols >> 2;
      const float4* a4 = reinterpret_cast<const float4*>(a);
      const float4* x4 = reinterpret_cast<const float4*>(x);
      int q = lane;
      for (; q + 96 < nq; q += 128) {
        float4 av[4], xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          av[u] = __ldcs(a4 + q + 32 * u);
          xv[u] = __ldg(x4 + q + 32 * u);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          acc0 = fmaf(av[u].x, xv[u].x, acc0);
          acc1 = fmaf(av[u].y, xv[u].y, acc1);
          acc2 = fmaf(av[u].z, xv[u].z, acc2);
          acc3 = fmaf(av[u].w, xv[u].w, acc3);
        }
      }
      for (; q < nq; q += 32) {
        const float4 av = __ldcs(a4 + q), xv = __ldg(x4 + q);
        acc0 = fmaf(av.x, xv.x, acc0);
        acc1 = fmaf(av.y, xv.y, acc1);
        acc2 = fmaf(av.z, xv.z, acc2);
        acc3 = fmaf(av.w, xv.w, acc3);
      }
    } else {
      for (int j = lane; j < cols; j += 32) acc0 = fmaf(__ldcs(a + j), __ldg(x + j), acc0);
    }
    const float s = warp_sum((acc0 + acc1) + (acc2 + acc3));
    if (lane == 0) y[i] = s;
  }
}

// y[i] = sum_j A[i][j] x[j] for wide rows, one CTA per row: thread t takes
// the quads t, t + 256, t + 512, ... (the CTA's eight warps read 4 KB of the
// row at once, eight such loads in flight per thread), a warp tree, then
// thread 0 adds the eight warp sums in order.  Two slots of warp sums let one
// barrier per row suffice.
__global__ void __launch_bounds__(256) k_matvec_cta(const float* __restrict__ A, int rows,
                                                    int cols, const float* __restrict__ x,
                                                    float* __restrict__ y) {
  __shared__ float s_part[2][8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nq = cols >> 2;
  const float4* x4 = reinterpret_cast<const float4*>(x);
  int slot = 0;
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const float4* a4 = reinterpret_cast<const float4*>(A + r * (long long)cols);
    float acc0 = 0.0f, acc1 = 0.0f, acc2 = 0.0f, acc3 = 0.0f;
    int q = threadIdx.x;
    for (; q + 7 * 256 < nq; q += 8 * 256) {
      float4 av[8], xv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        av[u] = __ldcs(a4 + q + 256 * u);
        xv[u] = __ldg(x4 + q + 256 * u);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        acc0 = fmaf(av[u].x, xv[u].x, acc0);
        acc1 = fmaf(av[u].y, xv[u].y, acc1);
        acc2 = fmaf(av[u].z, xv[u].z, acc2);
        acc3 = fmaf(av[u].w, xv[u].w, acc3);
      }
    }
    for (; q < nq; q += 256) {
      const float4 av = __ldcs(a4 + q), xv = __ldg(x4 + q);
      acc0 = fmaf(av.x, xv.x, acc0);
      acc1 = fmaf(av.y, xv.y, acc1);
      acc2 = fmaf(av.z, xv.z, acc2);
      acc3 = fmaf(av.w, xv.w, acc3);
    }
    const float sum = warp_sum((acc0 + acc1) + (acc2 + acc3));
    if (lane == 0) s_part[slot][w] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = s_part[slot][0];
#pragma unroll
      for (int k = 1; k < 8; ++k) t += s_part[slot][k];
      y[r] = t;
    }
    slot ^= 1;
  }
}

// partial[s][j] = sum over rows i of stripe s of x[i] A[i][j]
__global__ void __launch_bounds__(256) k_vecmat(const float* __restrict__ x,
                                                const float* __restrict__ A, int rows, int cols,
                                                int rows_per_stripe, float* __restrict__ partial,
                                                int vec) {
  const int s = blockIdx.y;
  const int i0 = s * rows_per_stripe;
  const int i1 = min(rows, i0 + rows_per_stripe);
  const int c = blockIdx.x * 1024 + threadIdx.x * 4;
  if (c >= cols) return;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (vec) {
    int i = i0;
    for (; i + 7 < i1; i += 8) {
      float4 av[8];
      float xv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        av[u] = __ldcs(reinterpret_cast<const float4*>(A + (size_t)(i + u) * cols + c));
        xv[u] = __ldg(x + i + u);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        acc.x = fmaf(xv[u], av[u].x, acc.x);
        acc.y = fmaf(xv[u], av[u].y, acc.y);
        acc.z = fmaf(xv[u], av[u].z, acc.z);
        acc.w = fmaf(xv[u], av[u].w, acc.w);
      }
    }
    for (; i < i1; ++i) {
      const float4 av = __ldcs(reinterpret_cast<const float4*>(A + (size_t)i * cols + c));
      const float xv = __ldg(x + i);
      acc.x = fmaf(xv, av.x, acc.x);
      acc.y = fmaf(xv, av.y, acc.y);
      acc.z = fmaf(xv, av.z, acc.z);
      acc.w = fmaf(xv, av.w, acc.w);
    }
    *reinterpret_cast<float4*>(partial + (size_t)s * cols + c) = acc;
  } else {
    float a4[4] = {0.f, 0.f, 0.f, 0.f};
    for (int i = i0; i < i1; ++i) {
      const float xv = __ldg(x + i);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (c + q < cols) a4[q] = fmaf(xv, __ldcs(A + (size_t)i * cols + c + q), a4[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (c + q < cols) partial[(size_t)s * cols + c + q] = a4[q];
  }
}

// y[j] = sum over stripes of partial[s][j]: 32 columns per CTA, its eight
// warps take the stripes k = w, w + 8, ... and thread row 0 adds the eight
// sums in order (a fixed order, so the result is deterministic)
__global__ void __launch_bounds__(256) k_vecmat_sum(const float* __restrict__ partial,
                                                    int stripes, int cols,
                                                    float* __restrict__ y) {
  __shared__ float sp[8][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + tx;
  float acc = 0.0f;
  if (j < cols) {
#pragma unroll 4
    for (int k = ty; k < stripes; k += 8) acc += __ldcg(partial + (size_t)k * cols + j);
  }
  sp[ty][tx] = acc;
  __syncthreads();
  if (ty == 0 && j < cols) {
    float t = sp[0][tx];
#pragma unroll
    for (int k = 1; k < 8; ++k) t += sp[k][tx];
    y[j] = t;
  }
}

int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms <= 0)
      sms = 1;
  }
  return sms;
}

// row stripes of the left product: enough CTAs for about 4 per SM, at least
// 16 rows per stripe
int vecmat_stripes(int rows, int cols) {
  const int colblocks = (cols + 1023) / 1024;
  int s = (4 * sm_count() + colblocks - 1) / colblocks;
  s = std::max(1, std::min(s, (rows + 15) / 16));
  return s;
}

}  // namespace

cudaError_t launch_transpose(const float* A, int rows, int cols, float* At, cudaStream_t s,
                             Prof* prof) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  const int vec = (rows % 4 == 0 && cols % 4 == 0 && ((uintptr_t)A % 16) == 0 &&
                   ((uintptr_t)At % 16) == 0)
                      ? 1
                      : 0;
  const dim3 grid((cols + kT - 1) / kT, (rows + kT - 1) / kT);
  prof_begin(prof, "transpose", s);
  k_transpose<<<grid, 256, 0, s>>>(A, rows, cols, At, vec);
  prof_end(prof, s);
  return cudaGetLastError();
}

cudaError_t launch_matvec(const float* A, int rows, int cols, const float* x, float* y,
                          cudaStream_t s, Prof* prof) {
  if (rows <= 0) return cudaSuccess;
  if (cols <= 0) return cudaMemsetAsync(y, 0, (size_t)rows * 4, s);
  const int vec = (cols % 4 == 0 && ((uintptr_t)A % 16) == 0 && ((uintptr_t)x % 16) == 0) ? 1 : 0;
  prof_begin(prof, "matvec", s);
  if (vec && cols >= 2048) {
    static int occ = 0;
    if (!occ && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_matvec_cta, 256, 0) !=
                    cudaSuccess)
      occ = 1;
    const long long blocks = std::min<long long>(rows, (long long)sm_count() * std::max(occ, 1));
    k_matvec_cta<<<(int)blocks, 256, 0, s>>>(A, rows, cols, x, y);
  } else {
    const long long blocks = std::min<long long>((rows + 7) / 8, (long long)sm_count() * 8);
    k_matvec<<<(int)blocks, 256, 0, s>>>(A, rows, cols, x, y, vec);
  }
  prof_end(prof, s);
  return cudaGetLastError();
}

size_t vecmat_scratch_bytes(int rows, int cols) {
  if (rows <= 0 || cols <= 0) return 0;
  return (size_t)vecmat_stripes(rows, cols) * cols * sizeof(float);
}

cudaError_t launch_vecmat(const float* x, const float* A, int rows, int cols, float* y,
                          void* scratch, cudaStream_t s, Prof* prof) {
  if (cols <= 0) return cudaSuccess;
  if (rows <= 0) return cudaMemsetAsync(y, 0, (size_t)cols * 4, s);
  const int stripes = vecmat_stripes(rows, cols);
  const int rps = (rows + stripes - 1) / stripes;
  const int vec = (cols % 4 == 0 && ((uintptr_t)A % 16) == 0 && ((uintptr_t)scratch % 16) == 0)
                      ? 1
                      : 0;
  float* partial = static_cast<float*>(scratch);
  prof_begin(prof, "vecmat", s);
  k_vecmat<<<dim3((cols + 1023) / 1024, stripes), 256, 0, s>>>(x, A, rows, cols, rps, partial, vec);
  k_vecmat_sum<<<(cols + 31) / 32, 256, 0, s>>>(partial, stripes, cols, y);
  prof_end(prof, s);
  return cudaGetLastError();
}

}  // namespace sgk
