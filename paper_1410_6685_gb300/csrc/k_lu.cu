// k_lu.cu -- Gaussian elimination (Sec. 5, Listing 6 read as elimination with
// partial pivoting) and the solve with iterative refinement (sm_103a).
//
// Right-looking blocked LU, panels of 32 columns:
//   k_lu_panel   : a cluster of 8 CTAs holds the panel (rows k..n-1) in their
//                  shared memories and eliminates it column by column.  Each
//                  column costs one hardware cluster barrier: every CTA
//                  publishes its best pivot candidate (largest |a|, then the
//                  lowest current row position) into every CTA's shared
//                  memory, all pick the same winner, read the pivot row from
//                  its owner over distributed shared memory, and update their
//                  own rows while finding the next column's candidate.  Row
//                  interchanges are tracked as a replicated position table
//                  and applied when the panel is written back, so the result
//                  equals the row-swapping textbook algorithm.
//   k_lu_laswp   : the panel's interchanges on the other columns.
//   k_lu_trsm    : U12 = L11^-1 A12 (unit lower, 32x32).
//   trailing update A22 -= L21 U12 : the tensor-core product (bf16/fp16
//                  operands, binary32 accumulate) or the binary32 SIMT form.
// Solve: pivots on the right-hand side, then forward / backward substitution
// by blocks of 32 rows in one launch each: CTAs take row blocks in order
// (ticket) and wait, with a bounded spin, for the blocks they depend on.
// Refinement: residual r = b - A x in binary64 from the binary32 A, and the
// update x += d with the norms the stopping test needs.
#include <cooperative_groups.h>

#include "sg_lu.h"
#include "sg_linalg_kernels.h"

namespace cg = cooperative_groups;

namespace sgk {
namespace {

constexpr int kPB = 32;       // panel width
constexpr int kPC = 8;        // CTAs per cluster
constexpr int kPT = 256;      // threads per CTA
constexpr int kStride = kPB + 1;
constexpr unsigned kSpin = 1u << 24;

__device__ __forceinline__ unsigned long long key_of(float v, int pos) {
  // larger |v| wins, then the lower position; NaN sorts above everything
  return ((unsigned long long)__float_as_uint(fabsf(v)) << 32) | (0xFFFFFFFFu - (unsigned)pos);
}

__device__ __forceinline__ unsigned long long block_max(unsigned long long v,
                                                        unsigned long long* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < kPT / 32 ? sh[lane] : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
      v = u > v ? u : v;
    }
    if (lane == 0) sh[0] = v;
  }
  __syncthreads();
  return sh[0];
}

// smem: slab[rs][33] floats, pos[m] ints, inv[m] ints, cand[2][8] u64,
// prow[32] floats, red[8] u64
__global__ void __cluster_dims__(kPC, 1, 1) __launch_bounds__(kPT)
    k_lu_panel(float* __restrict__ LU, int n, int k, int jb, int* __restrict__ piv,
               int* __restrict__ info) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int m = n - k;
  const int rs = (m + kPC - 1) / kPC;
  const int r0 = rank * rs;
  const int r1 = min(m, r0 + rs);
  float* slab = reinterpret_cast<float*>(smem);
  int* pos = reinterpret_cast<int*>(slab + (size_t)rs * kStride);
  int* inv = pos + m;
  unsigned long long* cand = reinterpret_cast<unsigned long long*>(
      (reinterpret_cast<uintptr_t>(inv + m) + 15) & ~(uintptr_t)15);
  float* prow = reinterpret_cast<float*>(cand + 2 * kPC);
  unsigned long long* red = reinterpret_cast<unsigned long long*>(prow + kPB);
  const int tid = threadIdx.x;

  // load my rows of the panel, initialise the position tables
  for (int t = tid; t < (r1 - r0) * kPB; t += kPT) {
    const int r = t / kPB, c = t % kPB;
    slab[r * kStride + c] = c < jb ? LU[(size_t)(k + r0 + r) * n + k + c] : 0.0f;
  }
  for (int i = tid; i < m; i += kPT) {
    pos[i] = i;
    inv[i] = i;
  }
  __syncthreads();
  // first column's candidate
  unsigned long long best = 0ull;
  for (int r = r0 + tid; r < r1; r += kPT) {
    const unsigned long long kk = key_of(slab[(r - r0) * kStride], r);
    best = kk > best ? kk : best;
  }
  best = block_max(best, red);
  int my_info = 0;
  for (int j = 0; j < jb; ++j) {
    const int par = j & 1;
    if (tid < kPC) {
      unsigned long long* dst = cluster.map_shared_rank(&cand[par * kPC + rank], tid);
      *dst = best;
    }
    cluster.sync();
    unsigned long long g = 0ull;
#pragma unroll
    for (int q = 0; q < kPC; ++q) g = cand[par * kPC + q] > g ? cand[par * kPC + q] : g;
    const int p = (int)(0xFFFFFFFFu - (unsigned)(g & 0xFFFFFFFFull));   // position
    const int gp = pos[p];                                               // physical row
    const int owner = gp / rs;
    // read the pivot row (columns j..jb-1) from its owner's shared memory
    if (tid < kPB) {
      const float* src = cluster.map_shared_rank(slab, owner);
      prow[tid] = (tid >= j && tid < jb) ? src[(gp - owner * rs) * kStride + tid] : 0.0f;
    }
    // replicated interchange of positions j and p
    __syncthreads();
    if (tid == 0) {
      const int gj = pos[j];
      pos[j] = gp;
      pos[p] = gj;
      inv[gp] = j;
      inv[gj] = p;
    }
    __syncthreads();
    const float d = prow[j];
    const bool zero = d == 0.0f;
    if (zero && my_info == 0) my_info = k + j + 1;
    // eliminate below the pivot; find the next column's candidate
    best = 0ull;
    for (int r = r0 + tid; r < r1; r += kPT) {
      const int lp = inv[r];
      if (lp <= j) continue;
      float* row = slab + (r - r0) * kStride;
      if (!zero) {
        const float l = row[j] / d;
        row[j] = l;
        for (int c = j + 1; c < jb; ++c) row[c] = fmaf(-l, prow[c], row[c]);
      }
      if (j + 1 < jb) {
        const unsigned long long kk = key_of(row[j + 1], lp);
        best = kk > best ? kk : best;
      }
    }
    if (tid == 0 && rank == 0) piv[k + j] = k + p;
    best = block_max(best, red);
  }
  cluster.sync();   // no CTA reads another's shared memory after this
  // write the panel back in its final row order
  for (int t = tid; t < (r1 - r0) * kPB; t += kPT) {
    const int r = t / kPB, c = t % kPB;
    if (c < jb) LU[(size_t)(k + inv[r0 + r]) * n + k + c] = slab[r * kStride + c];
  }
  if (tid == 0 && rank == 0 && my_info) atomicCAS(info, 0, my_info);
  cluster.sync();
}

// interchanges piv[k..k+jb) applied in order to columns [c0, c1)
__global__ void k_lu_laswp(float* LU, int n, int k, int jb, const int* __restrict__ piv, int c0,
                           int c1) {
  const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= c1) return;
  for (int j = 0; j < jb; ++j) {
    const int p = piv[k + j];
    if (p != k + j) {
      float* a = LU + (size_t)(k + j) * n + c;
      float* b = LU + (size_t)p * n + c;
      const float t = *a;
      *a = *b;
      *b = t;
    }
  }
}

// U12 = L11^-1 A12: one thread per column of A12
__global__ void k_lu_trsm(float* LU, int n, int k, int jb) {
  __shared__ float L[kPB][kPB + 1];
  for (int t = threadIdx.x; t < jb * jb; t += blockDim.x)
    L[t / jb][t % jb] = LU[(size_t)(k + t / jb) * n + k + t % jb];
  __syncthreads();
  const int c = k + jb + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  float x[kPB];
#pragma unroll
  for (int i = 0; i < kPB; ++i) x[i] = i < jb ? LU[(size_t)(k + i) * n + c] : 0.0f;
#pragma unroll
  for (int i = 1; i < kPB; ++i) {
    if (i >= jb) break;
    float s = x[i];
#pragma unroll
    for (int t = 0; t < i; ++t) s = fmaf(-L[i][t], x[t], s);
    x[i] = s;
  }
#pragma unroll
  for (int i = 1; i < kPB; ++i)
    if (i < jb) LU[(size_t)(k + i) * n + c] = x[i];
}

// ---------------------------------------------------------------------------
// solve

// y = P rhs (binary64 in, binary32 out): the row interchanges in order
__global__ void k_apply_piv(const double* __restrict__ rhs, float* y, int n,
                            const int* __restrict__ piv) {
  // one CTA: copy, then the interchanges in order by one thread
  for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = (float)rhs[i];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int j = 0; j < n; ++j) {
      const int p = piv[j];
      if (p != j) {
        const float t = y[j];
        y[j] = y[p];
        y[p] = t;
      }
    }
}

// Triangular solve by 32-row blocks.  LOWER: unit lower L, blocks in
// increasing order; else upper U with its diagonal, blocks in decreasing
// order.  Block b waits for the flags of the blocks it depends on.
template <bool LOWER>
__global__ void __launch_bounds__(256) k_trsv(const float* __restrict__ LU, int n, float* y,
                                              unsigned* flags, unsigned epoch, unsigned* ticket,
                                              int* err) {
  __shared__ unsigned s_b;
  __shared__ float part[8][32];
  __shared__ float yb[32];
  const int nb = (n + 31) / 32;
  if (threadIdx.x == 0) s_b = atomicAdd(ticket, 1u);
  __syncthreads();
  const int t = (int)s_b;
  const int b = LOWER ? t : nb - 1 - t;
  const int row0 = b * 32;
  const int rows = min(32, n - row0);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  // contributions of the finished blocks, in dependency order
  for (int q = 0; q < nb; ++q) {
    const int c = LOWER ? q : nb - 1 - q;
    if (c == b) break;
    if (threadIdx.x == 0) {
      unsigned spins = 0;
      while (atomicAdd(&flags[c], 0u) != epoch) {
        if (++spins > kSpin) {
          atomicExch(err, 1);
          break;
        }
        if (spins > 64) __nanosleep(100);
      }
      __threadfence();
    }
    __syncthreads();
    const int col = c * 32 + lane;
    const float yc = col < n ? __ldcg(&y[col]) : 0.0f;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int row = row0 + w * 4 + r;
      if (row < n && col < n) acc[r] = fmaf(LU[(size_t)row * n + col], yc, acc[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    float v = acc[r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) part[w][r] = v;
  }
  __syncthreads();
  // the diagonal block, by one warp
  if (w == 0) {
    float v = 0.0f;
    if (lane < rows) v = __ldcg(&y[row0 + lane]) - part[lane >> 2][lane & 3];
    if (LOWER) {
      for (int i = 0; i < rows; ++i) {
        const float yi = __shfl_sync(0xffffffffu, v, i);
        if (lane > i && lane < rows) v = fmaf(-LU[(size_t)(row0 + lane) * n + row0 + i], yi, v);
      }
    } else {
      for (int i = rows - 1; i >= 0; --i) {
        float vi = __shfl_sync(0xffffffffu, v, i);
        const float dii = LU[(size_t)(row0 + i) * n + row0 + i];
        vi = vi / dii;
        if (lane == i) v = vi;
        if (lane < i) v = fmaf(-LU[(size_t)(row0 + lane) * n + row0 + i], vi, v);
      }
    }
    if (lane < rows) yb[lane] = v;
    __syncwarp();
    if (lane < rows) y[row0 + lane] = yb[lane];
    __threadfence();
    __syncwarp();
    if (lane == 0) atomicExch(&flags[b], epoch);
  }
}

// r = b - A x (binary64), one warp per row; also |A|_inf rows when asked
__global__ void __launch_bounds__(256) k_residual(const float* __restrict__ A, int n,
                                                  const double* __restrict__ b,
                                                  const double* __restrict__ x, double* r,
                                                  double* norms, double thresh,
                                                  unsigned long long* viol) {
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  double rmax = 0.0;
  for (long long i = warp; i < n; i += nw) {
    const float* row = A + i * (long long)n;
    double s = 0.0;
    for (int j = lane; j < n; j += 32) s = fma((double)__ldcs(row + j), x[j], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const double ri = b[i] - s;
    if (lane == 0) {
      r[i] = ri;
      if (viol && !(fabs(ri) <= thresh)) atomicMax(viol, ~(unsigned long long)i);
    }
    rmax = fmax(rmax, fabs(ri));
  }
  if (lane == 0) atomicMax(reinterpret_cast<unsigned long long*>(&norms[0]),
                           (unsigned long long)__double_as_longlong(rmax));
}

// |A|_inf (binary64) once per solve
__global__ void __launch_bounds__(256) k_anorm(const float* __restrict__ A, int n, double* norms) {
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  double mx = 0.0;
  for (long long i = warp; i < n; i += nw) {
    const float* row = A + i * (long long)n;
    double s = 0.0;
    for (int j = lane; j < n; j += 32) s += fabs((double)row[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    mx = fmax(mx, s);
  }
  if (lane == 0) atomicMax(reinterpret_cast<unsigned long long*>(&norms[3]),
                           (unsigned long long)__double_as_longlong(mx));
}

// x += d (or x = d when init), with max|d|, max|x|, max|b| for the tests
__global__ void k_update(double* x, const float* __restrict__ d, const double* __restrict__ b,
                         int n, int init, double* norms) {
  double dm = 0.0, xm = 0.0, bm = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double di = (double)d[i];
    const double xi = init ? di : x[i] + di;
    x[i] = xi;
    dm = fmax(dm, fabs(di));
    xm = fmax(xm, fabs(xi));
    bm = fmax(bm, fabs(b[i]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
    xm = fmax(xm, __shfl_xor_sync(0xffffffffu, xm, o));
    bm = fmax(bm, __shfl_xor_sync(0xffffffffu, bm, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(reinterpret_cast<unsigned long long*>(&norms[1]),
              (unsigned long long)__double_as_longlong(dm));
    atomicMax(reinterpret_cast<unsigned long long*>(&norms[2]),
              (unsigned long long)__double_as_longlong(xm));
    atomicMax(reinterpret_cast<unsigned long long*>(&norms[4]),
              (unsigned long long)__double_as_longlong(bm));
  }
}

__global__ void k_residual_to_f32(const double* __restrict__ r, float* y, int n,
                                  const int* __restrict__ piv) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = (float)r[i];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int j = 0; j < n; ++j) {
      const int p = piv[j];
      if (p != j) {
        const float t = y[j];
        y[j] = y[p];
        y[p] = t;
      }
    }
}

size_t panel_smem(int n, int k) {
  const int m = n - k;
  const int rs = (m + kPC - 1) / kPC;
  return (size_t)rs * kStride * 4 + (size_t)m * 8 + 16 + 2 * kPC * 8 + kPB * 4 + 8 * 8 + 64;
}

}  // namespace

size_t lu_panel_max_smem(int n) { return panel_smem(n, 0); }

cudaError_t launch_lu_panel(float* LU, int n, int k, int jb, int* piv, int* info, cudaStream_t s,
                            Prof* prof) {
  const size_t sm = panel_smem(n, k);
  static size_t attr = 0;
  if (sm > attr) {
    cudaError_t e = cudaFuncSetAttribute(k_lu_panel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)panel_smem(n, 0));
    if (e != cudaSuccess) return e;
    attr = panel_smem(n, 0);
  }
  prof_begin(prof, "lu_panel", s);
  k_lu_panel<<<kPC, kPT, sm, s>>>(LU, n, k, jb, piv, info);
  prof_end(prof, s);
  return cudaGetLastError();
}

cudaError_t launch_lu_laswp_trsm(float* LU, int n, int k, int jb, const int* piv, cudaStream_t s,
                                 Prof* prof) {
  prof_begin(prof, "lu_laswp_trsm", s);
  if (k > 0) k_lu_laswp<<<(k + 255) / 256, 256, 0, s>>>(LU, n, k, jb, piv, 0, k);
  const int rest = n - k - jb;
  if (rest > 0) {
    k_lu_laswp<<<(rest + 255) / 256, 256, 0, s>>>(LU, n, k, jb, piv, k + jb, n);
    k_lu_trsm<<<(rest + 127) / 128, 128, 0, s>>>(LU, n, k, jb);
  }
  prof_end(prof, s);
  return cudaGetLastError();
}

cudaError_t launch_lu_solve(const float* LU, int n, const int* piv, const double* rhs,
                            bool rhs_is_residual, float* y, unsigned* flags, unsigned epoch,
                            unsigned* tickets, int* err, cudaStream_t s, Prof* prof) {
  const int nb = (n + 31) / 32;
  prof_begin(prof, "lu_trsv", s);
  if (rhs_is_residual)
    k_residual_to_f32<<<1, 1024, 0, s>>>(rhs, y, n, piv);
  else
    k_apply_piv<<<1, 1024, 0, s>>>(rhs, y, n, piv);
  cudaMemsetAsync(tickets, 0, 2 * sizeof(unsigned), s);
  k_trsv<true><<<nb, 256, 0, s>>>(LU, n, y, flags, epoch, tickets, err);
  k_trsv<false><<<nb, 256, 0, s>>>(LU, n, y, flags + nb, epoch, tickets + 1, err);
  prof_end(prof, s);
  return cudaGetLastError();
}

cudaError_t launch_residual(const float* A, int n, const double* b, const double* x, double* r,
                            double* norms, double thresh, unsigned long long* viol,
                            cudaStream_t s, Prof* prof) {
  prof_begin(prof, "residual_f64", s);
  k_residual<<<(n + 7) / 8, 256, 0, s>>>(A, n, b, x, r, norms, thresh, viol);
  prof_end(prof, s);
  return cudaGetLastError();
}

cudaError_t launch_anorm(const float* A, int n, double* norms, cudaStream_t s) {
  k_anorm<<<(n + 7) / 8, 256, 0, s>>>(A, n, norms);
  return cudaGetLastError();
}

cudaError_t launch_update(double* x, const float* d, const double* b, int n, bool init,
                          double* norms, cudaStream_t s) {
  k_update<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, s>>>(x, d, b, n,
                                                                            init ? 1 : 0, norms);
  return cudaGetLastError();
}

}  // namespace sgk
