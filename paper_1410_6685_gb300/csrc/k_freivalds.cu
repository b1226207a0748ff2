// k_freivalds.cu -- the postcondition of matrix `multiply` (Sec. 3.4):
// Freivalds' randomized check that C = A B, evaluated on the GPU.
//
// For each of `nvec` Rademacher vectors r (entries +-1 from the SplitMix64
// stream `seed`, draw t = v*N + j + 1 for entry j of vector v):
//   z = A (B r),  w = C r,  and row i is violated when |z_i - w_i| > tau_i,
//   tau_i = c * u_eff * sqrt( sum_k a_ik^2 ((B r)_k^2 + s_k) ),  s_k = sum_j b_kj^2,
// a c-sigma bound on the rounding noise of a product whose operand rounding
// and accumulation have unit roundoff u_eff.  Three streaming passes, one
// column stripe per CTA (8 warps side by side along 8 rows), each lane holding its columns' vector entries in
// registers while the rows stream by (their loads issued together); partial
// sums per stripe are then added in a fixed order: r, then B (B r and
// |B_k|^2), then A and C together, then the per-row test.
#include <math.h>

#include "sg_frv.cuh"
#include "sg_linalg_kernels.h"

namespace sgk {
namespace {

using frv::ldv;
using frv::ldvec;
using frv::warp_sum_spread;

constexpr int kMaxVec = 4;

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// r4[j] = (r_0(j), r_1(j), r_2(j), r_3(j)); unused vectors are 0
__global__ void k_frv_r(float4* r4, int N, int nvec, unsigned long long seed) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < N;
       j += (long long)gridDim.x * blockDim.x) {
    float v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const unsigned long long t = (unsigned long long)q * N + j + 1;
      const unsigned long long z = mix64(seed + t * 0x9E3779B97F4A7C15ull);
      v[q] = q < nvec ? ((z >> 63) ? -1.0f : 1.0f) : 0.0f;
    }
    r4[j] = make_float4(v[0], v[1], v[2], v[3]);
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int kRows = 8;            // rows per CTA (their loads issued together)
constexpr int kWarps = 8;           // warps per CTA, side by side along a row
constexpr int kWB = 256;            // columns per warp in the B pass (8 per lane)
constexpr int kWAC = 128;           // columns per warp in the A/C pass (4 per lane)
constexpr int kSwB = kWarps * kWB;  // stripe width of a CTA, B pass
constexpr int kSwAC = kWarps * kWAC;

constexpr int kIters = 4;   // row groups of kRows per CTA (vectors loaded once)

// partials over column stripes of B:  pb[s][k] = (sum_j B[k][j] r_v[j] for v<4,
// sum_j B[k][j]^2), j in stripe s; the warps' shares are added in warp order
__global__ void __launch_bounds__(256, 2) k_frv_b(const float* __restrict__ B, int N,
                                                  const float4* __restrict__ r4, float* pb) {
  __shared__ float red[2][kWarps][kRows][5];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int stripe = blockIdx.x;
  const long long c0 = (long long)stripe * kSwB + w * kWB + lane * 8;
  const bool vec = (N % 4) == 0 && ((uintptr_t)B % 16) == 0;
  float4 r[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) r[e] = ldvec(r4, c0 + e, N);
  const int slot = (lane >> 2) & 7;
#pragma unroll 1
  for (int it = 0; it < kIters; ++it) {
    const long long row0 = ((long long)blockIdx.y * kIters + it) * kRows;
    if (row0 >= N) break;
    float4 b[kRows][2];
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
      const long long row = row0 + i;
      const float* rp = B + (row < N ? row : 0) * (long long)N;
      b[i][0] = row < N ? ldv(rp, c0, N, vec) : make_float4(0.f, 0.f, 0.f, 0.f);
      b[i][1] = row < N ? ldv(rp, c0 + 4, N, vec) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
      const float bv[8] = {b[i][0].x, b[i][0].y, b[i][0].z, b[i][0].w,
                           b[i][1].x, b[i][1].y, b[i][1].z, b[i][1].w};
      float o[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        o[0] = fmaf(bv[e], r[e].x, o[0]);
        o[1] = fmaf(bv[e], r[e].y, o[1]);
        o[2] = fmaf(bv[e], r[e].z, o[2]);
        o[3] = fmaf(bv[e], r[e].w, o[3]);
        o[4] = fmaf(bv[e], bv[e], o[4]);
      }
      const float v = warp_sum_spread<8>(o, lane);
      if ((lane & 3) == 0 && slot < 5) red[it & 1][w][i][slot] = v;
    }
    __syncthreads();
    if (threadIdx.x < kRows * 5) {
      const int i = threadIdx.x / 5, t = threadIdx.x % 5;
      const long long row = row0 + i;
      float acc = 0.0f;
#pragma unroll
      for (int q = 0; q < kWarps; ++q) acc += red[it & 1][q][i][t];
      if (row < N) pb[((long long)stripe * N + row) * 5 + t] = acc;
    }
  }
}

// br4[k] = sum over stripes (fixed order), t4[k] = br4[k]^2 + |B_k|^2
__global__ void k_frv_b_reduce(const float* __restrict__ pb, int N, int nstripes, float4* br4,
                               float4* t4) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= N) return;
  float o[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  for (int s = 0; s < nstripes; ++s) {
#pragma unroll
    for (int t = 0; t < 5; ++t) o[t] += pb[((long long)s * N + k) * 5 + t];
  }
  br4[k] = make_float4(o[0], o[1], o[2], o[3]);
  t4[k] = make_float4(fmaf(o[0], o[0], o[4]), fmaf(o[1], o[1], o[4]), fmaf(o[2], o[2], o[4]),
                      fmaf(o[3], o[3], o[4]));
}

// partials over column stripes of A and C: z = A br, q = (A.A) t, w = C r
__global__ void __launch_bounds__(256, 2) k_frv_ac(const float* __restrict__ A,
                                                   const float* __restrict__ C, int N,
                                                   const float4* __restrict__ r4,
                                                   const float4* __restrict__ br4,
                                                   const float4* __restrict__ t4, float* pac) {
  __shared__ float red[2][kWarps][kRows][12];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int stripe = blockIdx.x;
  const long long c0 = (long long)stripe * kSwAC + w * kWAC + lane * 4;
  const bool vec = (N % 4) == 0 && ((uintptr_t)A % 16) == 0 && ((uintptr_t)C % 16) == 0;
  float4 vb[4], vt[4], vr[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    vb[e] = ldvec(br4, c0 + e, N);
    vt[e] = ldvec(t4, c0 + e, N);
    vr[e] = ldvec(r4, c0 + e, N);
  }
  const int slot = (lane >> 1) & 15;
#pragma unroll 1
  for (int it = 0; it < kIters; ++it) {
    const long long row0 = ((long long)blockIdx.y * kIters + it) * kRows;
    if (row0 >= N) break;
    float4 av[kRows], cv[kRows];
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
      const long long row = row0 + i;
      const long long rr = row < N ? row : 0;
      av[i] = row < N ? ldv(A + rr * (long long)N, c0, N, vec) : make_float4(0.f, 0.f, 0.f, 0.f);
      cv[i] = row < N ? ldv(C + rr * (long long)N, c0, N, vec) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
      const float a[4] = {av[i].x, av[i].y, av[i].z, av[i].w};
      const float c[4] = {cv[i].x, cv[i].y, cv[i].z, cv[i].w};
      float o[16];
#pragma unroll
      for (int t = 0; t < 16; ++t) o[t] = 0.0f;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float a2 = a[e] * a[e];
        o[0] = fmaf(a[e], vb[e].x, o[0]); o[1] = fmaf(a[e], vb[e].y, o[1]);
        o[2] = fmaf(a[e], vb[e].z, o[2]); o[3] = fmaf(a[e], vb[e].w, o[3]);
        o[4] = fmaf(a2, vt[e].x, o[4]); o[5] = fmaf(a2, vt[e].y, o[5]);
        o[6] = fmaf(a2, vt[e].z, o[6]); o[7] = fmaf(a2, vt[e].w, o[7]);
        o[8] = fmaf(c[e], vr[e].x, o[8]); o[9] = fmaf(c[e], vr[e].y, o[9]);
        o[10] = fmaf(c[e], vr[e].z, o[10]); o[11] = fmaf(c[e], vr[e].w, o[11]);
      }
      const float v = warp_sum_spread<16>(o, lane);
      if ((lane & 1) == 0 && slot < 12) red[it & 1][w][i][slot] = v;
    }
    __syncthreads();
    if (threadIdx.x < kRows * 12) {
      const int i = threadIdx.x / 12, t = threadIdx.x % 12;
      const long long row = row0 + i;
      float acc = 0.0f;
#pragma unroll
      for (int q = 0; q < kWarps; ++q) acc += red[it & 1][q][i][t];
      if (row < N) pac[((long long)stripe * N + row) * 12 + t] = acc;
    }
  }
}

// per row: sum the partials (fixed order), compare |z - w| with tau
__global__ void k_frv_check(const float* __restrict__ pac, int N, int nstripes, int nvec,
                            float c, float u_eff, FreivaldsResult* res) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  float worst = 0.0f;
  bool bad = false;
  if (i < N) {
    float o[12];
#pragma unroll
    for (int t = 0; t < 12; ++t) o[t] = 0.0f;
    for (int s = 0; s < nstripes; ++s) {
      const float* p = pac + ((long long)s * N + i) * 12;
#pragma unroll
      for (int t = 0; t < 12; t += 4) {
        const float4 v = *reinterpret_cast<const float4*>(p + t);
        o[t] += v.x; o[t + 1] += v.y; o[t + 2] += v.z; o[t + 3] += v.w;
      }
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      if (v >= nvec) continue;
      const float tau = c * u_eff * sqrtf(o[4 + v]);
      const float gap = fabsf(o[v] - o[8 + v]);
      const float ratio = tau > 0.0f ? gap / tau : (gap > 0.0f ? INFINITY : 0.0f);
      worst = fmaxf(worst, ratio);
      bad |= !(gap <= tau);
    }
    if (bad) atomicMax(&res->viol_enc, ~(unsigned long long)i);
  }
#pragma unroll
  for (int o2 = 16; o2 > 0; o2 >>= 1) worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, o2));
  // ratios are non-negative: their float bits order like unsigned ints
  if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned*>(&res->max_ratio), __float_as_uint(worst));
}

// The same test when the partial sums come from the fused product (the cast
// kernels and the GEMM epilogue): pzq[s][i] = (z_0..3, q_0..3) over column
// stripe s of A, pw[t][i] = (C r)_i over column tile t of C.
// Four threads per row: thread p of row i sums partials p, p + 4, p + 8,
// ... in order, then the four sums are added in a fixed order ((0 + 1) +
// (2 + 3)), so the result does not depend on the schedule.
__global__ void __launch_bounds__(256) k_frv_check_fused(const float* __restrict__ pzq, int nsa,
                                                         const float4* __restrict__ pw, int nsc,
                                                         int N, int nvec, float c, float u_eff,
                                                         FreivaldsResult* res) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long i = g >> 2;
  const int part = (int)(g & 3);
  float o[12];
#pragma unroll
  for (int t = 0; t < 12; ++t) o[t] = 0.0f;
  if (i < N) {
    for (int s = part; s < nsa; s += 4) {
      const float4* p = reinterpret_cast<const float4*>(pzq + ((long long)s * N + i) * 8);
      const float4 z = p[0], q = p[1];
      o[0] += z.x; o[1] += z.y; o[2] += z.z; o[3] += z.w;
      o[4] += q.x; o[5] += q.y; o[6] += q.z; o[7] += q.w;
    }
    // several partials in flight at once (each sum keeps its order)
#pragma unroll 4
    for (int t = part; t < nsc; t += 4) {
      const float4 w = pw[(long long)t * N + i];
      o[8] += w.x; o[9] += w.y; o[10] += w.z; o[11] += w.w;
    }
  }
#pragma unroll
  for (int t = 0; t < 12; ++t) {
    o[t] += __shfl_xor_sync(0xffffffffu, o[t], 1);
    o[t] += __shfl_xor_sync(0xffffffffu, o[t], 2);
  }
  float worst = 0.0f;
  bool bad = false;
  if (i < N && part == 0) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      if (v >= nvec) continue;
      const float tau = c * u_eff * sqrtf(o[4 + v]);
      const float gap = fabsf(o[v] - o[8 + v]);
      const float ratio = tau > 0.0f ? gap / tau : (gap > 0.0f ? INFINITY : 0.0f);
      worst = fmaxf(worst, ratio);
      bad |= !(gap <= tau);
    }
    if (bad) atomicMax(&res->viol_enc, ~(unsigned long long)i);
  }
#pragma unroll
  for (int o2 = 16; o2 > 0; o2 >>= 1) worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, o2));
  if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned*>(&res->max_ratio), __float_as_uint(worst));
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

size_t freivalds_scratch_bytes(int N, int nvec) {
  (void)nvec;
  const size_t nsb = (size_t)((N + kSwB - 1) / kSwB), nsa = (size_t)((N + kSwAC - 1) / kSwAC);
  return 3 * align256((size_t)N * sizeof(float4)) + align256(nsb * N * 5 * sizeof(float)) +
         align256(nsa * N * 12 * sizeof(float));
}

cudaError_t launch_freivalds(const float* A, const float* B, const float* C, int N,
                             unsigned long long seed, int nvec, float c, float u_eff,
                             void* scratch, FreivaldsResult* res, cudaStream_t st, Prof* prof,
                             int64_t* kernels) {
  if (N <= 0) return cudaSuccess;
  if (nvec < 1 || nvec > kMaxVec) return cudaErrorInvalidValue;
  const int nsb = (N + kSwB - 1) / kSwB, nsa = (N + kSwAC - 1) / kSwAC;
  char* p = static_cast<char*>(scratch);
  const size_t one = align256((size_t)N * sizeof(float4));
  float4* r4 = reinterpret_cast<float4*>(p);
  float4* br4 = reinterpret_cast<float4*>(p + one);
  float4* t4 = reinterpret_cast<float4*>(p + 2 * one);
  char* q = p + 3 * one;
  float* pb = reinterpret_cast<float*>(q);
  q += align256((size_t)nsb * N * 5 * sizeof(float));
  float* pac = reinterpret_cast<float*>(q);
  const int rowblocks = (N + kRows * kIters - 1) / (kRows * kIters);
  prof_begin(prof, "freivalds", st);
  k_frv_r<<<(N + 255) / 256, 256, 0, st>>>(r4, N, nvec, seed);
  k_frv_b<<<dim3(nsb, rowblocks), 256, 0, st>>>(B, N, r4, pb);
  k_frv_b_reduce<<<(N + 255) / 256, 256, 0, st>>>(pb, N, nsb, br4, t4);
  k_frv_ac<<<dim3(nsa, rowblocks), 256, 0, st>>>(A, C, N, r4, br4, t4, pac);
  k_frv_check<<<(N + 255) / 256, 256, 0, st>>>(pac, N, nsa, nvec, c, u_eff, res);
  prof_end(prof, st);
  *kernels += 5;
  return cudaGetLastError();
}

FrvFused frv_fused_layout(void* scratch, int N) {
  FrvFused f;
  char* p = static_cast<char*>(scratch);
  const size_t one = align256((size_t)N * sizeof(float4));
  f.r4 = reinterpret_cast<float4*>(p);
  f.br4 = reinterpret_cast<float4*>(p + one);
  f.t4 = reinterpret_cast<float4*>(p + 2 * one);
  p += 3 * one;
  f.nsb = (N + kFrvStripeB - 1) / kFrvStripeB;
  f.nsa = (N + kFrvStripeA - 1) / kFrvStripeA;
  f.nsc = (N + kFrvTileC - 1) / kFrvTileC;
  f.pb = reinterpret_cast<float*>(p);
  p += align256((size_t)f.nsb * N * 5 * sizeof(float));
  f.pzq = reinterpret_cast<float*>(p);
  p += align256((size_t)f.nsa * N * 8 * sizeof(float));
  f.pw = reinterpret_cast<float4*>(p);
  p += align256((size_t)f.nsc * N * sizeof(float4));
  f.bytes = (size_t)(p - static_cast<char*>(scratch));
  return f;
}

size_t frv_fused_scratch_bytes(int N) { return frv_fused_layout(nullptr, N).bytes; }

cudaError_t launch_frv_vectors(const FrvFused& f, int N, int nvec, unsigned long long seed,
                               cudaStream_t st) {
  if (nvec < 1 || nvec > kMaxVec) return cudaErrorInvalidValue;
  k_frv_r<<<(N + 255) / 256, 256, 0, st>>>(f.r4, N, nvec, seed);
  return cudaGetLastError();
}

cudaError_t launch_frv_b_reduce(const FrvFused& f, int N, cudaStream_t st) {
  k_frv_b_reduce<<<(N + 255) / 256, 256, 0, st>>>(f.pb, N, f.nsb, f.br4, f.t4);
  return cudaGetLastError();
}

cudaError_t launch_frv_check_fused(const FrvFused& f, int N, int nvec, float c, float u_eff,
                                   FreivaldsResult* res, cudaStream_t st) {
  // four threads per row: 128 CTAs of 256 threads at N = 8192
  k_frv_check_fused<<<(int)((4LL * N + 255) / 256), 256, 0, st>>>(f.pzq, f.nsa, f.pw, f.nsc, N,
                                                                  nvec, c, u_eff, res);
  return cudaGetLastError();
}

}  // namespace sgk
