// k_gemm_tc.cu -- matrix `multiply` of Sec. 3.4 on the 5th-generation tensor
// cores (sm_103a): C = A B (or C = C - A B for the elimination update) with
// bf16 or fp16 operands, rounded to nearest even from binary32, and binary32
// accumulation in tensor memory.
//
// Operands are first cast (and B transposed) into K-major 16-bit copies whose
// K extent is padded to a multiple of 64.  The product runs on CTA pairs
// (k_gemm_tc2, tcgen05 cta_group::2, 256 x 256 tiles, described there) where
// the device schedules clusters of two, else on single CTAs (k_gemm_tc), each
// computing a 128 x 256 tile of C:
//   warp 0, one lane : TMA producer -- 2-D tiled bulk-tensor loads of a 128x64
//                      A slice and a 256x64 B slice per stage (128-byte
//                      swizzle, no multicast), completion on a "full" mbarrier;
//   warp 1, one lane : MMA issuer -- four tcgen05.mma (M=128, N=256, K=16) per
//                      stage, accumulator in 256 TMEM columns, tcgen05.commit
//                      to the stage's "empty" mbarrier, and to "done" at the end;
//   warp 2           : allocates / frees the tensor memory;
//   all four warps   : epilogue -- tcgen05.ld of their 32 TMEM lanes (rows),
//                      binary32 stores (or read-modify-write for C - A B).
// Four pipeline stages of 48 KB.  Every mbarrier wait is bounded: on a
// timeout the kernel raises an error flag and finishes without hanging.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>

#include "sg_frv.cuh"
#include "sg_linalg_kernels.h"

namespace sgk {
namespace {

constexpr int TM = 128, TN = 256, TK = 64, STAGES = 4;
static_assert(kFrvTileC == TN / 2, "the fused check keeps one C r partial per epilogue warp's column half");
constexpr int A_BYTES = TM * TK * 2;            // 16 KB
constexpr int B_BYTES = TN * TK * 2;            // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;  // 48 KB
// Eight epilogue warps, two per quarter of the tensor memory's lanes, each
// draining one 128-column half of a tile (with four, each alone on its SM
// sub-partition, the dependent steps of the epilogue bounded short-K
// products such as the elimination's updates)
constexpr int kEpiWarps = 8;
constexpr int kGemmThreads = 64 + 32 * kEpiWarps;   // producer, MMA issuer, epilogue
constexpr int R_BYTES = kEpiWarps * (TN / 2) * 16;  // the fused check's r entries of each warp's half
// The epilogue turns each 32 x 32 chunk (lane = row, from the tensor
// memory) around in shared memory, 16 rows at a time, so that eight lanes
// cover one row's 128 bytes: a warp's access touches 4 rows instead of 32,
// and the L1 handles 4 lines per request instead of 32.  The 16-byte group
// g of row r sits at group g ^ (r & 7): conflict-free writes (lane = row)
// and reads (eight lanes = one row).
constexpr int T_BYTES = kEpiWarps * 16 * 32 * 4;    // one 16 x 32 buffer per epilogue warp
constexpr int SMEM_BYTES =
    STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/ + R_BYTES + T_BYTES;
constexpr unsigned kWaitLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

// bounded wait for the phase with the given parity to complete
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err) {
  for (unsigned i = 0; i < kWaitLimit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  atomicExch(err, 1);
  return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// UMMA shared-memory descriptor: K-major tile in the 128-byte swizzle
// layout (rows of 128 B, 8-row groups 1024 B apart).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address >> 4
  d |= (uint64_t)1 << 16;                      // leading byte offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;            // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                      // descriptor version
  d |= (uint64_t)2 << 61;                      // 128-byte swizzle
  return d;
}

// instruction descriptor, kind::f16: D f32, A/B bf16 or f16, both K-major
__host__ __device__ constexpr uint32_t idesc(bool fp16) {
  return (1u << 4) | ((fp16 ? 0u : 1u) << 7) | ((fp16 ? 0u : 1u) << 10) |
         ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id,
                                     uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(id), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// bounded wait that also gives up as soon as another role of the CTA has
// raised the abort flag (so one failed wait cannot leave the others spinning
// through every remaining tile)
__device__ __forceinline__ bool mbar_wait_ab(uint32_t bar, uint32_t parity, int* err,
                                             volatile int* abort_flag) {
  for (unsigned i = 0; i < kWaitLimit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((i & 255) == 255 && *abort_flag) return false;
  }
  atomicExch(err, 1);
  *abort_flag = 1;
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// arrive on a barrier anywhere in the cluster
__device__ __forceinline__ void mbar_arrive_cl(uint32_t bar_cl) {
  asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(bar_cl) : "memory");
}

// C rows m0q .. m0q + 31, columns col0 .. col0 + 31, as the epilogue's
// stores take them: access it, lane l: row m0q + 4 it + l / 8, columns
// col0 + 4 (l % 8) .. + 3 (zero outside M x N)
__device__ __forceinline__ void load_c(const float* __restrict__ C, int ldc, int M, int N, int m0q,
                                       int col0, int lane, float4 (&cv)[8]) {
#pragma unroll
  for (int it = 0; it < 8; ++it) {
    const int grow = m0q + it * 4 + (lane >> 3), gcol = col0 + (lane & 7) * 4;
    const float* cp = C + (size_t)grow * ldc + gcol;
    if (grow < M && gcol + 4 <= N && ((reinterpret_cast<uintptr_t>(cp) & 15) == 0)) {
      cv[it] = *reinterpret_cast<const float4*>(cp);
    } else {
      float e[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) e[u] = grow < M && gcol + u < N ? cp[u] : 0.0f;
      cv[it] = make_float4(e[0], e[1], e[2], e[3]);
    }
  }
}

// Row `row`, columns c0 .. c0 + w - 1 of C (clipped to N) into L2: the
// subtracting product's epilogue reads them a tile later
__device__ __forceinline__ void prefetch_c_row(const float* C, int ldc, int M, int N, int row,
                                               int c0, int w) {
  if (row >= M || c0 >= N) return;
  const float* p = C + (size_t)row * ldc + c0;
  const unsigned bytes = (unsigned)(min(w, N - c0) * 4) & ~15u;
  if ((reinterpret_cast<uintptr_t>(p) & 15) == 0 && bytes)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// One 32 x 32 chunk of the epilogue: lane l holds row m0q + l, columns
// col0 .. col0 + 31 (r); C := chunk, or C := cv - chunk when subtracting (cv
// from load_c), through the warp's transpose buffer s_tw (16 x 32 floats,
// rows 16 h .. 16 h + 15 in turn); rows outside M and columns outside N are
// left alone.
__device__ __forceinline__ void store_chunk(float* __restrict__ C, int ldc, int M, int N, int m0q,
                                            int col0, const uint32_t (&r)[32], float* s_tw,
                                            int lane, int subtract, const float4 (&cv)[8]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if ((lane >> 4) == h) {
      const int rw = lane & 15;
      float4* dst = reinterpret_cast<float4*>(s_tw + rw * 32);
#pragma unroll
      for (int j = 0; j < 8; ++j)
        dst[j ^ (rw & 7)] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                        __uint_as_float(r[4 * j + 2]),
                                        __uint_as_float(r[4 * j + 3]));
    }
    __syncwarp();
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int rr = it * 4 + (lane >> 3), g = lane & 7;
      const float4 v = reinterpret_cast<const float4*>(s_tw + rr * 32)[g ^ (rr & 7)];
      const int grow = m0q + 16 * h + rr, gcol = col0 + 4 * g;
      if (grow >= M) continue;
      const float4 c4 = cv[4 * h + it];
      const float4 o =
          subtract ? make_float4(c4.x - v.x, c4.y - v.y, c4.z - v.z, c4.w - v.w) : v;
      float* cp = C + (size_t)grow * ldc + gcol;
      if (gcol + 4 <= N && ((reinterpret_cast<uintptr_t>(cp) & 15) == 0)) {
        *reinterpret_cast<float4*>(cp) = o;
      } else {
        const float oe[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (gcol + u < N) cp[u] = oe[u];
      }
    }
    __syncwarp();
  }
}

// The epilogue of one tile by one epilogue warp: tensor-memory lane quarter
// q (rows m0q .. m0q + 31), column half hh (columns n0 + 128 hh .. + 127,
// four 32-column chunks) of accumulator acc.  The warp releases the
// accumulator with one arrival on `tempty` (a cluster address when CL) once
// its last chunk is read; the fused check's partial C r of its rows over its
// half goes to column tile 2 bn + hh of frv_pw.  false: the wait for the
// accumulator gave up.
template <bool CL>
__device__ __forceinline__ bool epilogue_tile(
    uint32_t tmem, int acc, int tl, uint32_t tfull, uint32_t tempty, int q, int hh, int m0q,
    int n0, int bn, float* __restrict__ C, int ldc, int M, int N, int subtract,
    const float4* __restrict__ frv_r, float4* __restrict__ frv_pw, int inj_row, int inj_col,
    float inj_delta, float4* s_rw, float* s_tw, int lane, int* err, volatile int* abort_flag) {
  const int c0 = n0 + hh * (TN / 2);
  if (frv_r) {
    // each epilogue warp keeps its own copy, so no barrier spans the warps
    __syncwarp();
    for (int j = lane; j < TN / 2; j += 32)
      s_rw[j] = c0 + j < N ? frv_r[c0 + j] : make_float4(0.f, 0.f, 0.f, 0.f);
    __syncwarp();
  }
  if (!mbar_wait_ab(tfull, (uint32_t)(tl >> 1) & 1u, err, abort_flag)) return false;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int row = m0q + lane;
  float4 wacc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
  for (int c = 0; c < TN / 64; ++c) {
    const int col0 = c0 + c * 32;
    float4 cv[8];
    if (subtract) load_c(C, ldc, M, N, m0q, col0, lane, cv);
    uint32_t r[32];
    tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * TN + col0 - n0), r);
    if (c == TN / 64 - 1) {
      // this warp's part of the accumulator is drained
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        if (CL)
          mbar_arrive_cl(tempty);
        else
          mbar_arrive(tempty);
      }
    }
    // contract testing: a planted error in one product element, applied
    // before it is stored (and before the fused check sees it)
    if (row == inj_row && inj_col >= col0 && inj_col < col0 + 32) {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (col0 + j == inj_col) r[j] = __float_as_uint(__uint_as_float(r[j]) + inj_delta);
    }
    if (frv_r) {
      // r of columns past N is zero in s_r (their accumulator entries are too)
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const float4 rj = s_rw[c * 32 + j];
        const float v = __uint_as_float(r[j]);
        wacc.x = fmaf(v, rj.x, wacc.x);
        wacc.y = fmaf(v, rj.y, wacc.y);
        wacc.z = fmaf(v, rj.z, wacc.z);
        wacc.w = fmaf(v, rj.w, wacc.w);
      }
    }
    store_chunk(C, ldc, M, N, m0q, col0, r, s_tw, lane, subtract, cv);
  }
  if (frv_r && row < M && c0 < N) frv_pw[(size_t)(2 * bn + hh) * M + row] = wacc;
  return true;
}

// Tile t of the persistent order: groups of kGroupM row blocks; inside a
// group the row block varies fastest.  The 76 pairs' concurrent 256 x 256
// tiles then span 8 row blocks x about 10 column blocks, whose A and B
// slices (some 75 MB at K = 8192) stay in L2 instead of all of B (groups of
// 8 measured 0.7% faster than 16, and 32 4% slower).
constexpr int kGroupM = 8;
__device__ __forceinline__ void tile_coords(int t, int nM, int nN, int* mb, int* nb) {
  const int per_group = kGroupM * nN;
  const int g = t / per_group;
  const int first = g * kGroupM;
  const int gm = min(kGroupM, nM - first);
  const int r = t - g * per_group;
  *mb = first + r % gm;
  *nb = r / gm;
}

// Persistent kernel, one CTA per SM, tiles t = blockIdx.x + i * gridDim.x in
// the grouped order of tile_coords:
//   warp 0, one lane : TMA producer over all of the CTA's tiles;
//   warp 1, one lane : MMA issuer; accumulators alternate between two
//                      256-column halves of the 512 TMEM columns, so the
//                      epilogue of one tile overlaps the main loop of the next;
//   warps 2..9       : epilogue, warp w reads TMEM lanes 32 (w % 4) .. + 31
//                      and the 128-column half (w - 2) / 4 of the tile;
//                      after draining an accumulator they release it to the
//                      MMA issuer through an mbarrier.
__global__ void __launch_bounds__(kGemmThreads, 1) k_gemm_tc(const __grid_constant__ CUtensorMap ma,
                                                    const __grid_constant__ CUtensorMap mb,
                                                    float* __restrict__ C, int ldc, int M,
                                                    int N, int KB, uint32_t id, int subtract,
                                                    int* err, const float4* __restrict__ frv_r,
                                                    float4* __restrict__ frv_pw, int inj_row,
                                                    int inj_col, float inj_delta) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  // bars[0..S): full, [S..2S): empty, [2S, 2S+2): accumulator full,
  // [2S+2, 2S+4): accumulator empty, [2S+4]: drain; then the TMEM slot and
  // the abort flag
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float4* s_r = reinterpret_cast<float4*>(smem + STAGES * STAGE_BYTES + 256);
  float* s_t = reinterpret_cast<float*>(smem + STAGES * STAGE_BYTES + 256 + R_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nN = (N + TN - 1) / TN, nM = (M + TM - 1) / TM;
  const int ntiles = nN * nM;
  const uint32_t tfull0 = smem_u32(&bars[2 * STAGES]), tempty0 = smem_u32(&bars[2 * STAGES + 2]);
  const uint32_t drain_bar = smem_u32(&bars[2 * STAGES + 4]);

  if (threadIdx.x == 0) {
    for (int s = 0; s < 2 * STAGES; ++s) mbar_init(smem_u32(&bars[s]), 1);
    mbar_init(tfull0, 1);
    mbar_init(tfull0 + 8, 1);
    mbar_init(tempty0, kEpiWarps);
    mbar_init(tempty0 + 8, kEpiWarps);
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(2 * TN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // producer
      int it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int bm, bn;
        tile_coords(t, nM, nN, &bm, &bn);
        const int m0 = bm * TM, n0 = bn * TN;
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
          if (it >= STAGES &&
              !mbar_wait_ab(smem_u32(&bars[STAGES + s]), ph ^ 1u, err, abort_flag)) {
            ok = false;
            break;
          }
          const uint32_t full = smem_u32(&bars[s]);
          mbar_expect_tx(full, STAGE_BYTES);
          const uint32_t a_dst = smem_u32(smem + s * STAGE_BYTES);
          tma_load_2d(a_dst, &ma, kb * TK, m0, full);
          tma_load_2d(a_dst + A_BYTES, &mb, kb * TK, n0, full);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer
      int it = 0, tl = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tl) {
        const int acc = tl & 1;
        if (tl >= 2 && !mbar_wait_ab(tempty0 + 8 * acc, (uint32_t)((tl >> 1) - 1) & 1u, err,
                                     abort_flag))
          break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dacc = tmem + (uint32_t)(acc * TN);
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
          if (!mbar_wait_ab(smem_u32(&bars[s]), ph, err, abort_flag)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a_base = smem_u32(smem + s * STAGE_BYTES);
          const uint64_t da = sdesc(a_base), db = sdesc(a_base + A_BYTES);
#pragma unroll
          for (int k = 0; k < TK / 16; ++k) {
            // advance 16 elements (32 bytes) along K inside the swizzled rows
            umma(dacc, da + (uint64_t)(k * 2), db + (uint64_t)(k * 2), id, (kb | k) != 0);
          }
          umma_commit(smem_u32(&bars[STAGES + s]));
        }
        if (ok) umma_commit(tfull0 + 8 * acc);
      }
      // completes when every MMA issued above has finished
      umma_commit(drain_bar);
    }
  } else {
    // epilogue warps 2..9: lane quarter warp % 4, column half (warp - 2) / 4
    const int q = warp & 3, hh = (warp - 2) >> 2;
    float4* s_rw = s_r + (warp - 2) * (TN / 2);
    float* s_tw = s_t + (warp - 2) * 16 * 32;
    int tl = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++tl) {
      int bm, bn;
      tile_coords(t, nM, nN, &bm, &bn);
      const int acc = tl & 1;
      if (subtract && t + (int)gridDim.x < ntiles) {
        int bm2, bn2;
        tile_coords(t + (int)gridDim.x, nM, nN, &bm2, &bn2);
        prefetch_c_row(C, ldc, M, N, bm2 * TM + q * 32 + lane, bn2 * TN + hh * (TN / 2), TN / 2);
      }
      if (!epilogue_tile<false>(tmem, acc, tl, tfull0 + 8 * acc, tempty0 + 8 * acc, q, hh,
                                bm * TM + q * 32, bn * TN, bn, C, ldc, M, N, subtract, frv_r,
                                frv_pw, inj_row, inj_col, inj_delta, s_rw, s_tw, lane, err,
                                abort_flag))
        break;
    }
  }
  __syncthreads();
  if (warp == 2) {
    // every MMA has completed before the tensor memory is released
    mbar_wait(drain_bar, 0, err);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TN)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// The same product on CTA pairs (a cluster of 2, tcgen05 cta_group::2): a pair
// computes a 256 x 256 tile of C, each CTA holding 128 rows of the A slice
// and 128 rows (half) of the B slice of every stage, so each CTA moves 32 KB
// per 64-deep K step instead of 48 KB for a 128 x 256 tile of its own.
//   warp 0, one lane, both CTAs : TMA producer of its CTA's halves; the loads
//       complete on the leader CTA's "full" barrier (.cta_group::2), which
//       expects both CTAs' bytes (each producer arrives with its own count);
//   warp 1, one lane, leader    : MMA issuer, tcgen05.mma.cta_group::2
//       (M = 256, N = 256, K = 16); commits multicast to both CTAs' "empty",
//       "accumulator full" and "drain" barriers;
//   warps 2..9, both CTAs       : epilogue of the CTA's 128 rows from its own
//       tensor memory (two warps per lane quarter, one per column half); they
//       release an accumulator by arriving on the leader's "accumulator
//       empty" barrier (sixteen arrivals, eight remote).
// Six stages of 32 KB.  Every mbarrier wait is bounded, as in k_gemm_tc.
constexpr int TM2 = 256, TH = 128, STAGES2 = 6;
constexpr int STAGE2_BYTES = TH * TK * 2 * 2;   // 128 A rows + 128 B rows
constexpr int SMEM2_BYTES = STAGES2 * STAGE2_BYTES + 1024 + 256 + R_BYTES + T_BYTES;

__host__ __device__ constexpr uint32_t idesc2(bool fp16) {
  return (1u << 4) | ((fp16 ? 0u : 1u) << 7) | ((fp16 ? 0u : 1u) << 10) |
         ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM2 >> 4) << 24);
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t map_rank(uint32_t local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
               ::: "memory");
}
// arrive (with a byte count to expect) on a barrier anywhere in the cluster;
// CTA-scope release: a cluster-scope one would wait for every earlier global
// store of the thread
__device__ __forceinline__ void mbar_expect_tx_cl(uint32_t bar_cl, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cluster.b64 _, [%0], %1;" ::"r"(bar_cl),
               "r"(bytes) : "memory");
}
// TMA load into this CTA's shared memory completing on a barrier of either CTA of the pair
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map, int x,
                                                 int y, uint32_t bar_cl) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar_cl)
      : "memory");
}
__device__ __forceinline__ void umma2(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id,
                                      uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(id), "r"(accumulate)
      : "memory");
}
// arrives once on the barrier at this offset in both CTAs of the pair when
// every MMA issued before it has completed
__device__ __forceinline__ void umma_commit_pair(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(bar), "h"((unsigned short)3)
      : "memory");
}

__global__ void __launch_bounds__(kGemmThreads, 1) k_gemm_tc2(const __grid_constant__ CUtensorMap ma,
                                                     const __grid_constant__ CUtensorMap mb,
                                                     float* __restrict__ C, int ldc, int M,
                                                     int N, int KB, uint32_t id, int subtract,
                                                     int* err, const float4* __restrict__ frv_r,
                                                     float4* __restrict__ frv_pw, int inj_row,
                                                     int inj_col, float inj_delta) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES2 * STAGE2_BYTES);
  // bars[0..S): full (leader's count), [S..2S): empty, [2S, 2S+2): accumulator
  // full, [2S+2, 2S+4): accumulator empty (leader's count), [2S+4]: drain
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES2 + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float4* s_r = reinterpret_cast<float4*>(smem + STAGES2 * STAGE2_BYTES + 256);
  float* s_t = reinterpret_cast<float*>(smem + STAGES2 * STAGE2_BYTES + 256 + R_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const int pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
  const int nN = (N + TN - 1) / TN, nM = (M + TM2 - 1) / TM2;
  const int ntiles = nN * nM;
  const uint32_t tfull0 = smem_u32(&bars[2 * STAGES2]), tempty0 = smem_u32(&bars[2 * STAGES2 + 2]);
  const uint32_t drain_bar = smem_u32(&bars[2 * STAGES2 + 4]);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES2; ++s) {
      mbar_init(smem_u32(&bars[s]), 2);
      mbar_init(smem_u32(&bars[STAGES2 + s]), 1);
    }
    mbar_init(tfull0, 1);
    mbar_init(tfull0 + 8, 1);
    mbar_init(tempty0, 2 * kEpiWarps);
    mbar_init(tempty0 + 8, 2 * kEpiWarps);
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(2 * TN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  cluster_sync();   // both CTAs' barriers exist, and the tensor memory, before use
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int t = pair; t < ntiles && ok; t += npairs) {
        int bm, bn;
        tile_coords(t, nM, nN, &bm, &bn);
        const int m0 = bm * TM2 + (int)rank * TH, n0 = bn * TN + (int)rank * TH;
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int s = it % STAGES2;
          const uint32_t ph = (uint32_t)(it / STAGES2) & 1u;
          if (it >= STAGES2 &&
              !mbar_wait_ab(smem_u32(&bars[STAGES2 + s]), ph ^ 1u, err, abort_flag)) {
            ok = false;
            break;
          }
          const uint32_t full_cl = map_rank(smem_u32(&bars[s]), 0);
          mbar_expect_tx_cl(full_cl, STAGE2_BYTES);
          const uint32_t a_dst = smem_u32(smem + s * STAGE2_BYTES);
          tma_load_2d_pair(a_dst, &ma, kb * TK, m0, full_cl);
          tma_load_2d_pair(a_dst + TH * TK * 2, &mb, kb * TK, n0, full_cl);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) {
      int it = 0, tl = 0;
      bool ok = true;
      for (int t = pair; t < ntiles && ok; t += npairs, ++tl) {
        const int acc = tl & 1;
        if (tl >= 2 && !mbar_wait_ab(tempty0 + 8 * acc, (uint32_t)((tl >> 1) - 1) & 1u, err,
                                     abort_flag))
          break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dacc = tmem + (uint32_t)(acc * TN);
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int s = it % STAGES2;
          const uint32_t ph = (uint32_t)(it / STAGES2) & 1u;
          if (!mbar_wait_ab(smem_u32(&bars[s]), ph, err, abort_flag)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a_base = smem_u32(smem + s * STAGE2_BYTES);
          const uint64_t da = sdesc(a_base), db = sdesc(a_base + TH * TK * 2);
#pragma unroll
          for (int k = 0; k < TK / 16; ++k)
            umma2(dacc, da + (uint64_t)(k * 2), db + (uint64_t)(k * 2), id, (kb | k) != 0);
          umma_commit_pair(smem_u32(&bars[STAGES2 + s]));
        }
        if (ok) umma_commit_pair(tfull0 + 8 * acc);
      }
      // completes, in both CTAs, when every MMA issued above has finished
      umma_commit_pair(drain_bar);
    }
  } else {
    // epilogue warps 2..9: lane quarter warp % 4, column half (warp - 2) / 4
    const int q = warp & 3, hh = (warp - 2) >> 2;
    float4* s_rw = s_r + (warp - 2) * (TN / 2);
    float* s_tw = s_t + (warp - 2) * 16 * 32;
    const uint32_t tempty_leader = map_rank(tempty0, 0);
    int tl = 0;
    for (int t = pair; t < ntiles; t += npairs, ++tl) {
      int bm, bn;
      tile_coords(t, nM, nN, &bm, &bn);
      const int acc = tl & 1;
      if (subtract && t + npairs < ntiles) {
        int bm2, bn2;
        tile_coords(t + npairs, nM, nN, &bm2, &bn2);
        prefetch_c_row(C, ldc, M, N, bm2 * TM2 + (int)rank * TH + q * 32 + lane,
                       bn2 * TN + hh * (TN / 2), TN / 2);
      }
      if (!epilogue_tile<true>(tmem, acc, tl, tfull0 + 8 * acc, tempty_leader + 8 * acc, q, hh,
                               bm * TM2 + (int)rank * TH + q * 32, bn * TN, bn, C, ldc, M, N,
                               subtract, frv_r, frv_pw, inj_row, inj_col, inj_delta, s_rw, s_tw,
                               lane, err, abort_flag))
        break;
    }
  }
  __syncthreads();
  if (warp == 2) {
    mbar_wait(drain_bar, 0, err);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TN)
                 : "memory");
  }
  // neither CTA leaves while the other may still signal its barriers
  cluster_sync();
}

// binary32 (rows x cols, leading dim ld) -> 16-bit rows x Kp, zero padded
template <bool FP16>
__global__ void k_cast_rows(const float* __restrict__ A, int lda, int rows, int cols, int Kp,
                            void* out) {
  const long long total = (long long)rows * (Kp / 8);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t / (Kp / 8));
    const int c0 = (int)(t % (Kp / 8)) * 8;
    const float* src = A + (size_t)r * lda + c0;
    uint16_t h[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float v = (c0 + j < cols) ? src[j] : 0.0f;
      if (FP16) {
        const __half x = __float2half_rn(v);
        h[j] = *reinterpret_cast<const uint16_t*>(&x);
      } else {
        const __nv_bfloat16 x = __float2bfloat16_rn(v);
        h[j] = *reinterpret_cast<const uint16_t*>(&x);
      }
    }
    uint4 pk;
    pk.x = h[0] | ((uint32_t)h[1] << 16);
    pk.y = h[2] | ((uint32_t)h[3] << 16);
    pk.z = h[4] | ((uint32_t)h[5] << 16);
    pk.w = h[6] | ((uint32_t)h[7] << 16);
    reinterpret_cast<uint4*>(out)[t] = pk;
  }
}

// B (K x N, leading dim ldb) -> Bt (N x Kp) 16-bit, transposed via 32x32 tiles
template <bool FP16>
__global__ void k_cast_transpose(const float* __restrict__ B, int ldb, int K, int N, int Kp,
                                 uint16_t* out) {
  __shared__ float t[32][33];
  const int k0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int k = k0 + i, n = n0 + threadIdx.x;
    t[i][threadIdx.x] = (k < K && n < N) ? B[(size_t)k * ldb + n] : 0.0f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int n = n0 + i, k = k0 + threadIdx.x;
    if (n < N && k < Kp) {
      const float v = t[threadIdx.x][i];
      uint16_t h;
      if (FP16) {
        const __half x = __float2half_rn(v);
        h = *reinterpret_cast<const uint16_t*>(&x);
      } else {
        const __nv_bfloat16 x = __float2bfloat16_rn(v);
        h = *reinterpret_cast<const uint16_t*>(&x);
      }
      out[(size_t)n * Kp + k] = h;
    }
  }
}

__device__ __forceinline__ uint16_t to16(float v, bool fp16) {
  if (fp16) {
    const __half x = __float2half_rn(v);
    return *reinterpret_cast<const uint16_t*>(&x);
  }
  const __nv_bfloat16 x = __float2bfloat16_rn(v);
  return *reinterpret_cast<const uint16_t*>(&x);
}

// Square B (N x N) -> Bt (N x Kp) 16-bit, with the fused Freivalds partial
// sums of row k over this CTA's stripe of kFrvStripeB columns:
// pb[stripe][k] = (sum_j B[k][j] r_v[j], v < 4;  sum_j B[k][j]^2).
// CTA: 64 rows of B, eight 64-column sub-tiles in turn, each staged in
// shared memory and written out transposed in 16-byte runs along k.
template <bool FP16>
__global__ void __launch_bounds__(256) k_cast_bt_frv(const float* __restrict__ B, int N, int Kp,
                                                     uint16_t* __restrict__ out,
                                                     const float4* __restrict__ r4,
                                                     float* __restrict__ pb) {
  __shared__ float t[64][65];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int k0 = blockIdx.y * 64;
  const bool vec2 = (N % 2) == 0 && ((uintptr_t)B % 8) == 0;
  float acc[8][5];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[i][q] = 0.0f;
  // the next step's 8 x 64 block is loaded while this step's is used
  auto load = [&](int n0, float* b0, float* b1) {
    const int nc = n0 + 2 * lane;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = k0 + w * 8 + i;
      b0[i] = 0.0f;
      b1[i] = 0.0f;
      if (k < N && n0 < N) {
        const float* rp = B + (size_t)k * N;
        if (vec2 && nc + 1 < N) {
          const float2 v = __ldcs(reinterpret_cast<const float2*>(rp + nc));
          b0[i] = v.x;
          b1[i] = v.y;
        } else {
          if (nc < N) b0[i] = __ldcs(rp + nc);
          if (nc + 1 < N) b1[i] = __ldcs(rp + nc + 1);
        }
      }
    }
  };
  float nb0[8], nb1[8];
  load(blockIdx.x * kFrvStripeB, nb0, nb1);
#pragma unroll 1
  for (int st = 0; st < kFrvStripeB / 64; ++st) {
    const int n0 = blockIdx.x * kFrvStripeB + st * 64;
    if (n0 >= N) break;   // the same for the whole CTA
    const int nc = n0 + 2 * lane;
    const float4 r0 = frv::ldvec(r4, nc, N), r1 = frv::ldvec(r4, nc + 1, N);
    float b0[8], b1[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      b0[i] = nb0[i];
      b1[i] = nb1[i];
    }
    if (st + 1 < kFrvStripeB / 64) load(n0 + 64, nb0, nb1);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      acc[i][0] = fmaf(b1[i], r1.x, fmaf(b0[i], r0.x, acc[i][0]));
      acc[i][1] = fmaf(b1[i], r1.y, fmaf(b0[i], r0.y, acc[i][1]));
      acc[i][2] = fmaf(b1[i], r1.z, fmaf(b0[i], r0.z, acc[i][2]));
      acc[i][3] = fmaf(b1[i], r1.w, fmaf(b0[i], r0.w, acc[i][3]));
      acc[i][4] = fmaf(b1[i], b1[i], fmaf(b0[i], b0[i], acc[i][4]));
      t[w * 8 + i][2 * lane] = b0[i];
      t[w * 8 + i][2 * lane + 1] = b1[i];
    }
    __syncthreads();
#pragma unroll
    for (int u = threadIdx.x; u < 512; u += 256) {
      const int nn = u >> 3, kc = u & 7;
      const int n = n0 + nn;
      if (n < N) {
        uint32_t h[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) h[j] = to16(t[kc * 8 + j][nn], FP16);
        uint4 pk;
        pk.x = h[0] | (h[1] << 16);
        pk.y = h[2] | (h[3] << 16);
        pk.z = h[4] | (h[5] << 16);
        pk.w = h[6] | (h[7] << 16);
        *reinterpret_cast<uint4*>(out + (size_t)n * Kp + k0 + kc * 8) = pk;
      }
    }
    __syncthreads();
  }
  const int slot = (lane >> 2) & 7;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    float o[8] = {acc[i][0], acc[i][1], acc[i][2], acc[i][3], acc[i][4], 0.0f, 0.0f, 0.0f};
    const float v = frv::warp_sum_spread<8>(o, lane);
    const int k = k0 + w * 8 + i;
    if ((lane & 3) == 0 && slot < 5 && k < N) pb[((size_t)blockIdx.x * N + k) * 5 + slot] = v;
  }
}

// Square A (N x N) -> A16 (N x Kp) 16-bit (zero padded), with the fused
// partial sums of row i over this CTA's stripe of kFrvStripeA columns:
// pzq[stripe][i] = (sum_k a_ik br_v[k], v < 4;  sum_k a_ik^2 t_v[k], v < 4).
// Eight warps side by side along the row (4 columns per lane), 8 rows per
// step, 4 steps per CTA.
template <bool FP16>
__global__ void __launch_bounds__(256, 2) k_cast_a_frv(const float* __restrict__ A, int N, int Kp,
                                                       uint16_t* __restrict__ out,
                                                       const float4* __restrict__ br4,
                                                       const float4* __restrict__ t4,
                                                       float* __restrict__ pzq) {
  __shared__ float red[2][8][8][8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long c0 = (long long)blockIdx.x * kFrvStripeA + w * 128 + lane * 4;
  const bool vec = (N % 4) == 0 && ((uintptr_t)A % 16) == 0;
  float4 vb[4], vt[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    vb[e] = frv::ldvec(br4, c0 + e, N);
    vt[e] = frv::ldvec(t4, c0 + e, N);
  }
  const int slot = (lane >> 2) & 7;
  // the next step's eight rows are loaded while this step's are used
  auto load8 = [&](long long row0, float4* av) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const long long row = row0 + i;
      av[i] = row < N ? frv::ldv(A + row * (long long)N, c0, N, vec)
                      : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  float4 nxt[8];
  load8((long long)blockIdx.y * 32, nxt);
#pragma unroll 1
  for (int it = 0; it < 4; ++it) {
    const long long row0 = ((long long)blockIdx.y * 4 + it) * 8;
    if (row0 >= N) break;
    float4 av[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) av[i] = nxt[i];
    if (it < 3) load8(row0 + 8, nxt);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const long long row = row0 + i;
      const float a[4] = {av[i].x, av[i].y, av[i].z, av[i].w};
      if (row < N && c0 < Kp) {
        uint2 pk;
        pk.x = (uint32_t)to16(a[0], FP16) | ((uint32_t)to16(a[1], FP16) << 16);
        pk.y = (uint32_t)to16(a[2], FP16) | ((uint32_t)to16(a[3], FP16) << 16);
        *reinterpret_cast<uint2*>(out + row * Kp + c0) = pk;
      }
      float o[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) o[q] = 0.0f;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float a2 = a[e] * a[e];
        o[0] = fmaf(a[e], vb[e].x, o[0]); o[1] = fmaf(a[e], vb[e].y, o[1]);
        o[2] = fmaf(a[e], vb[e].z, o[2]); o[3] = fmaf(a[e], vb[e].w, o[3]);
        o[4] = fmaf(a2, vt[e].x, o[4]); o[5] = fmaf(a2, vt[e].y, o[5]);
        o[6] = fmaf(a2, vt[e].z, o[6]); o[7] = fmaf(a2, vt[e].w, o[7]);
      }
      const float v = frv::warp_sum_spread<8>(o, lane);
      if ((lane & 3) == 0) red[it & 1][w][i][slot] = v;
    }
    __syncthreads();
    if (threadIdx.x < 64) {
      const int i = threadIdx.x >> 3, q = threadIdx.x & 7;
      const long long row = row0 + i;
      float s = 0.0f;
#pragma unroll
      for (int ww = 0; ww < 8; ++ww) s += red[it & 1][ww][i][q];
      if (row < N) pzq[((size_t)blockIdx.x * N + row) * 8 + q] = s;
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

bool make_map(CUtensorMap* m, const void* base, int rows, int Kp, int box_rows, bool fp16) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
  cuuint32_t box[2] = {(cuuint32_t)TK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return fn(m, fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
            const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// one CTA per SM (the pipeline's shared memory allows no second), at most
// one per tile
int persistent_grid(int M, int N) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms <= 0)
      sms = 1;
  }
  const long long tiles = (long long)((M + TM - 1) / TM) * ((N + TN - 1) / TN);
  return (int)std::max<long long>(1, std::min<long long>(tiles, sms));
}

// the CTA-pair kernel where the device schedules clusters of two with its
// shared memory (decided once)
bool use_pair() {
  static int v = -1;
  if (v < 0) {
    v = 0;
    if (cudaFuncSetAttribute(k_gemm_tc2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             SMEM2_BYTES) == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(2);
      cfg.blockDim = dim3(kGemmThreads);
      cfg.dynamicSmemBytes = SMEM2_BYTES;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = 2;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int nc = 0;
      if (cudaOccupancyMaxActiveClusters(&nc, k_gemm_tc2, &cfg) == cudaSuccess && nc >= 1) v = 1;
    }
    cudaGetLastError();
  }
  return v == 1;
}

// C (+)= A16 Bt16^T on the tensor cores: the CTA-pair kernel (form 2, or 0
// where the device schedules pairs), else the one-CTA kernel
cudaError_t launch_product(const uint16_t* a16, const uint16_t* bt16, int Kp, bool fp16, float* C,
                           int ldc, int M, int N, bool subtract, int* err, const float4* frv_r,
                           float4* frv_pw, int inj_row, int inj_col, float inj_delta,
                           cudaStream_t s, int form) {
  CUtensorMap ma, mb;
  if (!make_map(&ma, a16, M, Kp, TM, fp16)) return cudaErrorInvalidValue;
  if (form != 1 && !portable_kernels() && use_pair()) {
    if (!make_map(&mb, bt16, N, Kp, TH, fp16)) return cudaErrorInvalidValue;
    const long long tiles = (long long)((M + TM2 - 1) / TM2) * ((N + TN - 1) / TN);
    const int pairs = (int)std::max<long long>(
        1, std::min<long long>(tiles, persistent_grid(1 << 30, TN) / 2));   // SMs / 2
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * pairs);
    cfg.blockDim = dim3(kGemmThreads);
    cfg.dynamicSmemBytes = SMEM2_BYTES;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_gemm_tc2, ma, mb, C, ldc, M, N, Kp / TK, idesc2(fp16),
                              subtract ? 1 : 0, err, frv_r, frv_pw, inj_row, inj_col, inj_delta);
  }
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  if (!make_map(&mb, bt16, N, Kp, TN, fp16)) return cudaErrorInvalidValue;
  k_gemm_tc<<<persistent_grid(M, N), kGemmThreads, SMEM_BYTES, s>>>(ma, mb, C, ldc, M, N, Kp / TK,
                                                           idesc(fp16), subtract ? 1 : 0, err,
                                                           frv_r, frv_pw, inj_row, inj_col,
                                                           inj_delta);
  return cudaGetLastError();
}

}  // namespace

namespace {
bool g_portable = false;
}
void set_portable_kernels(bool on) { g_portable = on; }
bool portable_kernels() { return g_portable; }

void gemm_tc_prepare() {
  use_pair();
  cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  cudaGetLastError();
}

bool gemm_pair_available() { return !portable_kernels() && use_pair(); }

size_t gemm_tc_scratch_bytes(int M, int N, int K) {
  const size_t Kp = (size_t)((K + TK - 1) / TK) * TK;
  return 256 + align256((size_t)M * Kp * 2) + align256((size_t)N * Kp * 2);
}

namespace {

// the bf16 / fp16 operand copies: A by rows, B transposed (K padded to Kp)
void cast_operands(const float* A, int lda, const float* B, int ldb, int M, int N, int K, int Kp,
                   bool fp16, uint16_t* a16, uint16_t* bt16, cudaStream_t s) {
  const long long ca = (long long)M * (Kp / 8);
  const int ga = (int)std::min<long long>((ca + 255) / 256, 65535LL * 8);
  dim3 gt((N + 31) / 32, (Kp + 31) / 32), bt(32, 8);
  if (fp16) {
    k_cast_rows<true><<<ga, 256, 0, s>>>(A, lda, M, K, Kp, a16);
    k_cast_transpose<true><<<gt, bt, 0, s>>>(B, ldb, K, N, Kp, bt16);
  } else {
    k_cast_rows<false><<<ga, 256, 0, s>>>(A, lda, M, K, Kp, a16);
    k_cast_transpose<false><<<gt, bt, 0, s>>>(B, ldb, K, N, Kp, bt16);
  }
}

}  // namespace

cudaError_t time_gemm_forms(const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                            int M, int N, int K, bool fp16, void* scratch, cudaStream_t s,
                            const int* forms, int nforms, double* us, int64_t* kernels) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaErrorInvalidValue;
  const int Kp = ((K + TK - 1) / TK) * TK;
  char* p = static_cast<char*>(scratch);
  int* err = reinterpret_cast<int*>(p);
  uint16_t* a16 = reinterpret_cast<uint16_t*>(p + 256);
  uint16_t* bt16 = reinterpret_cast<uint16_t*>(p + 256 + align256((size_t)M * Kp * 2));
  cast_operands(A, lda, B, ldb, M, N, K, Kp, fp16, a16, bt16, s);
  *kernels += 2;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaError_t e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  for (int f = 0; f < nforms && e == cudaSuccess; ++f) {
    // a warm-up, then the better of two timed runs; a product shorter than
    // 16 us is repeated within each run (the events resolve about 0.5 us)
    double best = 1e300;
    int reps = 1;
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
      e = cudaEventRecord(ev[0], s);
      for (int k = 0; k < reps && e == cudaSuccess; ++k) {
        e = launch_product(a16, bt16, Kp, fp16, C, ldc, M, N, false, err, nullptr, nullptr, -1,
                           -1, 0.0f, s, forms[f]);
        *kernels += 1;
      }
      if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
      if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
      const double t = 1000.0 * ms / reps;
      if (r == 0)
        reps = t >= 16.0 ? 1 : (int)std::min(64.0, std::ceil(16.0 / std::max(t, 0.25)));
      else if (e == cudaSuccess)
        best = std::min(best, t);
    }
    us[f] = best;
  }
  for (cudaEvent_t v : ev)
    if (v) cudaEventDestroy(v);
  return e;
}

cudaError_t launch_gemm_tc(const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                           int M, int N, int K, bool fp16, bool subtract, void* scratch,
                           cudaStream_t s, Prof* prof, int64_t* kernels, int inj_row,
                           int inj_col, float inj_delta, int form) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (K <= 0) {   // empty inner dimension: C = 0 (or C unchanged for C - A B)
    if (subtract) return cudaSuccess;
    return cudaMemset2DAsync(C, (size_t)ldc * 4, 0, (size_t)N * 4, M, s);
  }
  const int Kp = ((K + TK - 1) / TK) * TK;
  char* p = static_cast<char*>(scratch);
  int* err = reinterpret_cast<int*>(p);
  uint16_t* a16 = reinterpret_cast<uint16_t*>(p + 256);
  uint16_t* bt16 = reinterpret_cast<uint16_t*>(p + 256 + align256((size_t)M * Kp * 2));
  prof_begin(prof, "cast_operands", s);
  cast_operands(A, lda, B, ldb, M, N, K, Kp, fp16, a16, bt16, s);
  prof_end(prof, s);
  prof_begin(prof, fp16 ? "gemm_tc_f16" : "gemm_tc_bf16", s);
  const cudaError_t e = launch_product(a16, bt16, Kp, fp16, C, ldc, M, N, subtract, err, nullptr,
                                       nullptr, inj_row, inj_col, inj_delta, s, form);
  prof_end(prof, s);
  *kernels += 3;
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_gemm_tc_checked(const float* A, const float* B, float* C, int N, bool fp16,
                                   unsigned long long seed, int nvec, float c, float u_eff,
                                   void* scratch, FreivaldsResult* res, cudaStream_t s,
                                   Prof* prof, int64_t* kernels, int inj_row, int inj_col,
                                   float inj_delta, int form) {
  if (N <= 0) return cudaSuccess;
  const int Kp = ((N + TK - 1) / TK) * TK;
  char* p = static_cast<char*>(scratch);
  int* err = reinterpret_cast<int*>(p);
  uint16_t* a16 = reinterpret_cast<uint16_t*>(p + 256);
  uint16_t* bt16 = reinterpret_cast<uint16_t*>(p + 256 + align256((size_t)N * Kp * 2));
  const FrvFused f = frv_fused_layout(p + gemm_tc_scratch_bytes(N, N, N), N);
  prof_begin(prof, "cast_operands", s);
  cudaError_t e = launch_frv_vectors(f, N, nvec, seed, s);
  if (e != cudaSuccess) return e;
  const dim3 gb((N + kFrvStripeB - 1) / kFrvStripeB, Kp / 64);
  const dim3 ga(f.nsa, (N + 31) / 32);
  if (fp16) k_cast_bt_frv<true><<<gb, 256, 0, s>>>(B, N, Kp, bt16, f.r4, f.pb);
  else k_cast_bt_frv<false><<<gb, 256, 0, s>>>(B, N, Kp, bt16, f.r4, f.pb);
  e = launch_frv_b_reduce(f, N, s);
  if (e != cudaSuccess) return e;
  if (fp16) k_cast_a_frv<true><<<ga, 256, 0, s>>>(A, N, Kp, a16, f.br4, f.t4, f.pzq);
  else k_cast_a_frv<false><<<ga, 256, 0, s>>>(A, N, Kp, a16, f.br4, f.t4, f.pzq);
  prof_end(prof, s);
  prof_begin(prof, fp16 ? "gemm_tc_f16" : "gemm_tc_bf16", s);
  e = launch_product(a16, bt16, Kp, fp16, C, N, N, N, false, err, f.r4, f.pw, inj_row, inj_col,
                     inj_delta, s, form);
  prof_end(prof, s);
  if (e != cudaSuccess) return e;
  prof_begin(prof, "freivalds_fused", s);
  e = launch_frv_check_fused(f, N, nvec, c, u_eff, res, s);
  prof_end(prof, s);
  *kernels += 6;
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace sgk
