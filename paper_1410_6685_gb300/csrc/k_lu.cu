// k_lu.cu -- Gaussian elimination (Sec. 5, Listing 6 read as elimination with
// partial pivoting) and the solve with iterative refinement (sm_103a).
//
// Right-looking blocked LU, panels of 32 columns:
//   k_lu_panel_reg / k_lu_panel : a cluster of 16 CTAs (8 where the device
//                  cannot schedule 16) holds the panel (rows k..n-1) -- in
//                  registers (16 CTAs) or in shared memory (8 CTAs) -- and
//                  eliminates it column by column.  Each
//                  column costs one exchange: every CTA sends its best pivot
//                  candidate (largest |a|, then the lowest current row
//                  position) together with that row into every CTA's shared
//                  memory with asynchronous remote stores that complete on
//                  the receiver's mbarrier; once its barrier completes a CTA
//                  picks the winner, finds its row in its own shared memory,
//                  and updates its own rows while finding the next column's
//                  candidate.  No cluster-wide barrier per column.  Row
//                  interchanges are tracked as a replicated position table
//                  and applied when the panel is written back, so the result
//                  equals the row-swapping textbook algorithm.
//                  At the end it applies its interchanges to the rest of
//                  its 128-column outer block.
//   k_lu_inner   : inside the outer block, after each panel, the columns to
//                  its right: U12 = L11^-1 A12 and A22 -= L21 U12, one launch.
//   k_lu_laswp_outer : the outer block's interchanges on every other column.
//   k_lu_trsm_outer  : U12 = L11^-1 A12 for the outer block (128 rows), L11
//                  and a 32-column strip per CTA in shared memory.
//   trailing update A22 -= L21 U12 (K = 128) : the tensor-core product
//                  (bf16/fp16 operands, binary32 accumulate) or the binary32
//                  SIMT form.
// Solve: pivots on the right-hand side, then forward / backward substitution
// by steps of 128 rows in one launch each: CTAs take steps in order
// (ticket) and wait, with a bounded spin, for the steps they depend on; each
// step's diagonal block is applied through its inverse (assembled from the
// 64 x 64 inverses formed once per factorisation), one short product
// instead of 128 dependent steps.
// Refinement: residual r = b - A x in binary64 from the binary32 A, and the
// update x += d with the norms the stopping test needs.
#include <cooperative_groups.h>

#include "sg_lu.h"
#include "sg_linalg_kernels.h"

namespace cg = cooperative_groups;

namespace sgk {
namespace {

constexpr int kPB = 32;       // panel width
// CTAs per cluster (PC): 16 where the device schedules clusters of 16
// (non-portable size), else 8
constexpr int kPT = 256;      // threads per CTA
constexpr int kStride = kPB + 1;
constexpr unsigned kSpin = 1u << 24;

// Pivot candidate: larger |v| wins, then the lower current position; the
// low 16 bits carry the candidate's row within the panel so one 64-bit max
// says who won.  NaN magnitudes sort above everything.
__device__ __forceinline__ unsigned long long key_of(float v, int pos, int row) {
  return ((unsigned long long)__float_as_uint(fabsf(v)) << 32) |
         ((unsigned long long)(0xFFFFu - (unsigned)pos) << 16) | (unsigned)row;
}

// rows per thread for the largest n: ceil(ceil(kLuMaxN / PC) / kPT)
template <int PC>
__host__ __device__ constexpr int max_rows_per_thread() { return (kLuMaxN / PC + kPT - 1) / kPT; }
// bytes every CTA receives per column: PC candidates and PC candidate rows
template <int PC>
__host__ __device__ constexpr unsigned col_bytes() { return PC * (8 + kPB * 4); }

__device__ __forceinline__ uint32_t sm_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// the same shared-memory offset in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cl_addr(uint32_t local, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
// asynchronous remote stores that complete bytes on the receiver's mbarrier
__device__ __forceinline__ void st_async_b64(uint32_t raddr, unsigned long long v, uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];"
               ::"r"(raddr), "l"(v), "r"(rbar) : "memory");
}
__device__ __forceinline__ void st_async_v4(uint32_t raddr, float4 v, uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];"
               ::"r"(raddr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(rbar) : "memory");
}
// bounded wait for phase `parity` of a local mbarrier
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  for (unsigned i = 0; i < kSpin; ++i) {
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
  return false;
}

// the outer block's columns outside the panel, per cluster CTA (PC >= 8)
constexpr int kXCols = (kLuOuter - kPB + 7) / 8;

// smem: slab[rs][33] floats, cand[2][PC] u64, best[2] u64, bar[2] u64,
// crow[2][PC][32] floats, xbuf[64][kXCols] floats, fpos[rs] ints
template <int PC>
__global__ void __launch_bounds__(kPT)
    k_lu_panel(float* __restrict__ LU, int n, int k, int jb, int* __restrict__ piv,
               int* __restrict__ info, int* __restrict__ moves, int c_lo, int c_hi) {
  constexpr int kRows = max_rows_per_thread<PC>();
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int m = n - k;
  const int rs = (m + PC - 1) / PC;
  const int r0 = rank * rs;
  const int r1 = min(m, r0 + rs);
  float* slab = reinterpret_cast<float*>(smem);
  unsigned long long* cand = reinterpret_cast<unsigned long long*>(
      (reinterpret_cast<uintptr_t>(slab + (size_t)rs * kStride) + 15) & ~(uintptr_t)15);
  unsigned long long* best = cand + 2 * PC;
  unsigned long long* bar = best + 2;
  // crow[par][q][c]: CTA q's candidate row for the column of parity par
  float* crow = reinterpret_cast<float*>(bar + 2);
  // xbuf[t][i]: moved row t of this CTA's i-th outer-block column
  float* xbuf = crow + 2 * PC * kPB;
  // fpos[r]: final position of this CTA's row r (for the write-back)
  int* fpos = reinterpret_cast<int*>(xbuf + 2 * kPB * kXCols);
  const int tid = threadIdx.x;
  const int lane = tid & 31;

  // my rows: r = r0 + tid + i*kPT; their current positions live in registers
  int lp[kRows];
#pragma unroll
  for (int i = 0; i < kRows; ++i) lp[i] = r0 + tid + i * kPT;
  // the slab, eight loads in flight per thread (a warp reads one row per load)
  const int total = (r1 - r0) * kPB;
  for (int base = 0; base < total; base += 8 * kPT) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int t = base + u * kPT + tid, r = t >> 5, c = t & 31;
      v[u] = (t < total && c < jb) ? __ldg(LU + (size_t)(k + r0 + r) * n + k + c) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int t = base + u * kPT + tid;
      if (t < total) slab[(t >> 5) * kStride + (t & 31)] = v[u];
    }
  }
  if (tid < 2) {
    best[tid] = 0ull;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sm_addr(&bar[tid])) : "memory");
  }
  if (tid == 0) asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  // every CTA's barriers exist before anyone sends
  cluster.sync();
  // the first column's candidate
  unsigned long long mine = 0ull;
#pragma unroll
  for (int i = 0; i < kRows; ++i) {
    const int r = r0 + tid + i * kPT;
    if (r < r1) {
      const unsigned long long kk = key_of(slab[(r - r0) * kStride], lp[i], r);
      mine = kk > mine ? kk : mine;
    }
  }
  int my_info = 0;
  bool failed = false;
  for (int j = 0; j < jb; ++j) {
    const int par = j & 1;
    const uint32_t mbar = sm_addr(&bar[par]);
    // this CTA's best candidate for column j
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long u = __shfl_xor_sync(0xffffffffu, mine, o);
      mine = u > mine ? u : mine;
    }
    if (lane == 0 && mine) atomicMax(&best[par], mine);
    if (tid == 0)   // this column's bytes from the cluster complete bar[par]
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar),
                   "r"(col_bytes<PC>()) : "memory");
    __syncthreads();
    // send the candidate and its row (the pivot row, should it win) to every
    // CTA of the cluster; the stores complete on the receivers' bar[par].
    // A CTA sends column j + 2 only after it has all of column j + 1, which
    // every CTA sends only after reading column j: two slots suffice.
    const unsigned long long bmine = best[par];
    if (tid < PC) {
      st_async_b64(cl_addr(sm_addr(&cand[par * PC + rank]), tid), bmine, cl_addr(mbar, tid));
    } else if (tid >= 32 && tid < 32 + kPB * PC / 4) {
      const int q = (tid - 32) / (kPB / 4), cq = ((tid - 32) % (kPB / 4)) * 4;
      const int lr = bmine ? (int)(bmine & 0xFFFFu) - r0 : 0;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (bmine) {
        v.x = (cq >= j && cq < jb) ? slab[lr * kStride + cq] : 0.0f;
        v.y = (cq + 1 >= j && cq + 1 < jb) ? slab[lr * kStride + cq + 1] : 0.0f;
        v.z = (cq + 2 >= j && cq + 2 < jb) ? slab[lr * kStride + cq + 2] : 0.0f;
        v.w = (cq + 3 >= j && cq + 3 < jb) ? slab[lr * kStride + cq + 3] : 0.0f;
      }
      st_async_v4(cl_addr(sm_addr(&crow[(par * PC + rank) * kPB + cq]), q), v, cl_addr(mbar, q));
    }
    if (tid == PC) best[par ^ 1] = 0ull;   // next column's slot (its last reader is done)
    if (!bar_wait(mbar, (uint32_t)(j >> 1) & 1u)) {
      failed = true;
      break;
    }
    unsigned long long g = 0ull;
    int wq = 0;
#pragma unroll
    for (int q = 0; q < PC; ++q) {
      const unsigned long long cq = cand[par * PC + q];
      if (cq > g) { g = cq; wq = q; }
    }
    const int p = (int)(0xFFFFu - (unsigned)((g >> 16) & 0xFFFFu));   // winning position
    const int gp = (int)(g & 0xFFFFu);                                // its row in the panel
    const float* prow = crow + (par * PC + wq) * kPB;
    // interchange of positions j and p (each thread for its own rows)
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
      const int r = r0 + tid + i * kPT;
      if (lp[i] == j) lp[i] = p;
      if (r == gp) lp[i] = j;
    }
    const float d = prow[j];
    const bool zero = d == 0.0f;
    if (zero && my_info == 0) my_info = k + j + 1;
    const float rd = 1.0f / d;
    // eliminate below the pivot; find the next column's candidate
    mine = 0ull;
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
      const int r = r0 + tid + i * kPT;
      if (r >= r1 || lp[i] <= j) continue;
      float* row = slab + (r - r0) * kStride;
      if (!zero) {
        const float l = row[j] * rd;   // a product with the reciprocal, as in the register form
        row[j] = l;
        for (int c = j + 1; c < jb; ++c) row[c] = fmaf(-l, prow[c], row[c]);
      }
      if (j + 1 < jb) {
        const unsigned long long kk = key_of(row[j + 1], lp[i], r);
        mine = kk > mine ? kk : mine;
      }
    }
    if (tid == 0 && rank == 0) piv[k + j] = k + p;
  }
  if (failed) atomicCAS(info, 0, -1);   // a wait gave up: report, write nothing
  const bool any_failed = __syncthreads_or(failed);
  cluster.sync();   // no CTA reads another's shared memory after this
  // list the rows that moved (at most 2 jb) for the other columns'
  // interchange; keep every row's final position for the write-back
  if (!any_failed) {
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
      const int r = r0 + tid + i * kPT;
      if (r >= r1) continue;
      fpos[r - r0] = lp[i];
      if (lp[i] != r) {
        const int t = atomicAdd(&moves[0], 1);
        if (t < 2 * kPB) {
          moves[1 + t] = k + r;
          moves[1 + 2 * kPB + t] = k + lp[i];
        }
      }
    }
  }
  __syncthreads();
  // write the panel back in its final row order, one row per warp store
  if (!any_failed) {
    for (int t = tid; t < total; t += kPT) {
      const int r = t >> 5, c = t & 31;
      if (c < jb) LU[(size_t)(k + fpos[r]) * n + k + c] = slab[r * kStride + c];
    }
  }
  if (tid == 0 && rank == 0 && my_info) atomicCAS(info, 0, my_info);
  cluster.sync();   // every CTA's moves are listed
  // the interchanges on the outer block's other columns [c_lo, k) and
  // [k + jb, c_hi) (at most kXCols * PC): CTA `rank` takes the columns
  // rank, rank + PC, ...; all their moved rows are read into shared memory
  // before any is written
  const int nl = k - c_lo, nc = nl + (c_hi - k - jb);
  const int nci = nc > rank ? (nc - rank + PC - 1) / PC : 0;
  if (!any_failed && nci > 0) {
    const int cnt = min(moves[0], 2 * kPB);
    for (int e = tid; e < cnt * nci; e += kPT) {
      const int t = e / nci, i = e % nci, g = rank + i * PC;
      const int c = g < nl ? c_lo + g : k + jb + (g - nl);
      xbuf[t * kXCols + i] = LU[(size_t)moves[1 + t] * n + c];
    }
    __syncthreads();
    for (int e = tid; e < cnt * nci; e += kPT) {
      const int t = e / nci, i = e % nci, g = rank + i * PC;
      const int c = g < nl ? c_lo + g : k + jb + (g - nl);
      LU[(size_t)moves[1 + 2 * kPB + t] * n + c] = xbuf[t * kXCols + i];
    }
  }
}

// The 16-CTA panel with each thread's rows in registers.  Shared memory
// traffic bounds the slab form above at large heights: every column reads
// and writes the whole remaining panel there.  Here a thread keeps its rows
// (at most kRows of them) as 32 registers each, in a layout shifted by one
// per column: at step j, register c of a row holds column j + c, so every
// register index is a compile-time constant although j is not.  An L entry
// goes to shared memory (lbuf, stride 33) when it is formed; a row chosen as
// the pivot writes its U part there and retires.  Per column: each warp's
// best candidate (two redux.sync maxima: magnitude, then position and row)
// stages its row (in the same shifted layout); one CTA barrier; every
// thread finds the CTA's best among the warps' keys by a lane-parallel
// maximum; the CTA's key and staged row go to every CTA of the cluster by
// asynchronous remote stores (as in the slab form); the cluster's winner is
// again a lane-parallel maximum, and its row arrives pre-shifted.  Once the
// pivot row is known a row forms its multiplier and only its next column
// (the next candidate); the rest of its update is done while the next
// exchange is in flight (a warp's winner completes its own row first, since
// that row is staged and sent).  The interchanges, the zero-pivot rule and
// the write-back are the slab form's.  KR: row slots per thread (2 when a
// CTA holds at most 2 kPT rows: fewer registers, measured 6% faster).
template <int PC, int KR>
__global__ void __launch_bounds__(kPT, 1)
    k_lu_panel_reg(float* __restrict__ LU, int n, int k, int jb, int* __restrict__ piv,
                   int* __restrict__ info, int* __restrict__ moves, int c_lo, int c_hi) {
  constexpr int kRows = KR;
  constexpr int kW = kPT / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int m = n - k;
  const int rs = (m + PC - 1) / PC;
  const int r0 = rank * rs;
  const int r1 = min(m, r0 + rs);
  float* lbuf = reinterpret_cast<float*>(smem);   // [rs][kStride]: the slab, then L\U
  float* stage = reinterpret_cast<float*>(
      (reinterpret_cast<uintptr_t>(lbuf + (size_t)rs * kStride) + 15) & ~(uintptr_t)15);  // [2][kW][32]
  float* crow = stage + 2 * kW * kPB;                                                    // [2][PC][32]
  unsigned long long* wkey = reinterpret_cast<unsigned long long*>(crow + 2 * PC * kPB);  // [2][kW]
  unsigned long long* cand = wkey + 2 * kW;                                              // [2][PC]
  unsigned long long* bar = cand + 2 * PC;                                               // [2]
  float* xbuf = reinterpret_cast<float*>(bar + 2);                                       // [2 kPB][kXCols]
  int* fpos = reinterpret_cast<int*>(xbuf + 2 * kPB * kXCols);                           // [rs]
  const int tid = threadIdx.x;
  const int lane = tid & 31, w = tid >> 5;

  const int total = (r1 - r0) * kPB;
  // my rows: r = r0 + tid + i * kPT, loaded whole into registers with every
  // load of the thread in flight at once (float4 where the rows start on 16
  // bytes); lbuf only receives the L and U entries as they form
  float x[kRows][kPB];
  float lr[kRows];       // a row's pending multiplier (0 after a zero pivot)
  int lp[kRows];
  bool act[kRows], pend[kRows];
  float pv[kPB];         // the last pivot row, shifted (pv[c] is column j + c of its step)
#pragma unroll
  for (int c = 0; c < kPB; ++c) pv[c] = 0.0f;
  const bool vec = ((n | k) & 3) == 0;   // then jb is a multiple of 4 too
#pragma unroll
  for (int i = 0; i < kRows; ++i) {
    const int r = r0 + tid + i * kPT;
    lp[i] = r;
    act[i] = r < r1;
    pend[i] = false;
    lr[i] = 0.0f;
    const float* src = LU + (size_t)(k + (act[i] ? r : 0)) * n + k;
    if (vec) {
#pragma unroll
      for (int q = 0; q < kPB / 4; ++q) {
        const float4 v = act[i] && 4 * q < jb ? __ldg(reinterpret_cast<const float4*>(src) + q)
                                              : make_float4(0.f, 0.f, 0.f, 0.f);
        x[i][4 * q] = v.x; x[i][4 * q + 1] = v.y; x[i][4 * q + 2] = v.z; x[i][4 * q + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int c = 0; c < kPB; ++c) x[i][c] = act[i] && c < jb ? __ldg(src + c) : 0.0f;
    }
  }
  if (tid < 2) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sm_addr(&bar[tid])) : "memory");
  if (tid == 0) asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  // every CTA's barriers exist before anyone sends
  cluster.sync();
  // the deferred part of a row's update: registers 1..30 of the shifted row
  // (register 0, the next column, was updated when the multiplier was formed).
  // After a zero pivot the multiplier and the pivot row are +0, and
  // x + (-0)(+0) = x for every x (signed zeros, infinities, NaN): the row is
  // only shifted, as the zero-pivot rule wants, without a select per entry.
  auto finish = [&](int i) {
#pragma unroll
    for (int c = 1; c + 1 < kPB; ++c) x[i][c] = fmaf(-lr[i], pv[c + 1], x[i][c + 1]);
    x[i][kPB - 1] = 0.0f;
    pend[i] = false;
  };
  int my_info = 0;
  bool failed = false;
  for (int j = 0; j < jb; ++j) {
    const int par = j & 1;
    const uint32_t mbar = sm_addr(&bar[par]);
    // this thread's and this warp's best candidate for column j (register 0)
    unsigned long long mine = 0ull;
    int mi = -1;
#pragma unroll
    for (int i = 0; i < kRows; ++i)
      if (act[i]) {
        const unsigned long long kk = key_of(x[i][0], lp[i], r0 + tid + i * kPT);
        if (kk > mine) { mine = kk; mi = i; }
      }
    const unsigned mh = __reduce_max_sync(0xffffffffu, (unsigned)(mine >> 32));
    const unsigned ml = __reduce_max_sync(0xffffffffu, (unsigned)(mine >> 32) == mh ? (unsigned)mine : 0u);
    const unsigned long long wk = ((unsigned long long)mh << 32) | ml;
    // the warp's winner completes and stages its row (keys carry the row:
    // the winner is unique)
    if (wk != 0ull && mine == wk) {
      float4* st = reinterpret_cast<float4*>(stage + (par * kW + w) * kPB);
#pragma unroll
      for (int i = 0; i < kRows; ++i)
        if (i == mi) {
          if (pend[i]) finish(i);
#pragma unroll
          for (int q = 0; q < kPB / 4; ++q)
            st[q] = make_float4(x[i][4 * q], x[i][4 * q + 1], x[i][4 * q + 2], x[i][4 * q + 3]);
        }
    }
    if (lane == 0) wkey[par * kW + w] = wk;
    if (tid == 0)   // this column's bytes from the cluster complete bar[par]
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar),
                   "r"(col_bytes<PC>()) : "memory");
    __syncthreads();
    // the CTA's best: lane q looks at warp q's key
    unsigned long long b;
    int bw;
    {
      const unsigned long long u = lane < kW ? wkey[par * kW + lane] : 0ull;
      const unsigned uh = (unsigned)(u >> 32);
      const unsigned bh = __reduce_max_sync(0xffffffffu, uh);
      const unsigned bl = __reduce_max_sync(0xffffffffu, uh == bh ? (unsigned)u : 0u);
      b = ((unsigned long long)bh << 32) | bl;
      const unsigned hit = __ballot_sync(0xffffffffu, b != 0ull && u == b);
      bw = hit ? __ffs(hit) - 1 : 0;
    }
    // send the key and its row to every CTA of the cluster; the stores
    // complete on the receivers' bar[par].  A CTA sends column j + 2 only
    // after it has all of column j + 1, which every CTA sends only after
    // reading column j: two slots suffice (for stage too).
    if (tid < PC) {
      st_async_b64(cl_addr(sm_addr(&cand[par * PC + rank]), tid), b, cl_addr(mbar, tid));
    } else if (tid >= 32) {
      const float4* srow = reinterpret_cast<const float4*>(stage + (par * kW + bw) * kPB);
      for (int e = tid - 32; e < PC * (kPB / 4); e += kPT - 32) {
        const int q = e / (kPB / 4), part = e % (kPB / 4);
        st_async_v4(cl_addr(sm_addr(&crow[(par * PC + rank) * kPB + 4 * part]), q),
                    b ? srow[part] : make_float4(0.f, 0.f, 0.f, 0.f), cl_addr(mbar, q));
      }
    }
    // the deferred updates, while the exchange is in flight
#pragma unroll
    for (int i = 0; i < kRows; ++i)
      if (pend[i]) finish(i);
    // after a wait gave up nothing is written back; later columns do not wait
    if (!failed && !bar_wait(mbar, (uint32_t)(j >> 1) & 1u)) failed = true;
    unsigned long long g;
    int wq;
    {
      const unsigned long long u = lane < PC ? cand[par * PC + lane] : 0ull;
      const unsigned uh = (unsigned)(u >> 32);
      const unsigned gh = __reduce_max_sync(0xffffffffu, uh);
      const unsigned gl = __reduce_max_sync(0xffffffffu, uh == gh ? (unsigned)u : 0u);
      g = ((unsigned long long)gh << 32) | gl;
      const unsigned hit = __ballot_sync(0xffffffffu, g != 0ull && u == g);
      wq = hit ? __ffs(hit) - 1 : 0;
    }
    const int p = (int)(0xFFFFu - (unsigned)((g >> 16) & 0xFFFFu));   // winning position
    const int gp = (int)(g & 0xFFFFu);                                // its row in the panel
    // the pivot row, shifted: pv[c] is column j + c (every pending update,
    // which used the previous one, is done)
    {
      const float4* pr = reinterpret_cast<const float4*>(crow + (par * PC + wq) * kPB);
#pragma unroll
      for (int q = 0; q < kPB / 4; ++q) {
        const float4 v = pr[q];
        pv[4 * q] = v.x; pv[4 * q + 1] = v.y; pv[4 * q + 2] = v.z; pv[4 * q + 3] = v.w;
      }
    }
    const float d = pv[0];
    const bool pzero = d == 0.0f;
    if (pzero) {
#pragma unroll
      for (int c = 0; c < kPB; ++c) pv[c] = 0.0f;
    }
    if (pzero && my_info == 0) my_info = k + j + 1;
    const float rd = 1.0f / d;
    // interchange of positions j and p; the pivot row writes its U part
    // (columns j..jb-1) and retires
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
      const int r = r0 + tid + i * kPT;
      if (lp[i] == j) lp[i] = p;
      if (act[i] && r == gp) {
        lp[i] = j;
        act[i] = false;
        float* dst = lbuf + (r - r0) * kStride + j;
#pragma unroll
        for (int c = 0; c < kPB; ++c)
          if (c < jb - j) dst[c] = x[i][c];
      }
    }
    // eliminate below the pivot: l = a_ij / u_jj (as a product with the
    // reciprocal); register 0 becomes the next column now, the rest of the
    // shifted update waits for the next exchange
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
      if (!act[i]) continue;
      const int r = r0 + tid + i * kPT;
      const float l = pzero ? x[i][0] : x[i][0] * rd;
      lbuf[(r - r0) * kStride + j] = l;
      lr[i] = pzero ? 0.0f : l;
      x[i][0] = fmaf(-lr[i], pv[1], x[i][1]);
      pend[i] = true;
    }
    if (tid == 0 && rank == 0) piv[k + j] = k + p;
  }
  if (failed) atomicCAS(info, 0, -1);   // a wait gave up: report, write nothing
  const bool any_failed = __syncthreads_or(failed);
  cluster.sync();   // no CTA reads another's shared memory after this
  // list the rows that moved (at most 2 jb) for the other columns'
  // interchange; keep every row's final position for the write-back
  if (!any_failed) {
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
      const int r = r0 + tid + i * kPT;
      if (r >= r1) continue;
      fpos[r - r0] = lp[i];
      if (lp[i] != r) {
        const int t = atomicAdd(&moves[0], 1);
        if (t < 2 * kPB) {
          moves[1 + t] = k + r;
          moves[1 + 2 * kPB + t] = k + lp[i];
        }
      }
    }
  }
  __syncthreads();
  // write the panel back in its final row order, one row per warp store
  if (!any_failed) {
    for (int t = tid; t < total; t += kPT) {
      const int r = t >> 5, c = t & 31;
      if (c < jb) LU[(size_t)(k + fpos[r]) * n + k + c] = lbuf[r * kStride + c];
    }
  }
  if (tid == 0 && rank == 0 && my_info) atomicCAS(info, 0, my_info);
  cluster.sync();   // every CTA's moves are listed
  // the interchanges on the outer block's other columns, as in the slab form
  const int nl = k - c_lo, nc = nl + (c_hi - k - jb);
  const int nci = nc > rank ? (nc - rank + PC - 1) / PC : 0;
  if (!any_failed && nci > 0) {
    const int cnt = min(moves[0], 2 * kPB);
    for (int e = tid; e < cnt * nci; e += kPT) {
      const int t = e / nci, i = e % nci, gg = rank + i * PC;
      const int c = gg < nl ? c_lo + gg : k + jb + (gg - nl);
      xbuf[t * kXCols + i] = LU[(size_t)moves[1 + t] * n + c];
    }
    __syncthreads();
    for (int e = tid; e < cnt * nci; e += kPT) {
      const int t = e / nci, i = e % nci, gg = rank + i * PC;
      const int c = gg < nl ? c_lo + gg : k + jb + (gg - nl);
      LU[(size_t)moves[1 + 2 * kPB + t] * n + c] = xbuf[t * kXCols + i];
    }
  }
}

// The interchanges of an outer block's panels (moves lists m0, m0 + 1, ...,
// in order) on the columns outside it, [0, K) and [K + KB, n), and on the
// row permutation perm: one thread per column; for each list every load of
// the column precedes its stores.
__global__ void __launch_bounds__(128) k_lu_laswp_outer(float* LU, int n, const int* __restrict__ moves,
                                                        int nlists, int K, int KB, int* perm) {
  __shared__ int s_cnt[kLuOuter / kPB], s_src[kLuOuter / kPB][2 * kPB],
      s_dst[kLuOuter / kPB][2 * kPB];
  for (int q = 0; q < nlists; ++q) {
    const int* m = moves + (size_t)q * kLuMoveInts;
    const int cnt = min(m[0], 2 * kPB);
    if (threadIdx.x == 0) s_cnt[q] = cnt;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      s_src[q][t] = m[1 + t];
      s_dst[q][t] = m[1 + 2 * kPB + t];
    }
  }
  __syncthreads();
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g == n - KB) {
    // one more column: the row permutation itself
    for (int q = 0; q < nlists; ++q) {
      const int cnt = s_cnt[q];
      int v[2 * kPB];
#pragma unroll
      for (int t = 0; t < 2 * kPB; ++t)
        if (t < cnt) v[t] = perm[s_src[q][t]];
#pragma unroll
      for (int t = 0; t < 2 * kPB; ++t)
        if (t < cnt) perm[s_dst[q][t]] = v[t];
    }
    return;
  }
  const int c = g < K ? g : g + KB;
  if (c >= n) return;
  for (int q = 0; q < nlists; ++q) {
    const int cnt = s_cnt[q];
    float v[2 * kPB];
#pragma unroll
    for (int t = 0; t < 2 * kPB; ++t)
      if (t < cnt) v[t] = LU[(size_t)s_src[q][t] * n + c];
#pragma unroll
    for (int t = 0; t < 2 * kPB; ++t)
      if (t < cnt) LU[(size_t)s_dst[q][t] * n + c] = v[t];
  }
}

// x := L^-1 x for one column x of 32 entries (stride xs) and the unit lower
// triangle of L (row stride ls, a multiple of 4; L 16-byte aligned), by
// forward substitution in registers: row i subtracts L[i][0] x[0], L[i][1]
// x[1], ... in that order, reading L's row four entries per shared-memory
// load.
__device__ __forceinline__ void unit_lower_solve_col4(const float* L, int ls, float* x, int xs) {
  float v[kPB];
#pragma unroll
  for (int i = 0; i < kPB; ++i) v[i] = x[i * xs];
#pragma unroll
  for (int i = 1; i < kPB; ++i) {
    float acc = v[i];
    const float4* Li = reinterpret_cast<const float4*>(L + i * ls);
#pragma unroll
    for (int g = 0; g < i / 4; ++g) {
      const float4 l = Li[g];
      acc = fmaf(-l.x, v[4 * g], acc);
      acc = fmaf(-l.y, v[4 * g + 1], acc);
      acc = fmaf(-l.z, v[4 * g + 2], acc);
      acc = fmaf(-l.w, v[4 * g + 3], acc);
    }
#pragma unroll
    for (int q = (i / 4) * 4; q < i; ++q) acc = fmaf(-L[i * ls + q], v[q], acc);
    v[i] = acc;
  }
#pragma unroll
  for (int i = 1; i < kPB; ++i) x[i * xs] = v[i];
}

// After panel j inside an outer block, for its columns [c0, c1) to the right
// of the panel (at most kLuOuter - kPB):
//   U12 = L11^-1 A12 (rows j..j+32; L11 the panel's unit lower triangle)
//   A22 -= L21 U12   (rows j+32..n)
// Each CTA solves U12 in shared memory (one thread per column) and updates
// kInRows rows of A22.  U12 replaces A12 in LU only after every
// CTA has read A12: the CTA that counts last on `counter` (zero before the
// launch) writes it.
constexpr int kInRows = 32;
constexpr int kInCols = kLuOuter - kPB;
__global__ void __launch_bounds__(256) k_lu_inner(float* LU, int n, int j, int c0, int c1,
                                                  unsigned* counter) {
  // rows of L and P padded to 36 floats: 16-byte loads of four entries
  __shared__ __align__(16) float L[kPB][kPB + 4];
  __shared__ float U[kPB][kInCols + 1];
  __shared__ __align__(16) float P[kInRows][kPB + 4];
  __shared__ bool s_last;
  const int tid = threadIdx.x;
  const int N = c1 - c0;
  const int rb = j + kPB + blockIdx.x * kInRows;
  const int nr = min(kInRows, n - rb);
  const int lane = tid & 31, w = tid >> 5;
  // staging: every thread issues all its loads before its shared stores;
  // thread (w, lane) owns rows w + 8 i (i < 4) and columns lane + 32 u (u < 3)
  {
    float l4[4], p4[4], u12[12];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = w + 8 * i;
      l4[i] = __ldg(LU + (size_t)(j + r) * n + j + lane);
      p4[i] = r < nr ? __ldg(LU + (size_t)(rb + r) * n + j + lane) : 0.0f;
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int c = lane + 32 * u;
        u12[i * 3 + u] = c < N ? __ldg(LU + (size_t)(j + r) * n + c0 + c) : 0.0f;
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = w + 8 * i;
      L[r][lane] = l4[i];
      P[r][lane] = p4[i];
#pragma unroll
      for (int u = 0; u < 3; ++u) U[r][lane + 32 * u] = u12[i * 3 + u];
    }
  }
  // this thread's A22 entries, loaded while U12 is solved
  float acc[12];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int r = w + 8 * i, c = lane + 32 * u;
      acc[i * 3 + u] = (r < nr && c < N) ? LU[(size_t)(rb + r) * n + c0 + c] : 0.0f;
    }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  if (tid < N) unit_lower_solve_col4(&L[0][0], kPB + 4, &U[0][tid], kInCols + 1);
  __syncthreads();
  if (s_last)
    for (int t = tid; t < kPB * N; t += 256) LU[(size_t)(j + t / N) * n + c0 + t % N] = U[t / N][t % N];
  // A22 -= L21 U12: twelve independent chains per thread, each over q in
  // order; four entries of each of the thread's P rows per load
#pragma unroll 2
  for (int q = 0; q < kPB; q += 4) {
    float4 p4[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) p4[i] = *reinterpret_cast<const float4*>(&P[w + 8 * i][q]);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float uq[3];
#pragma unroll
      for (int u = 0; u < 3; ++u) uq[u] = U[q + e][lane + 32 * u];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float pq = e == 0 ? p4[i].x : e == 1 ? p4[i].y : e == 2 ? p4[i].z : p4[i].w;
#pragma unroll
        for (int u = 0; u < 3; ++u) acc[i * 3 + u] = fmaf(-pq, uq[u], acc[i * 3 + u]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int r = w + 8 * i, c = lane + 32 * u;
      if (r < nr && c < N) LU[(size_t)(rb + r) * n + c0 + c] = acc[i * 3 + u];
    }
}

// Rows [K, K + KB) of columns [c0, c1) := L11^-1 (them), L11 the unit lower
// triangle of the KB x KB diagonal block at (K, K) (KB a multiple of 32, at
// most kLuOuter).  One CTA per 32 columns with L11 and its strip in shared
// memory; by 32-row blocks: the diagonal block solved one thread per column,
// then the rows below it updated by all threads.
__global__ void __launch_bounds__(256, 2) k_lu_trsm_outer(float* LU, int n, int K, int KB,
                                                          int c0, int c1) {
  extern __shared__ __align__(16) float sm_t[];
  const int ls = KB + 4;         // rows padded to a multiple of 4: 16-byte loads
  float* L = sm_t;               // KB x (KB + 4)
  float* X = sm_t + KB * ls;     // KB x 33
  const int tid = threadIdx.x;
  const int cb = c0 + blockIdx.x * kPB;
  const int nc = min(kPB, c1 - cb);
  const int lane = tid & 31, w = tid >> 5;
  // staging, eight loads in flight per thread before their shared stores:
  // warp w takes rows w, w + 8, ...; lane the column (of L11: lane + 32 u)
  for (int r0 = 0; r0 < KB; r0 += 32) {
    float v[4][4], x[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + w + 8 * i;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = lane + 32 * u;
        v[i][u] = (c < r) ? __ldg(LU + (size_t)(K + r) * n + K + c) : 0.0f;
      }
      x[i] = lane < nc ? __ldg(LU + (size_t)(K + r) * n + cb + lane) : 0.0f;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + w + 8 * i;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (lane + 32 * u < KB) L[r * ls + lane + 32 * u] = v[i][u];
      X[r * 33 + lane] = x[i];
    }
  }
  __syncthreads();
  for (int b = 0; b < KB; b += kPB) {
    if (tid < kPB) unit_lower_solve_col4(L + b * ls + b, ls, X + b * 33 + tid, 33);
    __syncthreads();
    // rows below: warp w takes rows b + 32 + w + 8 i, lane the column;
    // independent chains over q in order
    const int below = KB - b - kPB;
    float acc[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      const int r = b + kPB + w + 8 * i;
      acc[i] = (w + 8 * i < below) ? X[r * 33 + lane] : 0.0f;
    }
#pragma unroll 2
    for (int q = 0; q < kPB; q += 4) {
      float xq[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) xq[e] = X[(b + q + e) * 33 + lane];
#pragma unroll
      for (int i = 0; i < 12; ++i) {
        const int r = b + kPB + w + 8 * i;
        if (w + 8 * i < below) {
          const float4 l = *reinterpret_cast<const float4*>(L + r * ls + b + q);
          acc[i] = fmaf(-l.x, xq[0], acc[i]);
          acc[i] = fmaf(-l.y, xq[1], acc[i]);
          acc[i] = fmaf(-l.z, xq[2], acc[i]);
          acc[i] = fmaf(-l.w, xq[3], acc[i]);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      const int r = b + kPB + w + 8 * i;
      if (w + 8 * i < below) X[r * 33 + lane] = acc[i];
    }
    __syncthreads();
  }
  for (int t = tid; t < KB * kPB; t += 256) {
    const int r = t >> 5, c = t & 31;
    if (c < nc) LU[(size_t)(K + r) * n + cb + c] = X[r * 33 + c];
  }
}

// ---------------------------------------------------------------------------
// solve

// perm[i] = i (the interchanges are then applied to it like a column)
__global__ void k_lu_iota(int* perm, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) perm[i] = i;
}

// y = P rhs (binary64 in, binary32 out): y[i] = rhs[perm[i]]
__global__ void k_apply_perm(const double* __restrict__ rhs, float* y, int n,
                             const int* __restrict__ perm) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    y[i] = (float)rhs[perm[i]];
}

// Inverses of the 64x64 diagonal blocks of L (unit lower) and U (upper),
// once per factorisation, for the blocked substitutions: inv[0][b] = L_bb^-1,
// inv[1][b] = U_bb^-1, row-major; a block cut by n is padded with the
// identity.  One CTA per block: thread j < 64 forms column j of L_bb^-1 by
// forward substitution, thread 64 + j column j of U_bb^-1 by back
// substitution, both in registers.
constexpr int kTB = 64;   // rows of a substitution block
__global__ void __launch_bounds__(2 * kTB) k_lu_diag_inv(const float* __restrict__ LU, int n,
                                                         float* __restrict__ inv) {
  __shared__ float D[kTB][kTB + 1];
  const int b = blockIdx.x, row0 = b * kTB, tid = threadIdx.x;
  for (int t = tid; t < kTB * kTB; t += 2 * kTB) {
    const int r = t / kTB, c = t % kTB;
    D[r][c] = (row0 + r < n && row0 + c < n) ? LU[(size_t)(row0 + r) * n + row0 + c]
                                             : (r == c ? 1.0f : 0.0f);
  }
  __syncthreads();
  const int nb = gridDim.x;
  const int j = tid % kTB;
  float x[kTB];
  if (tid < kTB) {
#pragma unroll
    for (int i = 0; i < kTB; ++i) {
      float acc = i == j ? 1.0f : 0.0f;
#pragma unroll
      for (int q = 0; q < i; ++q) acc = fmaf(-D[i][q], x[q], acc);
      x[i] = acc;
    }
#pragma unroll
    for (int i = 0; i < kTB; ++i) inv[((size_t)b * kTB + i) * kTB + j] = x[i];
  } else {
#pragma unroll
    for (int i = kTB - 1; i >= 0; --i) {
      float acc = i == j ? 1.0f : 0.0f;
#pragma unroll
      for (int q = i + 1; q < kTB; ++q) acc = fmaf(-D[i][q], x[q], acc);
      x[i] = acc / D[i][i];
    }
#pragma unroll
    for (int i = 0; i < kTB; ++i) inv[((size_t)(nb + b) * kTB + i) * kTB + j] = x[i];
  }
}

// Triangular solve by steps of 128 rows (two 64-row blocks).  LOWER: unit
// lower L, steps in increasing order; else upper U with its diagonal, in
// decreasing order.  Each step first forms, in shared memory, the inverse of
// its 128 x 128 diagonal block from the two 64 x 64 inverses: with f the
// block solved first (the upper one for L, the lower one for U), s the
// other and X the rows of s over the columns of f, the inverse holds f's and
// s's inverses on its diagonal and -inv_s X inv_f in place of X.  This is
// done while earlier steps run, and each thread then keeps a 32-column
// quarter of one row of it in registers.  A step's 128 rows form four
// groups of 32, four warps per group sharing the step's dependencies in
// 32-column pieces (warp q of a group takes every fourth, in the order they
// are solved), each loading its piece row by row, coalesced (lane =
// column), before waiting, with a bounded spin, for the flag of the step the
// piece belongs to; one transposing warp reduction then gives lane r the sum
// of row r.  The right-hand sides minus those sums times the inverse give
// the step's solution, published with one flag (a release store).  The
// chain of global waits from step to step (a few microseconds each, the
// same at every size) bounds the solve.
constexpr int kRB = 2 * kTB;         // rows of a step
constexpr int kTrsvThreads = 512;
constexpr int kTS = kTB + 1;         // shared row strides (conflict-free lane = row reads)
constexpr int kRS = kRB + 1;
constexpr size_t kTrsvSmem =
    (kRB * kRS + 2 * kTB * kTS + (kTrsvThreads / 32) * 32 + kRB + 4 * kRB) * sizeof(float) + 16;
template <bool LOWER>
__global__ void __launch_bounds__(kTrsvThreads, 1) k_trsv(const float* __restrict__ LU,
                                                          const float* __restrict__ inv, int n,
                                                          float* y, unsigned* flags,
                                                          unsigned epoch, unsigned* ticket,
                                                          int* err) {
  extern __shared__ float tsm[];
  float* ib = tsm;                                     // [kRB][kRS] the step's inverse
  float* xa = ib + kRB * kRS;                          // [kTB][kTS] X
  float* xb = xa + kTB * kTS;                          // [kTB][kTS] X inv_f
  float* part = xb + kTB * kTS;                        // [16][32]
  float* vsh = part + (kTrsvThreads / 32) * 32;        // [kRB]
  float* xp = vsh + kRB;                               // [4][kRB] quarter sums
  unsigned* s_b = reinterpret_cast<unsigned*>(xp + 4 * kRB);
  const int tid = threadIdx.x;
  const int nb = (n + kTB - 1) / kTB;
  const int nst = (n + kRB - 1) / kRB;
  if (tid == 0) *s_b = atomicAdd(ticket, 1u);
  __syncthreads();
  const int t = (int)*s_b;
  const int c = LOWER ? t : nst - 1 - t;
  const int row0 = c * kRB;
  const int lane = tid & 31, w = tid >> 5;
  const int g = w >> 2, wq = w & 3;              // row group, and the warp's share of it
  const bool two = 2 * c + 1 < nb;
  const int nblk = two ? 2 : 1;
  const int kf = LOWER || !two ? 0 : 1, ks = 1 - kf;
  // warps 0-3 (lane + 32 w = row of the step) read their right-hand side now
  const int rs = 32 * (w & 3) + lane;
  const float bv = (w < 4 && row0 + rs < n) ? __ldcg(&y[row0 + rs]) : 0.0f;
  // the diagonal inverses (zero elsewhere), and X
  for (int e = tid; e < kRB * kRB; e += kTrsvThreads) {
    const int r = e / kRB, jj = e % kRB, kr = r / kTB;
    ib[r * kRS + jj] = (kr == jj / kTB && kr < nblk)
                           ? inv[((size_t)(2 * c + kr) * kTB + r % kTB) * kTB + jj % kTB]
                           : 0.0f;
  }
  if (two)
    for (int e = tid; e < kTB * kTB; e += kTrsvThreads) {
      const int r = e / kTB, jj = e % kTB;
      const int gr = row0 + kTB * ks + r, gc = (2 * c + kf) * kTB + jj;
      xa[r * kTS + jj] = (gr < n && gc < n) ? LU[(size_t)gr * n + gc] : 0.0f;
    }
  __syncthreads();
  if (two) {
    // X inv_f, then -inv_s (X inv_f): thread = one column, eight rows
    const int jj = tid % kTB, r8 = (tid / kTB) * 8;
    const float* fi = ib + (kTB * kf) * kRS + kTB * kf + jj;
    float a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = 0.0f;
#pragma unroll 8
    for (int m = 0; m < kTB; ++m) {
      const float bm = fi[m * kRS];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = fmaf(xa[(r8 + i) * kTS + m], bm, a[i]);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) xb[(r8 + i) * kTS + jj] = a[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = 0.0f;
    const float* si = ib + (kTB * ks) * kRS + kTB * ks;
#pragma unroll 8
    for (int m = 0; m < kTB; ++m) {
      const float bm = xb[m * kTS + jj];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = fmaf(si[(r8 + i) * kRS + m], bm, a[i]);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) ib[(kTB * ks + r8 + i) * kRS + kTB * kf + jj] = -a[i];
    __syncthreads();
  }
  // this thread's quarter of row rs of the inverse
  float iv[32];
  {
    const float* ir = ib + rs * kRS + 32 * g;
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) iv[jj] = ir[jj];
  }
  // the dependencies: lane = column, one transposing reduction at the end
  float acc[32];
#pragma unroll
  for (int r = 0; r < 32; ++r) acc[r] = 0.0f;
  const int rh = row0 + 32 * g;                  // the group's first row
  const int ns = (n + 31) / 32;   // 32-column pieces of the matrix
  const int ndep = LOWER ? 4 * c : max(0, ns - 4 * (c + 1));
  for (int q = wq; q < ndep; q += 4) {
    const int sp = LOWER ? q : ns - 1 - q;
    const int cb = sp * 32;
    const bool colok = cb + lane < n;
    float m[32];
#pragma unroll
    for (int r = 0; r < 32; ++r)
      m[r] = (colok && rh + r < n) ? LU[(size_t)(rh + r) * n + cb + lane] : 0.0f;
    if (lane == 0) {
      unsigned spins = 0;
      for (;;) {
        unsigned f;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(f) : "l"(&flags[sp >> 2]) : "memory");
        if (f == epoch) break;
        if (++spins > kSpin) {
          atomicExch(err, 1);
          break;
        }
        if (spins > 4096) __nanosleep(32);
      }
    }
    __syncwarp();
    const float yc = colok ? __ldcg(&y[cb + lane]) : 0.0f;
#pragma unroll
    for (int r = 0; r < 32; ++r) acc[r] = fmaf(m[r], yc, acc[r]);
  }
  // after the step of width o a lane keeps the half of its rows that its
  // bit o selects, added to its partner's: lane r ends with row r
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int r = 0; r < o; ++r) {
      const float send = up ? acc[r] : acc[r + o];
      const float keep = up ? acc[r + o] : acc[r];
      acc[r] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  part[w * 32 + lane] = acc[0];
  __syncthreads();
  if (w < 4) {
    const float* p = part + 4 * w * 32 + lane;
    vsh[rs] = row0 + rs < n ? bv - (((p[0] + p[32]) + p[64]) + p[96]) : 0.0f;
  }
  __syncthreads();
  {
    const float4* v4 = reinterpret_cast<const float4*>(vsh + 32 * g);
    float x0 = 0.0f, x1 = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float4 v = v4[k];
      x0 = fmaf(iv[4 * k], v.x, x0);
      x1 = fmaf(iv[4 * k + 1], v.y, x1);
      x0 = fmaf(iv[4 * k + 2], v.z, x0);
      x1 = fmaf(iv[4 * k + 3], v.w, x1);
    }
    xp[g * kRB + rs] = x0 + x1;
  }
  __syncthreads();
  if (w < 4) {
    const float x = ((xp[rs] + xp[kRB + rs]) + xp[2 * kRB + rs]) + xp[3 * kRB + rs];
    if (row0 + rs < n) y[row0 + rs] = x;
    __threadfence();
  }
  __syncthreads();
  if (tid == 0)
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(&flags[c]), "r"(epoch) : "memory");
}

// binary32 -> binary64, exactly, by the two formats' encodings: sign kept,
// exponent rebiased (127 -> 1023; all-ones stays all-ones for infinities and
// NaN), the 23-bit fraction moved to the top of the 52-bit one; zeros by
// their bits, subnormals (whose binary64 form is normal) by the conversion
// instruction.  On this part the conversion instruction shares the slow
// binary64 pipe with the products' fused multiply-adds: converting with
// integer operations measured 192 against 283 us for the residual at
// n = 8192, bit for bit the same.
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xFFu;
  if (e == 0u && (u & 0x7FFFFFu)) return (double)f;
  const uint64_t sign = (uint64_t)(u >> 31) << 63;
  const uint64_t frac = (uint64_t)(u & 0x7FFFFFu) << 29;
  const uint64_t ex = e == 0u ? 0ull : e == 0xFFu ? 0x7FFull : (uint64_t)(e + (1023u - 127u));
  return __longlong_as_double((long long)(sign | (ex << 52) | frac));
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
    for (int j = lane; j < n; j += 32) s = fma(f32_to_f64(__ldcs(row + j)), x[j], s);
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

// The determinant from the factors (the intent of Listing 6): det A =
// (-1)^(number of interchanges) * prod_i u_ii.  One block; every thread adds
// log|u_ii| of its diagonal entries in binary64, then a tree in a fixed
// order.  out[0] = sign (+1, -1, or 0 when some u_ii is zero), out[1] =
// log |det A| (-inf when zero).
__global__ void __launch_bounds__(1024) k_lu_det(const float* __restrict__ LU, int n,
                                                 const int* __restrict__ piv, double* out) {
  __shared__ double s_log[1024];
  __shared__ int s_neg[1024], s_zero[1024];
  double lg = 0.0;
  int neg = 0, zero = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float u = LU[(size_t)i * n + i];
    if (u == 0.0f) zero = 1;
    else lg += log(fabs((double)u));
    neg ^= (u < 0.0f) ? 1 : 0;
    neg ^= (piv[i] != i) ? 1 : 0;
  }
  s_log[threadIdx.x] = lg;
  s_neg[threadIdx.x] = neg;
  s_zero[threadIdx.x] = zero;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s_log[threadIdx.x] += s_log[threadIdx.x + o];
      s_neg[threadIdx.x] ^= s_neg[threadIdx.x + o];
      s_zero[threadIdx.x] |= s_zero[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s_zero[0] ? 0.0 : (s_neg[0] ? -1.0 : 1.0);
    out[1] = s_zero[0] ? -INFINITY : s_log[0];
  }
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
    for (int j = lane; j < n; j += 32) s += fabs(f32_to_f64(row[j]));
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

template <int PC>
size_t panel_smem(int n, int k) {
  const int m = n - k;
  const int rs = (m + PC - 1) / PC;
  return (size_t)rs * kStride * 4 + 16 + 2 * PC * 8 + 2 * 8 + 2 * 8 + 2 * PC * kPB * 4 +
         2 * kPB * kXCols * 4 + (size_t)rs * 4 + 64;
}

template <int PC>
size_t panel_reg_smem(int n, int k) {
  const int m = n - k;
  const int rs = (m + PC - 1) / PC;
  constexpr int kW = kPT / 32;
  return (size_t)rs * kStride * 4 + 16 + 2 * kW * kPB * 4 + 2 * PC * kPB * 4 + 2 * kW * 8 +
         2 * PC * 8 + 2 * 8 + 2 * kPB * kXCols * 4 + (size_t)rs * 4 + 64;
}

// the 16-CTA form keeps rows in registers (k_lu_panel_reg); the 8-CTA
// portable form keeps the slab in shared memory (k_lu_panel)
template <int PC>
cudaError_t launch_panel(float* LU, int n, int k, int jb, int* piv, int* info, int* moves,
                         int c_lo, int c_hi, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(PC);
  cfg.blockDim = dim3(kPT);
  cfg.dynamicSmemBytes = PC == 16 ? panel_reg_smem<PC>(n, k) : panel_smem<PC>(n, k);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = PC;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if constexpr (PC == 16) {
    if ((n - k + PC - 1) / PC <= 2 * kPT)
      return cudaLaunchKernelEx(&cfg, k_lu_panel_reg<PC, 2>, LU, n, k, jb, piv, info, moves, c_lo,
                                c_hi);
    return cudaLaunchKernelEx(&cfg, k_lu_panel_reg<PC, max_rows_per_thread<PC>()>, LU, n, k, jb,
                              piv, info, moves, c_lo, c_hi);
  } else
    return cudaLaunchKernelEx(&cfg, k_lu_panel<PC>, LU, n, k, jb, piv, info, moves, c_lo, c_hi);
}

// 16 when one cluster of 16 CTAs with the largest panel fits the device
bool use_cluster16() {
  static int v = -1;
  if (v < 0) {
    v = 0;
    if (cudaFuncSetAttribute(k_lu_panel_reg<16, max_rows_per_thread<16>()>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
            cudaSuccess &&
        cudaFuncSetAttribute(k_lu_panel_reg<16, max_rows_per_thread<16>()>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)panel_reg_smem<16>(kLuMaxN, 0)) == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(16);
      cfg.blockDim = dim3(kPT);
      cfg.dynamicSmemBytes = panel_reg_smem<16>(kLuMaxN, 0);
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = 16;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int clusters = 0;
      if (cudaOccupancyMaxActiveClusters(&clusters, k_lu_panel_reg<16, max_rows_per_thread<16>()>, &cfg) == cudaSuccess &&
          clusters >= 1)
        v = 1;
    }
    cudaGetLastError();
  }
  return v == 1;
}

}  // namespace

size_t lu_panel_max_smem(int n) { return panel_smem<8>(n, 0); }

cudaError_t lu_prepare(int n) {
  gemm_tc_prepare();
  const bool c16 = !portable_kernels() && use_cluster16();
  const size_t ps = c16 ? panel_reg_smem<16>(n, 0) : panel_smem<8>(n, 0);
  cudaError_t e;
  if (c16) {
    e = cudaFuncSetAttribute(k_lu_panel_reg<16, max_rows_per_thread<16>()>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ps);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_lu_panel_reg<16, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ps);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_lu_panel_reg<16, 2>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  } else {
    e = cudaFuncSetAttribute(k_lu_panel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ps);
  }
  if (e != cudaSuccess) return e;
  const size_t mx = ((size_t)kLuOuter * (kLuOuter + 4) + (size_t)kLuOuter * 33) * sizeof(float);
  return cudaFuncSetAttribute(k_lu_trsm_outer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
}

cudaError_t launch_lu_panel(float* LU, int n, int k, int jb, int* piv, int* info, int* moves,
                            int c_lo, int c_hi, cudaStream_t s, Prof* prof) {
  prof_begin(prof, "lu_panel", s);
  const cudaError_t e =
      !portable_kernels() && use_cluster16()
          ? launch_panel<16>(LU, n, k, jb, piv, info, moves, c_lo, c_hi, s)
                      : launch_panel<8>(LU, n, k, jb, piv, info, moves, c_lo, c_hi, s);
  prof_end(prof, s);
  return e;
}

cudaError_t launch_lu_laswp_outer(float* LU, int n, const int* moves, int nlists, int K, int KB,
                                  int* perm, cudaStream_t s, Prof* prof) {
  const int cols = n - KB + 1;   // and the permutation
  prof_begin(prof, "lu_laswp", s);
  k_lu_laswp_outer<<<(cols + 127) / 128, 128, 0, s>>>(LU, n, moves, nlists, K, KB, perm);
  prof_end(prof, s);
  return cudaGetLastError();
}

cudaError_t launch_lu_inner(float* LU, int n, int j, int c0, int c1, unsigned* counter,
                            cudaStream_t s, Prof* prof) {
  if (c1 <= c0 || n - j - kPB <= 0) return cudaSuccess;
  prof_begin(prof, "lu_inner", s);
  k_lu_inner<<<(n - j - kPB + kInRows - 1) / kInRows, 256, 0, s>>>(LU, n, j, c0, c1, counter);
  prof_end(prof, s);
  return cudaGetLastError();
}

cudaError_t launch_lu_trsm_outer(float* LU, int n, int K, int KB, int c0, int c1, cudaStream_t s,
                                 Prof* prof) {
  if (c1 <= c0) return cudaSuccess;
  const size_t sm = ((size_t)KB * (KB + 4) + (size_t)KB * 33) * sizeof(float);
  prof_begin(prof, "lu_trsm", s);
  k_lu_trsm_outer<<<(c1 - c0 + kPB - 1) / kPB, 256, sm, s>>>(LU, n, K, KB, c0, c1);
  prof_end(prof, s);
  return cudaGetLastError();
}

cudaError_t launch_lu_iota(int* perm, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_lu_iota<<<(n + 255) / 256 < 256 ? (n + 255) / 256 : 256, 256, 0, s>>>(perm, n);
  return cudaGetLastError();
}

size_t lu_diag_inv_bytes(int n) { return (size_t)2 * ((n + kTB - 1) / kTB) * kTB * kTB * 4; }

cudaError_t launch_lu_diag_inv(const float* LU, int n, float* inv, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_lu_diag_inv<<<(n + kTB - 1) / kTB, 2 * kTB, 0, s>>>(LU, n, inv);
  return cudaGetLastError();
}

cudaError_t launch_lu_solve(const float* LU, const float* inv, int n, const int* perm,
                            const double* rhs, bool rhs_is_residual, float* y, unsigned* flags,
                            unsigned epoch, unsigned* tickets, int* err, cudaStream_t s,
                            Prof* prof) {
  (void)rhs_is_residual;
  const int nb = (n + kTB - 1) / kTB;
  const int nst = (n + kRB - 1) / kRB;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_trsv<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTrsvSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_trsv<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kTrsvSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  prof_begin(prof, "lu_trsv", s);
  k_apply_perm<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, s>>>(rhs, y, n, perm);
  cudaMemsetAsync(tickets, 0, 2 * sizeof(unsigned), s);
  k_trsv<true><<<nst, kTrsvThreads, kTrsvSmem, s>>>(LU, inv, n, y, flags, epoch, tickets, err);
  k_trsv<false><<<nst, kTrsvThreads, kTrsvSmem, s>>>(LU, inv + (size_t)nb * kTB * kTB, n, y,
                                                     flags + nb, epoch, tickets + 1, err);
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

cudaError_t launch_lu_det(const float* LU, int n, const int* piv, double* out, cudaStream_t s,
                          Prof* prof) {
  prof_begin(prof, "lu_det", s);
  k_lu_det<<<1, 1024, 0, s>>>(LU, n, piv, out);
  prof_end(prof, s);
  return cudaGetLastError();
}

}  // namespace sgk
