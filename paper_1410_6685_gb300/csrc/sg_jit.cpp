// sg_jit.cpp -- run-time specialisation of fused element-wise passes.
//
// Sec. 5 of the paper instantiates a kernel template per library call and
// compiles it at run time.  Here the template is the hand-written streaming
// kernel below; what is instantiated is the body: the optimizer's fused
// postfix program (map chains, predicates, masked reduction) is turned into
// straight-line SSA code by symbolic execution of its stack, and compiled
// once per program structure with NVRTC for sm_103a (constants stay kernel
// arguments, so programs that differ only in constants share a kernel).
// The result record and the deterministic block / last-block combine are the
// same as those of the interpreting kernel (k_stream.cu), which remains the
// fallback when NVRTC is unavailable or specialisation is switched off.
#include <cuda_runtime.h>
#include <dlfcn.h>

#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "sg_internal.h"
#include "sg_jit.h"

namespace sgk {
namespace {

// ---- NVRTC, loaded on first use ------------------------------------------
typedef int nvrtcResult_t;
struct Nvrtc {
  void* h = nullptr;
  nvrtcResult_t (*create)(void**, const char*, const char*, int, const char* const*,
                          const char* const*) = nullptr;
  nvrtcResult_t (*compile)(void*, int, const char* const*) = nullptr;
  nvrtcResult_t (*cubin_size)(void*, size_t*) = nullptr;
  nvrtcResult_t (*cubin)(void*, char*) = nullptr;
  nvrtcResult_t (*log_size)(void*, size_t*) = nullptr;
  nvrtcResult_t (*log)(void*, char*) = nullptr;
  nvrtcResult_t (*destroy)(void**) = nullptr;
  bool ok = false;
};

Nvrtc& nvrtc() {
  static Nvrtc n;
  static std::once_flag once;
  std::call_once(once, [] {
    const char* names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                           "/usr/local/cuda/lib64/libnvrtc.so"};
    for (const char* nm : names) {
      n.h = dlopen(nm, RTLD_NOW | RTLD_LOCAL);
      if (n.h) break;
    }
    if (!n.h) return;
    n.create = (decltype(n.create))dlsym(n.h, "nvrtcCreateProgram");
    n.compile = (decltype(n.compile))dlsym(n.h, "nvrtcCompileProgram");
    n.cubin_size = (decltype(n.cubin_size))dlsym(n.h, "nvrtcGetCUBINSize");
    n.cubin = (decltype(n.cubin))dlsym(n.h, "nvrtcGetCUBIN");
    n.log_size = (decltype(n.log_size))dlsym(n.h, "nvrtcGetProgramLogSize");
    n.log = (decltype(n.log))dlsym(n.h, "nvrtcGetProgramLog");
    n.destroy = (decltype(n.destroy))dlsym(n.h, "nvrtcDestroyProgram");
    n.ok = n.create && n.compile && n.cubin_size && n.cubin && n.log_size && n.log && n.destroy;
  });
  return n;
}

// ---- the kernel template ---------------------------------------------------
// Layouts below must match PassResult (sg_internal.h) and JitArgs (sg_jit.h).
const char* kTemplateHead = R"SGJIT(
struct PassResult {
  double sum; long long count; float mn, mx; int nan_seen; int pad; long long first[4];
};
struct JitArgs {
  const float* in[4]; float* out[4]; long long n; float cst[48];
  PassResult* partials; unsigned* counter; PassResult* result; const long long* count;
  int vec4; int pad;
};
#define SG_NONE 0x7fffffffffffffffLL
__device__ __forceinline__ bool sg_nan(float v) { return v != v; }
__device__ __forceinline__ float sg_min(float a, float b) {
  return (sg_nan(a) || sg_nan(b)) ? __int_as_float(0x7fffffff) : (a < b ? a : b);
}
__device__ __forceinline__ float sg_max(float a, float b) {
  return (sg_nan(a) || sg_nan(b)) ? __int_as_float(0x7fffffff) : (a > b ? a : b);
}
__device__ __forceinline__ float sg_b(bool v) { return v ? 1.0f : 0.0f; }
struct Acc { double sum; float hi, lo; long long cnt; float mn, mx; int nan_seen; long long first[4]; };
__device__ __forceinline__ void acc_init(Acc& a) {
  a.sum = 0.0; a.hi = 0.0f; a.lo = 0.0f; a.cnt = 0;
  a.mn = __int_as_float(0x7f800000); a.mx = __int_as_float(0xff800000);
  a.nan_seen = 0;
  for (int p = 0; p < 4; ++p) a.first[p] = SG_NONE;
}
// Knuth's TwoSum: hi + v = s + e exactly; the error terms gather in lo
__device__ __forceinline__ void acc_add(Acc& a, float v) {
  const float s = __fadd_rn(a.hi, v);
  const float bp = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bp)), __fsub_rn(v, bp));
  a.hi = s;
  a.lo = __fadd_rn(a.lo, e);
}
__device__ __forceinline__ void acc_fold(Acc& a) {
  a.sum += (double)a.hi + (double)a.lo;
  a.hi = 0.0f; a.lo = 0.0f;
}
__device__ __forceinline__ void acc_merge(Acc& a, const Acc& b) {
  a.sum += b.sum; a.cnt += b.cnt;
  a.mn = b.mn < a.mn ? b.mn : a.mn; a.mx = b.mx > a.mx ? b.mx : a.mx;
  a.nan_seen |= b.nan_seen;
  for (int p = 0; p < 4; ++p) a.first[p] = b.first[p] < a.first[p] ? b.first[p] : a.first[p];
}
__device__ __forceinline__ void warp_reduce(Acc& a) {
  for (int o = 16; o > 0; o >>= 1) {
    Acc b;
    b.sum = __shfl_xor_sync(0xffffffffu, a.sum, o);
    b.cnt = __shfl_xor_sync(0xffffffffu, a.cnt, o);
    b.mn = __shfl_xor_sync(0xffffffffu, a.mn, o);
    b.mx = __shfl_xor_sync(0xffffffffu, a.mx, o);
    b.nan_seen = __shfl_xor_sync(0xffffffffu, a.nan_seen, o);
    for (int p = 0; p < 4; ++p) b.first[p] = __shfl_xor_sync(0xffffffffu, a.first[p], o);
    acc_merge(a, b);
  }
}
__device__ __forceinline__ void block_reduce(Acc& a) {
  __shared__ Acc sh[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  warp_reduce(a);
  if (lane == 0) sh[w] = a;
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    if (lane < nw) a = sh[lane]; else acc_init(a);
    warp_reduce(a);
  }
  __syncthreads();
}
// one masked value into the reduction (mn/mx skip NaN, which sets nan_seen)
__device__ __forceinline__ void acc_one(Acc& a, float v, bool m) {
  if (!m) return;
  a.cnt += 1;
  acc_add(a, v);
#if SG_MINMAX
  if (sg_nan(v)) a.nan_seen = 1;
  else { a.mn = v < a.mn ? v : a.mn; a.mx = v > a.mx ? v : a.mx; }
#endif
}
)SGJIT";

const char* kTemplateKernel = R"SGJIT(
extern "C" __global__ void __launch_bounds__(256) sg_fused(const JitArgs a) {
  Acc acc;
  acc_init(acc);
  long long n = a.n;
  if (a.count) {
    const long long c = *a.count;
    n = c < 0 ? 0 : c < n ? c : n;
  }
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long tail = 0;
  if (a.vec4) {
    const long long nv = n >> 2;
    tail = nv << 2;
    for (long long v = tid; v < nv; v += stride) {
      float xs[SG_NX][4];
#pragma unroll
      for (int k = 0; k < SG_NIN; ++k) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(a.in[k]) + v);
        xs[k][0] = t.x; xs[k][1] = t.y; xs[k][2] = t.z; xs[k][3] = t.w;
      }
      float os[SG_NO][4];
      float rv[4];
      bool rm[4];
      unsigned hit[4];
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        float x[SG_NX], o[SG_NO];
#pragma unroll
        for (int k = 0; k < SG_NIN; ++k) x[k] = xs[k][l];
        hit[l] = 0u; rv[l] = 0.0f; rm[l] = false;
        sg_body(a, x, (v << 2) + l, o, hit[l], rv[l], rm[l]);
#pragma unroll
        for (int k = 0; k < SG_NOUT; ++k) os[k][l] = o[k];
      }
#pragma unroll
      for (int k = 0; k < SG_NOUT; ++k)
        reinterpret_cast<float4*>(a.out[k])[v] = make_float4(os[k][0], os[k][1], os[k][2], os[k][3]);
#if SG_NPRED > 0
#pragma unroll
      for (int l = 3; l >= 0; --l)
#pragma unroll
        for (int p = 0; p < SG_NPRED; ++p)
          if ((hit[l] >> p) & 1u) acc.first[p] = (v << 2) + l < acc.first[p] ? (v << 2) + l : acc.first[p];
#endif
#if SG_RED
#pragma unroll
      for (int l = 0; l < 4; ++l) acc_one(acc, rv[l], rm[l]);
#endif
    }
  }
  for (long long i = tail + tid; i < n; i += stride) {
    float x[SG_NX], o[SG_NO];
#pragma unroll
    for (int k = 0; k < SG_NIN; ++k) x[k] = a.in[k][i];
    unsigned hit = 0u;
    float rv = 0.0f;
    bool rm = false;
    sg_body(a, x, i, o, hit, rv, rm);
#pragma unroll
    for (int k = 0; k < SG_NOUT; ++k) a.out[k][i] = o[k];
#if SG_NPRED > 0
#pragma unroll
    for (int p = 0; p < SG_NPRED; ++p)
      if ((hit >> p) & 1u) acc.first[p] = i < acc.first[p] ? i : acc.first[p];
#endif
#if SG_RED
    acc_one(acc, rv, rm);
#endif
  }
#if SG_RED || SG_NPRED > 0
  acc_fold(acc);
  block_reduce(acc);
  __shared__ bool am_last;
  if (threadIdx.x == 0) {
    PassResult r;
    r.sum = acc.sum; r.count = acc.cnt; r.mn = acc.mn; r.mx = acc.mx; r.nan_seen = acc.nan_seen;
    r.pad = 0;
    for (int p = 0; p < 4; ++p) r.first[p] = acc.first[p];
    a.partials[blockIdx.x] = r;
    __threadfence();
    am_last = atomicAdd(a.counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  Acc tot;
  acc_init(tot);
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    const PassResult* q = &a.partials[b];
    Acc p;
    p.hi = 0.0f; p.lo = 0.0f;
    p.sum = __ldcg(&q->sum); p.cnt = __ldcg(&q->count); p.mn = __ldcg(&q->mn);
    p.mx = __ldcg(&q->mx); p.nan_seen = __ldcg(&q->nan_seen);
    for (int k = 0; k < 4; ++k) p.first[k] = __ldcg(&q->first[k]);
    acc_merge(tot, p);
  }
  block_reduce(tot);
  if (threadIdx.x == 0) {
    PassResult r;
    r.sum = tot.sum; r.count = tot.cnt; r.mn = tot.mn; r.mx = tot.mx; r.nan_seen = tot.nan_seen;
    r.pad = 0;
    for (int p = 0; p < 4; ++p) r.first[p] = tot.first[p];
    *a.result = r;
    *a.counter = 0u;
  }
#endif
}
)SGJIT";

const char* kTemplateBatch = R"SGJIT(
struct ChunkPartial { double sum; long long cnt; long long first; };
struct BatchHdr { unsigned ticket; unsigned any_violation; unsigned long long total_chunks; unsigned pad[60]; };
struct BatchJitArgs {
  const float* data; const long long* off; long long nseg; long long chunk; float cst[48];
  const long long* chunk_start; const int* chunk_seg; ChunkPartial* partials; unsigned* seg_done;
  BatchHdr* hdr; double* sums; long long* first_viol; long long* kept; int vec4; int pad;
};
__device__ __forceinline__ void sg_elem(const BatchJitArgs& a, float v, long long i, Acc& acc) {
  float x[1] = {v};
  float o[1];
  unsigned hit = 0u;
  float rv = 0.0f;
  bool rm = false;
  sg_body(a, x, i, o, hit, rv, rm);
  if (hit & 1u) acc.first[0] = i < acc.first[0] ? i : acc.first[0];
  acc_one(acc, rv, rm);
}
// one quad wholly inside the collection: the four masked values are added in
// pairs, (v0 + v1) + (v2 + v3) (error at most 2u of their magnitudes), and the
// pair sum enters the compensated accumulator once; kept elements counted in
// 32 bits (a chunk holds far fewer than 2^31)
__device__ __forceinline__ void sg_quad_in(const BatchJitArgs& a, float4 t, long long i0, Acc& acc,
                                           int& cnt) {
  const float xv[4] = {t.x, t.y, t.z, t.w};
  float w[4];
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    float x[1] = {xv[l]};
    float o[1];
    unsigned hit = 0u;
    float rv = 0.0f;
    bool rm = false;
    sg_body(a, x, i0 + l, o, hit, rv, rm);
    if (hit & 1u) acc.first[0] = i0 + l < acc.first[0] ? i0 + l : acc.first[0];
    w[l] = rm ? rv : 0.0f;
    cnt += rm ? 1 : 0;
  }
  acc_add(acc, __fadd_rn(__fadd_rn(w[0], w[1]), __fadd_rn(w[2], w[3])));
}
// the three fields a chunk's result needs, combined like acc_merge
__device__ __forceinline__ void batch_warp_reduce(double& sum, long long& cnt, long long& first) {
  for (int o = 16; o > 0; o >>= 1) {
    const double s2 = __shfl_xor_sync(0xffffffffu, sum, o);
    const long long c2 = __shfl_xor_sync(0xffffffffu, cnt, o);
    const long long f2 = __shfl_xor_sync(0xffffffffu, first, o);
    sum += s2;
    cnt += c2;
    first = f2 < first ? f2 : first;
  }
}
extern "C" __global__ void __launch_bounds__(256) sg_batch(const BatchJitArgs a) {
  __shared__ unsigned long long s_item;
  __shared__ double s_sum[8];
  __shared__ long long s_cnt[8], s_first[8];
  __shared__ bool s_last;
  const unsigned long long total = a.hdr->total_chunks;
  const float4* d4 = reinterpret_cast<const float4*>(a.data);
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(&a.hdr->ticket, 1u);
    __syncthreads();
    const unsigned long long item = s_item;
    __syncthreads();
    if (item >= total) break;
    const long long s = a.chunk_seg[item];
    const long long cs = a.chunk_start[s];
    const long long c = (long long)item - cs;
    const long long nch = a.chunk_start[s + 1] - cs;
    const long long sb = a.off[s], se = a.off[s + 1];
    const long long b = sb + c * a.chunk;
    const long long e = b + a.chunk < se ? b + a.chunk : se;
    Acc acc;
    acc_init(acc);
    if (a.vec4) {
      // quads [qa, qz) lie wholly in [b, e); the at most three elements before
      // and after them go one by one.  Each thread visits quads q, q + 256,
      // q + 512, ... in that order, four loads issued before four are evaluated.
      const long long qa = (b + 3) >> 2;
      const long long qz = (e >> 2) > qa ? (e >> 2) : qa;
      const long long hb = b, he = (qa << 2) < e ? (qa << 2) : e;
      const long long tb = (qz << 2) > he ? (qz << 2) : he;
      if (threadIdx.x < he - hb) {
        const long long i = hb + threadIdx.x;
        sg_elem(a, __ldcs(a.data + i), i - sb, acc);
      } else if (threadIdx.x >= 4 && threadIdx.x - 4 < e - tb) {
        const long long i = tb + threadIdx.x - 4;
        sg_elem(a, __ldcs(a.data + i), i - sb, acc);
      }
      int cnt = 0;
      long long q = qa + threadIdx.x;
      const long long ib = -sb;
      for (; q + 768 < qz; q += 1024) {
        float4 t[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) t[u] = __ldcs(d4 + q + u * 256);
#pragma unroll
        for (int u = 0; u < 4; ++u) sg_quad_in(a, t[u], ((q + u * 256) << 2) + ib, acc, cnt);
      }
      for (; q < qz; q += 256) sg_quad_in(a, __ldcs(d4 + q), (q << 2) + ib, acc, cnt);
      acc.cnt += cnt;
    } else {
      for (long long i = b + threadIdx.x; i < e; i += 256) sg_elem(a, __ldcs(a.data + i), i - sb, acc);
    }
    acc_fold(acc);
    double sum = acc.sum;
    long long cnt = acc.cnt, first = acc.first[0];
    batch_warp_reduce(sum, cnt, first);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
      s_sum[w] = sum;
      s_cnt[w] = cnt;
      s_first[w] = first;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double tsum = s_sum[0];
      long long tcnt = s_cnt[0], tfirst = s_first[0];
      for (int k = 1; k < 8; ++k) {
        tsum += s_sum[k];
        tcnt += s_cnt[k];
        tfirst = s_first[k] < tfirst ? s_first[k] : tfirst;
      }
      if (nch == 1) {
        a.sums[s] = tsum;
        a.kept[s] = tcnt;
        a.first_viol[s] = tfirst == SG_NONE ? -1 : tfirst;
        if (tfirst != SG_NONE) atomicOr(&a.hdr->any_violation, 1u);
        s_last = false;
      } else {
        ChunkPartial p;
        p.sum = tsum; p.cnt = tcnt; p.first = tfirst;
        a.partials[cs + c] = p;
        __threadfence();
        s_last = atomicAdd(&a.seg_done[s], 1u) == (unsigned)(nch - 1);
      }
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
      __threadfence();
      double sum2 = 0.0;
      long long cnt2 = 0, first2 = SG_NONE;
      for (long long k = 0; k < nch; ++k) {
        const ChunkPartial* p = &a.partials[cs + k];
        sum2 += __ldcg(&p->sum);
        cnt2 += __ldcg(&p->cnt);
        const long long f = __ldcg(&p->first);
        first2 = f < first2 ? f : first2;
      }
      a.sums[s] = sum2;
      a.kept[s] = cnt2;
      a.first_viol[s] = first2 == SG_NONE ? -1 : first2;
      if (first2 != SG_NONE) atomicOr(&a.hdr->any_violation, 1u);
      a.seg_done[s] = 0;
    }
    __syncthreads();
  }
}
)SGJIT";

// The filter (Table 2), specialised: a stable compaction, one CTA per tile
// of 8192 items (or 2048 / 4096: SG_FQ = 2 / 4 float4s per thread, the
// schedule chooser's filter family) taken from a ticket counter when the CTA starts (so tiles
// start in ticket order and a look-back seldom waits on a tile that has not
// started).  Thread t loads float4s t + 256 q (q < 8) of the tile straight
// into registers; the order of kept items (round q, warp, lane, component)
// comes from four ballots per round and a scan of the 64 (round, warp)
// counts that every warp does itself.  The tile's aggregate is published at
// once, every warp packs its kept items into shared memory (unpredicated
// stores), warp 0 does the decoupled look-back over the tiles' words, 32
// tiles per memory round trip, and the packed items are written out
// contiguously.  Five CTAs per SM (48 registers, a few spilled).  Measured
// at 2^28 items: 0.41 ms, against 0.48 / 0.49 / 0.55 ms at six / four / three
// CTAs per SM (40 / 64 / 80 registers), 0.57 ms with 512 threads of 16
// items, 0.65 ms with 4096-item tiles, 0.71 / 0.85 ms with
// 64- / 128-tile look-back windows (more words re-polled while a predecessor
// is unpublished), and 0.92 ms for a persistent form prefetching its next
// tile by bulk copy (its tickets run ahead of the tiles it is still working
// on, so look-backs wait on them).
// Layouts below must match FilterResult (sg_internal.h) and FilterJitArgs
// (sg_jit.h).
const char* kTemplateFilter = R"SGJIT(
struct FilterResult { long long count; int timeout; int pad; unsigned long long post_enc; };
struct FilterJitArgs {
  const float* x; float* out; long long n; float cst[48];
  unsigned long long* st; unsigned* tile_ctr; FilterResult* res; unsigned ntiles; int skip_tile;
  unsigned spin_limit; int pad;
};
#define SG_AGG (1ull << 62)
#define SG_PRE (2ull << 62)
#define SG_CNT ((1ull << 62) - 1)
__device__ __forceinline__ unsigned long long sg_ld_relaxed(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void sg_st_relaxed(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

extern "C" __global__ void __launch_bounds__(256, SG_FMINB) sg_filter(const FilterJitArgs a) {
  __shared__ __align__(16) float s_pack[SG_FT];
  __shared__ float s_spare[256];
  __shared__ unsigned s_cnt[SG_FQ * 8];
  __shared__ unsigned s_tile;
  __shared__ unsigned long long s_excl;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long long n = a.n;
  unsigned lt;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
  if (tid == 0) s_tile = atomicAdd(a.tile_ctr, 1u);
  __syncthreads();
  const unsigned t = s_tile;
  const long long base = (long long)t * SG_FT;
  const int valid = (int)(n - base < SG_FT ? n - base : SG_FT);
  float v[4 * SG_FQ];
  if (valid == SG_FT && (((unsigned long long)(a.x + base)) & 15ull) == 0) {
#pragma unroll
    for (int q = 0; q < SG_FQ; ++q) {
      const float4 f = __ldcs(reinterpret_cast<const float4*>(a.x + base) + q * 256 + tid);
      v[4 * q] = f.x; v[4 * q + 1] = f.y; v[4 * q + 2] = f.z; v[4 * q + 3] = f.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < SG_FQ; ++q)
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const int li = 4 * (q * 256 + tid) + l;
        v[4 * q + l] = li < valid ? a.x[base + li] : 0.0f;
      }
  }
  // predicate on the thread's 32 items, masked to the valid ones
  unsigned keep = 0, vmask = 0;
#pragma unroll
  for (int q = 0; q < SG_FQ; ++q) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      float x[1], o[1];
      x[0] = v[4 * q + l];
      unsigned hit = 0u;
      float rv = 0.0f;
      bool rm = false;
      sg_body(a, x, base + 4 * (q * 256 + tid) + l, o, hit, rv, rm);
      keep |= (unsigned)(rv != 0.0f) << (4 * q + l);
    }
    const int rest = valid - 4 * (q * 256 + tid);
    vmask |= ((1u << min(max(rest, 0), 4)) - 1u) << (4 * q);
  }
  keep &= vmask;
  unsigned rbase[SG_FQ];
#pragma unroll
  for (int q = 0; q < SG_FQ; ++q) {
    unsigned below = 0, cnt = 0;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const unsigned m = __ballot_sync(0xffffffffu, (keep >> (4 * q + l)) & 1u);
      below += __popc(m & lt);
      cnt += __popc(m);
    }
    rbase[q] = below;
    if (lane == 0) s_cnt[q * 8 + w] = cnt;
  }
  __syncthreads();
  // every warp scans the 8 SG_FQ (round, warp) counts, two per lane when
  // there are 64
#if SG_FQ == 8
  const unsigned c0 = s_cnt[2 * lane], c1 = s_cnt[2 * lane + 1];
#else
  const unsigned c0 = lane < SG_FQ * 8 ? s_cnt[lane] : 0u, c1 = 0u;
#endif
  unsigned incl = c0 + c1;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
  const unsigned e0 = incl - c0 - c1;
  const bool publish = (int)t != a.skip_tile;
  if (tid == 0 && t > 0 && publish) sg_st_relaxed(&a.st[t], SG_AGG | total);
#pragma unroll
  for (int q = 0; q < SG_FQ; ++q) {
    const int entry = q * 8 + w;
#if SG_FQ == 8
    unsigned r = __shfl_sync(0xffffffffu, (entry & 1) ? e0 + c0 : e0, entry >> 1) + rbase[q];
#else
    unsigned r = __shfl_sync(0xffffffffu, e0, entry) + rbase[q];
#endif
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const unsigned bit = (keep >> (4 * q + l)) & 1u;
      *(bit ? s_pack + r : s_spare + tid) = v[4 * q + l];   // no predicated store
      r += bit;
    }
  }
  if (w == 0) {
    unsigned long long excl = 0;
    if (t == 0) {
      if (lane == 0 && publish) sg_st_relaxed(&a.st[0], SG_PRE | total);
    } else {
      long long j = (long long)t - 1;
      unsigned spins = 0;
      while (true) {
        const long long idx = j - lane;
        const unsigned long long wd = idx >= 0 ? sg_ld_relaxed(&a.st[idx]) : SG_PRE;
        const unsigned long long flag = wd & ~SG_CNT;
        const unsigned zero = __ballot_sync(0xffffffffu, flag == 0);
        const unsigned pre = __ballot_sync(0xffffffffu, flag == SG_PRE);
        const unsigned stop = zero ? (unsigned)(__ffs(zero) - 1) : 32u;
        const unsigned first_pre = pre ? (unsigned)(__ffs(pre) - 1) : 32u;
        const bool done = first_pre < stop;
        const unsigned take = done ? first_pre + 1 : stop;
        unsigned long long cc = (unsigned)lane < take ? (wd & SG_CNT) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cc += __shfl_xor_sync(0xffffffffu, cc, o);
        excl += cc;
        if (done) break;
        j -= take;
        if (stop < 32u) {
          if (++spins > a.spin_limit) {
            if (lane == 0) atomicExch(&a.res->timeout, 1);
            break;
          }
          if (spins > 32) __nanosleep(64);
        }
      }
      if (lane == 0 && publish) sg_st_relaxed(&a.st[t], SG_PRE | (excl + total));
    }
    if (lane == 0) {
      s_excl = excl;
      if (t == a.ntiles - 1) a.res->count = (long long)(excl + total);
    }
  }
  __syncthreads();
  const unsigned long long gb = s_excl;
#if SG_POST
  unsigned long long bad = 0ull;   // ~(lowest violating position), 0: none
#endif
  for (unsigned i = tid; i < total; i += 256) {
    const unsigned long long pos = gb + i;
    if (pos < (unsigned long long)n) {
      const float kv = s_pack[i];
      a.out[pos] = kv;
#if SG_POST
      // the folded postcondition on the kept item at its output position
      float x[1], o[1];
      x[0] = kv;
      unsigned hit = 0u;
      float rv = 0.0f;
      bool rm = false;
      sg_post(a, x, (long long)pos, o, hit, rv, rm);
      if (!(rv != 0.0f) && ~pos > bad) bad = ~pos;
#endif
    }
  }
#if SG_POST
#pragma unroll
  for (int o2 = 16; o2 > 0; o2 >>= 1) {
    const unsigned long long b2 = __shfl_xor_sync(0xffffffffu, bad, o2);
    bad = b2 > bad ? b2 : bad;
  }
  if (lane == 0 && bad) atomicMax(&a.res->post_enc, bad);
#endif
}
)SGJIT";

// ---- body generation: symbolic execution of the postfix program -----------
// cst_base: where the program's constants start in the argument block's
// cst array (a second program shares it)
bool gen_body(const Prog& pr, uint32_t pred_exists, std::string* body, int cst_base = 0) {
  std::vector<std::string> st;
  std::string b;
  int t = 0;
  auto tmp = [&](const std::string& expr) {
    std::string nm = "t" + std::to_string(t++);
    b += "  const float " + nm + " = " + expr + ";\n";
    return nm;
  };
  auto pop = [&](std::string* v) {
    if (st.empty()) return false;
    *v = st.back();
    st.pop_back();
    return true;
  };
  char buf[64];
  for (int pc = 0; pc < pr.nops; ++pc) {
    const int op = pr.op[pc];
    std::string x, y, z;
    switch (op) {
      case SG_OP_LOAD:
        snprintf(buf, sizeof buf, "x[%d]", (int)pr.arg[pc]);
        st.push_back(buf);
        break;
      case SG_OP_CONST:
        snprintf(buf, sizeof buf, "a.cst[%d]", cst_base + pc);
        st.push_back(buf);
        break;
      case SG_OP_INDEX: st.push_back(tmp("__ll2float_rn(i)")); break;
      case SG_OP_DUP:
        if (st.empty()) return false;
        st.push_back(st.back());
        break;
      case SG_OP_SWAP:
        if (st.size() < 2) return false;
        std::swap(st[st.size() - 1], st[st.size() - 2]);
        break;
      case SG_OP_NEG: case SG_OP_ABS: case SG_OP_SQRT: case SG_OP_NOT: {
        if (!pop(&x)) return false;
        const char* f = op == SG_OP_NEG ? "(-%s)" : op == SG_OP_ABS ? "fabsf(%s)"
                        : op == SG_OP_SQRT ? "__fsqrt_rn(%s)" : "sg_b(!(%s != 0.0f))";
        snprintf(buf, sizeof buf, f, x.c_str());
        st.push_back(tmp(buf));
        break;
      }
      case SG_OP_FMA: case SG_OP_SELECT: {
        if (!pop(&z) || !pop(&y) || !pop(&x)) return false;
        std::string e = op == SG_OP_FMA
                            ? "__fmaf_rn(" + x + ", " + y + ", " + z + ")"
                            : "((" + x + " != 0.0f) ? " + y + " : " + z + ")";
        st.push_back(tmp(e));
        break;
      }
      case K_STORE:
        if (st.empty()) return false;
        b += "  o[" + std::to_string((int)pr.arg[pc]) + "] = " + st.back() + ";\n";
        break;
      case K_PRED: {
        if (!pop(&x)) return false;
        const int p = pr.arg[pc];
        const bool ex = (pred_exists >> p) & 1u;
        b += std::string("  if (") + (ex ? "" : "!") + "(" + x + " != 0.0f)) hit |= " +
             std::to_string(1u << p) + "u;\n";
        break;
      }
      case K_MASK:
        if (!pop(&x)) return false;
        b += "  mask = (" + x + " != 0.0f);\n";
        break;
      case K_REDUCE:
        if (!pop(&x)) return false;
        b += "  rv = " + x + "; rm = mask; mask = true;\n";
        break;
      case K_POP:
        if (!pop(&x)) return false;
        break;
      default: {  // binary
        if (!pop(&y) || !pop(&x)) return false;
        std::string e;
        switch (op) {
          case SG_OP_ADD: e = "__fadd_rn(" + x + ", " + y + ")"; break;
          case SG_OP_SUB: e = "__fsub_rn(" + x + ", " + y + ")"; break;
          case SG_OP_MUL: e = "__fmul_rn(" + x + ", " + y + ")"; break;
          case SG_OP_DIV: e = "__fdiv_rn(" + x + ", " + y + ")"; break;
          case SG_OP_MIN: e = "sg_min(" + x + ", " + y + ")"; break;
          case SG_OP_MAX: e = "sg_max(" + x + ", " + y + ")"; break;
          case SG_OP_LT: e = "sg_b(" + x + " < " + y + ")"; break;
          case SG_OP_LE: e = "sg_b(" + x + " <= " + y + ")"; break;
          case SG_OP_GT: e = "sg_b(" + x + " > " + y + ")"; break;
          case SG_OP_GE: e = "sg_b(" + x + " >= " + y + ")"; break;
          case SG_OP_EQ: e = "sg_b(" + x + " == " + y + ")"; break;
          case SG_OP_NE: e = "sg_b(" + x + " != " + y + ")"; break;
          case SG_OP_AND: e = "sg_b(" + x + " != 0.0f && " + y + " != 0.0f)"; break;
          case SG_OP_OR: e = "sg_b(" + x + " != 0.0f || " + y + " != 0.0f)"; break;
          default: return false;
        }
        st.push_back(tmp(e));
      }
    }
  }
  *body = b;
  return true;
}

struct Cache {
  std::mutex mu;
  std::unordered_map<std::string, cudaKernel_t> kernels;
  std::unordered_map<std::string, bool> failed;
};
Cache& cache() {
  static Cache c;
  return c;
}

// Compiles `src` (once; cached by source text) and returns its kernel `name`,
// or nullptr when it cannot be built.
cudaKernel_t compile_cached(const std::string& src, const char* name, std::string* log) {
  Nvrtc& nv = nvrtc();
  Cache& c = cache();
  std::lock_guard<std::mutex> lk(c.mu);
  auto it = c.kernels.find(src);
  if (it != c.kernels.end()) return it->second;
  if (c.failed.count(src)) return nullptr;
  void* prog = nullptr;
  cudaKernel_t k = nullptr;
  if (nv.create(&prog, src.c_str(), "sg_fused.cu", 0, nullptr, nullptr) == 0) {
    const char* opts[] = {"--gpu-architecture=sm_103a", "--std=c++17", "-default-device",
                          "-fmad=false"};
    const int rc = nv.compile(prog, 4, opts);
    if (rc == 0) {
      size_t sz = 0;
      nv.cubin_size(prog, &sz);
      std::vector<char> cubin(sz);
      nv.cubin(prog, cubin.data());
      cudaLibrary_t lib = nullptr;
      if (cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) ==
              cudaSuccess &&
          cudaLibraryGetKernel(&k, lib, name) == cudaSuccess) {
        // the library stays loaded for the life of the process (cached kernel)
      } else {
        cudaGetLastError();
        k = nullptr;
        if (log) *log = "loading the specialised kernel failed";
      }
    } else if (log) {
      size_t ls = 0;
      nv.log_size(prog, &ls);
      std::string l(ls, '\0');
      nv.log(prog, &l[0]);
      *log = l;
    }
    nv.destroy(&prog);
  }
  if (k) c.kernels[src] = k;
  else c.failed[src] = true;
  return k;
}

std::string body_fn(const std::string& body, const char* name = "sg_body") {
  return std::string("template <class A> __device__ __forceinline__ void ") + name +
         "(const A& a, const float* x, "
         "long long i, float* o, unsigned& hit, float& rv, bool& rm) {\n"
         "  bool mask = true;\n  (void)x; (void)i; (void)o; (void)hit; (void)rv; "
         "(void)rm; (void)a;\n" +
         body + "  (void)mask;\n}\n";
}

}  // namespace

bool jit_available() { return nvrtc().ok; }

// Returns the specialised kernel, compiling it on first use; nullptr when it
// cannot be built (then the caller uses the interpreting kernel).
cudaKernel_t jit_stream_kernel(const Prog& pr, int nin, int nout, int npred, bool reduce,
                               bool minmax, uint32_t pred_exists, std::string* log) {
  if (!nvrtc().ok) {
    if (log) *log = "NVRTC library not found";
    return nullptr;
  }
  std::string body;
  if (!gen_body(pr, pred_exists, &body)) {
    if (log) *log = "program could not be specialised";
    return nullptr;
  }
  char defs[320];
  snprintf(defs, sizeof defs,
           "#define SG_NIN %d\n#define SG_NX %d\n#define SG_NOUT %d\n#define SG_NO %d\n"
           "#define SG_NPRED %d\n#define SG_RED %d\n#define SG_MINMAX %d\n",
           nin, nin > 0 ? nin : 1, nout, nout > 0 ? nout : 1, npred, reduce ? 1 : 0,
           minmax ? 1 : 0);
  const std::string src = std::string(defs) + kTemplateHead + body_fn(body) + kTemplateKernel;
  return compile_cached(src, "sg_fused", log);
}

cudaKernel_t jit_batch_kernel(const Prog& pr, std::string* log) {
  if (!nvrtc().ok) {
    if (log) *log = "NVRTC library not found";
    return nullptr;
  }
  std::string body;
  if (!gen_body(pr, 0u, &body)) {
    if (log) *log = "program could not be specialised";
    return nullptr;
  }
  const std::string src =
      std::string("#define SG_MINMAX 0\n") + kTemplateHead + body_fn(body) + kTemplateBatch;
  return compile_cached(src, "sg_batch", log);
}

namespace {

// the source of the specialised filter for `pred` with `tile`-item tiles;
// false (with a reason in *log) when it cannot be specialised
bool filter_source(const Prog& pred, int tile, std::string* src, std::string* log,
                   const Prog* post = nullptr) {
  if (tile != 2048 && tile != 4096 && tile != 8192) {
    if (log) *log = "unsupported filter tile";
    return false;
  }
  if (!nvrtc().ok) {
    if (log) *log = "NVRTC library not found";
    return false;
  }
  if (pred.nops <= 0 || pred.nops >= kMaxProg) {
    if (log) *log = "program could not be specialised";
    return false;
  }
  // the predicate's value is the program's result: a trailing reduce sink
  // hands it to the template as rv
  Prog pr = pred;
  pr.op[pr.nops] = K_REDUCE;
  pr.arg[pr.nops] = 0;
  pr.cst[pr.nops] = 0.0f;
  pr.nops += 1;
  std::string body;
  if (!gen_body(pr, 0u, &body)) {
    if (log) *log = "program could not be specialised";
    return false;
  }
  // the folded postcondition: the same form, its constants after the
  // predicate's and its sink
  std::string post_body;
  if (post) {
    const int b = jit_filter_post_base(pred);
    if (post->nops <= 0 || b + post->nops + 1 > kMaxProg) {
      if (log) *log = "postcondition could not be folded";
      return false;
    }
    Prog pp = *post;
    pp.op[pp.nops] = K_REDUCE;
    pp.arg[pp.nops] = 0;
    pp.cst[pp.nops] = 0.0f;
    pp.nops += 1;
    if (!gen_body(pp, 0u, &post_body, b)) {
      if (log) *log = "postcondition could not be specialised";
      return false;
    }
  }
  // resident CTAs per SM the compiler plans for: 48 registers at 8192
  // items, 40 at 4096, 32 at 2048
  char defs[160];
  snprintf(defs, sizeof defs, "#define SG_MINMAX 0\n#define SG_FT %d\n#define SG_FQ %d\n"
           "#define SG_FMINB %d\n#define SG_POST %d\n", tile, tile / 1024,
           filter_tile_occupancy(tile), post ? 1 : 0);
  *src = std::string(defs) + kTemplateHead + body_fn(body) +
         (post ? body_fn(post_body, "sg_post") : std::string()) + kTemplateFilter;
  return true;
}

}  // namespace

int filter_tile_occupancy(int tile) { return tile >= 8192 ? 5 : tile >= 4096 ? 6 : 8; }

cudaKernel_t jit_filter_kernel(const Prog& pred, std::string* log, int tile, const Prog* post) {
  std::string src;
  if (!filter_source(pred, tile, &src, log, post)) return nullptr;
  return compile_cached(src, "sg_filter", log);
}

bool jit_check_filter(const Prog& pred, std::string* log, const Prog* post) {
  Nvrtc& nv = nvrtc();
  if (!nv.ok) {
    if (log) *log = "NVRTC library not found";
    return false;
  }
  for (int tile : {2048, 4096, 8192}) {
    std::string src;
    if (!filter_source(pred, tile, &src, log, post)) return false;
    void* prog = nullptr;
    if (nv.create(&prog, src.c_str(), "sg_filter.cu", 0, nullptr, nullptr) != 0) {
      if (log) *log = "NVRTC could not create the program";
      return false;
    }
    const char* opts[] = {"--gpu-architecture=sm_103a", "--std=c++17", "-default-device",
                          "-fmad=false"};
    const bool ok = nv.compile(prog, 4, opts) == 0;
    if (!ok && log) {
      size_t ls = 0;
      nv.log_size(prog, &ls);
      std::string l(ls, '\0');
      nv.log(prog, &l[0]);
      *log = l;
    }
    nv.destroy(&prog);
    if (!ok) return false;
  }
  return true;
}

cudaError_t launch_jit_stream(cudaKernel_t k, const StreamArgs& s, int grid, int block,
                              cudaStream_t st, Prof* prof) {
  JitArgs a{};
  for (int i = 0; i < kMaxIn; ++i) a.in[i] = s.in[i];
  for (int i = 0; i < kMaxOut; ++i) a.out[i] = s.out[i];
  a.n = s.n;
  for (int i = 0; i < kMaxProg; ++i) a.cst[i] = s.prog.cst[i];
  a.partials = s.partials;
  a.counter = s.counter;
  a.result = s.result;
  a.count = s.count;
  a.vec4 = s.vec4;
  void* args[] = {&a};
  prof_begin(prof, "stream_jit", st);
  cudaError_t e = cudaLaunchKernel((const void*)k, dim3(grid), dim3(block), args, 0, st);
  prof_end(prof, st);
  return e;
}

}  // namespace sgk
