// k_filter.cu -- `filter` of Table 2 (sm_103a): the items for which the
// predicate holds, in index order (a stable stream compaction).
//
// One CTA per 4096-element tile, tiles taken in launch order from a global
// ticket.  The tile is staged through shared memory with 128-bit loads, each
// thread evaluates the predicate on 16 consecutive items, a block scan gives
// every kept item its rank inside the tile, and a decoupled look-back over
// the tile counts of earlier tiles (one warp, 32 tiles' words per memory
// round trip, bounded waits) gives the tile's global output offset.  Kept
// items are packed in shared memory and written out contiguously, so both the
// read and the write are coalesced: 4n bytes read, 4m bytes written for m
// kept items.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "sg_eval.cuh"
#include "sg_jit.h"

namespace sgk {
namespace {

constexpr int kFB = 256;
constexpr int kFK = 16;
constexpr int kFTile = kFB * kFK;
constexpr unsigned long long kFAgg = 1ull << 62;
constexpr unsigned long long kFPre = 2ull << 62;
constexpr unsigned long long kFCnt = (1ull << 62) - 1;
constexpr unsigned kFSpin = 1u << 22;

struct FilterHdr {
  unsigned tile_ctr;
  unsigned pad[63];
};

__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <int DEPTH>
__global__ void __launch_bounds__(kFB) k_filter(const float* __restrict__ x,
                                                float* __restrict__ out, long long n,
                                                const StreamArgs a, unsigned long long* st,
                                                FilterHdr* h, FilterResult* res,
                                                const LookbackCtl lb) {
  __shared__ float s_v[kFTile];
  __shared__ unsigned s_warp[kFB / 32];
  __shared__ unsigned s_tile;
  __shared__ unsigned s_total;
  __shared__ unsigned long long s_excl;
  const int tid = threadIdx.x;
  if (tid == 0) s_tile = atomicAdd(&h->tile_ctr, 1u);
  __syncthreads();
  const unsigned tile = s_tile;
  const long long base = (long long)tile * kFTile;
  const int valid = (int)(n - base < kFTile ? n - base : kFTile);

  // stage the tile (coalesced)
  if (valid == kFTile && (((uintptr_t)(x + base)) & 15) == 0) {
#pragma unroll
    for (int q = 0; q < kFK / 4; ++q) {
      const int i4 = tid + q * kFB;
      const float4 t = __ldcs(reinterpret_cast<const float4*>(x + base) + i4);
      reinterpret_cast<float4*>(s_v)[i4] = t;
    }
  } else {
    for (int i = tid; i < valid; i += kFB) s_v[i] = __ldcs(x + base + i);
  }
  __syncthreads();

  // predicate on 16 consecutive items per thread
  float v[kFK];
  unsigned keep = 0;
#pragma unroll
  for (int g = 0; g < kFK / 4; ++g) {
    float xx[1][4];
    const int i0 = tid * kFK + g * 4;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      xx[0][l] = (i0 + l < valid) ? s_v[i0 + l] : 0.0f;
      v[g * 4 + l] = xx[0][l];
    }
    float r[4];
    ev::eval_value<4, 1, DEPTH>(a, xx, base + i0, r);
#pragma unroll
    for (int l = 0; l < 4; ++l)
      if (i0 + l < valid && r[l] != 0.0f) keep |= 1u << (g * 4 + l);
  }
  const unsigned cnt = __popc(keep);

  // block exclusive scan of the counts
  const int lane = tid & 31, w = tid >> 5;
  unsigned incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[w] = incl;
  __syncthreads();
  if (w == 0) {
    unsigned t = lane < kFB / 32 ? s_warp[lane] : 0;
    unsigned ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += y;
    }
    if (lane < kFB / 32) s_warp[lane] = ti - t;
    if (lane == kFB / 32 - 1) s_total = ti;
  }
  __syncthreads();
  const unsigned excl_tile = incl - cnt + s_warp[w];
  const unsigned total = s_total;

  // decoupled look-back over earlier tiles' counts, by warp 0: lane l reads
  // the word of tile j - l, so one memory round trip covers up to 32 tiles.
  // The window is taken in order through its first inclusive prefix, or up
  // to its first word not yet published, which is then polled again.  Every
  // word is written once as an aggregate and once as an inclusive prefix
  // (tile 0 only as the prefix), so any published value read is a valid step;
  // below tile 0 stands an empty prefix (never reached).
  if (tid < 32) {
    unsigned long long excl = 0;
    const bool publish = (int)tile != lb.skip_tile;
    const unsigned limit = lb.spin_limit ? lb.spin_limit : kFSpin;
    if (tile == 0) {
      if (tid == 0 && publish) st_relaxed64(&st[0], kFPre | total);
    } else {
      if (tid == 0 && publish) st_relaxed64(&st[tile], kFAgg | total);
      long long j = (long long)tile - 1;
      unsigned spins = 0;
      while (true) {
        const long long idx = j - tid;
        const unsigned long long s = idx >= 0 ? ld_relaxed64(&st[idx]) : kFPre;
        const unsigned long long flag = s & ~kFCnt;
        const unsigned zero = __ballot_sync(0xffffffffu, flag == 0);
        const unsigned pre = __ballot_sync(0xffffffffu, flag == kFPre);
        const unsigned stop = zero ? (unsigned)(__ffs(zero) - 1) : 32u;
        const unsigned first_pre = pre ? (unsigned)(__ffs(pre) - 1) : 32u;
        const bool done = first_pre < stop;
        const unsigned take = done ? first_pre + 1 : stop;   // lanes [0, take) are added
        unsigned long long c = (unsigned)tid < take ? (s & kFCnt) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        excl += c;
        if (done) break;
        j -= take;
        if (stop < 32u) {
          if (++spins > limit) {
            if (tid == 0) atomicExch(&res->timeout, 1);
            break;
          }
          if (spins > 32) __nanosleep(64);
        }
      }
      if (tid == 0 && publish) st_relaxed64(&st[tile], kFPre | (excl + total));
    }
    if (tid == 0) {
      s_excl = excl;
      if (tile == gridDim.x - 1) res->count = (long long)(excl + total);
    }
  }
  __syncthreads();   // everyone has read s_v into registers

  // pack the kept items in shared memory, then write them out contiguously
  unsigned r = excl_tile;
#pragma unroll
  for (int k = 0; k < kFK; ++k)
    if (keep & (1u << k)) s_v[r++] = v[k];
  __syncthreads();
  const unsigned long long gb = s_excl;
  for (unsigned i = tid; i < total; i += kFB) {
    const unsigned long long pos = gb + i;
    if (pos < (unsigned long long)n) out[pos] = s_v[i];
  }
}

}  // namespace

size_t filter_scratch_bytes(long long n) {
  const size_t ntiles = (size_t)((n + kFTile - 1) / kFTile);
  return sizeof(FilterHdr) + ntiles * sizeof(unsigned long long) + 256;
}

size_t filter_jit_scratch_bytes(long long n) {
  const size_t ntiles = (size_t)((n + kJitFilterMinTile - 1) / kJitFilterMinTile);
  return std::max(filter_scratch_bytes(n), sizeof(FilterHdr) + ntiles * sizeof(unsigned long long) + 256);
}

cudaError_t launch_filter(const float* x, float* out, long long n, const Prog& pred,
                          int pred_depth, void* scratch, FilterResult* res, cudaStream_t s,
                          int num_sms, int64_t* kernels, Prof* prof, const LookbackCtl& lb) {
  (void)num_sms;
  if (n <= 0) return cudaSuccess;   // count stays 0 (result record was zeroed)
  const unsigned ntiles = (unsigned)((n + kFTile - 1) / kFTile);
  FilterHdr* h = static_cast<FilterHdr*>(scratch);
  unsigned long long* st = reinterpret_cast<unsigned long long*>(static_cast<char*>(scratch) +
                                                                 sizeof(FilterHdr));
  cudaError_t e = cudaMemsetAsync(scratch, 0, filter_scratch_bytes(n), s);
  if (e != cudaSuccess) return e;
  StreamArgs a{};
  a.prog = pred;
  a.nin = 1;
  a.depth = pred_depth;
  prof_begin(prof, "filter", s);
  if (pred_depth > 4)
    k_filter<8><<<ntiles, kFB, 0, s>>>(x, out, n, a, st, h, res, lb);
  else
    k_filter<4><<<ntiles, kFB, 0, s>>>(x, out, n, a, st, h, res, lb);
  prof_end(prof, s);
  *kernels += 1;
  return cudaGetLastError();
}

cudaError_t launch_filter_specialised(cudaKernel_t k, const float* x, float* out, long long n,
                                      const Prog& pred, void* scratch, FilterResult* res,
                                      cudaStream_t s, int num_sms, int64_t* kernels,
                                      Prof* prof, const LookbackCtl& lb, int tile,
                                      const Prog* post) {
  // the scratch (filter_jit_scratch_bytes) holds one look-back word per tile
  // of the smallest tile
  if (n <= 0) return cudaSuccess;
  if (tile < kJitFilterMinTile) return cudaErrorInvalidValue;
  const unsigned ntiles = (unsigned)((n + tile - 1) / tile);
  FilterHdr* h = static_cast<FilterHdr*>(scratch);
  cudaError_t e = cudaMemsetAsync(
      scratch, 0, sizeof(FilterHdr) + (size_t)ntiles * sizeof(unsigned long long) + 256, s);
  if (e != cudaSuccess) return e;
  (void)num_sms;   // one CTA per tile
  const void* fn = reinterpret_cast<const void*>(k);
  const int grid = (int)ntiles;
  FilterJitArgs a{};
  a.x = x;
  a.out = out;
  a.n = n;
  for (int i = 0; i < kMaxProg; ++i) a.cst[i] = pred.cst[i];
  if (post) {
    // the postcondition's constants follow the predicate's and its sink
    const int b = jit_filter_post_base(pred);
    if (b + post->nops > kMaxProg) return cudaErrorInvalidValue;
    for (int i = 0; i < post->nops; ++i) a.cst[b + i] = post->cst[i];
  }
  a.st = reinterpret_cast<unsigned long long*>(static_cast<char*>(scratch) + sizeof(FilterHdr));
  a.tile_ctr = &h->tile_ctr;
  a.res = res;
  a.ntiles = ntiles;
  a.skip_tile = lb.skip_tile;
  a.spin_limit = lb.spin_limit ? lb.spin_limit : kFSpin;
  void* args[] = {&a};
  prof_begin(prof, "filter_jit", s);
  e = cudaLaunchKernel(fn, dim3(grid), dim3(kFB), args, 0, s);
  prof_end(prof, s);
  *kernels += 1;
  return e;
}

// ---------------------------------------------------------------------------
// Allocation-free filter.  Some callers cannot allocate device memory: a
// serving runtime that reserves all of HBM in its own pool at start-up and
// forbids later allocations, a latency-critical path that cannot afford the
// device-wide synchronisation cudaMalloc may imply, or a plugin host that
// hands out only the input and output buffers.  For them the look-back
// scratch of the filter lives in this fixed device array instead of memory
// the library allocates.  Every GPU that loads the library holds the array
// until the process exits.  There is no counterpart in the paper.

static_assert(SG_FILTER_NOALLOC_SCRATCH_BYTES >=
                  256 + sizeof(FilterHdr) +
                      ((SG_FILTER_NOALLOC_MAX_N + kFTile - 1) / kFTile) * sizeof(unsigned long long) +
                      256,
              "the fixed scratch must hold the result record and the filter scratch");

static __device__ __align__(256) unsigned char sg_filter_noalloc_scratch[SG_FILTER_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices];   // device address of the array, per device

}  // namespace
}  // namespace sgk

namespace sgk {
namespace {

// the program of a filter predicate over input slot 0, with its stack
// depths; SG_ERR_INVALID_ARG when it is malformed (the library's one
// expression validator, as sg_filter uses)
sg_status filter_prog(const sg_expr* pred, Prog* pr, int* max_depth) {
  memset(pr, 0, sizeof *pr);
  const sg_status st = validate_expr(pred, 1, max_depth, pr->depth, nullptr, 0);
  if (st != SG_OK) return st;
  for (int p = 0; p < pred->nops; ++p) {
    pr->op[p] = (uint8_t)pred->ops[p].op;
    pr->arg[p] = 0;
    pr->cst[p] = pred->ops[p].value;
  }
  pr->nops = pred->nops;
  return SG_OK;
}

}  // namespace
}  // namespace sgk

extern "C" sg_status sg_debug_jit_check_filter_post(const sg_expr* pred, const sg_expr* post,
                                                     char* log, size_t cap) {
  using namespace sgk;
  if (log && cap > 0) log[0] = '\0';
  Prog pr, pp;
  int md = 0;
  sg_status st = filter_prog(pred, &pr, &md);
  if (st != SG_OK) return st;
  if (post) {
    st = filter_prog(post, &pp, &md);
    if (st != SG_OK) return st;
  }
  std::string l;
  if (jit_check_filter(pr, &l, post ? &pp : nullptr)) return SG_OK;
  if (log && cap > 0) {
    const size_t k = l.size() < cap - 1 ? l.size() : cap - 1;
    memcpy(log, l.data(), k);
    log[k] = '\0';
  }
  return SG_ERR_UNSUPPORTED;
}

extern "C" sg_status sg_debug_jit_check_filter(const sg_expr* pred, char* log, size_t cap) {
  return sg_debug_jit_check_filter_post(pred, nullptr, log, cap);
}

extern "C" sg_status sg_filter_noalloc(const sg_expr* pred, const float* dev_x, int64_t n,
                                       float* dev_out, int64_t* dev_count, void* stream) {
  using namespace sgk;
  if (!pred || n < 0 || (n > 0 && (!dev_x || !dev_out)) || !dev_count) return SG_ERR_INVALID_ARG;
  if (n > SG_FILTER_NOALLOC_MAX_N) return SG_ERR_SHAPE;
  // the predicate: one input slot, checked and given its stack depths here
  Prog pr;
  int md = 0;
  {
    const sg_status st = filter_prog(pred, &pr, &md);
    if (st != SG_OK) return st;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // set-up, once per device, with that device current: the array's device
  // address (the host-side symbol is only a stand-in, never a device pointer)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return SG_ERR_CUDA;
  }
  if (dev < 0 || dev >= kNoAllocMaxDevices) return SG_ERR_UNSUPPORTED;
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, sg_filter_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return SG_ERR_CUDA;
      }
      g_noalloc_ptr[dev] = p;
    }
    base = g_noalloc_ptr[dev];
  }
  FilterResult* res = static_cast<FilterResult*>(base);
  void* scratch = static_cast<char*>(base) + 256;

  // the array keeps the previous call's contents: clear the result record
  // and the look-back words this call uses
  cudaError_t e = cudaMemsetAsync(res, 0, sizeof(FilterResult), s);
  if (e == cudaSuccess && n > 0) {
    int64_t kernels = 0;
    // the interpreting kernel: the specialised one would need a module
    // load, which allocates device memory
    e = launch_filter(dev_x, dev_out, n, pr, md, scratch, res, s, 0, &kernels, nullptr,
                      LookbackCtl{0, -1});
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dev_count, &res->count, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
  FilterResult h{};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&h, res, sizeof h, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && h.timeout) {
    // the count of a compaction whose look-back gave up is not a count
    e = cudaMemsetAsync(dev_count, 0xff, sizeof(int64_t), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SG_ERR_CUDA;
  }
  return h.timeout ? SG_ERR_TIMEOUT : SG_OK;
}
