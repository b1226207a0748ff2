// k_batch.cu -- batched collections (sm_103a): thousands of collections of
// uneven size through one persistent launch, each running the chain
//     y = map(x);  require for_all(pre(y));  s = sum(filter(y, keep))
// (project / for_all / filter / sum of Table 2 and Sec. 3.3, per collection).
// The filter result is consumed only by the sum, so it is a masked sum and
// is never built.
//
// Work list: every collection is cut into chunks of `chunk` elements (an
// empty collection still gets one chunk).  A one-block prep kernel scans the
// chunk counts and a second kernel writes each chunk's collection; the
// persistent kernel's CTAs then take chunks from a global ticket, evaluate
// the fused program and leave a per-chunk partial.  The program is either
// interpreted (this file) or compiled at run time into straight-line code
// (the same kernel, specialised by sg_jit.cpp).  The CTA that finishes a
// collection's last chunk (per-collection counter) combines the partials in
// chunk order, so results do not depend on scheduling.  All counters return
// to zero, so the captured CUDA graph can be replayed as is.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "sg_batch.h"
#include "sg_eval.cuh"
#include "sg_jit.h"

namespace sgk {
namespace {

constexpr int kBB = 256;
constexpr long long kNone = 0x7fffffffffffffffLL;

struct ChunkPartial {
  double sum;
  long long cnt;
  long long first;
};

struct BatchHdr {
  unsigned ticket;
  unsigned any_violation;   // bit 0: a precondition failed; bit 1: overflow
  unsigned long long total_chunks;
  unsigned pad[60];
};

// chunk_start[s] = number of chunks before collection s (exclusive scan)
__global__ void __launch_bounds__(1024) k_batch_prep(const long long* __restrict__ off,
                                                     long long nseg, long long chunk,
                                                     long long capacity,
                                                     long long* chunk_start, BatchHdr* h) {
  __shared__ long long s_warp[32];
  __shared__ long long s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (long long b = 0; b < nseg; b += blockDim.x) {
    const long long s = b + threadIdx.x;
    long long c = 0;
    if (s < nseg) {
      const long long L = off[s + 1] - off[s];
      c = L > 0 ? (L + chunk - 1) / chunk : 1;
    }
    long long x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    if (w == 0) {
      const int nw = blockDim.x / 32;
      long long t = lane < nw ? s_warp[lane] : 0;
      long long ti = t;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, ti, o);
        if (lane >= o) ti += y;
      }
      if (lane < nw) s_warp[lane] = ti - t;
    }
    __syncthreads();
    const long long excl = s_carry + s_warp[w] + x - c;
    if (s < nseg) chunk_start[s] = excl;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_carry = excl + c;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    chunk_start[nseg] = s_carry;
    // more work items than the scratch holds: do nothing, report overflow
    h->total_chunks = s_carry <= capacity ? (unsigned long long)s_carry : 0ull;
    if (s_carry > capacity) h->any_violation |= 2u;
    h->ticket = 0;
  }
}

// chunk_seg[chunk_start[s] + c] = s for every chunk c of collection s
__global__ void k_batch_map(const long long* __restrict__ chunk_start, long long nseg,
                            long long capacity, int* chunk_seg) {
  if (chunk_start[nseg] > capacity) return;   // overflow: the batch kernel does nothing
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < nseg;
       s += (long long)gridDim.x * blockDim.x) {
    const long long c0 = chunk_start[s], c1 = chunk_start[s + 1];
    for (long long c = c0; c < c1; ++c) chunk_seg[c] = (int)s;
  }
}

template <int DEPTH, bool VEC>
__global__ void __launch_bounds__(kBB) k_batch(const float* __restrict__ data,
                                               const long long* __restrict__ off, long long nseg,
                                               long long chunk, const StreamArgs a,
                                               const long long* __restrict__ chunk_start,
                                               const int* __restrict__ chunk_seg,
                                               ChunkPartial* partials, unsigned* seg_done,
                                               BatchHdr* h, double* sums, long long* first_viol,
                                               long long* kept) {
  __shared__ unsigned long long s_item;
  __shared__ ev::Acc s_acc[kBB / 32];
  __shared__ bool s_last;
  const unsigned long long total = h->total_chunks;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(&h->ticket, 1u);
    __syncthreads();
    const unsigned long long item = s_item;
    __syncthreads();
    if (item >= total) break;
    const long long s = chunk_seg[item];
    const long long c = (long long)item - chunk_start[s];
    const long long nch = chunk_start[s + 1] - chunk_start[s];
    const long long sb = off[s], se = off[s + 1];
    const long long b = sb + c * chunk;
    const long long e = b + chunk < se ? b + chunk : se;

    ev::Acc acc;
    ev::acc_init(acc);
    if (VEC) {
      // 16-byte quads of the whole data array, four consecutive elements per
      // thread; lanes outside [b, e) are masked
      const long long q0 = b >> 2, q1 = (e + 3) >> 2;
      for (long long q = q0 + threadIdx.x; q < q1; q += kBB) {
        const float4 t = __ldcs(reinterpret_cast<const float4*>(data) + q);
        float x[1][4] = {{t.x, t.y, t.z, t.w}};
        bool vm[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          const long long j = (q << 2) + l;
          vm[l] = j >= b && j < e;
        }
        ev::run_prog<4, 1, DEPTH>(a, x, (q << 2) - sb, vm, acc);
      }
    } else {
      for (long long i = b + threadIdx.x; i < e; i += kBB) {
        float x[1][1] = {{__ldcs(data + i)}};
        const bool vm[1] = {true};
        ev::run_prog<1, 1, DEPTH>(a, x, i - sb, vm, acc);
      }
    }
    // block reduction (fixed order)
    ev::acc_fold(acc);
    ev::warp_reduce(acc);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) s_acc[w] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      ev::Acc tot = s_acc[0];
      for (int k = 1; k < kBB / 32; ++k) ev::acc_merge(tot, s_acc[k]);
      if (nch == 1) {
        sums[s] = tot.sum;
        kept[s] = tot.cnt;
        first_viol[s] = tot.first[0] == kNone ? -1 : tot.first[0];
        if (tot.first[0] != kNone) atomicOr(&h->any_violation, 1u);
        s_last = false;
      } else {
        ChunkPartial p{tot.sum, tot.cnt, tot.first[0]};
        partials[chunk_start[s] + c] = p;
        __threadfence();
        s_last = atomicAdd(&seg_done[s], 1u) == (unsigned)(nch - 1);
      }
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
      __threadfence();
      double sum = 0.0;
      long long cnt = 0, first = kNone;
      for (long long k = 0; k < nch; ++k) {
        const ChunkPartial* p = &partials[chunk_start[s] + k];
        sum += __ldcg(&p->sum);
        cnt += __ldcg(&p->cnt);
        const long long f = __ldcg(&p->first);
        first = f < first ? f : first;
      }
      sums[s] = sum;
      kept[s] = cnt;
      first_viol[s] = first == kNone ? -1 : first;
      if (first != kNone) atomicOr(&h->any_violation, 1u);
      seg_done[s] = 0;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// host: program building, scratch, graph cache

struct HostOp {
  uint8_t op;
  float cst;
};

void append_with(std::vector<HostOp>& out, const sg_expr& e, const std::vector<HostOp>& load0) {
  for (int p = 0; p < e.nops; ++p) {
    if (e.ops[p].op == SG_OP_LOAD) out.insert(out.end(), load0.begin(), load0.end());
    else out.push_back(HostOp{(uint8_t)e.ops[p].op, e.ops[p].value});
  }
}

int stack_delta(uint8_t op, int* need) {
  switch (op) {
    case SG_OP_LOAD: case SG_OP_CONST: case SG_OP_INDEX: *need = 0; return 1;
    case SG_OP_FMA: case SG_OP_SELECT: *need = 3; return -2;
    case SG_OP_NEG: case SG_OP_ABS: case SG_OP_SQRT: case SG_OP_NOT: *need = 1; return 0;
    case SG_OP_DUP: *need = 1; return 1;
    case SG_OP_SWAP: *need = 2; return 0;
    case K_STORE: *need = 1; return 0;
    case K_PRED: case K_MASK: case K_REDUCE: case K_POP: *need = 1; return -1;
    default: *need = 2; return -1;
  }
}

}  // namespace

bool build_chain_prog(const sg_chain& ch, Prog* pr, int* depth, bool with_pre) {
  std::vector<HostOp> x{{SG_OP_LOAD, 0.0f}}, y, prog;
  append_with(y, ch.map, x);                       // y = map(x)
  if (with_pre) {
    append_with(prog, ch.pre, y);                  // pre(y)
    prog.push_back(HostOp{K_PRED, 0.0f});
  }
  append_with(prog, ch.keep, y);                   // keep(y)
  prog.push_back(HostOp{K_MASK, 0.0f});
  prog.insert(prog.end(), y.begin(), y.end());     // y
  prog.push_back(HostOp{K_REDUCE, 0.0f});
  if ((int)prog.size() > kMaxProg) return false;
  int d = 0, mx = 0;
  std::memset(pr, 0, sizeof *pr);
  pr->nops = (int)prog.size();
  for (size_t p = 0; p < prog.size(); ++p) {
    int need = 0;
    const int delta = stack_delta(prog[p].op, &need);
    if (d < need) return false;
    pr->op[p] = prog[p].op;
    pr->arg[p] = 0;
    pr->cst[p] = prog[p].cst;
    pr->depth[p] = (uint8_t)d;
    d += delta;
    mx = d > mx ? d : mx;
  }
  if (d != 0 || mx > kMaxDepth) return false;
  *depth = mx;
  return true;
}

size_t batch_scratch_bytes(long long nseg, long long capacity) {
  return sizeof(BatchHdr) + (size_t)(nseg + 1) * sizeof(long long) +
         (size_t)nseg * sizeof(unsigned) + (size_t)capacity * sizeof(ChunkPartial) +
         (size_t)capacity * sizeof(int) + 1280;
}

cudaError_t launch_batch(const BatchLaunch& L, cudaStream_t s, Prof* prof) {
  char* base = static_cast<char*>(L.scratch);
  BatchHdr* h = reinterpret_cast<BatchHdr*>(base);
  size_t o = (sizeof(BatchHdr) + 255) & ~(size_t)255;
  long long* chunk_start = reinterpret_cast<long long*>(base + o);
  o = (o + (size_t)(L.nseg + 1) * sizeof(long long) + 255) & ~(size_t)255;
  unsigned* seg_done = reinterpret_cast<unsigned*>(base + o);
  o = (o + (size_t)L.nseg * sizeof(unsigned) + 255) & ~(size_t)255;
  ChunkPartial* partials = reinterpret_cast<ChunkPartial*>(base + o);
  o = (o + (size_t)L.capacity * sizeof(ChunkPartial) + 255) & ~(size_t)255;
  int* chunk_seg = reinterpret_cast<int*>(base + o);

  StreamArgs a{};
  a.prog = L.prog;
  a.nin = 1;
  a.depth = L.depth;
  a.npred = 1;
  a.has_reduce = 1;
  cudaError_t e = cudaMemsetAsync(h, 0, sizeof(BatchHdr), s);
  if (e != cudaSuccess) return e;
  if (L.nseg == 0) return cudaSuccess;
  prof_begin(prof, "batch_prep", s);
  k_batch_prep<<<1, 1024, 0, s>>>(L.offsets, L.nseg, L.chunk, L.capacity, chunk_start, h);
  k_batch_map<<<(int)std::min<long long>((L.nseg + 255) / 256, 1024), 256, 0, s>>>(
      chunk_start, L.nseg, L.capacity, chunk_seg);
  prof_end(prof, s);
  const bool vec = ((uintptr_t)L.data & 15) == 0;
  if (L.jit) {
    BatchJitArgs ja{};
    ja.data = L.data;
    ja.off = L.offsets;
    ja.nseg = L.nseg;
    ja.chunk = L.chunk;
    for (int i = 0; i < kMaxProg; ++i) ja.cst[i] = L.prog.cst[i];
    ja.chunk_start = chunk_start;
    ja.chunk_seg = chunk_seg;
    ja.partials = partials;
    ja.seg_done = seg_done;
    ja.hdr = h;
    ja.sums = L.sums;
    ja.first_viol = L.first_viol;
    ja.kept = L.kept;
    ja.vec4 = vec ? 1 : 0;
    void* args[] = {&ja};
    prof_begin(prof, "batch_jit", s);
    e = cudaLaunchKernel((const void*)L.jit, dim3(L.grid), dim3(kBB), args, 0, s);
    prof_end(prof, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(L.host_flag, &h->any_violation, sizeof(unsigned), cudaMemcpyDeviceToHost,
                        s);
    return e == cudaSuccess ? cudaGetLastError() : e;
  }
  prof_begin(prof, "batch", s);
#define SG_BATCH(D, V)                                                                  \
  k_batch<D, V><<<L.grid, kBB, 0, s>>>(L.data, L.offsets, L.nseg, L.chunk, a, chunk_start, \
                                       chunk_seg, partials, seg_done, h, L.sums, L.first_viol, L.kept)
  if (L.depth > 4) {
    if (vec) SG_BATCH(8, true); else SG_BATCH(8, false);
  } else {
    if (vec) SG_BATCH(4, true); else SG_BATCH(4, false);
  }
#undef SG_BATCH
  prof_end(prof, s);
  e = cudaMemcpyAsync(L.host_flag, &h->any_violation, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

int batch_blocks_per_sm(int depth) {
  int nb = 0;
  cudaError_t e = depth > 4
      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<8, true>, kBB, 0)
      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<4, true>, kBB, 0);
  return e == cudaSuccess && nb > 0 ? nb : 1;
}

}  // namespace sgk
