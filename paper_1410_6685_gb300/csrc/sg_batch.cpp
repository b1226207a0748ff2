// sg_batch.cpp -- sg_batch_run: the batched-collections chain, captured once
// into a CUDA graph per (chain, pointers, sizes, schedule) and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>

#include "sg_batch.h"
#include "sg_runtime.h"
#include "sg_sched.h"

namespace {

sg_status bad(sg_ctx* c, sg_status s, const char* msg) {
  if (c) c->err = msg;
  return s;
}

bool expr_ok(const sg_expr& e) {
  if (e.nops <= 0 || e.nops > SG_MAX_EXPR_OPS) return false;
  int d = 0;
  for (int p = 0; p < e.nops; ++p) {
    const int op = e.ops[p].op;
    int need = 0, delta = 0;
    switch (op) {
      case SG_OP_LOAD: if (e.ops[p].arg != 0) return false; delta = 1; break;
      case SG_OP_CONST: case SG_OP_INDEX: delta = 1; break;
      case SG_OP_FMA: case SG_OP_SELECT: need = 3; delta = -2; break;
      case SG_OP_NEG: case SG_OP_ABS: case SG_OP_SQRT: case SG_OP_NOT: need = 1; break;
      case SG_OP_DUP: need = 1; delta = 1; break;
      case SG_OP_SWAP: need = 2; break;
      default:
        if (op < SG_OP_ADD || op > SG_OP_INDEX) return false;
        need = 2; delta = -1;
    }
    if (d < need) return false;
    d += delta;
    if (d > SG_MAX_EXPR_DEPTH) return false;
  }
  return d == 1;
}

}  // namespace

BatchPlanCache::~BatchPlanCache() {
  for (auto& kv : plans) {
    BatchPlan& p = kv.second;
    if (p.exec) cudaGraphExecDestroy(p.exec);
    if (p.scratch) cudaFree(p.scratch);
    if (p.host_flag) cudaFreeHost(p.host_flag);
  }
  if (capture_stream) cudaStreamDestroy(capture_stream);
}

extern "C" sg_status sg_batch_run(sg_ctx* c, const sg_chain* ch, const float* data,
                                  const int64_t* offsets, int64_t nseg, double* sums,
                                  int64_t* first_viol, int64_t* kept) {
  if (!c || !ch || nseg < 0) return bad(c, SG_ERR_INVALID_ARG, "bad batch arguments");
  if (c->planning_only) return bad(c, SG_ERR_UNSUPPORTED, "planning-only context");
  if (nseg > 0 && (!data || !offsets || !sums || !first_viol || !kept))
    return bad(c, SG_ERR_INVALID_ARG, "null device pointer");
  if (!expr_ok(ch->map) || !expr_ok(ch->pre) || !expr_ok(ch->keep))
    return bad(c, SG_ERR_INVALID_ARG, "chain expressions must be 1-input programs");
  if (nseg == 0) return SG_OK;
  sgk::Prog prog;
  int depth = 0;
  if (!sgk::build_chain_prog(*ch, &prog, &depth))
    return bad(c, SG_ERR_INVALID_ARG, "chain program too long or too deep");

  // everything queued before runs first (same stream order as a flush)
  sg_status st = sg_flush(c);
  if (st && st != SG_ERR_PRECONDITION && st != SG_ERR_POSTCONDITION) return st;

  const sg_sched_choice sch = sg_choose_batch_schedule(c, nseg, depth);
  BatchKey key;
  memcpy(&key.chain, ch, sizeof *ch);
  key.data = data;
  key.offsets = offsets;
  key.nseg = nseg;
  key.sums = sums;
  key.first = first_viol;
  key.kept = kept;
  key.chunk = sch.chunk;
  key.grid_per_sm = sch.blocks_per_sm;
  BatchPlanCache& cache = c->batch;
  if (!cache.capture_stream) {
    if (cudaStreamCreateWithFlags(&cache.capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return bad(c, SG_ERR_CUDA, "capture stream creation failed");
    }
  }
  for (int attempt = 0; attempt < 3; ++attempt) {
    BatchPlan* plan = nullptr;
    for (auto& kv : cache.plans)
      if (memcmp(&kv.first, &key, sizeof key) == 0) plan = &kv.second;
    if (!plan) {
      // capacity: one chunk per collection plus the chunks the elements need
      // (the total is read once; the kernel reports an overflow if the
      // offsets change under the same pointers)
      int64_t total = 0;
      cudaError_t e = cudaMemcpyAsync(&total, offsets + nseg, sizeof total,
                                      cudaMemcpyDeviceToHost, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      if (e != cudaSuccess) return bad(c, SG_ERR_CUDA, cudaGetErrorString(e));
      BatchPlan p;
      p.capacity = nseg + total / sch.chunk + 1 + (attempt ? 2 * nseg : 0);
      if (cudaMalloc(&p.scratch, sgk::batch_scratch_bytes(nseg, p.capacity)) != cudaSuccess ||
          cudaMallocHost((void**)&p.host_flag, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return bad(c, SG_ERR_OOM, "batch scratch allocation failed");
      }
      // the per-collection counters start at zero and return to zero
      cudaMemset(p.scratch, 0, sgk::batch_scratch_bytes(nseg, p.capacity));
      sgk::BatchLaunch L{};
      L.data = data;
      L.offsets = reinterpret_cast<const long long*>(offsets);
      L.nseg = nseg;
      L.chunk = sch.chunk;
      L.capacity = p.capacity;
      L.grid = std::max(1, c->num_sms * sch.blocks_per_sm);
      L.prog = prog;
      L.depth = depth;
      L.scratch = p.scratch;
      L.sums = sums;
      L.first_viol = reinterpret_cast<long long*>(first_viol);
      L.kept = reinterpret_cast<long long*>(kept);
      L.host_flag = p.host_flag;
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(cache.capture_stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t le = sgk::launch_batch(L, cache.capture_stream, nullptr);
        e = cudaStreamEndCapture(cache.capture_stream, &g);
        if (e == cudaSuccess) e = le;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&p.exec, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(p.scratch);
        cudaFreeHost(p.host_flag);
        return bad(c, SG_ERR_CUDA, "batch graph capture failed");
      }
      cache.plans.emplace_back(key, p);
      plan = &cache.plans.back().second;
    }
    const bool prof = c->prof.on;
    if (prof) sgk::prof_begin(&c->prof, "batch_graph", c->stream);
    cudaError_t e = cudaGraphLaunch(plan->exec, c->stream);
    if (prof) sgk::prof_end(&c->prof, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return bad(c, SG_ERR_CUDA, cudaGetErrorString(e));
    if (prof) c->prof.collect();
    c->kernels += 2;
    const unsigned flag = *plan->host_flag;
    if (flag & 2u) {
      // offsets changed under the same pointers: rebuild with more room
      cudaGraphExecDestroy(plan->exec);
      cudaFree(plan->scratch);
      cudaFreeHost(plan->host_flag);
      for (auto it = cache.plans.begin(); it != cache.plans.end(); ++it)
        if (&it->second == plan) {
          cache.plans.erase(it);
          break;
        }
      continue;
    }
    sg_record_batch_timing(c, nseg, sch);
    if (flag & 1u) {
      c->err = "a collection violated the batch precondition";
      return SG_ERR_PRECONDITION;
    }
    return SG_OK;
  }
  return bad(c, SG_ERR_CUDA, "batch work list overflowed twice");
}
