// sg_batch.cpp -- sg_batch_run: the batched-collections chain, captured once
// into a CUDA graph per (chain, pointers, sizes, schedule) and replayed, with
// the schedule from the plain table, the autotuner or the learned model.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "sg_batch.h"
#include "sg_jit.h"
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

uint64_t chain_hash(const sg_chain& ch) {
  const unsigned char* p = reinterpret_cast<const unsigned char*>(&ch);
  uint64_t h = 1469598103934665603ull;   // FNV-1a
  for (size_t i = 0; i < sizeof ch; ++i) h = (h ^ p[i]) * 1099511628211ull;
  return h;
}

struct Job {
  const sg_chain* ch;
  const float* data;
  const int64_t* offsets;
  int64_t nseg;
  double* sums;
  int64_t* first;
  int64_t* kept;
  sgk::Prog prog;
  int depth;
  int occ;          // resident CTAs per SM of the kernel that will run
  bool with_pre;    // the precondition is checked (contract mode PRE or above)
  BatchStats stats;
};

sg_status read_stats(sg_ctx* c, Job& j) {
  std::vector<int64_t> off(j.nseg + 1);
  cudaError_t e = cudaMemcpyAsync(off.data(), j.offsets, off.size() * 8, cudaMemcpyDeviceToHost,
                                  c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bad(c, SG_ERR_CUDA, cudaGetErrorString(e));
  }
  BatchStats& w = j.stats;
  w.nseg = j.nseg;
  w.total = off[j.nseg] - off[0];
  double s = 0, s2 = 0, mn = 1e300, mx = -1e300;
  for (int64_t i = 0; i < j.nseg; ++i) {
    const int64_t L = off[i + 1] - off[i];
    if (L < 0) return bad(c, SG_ERR_INVALID_ARG, "offsets must be non-decreasing");
    const double l = std::log2((double)L + 1.0);
    s += l;
    s2 += l * l;
    mn = std::min(mn, l);
    mx = std::max(mx, l);
  }
  w.mean_log = s / (double)j.nseg;
  w.std_log = std::sqrt(std::max(0.0, s2 / (double)j.nseg - w.mean_log * w.mean_log));
  w.min_log = mn;
  w.max_log = mx;
  w.ops = j.prog.nops;
  w.depth = j.depth;
  return SG_OK;
}

// Runs the batch once with schedule `sch` (capturing its graph on first use)
// and times it with CUDA events.  *violated: a precondition failed.
sg_status run_with(sg_ctx* c, const Job& j, const sg_sched_choice& sch, double* us,
                   bool* violated) {
  BatchKey key;
  memset(&key, 0, sizeof key);
  memcpy(&key.chain, j.ch, sizeof *j.ch);
  key.data = j.data;
  key.offsets = j.offsets;
  key.nseg = j.nseg;
  key.sums = j.sums;
  key.first = j.first;
  key.kept = j.kept;
  key.chunk = sch.chunk;
  key.grid_per_sm = sch.blocks_per_sm;
  key.pad = c->codegen | (j.with_pre ? 0x100 : 0);
  BatchPlanCache& cache = c->batch;
  if (!cache.capture_stream) {
    if (cudaStreamCreateWithFlags(&cache.capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return bad(c, SG_ERR_CUDA, "capture stream creation failed");
    }
  }
  if (!cache.ev[0]) {
    cudaEventCreate(&cache.ev[0]);
    cudaEventCreate(&cache.ev[1]);
  }
  for (int attempt = 0; attempt < 3; ++attempt) {
    BatchPlan* plan = nullptr;
    for (auto& kv : cache.plans)
      if (memcmp(&kv.first, &key, sizeof key) == 0) plan = &kv.second;
    if (!plan) {
      BatchPlan p;
      p.capacity = j.nseg + j.stats.total / sch.chunk + 1 + (attempt ? 4 * j.nseg + 1024 : 0);
      if (cudaMalloc(&p.scratch, sgk::batch_scratch_bytes(j.nseg, p.capacity)) != cudaSuccess ||
          cudaMallocHost((void**)&p.host_flag, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return bad(c, SG_ERR_OOM, "batch scratch allocation failed");
      }
      // the per-collection counters start at zero and return to zero
      cudaMemset(p.scratch, 0, sgk::batch_scratch_bytes(j.nseg, p.capacity));
      sgk::BatchLaunch L{};
      L.data = j.data;
      L.offsets = reinterpret_cast<const long long*>(j.offsets);
      L.nseg = j.nseg;
      L.chunk = sch.chunk;
      L.capacity = p.capacity;
      L.grid = std::max(1, c->num_sms * sch.blocks_per_sm);
      L.prog = j.prog;
      L.depth = j.depth;
      L.scratch = p.scratch;
      L.sums = j.sums;
      L.first_viol = reinterpret_cast<long long*>(j.first);
      L.kept = reinterpret_cast<long long*>(j.kept);
      L.host_flag = p.host_flag;
      L.jit = c->codegen == SG_CODEGEN_SPECIALIZE ? sgk::jit_batch_kernel(j.prog, nullptr)
                                                  : nullptr;
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(cache.capture_stream, cudaStreamCaptureModeThreadLocal);
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
    cudaEventRecord(cache.ev[0], c->stream);
    cudaError_t e = cudaGraphLaunch(plan->exec, c->stream);
    cudaEventRecord(cache.ev[1], c->stream);
    if (prof) sgk::prof_end(&c->prof, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return bad(c, SG_ERR_CUDA, cudaGetErrorString(e));
    if (prof) c->prof.collect();
    c->kernels += 2;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, cache.ev[0], cache.ev[1]);
    const unsigned flag = *plan->host_flag;
    if (flag & 2u) {
      // the offsets changed under the same pointers: rebuild with more room
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
    if (us) *us = ms * 1000.0;
    *violated = (flag & 1u) != 0;
    return SG_OK;
  }
  return bad(c, SG_ERR_CUDA, "batch work list overflowed twice");
}

sg_status prepare(sg_ctx* c, const sg_chain* ch, const float* data, const int64_t* offsets,
                  int64_t nseg, double* sums, int64_t* first, int64_t* kept, Job* j) {
  if (!c || !ch || nseg < 0) return bad(c, SG_ERR_INVALID_ARG, "bad batch arguments");
  if (c->planning_only) return bad(c, SG_ERR_UNSUPPORTED, "planning-only context");
  if (nseg > 0 && (!data || !offsets || !sums || !first || !kept))
    return bad(c, SG_ERR_INVALID_ARG, "null device pointer");
  if (!expr_ok(ch->map) || !expr_ok(ch->pre) || !expr_ok(ch->keep))
    return bad(c, SG_ERR_INVALID_ARG, "chain expressions must be 1-input programs");
  j->ch = ch;
  j->data = data;
  j->offsets = offsets;
  j->nseg = nseg;
  j->sums = sums;
  j->first = first;
  j->kept = kept;
  // contract mode OFF (Sec. 6.3): the precondition is not compiled in, and
  // every first-violation index comes back -1
  j->with_pre = c->mode >= SG_CONTRACTS_PRE;
  if (!sgk::build_chain_prog(*ch, &j->prog, &j->depth, j->with_pre))
    return bad(c, SG_ERR_INVALID_ARG, "chain program too long or too deep");
  // the candidates' CTAs per SM follow the kernel that will run: the
  // specialised one when code generation is on, else the interpreter
  j->occ = 0;
  if (c->codegen == SG_CODEGEN_SPECIALIZE) {
    if (cudaKernel_t k = sgk::jit_batch_kernel(j->prog, nullptr)) {
      int nb = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)k, 256, 0) == cudaSuccess)
        j->occ = nb;
      cudaGetLastError();
    }
  }
  if (j->occ <= 0) j->occ = sgk::batch_blocks_per_sm(j->depth);
  if (nseg == 0) return SG_OK;
  // everything queued before runs first (same stream order as a flush)
  sg_status st = sg_flush(c);
  if (st && st != SG_ERR_PRECONDITION && st != SG_ERR_POSTCONDITION) return st;
  return read_stats(c, *j);
}

// Autotune: measure every candidate -- a warm-up run (graph capture, cold
// caches), then the better of two timed runs -- and log the sweep with each
// time relative to the plain table's choice.
sg_status autotune(sg_ctx* c, const Job& j, const std::vector<sg_sched_choice>& cand,
                   const std::vector<float>& X, int def, std::vector<double>* times, int* best) {
  times->assign(cand.size(), 0.0);
  double bt = 1e300;
  *best = 0;
  for (size_t i = 0; i < cand.size(); ++i) {
    bool viol = false;
    double us = 0.0, u2 = 0.0;
    sg_status st = run_with(c, j, cand[i], &us, &viol);
    if (!st) st = run_with(c, j, cand[i], &us, &viol);
    if (!st) st = run_with(c, j, cand[i], &u2, &viol);
    if (st) return st;
    us = std::min(us, u2);
    (*times)[i] = us;
    if (us < bt) {
      bt = us;
      *best = (int)i;
    }
  }
  sg_sched_log_sweep(c, SG_SCHED_BATCH, X, *times, def);
  return SG_OK;
}

// candidates, their features and the plain choice's index
void batch_candidates(sg_ctx* c, const Job& j, std::vector<sg_sched_choice>* cand,
                      std::vector<float>* X, int* def) {
  *cand = sg_batch_candidates(j.occ);
  const sg_sched_choice d = sg_batch_default(j.occ);
  X->assign(cand->size() * kSchedFeatures, 0.0f);
  *def = 0;
  for (size_t i = 0; i < cand->size(); ++i) {
    sg_batch_features(j.stats, (*cand)[i], c->num_sms, &(*X)[i * kSchedFeatures]);
    if ((*cand)[i].chunk == d.chunk && (*cand)[i].blocks_per_sm == d.blocks_per_sm) *def = (int)i;
  }
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
  if (ev[0]) cudaEventDestroy(ev[0]);
  if (ev[1]) cudaEventDestroy(ev[1]);
}

extern "C" sg_status sg_batch_run(sg_ctx* c, const sg_chain* ch, const float* data,
                                  const int64_t* offsets, int64_t nseg, double* sums,
                                  int64_t* first_viol, int64_t* kept) {
  Job j;
  sg_status st = prepare(c, ch, data, offsets, nseg, sums, first_viol, kept, &j);
  if (st || nseg == 0) return st;
  std::vector<sg_sched_choice> cand;
  std::vector<float> X;
  int def = 0;
  batch_candidates(c, j, &cand, &X, &def);
  // the autotuned table is kept per workload (offsets, count, lengths) and
  // chain
  uint64_t mb;
  memcpy(&mb, &j.stats.mean_log, 8);
  const uint64_t key =
      sg_sched_key(SG_SCHED_BATCH, {(uint64_t)(uintptr_t)offsets, (uint64_t)nseg,
                                    (uint64_t)j.stats.total, mb, chain_hash(*ch)});
  int learned = -1;
  std::vector<float> pred;
  std::vector<double> times;
  int idx = sg_sched_lookup(c, SG_SCHED_BATCH, key, X, def, &learned, &pred, &times);
  if (idx < 0) {
    st = autotune(c, j, cand, X, def, &times, &idx);
    if (st) return st;
    learned = sg_sched_learned_index(c, SG_SCHED_BATCH, X, def, &pred);
    sg_sched_set_tuned(c, SG_SCHED_BATCH, key, idx, times, learned);
  }
  sg_sched_note(c, SG_SCHED_BATCH, cand, times, def, learned, idx, pred);
  bool viol = false;
  st = run_with(c, j, cand[idx], nullptr, &viol);
  if (st) return st;
  if (viol) {
    c->err = "a collection violated the batch precondition";
    return SG_ERR_PRECONDITION;
  }
  return SG_OK;
}

extern "C" sg_status sg_batch_report(sg_ctx* c, const sg_chain* ch, const float* data,
                                     const int64_t* offsets, int64_t nseg, double* sums,
                                     int64_t* first_viol, int64_t* kept, sg_sched_report* out) {
  if (!out) return bad(c, SG_ERR_INVALID_ARG, "null report");
  Job j;
  sg_status st = prepare(c, ch, data, offsets, nseg, sums, first_viol, kept, &j);
  if (st) return st;
  if (nseg == 0) return bad(c, SG_ERR_INVALID_ARG, "empty batch");
  std::vector<sg_sched_choice> cand;
  std::vector<float> X;
  int def = 0;
  batch_candidates(c, j, &cand, &X, &def);
  std::vector<double> times;
  int best = 0;
  st = autotune(c, j, cand, X, def, &times, &best);
  if (st) return st;
  std::vector<float> pred;
  const int li = sg_sched_learned_index(c, SG_SCHED_BATCH, X, def, &pred);
  sg_sched_note(c, SG_SCHED_BATCH, cand, times, def, li, best, pred);
  *out = c->schedst.last[SG_SCHED_BATCH];
  return SG_OK;
}

extern "C" sg_status sg_sched_train(sg_ctx* c, int32_t epochs, float lr, uint64_t seed,
                                    float* final_loss) {
  if (!c || epochs <= 0 || !(lr > 0.0f)) return bad(c, SG_ERR_INVALID_ARG, "bad training arguments");
  if (c->planning_only) return bad(c, SG_ERR_UNSUPPORTED, "planning-only context");
  return sg_sched_train_impl(c, epochs, lr, seed, final_loss);
}

extern "C" sg_status sg_sched_log_size(sg_ctx* c, int64_t* records, int32_t* features) {
  if (!c || !records || !features) return SG_ERR_INVALID_ARG;
  *records = (int64_t)c->schedst.log_y.size();
  *features = kSchedFeatures;
  return SG_OK;
}

extern "C" sg_status sg_sched_log_read(sg_ctx* c, float* features, float* log_us,
                                       int32_t* family, int64_t records) {
  if (!c || records < 0 || records > (int64_t)c->schedst.log_y.size()) return SG_ERR_INVALID_ARG;
  if (records && (!features || !log_us)) return SG_ERR_INVALID_ARG;
  if (records == 0) return SG_OK;
  memcpy(features, c->schedst.log_x.data(), (size_t)records * kSchedFeatures * 4);
  memcpy(log_us, c->schedst.log_y.data(), (size_t)records * 4);
  if (family)
    for (int64_t r = 0; r < records; ++r) family[r] = (int32_t)c->schedst.log_fam[r];
  return SG_OK;
}

extern "C" sg_status sg_sched_last(sg_ctx* c, int32_t family, sg_sched_report* out) {
  if (!c || !out || family < 0 || family >= kSchedFamilies) return SG_ERR_INVALID_ARG;
  if (!c->schedst.has_last[family]) return bad(c, SG_ERR_INVALID_ARG, "no decision of that family yet");
  *out = c->schedst.last[family];
  return SG_OK;
}

extern "C" sg_status sg_sched_forget(sg_ctx* c, int32_t family) {
  if (!c || family < -1 || family >= kSchedFamilies) return SG_ERR_INVALID_ARG;
  auto& t = c->schedst.tuned;
  t.erase(std::remove_if(t.begin(), t.end(),
                         [&](const SchedState::Tuned& x) { return family < 0 || x.family == family; }),
          t.end());
  return SG_OK;
}

extern "C" sg_status sg_sched_force(sg_ctx* c, int32_t family, int32_t index) {
  if (!c || family < 0 || family >= kSchedFamilies || index < -1 || index >= SG_SCHED_MAX_CANDIDATES)
    return SG_ERR_INVALID_ARG;
  c->schedst.forced[family] = index;
  return SG_OK;
}
