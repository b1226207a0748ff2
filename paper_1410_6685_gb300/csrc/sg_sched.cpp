// sg_sched.cpp -- schedule choice for launch and tile shapes: the plain
// table, the autotuner, and the learned 2x64 MLP cost models, one per
// decision family (sg_sched_family).
//
// A family lists candidate schedules for a workload and describes each
// (workload, candidate) pair by 12 features:
//   batch    [log2 nseg, log2 total, mean / std / min / max of log2(L+1),
//             log2 of the work items, program ops / 48, depth / 8, log2
//             chunk, CTAs per SM / 8, work items per CTA slot (log2)]
//   stream   [log2 n, inputs, outputs, ops / 48, depth / 8, predicates,
//             reduce + min/max, log2 threads per CTA, CTAs per SM / 8,
//             log2 grid, log2 float4s per thread, grid / SMs]
//   filter   [log2 n, ops / 48, log2 tile, log2 tiles, log2 waves of
//             resident CTAs, resident CTAs per SM / 8, tiles / SMs (capped
//             at 64) / 64, the last tile's fill, 0...]
//   product  [log2 M, log2 N, log2 K, fp16, CTAs per tile, log2 tiles,
//             SMs busy / SMs, row and column padding of the tiles, log2
//             flops, tiles per busy SM (log2), 0]
//   fusion   [log2 n, queued calls, the plan's kernels, the unfused plan's
//             extra kernels, reductions, predicates, ops / 48, unfused,
//             log2 of the plan's bytes, its bytes / the fused plan's, log2
//             bytes per kernel, 0]
// The autotuner measures every candidate of a workload (a warm-up run, then
// the better of two timed runs, CUDA events) and keeps the fastest; each
// measurement is logged as (family, features, log microseconds, log of the
// time relative to the plain table's choice on the same workload).  The
// family's MLP, trained on the GPU by the library's own kernels, predicts
// that relative log-time; the learned chooser runs the predicted-fastest
// candidate when it is predicted to beat the plain choice by more than 2%,
// else the plain choice, without measuring.
#include "sg_sched.h"

#include <algorithm>
#include <cmath>
#include <cstring>

#include "sg_batch.h"
#include "sg_mlp.h"

namespace {

const long long kChunks[] = {2048, 4096, 8192, 16384, 32768, 65536};
const int kPerSm[] = {1, 2, 4, 8};   // capped at the kernel's occupancy
const int kStreamThreads[] = {64, 128, 256};
const long long kFilterTiles[] = {2048, 4096, 8192};

uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

float lg2(double x) { return (float)std::log2(std::max(1.0, x)); }

}  // namespace

std::vector<sg_sched_choice> sg_batch_candidates(int occ) {
  std::vector<sg_sched_choice> out;
  occ = std::max(1, occ);
  for (long long ch : kChunks)
    for (int p : kPerSm) {
      const int bps = std::min(p, occ);
      bool dup = false;
      for (auto& c : out) dup |= c.chunk == ch && c.blocks_per_sm == bps;
      if (!dup) out.push_back(sg_sched_choice{ch, bps});
    }
  return out;
}

sg_sched_choice sg_batch_default(int occ) {
  return sg_sched_choice{16384, std::max(1, std::min(occ, 8))};
}

void sg_batch_features(const BatchStats& w, const sg_sched_choice& ch, int num_sms, float* f) {
  const double items = (double)w.nseg + (double)w.total / (double)ch.chunk;
  const double slots = (double)num_sms * ch.blocks_per_sm;
  f[0] = lg2((double)w.nseg);
  f[1] = lg2((double)w.total);
  f[2] = (float)w.mean_log;
  f[3] = (float)w.std_log;
  f[4] = (float)w.min_log;
  f[5] = (float)w.max_log;
  f[6] = lg2(items);
  f[7] = (float)w.ops / 48.0f;
  f[8] = (float)w.depth / 8.0f;
  f[9] = (float)std::log2((double)ch.chunk);
  f[10] = (float)ch.blocks_per_sm / 8.0f;
  f[11] = lg2(items / slots);
}

// ---- stream passes: grid-stride grid of float4 units ----------------------

int sg_stream_grid(long long n, const sg_sched_choice& ch, int num_sms) {
  const long long units = std::max<long long>(1, (n + 3) / 4);
  const long long want = (units + ch.chunk - 1) / ch.chunk;
  return (int)std::max<long long>(1, std::min<long long>(want, (long long)num_sms * ch.blocks_per_sm));
}

std::vector<sg_sched_choice> sg_stream_candidates(long long n, int num_sms) {
  std::vector<sg_sched_choice> out;
  for (int t : kStreamThreads)
    for (int p : kPerSm) {
      const sg_sched_choice c{t, p};
      const int g = sg_stream_grid(n, c, num_sms);
      bool dup = false;
      for (auto& o : out) dup |= o.chunk == t && sg_stream_grid(n, o, num_sms) == g;
      if (!dup) out.push_back(c);
    }
  return out;
}

sg_sched_choice sg_stream_default() { return sg_sched_choice{256, 8}; }

void sg_stream_features(const StreamWork& w, const sg_sched_choice& ch, int num_sms, float* f) {
  const int g = sg_stream_grid(w.n, ch, num_sms);
  const double units = std::max<long long>(1, (w.n + 3) / 4);
  f[0] = lg2((double)w.n);
  f[1] = (float)w.nin;
  f[2] = (float)w.nout;
  f[3] = (float)w.ops / 48.0f;
  f[4] = (float)w.depth / 8.0f;
  f[5] = (float)w.npred;
  f[6] = (w.reduce ? 1.0f : 0.0f) + (w.minmax ? 1.0f : 0.0f);
  f[7] = (float)std::log2((double)ch.chunk);
  f[8] = (float)ch.blocks_per_sm / 8.0f;
  f[9] = lg2((double)g);
  f[10] = lg2(units / ((double)g * ch.chunk));
  f[11] = (float)g / (float)num_sms;
}

// ---- the filter's tile --------------------------------------------------------

std::vector<sg_sched_choice> sg_filter_candidates() {
  std::vector<sg_sched_choice> out;
  for (long long t : kFilterTiles) out.push_back(sg_sched_choice{t, 0});
  return out;
}

sg_sched_choice sg_filter_default() { return sg_sched_choice{8192, 0}; }

void sg_filter_features(const FilterWork& w, const sg_sched_choice& ch, int occ, int num_sms,
                        float* f) {
  const double tiles = (double)((w.n + ch.chunk - 1) / ch.chunk);
  const double slots = (double)num_sms * std::max(1, occ);
  const long long rem = w.n % ch.chunk;
  f[0] = lg2((double)w.n);
  f[1] = (float)w.ops / 48.0f;
  f[2] = (float)std::log2((double)ch.chunk);
  f[3] = lg2(tiles);
  f[4] = lg2(tiles / slots * 2.0);
  f[5] = (float)occ / 8.0f;
  f[6] = (float)std::min(64.0, tiles / num_sms) / 64.0f;
  f[7] = rem == 0 ? 1.0f : (float)rem / (float)ch.chunk;
  for (int k = 8; k < kSchedFeatures; ++k) f[k] = 0.0f;
}

// ---- the product's tile form --------------------------------------------------

std::vector<sg_sched_choice> sg_product_candidates(bool pair_available) {
  std::vector<sg_sched_choice> out;
  if (pair_available) out.push_back(sg_sched_choice{256, 2});
  out.push_back(sg_sched_choice{128, 1});
  return out;
}

sg_sched_choice sg_product_default(bool pair_available) {
  return pair_available ? sg_sched_choice{256, 2} : sg_sched_choice{128, 1};
}

void sg_product_features(const ProductWork& w, const sg_sched_choice& ch, int num_sms, float* f) {
  const long long tm = ch.chunk, tn = 256;
  const long long rt = (w.M + tm - 1) / tm, ct = (w.N + tn - 1) / tn;
  const double tiles = (double)(rt * ct);
  const double units = (double)num_sms / ch.blocks_per_sm;   // tiles in flight
  const double busy = std::min(tiles, units) * ch.blocks_per_sm;
  f[0] = lg2((double)w.M);
  f[1] = lg2((double)w.N);
  f[2] = lg2((double)w.K);
  f[3] = w.fp16 ? 1.0f : 0.0f;
  f[4] = (float)ch.blocks_per_sm;
  f[5] = lg2(tiles);
  f[6] = (float)(busy / num_sms);
  f[7] = 1.0f - (float)w.M / (float)(rt * tm);
  f[8] = 1.0f - (float)w.N / (float)(ct * tn);
  f[9] = lg2(2.0 * w.M * (double)w.N * w.K) / 48.0f;
  f[10] = lg2(tiles / std::max(1.0, std::min(tiles, units)));
  f[11] = 0.0f;
}

// ---- the fusion boundaries ------------------------------------------------------

std::vector<sg_sched_choice> sg_fusion_candidates(const FusionWork& w) {
  return {sg_sched_choice{w.passes[0], 1}, sg_sched_choice{w.passes[1], 0}};
}

void sg_fusion_features(const FusionWork& w, int cand, float* f) {
  f[0] = lg2((double)w.n);
  f[1] = (float)w.nodes;
  f[2] = (float)w.passes[cand];
  f[3] = (float)(w.passes[1] - w.passes[0]);
  f[4] = (float)w.reduces;
  f[5] = (float)w.preds;
  f[6] = (float)w.ops / 48.0f;
  f[7] = (float)cand;
  f[8] = lg2(w.bytes[cand]);
  f[9] = (float)(w.bytes[cand] / std::max(1.0, w.bytes[0]));
  f[10] = lg2(w.bytes[cand] / std::max(1.0, (double)w.passes[cand]));
  f[11] = 0.0f;
}

// ---- the log, the tuned table and the last decisions --------------------------

void sg_sched_log_add(sg_ctx* c, int family, const float* f, double us, float rel) {
  SchedState& s = c->schedst;
  s.log_x.insert(s.log_x.end(), f, f + kSchedFeatures);
  s.log_y.push_back((float)std::log(std::max(us, 1e-3)));
  s.log_rel.push_back(rel);
  s.log_fam.push_back(family);
}

void sg_sched_log_sweep(sg_ctx* c, int family, const std::vector<float>& X,
                        const std::vector<double>& us, int def) {
  const double tdef = def >= 0 && def < (int)us.size() ? us[def] : 0.0;
  for (size_t i = 0; i < us.size(); ++i) {
    const float rel = tdef > 0.0 ? (float)std::log(us[i] / tdef) : NAN;
    sg_sched_log_add(c, family, &X[i * kSchedFeatures], us[i], rel);
  }
}

uint64_t sg_sched_key(int family, std::initializer_list<uint64_t> parts) {
  uint64_t h = mix64(0x5C4EDull + (uint64_t)family);
  for (uint64_t p : parts) h = mix64(h ^ (p + 0x9E3779B97F4A7C15ull));
  return h;
}

int sg_sched_tuned(const sg_ctx* c, uint64_t key, std::vector<double>* us, int* learned) {
  for (auto& t : c->schedst.tuned)
    if (t.key == key) {
      if (us) *us = t.us;
      if (learned) *learned = t.learned;
      return t.idx;
    }
  return -1;
}

void sg_sched_set_tuned(sg_ctx* c, int family, uint64_t key, int idx,
                        const std::vector<double>& us, int learned) {
  for (auto& t : c->schedst.tuned)
    if (t.key == key) {
      t.idx = idx;
      t.us = us;
      t.learned = learned;
      return;
    }
  c->schedst.tuned.push_back({key, idx, family, us, learned});
}

void sg_sched_note(sg_ctx* c, int family, const std::vector<sg_sched_choice>& cand,
                   const std::vector<double>& us, int def, int learned, int chosen,
                   const std::vector<float>& pred) {
  if (family < 0 || family >= kSchedFamilies) return;
  sg_sched_report& r = c->schedst.last[family];
  memset(&r, 0, sizeof r);
  r.family = family;
  r.ncand = (int32_t)std::min<size_t>(cand.size(), SG_SCHED_MAX_CANDIDATES);
  r.default_index = def;
  r.learned_index = learned;
  r.chosen_index = chosen;
  r.best_index = -1;
  double bt = 1e300;
  for (int i = 0; i < r.ncand; ++i) {
    r.chunk[i] = cand[i].chunk;
    r.ctas_per_sm[i] = cand[i].blocks_per_sm;
    if ((size_t)i < us.size()) {
      r.measured_us[i] = us[i];
      if (us[i] < bt) {
        bt = us[i];
        r.best_index = i;
      }
    }
  }
  // the model predicts times relative to the plain choice: scale by its
  // measured time
  const double tdef = def >= 0 && (size_t)def < us.size() ? us[def] : 0.0;
  if (!pred.empty())
    for (int i = 0; i < r.ncand && (size_t)i < pred.size(); ++i)
      r.predicted_us[i] = std::exp((double)pred[i]) * tdef;
  c->schedst.has_last[family] = true;
}

int sg_sched_lookup(sg_ctx* c, int family, uint64_t key, const std::vector<float>& X, int def,
                    int* learned, std::vector<float>* pred, std::vector<double>* us) {
  *learned = -1;
  const int f = c->schedst.forced[family];
  if (f >= 0 && f < (int)(X.size() / kSchedFeatures)) return f;
  if (c->sched == SG_SCHED_LEARNED && c->schedst.model[family].trained) {
    // one prediction per workload while the model stands
    for (auto& t : c->schedst.learned_memo)
      if (t.first == key) return *learned = t.second;
    *learned = sg_sched_learned_index(c, family, X, def, pred);
    if (*learned >= 0) {
      c->schedst.learned_memo.push_back({key, *learned});
      return *learned;
    }
  }
  return sg_sched_tuned(c, key, us, learned);
}

// ---------------------------------------------------------------------------
// training on the GPU with the library's kernels

SchedModel::~SchedModel() {
  if (dev) cudaFree(dev);
}

static void init_params(std::vector<float>& P, int d_in, uint64_t seed) {
  const int H = sgk::kMlpHidden;
  P.assign(sgk::mlp_nparams(d_in), 0.0f);
  uint64_t t = seed;
  auto normal = [&]() {
    // Box-Muller from two SplitMix64 draws
    const double u1 = ((mix64(t += 0x9E3779B97F4A7C15ull) >> 11) + 1.0) / 9007199254740993.0;
    const double u2 = (mix64(t += 0x9E3779B97F4A7C15ull) >> 11) / 9007199254740992.0;
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
  };
  float* W1 = P.data();
  float* W2 = W1 + H * d_in + H;
  float* W3 = W2 + H * H + H;
  for (int i = 0; i < H * d_in; ++i) W1[i] = (float)(normal() * std::sqrt(2.0 / d_in));
  for (int i = 0; i < H * H; ++i) W2[i] = (float)(normal() * std::sqrt(2.0 / H));
  for (int i = 0; i < H; ++i) W3[i] = (float)(normal() * std::sqrt(1.0 / H));
}

namespace {

// Fits one family's model to its sweep records; *sq: summed squared error
// on the standardised targets, *count: the records.  SG_ERR_INVALID_ARG
// when the family has fewer than 8.
sg_status train_family(sg_ctx* c, int fam, int epochs, float lr, uint64_t seed, double* sq,
                       long long* count) {
  SchedState& s = c->schedst;
  SchedModel& md = s.model[fam];
  const int d = kSchedFeatures;
  std::vector<long long> rows;
  for (long long r = 0; r < (long long)s.log_rel.size(); ++r)
    if (s.log_fam[r] == fam && std::isfinite(s.log_rel[r])) rows.push_back(r);
  const long long R = (long long)rows.size();
  if (R < 8) return SG_ERR_INVALID_ARG;
  // feature / target normalisation from those records
  md.mu.assign(d, 0.0f);
  md.sd.assign(d, 0.0f);
  double ym = 0.0, ys = 0.0;
  for (long long r : rows) {
    for (int k = 0; k < d; ++k) md.mu[k] += s.log_x[r * d + k];
    ym += s.log_rel[r];
  }
  for (int k = 0; k < d; ++k) md.mu[k] /= (float)R;
  ym /= (double)R;
  for (long long r : rows) {
    for (int k = 0; k < d; ++k) {
      const float q = s.log_x[r * d + k] - md.mu[k];
      md.sd[k] += q * q;
    }
    ys += (s.log_rel[r] - ym) * (s.log_rel[r] - ym);
  }
  for (int k = 0; k < d; ++k) md.sd[k] = std::sqrt(md.sd[k] / (float)R) + 1e-6f;
  md.ymu = (float)ym;
  md.ysd = (float)std::sqrt(ys / (double)R) + 1e-6f;
  std::vector<float> X((size_t)R * d), Y(R);
  for (long long i = 0; i < R; ++i) {
    const long long r = rows[i];
    for (int k = 0; k < d; ++k) X[i * d + k] = (s.log_x[r * d + k] - md.mu[k]) / md.sd[k];
    Y[i] = (s.log_rel[r] - md.ymu) / md.ysd;
  }
  // device buffers: params, grad, m, v, X, Y, loss, predictions, work
  const int np = sgk::mlp_nparams(d);
  const int B = (int)std::min<long long>(R, 512);
  const size_t bytes = (size_t)np * 16 + (size_t)R * (d + 1) * 4 + sgk::mlp_work_bytes(B) +
                       (size_t)kSchedMaxCand * (d + 1) * 4 + 2048;
  md.trained = false;
  if (md.dev) cudaFree(md.dev);
  md.dev = nullptr;
  if (cudaMalloc(&md.dev, bytes) != cudaSuccess) {
    cudaGetLastError();
    c->err = "model allocation failed";
    return SG_ERR_OOM;
  }
  float* P = static_cast<float*>(md.dev);
  float* G = P + np;
  float* m = G + np;
  float* v = m + np;
  float* dX = v + np;
  float* dY = dX + (size_t)R * d;
  float* loss = dY + R;
  float* pred = loss + 64;
  void* work = pred + (size_t)kSchedMaxCand * (d + 1);
  std::vector<float> P0;
  init_params(P0, d, seed + (uint64_t)fam * 0x1000193ull);
  cudaStream_t st = c->stream;
  cudaError_t e = cudaMemcpyAsync(P, P0.data(), np * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m, 0, (size_t)np * 8, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dX, X.data(), X.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dY, Y.data(), Y.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  // mini-batches over a shuffled order (shuffled on the host, rows copied
  // once per epoch)
  std::vector<long long> order(R);
  for (long long r = 0; r < R; ++r) order[r] = r;
  std::vector<float> Xe((size_t)R * d), Ye(R);
  long long t = 0;
  uint64_t rs = seed ^ 0x5151ull ^ ((uint64_t)fam << 40);
  for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
    for (long long r = R - 1; r > 0; --r) {
      const long long j = (long long)(mix64(rs += 0x9E3779B97F4A7C15ull) % (uint64_t)(r + 1));
      std::swap(order[r], order[j]);
    }
    for (long long r = 0; r < R; ++r) {
      memcpy(&Xe[r * d], &X[order[r] * d], d * 4);
      Ye[r] = Y[order[r]];
    }
    e = cudaMemcpyAsync(dX, Xe.data(), Xe.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dY, Ye.data(), Ye.size() * 4, cudaMemcpyHostToDevice, st);
    for (long long b0 = 0; b0 < R && e == cudaSuccess; b0 += B) {
      const int bb = (int)std::min<long long>(B, R - b0);
      e = sgk::launch_mlp_loss_grad(P, d, dX + b0 * d, dY + b0, bb, G, nullptr, work, st);
      if (e == cudaSuccess)
        e = sgk::launch_mlp_adam(P, G, m, v, np, ++t, lr, 0.9f, 0.999f, 1e-8f, st);
      c->kernels += 4;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  // final loss over the family's records (original order)
  if (e == cudaSuccess) e = cudaMemcpyAsync(dX, X.data(), X.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dY, Y.data(), Y.size() * 4, cudaMemcpyHostToDevice, st);
  float hl = 0.0f;
  double tot = 0.0;
  for (long long b0 = 0; b0 < R && e == cudaSuccess; b0 += B) {
    const int bb = (int)std::min<long long>(B, R - b0);
    e = sgk::launch_mlp_loss_grad(P, d, dX + b0 * d, dY + b0, bb, G, loss, work, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hl, loss, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    tot += (double)hl * bb;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->err = cudaGetErrorString(e);
    return SG_ERR_CUDA;
  }
  md.trained = true;
  md.params = P;
  md.pred = pred;
  *sq += tot;
  *count += R;
  return SG_OK;
}

}  // namespace

sg_status sg_sched_train_impl(sg_ctx* c, int epochs, float lr, uint64_t seed, float* final_loss) {
  double sq = 0.0;
  long long count = 0;
  int trained = 0;
  c->schedst.learned_memo.clear();
  for (int f = 0; f < kSchedFamilies; ++f) {
    const sg_status st = train_family(c, f, epochs, lr, seed, &sq, &count);
    if (st == SG_OK) ++trained;
    else if (st != SG_ERR_INVALID_ARG) return st;
  }
  if (!trained) {
    c->err = "the schedule log needs at least 8 records from candidate sweeps of one family";
    return SG_ERR_INVALID_ARG;
  }
  if (final_loss) *final_loss = (float)(sq / (double)count);
  return SG_OK;
}

// predicted log-time of each candidate (the family's model), on the GPU
bool sg_sched_predict(sg_ctx* c, int family, const std::vector<float>& Xraw,
                      std::vector<float>* pred) {
  if (family < 0 || family >= kSchedFamilies) return false;
  SchedModel& md = c->schedst.model[family];
  if (!md.trained) return false;
  const int d = kSchedFeatures;
  const int n = (int)(Xraw.size() / d);
  if (n <= 0 || n > kSchedMaxCand) return false;
  std::vector<float> X((size_t)n * d);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < d; ++k) X[(size_t)i * d + k] = (Xraw[(size_t)i * d + k] - md.mu[k]) / md.sd[k];
  float* dX = md.pred;
  float* dY = dX + (size_t)n * d;
  pred->assign(n, 0.0f);
  cudaError_t e = cudaMemcpyAsync(dX, X.data(), X.size() * 4, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = sgk::launch_mlp_forward(md.params, d, dX, n, dY, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(pred->data(), dY, n * 4, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  c->kernels += 1;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  for (float& p : *pred) p = p * md.ysd + md.ymu;
  return true;
}

int sg_sched_learned_index(sg_ctx* c, int family, const std::vector<float>& X, int def,
                           std::vector<float>* pred) {
  std::vector<float> local;
  std::vector<float>& p = pred ? *pred : local;
  if (!sg_sched_predict(c, family, X, &p)) return -1;
  const int bi = (int)(std::min_element(p.begin(), p.end()) - p.begin());
  // a predicted gain against the plain choice, beyond the model's noise
  return p[bi] < p[def] - kLearnedMargin ? bi : def;
}
