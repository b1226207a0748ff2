// sg_sched.cpp -- schedule choice for the batched-collections launch: the
// plain table, the autotuner, and the learned 2x64 MLP cost model.
//
// A schedule is (chunk: elements per work item, CTAs per SM).  For a
// workload (the collection lengths, the chain) and a candidate schedule the
// features are
//   [log2 nseg, log2 total, mean / std / min / max of log2(L+1), log2 of the
//    work items, program ops / 48, depth / 8, log2 chunk, CTAs per SM / 8,
//    work items per CTA slot (log2)]                              (d_in = 12)
// The autotuner measures every candidate of a workload (a warm-up run, then
// the better of two timed runs, CUDA events) and keeps the fastest; each
// measurement is logged as (features, log microseconds, log of the time
// relative to the plain table's choice on the same workload).  The MLP,
// trained on the GPU by the library's own kernels, predicts that relative
// log-time; the learned chooser runs the predicted-fastest candidate when it
// is predicted to beat the plain choice by more than 2%, else the plain
// choice, without measuring.
#include "sg_sched.h"

#include <algorithm>
#include <cmath>
#include <cstring>

#include "sg_batch.h"
#include "sg_mlp.h"

namespace {

const long long kChunks[] = {2048, 4096, 8192, 16384, 32768, 65536};
const int kPerSm[] = {1, 2, 4, 8};   // capped at the kernel's occupancy

uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

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
  f[0] = (float)std::log2(std::max<double>(1, w.nseg));
  f[1] = (float)std::log2(std::max<double>(1, w.total));
  f[2] = (float)w.mean_log;
  f[3] = (float)w.std_log;
  f[4] = (float)w.min_log;
  f[5] = (float)w.max_log;
  f[6] = (float)std::log2(std::max(1.0, items));
  f[7] = (float)w.ops / 48.0f;
  f[8] = (float)w.depth / 8.0f;
  f[9] = (float)std::log2((double)ch.chunk);
  f[10] = (float)ch.blocks_per_sm / 8.0f;
  f[11] = (float)std::log2(std::max(1.0, items / slots));
}

void sg_sched_log_add(sg_ctx* c, const float* f, double us, float rel) {
  SchedState& s = c->schedst;
  s.log_x.insert(s.log_x.end(), f, f + kSchedFeatures);
  s.log_y.push_back((float)std::log(std::max(us, 1e-3)));
  s.log_rel.push_back(rel);
}

// ---------------------------------------------------------------------------
// training on the GPU with the library's kernels

SchedState::~SchedState() {
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

sg_status sg_sched_train_impl(sg_ctx* c, int epochs, float lr, uint64_t seed, float* final_loss) {
  SchedState& s = c->schedst;
  const int d = kSchedFeatures;
  // the sweep records: features and time relative to the plain choice
  std::vector<long long> rows;
  for (long long r = 0; r < (long long)s.log_rel.size(); ++r)
    if (std::isfinite(s.log_rel[r])) rows.push_back(r);
  const long long R = (long long)rows.size();
  if (R < 8) {
    c->err = "the schedule log needs at least 8 records from candidate sweeps";
    return SG_ERR_INVALID_ARG;
  }
  // feature / target normalisation from those records
  s.mu.assign(d, 0.0f);
  s.sd.assign(d, 0.0f);
  double ym = 0.0, ys = 0.0;
  for (long long r : rows) {
    for (int k = 0; k < d; ++k) s.mu[k] += s.log_x[r * d + k];
    ym += s.log_rel[r];
  }
  for (int k = 0; k < d; ++k) s.mu[k] /= (float)R;
  ym /= (double)R;
  for (long long r : rows) {
    for (int k = 0; k < d; ++k) {
      const float q = s.log_x[r * d + k] - s.mu[k];
      s.sd[k] += q * q;
    }
    ys += (s.log_rel[r] - ym) * (s.log_rel[r] - ym);
  }
  for (int k = 0; k < d; ++k) s.sd[k] = std::sqrt(s.sd[k] / (float)R) + 1e-6f;
  s.ymu = (float)ym;
  s.ysd = (float)std::sqrt(ys / (double)R) + 1e-6f;
  std::vector<float> X((size_t)R * d), Y(R);
  for (long long i = 0; i < R; ++i) {
    const long long r = rows[i];
    for (int k = 0; k < d; ++k) X[i * d + k] = (s.log_x[r * d + k] - s.mu[k]) / s.sd[k];
    Y[i] = (s.log_rel[r] - s.ymu) / s.ysd;
  }
  // device buffers: params, grad, m, v, X, Y, work, loss
  const int np = sgk::mlp_nparams(d);
  const int B = (int)std::min<long long>(R, 512);
  const size_t bytes = (size_t)np * 16 + (size_t)R * (d + 1) * 4 + sgk::mlp_work_bytes(B) +
                       (size_t)kSchedMaxCand * (d + 1) * 4 + 2048;
  if (s.dev) cudaFree(s.dev);
  s.dev = nullptr;
  if (cudaMalloc(&s.dev, bytes) != cudaSuccess) {
    cudaGetLastError();
    c->err = "model allocation failed";
    return SG_ERR_OOM;
  }
  float* P = static_cast<float*>(s.dev);
  float* G = P + np;
  float* m = G + np;
  float* v = m + np;
  float* dX = v + np;
  float* dY = dX + (size_t)R * d;
  float* loss = dY + R;
  float* pred = loss + 64;
  void* work = pred + (size_t)kSchedMaxCand * (d + 1);
  std::vector<float> P0;
  init_params(P0, d, seed);
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
  uint64_t rs = seed ^ 0x5151ull;
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
  // final loss over the whole log (original order)
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
  s.trained = true;
  s.params = P;
  s.pred = pred;
  if (final_loss) *final_loss = (float)(tot / (double)R);
  return SG_OK;
}

// predicted log-time of each candidate (learned model), on the GPU
bool sg_sched_predict(sg_ctx* c, const BatchStats& w, const std::vector<sg_sched_choice>& cand,
                      std::vector<float>* pred) {
  SchedState& s = c->schedst;
  if (!s.trained) return false;
  const int d = kSchedFeatures;
  const int n = (int)cand.size();
  std::vector<float> X((size_t)n * d);
  for (int i = 0; i < n; ++i) {
    float f[kSchedFeatures];
    sg_batch_features(w, cand[i], c->num_sms, f);
    for (int k = 0; k < d; ++k) X[(size_t)i * d + k] = (f[k] - s.mu[k]) / s.sd[k];
  }
  if (n > kSchedMaxCand) return false;
  float* dX = s.pred;
  float* dY = dX + (size_t)n * d;
  pred->assign(n, 0.0f);
  cudaError_t e = cudaMemcpyAsync(dX, X.data(), X.size() * 4, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = sgk::launch_mlp_forward(s.params, d, dX, n, dY, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(pred->data(), dY, n * 4, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  c->kernels += 1;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  for (float& p : *pred) p = p * s.ysd + s.ymu;
  return true;
}

int sg_sched_learned_index(sg_ctx* c, const BatchStats& w, const std::vector<sg_sched_choice>& cand,
                           const sg_sched_choice& def, std::vector<float>* pred) {
  std::vector<float> local;
  std::vector<float>& p = pred ? *pred : local;
  if (!sg_sched_predict(c, w, cand, &p)) return -1;
  int di = 0;
  for (size_t i = 0; i < cand.size(); ++i)
    if (cand[i].chunk == def.chunk && cand[i].blocks_per_sm == def.blocks_per_sm) di = (int)i;
  const int bi = (int)(std::min_element(p.begin(), p.end()) - p.begin());
  // a predicted gain against the plain choice, beyond the model's noise
  return p[bi] < p[di] - kLearnedMargin ? bi : di;
}
