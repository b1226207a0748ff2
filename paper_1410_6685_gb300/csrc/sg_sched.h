// sg_sched.h -- schedule choice for launch and tile shapes: the plain
// table, the autotuner and the learned cost models (sg_set_scheduler), per
// decision family (sg_sched_family).  Internal.
#pragma once
#include <cstdint>
#include <initializer_list>
#include <vector>

#include "sg_runtime.h"

struct sg_sched_choice {
  long long chunk;      // batch: elements per work item; stream: threads per
                        // CTA; filter: tile items; product: tile rows
  int blocks_per_sm;    // batch, stream: CTAs per SM; product: CTAs per tile
};

// Length statistics of a batched workload (from its offsets) and program size
struct BatchStats {
  long long nseg = 0, total = 0;
  double mean_log = 0, std_log = 0, min_log = 0, max_log = 0;
  int ops = 0, depth = 0;
};

// A fused element-wise pass: its length and program shape
struct StreamWork {
  long long n = 0;
  int nin = 0, nout = 0, ops = 0, depth = 0, npred = 0;
  bool reduce = false, minmax = false, vec4 = true;
};

// The specialised filter: length and predicate size
struct FilterWork {
  long long n = 0;
  int ops = 0;
};

// The tensor-core product C (M x N) = A (M x K) B (K x N)
struct ProductWork {
  int M = 0, N = 0, K = 0;
  bool fp16 = false;
};

// A flush of element-wise passes, under its fused and its unfused plan
struct FusionWork {
  long long n = 0;           // the longest pass
  int nodes = 0, reduces = 0, preds = 0, ops = 0;
  int passes[2] = {0, 0};    // kernels of the fused / unfused plan
  double bytes[2] = {0, 0};  // bytes those kernels read and write
};

// occ: resident CTAs per SM of the batch kernel that will run
std::vector<sg_sched_choice> sg_batch_candidates(int occ);
sg_sched_choice sg_batch_default(int occ);
void sg_batch_features(const BatchStats& w, const sg_sched_choice& ch, int num_sms, float* f);

// Stream passes: (threads per CTA, CTAs per SM); candidates whose grids
// coincide for this length are listed once
std::vector<sg_sched_choice> sg_stream_candidates(long long n, int num_sms);
sg_sched_choice sg_stream_default();
int sg_stream_grid(long long n, const sg_sched_choice& ch, int num_sms);
void sg_stream_features(const StreamWork& w, const sg_sched_choice& ch, int num_sms, float* f);

// The filter: tile items; occ = resident CTAs per SM of that tile's kernel
std::vector<sg_sched_choice> sg_filter_candidates();
sg_sched_choice sg_filter_default();
void sg_filter_features(const FilterWork& w, const sg_sched_choice& ch, int occ, int num_sms,
                        float* f);

// The product: (256, 2) CTA-pair tiles and (128, 1) one-CTA tiles
std::vector<sg_sched_choice> sg_product_candidates(bool pair_available);
sg_sched_choice sg_product_default(bool pair_available);
void sg_product_features(const ProductWork& w, const sg_sched_choice& ch, int num_sms, float* f);

// The fusion boundaries: candidate 0 the fused plan (kernels, 1), candidate
// 1 one kernel per queued call (kernels, 0)
std::vector<sg_sched_choice> sg_fusion_candidates(const FusionWork& w);
void sg_fusion_features(const FusionWork& w, int cand, float* f);
// the autotuner takes the unfused plan only when it measured this much faster
constexpr double kFusionMargin = 0.97;

// One timing record: family, features, microseconds, and log(us / us of the
// plain table's choice on the same workload) when the record comes from a
// sweep of every candidate (NaN otherwise).
void sg_sched_log_add(sg_ctx* c, int family, const float* f, double us, float rel);
// Logs a sweep: every candidate's features (n x kSchedFeatures) and time,
// relative to the plain choice `def`.
void sg_sched_log_sweep(sg_ctx* c, int family, const std::vector<float>& X,
                        const std::vector<double>& us, int def);
sg_status sg_sched_train_impl(sg_ctx* c, int epochs, float lr, uint64_t seed, float* final_loss);
// Predicted log(time / time of the plain table's choice) of each candidate
// (rows of X, n x kSchedFeatures).  false when the family has no model.
bool sg_sched_predict(sg_ctx* c, int family, const std::vector<float>& X,
                      std::vector<float>* pred);
// The learned choice: the predicted-fastest candidate when it is predicted
// to beat the plain table's choice `def` by more than kLearnedMargin, else
// `def`.  -1 when the family has no trained model.
constexpr float kLearnedMargin = 0.02f;
int sg_sched_learned_index(sg_ctx* c, int family, const std::vector<float>& X, int def,
                           std::vector<float>* pred);

// A workload's autotuned choice: the candidate index (and, when us is not
// null, the times its sweep measured), or -1 when none yet
int sg_sched_tuned(const sg_ctx* c, uint64_t key, std::vector<double>* us = nullptr,
                   int* learned = nullptr);
// learned: the model's choice for the workload when it was swept (-1: none)
void sg_sched_set_tuned(sg_ctx* c, int family, uint64_t key, int idx,
                        const std::vector<double>& us = {}, int learned = -1);
uint64_t sg_sched_key(int family, std::initializer_list<uint64_t> parts);

// Records a decision for sg_sched_last: the candidates, the measured times
// (empty when nothing was measured), the plain, learned and chosen indices
// and the predictions (empty without a model).
void sg_sched_note(sg_ctx* c, int family, const std::vector<sg_sched_choice>& cand,
                   const std::vector<double>& us, int def, int learned, int chosen,
                   const std::vector<float>& pred);

// The decision of one family for one workload: a forced index
// (sg_sched_force) when it names a candidate; under SG_SCHED_LEARNED with
// a trained model the learned index; otherwise the autotuned index when
// `key` was swept before, else -1 (the caller sweeps when it can, or takes
// `def`).  *pred receives the model's predictions when there is a model,
// *us and *learned an autotuned choice's measured times and the model's
// choice when it was measured.
int sg_sched_lookup(sg_ctx* c, int family, uint64_t key, const std::vector<float>& X, int def,
                    int* learned, std::vector<float>* pred, std::vector<double>* us);
