// sg_sched.h -- schedule choice for launch shapes: the plain table, the
// autotuner and the learned cost model (sg_set_scheduler).  Internal.
#pragma once
#include <cstdint>
#include <vector>

#include "sg_runtime.h"

struct sg_sched_choice {
  long long chunk;      // batched collections: elements per work item
  int blocks_per_sm;    // persistent CTAs per SM
};

// Length statistics of a batched workload (from its offsets) and program size
struct BatchStats {
  long long nseg = 0, total = 0;
  double mean_log = 0, std_log = 0, min_log = 0, max_log = 0;
  int ops = 0, depth = 0;
};

// occ: resident CTAs per SM of the batch kernel that will run
std::vector<sg_sched_choice> sg_batch_candidates(int occ);
sg_sched_choice sg_batch_default(int occ);
void sg_batch_features(const BatchStats& w, const sg_sched_choice& ch, int num_sms, float* f);
// One timing record: features, microseconds, and log(us / us of the plain
// table's choice on the same workload) when the record comes from a sweep
// of every candidate (NaN otherwise).
void sg_sched_log_add(sg_ctx* c, const float* f, double us, float rel);
sg_status sg_sched_train_impl(sg_ctx* c, int epochs, float lr, uint64_t seed, float* final_loss);
// Predicted log(time / time of the plain table's choice) of each candidate.
bool sg_sched_predict(sg_ctx* c, const BatchStats& w, const std::vector<sg_sched_choice>& cand,
                      std::vector<float>* pred);
// The learned choice: the predicted-fastest candidate when it is predicted
// to beat the plain table's choice by more than kLearnedMargin, else that
// choice.  -1 when no model is trained.
constexpr float kLearnedMargin = 0.02f;
int sg_sched_learned_index(sg_ctx* c, const BatchStats& w, const std::vector<sg_sched_choice>& cand,
                           const sg_sched_choice& def, std::vector<float>* pred);
