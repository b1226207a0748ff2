// sg_sched.h -- schedule choice for launch shapes: the autotuned plain table
// or the learned cost model (sg_set_scheduler).  Internal.
#pragma once
#include <cstdint>

#include "sg_runtime.h"

struct sg_sched_choice {
  long long chunk;      // batched collections: elements per work item
  int blocks_per_sm;    // persistent CTAs per SM
};

sg_sched_choice sg_choose_batch_schedule(sg_ctx* c, int64_t nseg, int depth);
void sg_record_batch_timing(sg_ctx* c, int64_t nseg, const sg_sched_choice& ch);
