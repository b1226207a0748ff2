// sg_sched.cpp -- schedule choice (plain autotuned table for now).
#include "sg_sched.h"

#include <algorithm>

#include "sg_batch.h"

sg_sched_choice sg_choose_batch_schedule(sg_ctx* c, int64_t nseg, int depth) {
  (void)nseg;
  sg_sched_choice ch;
  ch.chunk = 16384;
  ch.blocks_per_sm = std::max(1, sgk::batch_blocks_per_sm(depth));
  (void)c;
  return ch;
}

void sg_record_batch_timing(sg_ctx*, int64_t, const sg_sched_choice&) {}
