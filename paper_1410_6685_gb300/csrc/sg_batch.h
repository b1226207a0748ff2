// sg_batch.h -- the batched-collections kernels (k_batch.cu) and their host
// driver (sg_batch.cpp).  Internal.
#pragma once
#include "sg_internal.h"

namespace sgk {

struct BatchLaunch {
  const float* data;
  const long long* offsets;
  long long nseg;
  long long chunk;          // elements per work item
  long long capacity;       // chunk partials the scratch holds
  int grid;                 // persistent CTAs
  Prog prog;
  int depth;
  void* scratch;
  double* sums;
  long long* first_viol;
  long long* kept;
  unsigned* host_flag;      // pinned: bit 0 violation, bit 1 capacity overflow
  cudaKernel_t jit;         // run-time specialised kernel, or nullptr (interpreter)
};

// with_pre: the precondition is evaluated (contract mode PRE or above)
bool build_chain_prog(const sg_chain& ch, Prog* pr, int* depth, bool with_pre = true);
size_t batch_scratch_bytes(long long nseg, long long capacity);
cudaError_t launch_batch(const BatchLaunch& L, cudaStream_t s, Prof* prof);
int batch_blocks_per_sm(int depth);

}  // namespace sgk
