// sg_jit.h -- run-time specialised fused passes (sg_jit.cpp).  Internal.
#pragma once
#include <string>

#include "sg_internal.h"

namespace sgk {

// Kernel argument block of the specialised kernel; its layout is repeated
// verbatim in the kernel template source inside sg_jit.cpp.
struct JitArgs {
  const float* in[kMaxIn];
  float* out[kMaxOut];
  long long n;
  float cst[kMaxProg];
  PassResult* partials;
  unsigned* counter;
  PassResult* result;
  const long long* count;   // StreamArgs::count
  int vec4;
  int pad;
};
static_assert(kMaxIn == 4 && kMaxOut == 4 && kMaxProg == 48 && kMaxPred == 4,
              "the kernel template hard-codes these sizes");
static_assert(sizeof(JitArgs) == 304, "JitArgs layout changed: update the template");

// Kernel argument block of the specialised batch kernel (k_batch.cu holds the
// interpreting twin); repeated verbatim in the template source.
struct BatchJitArgs {
  const float* data;
  const long long* off;
  long long nseg;
  long long chunk;
  float cst[kMaxProg];
  const long long* chunk_start;
  const int* chunk_seg;
  void* partials;
  unsigned* seg_done;
  void* hdr;
  double* sums;
  long long* first_viol;
  long long* kept;
  int vec4;
  int pad;
};
static_assert(sizeof(BatchJitArgs) == 296, "BatchJitArgs layout changed: update the template");

// Kernel argument block of the specialised filter (k_filter.cu holds the
// interpreting twin and the launch); repeated verbatim in the template source.
struct FilterJitArgs {
  const float* x;
  float* out;
  long long n;
  float cst[kMaxProg];
  unsigned long long* st;   // look-back words, one per tile
  unsigned* tile_ctr;       // tile tickets
  FilterResult* res;
  unsigned ntiles;
  int skip_tile;            // look-back testing switch: this tile publishes nothing
  unsigned spin_limit;      // polls before a look-back wait gives up
  int pad;
};
static_assert(sizeof(FilterJitArgs) == 256, "FilterJitArgs layout changed: update the template");
// tile of the specialised filter (items); its shared memory is static
constexpr int kJitFilterTile = 8192;

bool jit_available();
// minmax: the pass also tracks min / max / NaN (a min, max or avg is asked)
cudaKernel_t jit_stream_kernel(const Prog& pr, int nin, int nout, int npred, bool reduce,
                               bool minmax, uint32_t pred_exists, std::string* log);
// the batched map -> for_all -> masked sum chain of one program (k_batch.cu)
cudaKernel_t jit_batch_kernel(const Prog& pr, std::string* log);
// the stable compaction of one predicate (one input slot), one CTA per
// tile of `tile` items: 2048, 4096 or 8192 (k_filter.cu launches it)
// post: a for_all postcondition (one input slot) on the kept items, checked
// as they are written (FilterResult::post_enc), or null
cudaKernel_t jit_filter_kernel(const Prog& pred, std::string* log, int tile = kJitFilterTile,
                               const Prog* post = nullptr);
// index of the postcondition's first constant in FilterJitArgs::cst
inline int jit_filter_post_base(const Prog& pred) { return pred.nops + 1; }
// resident CTAs per SM that filter kernel is compiled for
int filter_tile_occupancy(int tile);
// the smallest tile of the specialised filter (sizes its look-back scratch)
constexpr int kJitFilterMinTile = 2048;
// compiles that kernel's source with NVRTC without loading it (no device
// needed); false with the compiler's log when it does not compile
bool jit_check_filter(const Prog& pred, std::string* log, const Prog* post = nullptr);
cudaError_t launch_jit_stream(cudaKernel_t k, const StreamArgs& s, int grid, int block,
                              cudaStream_t st, Prof* prof);

}  // namespace sgk
