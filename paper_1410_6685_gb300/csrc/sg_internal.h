// sg_internal.h -- declarations shared by the host runtime (sg_api.cpp) and
// the sm_103a kernels (k_*.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "safegpu.h"

namespace sgk {

// Per-kernel CUDA-event tracing of one context (off unless enabled).
struct Prof {
  int on = 0;
  struct Rec {
    const char* name;
    cudaEvent_t a, b;
  };
  std::vector<Rec> open;                                  // this flush
  std::vector<cudaEvent_t> pool;
  std::map<std::string, std::pair<long long, double>> agg;  // launches, ms
  cudaEvent_t take();
  void begin(const char* name, cudaStream_t s);
  void end(cudaStream_t s);
  void collect();   // after the stream is synchronised
  ~Prof();
};
inline void prof_begin(Prof* p, const char* name, cudaStream_t s) {
  if (p && p->on) p->begin(name, s);
}
inline void prof_end(Prof* p, cudaStream_t s) {
  if (p && p->on) p->end(s);
}

// ---------------------------------------------------------------------------
// Fused element-wise program (the optimizer's output for one pass, Sec. 5).
// Ops are the public SG_OP_* arithmetic ops plus sinks.  For every op the host
// stores the stack depth *before* it executes, so the kernel addresses stack
// slots by compile-time index (slot 0 = bottom).
constexpr int kMaxProg = 48;
constexpr int kMaxDepth = 8;
constexpr int kMaxIn = 4;
constexpr int kMaxOut = 4;
constexpr int kMaxPred = 4;

enum : uint8_t {
  K_STORE = 64,   // out[arg][i] = top (no pop)
  K_PRED = 65,    // pop; record i in first[arg] when the predicate fails (for_all)
                  // or holds (exists, bit arg of pred_exists)
  K_MASK = 66,    // pop; the next K_REDUCE only takes elements where it is true
  K_REDUCE = 67,  // pop value; accumulate sum/count/min/max over the mask
  K_POP = 68      // pop and discard
};

struct Prog {
  int32_t nops;
  uint8_t op[kMaxProg];
  uint8_t depth[kMaxProg];
  int8_t arg[kMaxProg];
  float cst[kMaxProg];
};

// Result of one pass: the reduction and the first violating index of each
// predicate (INT64_MAX = none).  64 bytes.
struct PassResult {
  double sum;
  long long count;
  float mn, mx;
  int nan_seen;
  int pad;
  long long first[kMaxPred];
};

struct StreamArgs {
  const float* in[kMaxIn];
  float* out[kMaxOut];
  long long n;
  Prog prog;
  int nin;               // number of input slots used (0..4)
  int depth;             // largest stack depth the program reaches (<= 8)
  int has_reduce;
  int npred;
  uint32_t pred_exists;  // bit p set: predicate p is an `exists`
  PassResult* partials;  // one per block (scratch)
  unsigned int* counter; // last-block-done counter; zero before and after
  PassResult* result;    // final record (scratch or caller memory)
  int vec4;              // every pointer 16-byte aligned: use 128-bit accesses
  // when set, the pass covers min(n, *count) elements: a compacted filter's
  // count, which the filter kernel earlier in the stream wrote on the device
  const long long* count;
};

// Stack check of a postfix expression over `nin` input slots (the one
// validator of every entry point that takes an sg_expr).  SG_OK with the
// largest stack depth in *max_depth and, when `depth_before` is given, the
// depth before each op; else SG_ERR_INVALID_ARG with a message in msg.
sg_status validate_expr(const sg_expr* f, int nin, int* max_depth, uint8_t* depth_before,
                        char* msg, size_t cap);

cudaError_t launch_stream(const StreamArgs& a, int grid, int block,
                          cudaStream_t s, Prof* prof);
int stream_max_blocks_per_sm(int nin, int depth, int block);

// Every result record the executor copies back fits in this many bytes.
constexpr int kResultBytes = 128;

// ---------------------------------------------------------------------------
// Sort (k_sort.cu): LSD radix sort of signed int32 keys, 8-bit digits, one
// histogram pass and four onesweep passes.  With `contracts`, the last pass
// also checks sortedness and the multiset fingerprint of its output.
struct SortResult {
  unsigned long long unsorted_enc;     // ~i of the smallest i with out[i] >
                                       // out[i+1]; 0 when sorted (max-combined)
  unsigned long long fp_in[2];         // sum mix(k), sum mix(k)^2  (mod 2^64)
  unsigned long long fp_out[2];
  long long cnt_in, cnt_out;
  int timeout;                         // a look-back wait gave up
  int checked;                         // contracts were evaluated
};
static_assert(sizeof(SortResult) <= kResultBytes, "result too large");

// Bounds of the decoupled look-back waits (sort passes, filter).  The
// default (spin_limit 0, skip_tile -1) is the kernels' own limit and every
// tile publishing; the testing switch sg_debug_lookback sets a short limit
// and a tile that publishes nothing, so that its successors' waits run out.
struct LookbackCtl {
  unsigned spin_limit;   // polls before a wait gives up (0 = the kernel's default)
  int skip_tile;         // this tile publishes no look-back word (-1 = none)
};

// bytes from src to dst (no overlap), on stream s
cudaError_t launch_copy(void* dst, const void* src, size_t bytes, int num_sms, cudaStream_t s);

size_t sort_scratch_bytes(long long n);
// Host-side fault planted before the last pass (contract tests only).
struct SortInject {
  int mode;         // 0 none, 1 swap i and j, 2 overwrite i with value j
  long long i, j;
};
// in -> out (distinct buffers).  Scratch must hold sort_scratch_bytes(n).
// flt: the 32-bit keys are binary32 patterns sorted in IEEE totalOrder
// (else signed int32 order).
cudaError_t launch_sort(const int32_t* in, int32_t* out, long long n,
                        bool contracts, void* scratch, SortResult* res,
                        cudaStream_t s, int num_sms, int64_t* kernels,
                        const SortInject* inject, Prof* prof, bool flt,
                        const LookbackCtl& lb);
// Stand-alone checks on any 32-bit vector (re-read).  `res` must be zeroed
// by the caller's conventions: these kernels set only their own fields.
size_t check_scratch_bytes();
// flt: binary32 values in the IEEE comparison (NaN never out of order)
cudaError_t launch_check_sorted(const int32_t* x, long long n, SortResult* res,
                                void* scratch, cudaStream_t s, int num_sms,
                                int64_t* kernels, Prof* prof, bool flt);
cudaError_t launch_check_perm(const int32_t* x, const int32_t* ref, long long n,
                              SortResult* res, void* scratch, cudaStream_t s,
                              int num_sms, int64_t* kernels, Prof* prof);

// Position-dependent fingerprint of `bytes` bytes at x, read in units of
// unit_bytes (2 or 4): out[0] = sum of h_i, out[1] = sum of hi32(h_i)
// lo32(h_i) mod 2^64 with h_i = mix64(i 2^32 + unit_i) (k_fprint.cu); out is
// cleared first.  The `old` of a postcondition (Sec. 4, Listing 3).
cudaError_t launch_fprint(const void* x, size_t bytes, int unit_bytes, unsigned long long* out,
                          cudaStream_t s, int num_sms, int64_t* kernels, Prof* prof);

// ---------------------------------------------------------------------------
// Filter (k_filter.cu): stable stream compaction with a decoupled look-back
// scan of tile counts.
struct FilterResult {
  long long count;
  int timeout;
  int pad;
  // a for_all postcondition on the kept items checked as they are written
  // (the specialised kernel's folded check): ~(first violating position), 0
  // when none
  unsigned long long post_enc;
};
size_t filter_scratch_bytes(long long n);
cudaError_t launch_filter(const float* x, float* out, long long n,
                          const Prog& pred, int pred_depth, void* scratch,
                          FilterResult* res, cudaStream_t s, int num_sms,
                          int64_t* kernels, Prof* prof, const LookbackCtl& lb);
// the same filter through its run-time specialised kernel (sg_jit.h), whose
// tiles hold `tile` items; scratch: filter_jit_scratch_bytes(n)
size_t filter_jit_scratch_bytes(long long n);
// post: the folded postcondition's program (its constants follow the
// predicate's), or null; the kernel must have been built with it
cudaError_t launch_filter_specialised(cudaKernel_t k, const float* x, float* out, long long n,
                                      const Prog& pred, void* scratch, FilterResult* res,
                                      cudaStream_t s, int num_sms, int64_t* kernels,
                                      Prof* prof, const LookbackCtl& lb, int tile,
                                      const Prog* post = nullptr);

}  // namespace sgk
