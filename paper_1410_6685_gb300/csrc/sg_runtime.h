// sg_runtime.h -- host-side objects of the library: values, handles, the
// deferred-execution graph (Sec. 5) and the context.  Internal.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "safegpu.h"
#include "sg_internal.h"

struct Node;

// Device storage shared by the values that alias it (for_each writes in place).
struct Storage {
  void* ptr = nullptr;
  size_t bytes = 0;
  bool owned = false;
  cudaStream_t stream = nullptr;     // the stream the allocation is freed on
  cudaEvent_t ul_event = nullptr;    // the asynchronous create's copy, until first used
  cudaEvent_t dl_event = nullptr;    // an asynchronous read still in flight
  std::shared_ptr<Storage> parent;   // a subset's view keeps its source alive
  ~Storage();
};

// One value of a collection / vector / matrix (an SSA value of the graph).
struct Value {
  sg_dtype dt = SG_F32;
  int64_t n = 0;          // element count (capacity for a pending filter)
  int64_t rows = 0, cols = 1;
  std::shared_ptr<Storage> st;   // null until materialised
  Node* producer = nullptr;      // pending producer (valid until the flush)
  bool poisoned = false;
  bool count_known = true;       // false for a filter result before its flush
  int handles = 0;               // user handles that point at this value
  int pending_uses = 0;          // uses by queued nodes
};
using ValueP = std::shared_ptr<Value>;

// Two storages share memory: the same allocation, or subset views of one.
inline bool storage_related(const Storage* a, const Storage* b) {
  if (!a || !b) return false;
  while (a->parent) a = a->parent.get();
  while (b->parent) b = b->parent.get();
  return a == b;
}

struct ScalarVal {
  bool done = false;
  bool poisoned = false;
  double value = 0.0;
  int64_t index = -1;
  Node* producer = nullptr;
};
using ScalarP = std::shared_ptr<ScalarVal>;

enum class NK { MAP, REDUCE, QUANT, CHECK, FILTER, SORT, MATMUL, TRANSPOSE, MATVEC, CONCAT,
                SNAPSHOT };

struct Node {
  int id = 0;
  NK kind = NK::MAP;
  sg_expr expr{};                // MAP / QUANT / CHECK(for_all, exists) / FILTER
  int nin = 0;
  ValueP in[4];
  ValueP out;
  bool inplace = false;          // MAP as for_each
  ScalarP sout;                  // REDUCE / QUANT
  int rop = 0;                   // sg_reduce_op
  bool exists = false;           // QUANT: exists (else for_all)
  // CHECK
  int ckind = 0, role = 0, cid = -1;
  bool builtin = false;
  uint64_t seed = 0;
  int nvec = 4;
  double tol = 0.0;
  int prec = 0;                  // MATMUL precision
  bool left = false;             // MATVEC: y = x^T A (in[0] = x, in[1] = A), else y = A x
  // results filled at execution
  int64_t first = -1;
  double observed = 0.0;
  bool failed = false;
};
using NodeP = std::shared_ptr<Node>;

// Captured batched-collections launches, keyed by everything baked into
// the CUDA graph.
struct BatchKey {
  sg_chain chain;
  const float* data;
  const int64_t* offsets;
  int64_t nseg;
  double* sums;
  int64_t* first;
  int64_t* kept;
  long long chunk;
  int grid_per_sm;
  int pad;
};

struct BatchPlan {
  cudaGraphExec_t exec = nullptr;
  void* scratch = nullptr;
  unsigned* host_flag = nullptr;
  long long capacity = 0;
};

struct BatchPlanCache {
  std::vector<std::pair<BatchKey, BatchPlan>> plans;
  cudaStream_t capture_stream = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};   // timing of each batched run
  ~BatchPlanCache();
};

// Timing log and learned cost models of the schedule chooser: one 2x64
// MLP per decision family (sg_sched_family).
constexpr int kSchedFeatures = 12;
constexpr int kSchedMaxCand = 64;
constexpr int kSchedFamilies = 5;
struct SchedModel {
  bool trained = false;
  std::vector<float> mu, sd;  // feature normalisation
  float ymu = 0.0f, ysd = 1.0f;
  void* dev = nullptr;        // params, grads, Adam moments, data (device)
  float* params = nullptr;
  float* pred = nullptr;
  ~SchedModel();
};
struct SchedState {
  std::vector<float> log_x;   // records x kSchedFeatures
  std::vector<float> log_y;   // log microseconds
  std::vector<float> log_rel; // log(us / us of the plain choice), NaN outside sweeps
  std::vector<int> log_fam;   // the record's decision family
  SchedModel model[kSchedFamilies];
  // autotuned choices: hash of (family, workload) -> candidate index
  struct Tuned {
    uint64_t key;
    int idx, family;
    std::vector<double> us;   // the sweep's times, for sg_sched_last
    int learned;              // the model's choice when the sweep ran, or -1
  };
  std::vector<Tuned> tuned;
  // learned choices under the current models (cleared when they are trained)
  std::vector<std::pair<uint64_t, int>> learned_memo;
  // sg_sched_force: a candidate index every decision of the family takes
  int forced[kSchedFamilies] = {-1, -1, -1, -1, -1};
  // the last decision of each family (sg_sched_last)
  sg_sched_report last[kSchedFamilies];
  bool has_last[kSchedFamilies] = {};
};

// The blocked factorisation of one size and precision, captured once as a
// CUDA graph over a workspace the context keeps (factors, pivots, the
// panels' interchange lists, tensor-core operand copies).
struct LuCache {
  int n = 0, prec = -1;
  void* base = nullptr;
  float* lu = nullptr;
  int* piv = nullptr;
  int* perm = nullptr;          // row i of the factors is row perm[i] of A
  float* inv = nullptr;         // inverses of the factors' 32x32 diagonal blocks
  int* info = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  int64_t kernels = 0;          // kernel launches in one replay
  void clear();
  ~LuCache() { clear(); }
};

struct sg_ctx {
  int device = -1;
  bool planning_only = true;
  cudaStream_t stream = nullptr;
  cudaStream_t upload = nullptr;       // asynchronous host-to-device creates
  cudaStream_t download = nullptr;     // asynchronous device-to-host reads
  cudaEvent_t last_download = nullptr; // the latest of them
  int num_sms = 0;
  int mode = SG_CONTRACTS_PRE_POST;
  int fusion = SG_FUSE_ON;
  int sched = SG_SCHED_AUTOTUNE;
  int codegen = SG_CODEGEN_SPECIALIZE;
  std::vector<NodeP> pending;
  int next_node = 0;
  int next_contract = 0;
  std::string err;
  bool has_violation = false;
  sg_violation last_violation{};
  int64_t kernels = 0;
  // device resources
  unsigned int* counter = nullptr;     // last-block-done counter (stays zero)
  void* scratch = nullptr;             // per-flush scratch arena
  size_t scratch_bytes = 0;
  void* host_res = nullptr;            // pinned host copy of pass results
  size_t host_res_bytes = 0;
  bool host_res_mapped = false;        // kernels can store into host_res directly
  sgk::SortInject inject{};            // contract-test fault for the next sort
  sgk::LookbackCtl lookback{0, -1};    // testing switch of the look-back waits
  struct {
    int64_t row = -1, col = -1;
    float delta = 0.0f;
  } mm_inject;                          // contract-test fault for the next tc product
  sgk::Prof prof;                      // per-kernel event tracing
  BatchPlanCache batch;                // captured batched launches
  SchedState schedst;                  // schedule log and cost model
  LuCache lu;                          // factorisation workspace + graph
};

// Makes work enqueued next on the context's stream wait for the
// asynchronous copies of `st` (sg_vector_create_async, sg_vector_read_async)
// still in flight.
void join_transfers(sg_ctx* c, Storage* st);

struct sg_vector {
  sg_ctx* ctx = nullptr;
  ValueP v;
  bool matrix = false;
};

struct sg_scalar {
  sg_ctx* ctx = nullptr;
  ScalarP s;
};
