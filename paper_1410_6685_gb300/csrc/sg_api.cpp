// sg_api.cpp -- the C ABI: contexts, handles, deferred queue, contracts.
//
// Calls are queued on the context (Sec. 5: "a method call is not executed,
// but rather added to a list of pending actions") and run at one of the
// three triggers: a scalar query (sg_scalar_get), a read back to the host
// (sg_vector_read) or an explicit update (sg_flush).  The planner that turns
// the queue into kernels lives in sg_plan.cpp.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "sg_jit.h"
#include "sg_linalg_kernels.h"
#include "sg_plan.h"
#include "sg_runtime.h"

Storage::~Storage() {
  if (ul_event) {
    // never used: free it behind its copy in
    if (owned && ptr) cudaStreamWaitEvent(stream, ul_event, 0);
    cudaEventDestroy(ul_event);
  }
  if (owned && ptr) cudaFreeAsync(ptr, stream);
  if (dl_event) cudaEventDestroy(dl_event);
}

// The storage that owns a view's memory.
static Storage* root_storage(Storage* st) {
  while (st && st->parent) st = st->parent.get();
  return st;
}

// Work about to be enqueued on the context's stream that touches a storage
// waits for its asynchronous copy in, and for an asynchronous read in
// flight (after which the storage is freed on the context's stream again).
void join_transfers(sg_ctx* c, Storage* st) {
  st = root_storage(st);
  if (!st) return;
  if (st->ul_event) {
    cudaStreamWaitEvent(c->stream, st->ul_event, 0);
    cudaEventDestroy(st->ul_event);
    st->ul_event = nullptr;
  }
  if (st->dl_event) {
    cudaStreamWaitEvent(c->stream, st->dl_event, 0);
    cudaEventDestroy(st->dl_event);
    st->dl_event = nullptr;
    st->stream = c->stream;
  }
}

static void join_downloads_of_pending(sg_ctx* c) {
  for (auto& n : c->pending) {
    for (int i = 0; i < n->nin; ++i)
      if (n->in[i] && n->in[i]->st) join_transfers(c, n->in[i]->st.get());
    if (n->out && n->out->st) join_transfers(c, n->out->st.get());
  }
}

struct sg_matrix : public sg_vector {};

namespace {

sg_status fail(sg_ctx* c, sg_status s, const char* fmt, ...)
    __attribute__((format(printf, 3, 4)));

sg_status fail(sg_ctx* c, sg_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return s;
}

size_t dtype_size(sg_dtype dt) {
  switch (dt) {
    case SG_F32: case SG_I32: return 4;
    case SG_F64: case SG_I64: return 8;
    case SG_BF16: case SG_F16: return 2;
  }
  return 0;
}

bool valid_dtype(int dt) { return dt >= SG_F32 && dt <= SG_I64; }

sg_status alloc_storage(sg_ctx* c, size_t bytes, std::shared_ptr<Storage>* out) {
  auto st = std::make_shared<Storage>();
  st->bytes = bytes;
  st->stream = c->stream;
  if (!c->planning_only && bytes) {
    cudaError_t e = cudaMallocAsync(&st->ptr, bytes, c->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(c, SG_ERR_OOM, "device allocation of %zu bytes failed: %s", bytes,
                  cudaGetErrorString(e));
    }
    st->owned = true;
  }
  *out = std::move(st);
  return SG_OK;
}

// Validates a user expression over `nin` input slots; returns its max depth.
sg_status check_expr(sg_ctx* c, const sg_expr* f, int nin, int* depth_out) {
  char msg[160];
  const sg_status s = sgk::validate_expr(f, nin, depth_out, nullptr, msg, sizeof msg);
  if (s) return fail(c, s, "%s", msg);
  return SG_OK;
}

sg_status check_vec(sg_vector* v) {
  if (!v || !v->ctx || !v->v) return SG_ERR_INVALID_ARG;
  return SG_OK;
}

// A scalar contract needs counts: a pending filter's count is only known
// after its flush (trigger 1 of Sec. 5 applies).
sg_status known_count(sg_vector* v) {
  if (v->v->count_known) return SG_OK;
  return sg_flush(v->ctx);
}

// A queued in-place write (for_each) lands in memory that v shares (v
// itself, or a subset view of the same allocation): reading v must flush.
bool pending_write_to(sg_ctx* c, const Value* v) {
  for (auto& n : c->pending)
    if (n->inplace && n->out && storage_related(n->out->st.get(), v->st.get())) return true;
  return false;
}

sg_vector* new_handle(sg_ctx* c, ValueP v, bool matrix) {
  sg_vector* h = matrix ? static_cast<sg_vector*>(new sg_matrix) : new sg_vector;
  h->ctx = c;
  h->v = std::move(v);
  h->matrix = matrix;
  h->v->handles++;
  return h;
}

NodeP new_node(sg_ctx* c, NK k) {
  auto n = std::make_shared<Node>();
  n->id = c->next_node++;
  n->kind = k;
  return n;
}

void use(Node* n, int slot, const ValueP& v) {
  n->in[slot] = v;
  v->pending_uses++;
}

void enqueue(sg_ctx* c, NodeP n) {
  if (n->out) n->out->producer = n.get();
  if (n->sout) n->sout->producer = n.get();
  c->pending.push_back(std::move(n));
}

sg_status make_out(sg_ctx* c, sg_dtype dt, int64_t n, int64_t rows, int64_t cols,
                   ValueP* out) {
  auto v = std::make_shared<Value>();
  v->dt = dt;
  v->n = n;
  v->rows = rows;
  v->cols = cols;
  (void)c;
  *out = std::move(v);
  return SG_OK;
}

sg_status new_scalar(sg_ctx* c, ScalarP s, sg_scalar** out) {
  auto* h = new sg_scalar;
  h->ctx = c;
  h->s = std::move(s);
  *out = h;
  return SG_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" {

const char* sg_status_name(sg_status s) {
  switch (s) {
    case SG_OK: return "SG_OK";
    case SG_ERR_INVALID_ARG: return "SG_ERR_INVALID_ARG";
    case SG_ERR_SHAPE: return "SG_ERR_SHAPE";
    case SG_ERR_DTYPE: return "SG_ERR_DTYPE";
    case SG_ERR_OOM: return "SG_ERR_OOM";
    case SG_ERR_CUDA: return "SG_ERR_CUDA";
    case SG_ERR_PRECONDITION: return "SG_ERR_PRECONDITION";
    case SG_ERR_POSTCONDITION: return "SG_ERR_POSTCONDITION";
    case SG_ERR_TIMEOUT: return "SG_ERR_TIMEOUT";
    case SG_ERR_NOT_CONVERGED: return "SG_ERR_NOT_CONVERGED";
    case SG_ERR_POISONED: return "SG_ERR_POISONED";
    case SG_ERR_UNSUPPORTED: return "SG_ERR_UNSUPPORTED";
    case SG_ERR_SINGULAR: return "SG_ERR_SINGULAR";
  }
  return "SG_ERR_?";
}

sg_status sg_init(int device, void* stream, sg_ctx** out) {
  if (!out) return SG_ERR_INVALID_ARG;
  auto* c = new sg_ctx;
  c->device = device;
  if (const char* g = getenv("SG_CODEGEN"))
    if (strcmp(g, "interpret") == 0) c->codegen = SG_CODEGEN_INTERPRET;
  c->stream = static_cast<cudaStream_t>(stream);
  if (device >= 0) {
    c->planning_only = false;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->upload, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->download, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->last_download, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&c->counter, 64 * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(c->counter, 0, 64 * sizeof(unsigned int));
    if (e == cudaSuccess) {
      // library values come from the device's stream-ordered pool; keep freed
      // blocks in the pool (this process only) so that a value of the same
      // size in the next step does not go back to the driver
      cudaMemPool_t pool = nullptr;
      if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        // a block freed on one of the context's streams is not handed to an
        // allocation on another by making that stream wait (it would chain
        // an asynchronous copy in behind an asynchronous read): such a block
        // is reused once its free has completed, else a new one is taken
        int no = 0;
        cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
      }
      cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (c->counter) cudaFree(c->counter);
      if (c->upload) cudaStreamDestroy(c->upload);
      if (c->download) cudaStreamDestroy(c->download);
      if (c->last_download) cudaEventDestroy(c->last_download);
      delete c;
      return SG_ERR_CUDA;
    }
  }
  *out = c;
  return SG_OK;
}

sg_status sg_destroy(sg_ctx* c) {
  if (!c) return SG_ERR_INVALID_ARG;
  c->pending.clear();
  if (!c->planning_only) {
    cudaStreamSynchronize(c->upload);
    cudaStreamSynchronize(c->download);
    cudaStreamSynchronize(c->stream);
    cudaStreamDestroy(c->upload);
    cudaStreamDestroy(c->download);
    cudaEventDestroy(c->last_download);
    if (c->scratch) cudaFree(c->scratch);
    if (c->counter) cudaFree(c->counter);
    if (c->host_res) cudaFreeHost(c->host_res);
  }
  delete c;
  return SG_OK;
}

const char* sg_last_error(sg_ctx* c) { return c ? c->err.c_str() : "null context"; }

// ---------------------------------------------------------------------------
// vectors and matrices

static sg_status create_common(sg_ctx* c, sg_dtype dt, int64_t rows, int64_t cols,
                               const void* host, bool matrix, sg_vector** out) {
  if (!c || !out || !valid_dtype(dt) || rows < 0 || cols < 0)
    return fail(c, SG_ERR_INVALID_ARG, "bad create arguments");
  const int64_t n = rows * cols;
  ValueP v;
  make_out(c, dt, n, rows, cols, &v);
  sg_status s = alloc_storage(c, (size_t)n * dtype_size(dt), &v->st);
  if (s) return s;
  if (host && n && !c->planning_only) {
    cudaError_t e = cudaMemcpyAsync(v->st->ptr, host, (size_t)n * dtype_size(dt),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess)
      return fail(c, SG_ERR_CUDA, "host to device copy failed: %s", cudaGetErrorString(e));
  }
  *out = new_handle(c, v, matrix);
  return SG_OK;
}

static sg_status wrap_common(sg_ctx* c, sg_dtype dt, int64_t rows, int64_t cols, void* p,
                             bool matrix, sg_vector** out) {
  if (!c || !out || !valid_dtype(dt) || rows < 0 || cols < 0 || (!p && rows * cols > 0))
    return fail(c, SG_ERR_INVALID_ARG, "bad wrap arguments");
  ValueP v;
  make_out(c, dt, rows * cols, rows, cols, &v);
  v->st = std::make_shared<Storage>();
  v->st->ptr = p;
  v->st->bytes = (size_t)(rows * cols) * dtype_size(dt);
  v->st->owned = false;
  *out = new_handle(c, v, matrix);
  return SG_OK;
}

sg_status sg_vector_create(sg_ctx* c, sg_dtype dt, int64_t n, const void* host,
                           sg_vector** out) {
  return create_common(c, dt, n, 1, host, false, out);
}

sg_status sg_vector_wrap(sg_ctx* c, sg_dtype dt, int64_t n, void* p, sg_vector** out) {
  return wrap_common(c, dt, n, 1, p, false, out);
}

static sg_status read_common(sg_vector* h, void* host, int64_t n) {
  if (check_vec(h) || (!host && n > 0)) return SG_ERR_INVALID_ARG;
  sg_ctx* c = h->ctx;
  if (h->v->producer || !h->v->count_known || pending_write_to(c, h->v.get())) {
    sg_status s = sg_flush(c);
    if (s && s != SG_ERR_PRECONDITION && s != SG_ERR_POSTCONDITION) return s;
  }
  if (h->v->poisoned) return fail(c, SG_ERR_POISONED, "value depends on a failed contract");
  if (n != h->v->n) return fail(c, SG_ERR_SHAPE, "read of %lld elements, count is %lld",
                                (long long)n, (long long)h->v->n);
  if (c->planning_only) return fail(c, SG_ERR_UNSUPPORTED, "planning-only context");
  if (n == 0) return SG_OK;
  join_transfers(c, h->v->st.get());
  cudaError_t e = cudaMemcpyAsync(host, h->v->st->ptr, (size_t)n * dtype_size(h->v->dt),
                                  cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess)
    return fail(c, SG_ERR_CUDA, "device to host copy failed: %s", cudaGetErrorString(e));
  return SG_OK;
}

sg_status sg_vector_read(sg_vector* h, void* host, int64_t n) { return read_common(h, host, n); }

sg_status sg_vector_create_async(sg_ctx* c, sg_dtype dt, int64_t n, const void* host,
                                 sg_vector** out) {
  if (!c || !out || !valid_dtype(dt) || n < 0 || (!host && n > 0))
    return fail(c, SG_ERR_INVALID_ARG, "bad create arguments");
  if (c->planning_only) return fail(c, SG_ERR_UNSUPPORTED, "planning-only context");
  ValueP v;
  make_out(c, dt, n, n, 1, &v);
  auto st = std::make_shared<Storage>();
  st->bytes = (size_t)n * dtype_size(dt);
  st->stream = c->stream;   // freed behind the work that uses it
  if (st->bytes) {
    cudaError_t e = cudaMallocAsync(&st->ptr, st->bytes, c->upload);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(c, SG_ERR_OOM, "device allocation of %zu bytes failed", st->bytes);
    }
    st->owned = true;
    e = cudaMemcpyAsync(st->ptr, host, st->bytes, cudaMemcpyHostToDevice, c->upload);
    // the first work on the context's stream that uses the value waits for it
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&st->ul_event, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(st->ul_event, c->upload);
    if (e != cudaSuccess)
      return fail(c, SG_ERR_CUDA, "host to device copy failed: %s", cudaGetErrorString(e));
  }
  v->st = std::move(st);
  *out = new_handle(c, v, false);
  return SG_OK;
}

sg_status sg_vector_read_async(sg_vector* h, void* host, int64_t n) {
  if (check_vec(h) || (!host && n > 0)) return SG_ERR_INVALID_ARG;
  sg_ctx* c = h->ctx;
  if (h->v->producer || !h->v->count_known || pending_write_to(c, h->v.get())) {
    sg_status s = sg_flush(c);
    if (s && s != SG_ERR_PRECONDITION && s != SG_ERR_POSTCONDITION) return s;
  }
  if (h->v->poisoned) return fail(c, SG_ERR_POISONED, "value depends on a failed contract");
  if (n != h->v->n) return fail(c, SG_ERR_SHAPE, "read of %lld elements, count is %lld",
                                (long long)n, (long long)h->v->n);
  if (c->planning_only) return fail(c, SG_ERR_UNSUPPORTED, "planning-only context");
  if (n == 0) return SG_OK;
  Storage* root = root_storage(h->v->st.get());
  cudaEvent_t made = nullptr, done = nullptr;
  cudaError_t e = cudaEventCreateWithFlags(&made, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
  // the copy follows everything enqueued so far on the context's stream
  if (e == cudaSuccess) e = cudaEventRecord(made, c->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->download, made, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host, h->v->st->ptr, (size_t)n * dtype_size(h->v->dt),
                        cudaMemcpyDeviceToHost, c->download);
  if (e == cudaSuccess) e = cudaEventRecord(done, c->download);
  if (made) cudaEventDestroy(made);
  if (e != cudaSuccess) {
    if (done) cudaEventDestroy(done);
    return fail(c, SG_ERR_CUDA, "device to host copy failed: %s", cudaGetErrorString(e));
  }
  if (root->dl_event) cudaEventDestroy(root->dl_event);
  root->dl_event = done;
  cudaEventRecord(c->last_download, c->download);
  // released before any further use: freed behind the copy
  root->stream = c->download;
  return SG_OK;
}

sg_status sg_sync(sg_ctx* c) {
  if (!c) return SG_ERR_INVALID_ARG;
  if (c->planning_only) return SG_OK;
  cudaError_t e = cudaStreamSynchronize(c->upload);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->download);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(c, SG_ERR_CUDA, "synchronisation failed: %s", cudaGetErrorString(e));
  return SG_OK;
}

sg_status sg_vector_count(sg_vector* h, int64_t* n) {
  if (check_vec(h) || !n) return SG_ERR_INVALID_ARG;
  sg_status s = known_count(h);
  if (s && s != SG_ERR_PRECONDITION && s != SG_ERR_POSTCONDITION) return s;
  *n = h->v->n;
  return SG_OK;
}

static sg_status devptr_common(sg_vector* h, void** p) {
  if (check_vec(h) || !p) return SG_ERR_INVALID_ARG;
  if (h->v->producer || !h->v->count_known || pending_write_to(h->ctx, h->v.get())) {
    sg_status s = sg_flush(h->ctx);
    if (s && s != SG_ERR_PRECONDITION && s != SG_ERR_POSTCONDITION) return s;
  }
  if (!h->v->st) return fail(h->ctx, SG_ERR_UNSUPPORTED, "value was never materialised");
  // work the caller enqueues on the context's stream sees its copies done
  if (!h->ctx->planning_only) join_transfers(h->ctx, h->v->st.get());
  *p = h->v->st->ptr;
  return SG_OK;
}

sg_status sg_vector_device_ptr(sg_vector* h, void** p) { return devptr_common(h, p); }

sg_status sg_vector_item(sg_vector* h, int64_t i, void* value) {
  if (check_vec(h) || !value) return SG_ERR_INVALID_ARG;
  sg_ctx* c = h->ctx;
  if (h->v->producer || !h->v->count_known || pending_write_to(c, h->v.get())) {
    sg_status s = sg_flush(c);
    if (s && s != SG_ERR_PRECONDITION && s != SG_ERR_POSTCONDITION) return s;
  }
  if (h->v->poisoned) return fail(c, SG_ERR_POISONED, "value depends on a failed contract");
  if (i < 0 || i >= h->v->n)
    return fail(c, SG_ERR_SHAPE, "item %lld of a vector of %lld", (long long)i, (long long)h->v->n);
  if (c->planning_only) return fail(c, SG_ERR_UNSUPPORTED, "planning-only context");
  const size_t es = dtype_size(h->v->dt);
  join_transfers(c, h->v->st.get());
  cudaError_t e = cudaMemcpyAsync(value, static_cast<const char*>(h->v->st->ptr) + (size_t)i * es,
                                  es, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(c, SG_ERR_CUDA, "item copy failed: %s", cudaGetErrorString(e));
  return SG_OK;
}

sg_status sg_concat(sg_ctx* c, sg_vector* a, sg_vector* b, sg_vector** out) {
  if (!c || check_vec(a) || check_vec(b) || a->ctx != c || b->ctx != c || !out)
    return fail(c, SG_ERR_INVALID_ARG, "bad concatenate");
  if (a->v->dt != b->v->dt) return fail(c, SG_ERR_DTYPE, "concatenate of different dtypes");
  sg_status s = known_count(a);
  if (!s) s = known_count(b);
  if (s && s != SG_ERR_PRECONDITION && s != SG_ERR_POSTCONDITION) return s;
  NodeP n = new_node(c, NK::CONCAT);
  n->nin = 2;
  use(n.get(), 0, a->v);
  use(n.get(), 1, b->v);
  const int64_t len = a->v->n + b->v->n;
  make_out(c, a->v->dt, len, len, 1, &n->out);
  sg_vector* h = new_handle(c, n->out, false);
  enqueue(c, std::move(n));
  *out = h;
  return SG_OK;
}

sg_status sg_subset(sg_ctx* c, sg_vector* v, int64_t start, int64_t finish, sg_vector** out) {
  if (!c || check_vec(v) || v->ctx != c || !out) return fail(c, SG_ERR_INVALID_ARG, "bad subset");
  if (v->v->producer || !v->v->count_known) {
    sg_status s = sg_flush(c);
    if (s && s != SG_ERR_PRECONDITION && s != SG_ERR_POSTCONDITION) return s;
  }
  if (v->v->poisoned) return fail(c, SG_ERR_POISONED, "value depends on a failed contract");
  if (start < 0 || start > finish || finish > v->v->n)
    return fail(c, SG_ERR_SHAPE, "subset [%lld, %lld) of a vector of %lld", (long long)start,
                (long long)finish, (long long)v->v->n);
  const size_t es = dtype_size(v->v->dt);
  auto view = std::make_shared<Storage>();
  view->ptr = v->v->st ? static_cast<char*>(v->v->st->ptr) + (size_t)start * es : nullptr;
  view->bytes = (size_t)(finish - start) * es;
  view->owned = false;
  view->parent = v->v->st;
  ValueP nv;
  make_out(c, v->v->dt, finish - start, finish - start, 1, &nv);
  nv->st = std::move(view);
  *out = new_handle(c, nv, false);
  return SG_OK;
}

sg_status sg_vector_release(sg_vector* h) {
  if (!h) return SG_ERR_INVALID_ARG;
  if (h->v) h->v->handles--;
  if (h->matrix) delete static_cast<sg_matrix*>(h);
  else delete h;
  return SG_OK;
}

sg_status sg_matrix_create(sg_ctx* c, sg_dtype dt, int64_t rows, int64_t cols,
                           const void* host, sg_matrix** out) {
  sg_vector* h = nullptr;
  sg_status s = create_common(c, dt, rows, cols, host, true, &h);
  if (!s) *out = static_cast<sg_matrix*>(h);
  return s;
}

sg_status sg_matrix_wrap(sg_ctx* c, sg_dtype dt, int64_t rows, int64_t cols, void* p,
                         sg_matrix** out) {
  sg_vector* h = nullptr;
  sg_status s = wrap_common(c, dt, rows, cols, p, true, &h);
  if (!s) *out = static_cast<sg_matrix*>(h);
  return s;
}

sg_status sg_matrix_read(sg_matrix* m, void* host, int64_t count) {
  return read_common(m, host, count);
}

sg_status sg_matrix_shape(sg_matrix* m, int64_t* rows, int64_t* cols) {
  if (check_vec(m) || !rows || !cols) return SG_ERR_INVALID_ARG;
  *rows = m->v->rows;
  *cols = m->v->cols;
  return SG_OK;
}

sg_status sg_matrix_device_ptr(sg_matrix* m, void** p) { return devptr_common(m, p); }

sg_status sg_matrix_release(sg_matrix* m) { return sg_vector_release(m); }

sg_status sg_matrix_as_vector(sg_matrix* m, sg_vector** out) {
  if (check_vec(m) || !out) return SG_ERR_INVALID_ARG;
  *out = new_handle(m->ctx, m->v, false);
  return SG_OK;
}

// ---------------------------------------------------------------------------
// collection operations

sg_status sg_mapn(sg_ctx* c, const sg_expr* f, int nin, sg_vector* const* ins,
                  sg_vector** out) {
  if (!c || !out || nin < 1 || nin > 4 || !ins)
    return fail(c, SG_ERR_INVALID_ARG, "map needs 1..4 inputs and an output");
  for (int k = 0; k < nin; ++k) {
    if (check_vec(ins[k]) || ins[k]->ctx != c) return fail(c, SG_ERR_INVALID_ARG, "bad input %d", k);
    if (ins[k]->v->dt != SG_F32) return fail(c, SG_ERR_DTYPE, "map inputs must be SG_F32");
    sg_status s = known_count(ins[k]);
    if (s && s != SG_ERR_PRECONDITION && s != SG_ERR_POSTCONDITION) return s;
  }
  for (int k = 1; k < nin; ++k)
    if (ins[k]->v->n != ins[0]->v->n)
      return fail(c, SG_ERR_SHAPE, "input %d has count %lld, input 0 has %lld", k,
                  (long long)ins[k]->v->n, (long long)ins[0]->v->n);
  sg_status s = check_expr(c, f, nin, nullptr);
  if (s) return s;
  NodeP n = new_node(c, NK::MAP);
  n->expr = *f;
  n->nin = nin;
  for (int k = 0; k < nin; ++k) use(n.get(), k, ins[k]->v);
  make_out(c, SG_F32, ins[0]->v->n, ins[0]->v->n, 1, &n->out);
  sg_vector* h = new_handle(c, n->out, false);
  enqueue(c, std::move(n));
  *out = h;
  return SG_OK;
}

sg_status sg_map(sg_ctx* c, const sg_expr* f, sg_vector* x, sg_vector** out) {
  sg_vector* ins[1] = {x};
  return sg_mapn(c, f, 1, ins, out);
}

sg_status sg_zip(sg_ctx* c, const sg_expr* f, sg_vector* x, sg_vector* y, sg_vector** out) {
  sg_vector* ins[2] = {x, y};
  return sg_mapn(c, f, 2, ins, out);
}

sg_status sg_for_each(sg_ctx* c, const sg_expr* f, sg_vector* x) {
  if (!c || check_vec(x) || x->ctx != c) return fail(c, SG_ERR_INVALID_ARG, "bad for_each");
  if (x->v->dt != SG_F32) return fail(c, SG_ERR_DTYPE, "for_each needs SG_F32");
  sg_status s = known_count(x);
  if (s && s != SG_ERR_PRECONDITION && s != SG_ERR_POSTCONDITION) return s;
  s = check_expr(c, f, 1, nullptr);
  if (s) return s;
  NodeP n = new_node(c, NK::MAP);
  n->expr = *f;
  n->nin = 1;
  n->inplace = true;
  use(n.get(), 0, x->v);
  make_out(c, SG_F32, x->v->n, x->v->rows, x->v->cols, &n->out);
  // the new value writes over the old one's storage (allocated now if the
  // old value was itself never materialised)
  if (!x->v->st) {
    s = alloc_storage(c, (size_t)x->v->n * 4, &x->v->st);
    if (s) return s;
  }
  n->out->st = x->v->st;
  x->v->handles--;
  x->v = n->out;
  x->v->handles++;
  enqueue(c, std::move(n));
  return SG_OK;
}

sg_status sg_filter(sg_ctx* c, const sg_expr* pred, sg_vector* x, sg_vector** out) {
  if (!c || check_vec(x) || !out || x->ctx != c) return fail(c, SG_ERR_INVALID_ARG, "bad filter");
  if (x->v->dt != SG_F32) return fail(c, SG_ERR_DTYPE, "filter needs SG_F32");
  sg_status s = known_count(x);
  if (s && s != SG_ERR_PRECONDITION && s != SG_ERR_POSTCONDITION) return s;
  s = check_expr(c, pred, 1, nullptr);
  if (s) return s;
  NodeP n = new_node(c, NK::FILTER);
  n->expr = *pred;
  n->nin = 1;
  use(n.get(), 0, x->v);
  make_out(c, SG_F32, x->v->n, x->v->n, 1, &n->out);
  n->out->count_known = false;
  sg_vector* h = new_handle(c, n->out, false);
  enqueue(c, std::move(n));
  *out = h;
  return SG_OK;
}

sg_status sg_reduce(sg_ctx* c, sg_reduce_op op, sg_vector* x, sg_scalar** out) {
  if (!c || check_vec(x) || !out || x->ctx != c || op < SG_REDUCE_SUM || op > SG_REDUCE_COUNT)
    return fail(c, SG_ERR_INVALID_ARG, "bad reduce");
  if (x->v->dt != SG_F32) return fail(c, SG_ERR_DTYPE, "reduce needs SG_F32");
  NodeP n = new_node(c, NK::REDUCE);
  n->rop = op;
  n->nin = 1;
  use(n.get(), 0, x->v);
  n->sout = std::make_shared<ScalarVal>();
  ScalarP sv = n->sout;
  enqueue(c, std::move(n));
  return new_scalar(c, sv, out);
}

static sg_status quant(sg_ctx* c, const sg_expr* pred, int nin, sg_vector* const* ins,
                       sg_scalar** out, bool exists) {
  if (!c || !out || nin < 1 || nin > 4 || !ins)
    return fail(c, SG_ERR_INVALID_ARG, "for_all/exists need 1..4 inputs");
  for (int k = 0; k < nin; ++k) {
    if (check_vec(ins[k]) || ins[k]->ctx != c) return fail(c, SG_ERR_INVALID_ARG, "bad input %d", k);
    if (ins[k]->v->dt != SG_F32) return fail(c, SG_ERR_DTYPE, "inputs must be SG_F32");
    sg_status s = known_count(ins[k]);
    if (s && s != SG_ERR_PRECONDITION && s != SG_ERR_POSTCONDITION) return s;
    if (ins[k]->v->n != ins[0]->v->n) return fail(c, SG_ERR_SHAPE, "input counts differ");
  }
  sg_status s = check_expr(c, pred, nin, nullptr);
  if (s) return s;
  NodeP n = new_node(c, NK::QUANT);
  n->expr = *pred;
  n->nin = nin;
  n->exists = exists;
  for (int k = 0; k < nin; ++k) use(n.get(), k, ins[k]->v);
  n->sout = std::make_shared<ScalarVal>();
  ScalarP sv = n->sout;
  enqueue(c, std::move(n));
  return new_scalar(c, sv, out);
}

sg_status sg_for_all(sg_ctx* c, const sg_expr* pred, int nin, sg_vector* const* ins,
                     sg_scalar** out) {
  return quant(c, pred, nin, ins, out, false);
}

sg_status sg_exists(sg_ctx* c, const sg_expr* pred, int nin, sg_vector* const* ins,
                    sg_scalar** out) {
  return quant(c, pred, nin, ins, out, true);
}

static sg_status scalar_ready(sg_scalar* s) {
  if (!s || !s->s) return SG_ERR_INVALID_ARG;
  if (!s->s->done) {
    sg_status st = sg_flush(s->ctx);
    if (st && st != SG_ERR_PRECONDITION && st != SG_ERR_POSTCONDITION) return st;
  }
  if (s->s->poisoned) return fail(s->ctx, SG_ERR_POISONED, "scalar depends on a failed contract");
  return SG_OK;
}

sg_status sg_scalar_get(sg_scalar* s, double* value) {
  if (!value) return SG_ERR_INVALID_ARG;
  sg_status st = scalar_ready(s);
  if (st) return st;
  *value = s->s->value;
  return SG_OK;
}

sg_status sg_scalar_index(sg_scalar* s, int64_t* index) {
  if (!index) return SG_ERR_INVALID_ARG;
  sg_status st = scalar_ready(s);
  if (st) return st;
  *index = s->s->index;
  return SG_OK;
}

sg_status sg_scalar_release(sg_scalar* s) {
  if (!s) return SG_ERR_INVALID_ARG;
  delete s;
  return SG_OK;
}

// ---------------------------------------------------------------------------
// sort, matmul

sg_status sg_sort(sg_ctx* c, sg_vector* keys, sg_vector** out) {
  if (!c || check_vec(keys) || !out || keys->ctx != c) return fail(c, SG_ERR_INVALID_ARG, "bad sort");
  if (keys->v->dt != SG_I32 && keys->v->dt != SG_F32)
    return fail(c, SG_ERR_DTYPE, "sort keys must be SG_I32 or SG_F32");
  sg_status s = known_count(keys);
  if (s && s != SG_ERR_PRECONDITION && s != SG_ERR_POSTCONDITION) return s;
  if (keys->v->n >= (int64_t(1) << 30)) return fail(c, SG_ERR_SHAPE, "sort supports n < 2^30");
  NodeP n = new_node(c, NK::SORT);
  n->nin = 1;
  use(n.get(), 0, keys->v);
  make_out(c, keys->v->dt, keys->v->n, keys->v->n, 1, &n->out);
  ValueP outv = n->out, inv = keys->v;
  sg_vector* h = new_handle(c, n->out, false);
  enqueue(c, std::move(n));
  if (c->mode >= SG_CONTRACTS_PRE_POST) {
    // Listing 4: ensure Result.is_sorted; Result.count = a.count (as a
    // permutation check).  Queued right behind the sort so the planner fuses
    // them into its last pass.
    NodeP k1 = new_node(c, NK::CHECK);
    k1->ckind = SG_C_SORTED; k1->role = SG_POST; k1->builtin = true; k1->nin = 1;
    use(k1.get(), 0, outv);
    enqueue(c, std::move(k1));
    NodeP k2 = new_node(c, NK::CHECK);
    k2->ckind = SG_C_PERMUTATION; k2->role = SG_POST; k2->builtin = true; k2->nin = 2;
    use(k2.get(), 0, outv);
    use(k2.get(), 1, inv);
    enqueue(c, std::move(k2));
  }
  *out = h;
  return SG_OK;
}

sg_status sg_transpose(sg_ctx* c, sg_matrix* A, sg_matrix** At) {
  if (!c || check_vec(A) || A->ctx != c || !At) return fail(c, SG_ERR_INVALID_ARG, "bad transpose");
  if (A->v->dt != SG_F32) return fail(c, SG_ERR_DTYPE, "transpose needs SG_F32");
  NodeP n = new_node(c, NK::TRANSPOSE);
  n->nin = 1;
  use(n.get(), 0, A->v);
  make_out(c, SG_F32, A->v->n, A->v->cols, A->v->rows, &n->out);
  sg_vector* h = new_handle(c, n->out, true);
  enqueue(c, std::move(n));
  *At = static_cast<sg_matrix*>(h);
  return SG_OK;
}

sg_status sg_matvec(sg_ctx* c, sg_matrix* A, sg_vector* x, sg_vector** y) {
  if (!c || check_vec(A) || check_vec(x) || A->ctx != c || x->ctx != c || !y)
    return fail(c, SG_ERR_INVALID_ARG, "bad matvec");
  if (A->v->dt != SG_F32 || x->v->dt != SG_F32) return fail(c, SG_ERR_DTYPE, "matvec needs SG_F32");
  sg_status ks = known_count(x);
  if (ks && ks != SG_ERR_PRECONDITION && ks != SG_ERR_POSTCONDITION) return ks;
  // precondition of Listing 1: the vector's count matches the matrix
  if (x->v->n != A->v->cols)
    return fail(c, SG_ERR_SHAPE, "A is %lldx%lld, x has %lld elements", (long long)A->v->rows,
                (long long)A->v->cols, (long long)x->v->n);
  NodeP n = new_node(c, NK::MATVEC);
  n->nin = 2;
  n->left = false;
  use(n.get(), 0, A->v);
  use(n.get(), 1, x->v);
  make_out(c, SG_F32, A->v->rows, A->v->rows, 1, &n->out);
  sg_vector* h = new_handle(c, n->out, false);
  enqueue(c, std::move(n));
  *y = h;
  return SG_OK;
}

sg_status sg_vecmat(sg_ctx* c, sg_vector* x, sg_matrix* A, sg_vector** y) {
  if (!c || check_vec(A) || check_vec(x) || A->ctx != c || x->ctx != c || !y)
    return fail(c, SG_ERR_INVALID_ARG, "bad vecmat");
  if (A->v->dt != SG_F32 || x->v->dt != SG_F32) return fail(c, SG_ERR_DTYPE, "vecmat needs SG_F32");
  sg_status ks = known_count(x);
  if (ks && ks != SG_ERR_PRECONDITION && ks != SG_ERR_POSTCONDITION) return ks;
  if (x->v->n != A->v->rows)
    return fail(c, SG_ERR_SHAPE, "x has %lld elements, A is %lldx%lld", (long long)x->v->n,
                (long long)A->v->rows, (long long)A->v->cols);
  NodeP n = new_node(c, NK::MATVEC);
  n->nin = 2;
  n->left = true;
  use(n.get(), 0, x->v);
  use(n.get(), 1, A->v);
  make_out(c, SG_F32, A->v->cols, A->v->cols, 1, &n->out);
  sg_vector* h = new_handle(c, n->out, false);
  enqueue(c, std::move(n));
  *y = h;
  return SG_OK;
}

sg_status sg_matmul(sg_ctx* c, sg_matrix* A, sg_matrix* B, sg_precision p, sg_matrix** C) {
  if (!c || check_vec(A) || check_vec(B) || !C || p < SG_PREC_F32_SIMT || p > SG_PREC_F16_TC)
    return fail(c, SG_ERR_INVALID_ARG, "bad matmul");
  if (A->v->dt != SG_F32 || B->v->dt != SG_F32) return fail(c, SG_ERR_DTYPE, "matmul needs SG_F32");
  if (A->v->cols != B->v->rows)
    return fail(c, SG_ERR_SHAPE, "A is %lldx%lld, B is %lldx%lld", (long long)A->v->rows,
                (long long)A->v->cols, (long long)B->v->rows, (long long)B->v->cols);
  NodeP n = new_node(c, NK::MATMUL);
  n->nin = 2;
  n->prec = p;
  use(n.get(), 0, A->v);
  use(n.get(), 1, B->v);
  make_out(c, SG_F32, A->v->rows * B->v->cols, A->v->rows, B->v->cols, &n->out);
  ValueP cv = n->out, av = A->v, bv = B->v;
  sg_vector* h = new_handle(c, n->out, true);
  enqueue(c, std::move(n));
  if (c->mode >= SG_CONTRACTS_PRE_POST && A->v->rows == A->v->cols && B->v->rows == B->v->cols) {
    NodeP k = new_node(c, NK::CHECK);
    k->ckind = SG_C_FREIVALDS; k->role = SG_POST; k->builtin = true; k->nin = 3;
    k->seed = 6; k->nvec = 4; k->tol = 8.0; k->prec = p;
    use(k.get(), 0, cv);
    use(k.get(), 1, av);
    use(k.get(), 2, bv);
    enqueue(c, std::move(k));
  }
  *C = static_cast<sg_matrix*>(h);
  return SG_OK;
}

// ---------------------------------------------------------------------------
// contracts

static sg_status attach(sg_ctx* c, void* target, const sg_contract* k, int32_t* id, int role) {
  if (!c || !target || !k) return fail(c, SG_ERR_INVALID_ARG, "bad contract");
  sg_vector* t = static_cast<sg_vector*>(target);
  if (check_vec(t) || t->ctx != c) return fail(c, SG_ERR_INVALID_ARG, "bad contract target");
  if (k->nother < 0 || k->nother > 3) return fail(c, SG_ERR_INVALID_ARG, "nother must be 0..3");
  for (int i = 0; i < k->nother; ++i) {
    sg_vector* o = static_cast<sg_vector*>(k->other[i]);
    if (check_vec(o) || o->ctx != c) return fail(c, SG_ERR_INVALID_ARG, "bad contract operand %d", i);
  }
  const int cid = c->next_contract++;
  if (id) *id = cid;
  // Sec. 6.3 modes: OFF checks nothing, PRE only preconditions.
  const bool active = (role == SG_PRE) ? c->mode >= SG_CONTRACTS_PRE : c->mode >= SG_CONTRACTS_PRE_POST;
  NodeP n = new_node(c, NK::CHECK);
  n->ckind = k->kind;
  n->role = role;
  n->cid = cid;
  switch (k->kind) {
    case SG_C_FOR_ALL:
    case SG_C_EXISTS: {
      const int nin = 1 + k->nother;
      if (t->v->dt != SG_F32) return fail(c, SG_ERR_DTYPE, "for_all/exists need SG_F32");
      // a contract on a queued filter's result alone needs no count now: it
      // runs in the same flush, over the count the filter finds on the device
      // (checked by the filter itself where the plan folds it in)
      const bool behind_filter = !t->v->count_known && k->nother == 0 && t->v->producer &&
                                 t->v->producer->kind == NK::FILTER;
      sg_status s = behind_filter ? SG_OK : known_count(t);
      if (s && s != SG_ERR_PRECONDITION && s != SG_ERR_POSTCONDITION) return s;
      for (int i = 0; i < k->nother; ++i) {
        sg_vector* o = static_cast<sg_vector*>(k->other[i]);
        if (o->v->dt != SG_F32) return fail(c, SG_ERR_DTYPE, "contract operands must be SG_F32");
        s = known_count(o);
        if (s && s != SG_ERR_PRECONDITION && s != SG_ERR_POSTCONDITION) return s;
        if (o->v->n != t->v->n) return fail(c, SG_ERR_SHAPE, "contract operand %d count differs", i);
      }
      s = check_expr(c, &k->expr, nin, nullptr);
      if (s) return s;
      if (!active) return SG_OK;
      n->expr = k->expr;
      n->nin = nin;
      use(n.get(), 0, t->v);
      for (int i = 0; i < k->nother; ++i) use(n.get(), 1 + i, static_cast<sg_vector*>(k->other[i])->v);
      break;
    }
    case SG_C_SORTED:
      if (t->v->dt != SG_I32 && t->v->dt != SG_F32)
        return fail(c, SG_ERR_DTYPE, "sortedness contract needs SG_I32 or SG_F32");
      if (!active) return SG_OK;
      n->nin = 1;
      use(n.get(), 0, t->v);
      break;
    case SG_C_PERMUTATION: {
      if (k->nother != 1) return fail(c, SG_ERR_INVALID_ARG, "permutation needs other[0]");
      sg_vector* o = static_cast<sg_vector*>(k->other[0]);
      if ((t->v->dt != SG_I32 && t->v->dt != SG_F32) || o->v->dt != t->v->dt)
        return fail(c, SG_ERR_DTYPE, "permutation contract needs two SG_I32 or two SG_F32 vectors");
      sg_status s = known_count(t);
      if (!s) s = known_count(o);
      if (s && s != SG_ERR_PRECONDITION && s != SG_ERR_POSTCONDITION) return s;
      if (o->v->n != t->v->n) return fail(c, SG_ERR_SHAPE, "permutation of a different count");
      if (!active) return SG_OK;
      n->nin = 2;
      use(n.get(), 0, t->v);
      use(n.get(), 1, o->v);
      break;
    }
    case SG_C_FREIVALDS: {
      if (k->nother != 2) return fail(c, SG_ERR_INVALID_ARG, "Freivalds needs A and B");
      sg_vector* a = static_cast<sg_vector*>(k->other[0]);
      sg_vector* b = static_cast<sg_vector*>(k->other[1]);
      const int64_t N = t->v->rows;
      if (t->v->cols != N || a->v->rows != N || a->v->cols != N || b->v->rows != N || b->v->cols != N)
        return fail(c, SG_ERR_SHAPE, "Freivalds check needs square matrices of one size");
      if (t->v->dt != SG_F32 || a->v->dt != SG_F32 || b->v->dt != SG_F32)
        return fail(c, SG_ERR_DTYPE, "Freivalds check needs SG_F32");
      if (!active) return SG_OK;
      n->nin = 3;
      n->seed = k->seed;
      n->nvec = k->nvec > 0 ? k->nvec : 4;
      if (n->nvec > 4) return fail(c, SG_ERR_INVALID_ARG, "Freivalds uses at most 4 vectors");
      n->tol = k->tol > 0 ? k->tol : 8.0;
      n->prec = SG_PREC_F32_SIMT;
      use(n.get(), 0, t->v);
      use(n.get(), 1, a->v);
      use(n.get(), 2, b->v);
      break;
    }
    case SG_C_UNCHANGED: {
      // Listing 3: Current = old Current, against the fingerprint sg_old took
      if (k->nother != 1) return fail(c, SG_ERR_INVALID_ARG, "unchanged needs other[0] from sg_old");
      sg_vector* o = static_cast<sg_vector*>(k->other[0]);
      if (o->v->dt != SG_I64 || o->v->n != 2)
        return fail(c, SG_ERR_INVALID_ARG, "other[0] must be the 2-element vector sg_old returns");
      sg_status s = known_count(t);
      if (s && s != SG_ERR_PRECONDITION && s != SG_ERR_POSTCONDITION) return s;
      if (!active) return SG_OK;
      n->nin = 2;
      use(n.get(), 0, t->v);
      use(n.get(), 1, o->v);
      break;
    }
    default:
      return fail(c, SG_ERR_INVALID_ARG, "contract kind %d not supported here", k->kind);
  }
  enqueue(c, std::move(n));
  return SG_OK;
}

sg_status sg_old(sg_ctx* c, void* target, sg_vector** old) {
  if (!c || !target || !old) return fail(c, SG_ERR_INVALID_ARG, "bad sg_old arguments");
  sg_vector* t = static_cast<sg_vector*>(target);
  if (check_vec(t) || t->ctx != c) return fail(c, SG_ERR_INVALID_ARG, "bad sg_old target");
  sg_status s = known_count(t);
  if (s && s != SG_ERR_PRECONDITION && s != SG_ERR_POSTCONDITION) return s;
  if (t->v->poisoned) return fail(c, SG_ERR_POISONED, "sg_old of a value that failed a contract");
  NodeP n = new_node(c, NK::SNAPSHOT);
  n->nin = 1;
  use(n.get(), 0, t->v);
  make_out(c, SG_I64, 2, 2, 1, &n->out);
  sg_vector* h = new_handle(c, n->out, false);
  enqueue(c, std::move(n));
  *old = h;
  return SG_OK;
}

sg_status sg_require(sg_ctx* c, void* target, const sg_contract* k, int32_t* id) {
  return attach(c, target, k, id, SG_PRE);
}

sg_status sg_ensure(sg_ctx* c, void* target, const sg_contract* k, int32_t* id) {
  return attach(c, target, k, id, SG_POST);
}

sg_status sg_last_violation(sg_ctx* c, sg_violation* out) {
  if (!c || !out) return SG_ERR_INVALID_ARG;
  if (!c->has_violation) return SG_ERR_INVALID_ARG;
  *out = c->last_violation;
  return SG_OK;
}

// ---------------------------------------------------------------------------
// execution and settings

sg_status sg_flush(sg_ctx* c) {
  if (!c) return SG_ERR_INVALID_ARG;
  if (c->pending.empty()) return SG_OK;
  if (c->planning_only) return fail(c, SG_ERR_UNSUPPORTED, "planning-only context cannot execute");
  join_downloads_of_pending(c);
  return sg_execute_pending(c);
}

sg_status sg_set_contract_mode(sg_ctx* c, sg_contract_mode m) {
  if (!c || m < SG_CONTRACTS_OFF || m > SG_CONTRACTS_FULL) return SG_ERR_INVALID_ARG;
  c->mode = m;
  return SG_OK;
}

sg_status sg_set_fusion(sg_ctx* c, sg_fusion f) {
  if (!c || (f != SG_FUSE_OFF && f != SG_FUSE_ON)) return SG_ERR_INVALID_ARG;
  c->fusion = f;
  return SG_OK;
}

sg_status sg_set_codegen(sg_ctx* c, sg_codegen g) {
  if (!c || (g != SG_CODEGEN_INTERPRET && g != SG_CODEGEN_SPECIALIZE)) return SG_ERR_INVALID_ARG;
  if (g == SG_CODEGEN_SPECIALIZE && !sgk::jit_available()) {
    c->codegen = SG_CODEGEN_INTERPRET;
    return fail(c, SG_ERR_UNSUPPORTED, "NVRTC is not available; fused passes are interpreted");
  }
  c->codegen = g;
  return SG_OK;
}

sg_status sg_set_scheduler(sg_ctx* c, sg_sched s) {
  if (!c || (s != SG_SCHED_AUTOTUNE && s != SG_SCHED_LEARNED)) return SG_ERR_INVALID_ARG;
  c->sched = s;
  return SG_OK;
}

sg_status sg_plan_describe(sg_ctx* c, char* buf, size_t cap, size_t* len) {
  if (!c) return SG_ERR_INVALID_ARG;
  std::string d;
  sg_status s = sg_describe_pending(c, &d);
  if (s) return s;
  if (len) *len = d.size() + 1;
  if (buf && cap) {
    size_t m = std::min(cap - 1, d.size());
    memcpy(buf, d.data(), m);
    buf[m] = 0;
  }
  return SG_OK;
}

sg_status sg_debug_inject_sort(sg_ctx* c, sg_inject_mode mode, int64_t i, int64_t j) {
  if (!c || mode < SG_INJECT_NONE || mode > SG_INJECT_OVERWRITE || i < 0 ||
      (mode == SG_INJECT_SWAP && j < 0))
    return SG_ERR_INVALID_ARG;
  c->inject.mode = mode;
  c->inject.i = i;
  c->inject.j = j;
  return SG_OK;
}

sg_status sg_debug_lookback(sg_ctx* c, uint32_t spin_limit, int64_t skip_tile) {
  if (!c || skip_tile < -1 || skip_tile > INT32_MAX) return SG_ERR_INVALID_ARG;
  c->lookback.spin_limit = spin_limit;
  c->lookback.skip_tile = (int)skip_tile;
  return SG_OK;
}

sg_status sg_debug_inject_matmul(sg_ctx* c, int64_t row, int64_t col, float delta) {
  if (!c || row < -1 || col < -1 || (row < 0) != (col < 0) || row > INT32_MAX || col > INT32_MAX)
    return SG_ERR_INVALID_ARG;
  c->mm_inject.row = row;
  c->mm_inject.col = col;
  c->mm_inject.delta = delta;
  return SG_OK;
}

sg_status sg_debug_portable_kernels(sg_ctx* c, int on) {
  if (!c) return SG_ERR_INVALID_ARG;
  sgk::set_portable_kernels(on != 0);
  c->lu.clear();
  return SG_OK;
}

sg_status sg_kernel_count(sg_ctx* c, int64_t* count) {
  if (!c || !count) return SG_ERR_INVALID_ARG;
  *count = c->kernels;
  return SG_OK;
}

}  // extern "C"

namespace sgk {

static sg_status expr_error(char* msg, size_t cap, const char* fmt, ...)
    __attribute__((format(printf, 3, 4)));

static sg_status expr_error(char* msg, size_t cap, const char* fmt, ...) {
  if (msg && cap) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, cap, fmt, ap);
    va_end(ap);
  }
  return SG_ERR_INVALID_ARG;
}

sg_status validate_expr(const sg_expr* f, int nin, int* max_depth, uint8_t* depth_before,
                        char* msg, size_t cap) {
  if (!f) return expr_error(msg, cap, "null expression");
  if (f->nops <= 0 || f->nops > SG_MAX_EXPR_OPS)
    return expr_error(msg, cap, "expression has %d ops (1..%d allowed)", f->nops,
                      SG_MAX_EXPR_OPS);
  int d = 0, mx = 0;
  for (int p = 0; p < f->nops; ++p) {
    const sg_expr_op& o = f->ops[p];
    int need = 0, delta = 0;
    switch (o.op) {
      case SG_OP_LOAD:
        if (o.arg < 0 || o.arg >= nin)
          return expr_error(msg, cap, "op %d loads slot %d of %d", p, o.arg, nin);
        delta = 1;
        break;
      case SG_OP_CONST: case SG_OP_INDEX: delta = 1; break;
      case SG_OP_ADD: case SG_OP_SUB: case SG_OP_MUL: case SG_OP_DIV: case SG_OP_MIN:
      case SG_OP_MAX: case SG_OP_LT: case SG_OP_LE: case SG_OP_GT: case SG_OP_GE:
      case SG_OP_EQ: case SG_OP_NE: case SG_OP_AND: case SG_OP_OR:
        need = 2; delta = -1; break;
      case SG_OP_FMA: case SG_OP_SELECT: need = 3; delta = -2; break;
      case SG_OP_NEG: case SG_OP_ABS: case SG_OP_SQRT: case SG_OP_NOT: need = 1; break;
      case SG_OP_DUP: need = 1; delta = 1; break;
      case SG_OP_SWAP: need = 2; break;
      default:
        return expr_error(msg, cap, "op %d has unknown opcode %d", p, o.op);
    }
    if (d < need)
      return expr_error(msg, cap, "op %d needs %d operands, stack has %d", p, need, d);
    if (depth_before) depth_before[p] = (uint8_t)d;
    d += delta;
    mx = std::max(mx, d);
    if (mx > SG_MAX_EXPR_DEPTH)
      return expr_error(msg, cap, "expression stack deeper than %d", SG_MAX_EXPR_DEPTH);
  }
  if (d != 1) return expr_error(msg, cap, "expression leaves %d values (must be 1)", d);
  if (max_depth) *max_depth = mx;
  return SG_OK;
}

}  // namespace sgk
