/*
 * safegpu.h -- C ABI of the GB300 (sm_103a) SafeGPU library.
 *
 * The library implements the data-parallel collection operations and the
 * on-device design-by-contract checks of Kolesnichenko, Poskitt, Nanz, Meyer,
 * "Contract-Based General-Purpose GPU Programming" (SafeGPU):
 *   - collections, vectors and matrices held in device memory (Sec. 3.1-3.4,
 *     Table 1 CUDA_DATA_HANDLE, Table 2 collection API);
 *   - deferred execution: calls are queued and run at a trigger -- a scalar
 *     query, a read back to the host, or an explicit flush (Sec. 5, the
 *     three triggers) -- after an optimizer merges the queued calls into
 *     fewer kernels (Sec. 5, Fig. 2 map+reduce merge, Fig. 3 expression
 *     rewrite);
 *   - pre- and postconditions evaluated on the GPU, scalar ones on the host
 *     and range ones (for_all, exists, is_sorted, ...) on the device
 *     (Sec. 4; contract modes of Sec. 6.3).
 *
 * Conventions for every call:
 *   - Every function returns an sg_status; results come back through
 *     out-parameters, which are written only on SG_OK.
 *   - Sizes and indices are int64_t.  Vectors are contiguous 1-D arrays;
 *     matrices are row-major (Sec. 3.4: "a single-dimensional array with
 *     row-wise alignment").
 *   - Handles returned through an out-parameter are owned by the caller, who
 *     releases them with the matching *_release call.  Releasing a handle
 *     whose value is still pending is allowed: the queued work keeps what it
 *     needs alive, and an unread intermediate whose handle was released is
 *     never materialised when the optimizer can fuse it away.
 *   - Device pointers passed to *_wrap are borrowed: the caller keeps the
 *     memory alive and unmodified until the next sg_flush returns.
 *   - Shape and dtype errors (the paper's scalar contracts) are detected on
 *     the host at the call and nothing is queued.  Range contracts are
 *     evaluated on the device at the flush: the flush then returns
 *     SG_ERR_PRECONDITION / SG_ERR_POSTCONDITION, the checked value and its
 *     dependants are poisoned (reading them returns SG_ERR_POISONED) and
 *     sg_last_violation() reports the first (smallest) violating index.
 *   - No call falls back to the CPU.  A context needs a CUDA device; the one
 *     exception is a planning-only context (device = -1), on which handles
 *     carry shapes only and sg_plan_describe() shows what a flush would
 *     launch.
 *   - All work of a context runs in order on the stream given to sg_init.
 *     A context is not thread-safe; use one per host thread.
 */
#ifndef SAFEGPU_H
#define SAFEGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SG_ABI_VERSION 1

typedef enum {
  SG_OK = 0,
  SG_ERR_INVALID_ARG = 1,   /* null handle, bad enum, malformed expression   */
  SG_ERR_SHAPE = 2,         /* count / rows / columns mismatch (scalar contract) */
  SG_ERR_DTYPE = 3,         /* element type not supported by the operation   */
  SG_ERR_OOM = 4,           /* device allocation failed                      */
  SG_ERR_CUDA = 5,          /* a CUDA runtime call failed                    */
  SG_ERR_PRECONDITION = 6,  /* a `require` range contract failed on device   */
  SG_ERR_POSTCONDITION = 7, /* an `ensure` range contract failed on device   */
  SG_ERR_TIMEOUT = 8,       /* a bounded device-side wait gave up            */
  SG_ERR_NOT_CONVERGED = 9, /* iterative refinement hit its iteration limit  */
  SG_ERR_POISONED = 10,     /* value depends on a failed contract            */
  SG_ERR_UNSUPPORTED = 11,  /* e.g. compute on a planning-only context       */
  SG_ERR_SINGULAR = 12      /* exactly zero pivot in elimination             */
} sg_status;

typedef enum {
  SG_F32 = 0, SG_F64 = 1, SG_BF16 = 2, SG_F16 = 3, SG_I32 = 4, SG_I64 = 5
} sg_dtype;

typedef struct sg_ctx sg_ctx;
typedef struct sg_vector sg_vector;   /* collection / vector (Sec. 3.2-3.3) */
typedef struct sg_matrix sg_matrix;   /* row-major matrix (Sec. 3.4)        */
typedef struct sg_scalar sg_scalar;   /* deferred scalar result             */

/* ------------------------------------------------------------------------ */
/* Expressions: the agents of Sec. 3.2 (functions and predicates applied to
 * every element).  A postfix program over a stack of IEEE binary32 values,
 * evaluated per element index i.  Booleans are 1.0f / 0.0f and a value is
 * true when it compares unequal to 0.0f (NaN is true).  Every operation is
 * one IEEE operation rounded to nearest-even; nothing is contracted into an
 * FMA unless SG_OP_FMA says so.  At most SG_MAX_EXPR_OPS ops and a stack
 * depth of at most SG_MAX_EXPR_DEPTH.                                       */

#define SG_MAX_EXPR_OPS 24
#define SG_MAX_EXPR_DEPTH 6

typedef enum {
  SG_OP_LOAD = 1,   /* arg = input slot k: push in_k[i]                   */
  SG_OP_CONST,      /* push `value`                                       */
  SG_OP_ADD, SG_OP_SUB, SG_OP_MUL, SG_OP_DIV,   /* pop b, a; push a op b  */
  SG_OP_FMA,        /* pop c, b, a; push a*b+c with one rounding          */
  SG_OP_MIN, SG_OP_MAX, /* NaN if either is NaN, else a<b?a:b / a>b?a:b   */
  SG_OP_NEG, SG_OP_ABS, SG_OP_SQRT,
  SG_OP_LT, SG_OP_LE, SG_OP_GT, SG_OP_GE, SG_OP_EQ, SG_OP_NE,
  SG_OP_AND, SG_OP_OR, SG_OP_NOT,
  SG_OP_SELECT,     /* pop f, t, c; push c ? t : f                        */
  SG_OP_DUP, SG_OP_SWAP,
  SG_OP_INDEX       /* push (float)i                                      */
} sg_opcode;

typedef struct {
  int32_t op;      /* sg_opcode                      */
  int32_t arg;     /* input slot for SG_OP_LOAD      */
  float value;     /* constant for SG_OP_CONST       */
} sg_expr_op;

typedef struct {
  int32_t nops;
  sg_expr_op ops[SG_MAX_EXPR_OPS];
} sg_expr;

/* ------------------------------------------------------------------------ */
/* Context (Table 1, CUDA_INTEROP: initialisation and device handling).
 * device  : CUDA ordinal, or -1 for a planning-only context (no GPU needed).
 * stream  : a cudaStream_t (as void*), or NULL for the legacy default stream.
 *           All kernels and copies of this context are issued on it.
 * Errors  : SG_ERR_INVALID_ARG (out is NULL), SG_ERR_CUDA (no such device). */
sg_status sg_init(int device, void* stream, sg_ctx** out);
/* Waits for the stream, frees every device allocation the context made.
 * Handles still alive become invalid. */
sg_status sg_destroy(sg_ctx* ctx);
/* Message of the last error on this context (static storage until the next
 * call on it). */
const char* sg_last_error(sg_ctx* ctx);
const char* sg_status_name(sg_status s);

/* ------------------------------------------------------------------------ */
/* Vectors (Table 2: from_array, count, item; Table 1 CUDA_DATA_HANDLE).      */

/* from_array: allocates n elements on the device (owned by the handle) and,
 * when host is not NULL, copies n elements from host memory (one memcpy,
 * Sec. 3.2).  host == NULL leaves the contents undefined. */
sg_status sg_vector_create(sg_ctx* ctx, sg_dtype dt, int64_t n,
                           const void* host, sg_vector** out);
/* Borrows n elements at dev_ptr (e.g. a torch tensor's storage). */
sg_status sg_vector_wrap(sg_ctx* ctx, sg_dtype dt, int64_t n, void* dev_ptr,
                         sg_vector** out);
/* to_array: flushes the work the vector depends on (trigger 2 of Sec. 5),
 * then copies n == count elements into host memory and waits for them.
 * SG_ERR_POISONED if the value depends on a failed contract. */
sg_status sg_vector_read(sg_vector* v, void* host, int64_t n);

/* Asynchronous forms of create and read, for pipelines of many steps (Sec. 3.1:
 * the data is copied to the device when the collection is created and back
 * when it is read).  Both return without waiting:
 *   sg_vector_create_async copies `host` (n elements) on a separate upload
 *     stream; the first work on the context's stream that uses the vector
 *     waits for the copy (other work does not, so the copy of the next
 *     step's input can overlap this step's compute).  `host` must stay
 *     valid and unchanged until the copy completes
 *     (sg_sync, or any later call that waits, such as a flush that reads
 *     back contract results).  Pinned (page-locked) host memory gives the
 *     full link bandwidth.
 *   sg_vector_read_async flushes the value's pending work first (like
 *     sg_vector_read: precondition / postcondition failures are reported
 *     there) and then enqueues its copy into `host` on a separate download
 *     stream, after everything enqueued so far on the context's stream.
 *     `host` holds the data only after sg_sync.  Later work that touches the
 *     value waits for the copy; a value released right away is freed behind it.
 * So one step's read can overlap the next step's create and compute.
 *   sg_sync waits for every copy and kernel the context has enqueued.
 * Values must be released before sg_destroy.  Errors as for the synchronous
 * forms; copy failures give SG_ERR_CUDA. */
sg_status sg_vector_create_async(sg_ctx* ctx, sg_dtype dtype, int64_t n, const void* host,
                                 sg_vector** out);
sg_status sg_vector_read_async(sg_vector* v, void* host, int64_t n);
sg_status sg_sync(sg_ctx* ctx);
/* count (Table 2): scalar query, no flush.  May be called on a pending
 * filter result only after a flush (its count is data-dependent); before
 * that it flushes. */
sg_status sg_vector_count(sg_vector* v, int64_t* n);
/* Device address of the vector's storage after flushing it (for interop).
 * Work the caller enqueues on the context's stream afterwards sees the
 * vector's asynchronous copies completed; on another stream, sg_sync first. */
sg_status sg_vector_device_ptr(sg_vector* v, void** dev_ptr);
sg_status sg_vector_release(sg_vector* v);
/* item (Table 2): element i (0-based) into *value (dtype-sized); flushes the
 * work the vector depends on.  SG_ERR_SHAPE for i outside [0, count),
 * SG_ERR_POISONED as sg_vector_read. */
sg_status sg_vector_item(sg_vector* v, int64_t i, void* value);
/* concatenate (Table 2): a new vector, a's elements then b's (same dtype),
 * deferred; counts must be known, so a pending filter operand is flushed
 * first (its count is data-dependent).  Errors: SG_ERR_DTYPE. */
sg_status sg_concat(sg_ctx* ctx, sg_vector* a, sg_vector* b, sg_vector** out);
/* subset (Table 2): elements [start, finish) of v (0-based, half-open) as a
 * vector that shares v's memory: writes through either are seen by both.
 * v is flushed first if pending.  Errors: SG_ERR_SHAPE unless
 * 0 <= start <= finish <= count. */
sg_status sg_subset(sg_ctx* ctx, sg_vector* v, int64_t start, int64_t finish,
                    sg_vector** out);

/* Matrices (Sec. 3.4): rows x cols, row-major, same ownership rules. */
sg_status sg_matrix_create(sg_ctx* ctx, sg_dtype dt, int64_t rows, int64_t cols,
                           const void* host, sg_matrix** out);
sg_status sg_matrix_wrap(sg_ctx* ctx, sg_dtype dt, int64_t rows, int64_t cols,
                         void* dev_ptr, sg_matrix** out);
sg_status sg_matrix_read(sg_matrix* m, void* host, int64_t count);
sg_status sg_matrix_shape(sg_matrix* m, int64_t* rows, int64_t* cols);
sg_status sg_matrix_device_ptr(sg_matrix* m, void** dev_ptr);
sg_status sg_matrix_release(sg_matrix* m);
/* A vector view of all rows*cols elements (the matrix stays valid). */
sg_status sg_matrix_as_vector(sg_matrix* m, sg_vector** out);

/* ------------------------------------------------------------------------ */
/* Collection operations (Table 2, Sec. 3.2-3.3).  All are deferred.
 * Element type: SG_F32.  Every input must have the same count (scalar
 * contract, else SG_ERR_SHAPE).                                             */

/* project (Table 2): out[i] = f(x[i]); input slot 0 = x.  New vector. */
sg_status sg_map(sg_ctx* ctx, const sg_expr* f, sg_vector* x, sg_vector** out);
/* Component-wise vector arithmetic (Sec. 3.3 plus/minus/compwise_*):
 * out[i] = f(x[i], y[i]); slots 0 = x, 1 = y. */
sg_status sg_zip(sg_ctx* ctx, const sg_expr* f, sg_vector* x, sg_vector* y,
                 sg_vector** out);
/* General n-ary form (1..4 inputs in slots 0..nin-1). */
sg_status sg_mapn(sg_ctx* ctx, const sg_expr* f, int nin, sg_vector* const* ins,
                  sg_vector** out);
/* for_each (Table 2): x[i] = f(x[i]) in place. */
sg_status sg_for_each(sg_ctx* ctx, const sg_expr* f, sg_vector* x);
/* filter (Table 2): a new vector of the x[i] for which pred(x[i]) holds, in
 * index order (stable).  Its count is known after the flush. */
sg_status sg_filter(sg_ctx* ctx, const sg_expr* pred, sg_vector* x,
                    sg_vector** out);

typedef enum {
  SG_REDUCE_SUM = 0,  /* binary64 value of the sum of the elements (an empty
                         sum is 0)                                          */
  SG_REDUCE_MIN = 1,  /* NaN if any element is NaN; count must be > 0       */
  SG_REDUCE_MAX = 2,
  SG_REDUCE_AVG = 3,  /* sum / count; count must be > 0                     */
  SG_REDUCE_COUNT = 4
} sg_reduce_op;

/* sum / avg / min / max (Sec. 3.3): a deferred scalar. */
sg_status sg_reduce(sg_ctx* ctx, sg_reduce_op op, sg_vector* x, sg_scalar** out);
/* for_all / exists (Table 2): deferred Boolean; pred over slots 0..nin-1
 * (slot 0 = x).  sg_scalar_index gives the first failing (for_all) or first
 * witnessing (exists) index, -1 if none. */
sg_status sg_for_all(sg_ctx* ctx, const sg_expr* pred, int nin,
                     sg_vector* const* ins, sg_scalar** out);
sg_status sg_exists(sg_ctx* ctx, const sg_expr* pred, int nin,
                    sg_vector* const* ins, sg_scalar** out);
/* Trigger 1 of Sec. 5: reading a scalar flushes what it depends on. */
sg_status sg_scalar_get(sg_scalar* s, double* value);
sg_status sg_scalar_index(sg_scalar* s, int64_t* index);
sg_status sg_scalar_release(sg_scalar* s);

/* ------------------------------------------------------------------------ */
/* Sorting (Listing 4: ascending, left < mid = right >).  Keys SG_I32 in
 * signed order, or SG_F32 (Listing 4 sorts REAL_32) in IEEE 754 totalOrder:
 * -NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN, equal bit patterns being
 * indistinguishable, so the output is unique.  With contract mode >=
 * SG_CONTRACTS_PRE_POST the built-in postconditions `Result.is_sorted` and
 * `Result is a permutation of keys` (Listing 4 `Result.count = a.count`,
 * strengthened to multiset equality of the bit patterns) are evaluated
 * inside the sort's last pass; there `is_sorted` is checked in the sort's
 * own order.  A stand-alone SG_C_SORTED contract on SG_F32 uses the IEEE
 * comparison (x[i] > x[i+1] is a violation; NaN never is).  n < 2^30. */
sg_status sg_sort(sg_ctx* ctx, sg_vector* keys, sg_vector** out);

/* ------------------------------------------------------------------------ */
/* Matrix product (Sec. 3.4 `multiply`): C = A B.  A: M x K, B: K x N, SG_F32
 * storage; C: M x N SG_F32.  `precision` selects binary32 SIMT arithmetic or
 * bf16 / fp16 operands (rounded to nearest even) on the tensor cores with
 * binary32 accumulation.  Built-in postcondition (mode >= PRE_POST):
 * Freivalds' check with 4 Rademacher vectors (see sg_contract). */
typedef enum {
  SG_PREC_F32_SIMT = 0,
  SG_PREC_BF16_TC = 1,
  SG_PREC_F16_TC = 2
} sg_precision;
sg_status sg_matmul(sg_ctx* ctx, sg_matrix* A, sg_matrix* B, sg_precision p,
                    sg_matrix** C);

/* Matrix `transpose` and the matrix-vector products `right_multiply` and
 * `left_multiply` of Sec. 3.4 (Listing 1 chains the first two).  SG_F32,
 * row-major; all three are deferred like the collection operations.
 *   sg_transpose: At = A^T (cols x rows, a new matrix owned by the caller).
 *   sg_matvec:    y = A x; A rows x cols, x of cols elements (Listing 1's
 *                 precondition: checked at the call, SG_ERR_SHAPE), y of rows.
 *   sg_vecmat:    y = x^T A; x of rows elements, y of cols.
 * Sums are binary32 (FMA per lane, then fixed-order trees and stripe sums):
 * |y_i - y*_i| <= (terms + 8) 2^-24 sum |a x| with terms = cols (matvec) or
 * rows (vecmat).  With fusion on, sg_matvec on the pending transpose of A
 * whose handle has been released reads A once as sg_vecmat does and never
 * materialises A^T.
 * Errors: SG_ERR_INVALID_ARG, SG_ERR_DTYPE, SG_ERR_SHAPE. */
sg_status sg_transpose(sg_ctx* ctx, sg_matrix* A, sg_matrix** At);
sg_status sg_matvec(sg_ctx* ctx, sg_matrix* A, sg_vector* x, sg_vector** y);
sg_status sg_vecmat(sg_ctx* ctx, sg_vector* x, sg_matrix* A, sg_vector** y);

/* ------------------------------------------------------------------------ */
/* Gaussian elimination (Sec. 5, Listing 6; read as elimination with partial
 * pivoting) and solve.  A: n x n SG_F32, b: n SG_F64; x: n SG_F64.
 * The factorisation runs with `precision` operands for the trailing update
 * (binary32 accumulation), then iterative refinement with the residual
 * r = b - A x in binary64 until max|d| <= refine_tol * max|x| or max_iter.
 * Built-in postcondition (mode >= PRE_POST): max|b - A x| /
 * (|A|_inf |x|_inf + |b|_inf) <= residual_tol, evaluated in binary64. */
typedef struct {
  sg_precision precision;  /* trailing-update operands                */
  int32_t max_iter;        /* refinement iterations (default 30)      */
  double refine_tol;       /* default 1e-14                           */
  double residual_tol;     /* default 1e-12                           */
  int32_t block;           /* panel width nb (0 = library choice)     */
} sg_solve_opts;

typedef struct {
  int32_t iterations;      /* refinement steps taken                  */
  int32_t info;            /* 0, or k+1 for an exactly zero pivot     */
  double residual;         /* final normwise backward error           */
  double last_correction;  /* max|d| / max|x| of the last step        */
} sg_solve_info;

sg_status sg_solve(sg_ctx* ctx, sg_matrix* A, sg_vector* b,
                   const sg_solve_opts* opts, sg_vector** x,
                   sg_solve_info* info);

/* The determinant (the intent of Listing 6, Sec. 5: elimination that returns
 * the product of the pivots), from the same elimination with partial
 * pivoting: det A = (-1)^(row interchanges) * prod_i u_ii.  A: n x n SG_F32
 * (n <= 9216), factored in a workspace copy with `precision` operands for
 * the trailing updates (SG_PREC_F32_SIMT keeps every update in binary32).
 * The log of |det| is summed in binary64, so it neither overflows nor
 * underflows; `det` = sign * exp(log_abs) may be +-inf or 0 in binary64.
 * An exactly singular A (a zero pivot) is not an error: sign = 0,
 * det = 0, log_abs = -inf, info = k+1 for the first zero pivot at step k.
 * Errors: SG_ERR_SHAPE (not square, n too large), SG_ERR_DTYPE,
 * SG_ERR_POISONED, SG_ERR_OOM, SG_ERR_CUDA. */
typedef struct {
  int32_t sign;        /* +1, -1, or 0 for an exactly singular A            */
  int32_t info;        /* 0, or k+1 for the first exactly zero pivot        */
  double log_abs;      /* natural log of |det A| (-inf when singular)       */
  double det;          /* sign * exp(log_abs) in binary64                   */
} sg_det_result;
sg_status sg_det(sg_ctx* ctx, sg_matrix* A, sg_precision precision, sg_det_result* out);

/* ------------------------------------------------------------------------ */
/* Contracts (Sec. 4).  sg_require attaches a precondition, sg_ensure a
 * postcondition, to the current (possibly pending) value of `target`.  They
 * are evaluated at the next flush, fused into the pass that produces the
 * target whenever possible.  Scalar parts (counts, shapes) are checked at
 * the call; a FOR_ALL or EXISTS with no other[] operand on a pending filter
 * result has none, so it does not flush the filter: it runs in the filter's
 * flush, over the count the filter finds (a FOR_ALL there is checked by the
 * run-time specialised filter itself, on each kept item as it is written,
 * when fusion is on), and its first index is a position in the result.
 * Returns an id in *contract_id (may be NULL) that sg_last_violation()
 * reports.                                                                  */
typedef enum {
  SG_C_FOR_ALL = 0,     /* expr over slots: 0 = target, 1.. = other[]   */
  SG_C_EXISTS = 1,
  SG_C_SORTED = 2,      /* target ascending; first i with t[i] > t[i+1]   */
  SG_C_PERMUTATION = 3, /* target is a permutation of other[0]            */
  SG_C_FREIVALDS = 4,   /* target C = other[0] (A) x other[1] (B), matrices */
  SG_C_RESIDUAL = 5,    /* target x solves other[0] (A) x = other[1] (b)    */
  SG_C_UNCHANGED = 6    /* target equals its value when other[0] was taken
                           by sg_old (Listing 3: Current = old Current)   */
} sg_contract_kind;

typedef struct {
  int32_t kind;          /* sg_contract_kind                              */
  sg_expr expr;          /* FOR_ALL / EXISTS predicate                    */
  int32_t nother;        /* number of entries used in other[]             */
  void* other[3];        /* sg_vector* (or sg_matrix* for FREIVALDS,
                            RESIDUAL's A)                                 */
  uint64_t seed;         /* FREIVALDS: Rademacher stream seed             */
  int32_t nvec;          /* FREIVALDS: number of vectors, 1..4 (0 = 4)    */
  double tol;            /* FREIVALDS: c in tau = c u sigma (default 8);
                            RESIDUAL: bound (default 1e-12)               */
} sg_contract;

sg_status sg_require(sg_ctx* ctx, void* target, const sg_contract* c,
                     int32_t* contract_id);

sg_status sg_ensure(sg_ctx* ctx, void* target, const sg_contract* c,
                    int32_t* contract_id);

/* Eiffel's `old` (Sec. 4, Listing 3's postcondition Current = old Current):
 * takes the state of `target` (a vector or a matrix) at this point of the
 * queue, kept as a position-dependent fingerprint -- two 64-bit sums of
 * mix64(i 2^32 + unit_i) over its 16-bit (bf16, fp16) or 32-bit units, mix64
 * being SplitMix64's output function -- instead of a copy: one read of the
 * target when the queue reaches it, 16 bytes kept.  *old is a new SG_I64
 * vector of 2 elements (owned by the caller) holding the fingerprint; pass
 * it as other[0] of an SG_C_UNCHANGED contract on the same target.  A
 * change of any single unit always changes the fingerprint (mix64 is a
 * bijection); several changes go unseen only if their sums cancel mod 2^64
 * in both sums.  Errors: SG_ERR_INVALID_ARG, SG_ERR_POISONED. */
sg_status sg_old(sg_ctx* ctx, void* target, sg_vector** old);

typedef enum { SG_PRE = 0, SG_POST = 1 } sg_contract_role;

typedef struct {
  int32_t contract_id;   /* id from sg_require / sg_ensure, or -1 for a
                            built-in contract of an operation             */
  int32_t role;          /* sg_contract_role                              */
  int32_t kind;          /* sg_contract_kind                              */
  int32_t op_id;         /* sequence number of the checked operation      */
  int64_t first_index;   /* smallest violating index (row for FREIVALDS), -1
                            when the contract has no index (PERMUTATION)  */
  double observed;       /* e.g. the residual or |z_i - w_i| / tau_i      */
} sg_violation;

/* The first violation found by the last flush; SG_ERR_INVALID_ARG if none. */
sg_status sg_last_violation(sg_ctx* ctx, sg_violation* out);

/* ------------------------------------------------------------------------ */
/* Execution (Sec. 5).                                                       */

/* update (Table 2): run every pending operation of the context, merged by
 * the optimizer, and wait for it.  Returns the first failure. */
sg_status sg_flush(sg_ctx* ctx);

typedef enum {
  SG_CONTRACTS_OFF = 0,
  SG_CONTRACTS_PRE = 1,       /* preconditions only        (Sec. 6.3 mode 1) */
  SG_CONTRACTS_PRE_POST = 2,  /* pre- and postconditions   (mode 2)          */
  SG_CONTRACTS_FULL = 3       /* plus handle invariants    (mode 3)          */
} sg_contract_mode;
sg_status sg_set_contract_mode(sg_ctx* ctx, sg_contract_mode m);

/* Fusion of queued calls (Sec. 5): SG_FUSE_ON merges map chains, map+reduce
 * and contract predicates into single passes; SG_FUSE_OFF launches one
 * kernel per queued call (the plain unfused schedule). */
typedef enum { SG_FUSE_OFF = 0, SG_FUSE_ON = 1 } sg_fusion;
sg_status sg_set_fusion(sg_ctx* ctx, sg_fusion f);

/* Schedule choice for launch and tile shapes (the families below): the
 * autotuned plain table, or the learned MLP cost model. */
typedef enum { SG_SCHED_AUTOTUNE = 0, SG_SCHED_LEARNED = 1 } sg_sched;
sg_status sg_set_scheduler(sg_ctx* ctx, sg_sched s);

/* Code generation for fused element-wise passes (Sec. 5 generates a kernel
 * per plan).  SG_CODEGEN_SPECIALIZE (default): the fused program (and a
 * filter's predicate) is compiled once per program structure into
 * straight-line code inside the streaming (or filter) kernel template
 * (NVRTC, sm_103a) and cached for the process; a program whose kernel does
 * not compile is interpreted instead.  SG_CODEGEN_INTERPRET: the
 * precompiled kernels evaluate the program.  Both give identical results.  SG_ERR_UNSUPPORTED if
 * specialisation was requested but NVRTC cannot be loaded (the context keeps
 * interpreting).  The environment variable SG_CODEGEN=interpret sets the
 * default of new contexts. */
typedef enum { SG_CODEGEN_INTERPRET = 0, SG_CODEGEN_SPECIALIZE = 1 } sg_codegen;
sg_status sg_set_codegen(sg_ctx* ctx, sg_codegen g);

/* Compiles, and only compiles, the run-time specialised filter kernel of
 * `pred` (a predicate over slot 0, as for sg_filter) in each of its tile
 * sizes (2048, 4096, 8192 items) with NVRTC for sm_103a; nothing is
 * loaded, so no GPU is needed.  SG_OK when it compiles;
 * SG_ERR_UNSUPPORTED when NVRTC cannot be loaded or the compile fails (the
 * reason or the compiler's log, truncated to cap - 1 bytes and terminated,
 * goes to `log` unless it is NULL); SG_ERR_INVALID_ARG for a malformed
 * predicate.  A predicate whose kernel does not compile still filters
 * correctly: sg_filter then uses the interpreting kernel. */
sg_status sg_debug_jit_check_filter(const sg_expr* pred, char* log, size_t cap);

/* The same compile check for the specialised filter that also evaluates a
 * for_all postcondition `post` (one input slot, as for sg_filter's
 * predicate; NULL: none) on each kept item as it writes it -- the form
 * sg_flush uses when a `Result.for_all` contract (sg_ensure) on a filter's
 * result of the same flush is folded into the filter (Sec. 4: contracts
 * checked on the device; no pass over the result).  Status and log as for
 * sg_debug_jit_check_filter; SG_ERR_UNSUPPORTED also when the two programs
 * together have more than 46 operations. */
sg_status sg_debug_jit_check_filter_post(const sg_expr* pred, const sg_expr* post, char* log,
                                         size_t cap);

/* Writes a one-line-per-kernel description of what sg_flush would launch
 * for the currently queued work (no execution; works on a planning-only
 * context).  *len receives the length needed, including the terminator. */
sg_status sg_plan_describe(sg_ctx* ctx, char* buf, size_t cap, size_t* len);

/* Number of kernels this context has launched so far. */
sg_status sg_kernel_count(sg_ctx* ctx, int64_t* count);

/* Tracing.  With `on` != 0 every kernel this context launches is bracketed
 * by two CUDA events recorded on its stream (a few microseconds per launch;
 * off by default).  sg_profile_report writes one line per kernel name,
 * "name launches total_ms", accumulated since the last reset (reset != 0
 * clears the totals after writing); *len receives the size needed. */
sg_status sg_profile_enable(sg_ctx* ctx, int on);
sg_status sg_profile_report(sg_ctx* ctx, char* buf, size_t cap, size_t* len,
                            int reset);

/* Contract testing (Sec. 4 contracts must be seen to fire): plant a fault
 * in the NEXT sort of this context, on the host side, between its third and
 * its last pass: the host copies into the intermediate buffer (which holds
 * the keys ordered by their low 24 bits) either
 *   SG_INJECT_SWAP:      positions i and j exchanged, or
 *   SG_INJECT_OVERWRITE: position i set to the int32 value j.
 * Nothing is planted on the device side; the fused postconditions of the
 * last pass then report what they see.  mode SG_INJECT_NONE cancels.
 * Errors: SG_ERR_INVALID_ARG for a bad mode or negative index. */
typedef enum { SG_INJECT_NONE = 0, SG_INJECT_SWAP = 1, SG_INJECT_OVERWRITE = 2 } sg_inject_mode;
sg_status sg_debug_inject_sort(sg_ctx* ctx, sg_inject_mode mode, int64_t i, int64_t j);

/* Failure-detection testing of the bounded waits (no counterpart in the
 * paper; its kernels have no inter-block waits).  The sort passes and the
 * filter find their tiles' output offsets by a decoupled look-back: a tile
 * waits for words that earlier tiles publish, and every wait gives up after
 * a bounded number of polls, marks the flush SG_ERR_TIMEOUT and leaves the
 * context usable.  For the sorts and filters of this context's later
 * flushes: spin_limit bounds each wait (0 restores the default of 2^22
 * polls), and skip_tile >= 0 makes that tile of every look-back pass publish
 * nothing, so that the tiles after it wait until the limit (the planted
 * fault is on the host side: a kernel argument).  (0, -1) switches both off.
 * A timed-out pass writes nothing at unknown offsets and later passes of
 * the same sort do nothing; the outputs of the flush are undefined.
 * Errors: SG_ERR_INVALID_ARG for skip_tile < -1 or > INT32_MAX. */
sg_status sg_debug_lookback(sg_ctx* ctx, uint32_t spin_limit, int64_t skip_tile);

/* Contract testing of `multiply` (Sec. 3.4): plant an error in the NEXT
 * tensor-core product (SG_PREC_BF16_TC / SG_PREC_F16_TC) of this context:
 * `delta` is added to element (row, col) of the product as the kernel's
 * epilogue stores it, so every later reader -- the Freivalds
 * postcondition, fused into the product or not -- sees the wrong value.
 * The planted value is a kernel argument; nothing faults.  row = col = -1
 * cancels; an index outside the product plants nothing.  Binary32 products
 * ignore it.  Errors: SG_ERR_INVALID_ARG for indices below -1, one of them
 * negative, or above INT32_MAX. */
sg_status sg_debug_inject_matmul(sg_ctx* ctx, int64_t row, int64_t col, float delta);

/* Testing aid for the portable kernel forms.  On devices that schedule them,
 * tensor-core products run on CTA pairs (clusters of two, tcgen05
 * cta_group::2) and the elimination's panel on a 16-CTA cluster; the
 * one-CTA product and the 8-CTA panel remain for devices that do not.
 * on != 0 makes every later product and factorisation in this PROCESS use
 * the portable forms (so that they can be tested where the fast ones run);
 * 0 restores the choice by the device.  Clears this context's cached
 * factorisation graph.  Results of both forms are equal up to rounding
 * order.  Errors: SG_ERR_INVALID_ARG for a null context. */
sg_status sg_debug_portable_kernels(sg_ctx* ctx, int on);

/* ------------------------------------------------------------------------ */
/* Batched collections: one persistent launch over many collections of uneven
 * size, each running the chain
 *     y = map(x);  require for_all(pre(y));  s = sum(filter(y, keep))
 * (Sec. 3.2-3.3 operations per collection; the filter output is consumed only
 * by the sum, so it is never materialised).  Captured once into a CUDA graph
 * per (context, chain, nseg) and replayed.  Device pointers, caller-owned:
 *   data     : concatenated SG_F32 elements
 *   offsets  : nseg+1 int64, offsets[0] = 0, non-decreasing
 *   sums     : nseg binary64 sums of the kept y
 *   first_viol: nseg int64, first index (within the collection) where pre
 *               fails, -1 if none
 *   kept     : nseg int64 counts of kept elements
 * Returns SG_ERR_PRECONDITION if any collection violated `pre` (outputs are
 * still written).  In contract mode SG_CONTRACTS_OFF the precondition is not
 * evaluated (it is not compiled into the pass) and every first_viol is -1. */
typedef struct {
  sg_expr map;
  sg_expr pre;
  sg_expr keep;
} sg_chain;

sg_status sg_batch_run(sg_ctx* ctx, const sg_chain* chain, const float* data,
                       const int64_t* offsets, int64_t nseg, double* sums,
                       int64_t* first_viol, int64_t* kept);

/* ------------------------------------------------------------------------ */
/* Schedule choice.  A decision family is a point where the library picks a
 * launch or tile shape from a candidate list; a schedule is one candidate,
 * given as (chunk, ctas_per_sm):
 *   SG_SCHED_BATCH    the batched launch (sg_batch_run): chunk = elements
 *                     per work item, ctas_per_sm = persistent CTAs per SM;
 *                     plain table (16384, 8)
 *   SG_SCHED_STREAM   a fused element-wise pass (Sec. 5's generated kernel,
 *                     specialised code): chunk = threads per CTA (64, 128,
 *                     256), ctas_per_sm = CTAs per SM of the grid-stride
 *                     grid (1, 2, 4, 8; the grid never exceeds one float4
 *                     per thread); plain table (256, 8)
 *   SG_SCHED_FILTER   the specialised filter (Table 2): chunk = items per
 *                     tile (2048, 4096, 8192), ctas_per_sm = 0; plain
 *                     table 8192
 *   SG_SCHED_PRODUCT  the tensor-core product (Sec. 3.4 multiply, sg_matmul
 *                     in bf16 / fp16): chunk = tile rows, ctas_per_sm =
 *                     CTAs per tile (256, 2: a CTA pair; 128, 1: one CTA);
 *                     plain table the pair (on devices that schedule pairs)
 *   SG_SCHED_FUSION   the fusion boundaries of a flush whose work is only
 *                     element-wise passes (maps, zips, reductions, for_all /
 *                     exists and range contracts, no call writing in place)
 *                     and whose fused and unfused plans differ: chunk = the
 *                     candidate plan's kernels, ctas_per_sm = 1 for the
 *                     fused plan (Sec. 5's merges), 0 for one kernel per
 *                     queued call; plain table the fused plan.  Under
 *                     SG_FUSE_OFF nothing is decided.  The autotuner takes
 *                     the unfused plan only when it measured more than 3%
 *                     faster
 * SG_SCHED_AUTOTUNE measures every candidate the first time a workload is
 * seen -- a warm-up run, then the better of two runs timed with CUDA
 * events -- and keeps the fastest (the batch: per offsets pointer, count
 * and chain; a stream pass: per length, program shape and alignment; the
 * filter: per length and predicate shape; the product: per M, N, K and
 * precision; the fusion boundaries: per shape of the queued calls, timing
 * each plan's kernels over the whole flush).  A stream pass that writes over one of its inputs is not
 * re-run: it takes the plain table's choice.  Each measurement is logged
 * as (family, 12 features, log microseconds, log of the time relative to
 * the plain table's choice on that workload).  sg_sched_train fits one 2x64
 * MLP cost model per family to the relative log-times on the GPU with the
 * kernels below.  SG_SCHED_LEARNED then runs, without measuring, the
 * candidate the family's model predicts fastest when it is predicted to
 * beat the plain table's choice by more than 2%, else that choice (a family
 * with no trained model behaves as under SG_SCHED_AUTOTUNE).  In a report,
 * predicted_us is the model's relative prediction times the plain choice's
 * measured time (0 where nothing was measured).                          */
typedef enum {
  SG_SCHED_BATCH = 0,
  SG_SCHED_STREAM = 1,
  SG_SCHED_FILTER = 2,
  SG_SCHED_PRODUCT = 3,
  SG_SCHED_FUSION = 4
} sg_sched_family;
#define SG_SCHED_MAX_CANDIDATES 32
typedef struct {
  int32_t ncand;          /* candidates                                        */
  int32_t best_index;     /* fastest measured (the autotuner's choice), -1 when
                             nothing was measured                              */
  int32_t default_index;  /* the plain table's choice                          */
  int32_t learned_index;  /* the model's choice, -1 when no model is trained
                             (for an autotuned choice: when it was measured)  */
  int64_t chunk[SG_SCHED_MAX_CANDIDATES];
  int32_t ctas_per_sm[SG_SCHED_MAX_CANDIDATES];
  double measured_us[SG_SCHED_MAX_CANDIDATES];   /* 0: not measured         */
  double predicted_us[SG_SCHED_MAX_CANDIDATES];
  int32_t family;         /* sg_sched_family                                   */
  int32_t chosen_index;   /* the candidate that ran                            */
} sg_sched_report;

/* Runs the batch once under every candidate schedule (the outputs hold the
 * last run's results) and reports the measured times, the plain table's,
 * the autotuner's and the learned model's choices.  For regret studies. */
sg_status sg_batch_report(sg_ctx* ctx, const sg_chain* chain, const float* data,
                          const int64_t* offsets, int64_t nseg, double* sums,
                          int64_t* first_viol, int64_t* kept, sg_sched_report* out);
/* Trains the cost models on the context's log: every family with at least 8
 * sweep records gets its own model (SG_ERR_INVALID_ARG when none has),
 * features and targets standardised per family, minibatches of up to 512,
 * Adam(lr), `epochs` passes, initial weights from `seed`.  *final_loss:
 * mean squared error on the standardised log-time over the trained
 * families' records. */
sg_status sg_sched_train(sg_ctx* ctx, int32_t epochs, float lr, uint64_t seed,
                         float* final_loss);
/* The log: records x 12 features, log microseconds, and (family may be
 * NULL) each record's sg_sched_family; host buffers of the caller. */
sg_status sg_sched_log_size(sg_ctx* ctx, int64_t* records, int32_t* features);
sg_status sg_sched_log_read(sg_ctx* ctx, float* features, float* log_us,
                            int32_t* family, int64_t records);
/* The last decision the context took in `family` (its candidates, the
 * measured times of a sweep, the plain, autotuned, learned and chosen
 * indices).  SG_ERR_INVALID_ARG when that family has decided nothing yet. */
sg_status sg_sched_last(sg_ctx* ctx, int32_t family, sg_sched_report* out);
/* Drops the autotuned choices of `family` (-1: of every family), so that the
 * next workload of each kind is measured again (after a change of
 * conditions: another process on the device, other clocks).  The log and
 * the models are kept. */
sg_status sg_sched_forget(sg_ctx* ctx, int32_t family);
/* Testing aid: every later decision of `family` takes candidate `index` (in
 * the order sg_sched_last lists them) when the workload has that many
 * candidates, without measuring or predicting; -1 restores the scheduler.
 * Lets a test check each candidate's results. */
sg_status sg_sched_force(sg_ctx* ctx, int32_t family, int32_t index);

/* The cost model's network on caller device buffers (binary32), stream of
 * ctx: yhat = W3 relu(W2 relu(W1 x + b1) + b2) + b3, hidden width 64, flat
 * parameters [W1 (64 x d_in), b1, W2 (64 x 64), b2, W3 (64), b3];
 * loss = mean (yhat - y)^2, gradient in the same layout; Adam with bias
 * correction at step `step` (1-based).  X is B x d_in row-major, 1 <= d_in
 * <= 32.  The calls wait for the stream. */
sg_status sg_mlp_forward(sg_ctx* ctx, const float* params, int32_t d_in,
                         const float* X, int64_t B, float* yhat);
sg_status sg_mlp_loss_grad(sg_ctx* ctx, const float* params, int32_t d_in,
                           const float* X, const float* y, int64_t B,
                           float* grad, float* loss);
sg_status sg_mlp_adam(sg_ctx* ctx, float* params, const float* grad, float* m,
                      float* v, int64_t nparams, int64_t step, float lr,
                      float beta1, float beta2, float eps);

/* ------------------------------------------------------------------------ */
/* Allocation-free filter (the paper has no counterpart).  Some callers
 * cannot allocate device memory: a serving runtime that reserves all of HBM
 * in its own pool at start-up and forbids later allocations, a
 * latency-critical path that cannot afford the device-wide synchronisation
 * an allocation may imply, a plugin host that only hands out the input and
 * output buffers.  This call runs the filter of sg_filter on caller-owned
 * device buffers, needs no context, and keeps its scratch (the look-back
 * words of the stream compaction) in one fixed array of
 * SG_FILTER_NOALLOC_SCRATCH_BYTES (about 513 KB) in the library's device
 * memory, which every GPU that loads the library holds until the process
 * exits.  It calls no cudaMalloc, cudaFree or other allocating routine.
 *   pred      : predicate over slot 0, as for sg_filter
 *   dev_x     : n binary32 inputs (device memory)
 *   dev_out   : room for n binary32 outputs (device memory); the kept items,
 *               in index order, are written to its start
 *   dev_count : one int64 in device memory, receives the number kept
 *   stream    : a cudaStream_t, or NULL for the legacy default stream; the
 *               call waits for the stream before it returns
 * Errors: n > SG_FILTER_NOALLOC_MAX_N (2^28) gives SG_ERR_SHAPE; a malformed
 * predicate or a null buffer SG_ERR_INVALID_ARG; a look-back wait that gave
 * up SG_ERR_TIMEOUT, with *dev_count set to -1 (the kept items written so far
 * are not a result); a CUDA failure SG_ERR_CUDA.
 * Every call waits for its stream (it reads the look-back's timeout flag
 * back), so no call can be captured in a CUDA graph.  The first call on each
 * device looks up the array's device address, with that device current.
 * Loading is the one exception to "allocates nothing": under CUDA's default
 * lazy module loading, that first call loads the library's device code on
 * the device, and the loader then takes the array's 513 KB (and the code's
 * own memory) from the device; the first call with a predicate whose stack
 * is deeper than 4 loads a second kernel the same way.  A caller that is
 * about to reserve all of HBM should make one call with a shallow and one
 * with a deep predicate first (or run with CUDA_MODULE_LOADING=EAGER, which
 * loads everything when the process starts); after that no call takes
 * device memory.
 * All calls on a device share the one array, which keeps the last call's
 * contents (each call clears what it needs first): calls whose GPU work
 * overlaps -- from several host threads or streams -- race on it, so the
 * caller must serialise them. */
#define SG_FILTER_NOALLOC_MAX_N (1LL << 28)
#define SG_FILTER_NOALLOC_SCRATCH_BYTES \
  (768 + ((SG_FILTER_NOALLOC_MAX_N + 4095) / 4096) * 8)
sg_status sg_filter_noalloc(const sg_expr* pred, const float* dev_x, int64_t n,
                            float* dev_out, int64_t* dev_count, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SAFEGPU_H */
