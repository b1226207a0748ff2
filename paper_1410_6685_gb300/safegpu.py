"""Thin Python binding of the C ABI in include/safegpu.h (ctypes).

Names follow the C functions one to one; this module only marshals
arguments (expressions given as tuples, torch tensors wrapped by address)
and turns a non-OK sg_status into SgError.  Every operation runs in the CUDA
library libsafegpu.so: if the library is missing the import fails -- there is
no CPU fallback.

Expressions are postfix tuples, e.g. ``[("x", 0), ("x", 1), ("add",)]``;
``("x", k)`` loads input slot k, ``("c", v)`` pushes a binary32 constant.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsafegpu.so")

# ---- enums (values from include/safegpu.h) -----------------------------------
SG_OK = 0
STATUS = ["SG_OK", "SG_ERR_INVALID_ARG", "SG_ERR_SHAPE", "SG_ERR_DTYPE", "SG_ERR_OOM",
          "SG_ERR_CUDA", "SG_ERR_PRECONDITION", "SG_ERR_POSTCONDITION", "SG_ERR_TIMEOUT",
          "SG_ERR_NOT_CONVERGED", "SG_ERR_POISONED", "SG_ERR_UNSUPPORTED", "SG_ERR_SINGULAR"]
for _i, _n in enumerate(STATUS):
    globals()[_n] = _i

SG_F32, SG_F64, SG_BF16, SG_F16, SG_I32, SG_I64 = range(6)
SG_REDUCE_SUM, SG_REDUCE_MIN, SG_REDUCE_MAX, SG_REDUCE_AVG, SG_REDUCE_COUNT = range(5)
SG_PREC_F32_SIMT, SG_PREC_BF16_TC, SG_PREC_F16_TC = range(3)
(SG_C_FOR_ALL, SG_C_EXISTS, SG_C_SORTED, SG_C_PERMUTATION, SG_C_FREIVALDS, SG_C_RESIDUAL,
 SG_C_UNCHANGED) = range(7)
SG_PRE, SG_POST = 0, 1
SG_CONTRACTS_OFF, SG_CONTRACTS_PRE, SG_CONTRACTS_PRE_POST, SG_CONTRACTS_FULL = range(4)
SG_FUSE_OFF, SG_FUSE_ON = 0, 1
SG_SCHED_AUTOTUNE, SG_SCHED_LEARNED = 0, 1
SG_SCHED_BATCH, SG_SCHED_STREAM, SG_SCHED_FILTER, SG_SCHED_PRODUCT, SG_SCHED_FUSION = 0, 1, 2, 3, 4

SG_MAX_EXPR_OPS = 24
OPCODES = {
    "x": 1, "c": 2, "add": 3, "sub": 4, "mul": 5, "div": 6, "fma": 7, "min": 8, "max": 9,
    "neg": 10, "abs": 11, "sqrt": 12, "lt": 13, "le": 14, "gt": 15, "ge": 16, "eq": 17,
    "ne": 18, "and": 19, "or": 20, "not": 21, "select": 22, "dup": 23, "swap": 24, "index": 25,
}


class SgExprOp(C.Structure):
    _fields_ = [("op", C.c_int32), ("arg", C.c_int32), ("value", C.c_float)]


class SgExpr(C.Structure):
    _fields_ = [("nops", C.c_int32), ("ops", SgExprOp * SG_MAX_EXPR_OPS)]


class SgContract(C.Structure):
    _fields_ = [("kind", C.c_int32), ("expr", SgExpr), ("nother", C.c_int32),
                ("other", C.c_void_p * 3), ("seed", C.c_uint64), ("nvec", C.c_int32),
                ("tol", C.c_double)]


class SgViolation(C.Structure):
    _fields_ = [("contract_id", C.c_int32), ("role", C.c_int32), ("kind", C.c_int32),
                ("op_id", C.c_int32), ("first_index", C.c_int64), ("observed", C.c_double)]


class SgSolveOpts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("max_iter", C.c_int32), ("refine_tol", C.c_double),
                ("residual_tol", C.c_double), ("block", C.c_int32)]


class SgSolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("info", C.c_int32), ("residual", C.c_double),
                ("last_correction", C.c_double)]


class SgDetResult(C.Structure):
    _fields_ = [("sign", C.c_int32), ("info", C.c_int32), ("log_abs", C.c_double),
                ("det", C.c_double)]


SG_SCHED_MAX_CANDIDATES = 32


class SgSchedReport(C.Structure):
    _fields_ = [("ncand", C.c_int32), ("best_index", C.c_int32), ("default_index", C.c_int32),
                ("learned_index", C.c_int32), ("chunk", C.c_int64 * SG_SCHED_MAX_CANDIDATES),
                ("ctas_per_sm", C.c_int32 * SG_SCHED_MAX_CANDIDATES),
                ("measured_us", C.c_double * SG_SCHED_MAX_CANDIDATES),
                ("predicted_us", C.c_double * SG_SCHED_MAX_CANDIDATES),
                ("family", C.c_int32), ("chosen_index", C.c_int32)]


class SgChain(C.Structure):
    _fields_ = [("map", SgExpr), ("pre", SgExpr), ("keep", SgExpr)]


class SgError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        self.status = status
        name = STATUS[status] if 0 <= status < len(STATUS) else str(status)
        super().__init__("%s%s" % (name, (": " + msg) if msg else ""))


# ---- library -------------------------------------------------------------------
def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libsafegpu.so is not built (run __graft_entry__.build()): " + LIB_PATH)
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl, sz = C.c_void_p, C.c_int, C.c_int64, C.c_double, C.c_size_t
    P = C.POINTER
    protos = {
        "sg_init": [i32, vp, P(vp)], "sg_destroy": [vp],
        "sg_vector_create": [vp, i32, i64, vp, P(vp)],
        "sg_vector_create_async": [vp, i32, i64, vp, P(vp)], "sg_vector_read_async": [vp, vp, i64],
        "sg_sync": [vp],
        "sg_vector_wrap": [vp, i32, i64, vp, P(vp)],
        "sg_vector_read": [vp, vp, i64], "sg_vector_count": [vp, P(i64)],
        "sg_vector_device_ptr": [vp, P(vp)], "sg_vector_release": [vp],
        "sg_matrix_create": [vp, i32, i64, i64, vp, P(vp)],
        "sg_matrix_wrap": [vp, i32, i64, i64, vp, P(vp)],
        "sg_matrix_read": [vp, vp, i64], "sg_matrix_shape": [vp, P(i64), P(i64)],
        "sg_matrix_device_ptr": [vp, P(vp)], "sg_matrix_release": [vp],
        "sg_matrix_as_vector": [vp, P(vp)],
        "sg_map": [vp, P(SgExpr), vp, P(vp)], "sg_zip": [vp, P(SgExpr), vp, vp, P(vp)],
        "sg_mapn": [vp, P(SgExpr), i32, P(vp), P(vp)], "sg_for_each": [vp, P(SgExpr), vp],
        "sg_filter": [vp, P(SgExpr), vp, P(vp)], "sg_reduce": [vp, i32, vp, P(vp)],
        "sg_for_all": [vp, P(SgExpr), i32, P(vp), P(vp)],
        "sg_exists": [vp, P(SgExpr), i32, P(vp), P(vp)],
        "sg_scalar_get": [vp, P(dbl)], "sg_scalar_index": [vp, P(i64)],
        "sg_scalar_release": [vp], "sg_sort": [vp, vp, P(vp)],
        "sg_matmul": [vp, vp, vp, i32, P(vp)],
        "sg_transpose": [vp, vp, P(vp)], "sg_matvec": [vp, vp, vp, P(vp)],
        "sg_vector_item": [vp, i64, vp], "sg_concat": [vp, vp, vp, P(vp)],
        "sg_subset": [vp, vp, i64, i64, P(vp)],
        "sg_vecmat": [vp, vp, vp, P(vp)],
        "sg_solve": [vp, vp, vp, P(SgSolveOpts), P(vp), P(SgSolveInfo)],
        "sg_det": [vp, vp, i32, P(SgDetResult)],
        "sg_require": [vp, vp, P(SgContract), P(C.c_int32)],
        "sg_ensure": [vp, vp, P(SgContract), P(C.c_int32)], "sg_old": [vp, vp, P(vp)],
        "sg_last_violation": [vp, P(SgViolation)], "sg_flush": [vp],
        "sg_set_contract_mode": [vp, i32], "sg_set_fusion": [vp, i32],
        "sg_set_scheduler": [vp, i32], "sg_set_codegen": [vp, i32], "sg_plan_describe": [vp, C.c_char_p, sz, P(sz)],
        "sg_kernel_count": [vp, P(i64)], "sg_profile_enable": [vp, i32], "sg_profile_report": [vp, C.c_char_p, sz, P(sz), i32], "sg_debug_inject_sort": [vp, i32, i64, i64], "sg_debug_lookback": [vp, C.c_uint32, i64], "sg_debug_inject_matmul": [vp, i64, i64, C.c_float], "sg_debug_portable_kernels": [vp, i32],
        "sg_batch_run": [vp, P(SgChain), vp, vp, i64, vp, vp, vp],
        "sg_filter_noalloc": [P(SgExpr), vp, i64, vp, vp, vp],
        "sg_debug_jit_check_filter": [P(SgExpr), C.c_char_p, sz],
        "sg_debug_jit_check_filter_post": [P(SgExpr), P(SgExpr), C.c_char_p, sz],
        "sg_batch_report": [vp, P(SgChain), vp, vp, i64, vp, vp, vp, P(SgSchedReport)],
        "sg_sched_train": [vp, i32, C.c_float, C.c_uint64, P(C.c_float)],
        "sg_sched_log_size": [vp, P(i64), P(C.c_int32)],
        "sg_sched_log_read": [vp, vp, vp, vp, i64],
        "sg_sched_last": [vp, i32, P(SgSchedReport)],
        "sg_sched_forget": [vp, i32],
        "sg_sched_force": [vp, i32, i32],
        "sg_mlp_forward": [vp, vp, i32, vp, i64, vp],
        "sg_mlp_loss_grad": [vp, vp, i32, vp, vp, i64, vp, vp],
        "sg_mlp_adam": [vp, vp, vp, vp, vp, i64, i64, C.c_float, C.c_float, C.c_float, C.c_float],
    }
    for name, args in protos.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.sg_last_error.argtypes = [vp]
    L.sg_last_error.restype = C.c_char_p
    L.sg_status_name.argtypes = [C.c_int]
    L.sg_status_name.restype = C.c_char_p
    return L


lib = _load()


def _check(rc: int, ctx=None):
    if rc != SG_OK:
        msg = lib.sg_last_error(ctx).decode() if ctx else ""
        raise SgError(rc, msg)


def expr(ops) -> SgExpr:
    """Marshal a postfix tuple list into an sg_expr."""
    if isinstance(ops, SgExpr):
        return ops
    if len(ops) > SG_MAX_EXPR_OPS:
        raise ValueError("expression longer than %d ops" % SG_MAX_EXPR_OPS)
    e = SgExpr()
    e.nops = len(ops)
    for i, t in enumerate(ops):
        e.ops[i].op = OPCODES[t[0]]
        e.ops[i].arg = int(t[1]) if t[0] == "x" else 0
        e.ops[i].value = float(t[1]) if t[0] == "c" else 0.0
    return e


def _out(fn, ctx, *args):
    h = C.c_void_p()
    _check(fn(*args, C.byref(h)), ctx)
    return h


# ---- context -------------------------------------------------------------------
def sg_init(device: int = 0, stream: int | None = None):
    h = C.c_void_p()
    _check(lib.sg_init(device, C.c_void_p(stream or 0), C.byref(h)))
    return h


def sg_destroy(ctx):
    _check(lib.sg_destroy(ctx))


def sg_flush(ctx):
    _check(lib.sg_flush(ctx), ctx)


def sg_set_contract_mode(ctx, m):
    _check(lib.sg_set_contract_mode(ctx, m), ctx)


def sg_set_fusion(ctx, f):
    _check(lib.sg_set_fusion(ctx, f), ctx)


def sg_set_scheduler(ctx, s):
    _check(lib.sg_set_scheduler(ctx, s), ctx)


def sg_plan_describe(ctx) -> str:
    n = C.c_size_t()
    _check(lib.sg_plan_describe(ctx, None, 0, C.byref(n)), ctx)
    buf = C.create_string_buffer(n.value)
    _check(lib.sg_plan_describe(ctx, buf, n.value, C.byref(n)), ctx)
    return buf.value.decode()


def sg_kernel_count(ctx) -> int:
    n = C.c_int64()
    _check(lib.sg_kernel_count(ctx, C.byref(n)), ctx)
    return n.value


def sg_last_violation(ctx):
    v = SgViolation()
    rc = lib.sg_last_violation(ctx, C.byref(v))
    return v if rc == SG_OK else None


# ---- vectors / matrices --------------------------------------------------------
def sg_vector_create(ctx, dtype, n, host=None):
    """host: None or a numpy array (contiguous, matching dtype)."""
    ptr = host.ctypes.data if host is not None else None
    return _out(lib.sg_vector_create, ctx, ctx, dtype, n, C.c_void_p(ptr))


def sg_vector_wrap(ctx, dtype, n, dev_ptr):
    return _out(lib.sg_vector_wrap, ctx, ctx, dtype, n, C.c_void_p(dev_ptr))


def sg_vector_read(ctx, v, out):
    """out: a numpy array with count elements of the vector's dtype."""
    _check(lib.sg_vector_read(v, C.c_void_p(out.ctypes.data), out.size), ctx)
    return out


def sg_vector_create_async(ctx, dtype, n, host):
    """host: a numpy array (contiguous, matching dtype, ideally over pinned
    memory) that must stay alive and unchanged until sg_sync."""
    return _out(lib.sg_vector_create_async, ctx, ctx, dtype, n, C.c_void_p(host.ctypes.data))


def sg_vector_read_async(ctx, v, out):
    """Enqueues the copy into `out` (count elements); valid after sg_sync."""
    _check(lib.sg_vector_read_async(v, C.c_void_p(out.ctypes.data), out.size), ctx)
    return out


def sg_sync(ctx):
    _check(lib.sg_sync(ctx), ctx)


def sg_vector_count(ctx, v) -> int:
    n = C.c_int64()
    _check(lib.sg_vector_count(v, C.byref(n)), ctx)
    return n.value


def sg_vector_device_ptr(ctx, v) -> int:
    p = C.c_void_p()
    _check(lib.sg_vector_device_ptr(v, C.byref(p)), ctx)
    return p.value or 0


def sg_vector_release(v):
    _check(lib.sg_vector_release(v))


def sg_matrix_create(ctx, dtype, rows, cols, host=None):
    ptr = host.ctypes.data if host is not None else None
    return _out(lib.sg_matrix_create, ctx, ctx, dtype, rows, cols, C.c_void_p(ptr))


def sg_matrix_wrap(ctx, dtype, rows, cols, dev_ptr):
    return _out(lib.sg_matrix_wrap, ctx, ctx, dtype, rows, cols, C.c_void_p(dev_ptr))


def sg_matrix_read(ctx, m, out):
    _check(lib.sg_matrix_read(m, C.c_void_p(out.ctypes.data), out.size), ctx)
    return out


def sg_matrix_shape(ctx, m):
    r, c = C.c_int64(), C.c_int64()
    _check(lib.sg_matrix_shape(m, C.byref(r), C.byref(c)), ctx)
    return r.value, c.value


def sg_matrix_device_ptr(ctx, m) -> int:
    p = C.c_void_p()
    _check(lib.sg_matrix_device_ptr(m, C.byref(p)), ctx)
    return p.value or 0


def sg_matrix_release(m):
    _check(lib.sg_matrix_release(m))


def sg_matrix_as_vector(ctx, m):
    return _out(lib.sg_matrix_as_vector, ctx, m)


# ---- operations ----------------------------------------------------------------
def sg_map(ctx, f, x):
    e = expr(f)
    return _out(lib.sg_map, ctx, ctx, C.byref(e), x)


def sg_zip(ctx, f, x, y):
    e = expr(f)
    return _out(lib.sg_zip, ctx, ctx, C.byref(e), x, y)


def sg_mapn(ctx, f, ins):
    e = expr(f)
    arr = (C.c_void_p * len(ins))(*[h.value for h in ins])
    return _out(lib.sg_mapn, ctx, ctx, C.byref(e), len(ins), arr)


def sg_for_each(ctx, f, x):
    e = expr(f)
    _check(lib.sg_for_each(ctx, C.byref(e), x), ctx)


def sg_filter(ctx, pred, x):
    e = expr(pred)
    return _out(lib.sg_filter, ctx, ctx, C.byref(e), x)


def sg_reduce(ctx, op, x):
    return _out(lib.sg_reduce, ctx, ctx, op, x)


def sg_for_all(ctx, pred, ins):
    e = expr(pred)
    arr = (C.c_void_p * len(ins))(*[h.value for h in ins])
    return _out(lib.sg_for_all, ctx, ctx, C.byref(e), len(ins), arr)


def sg_exists(ctx, pred, ins):
    e = expr(pred)
    arr = (C.c_void_p * len(ins))(*[h.value for h in ins])
    return _out(lib.sg_exists, ctx, ctx, C.byref(e), len(ins), arr)


def sg_scalar_get(ctx, s) -> float:
    v = C.c_double()
    _check(lib.sg_scalar_get(s, C.byref(v)), ctx)
    return v.value


def sg_scalar_index(ctx, s) -> int:
    v = C.c_int64()
    _check(lib.sg_scalar_index(s, C.byref(v)), ctx)
    return v.value


def sg_scalar_release(s):
    _check(lib.sg_scalar_release(s))


def sg_sort(ctx, keys):
    return _out(lib.sg_sort, ctx, ctx, keys)


def sg_matmul(ctx, A, B, precision=SG_PREC_F32_SIMT):
    return _out(lib.sg_matmul, ctx, ctx, A, B, precision)


def sg_vector_item(ctx, v, i, dtype=np.float32):
    out = np.zeros(1, dtype=dtype)
    _check(lib.sg_vector_item(v, i, C.c_void_p(out.ctypes.data)), ctx)
    return out[0]


def sg_concat(ctx, a, b):
    return _out(lib.sg_concat, ctx, ctx, a, b)


def sg_subset(ctx, v, start, finish):
    return _out(lib.sg_subset, ctx, ctx, v, start, finish)


def sg_transpose(ctx, A):
    return _out(lib.sg_transpose, ctx, ctx, A)


def sg_matvec(ctx, A, x):
    return _out(lib.sg_matvec, ctx, ctx, A, x)


def sg_vecmat(ctx, x, A):
    return _out(lib.sg_vecmat, ctx, ctx, x, A)


def sg_solve(ctx, A, b, opts: SgSolveOpts | None = None):
    x = C.c_void_p()
    info = SgSolveInfo()
    rc = lib.sg_solve(ctx, A, b, C.byref(opts) if opts is not None else None, C.byref(x),
                      C.byref(info))
    _check(rc, ctx)
    return x, info


def sg_det(ctx, A, precision=SG_PREC_F32_SIMT) -> SgDetResult:
    out = SgDetResult()
    _check(lib.sg_det(ctx, A, precision, C.byref(out)), ctx)
    return out


def contract(kind, expr_ops=None, other=(), seed=0, nvec=4, tol=0.0) -> SgContract:
    k = SgContract()
    k.kind = kind
    if expr_ops is not None:
        k.expr = expr(expr_ops)
    k.nother = len(other)
    for i, h in enumerate(other):
        k.other[i] = h.value
    k.seed = seed
    k.nvec = nvec
    k.tol = tol
    return k


def sg_require(ctx, target, c: SgContract) -> int:
    cid = C.c_int32()
    _check(lib.sg_require(ctx, target, C.byref(c), C.byref(cid)), ctx)
    return cid.value


def sg_old(ctx, target):
    """Eiffel's `old`: the fingerprint of target at this point of the queue."""
    return _out(lib.sg_old, ctx, ctx, target)


def sg_ensure(ctx, target, c: SgContract) -> int:
    cid = C.c_int32()
    _check(lib.sg_ensure(ctx, target, C.byref(c), C.byref(cid)), ctx)
    return cid.value


def sg_batch_run(ctx, chain: SgChain, data_ptr, offsets_ptr, nseg, sums_ptr, first_ptr, kept_ptr):
    rc = lib.sg_batch_run(ctx, C.byref(chain), C.c_void_p(data_ptr), C.c_void_p(offsets_ptr),
                          nseg, C.c_void_p(sums_ptr), C.c_void_p(first_ptr),
                          C.c_void_p(kept_ptr))
    _check(rc, ctx)


def chain(map_ops, pre_ops, keep_ops) -> SgChain:
    c = SgChain()
    c.map = expr(map_ops)
    c.pre = expr(pre_ops)
    c.keep = expr(keep_ops)
    return c


# ---- torch interop (device memory only) -----------------------------------------
_TORCH_DT = {"torch.float32": SG_F32, "torch.float64": SG_F64, "torch.bfloat16": SG_BF16,
             "torch.float16": SG_F16, "torch.int32": SG_I32, "torch.int64": SG_I64}


def wrap_tensor(ctx, t):
    """Borrow a contiguous CUDA tensor as a vector (1-D) or matrix (2-D)."""
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    dt = _TORCH_DT[str(t.dtype)]
    if t.dim() == 2:
        return sg_matrix_wrap(ctx, dt, t.shape[0], t.shape[1], t.data_ptr())
    return sg_vector_wrap(ctx, dt, t.numel(), t.data_ptr())


SG_INJECT_NONE, SG_INJECT_SWAP, SG_INJECT_OVERWRITE = 0, 1, 2


def sg_debug_lookback(ctx, spin_limit=0, skip_tile=-1):
    _check(lib.sg_debug_lookback(ctx, spin_limit, skip_tile), ctx)


def sg_debug_inject_sort(ctx, mode, i, j=0):
    _check(lib.sg_debug_inject_sort(ctx, mode, i, j), ctx)


def sg_debug_inject_matmul(ctx, row, col, delta):
    _check(lib.sg_debug_inject_matmul(ctx, row, col, delta), ctx)


def sg_debug_portable_kernels(ctx, on=True):
    _check(lib.sg_debug_portable_kernels(ctx, 1 if on else 0), ctx)


def sg_profile_enable(ctx, on=True):
    _check(lib.sg_profile_enable(ctx, 1 if on else 0), ctx)


def sg_profile_report(ctx, reset=False) -> dict:
    """{kernel name: (launches, total_ms)} since the last reset."""
    n = C.c_size_t()
    _check(lib.sg_profile_report(ctx, None, 0, C.byref(n), 0), ctx)
    buf = C.create_string_buffer(n.value)
    _check(lib.sg_profile_report(ctx, buf, n.value, C.byref(n), 1 if reset else 0), ctx)
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt, ms = line.split()
        out[name] = (int(cnt), float(ms))
    return out


SG_CODEGEN_INTERPRET, SG_CODEGEN_SPECIALIZE = 0, 1


def sg_set_codegen(ctx, g):
    _check(lib.sg_set_codegen(ctx, g), ctx)


def sg_debug_jit_check_filter(pred):
    """Compile (only) the specialised filter kernel of `pred` with NVRTC.
    Returns (status, log): status 0 when it compiles."""
    e = expr(pred)
    buf = C.create_string_buffer(1 << 14)
    st = lib.sg_debug_jit_check_filter(C.byref(e), buf, len(buf))
    return int(st), buf.value.decode(errors="replace")


def sg_debug_jit_check_filter_post(pred, post):
    """Compile (only) the specialised filter of `pred` with the for_all
    postcondition `post` folded in.  Returns (status, log)."""
    e, q = expr(pred), expr(post)
    buf = C.create_string_buffer(1 << 14)
    st = lib.sg_debug_jit_check_filter_post(C.byref(e), C.byref(q), buf, len(buf))
    return int(st), buf.value.decode(errors="replace")


SG_FILTER_NOALLOC_MAX_N = 1 << 28


def sg_filter_noalloc(pred, dev_x, n, dev_out, dev_count, stream=None):
    """Allocation-free filter on caller-owned device buffers (no context)."""
    e = expr(pred)
    _check(lib.sg_filter_noalloc(C.byref(e), C.c_void_p(dev_x), n, C.c_void_p(dev_out),
                                 C.c_void_p(dev_count), C.c_void_p(stream or 0)))


def sg_batch_report(ctx, chain: SgChain, data_ptr, offsets_ptr, nseg, sums_ptr, first_ptr,
                    kept_ptr) -> SgSchedReport:
    r = SgSchedReport()
    _check(lib.sg_batch_report(ctx, C.byref(chain), C.c_void_p(data_ptr), C.c_void_p(offsets_ptr),
                               nseg, C.c_void_p(sums_ptr), C.c_void_p(first_ptr),
                               C.c_void_p(kept_ptr), C.byref(r)), ctx)
    return r


def sg_sched_train(ctx, epochs=200, lr=1e-3, seed=1) -> float:
    loss = C.c_float()
    _check(lib.sg_sched_train(ctx, epochs, lr, seed, C.byref(loss)), ctx)
    return loss.value


def sg_sched_log(ctx):
    """The timing log: features (records x 12), log microseconds, family."""
    import numpy as np
    n, d = C.c_int64(), C.c_int32()
    _check(lib.sg_sched_log_size(ctx, C.byref(n), C.byref(d)), ctx)
    X = np.empty((n.value, d.value), np.float32)
    y = np.empty(n.value, np.float32)
    fam = np.empty(n.value, np.int32)
    _check(lib.sg_sched_log_read(ctx, C.c_void_p(X.ctypes.data), C.c_void_p(y.ctypes.data),
                                 C.c_void_p(fam.ctypes.data), n.value), ctx)
    return X, y, fam


def sg_sched_forget(ctx, family=-1):
    """Drops the autotuned choices of `family` (-1: all) so they are measured again."""
    _check(lib.sg_sched_forget(ctx, family), ctx)


def sg_sched_force(ctx, family, index):
    """Every later decision of `family` takes candidate `index` (-1: none)."""
    _check(lib.sg_sched_force(ctx, family, index), ctx)


def sg_sched_last(ctx, family) -> SgSchedReport:
    """The last decision the context took in `family` (SG_SCHED_*)."""
    r = SgSchedReport()
    _check(lib.sg_sched_last(ctx, family, C.byref(r)), ctx)
    return r


def sg_mlp_forward(ctx, p_ptr, d_in, x_ptr, B, yhat_ptr):
    _check(lib.sg_mlp_forward(ctx, C.c_void_p(p_ptr), d_in, C.c_void_p(x_ptr), B,
                              C.c_void_p(yhat_ptr)), ctx)


def sg_mlp_loss_grad(ctx, p_ptr, d_in, x_ptr, y_ptr, B, g_ptr, loss_ptr):
    _check(lib.sg_mlp_loss_grad(ctx, C.c_void_p(p_ptr), d_in, C.c_void_p(x_ptr),
                                C.c_void_p(y_ptr), B, C.c_void_p(g_ptr),
                                C.c_void_p(loss_ptr)), ctx)


def sg_mlp_adam(ctx, p_ptr, g_ptr, m_ptr, v_ptr, nparams, step, lr=1e-3, b1=0.9, b2=0.999,
                eps=1e-8):
    _check(lib.sg_mlp_adam(ctx, C.c_void_p(p_ptr), C.c_void_p(g_ptr), C.c_void_p(m_ptr),
                           C.c_void_p(v_ptr), nparams, step, lr, b1, b2, eps), ctx)
