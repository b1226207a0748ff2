"""Plain CPU oracle for the SafeGPU operations -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
library (``paper_1410_6685_gb300``) never imports it, and this package never
imports the library: the two share no code.  Inputs come from
``paper_1410_6685_gb300.inputs`` (seeded generators with none of the
method's arithmetic) or from the tests themselves.

The arithmetic lives in ``sg_oracle.c`` (plain C, compiled with
``-ffp-contract=off``); this module only compiles it and marshals arrays.
Expressions use a neutral form: a list of tuples such as
``[("x", 0), ("x", 1), ("add",)]`` (postfix; ``("c", v)`` pushes a binary32
constant).  The op table below is the oracle's own numbering.
"""
from __future__ import annotations

import builtins
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sg_oracle.c")
_LIB = os.path.join(_HERE, "libsg_oracle.so")
_lock = threading.Lock()
_lib = None

# oracle op numbering (matches the enum in sg_oracle.h)
_OPS = {
    "x": 1, "c": 2, "add": 3, "sub": 4, "mul": 5, "div": 6, "fma": 7,
    "min": 8, "max": 9, "neg": 10, "abs": 11, "sqrt": 12,
    "lt": 13, "le": 14, "gt": 15, "ge": 16, "eq": 17, "ne": 18,
    "and": 19, "or": 20, "not": 21, "select": 22, "dup": 23, "swap": 24,
    "index": 25,
}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB) or \
                os.path.getmtime(_LIB) < builtins.max(os.path.getmtime(_SRC),
                                             os.path.getmtime(_SRC[:-1] + "h")):
            tmp = _LIB + ".%d.tmp" % os.getpid()
            subprocess.check_call([
                "gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                "-ffp-contract=off", "-fno-fast-math", "-Wall",
                "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        i64, i32, dbl, flt, vp = C.c_int64, C.c_int, C.c_double, C.c_float, C.c_void_p
        u64 = C.c_uint64
        sig = {
            "or_map": (i32, [i32, vp, vp, vp, i32, vp, i64, vp]),
            "or_first_false": (i64, [i32, vp, vp, vp, i32, vp, i64]),
            "or_first_true": (i64, [i32, vp, vp, vp, i32, vp, i64]),
            "or_filter": (i64, [i32, vp, vp, vp, i32, vp, i64, vp]),
            "or_sum_f32": (dbl, [vp, i64]),
            "or_min_f32": (flt, [vp, i64]),
            "or_max_f32": (flt, [vp, i64]),
            "or_sort_i32": (None, [vp, i64, vp]),
            "or_first_unsorted_i32": (i64, [vp, i64]),
            "or_same_multiset_i32": (i32, [vp, vp, i64]),
            "or_matmul_f64": (None, [vp, vp, i64, i64, i64, vp]),
            "or_sort_f32": (None, [vp, i64, vp]),
            "or_first_unsorted_f32": (i64, [vp, i64]),
            "or_transpose_f32": (None, [vp, i64, i64, vp]),
            "or_matvec_f64": (None, [vp, i64, i64, vp, vp]),
            "or_vecmat_f64": (None, [vp, vp, i64, i64, vp]),
            "or_matmul_rows_f64": (None, [vp, vp, i64, i64, i64, vp, i64, vp]),
            "or_splitmix64": (u64, [u64]),
            "or_first_changed": (i64, [vp, vp, i64, i32]),
            "or_fingerprint_old": (None, [vp, i64, i32, vp]),
            "or_rademacher": (dbl, [u64, i64, i64, i64]),
            "or_freivalds": (i64, [vp, vp, vp, i64, u64, i32, dbl, dbl, vp, vp]),
            "or_gepp_f64": (i32, [vp, i64, vp]),
            "or_lu_solve_f64": (None, [vp, vp, i64, vp]),
            "or_solve_f32a": (i32, [vp, vp, i64, vp]),
            "or_det_f64": (dbl, [vp, vp, i64]),
            "or_batch_chain": (i32, [i32, vp, vp, vp, i32, vp, vp, vp, i32, vp, vp, vp,
                                     vp, vp, i64, vp, vp, vp]),
            "or_mlp_forward": (None, [vp, i32, i32, vp, i64, vp]),
            "or_mlp_loss_grad": (dbl, [vp, i32, i32, vp, vp, i64, vp]),
            "or_adam_step": (None, [vp, vp, vp, vp, i64, i64, dbl, dbl, dbl, dbl]),
            "or_mlp_nparams": (i64, [i32, i32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class _Expr:
    """An expression in the oracle's numbering, kept alive with its arrays."""

    def __init__(self, expr):
        self.op = np.array([_OPS[t[0]] for t in expr], dtype=np.int32)
        self.arg = np.array([int(t[1]) if t[0] == "x" else 0 for t in expr],
                            dtype=np.int32)
        self.cst = np.array([float(t[1]) if t[0] == "c" else 0.0 for t in expr],
                            dtype=np.float32)
        self.n = len(expr)

    def args(self):
        return (self.n, _p(self.op), _p(self.arg), _p(self.cst))


def _inputs(ins):
    arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in ins]
    ptrs = (C.c_void_p * builtins.max(1, len(arrs)))(*[a.ctypes.data for a in arrs])
    n = len(arrs[0]) if arrs else 0
    for a in arrs:
        if len(a) != n:
            raise ValueError("inputs differ in length")
    return arrs, ptrs, n


def map(expr, *ins, n=None) -> np.ndarray:
    e = _Expr(expr)
    arrs, ptrs, m = _inputs(ins)
    if n is None:
        n = m
    out = np.empty(n, dtype=np.float32)
    rc = lib().or_map(*e.args(), len(arrs), C.cast(ptrs, C.c_void_p), n, _p(out))
    if rc:
        raise ValueError("malformed expression")
    return out


def first_false(expr, *ins) -> int:
    """for_all: smallest failing index, or -1."""
    e = _Expr(expr)
    arrs, ptrs, n = _inputs(ins)
    r = lib().or_first_false(*e.args(), len(arrs), C.cast(ptrs, C.c_void_p), n)
    if r < -1:
        raise ValueError("malformed expression")
    return int(r)


def first_true(expr, *ins) -> int:
    """exists: smallest witnessing index, or -1."""
    e = _Expr(expr)
    arrs, ptrs, n = _inputs(ins)
    r = lib().or_first_true(*e.args(), len(arrs), C.cast(ptrs, C.c_void_p), n)
    if r < -1:
        raise ValueError("malformed expression")
    return int(r)


def filter(expr, *ins) -> np.ndarray:
    e = _Expr(expr)
    arrs, ptrs, n = _inputs(ins)
    out = np.empty(builtins.max(n, 1), dtype=np.float32)
    m = lib().or_filter(*e.args(), len(arrs), C.cast(ptrs, C.c_void_p), n, _p(out))
    if m < 0:
        raise ValueError("malformed expression")
    return out[:m].copy()


def sum(x) -> float:
    x = np.ascontiguousarray(x, dtype=np.float32)
    return float(lib().or_sum_f32(_p(x), len(x)))


def min(x) -> float:
    x = np.ascontiguousarray(x, dtype=np.float32)
    if len(x) == 0:
        raise ValueError("min of an empty collection")
    return float(lib().or_min_f32(_p(x), len(x)))


def max(x) -> float:
    x = np.ascontiguousarray(x, dtype=np.float32)
    if len(x) == 0:
        raise ValueError("max of an empty collection")
    return float(lib().or_max_f32(_p(x), len(x)))


def avg(x) -> float:
    return sum(x) / len(x)


def sort_i32(x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.int32)
    out = np.empty_like(x)
    lib().or_sort_i32(_p(x), len(x), _p(out))
    return out


def first_unsorted_i32(x) -> int:
    x = np.ascontiguousarray(x, dtype=np.int32)
    return int(lib().or_first_unsorted_i32(_p(x), len(x)))


def sort_f32(x) -> np.ndarray:
    """Listing 4's REAL_32 sort: ascending in IEEE 754 totalOrder."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty_like(x)
    lib().or_sort_f32(_p(x), len(x), _p(out))
    return out


def first_unsorted_f32(x) -> int:
    """is_sorted in the IEEE comparison: first i with x[i] > x[i+1], else -1."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    return int(lib().or_first_unsorted_f32(_p(x), len(x)))


def same_multiset_i32(a, b) -> bool:
    a = np.ascontiguousarray(a, dtype=np.int32)
    b = np.ascontiguousarray(b, dtype=np.int32)
    if len(a) != len(b):
        return False
    r = lib().or_same_multiset_i32(_p(a), _p(b), len(a))
    if r < 0:
        raise MemoryError
    return bool(r)


def transpose_f32(A) -> np.ndarray:
    """Sec. 3.4 `transpose` (Listing 1): At[j][i] = A[i][j]."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    r, c = A.shape
    At = np.empty((c, r), dtype=np.float32)
    lib().or_transpose_f32(_p(A), r, c, _p(At))
    return At


def matvec_f64(A, x) -> np.ndarray:
    """Sec. 3.4 `right_multiply` (Listing 1): y = A x in binary64."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    r, c = A.shape
    assert x.shape == (c,)
    y = np.empty(r, dtype=np.float64)
    lib().or_matvec_f64(_p(A), r, c, _p(x), _p(y))
    return y


def vecmat_f64(x, A) -> np.ndarray:
    """Sec. 3.4 `left_multiply`: y = x^T A in binary64."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    r, c = A.shape
    assert x.shape == (r,)
    y = np.empty(c, dtype=np.float64)
    lib().or_vecmat_f64(_p(x), _p(A), r, c, _p(y))
    return y


def matmul_f64(A, B) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    Cm = np.empty((M, N), dtype=np.float64)
    lib().or_matmul_f64(_p(A), _p(B), M, K, N, _p(Cm))
    return Cm


def matmul_rows_f64(A, B, rows) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    M, K = A.shape
    _, N = B.shape
    Cm = np.empty((len(rows), N), dtype=np.float64)
    lib().or_matmul_rows_f64(_p(A), _p(B), M, K, N, _p(rows), len(rows), _p(Cm))
    return Cm


def _units(x):
    x = np.ascontiguousarray(x)
    ub = 2 if x.dtype.itemsize == 2 else 4
    return x, x.nbytes // ub, ub


def first_changed(before, after) -> int:
    """Listing 3's Current = old Current: first unit whose bits differ, -1."""
    a, units, ub = _units(before)
    b = np.ascontiguousarray(after)
    assert a.dtype == b.dtype and a.shape == b.shape
    return int(lib().or_first_changed(_p(a), _p(b), units, ub))


def fingerprint_old(x) -> tuple:
    """The (F1, F2) fingerprint that stands for `old` of a collection."""
    a, units, ub = _units(x)
    f = np.zeros(2, dtype=np.uint64)
    lib().or_fingerprint_old(_p(a), units, ub, _p(f))
    return int(f[0]), int(f[1])


def splitmix64(z: int) -> int:
    return int(lib().or_splitmix64(z & 0xFFFFFFFFFFFFFFFF))


def rademacher(seed: int, v: int, n: int) -> np.ndarray:
    L = lib()
    return np.array([L.or_rademacher(seed, v, n, j) for j in range(n)])


def freivalds(A, B, Cm, seed: int, nvec: int = 4, c: float = 8.0,
              u_eff: float = 2.0 ** -24):
    """Returns (first violated row or -1, gap per row, tau per row)."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    Cm = np.ascontiguousarray(Cm, dtype=np.float32)
    N = A.shape[0]
    gap = np.zeros(N)
    tau = np.zeros(N)
    r = lib().or_freivalds(_p(A), _p(B), _p(Cm), N, seed, nvec, c, u_eff,
                           _p(gap), _p(tau))
    return int(r), gap, tau


def gepp_f64(A):
    LU = np.array(A, dtype=np.float64, order="C", copy=True)
    n = LU.shape[0]
    piv = np.empty(n, dtype=np.int32)
    info = lib().or_gepp_f64(_p(LU), n, _p(piv))
    return LU, piv, int(info)


def lu_solve_f64(LU, piv, b):
    x = np.array(b, dtype=np.float64, copy=True)
    lib().or_lu_solve_f64(_p(np.ascontiguousarray(LU)), _p(np.ascontiguousarray(piv)),
                          len(x), _p(x))
    return x


def solve(A, b):
    A = np.ascontiguousarray(A, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.empty_like(b)
    info = lib().or_solve_f32a(_p(A), _p(b), len(b), _p(x))
    if info:
        raise ZeroDivisionError("singular matrix (zero pivot at step %d)" % (info - 1))
    return x


def det_f64(LU, piv) -> float:
    return float(lib().or_det_f64(_p(np.ascontiguousarray(LU)),
                                  _p(np.ascontiguousarray(piv)), LU.shape[0]))


def batch_chain(map_expr, pre_expr, filt_expr, x, offsets):
    m, p, f = _Expr(map_expr), _Expr(pre_expr), _Expr(filt_expr)
    x = np.ascontiguousarray(x, dtype=np.float32)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    nseg = len(off) - 1
    sums = np.empty(nseg, dtype=np.float64)
    fv = np.empty(nseg, dtype=np.int64)
    kept = np.empty(nseg, dtype=np.int64)
    rc = lib().or_batch_chain(*m.args(), *p.args(), *f.args(), _p(x), _p(off), nseg,
                              _p(sums), _p(fv), _p(kept))
    if rc:
        raise ValueError("malformed expression")
    return sums, fv, kept


def mlp_nparams(d_in: int, H: int = 64) -> int:
    return int(lib().or_mlp_nparams(d_in, H))


def mlp_forward(P, X, d_in: int, H: int = 64) -> np.ndarray:
    P = np.ascontiguousarray(P, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    y = np.empty(X.shape[0])
    lib().or_mlp_forward(_p(P), d_in, H, _p(X), X.shape[0], _p(y))
    return y


def mlp_loss_grad(P, X, y, d_in: int, H: int = 64):
    P = np.ascontiguousarray(P, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    G = np.empty_like(P)
    loss = lib().or_mlp_loss_grad(_p(P), d_in, H, _p(X), _p(y), X.shape[0], _p(G))
    return float(loss), G


def adam_step(P, G, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In place on P, m, v (float64 arrays)."""
    lib().or_adam_step(_p(P), _p(np.ascontiguousarray(G)), _p(m), _p(v), len(P), t,
                       lr, b1, b2, eps)
