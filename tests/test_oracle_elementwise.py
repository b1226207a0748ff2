"""Pins for the oracle's expression evaluation, reductions, for_all/exists and
filter (Table 2 and Sec. 3.2-3.3 of the paper).  CPU only.

Each pin is independent of the oracle's own code: IEEE facts with known bit
patterns, numpy's binary32 arithmetic (correctly rounded, a separate
implementation), Python's math.fsum, closed forms and brute force.
"""
import itertools
import math
import struct

import numpy as np
import pytest

import oracle

f32 = np.float32


def bits(v):
    return struct.unpack("<I", struct.pack("<f", float(v)))[0]


def X(k=0):
    return ("x", k)


# --------------------------------------------------------------------------
# expressions
# --------------------------------------------------------------------------

def test_map_plus_one_closed_form():
    # map(x + 1) over 0..n-1 is 1..n exactly (all values < 2^24)
    n = 5000
    x = np.arange(n, dtype=f32)
    y = oracle.map([X(), ("c", 1.0), ("add",)], x)
    assert np.array_equal(y, np.arange(1, n + 1, dtype=f32))


def test_ieee_known_bit_patterns():
    one = np.array([0.1], f32)
    two = np.array([0.2], f32)
    # 0.1f + 0.2f rounds to 0x3E99999A (== 0.3f)
    assert bits(oracle.map([X(0), X(1), ("add",)], one, two)[0]) == 0x3E99999A
    # sqrt(2) correctly rounded to binary32 is 0x3FB504F3
    assert bits(oracle.map([X(), ("sqrt",)], np.array([2.0], f32))[0]) == 0x3FB504F3
    # 1/3 in binary32 is 0x3EAAAAAB
    r = oracle.map([("c", 1.0), X(), ("div",)], np.array([3.0], f32))[0]
    assert bits(r) == 0x3EAAAAAB


def test_fma_single_rounding():
    # a = b = 1 + 2^-23; a*b = 1 + 2^-22 + 2^-46; fma(a, b, -(1 + 2^-22)) is
    # exactly 2^-46, whereas a rounded product followed by the add gives 0.
    a = np.array([1 + 2.0 ** -23], f32)
    c = np.array([-(1 + 2.0 ** -22)], f32)
    r = oracle.map([X(0), X(0), X(1), ("fma",)], a, c)[0]
    assert r == 2.0 ** -46
    r2 = oracle.map([X(0), X(0), ("mul",), X(1), ("add",)], a, c)[0]
    assert r2 == 0.0


@pytest.mark.parametrize("name,fn", [
    ("add", np.add), ("sub", np.subtract), ("mul", np.multiply),
    ("div", np.divide)])
def test_binary_ops_match_numpy_binary32(name, fn):
    g = np.random.default_rng(123)
    a = (g.standard_normal(4096) * 10).astype(f32)
    b = (g.standard_normal(4096) * 10).astype(f32)
    b[b == 0] = 1.0
    y = oracle.map([X(0), X(1), (name,)], a, b)
    with np.errstate(all="ignore"):
        ref = fn(a, b).astype(f32)
    assert np.array_equal(y.view(np.uint32), ref.view(np.uint32))


def test_unary_ops_match_numpy_binary32():
    g = np.random.default_rng(7)
    a = (g.standard_normal(2048) * 100).astype(f32)
    assert np.array_equal(oracle.map([X(), ("neg",)], a), -a)
    assert np.array_equal(oracle.map([X(), ("abs",)], a), np.abs(a))
    pos = np.abs(a)
    assert np.array_equal(oracle.map([X(), ("sqrt",)], pos).view(np.uint32),
                          np.sqrt(pos).view(np.uint32))


def test_comparisons_and_nan():
    nan = np.array([np.nan], f32)
    one = np.array([1.0], f32)
    for name, expect in [("lt", 0), ("le", 0), ("gt", 0), ("ge", 0), ("eq", 0), ("ne", 1)]:
        assert oracle.map([X(0), X(1), (name,)], nan, one)[0] == expect
        assert oracle.map([X(0), X(0), (name,)], nan, nan)[0] == expect
    a = np.array([1, 2, 3], f32)
    b = np.array([2, 2, 2], f32)
    assert list(oracle.map([X(0), X(1), ("lt",)], a, b)) == [1, 0, 0]
    assert list(oracle.map([X(0), X(1), ("le",)], a, b)) == [1, 1, 0]
    assert list(oracle.map([X(0), X(1), ("gt",)], a, b)) == [0, 0, 1]
    assert list(oracle.map([X(0), X(1), ("ge",)], a, b)) == [0, 1, 1]
    assert list(oracle.map([X(0), X(1), ("eq",)], a, b)) == [0, 1, 0]


def test_boolean_ops_truth_tables():
    a = np.array([0, 0, 1, 1], f32)
    b = np.array([0, 1, 0, 1], f32)
    assert list(oracle.map([X(0), X(1), ("and",)], a, b)) == [0, 0, 0, 1]
    assert list(oracle.map([X(0), X(1), ("or",)], a, b)) == [0, 1, 1, 1]
    assert list(oracle.map([X(0), ("not",)], a)) == [1, 1, 0, 0]
    # NaN counts as true (it compares unequal to zero)
    assert oracle.map([X(0), ("not",)], np.array([np.nan], f32))[0] == 0


def test_select_dup_swap_index():
    c = np.array([1, 0, 2], f32)
    t = np.array([10, 20, 30], f32)
    f = np.array([-1, -2, -3], f32)
    assert list(oracle.map([X(0), X(1), X(2), ("select",)], c, t, f)) == [10, -2, 30]
    a = np.array([3.0], f32)
    b = np.array([5.0], f32)
    assert oracle.map([X(0), X(1), ("swap",), ("sub",)], a, b)[0] == 2.0
    assert oracle.map([X(0), ("dup",), ("mul",)], a)[0] == 9.0
    assert list(oracle.map([("index",)], n=4)) == [0, 1, 2, 3]


def test_min_max_ops():
    a = np.array([1, 5, np.nan, 2], f32)
    b = np.array([3, 4, 1, np.nan], f32)
    mn = oracle.map([X(0), X(1), ("min",)], a, b)
    mx = oracle.map([X(0), X(1), ("max",)], a, b)
    assert mn[0] == 1 and mn[1] == 4 and np.isnan(mn[2]) and np.isnan(mn[3])
    assert mx[0] == 3 and mx[1] == 5 and np.isnan(mx[2]) and np.isnan(mx[3])


@pytest.mark.parametrize("expr", [
    [("add",)], [X(0), ("add",)], [X(0), X(0)], [X(3)], [], [("fma",)],
    [X(0), X(0), ("select",)], [("swap",)]])
def test_malformed_programs_rejected(expr):
    with pytest.raises(ValueError):
        oracle.map(expr, np.ones(2, f32))


def test_axpy_rewrite_is_one_expression():
    # Fig. 3: a*X[i] + Y[i] evaluated as one expression equals the two-step
    # plan (smult then plus) element by element (same roundings).
    g = np.random.default_rng(5)
    x = g.standard_normal(1000).astype(f32)
    y = g.standard_normal(1000).astype(f32)
    ax = oracle.map([("c", 2.5), X(0), ("mul",)], x)
    two_step = oracle.map([X(0), X(1), ("add",)], ax, y)
    fused = oracle.map([("c", 2.5), X(0), ("mul",), X(1), ("add",)], x, y)
    assert np.array_equal(two_step, fused)
    assert np.array_equal(fused, (f32(2.5) * x + y).astype(f32))


# --------------------------------------------------------------------------
# reductions
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [0, 1, 2, 3, 100, 4095, 4096])
def test_sum_closed_form(n):
    x = np.arange(1, n + 1, dtype=f32)
    assert oracle.sum(x) == n * (n + 1) // 2


def test_sum_cancelling_pairs_and_fsum():
    g = np.random.default_rng(0)
    v = g.standard_normal(10000).astype(f32)
    assert oracle.sum(np.concatenate([v, -v])) == 0.0
    x = g.uniform(-1, 1, 100000).astype(f32)
    exact = math.fsum(float(t) for t in x)
    assert abs(oracle.sum(x) - exact) <= 1e-12 * np.abs(x.astype(np.float64)).sum()


def test_min_max_avg_brute_force():
    g = np.random.default_rng(1)
    for n in range(1, 9):
        for _ in range(20):
            x = g.standard_normal(n).astype(f32)
            assert oracle.min(x) == min(x.tolist())
            assert oracle.max(x) == max(x.tolist())
            assert abs(oracle.avg(x) - math.fsum(x.tolist()) / n) < 1e-12
    x = np.array([1, np.nan, 0], f32)
    assert math.isnan(oracle.min(x)) and math.isnan(oracle.max(x))
    with pytest.raises(ValueError):
        oracle.min(np.zeros(0, f32))


# --------------------------------------------------------------------------
# for_all / exists
# --------------------------------------------------------------------------

def brute_first(pred, xs, want):
    for i, v in enumerate(xs):
        if bool(pred(v)) == want:
            return i
    return -1


def test_for_all_exists_brute_force():
    g = np.random.default_rng(2)
    for n in range(0, 9):
        for _ in range(30):
            x = g.integers(-3, 4, n).astype(f32)
            pe = [X(), ("c", 0.0), ("ge",)]
            assert oracle.first_false(pe, x) == brute_first(lambda v: v >= 0, x, False)
            assert oracle.first_true(pe, x) == brute_first(lambda v: v >= 0, x, True)


def test_for_all_empty_and_planted():
    pe = [X(), ("c", 1.0), ("ge",)]
    assert oracle.first_false(pe, np.zeros(0, f32)) == -1   # for_all(empty) holds
    assert oracle.first_true(pe, np.zeros(0, f32)) == -1    # exists(empty) is false
    n = 100000
    x = np.full(n, 2.0, f32)
    assert oracle.first_false(pe, x) == -1
    for idx in [0, n - 1, 777]:
        y = x.copy()
        y[idx] = 0.5
        assert oracle.first_false(pe, y) == idx
    y = x.copy()
    y[900] = 0.0
    y[300] = np.nan     # NaN >= 1 is false: a violation too; the minimum wins
    assert oracle.first_false(pe, y) == 300


def test_vadd_postcondition():
    # the vector-addition postcondition z[i] == a[i] + b[i]
    a = np.array([1, 2, 3], f32)
    b = np.array([4, 5, 6], f32)
    z = np.array([5, 7, 10], f32)
    post = [X(2), X(0), X(1), ("add",), ("eq",)]
    assert oracle.first_false(post, a, b, z) == 2


# --------------------------------------------------------------------------
# filter
# --------------------------------------------------------------------------

def test_filter_all_masks_on_8():
    vals = np.arange(1, 9, dtype=f32) * 10
    for mask in range(256):
        keep = np.array([(mask >> i) & 1 for i in range(8)], f32)
        # predicate: x[1] != 0 selects the items of x[0] whose mask bit is set
        out = oracle.filter([X(1), ("c", 0.0), ("ne",)], vals, keep)
        assert out.tolist() == [v for v, k in zip(vals.tolist(), keep) if k]


def test_filter_paper_example_and_order():
    # Sec. 3.2: c.filter(a < 5)
    c = np.array([7, 1, 9, 4, 5, 3, 0], f32)
    out = oracle.filter([X(), ("c", 5.0), ("lt",)], c)
    assert out.tolist() == [1, 4, 3, 0]
    assert len(oracle.filter([X(), ("c", 5.0), ("lt",)], np.zeros(0, f32))) == 0


def test_filter_count_complements_for_all():
    g = np.random.default_rng(3)
    x = g.uniform(-1, 1, 5000).astype(f32)
    keep = oracle.filter([X(), ("c", 0.25), ("gt",)], x)
    drop = oracle.filter([X(), ("c", 0.25), ("le",)], x)
    assert len(keep) + len(drop) == len(x)
    assert sorted(keep.tolist() + drop.tolist()) == sorted(x.tolist())
