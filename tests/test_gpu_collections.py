"""GPU parity of the rest of the collection API of Table 2 -- `item`,
`concatenate`, `subset` -- and of the paper's two composed examples built on
it: component-wise division with the contracts of Listing 3, and quicksort
by three filters and two concatenations with the contracts of Listing 4
(REAL_32 keys).  Through the C ABI; every element-wise result is compared
bit for bit with the oracle."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_6685_gb300 import safegpu as sg
    ctx = sg.sg_init(0, torch.cuda.current_stream().cuda_stream)
    yield sg, ctx, torch
    sg.sg_destroy(ctx)


def dev(env, a):
    sg, ctx, torch = env
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t, sg.wrap_tensor(ctx, t)


def read(env, h, dt=np.float32):
    sg, ctx, _ = env
    n = sg.sg_vector_count(ctx, h)
    return sg.sg_vector_read(ctx, h, np.empty(n, dt))


def test_item(env):
    sg, ctx, _ = env
    x = np.arange(1000, dtype=np.float32) * np.float32(0.5)
    t, v = dev(env, x)
    y = sg.sg_map(ctx, [("x", 0), ("c", 3.0), ("add",)], v)     # pending: item flushes it
    assert sg.sg_vector_item(ctx, y, 0) == np.float32(3.0)
    assert sg.sg_vector_item(ctx, y, 999) == x[999] + np.float32(3.0)
    ti, vi = dev(env, np.array([7, -8, 9], np.int32))
    assert sg.sg_vector_item(ctx, vi, 1, np.int32) == -8
    for bad in (-1, 1000):
        with pytest.raises(sg.SgError) as e:
            sg.sg_vector_item(ctx, y, bad)
        assert e.value.status == sg.SG_ERR_SHAPE


@pytest.mark.parametrize("na,nb", [(0, 0), (0, 5), (5, 0), (1, 1), (1023, 4097),
                                   (1 << 20, 3)])
def test_concat(env, na, nb):
    sg, ctx, _ = env
    g = np.random.default_rng(na + 7 * nb)
    a = g.standard_normal(na).astype(np.float32)
    b = g.standard_normal(nb).astype(np.float32)
    ta, va = dev(env, a)
    tb, vb = dev(env, b)
    c = sg.sg_concat(ctx, va, vb)
    assert sg.sg_vector_count(ctx, c) == na + nb
    assert np.array_equal(read(env, c).view(np.uint32), np.concatenate([a, b]).view(np.uint32))


def test_concat_of_pending_filters_and_dtypes(env):
    sg, ctx, _ = env
    x = np.random.default_rng(1).standard_normal(100_000).astype(np.float32)
    t, v = dev(env, x)
    lo = sg.sg_filter(ctx, [("x", 0), ("c", -1.0), ("lt",)], v)
    hi = sg.sg_filter(ctx, [("x", 0), ("c", 1.0), ("gt",)], v)
    c = sg.sg_concat(ctx, lo, hi)    # counts are data-dependent: the filters run first
    want = np.concatenate([oracle.filter([("x", 0), ("c", -1.0), ("lt",)], x),
                           oracle.filter([("x", 0), ("c", 1.0), ("gt",)], x)])
    assert np.array_equal(read(env, c), want)
    ti, vi = dev(env, np.arange(4, dtype=np.int32))
    with pytest.raises(sg.SgError) as e:
        sg.sg_concat(ctx, v, vi)
    assert e.value.status == sg.SG_ERR_DTYPE


def test_subset_shares_memory(env):
    """subset: "shares the same memory as the original" -- an in-place
    for_each on the subset is seen through the original."""
    sg, ctx, _ = env
    x = np.arange(100, dtype=np.float32)
    t, v = dev(env, x)
    s = sg.sg_subset(ctx, v, 10, 20)
    assert sg.sg_vector_count(ctx, s) == 10
    assert np.array_equal(read(env, s), x[10:20])
    sg.sg_for_each(ctx, [("x", 0), ("c", 1000.0), ("add",)], s)
    got = read(env, v)
    want = x.copy()
    want[10:20] += 1000
    assert np.array_equal(got, want)
    e = sg.sg_subset(ctx, v, 50, 50)
    assert sg.sg_vector_count(ctx, e) == 0
    for a, b in [(-1, 5), (5, 4), (0, 101)]:
        with pytest.raises(sg.SgError) as err:
            sg.sg_subset(ctx, v, a, b)
        assert err.value.status == sg.SG_ERR_SHAPE


# ---- Listing 3: component-wise division with its contracts ----

NONZERO = [("x", 0), ("c", 0.0), ("ne",)]
# Result * other = Current, read within 2^-22 |Current| (two roundings: the
# quotient and the product each within half an ulp)
RECOVERS = [("x", 0), ("x", 1), ("mul",), ("x", 2), ("sub",), ("abs",),
            ("c", 2.0 ** -22), ("x", 2), ("abs",), ("mul",), ("le",)]


def compwise_divide(env, va, vb):
    sg, ctx, _ = env
    sg.sg_require(ctx, vb, sg.contract(sg.SG_C_FOR_ALL, NONZERO))
    r = sg.sg_zip(ctx, [("x", 0), ("x", 1), ("div",)], va, vb)
    sg.sg_ensure(ctx, r, sg.contract(sg.SG_C_FOR_ALL, RECOVERS, other=[vb, va]))
    return r


def test_compwise_divide_listing3(env):
    sg, ctx, _ = env
    g = np.random.default_rng(3)
    n = 1_000_003
    a = g.standard_normal(n).astype(np.float32)
    b = (g.standard_normal(n) + np.float32(0.1)).astype(np.float32)
    b[b == 0] = 1.0
    ta, va = dev(env, a)
    tb, vb = dev(env, b)
    r = compwise_divide(env, va, vb)
    got = read(env, r)
    assert np.array_equal(got.view(np.uint32),
                          oracle.map([("x", 0), ("x", 1), ("div",)], a, b).view(np.uint32))
    assert oracle.first_false(RECOVERS, got, b, a) == -1
    # a zero divisor violates the precondition at its (first) index
    b2 = b.copy()
    b2[[123_456, 777_777]] = 0.0
    tb2, vb2 = dev(env, b2)
    r = compwise_divide(env, va, vb2)
    with pytest.raises(sg.SgError) as e:
        sg.sg_flush(ctx)
    assert e.value.status == sg.SG_ERR_PRECONDITION
    assert sg.sg_last_violation(ctx).first_index == 123_456
    assert oracle.first_false(NONZERO, b2) == 123_456


# ---- Listing 4: quicksort by filters and concatenation (REAL_32) ----

def quicksort(env, v):
    """Listing 4 through the library: pivot = a[count // 2], three filters,
    recursion on the outer two, two concatenations."""
    sg, ctx, _ = env
    n = sg.sg_vector_count(ctx, v)
    if n <= 1:
        return v
    pivot = float(sg.sg_vector_item(ctx, v, n // 2))
    left = sg.sg_filter(ctx, [("x", 0), ("c", pivot), ("lt",)], v)
    right = sg.sg_filter(ctx, [("x", 0), ("c", pivot), ("gt",)], v)
    mid = sg.sg_filter(ctx, [("x", 0), ("c", pivot), ("eq",)], v)
    ls, rs = quicksort(env, left), quicksort(env, right)
    out = sg.sg_concat(ctx, sg.sg_concat(ctx, ls, mid), rs)
    return out


def checked_quicksort(env, x):
    """require a.count > 0; ensure Result.is_sorted, Result.count = a.count."""
    sg, ctx, _ = env
    t, v = dev(env, x)
    assert sg.sg_vector_count(ctx, v) > 0
    r = quicksort(env, v)
    sg.sg_ensure(ctx, r, sg.contract(sg.SG_C_SORTED))
    sg.sg_flush(ctx)
    return r, sg.sg_vector_count(ctx, r) == len(x)


@pytest.mark.parametrize("n,distinct", [(1, 1), (2, 2), (1000, 1000), (20_000, 50)])
def test_quicksort_listing4(env, n, distinct):
    g = np.random.default_rng(n)
    vals = (g.standard_normal(distinct) * 100).astype(np.float32)
    x = vals[g.integers(0, distinct, n)]
    r, count_ok = checked_quicksort(env, x)
    assert count_ok
    got = read(env, r)
    assert np.array_equal(got.view(np.uint32), oracle.sort_f32(x).view(np.uint32))


def test_quicksort_count_postcondition_catches_nan(env):
    """A NaN is neither <, > nor = the pivot: every filter drops it, and the
    count postcondition of Listing 4 is what notices."""
    x = np.array([3.0, np.nan, 1.0, 2.0], np.float32)
    r, count_ok = checked_quicksort(env, x)
    assert not count_ok
    assert np.array_equal(read(env, r), np.array([1.0, 2.0, 3.0], np.float32))
