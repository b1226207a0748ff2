"""GPU parity of the fused streaming pass against the oracle (Table 2 and
Sec. 3.2-3.3 operations, Sec. 4 range contracts, Sec. 5 fusion), through the
C ABI.  Element-wise results must be bit-identical; sums within 1e-5
relative (they come out far tighter: binary64 accumulation)."""
import numpy as np
import pytest

import oracle
from paper_1410_6685_gb300 import inputs

pytestmark = pytest.mark.gpu

f32 = np.float32
SIZES = [1, 3, 4, 5, 255, 1024 + 3, 256 * 4 * 37 + 1, (1 << 20) + 7]
ADD = [("x", 0), ("x", 1), ("add",)]


@pytest.fixture(scope="module", params=["specialize", "interpret"])
def env(request):
    """Every test runs with the run-time specialised kernels and with the
    interpreting kernel: both must match the oracle."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_6685_gb300 import safegpu as sg
    assert torch.cuda.is_available()
    ctx = sg.sg_init(0, torch.cuda.current_stream().cuda_stream)
    sg.sg_set_codegen(ctx, sg.SG_CODEGEN_SPECIALIZE if request.param == "specialize"
                      else sg.SG_CODEGEN_INTERPRET)
    yield sg, ctx, torch
    sg.sg_destroy(ctx)


def dev(env, a):
    sg, ctx, torch = env
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t, sg.wrap_tensor(ctx, t)


def read(env, h, n, dt=np.float32):
    sg, ctx, _ = env
    return sg.sg_vector_read(ctx, h, np.empty(n, dt))


def bits_equal(x, y):
    """Bit-identical, except that any NaN equals any NaN (IEEE 754 leaves the
    payload of a NaN result unspecified; the GPU returns its canonical NaN)."""
    x = np.asarray(x, f32)
    y = np.asarray(y, f32)
    if x.shape != y.shape:
        return False
    nx, ny = np.isnan(x), np.isnan(y)
    if not np.array_equal(nx, ny):
        return False
    return np.array_equal(x[~nx].view(np.uint32), y[~ny].view(np.uint32))


def sum_ok(got, xs):
    """Within 1e-5 relative wherever the sum is well posed (|s| >= 1e-3
    sum|x|); where the terms cancel, within the kernel's proven bound: groups
    of four are added in binary32 (two roundings, <= 2^-23 sum|x|) and the
    group sums in binary64."""
    ref = oracle.sum(xs)
    scale = np.abs(np.asarray(xs, np.float64)).sum()
    if abs(ref) >= 1e-3 * scale:
        return abs(got - ref) <= 1e-5 * abs(ref)
    return abs(got - ref) <= 2.0 ** -22 * scale


@pytest.mark.parametrize("n", SIZES)
def test_zip_add_and_sum(env, n):
    sg, ctx, _ = env
    a, b = inputs.vadd_inputs(n, seed=n)
    ta, va = dev(env, a)
    tb, vb = dev(env, b)
    z = sg.sg_zip(ctx, ADD, va, vb)
    s = sg.sg_reduce(ctx, sg.SG_REDUCE_SUM, z)
    got = sg.sg_scalar_get(ctx, s)
    zo = oracle.map(ADD, a, b)
    assert bits_equal(read(env, z, n), zo)
    assert sum_ok(got, zo)


EXPRS = [
    [("x", 0), ("x", 1), ("sub",)],
    [("x", 0), ("x", 1), ("mul",)],
    [("x", 0), ("x", 1), ("div",)],
    [("x", 0), ("x", 0), ("x", 1), ("fma",)],
    [("x", 0), ("x", 1), ("min",)],
    [("x", 0), ("x", 1), ("max",)],
    [("x", 0), ("abs",), ("sqrt",), ("neg",)],
    [("x", 0), ("x", 1), ("lt",), ("x", 0), ("x", 1), ("select",)],
    [("x", 0), ("x", 1), ("le",), ("x", 0), ("c", 0.0), ("gt",), ("and",), ("not",)],
    [("x", 0), ("x", 1), ("ge",), ("x", 0), ("x", 1), ("eq",), ("or",)],
    [("x", 0), ("x", 1), ("ne",), ("x", 0), ("x", 1), ("gt",), ("sub",)],
    [("x", 1), ("x", 0), ("swap",), ("sub",), ("dup",), ("mul",)],
    [("index",), ("c", 0.5), ("mul",), ("x", 0), ("add",)],
    [("c", 2.5), ("x", 0), ("mul",), ("x", 1), ("add",)],
]


@pytest.mark.parametrize("k", range(len(EXPRS)))
def test_expression_ops_bit_exact(env, k):
    sg, ctx, _ = env
    n = 100_003
    g = np.random.default_rng(k)
    a = (g.standard_normal(n) * 3).astype(f32)
    b = (g.standard_normal(n) * 3).astype(f32)
    a[::97] = np.nan
    b[::89] = 0.0
    a[5::101] = b[5::101]           # ties for comparisons
    ta, va = dev(env, a)
    tb, vb = dev(env, b)
    z = sg.sg_zip(ctx, EXPRS[k], va, vb)
    assert bits_equal(read(env, z, n), oracle.map(EXPRS[k], a, b))


def test_unaligned_views_use_the_scalar_path(env):
    sg, ctx, torch = env
    n = 5000
    a, b = inputs.vadd_inputs(n + 1, seed=3)
    ta = torch.from_numpy(a).cuda()
    tb = torch.from_numpy(b).cuda()
    va = sg.sg_vector_wrap(ctx, sg.SG_F32, n, ta.data_ptr() + 4)   # 4-byte offset
    vb = sg.sg_vector_wrap(ctx, sg.SG_F32, n, tb.data_ptr())
    z = sg.sg_zip(ctx, ADD, va, vb)
    assert bits_equal(read(env, z, n), oracle.map(ADD, a[1:], b[:n]))


@pytest.mark.parametrize("n", [1, 7, 4096, 300_001])
def test_min_max_avg_count(env, n):
    sg, ctx, _ = env
    x = inputs.uniform_pm1(inputs.rng(n), n) * f32(100)
    tx, vx = dev(env, x)
    res = {}
    for op in (sg.SG_REDUCE_MIN, sg.SG_REDUCE_MAX, sg.SG_REDUCE_AVG, sg.SG_REDUCE_COUNT):
        res[op] = sg.sg_reduce(ctx, op, vx)
    assert sg.sg_scalar_get(ctx, res[sg.SG_REDUCE_MIN]) == oracle.min(x)
    assert sg.sg_scalar_get(ctx, res[sg.SG_REDUCE_MAX]) == oracle.max(x)
    assert abs(sg.sg_scalar_get(ctx, res[sg.SG_REDUCE_AVG]) - oracle.avg(x)) <= \
        2.0 ** -22 * np.abs(x.astype(np.float64)).mean()
    assert sg.sg_scalar_get(ctx, res[sg.SG_REDUCE_COUNT]) == n


def test_min_max_nan_propagates(env):
    sg, ctx, _ = env
    x = np.arange(1000, dtype=f32)
    x[777] = np.nan
    tx, vx = dev(env, x)
    assert np.isnan(sg.sg_scalar_get(ctx, sg.sg_reduce(ctx, sg.SG_REDUCE_MIN, vx)))
    assert np.isnan(sg.sg_scalar_get(ctx, sg.sg_reduce(ctx, sg.SG_REDUCE_MAX, vx)))


def test_sum_closed_form(env):
    sg, ctx, _ = env
    n = 4096
    x = np.arange(1, n + 1, dtype=f32)
    tx, vx = dev(env, x)
    assert sg.sg_scalar_get(ctx, sg.sg_reduce(ctx, sg.SG_REDUCE_SUM, vx)) == n * (n + 1) // 2


@pytest.mark.parametrize("n", [1, 33, 1 << 16, (1 << 20) + 3])
def test_for_all_exists_first_index(env, n):
    sg, ctx, _ = env
    x = np.full(n, 2.0, f32)
    ge1 = [("x", 0), ("c", 1.0), ("ge",)]
    lt1 = [("x", 0), ("c", 1.0), ("lt",)]
    plants = sorted({0, n - 1, n // 2, n // 3})
    for cut in range(len(plants) + 1):
        y = x.copy()
        y[plants[cut:]] = 0.5
        ty, vy = dev(env, y)
        fa = sg.sg_for_all(ctx, ge1, [vy])
        ex = sg.sg_exists(ctx, lt1, [vy])
        want = oracle.first_false(ge1, y)
        assert want == oracle.first_true(lt1, y)
        assert sg.sg_scalar_index(ctx, fa) == want
        assert sg.sg_scalar_get(ctx, fa) == (1.0 if want < 0 else 0.0)
        assert sg.sg_scalar_index(ctx, ex) == want
        assert sg.sg_scalar_get(ctx, ex) == (0.0 if want < 0 else 1.0)


def test_vadd_postcondition_and_violation(env):
    """The vector-add workload: postcondition for_all(z == a + b)."""
    sg, ctx, torch = env
    n = 1 << 20
    a, b = inputs.vadd_inputs(n)
    for fusion in (sg.SG_FUSE_ON, sg.SG_FUSE_OFF):
        sg.sg_set_fusion(ctx, fusion)
        ta, va = dev(env, a)
        tb, vb = dev(env, b)
        z = sg.sg_zip(ctx, ADD, va, vb)
        post = sg.contract(sg.SG_C_FOR_ALL, [("x", 0), ("x", 1), ("x", 2), ("add",), ("eq",)],
                           other=[va, vb])
        sg.sg_ensure(ctx, z, post)
        s = sg.sg_reduce(ctx, sg.SG_REDUCE_SUM, z)
        got = sg.sg_scalar_get(ctx, s)
        zo = oracle.map(ADD, a, b)
        assert sum_ok(got, zo)
        assert bits_equal(read(env, z, n), zo)
        # a NaN in the inputs makes z == a + b false at that index (IEEE)
        a2 = a.copy()
        a2[123457] = np.nan
        a2[900001] = np.nan
        ta2, va2 = dev(env, a2)
        z2 = sg.sg_zip(ctx, ADD, va2, vb)
        cid = sg.sg_ensure(ctx, z2, sg.contract(sg.SG_C_FOR_ALL,
                                                [("x", 0), ("x", 1), ("x", 2), ("add",), ("eq",)],
                                                other=[va2, vb]))
        with pytest.raises(sg.SgError) as e:
            sg.sg_flush(ctx)
        assert e.value.status == sg.SG_ERR_POSTCONDITION
        v = sg.sg_last_violation(ctx)
        assert v.first_index == 123457 and v.contract_id == cid and v.role == sg.SG_POST
        zo2 = oracle.map(ADD, a2, b)
        assert oracle.first_false([("x", 2), ("x", 0), ("x", 1), ("add",), ("eq",)],
                                  a2, b, zo2) == 123457
        with pytest.raises(sg.SgError) as e:
            read(env, z2, n)
        assert e.value.status == sg.SG_ERR_POISONED
    sg.sg_set_fusion(ctx, sg.SG_FUSE_ON)


def test_precondition_poisons_dependants(env):
    """Listing 3: compwise_divide requires other.for_all(el /= 0)."""
    sg, ctx, _ = env
    n = 50_000
    g = np.random.default_rng(4)
    v1 = g.standard_normal(n).astype(f32)
    v2 = g.standard_normal(n).astype(f32)
    v2[31337] = 0.0
    t1, h1 = dev(env, v1)
    t2, h2 = dev(env, v2)
    nz = [("x", 0), ("c", 0.0), ("ne",)]
    sg.sg_require(ctx, h2, sg.contract(sg.SG_C_FOR_ALL, nz))
    q = sg.sg_zip(ctx, [("x", 0), ("x", 1), ("div",)], h1, h2)
    s = sg.sg_reduce(ctx, sg.SG_REDUCE_SUM, q)
    with pytest.raises(sg.SgError) as e:
        sg.sg_flush(ctx)
    assert e.value.status == sg.SG_ERR_PRECONDITION
    assert sg.sg_last_violation(ctx).first_index == 31337
    with pytest.raises(sg.SgError) as e:
        sg.sg_scalar_get(ctx, s)
    assert e.value.status == sg.SG_ERR_POISONED
    # with checking off the same program runs and divides by zero (inf)
    sg.sg_set_contract_mode(ctx, sg.SG_CONTRACTS_OFF)
    t2b, h2b = dev(env, v2)
    sg.sg_require(ctx, h2b, sg.contract(sg.SG_C_FOR_ALL, nz))
    q2 = sg.sg_zip(ctx, [("x", 0), ("x", 1), ("div",)], h1, h2b)
    out = read(env, q2, n)
    assert np.isinf(out[31337])
    sg.sg_set_contract_mode(ctx, sg.SG_CONTRACTS_PRE_POST)


def test_dot_product_fused_one_kernel(env):
    """Listing 5: a.compwise_multiply(b).sum runs as one kernel."""
    sg, ctx, _ = env
    n = 3_000_001
    a, b = inputs.vadd_inputs(n, seed=5)
    ta, va = dev(env, a)
    tb, vb = dev(env, b)
    # the first flush of a workload measures its launch shapes (the
    # autotuner); the second runs the plan alone
    for rep in range(2):
        k0 = sg.sg_kernel_count(ctx)
        t = sg.sg_zip(ctx, [("x", 0), ("x", 1), ("mul",)], va, vb)
        s = sg.sg_reduce(ctx, sg.SG_REDUCE_SUM, t)
        sg.sg_vector_release(t)
        got = sg.sg_scalar_get(ctx, s)
    assert sg.sg_kernel_count(ctx) - k0 == 1
    assert sum_ok(got, oracle.map([("x", 0), ("x", 1), ("mul",)], a, b))


def test_map_chain_matches_unfused(env):
    sg, ctx, _ = env
    n = 777_777
    x, y = inputs.vadd_inputs(n, seed=6)
    tx, vx = dev(env, x)
    ty, vy = dev(env, y)
    results = []
    for fusion in (sg.SG_FUSE_ON, sg.SG_FUSE_OFF):
        sg.sg_set_fusion(ctx, fusion)
        ax = sg.sg_map(ctx, [("c", 2.5), ("x", 0), ("mul",)], vx)
        r = sg.sg_zip(ctx, ADD, ax, vy)
        w = sg.sg_map(ctx, [("x", 0), ("x", 0), ("mul",), ("sqrt",)], r)
        sg.sg_vector_release(ax)
        results.append((read(env, r, n), read(env, w, n)))
    sg.sg_set_fusion(ctx, sg.SG_FUSE_ON)
    r_or = oracle.map([("c", 2.5), ("x", 0), ("mul",), ("x", 1), ("add",)], x, y)
    w_or = oracle.map([("x", 0), ("x", 0), ("mul",), ("sqrt",)], r_or)
    for r, w in results:
        assert bits_equal(r, r_or) and bits_equal(w, w_or)


def test_for_each_in_place(env):
    sg, ctx, _ = env
    n = 10_001
    x = np.arange(n, dtype=f32)
    tx, vx = dev(env, x)
    before = sg.sg_reduce(ctx, sg.SG_REDUCE_SUM, vx)
    sg.sg_for_each(ctx, [("x", 0), ("c", 2.0), ("mul",)], vx)    # Sec. 3.2 example
    after = sg.sg_reduce(ctx, sg.SG_REDUCE_SUM, vx)
    assert sg.sg_scalar_get(ctx, before) == n * (n - 1) // 2
    assert sg.sg_scalar_get(ctx, after) == n * (n - 1)
    assert bits_equal(read(env, vx, n), x * 2)


def test_masked_filter_sum_and_count(env):
    sg, ctx, _ = env
    n = 1_000_003
    x = inputs.batch_data(n, seed=12)
    tx, vx = dev(env, x)
    fma = [("x", 0), ("x", 0), ("c", 1.0), ("fma",)]
    keep = [("x", 0), ("c", 1.5), ("gt",)]
    for rep in range(2):   # the second flush, after the autotuner has measured
        k0 = sg.sg_kernel_count(ctx)
        y = sg.sg_map(ctx, fma, vx)
        k = sg.sg_filter(ctx, keep, y)
        s = sg.sg_reduce(ctx, sg.SG_REDUCE_SUM, k)
        c = sg.sg_reduce(ctx, sg.SG_REDUCE_COUNT, k)
        sg.sg_vector_release(y)
        sg.sg_vector_release(k)
        got_s, got_c = sg.sg_scalar_get(ctx, s), sg.sg_scalar_get(ctx, c)
    assert sg.sg_kernel_count(ctx) - k0 == 1
    kept = oracle.filter(keep, oracle.map(fma, x))
    assert got_c == len(kept)
    assert sum_ok(got_s, kept)


def test_e2e_host_create_and_read(env):
    sg, ctx, _ = env
    n = 65_537
    a, b = inputs.vadd_inputs(n, seed=8)
    va = sg.sg_vector_create(ctx, sg.SG_F32, n, a)
    vb = sg.sg_vector_create(ctx, sg.SG_F32, n, b)
    z = sg.sg_zip(ctx, ADD, va, vb)
    assert bits_equal(read(env, z, n), oracle.map(ADD, a, b))
    assert sg.sg_vector_count(ctx, z) == n
    for h in (va, vb, z):
        sg.sg_vector_release(h)


def test_empty_vector(env):
    sg, ctx, _ = env
    e = sg.sg_vector_create(ctx, sg.SG_F32, 0)
    s = sg.sg_reduce(ctx, sg.SG_REDUCE_SUM, e)
    fa = sg.sg_for_all(ctx, [("x", 0), ("c", 1.0), ("ge",)], [e])
    ex = sg.sg_exists(ctx, [("x", 0), ("c", 1.0), ("ge",)], [e])
    assert sg.sg_scalar_get(ctx, s) == 0.0
    assert sg.sg_scalar_get(ctx, fa) == 1.0 and sg.sg_scalar_get(ctx, ex) == 0.0
