"""GPU parity of `filter` (Table 2; Sec. 3.2 example `a < 5`): the kept items
in index order, bit-identical to the oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_1410_6685_gb300 import inputs

pytestmark = pytest.mark.gpu
f32 = np.float32


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_6685_gb300 import safegpu as sg
    ctx = sg.sg_init(0, torch.cuda.current_stream().cuda_stream)
    yield sg, ctx, torch
    sg.sg_destroy(ctx)


def run_filter(env, x, pred):
    sg, ctx, torch = env
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=f32)).cuda()
    v = sg.sg_vector_wrap(ctx, sg.SG_F32, len(x), t.data_ptr())
    k = sg.sg_filter(ctx, pred, v)
    m = sg.sg_vector_count(ctx, k)
    out = sg.sg_vector_read(ctx, k, np.empty(m, f32))
    return out, t


PREDS = [
    [("x", 0), ("c", 0.25), ("gt",)],
    [("x", 0), ("c", 5.0), ("lt",)],
    [("x", 0), ("abs",), ("c", 0.5), ("lt",), ("x", 0), ("c", -0.9), ("lt",), ("or",)],
    [("index",), ("c", 3.0), ("div",), ("dup",), ("c", 0.5), ("add",), ("c", 0.0), ("add",),
     ("swap",), ("sub",), ("c", 0.4), ("gt",)],
]


@pytest.mark.parametrize("n", [1, 2, 4095, 4096, 4097, 3 * 4096 + 5, 1_000_003])
@pytest.mark.parametrize("k", range(len(PREDS)))
def test_filter_bit_exact(env, n, k):
    x = inputs.uniform_pm1(inputs.rng(n + k), n)
    got, _ = run_filter(env, x, PREDS[k])
    ref = oracle.filter(PREDS[k], x)
    assert len(got) == len(ref)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_filter_none_and_all(env):
    x = inputs.uniform_pm1(inputs.rng(5), 100_000)
    none, _ = run_filter(env, x, [("x", 0), ("c", 2.0), ("gt",)])
    every, _ = run_filter(env, x, [("x", 0), ("c", 2.0), ("lt",)])
    assert len(none) == 0
    assert np.array_equal(every, x)


def test_filter_paper_example(env):
    c = np.array([7, 1, 9, 4, 5, 3, 0], f32)
    got, _ = run_filter(env, c, [("x", 0), ("c", 5.0), ("lt",)])
    assert got.tolist() == [1, 4, 3, 0]


def test_filter_large_full_size(env):
    n = 1 << 26
    x = inputs.batch_data(n, seed=21)
    pred = [("x", 0), ("x", 0), ("mul",), ("c", 0.5), ("gt",)]
    got, _ = run_filter(env, x, pred)
    ref = oracle.filter(pred, x)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("n", [5, 300_007, (1 << 22) + 3])
def test_reductions_of_a_kept_filter_result(env, n):
    """Reductions queued over a filter's result that a handle keeps (so it is
    compacted, not masked) cover the filter's count, which only the device
    knows when they are planned: count, sum and max against the oracle, after
    a flush that leaves large stale values in the allocator's memory."""
    sg, ctx, torch = env
    big = torch.full((n,), 1000.0, device="cuda")
    vb = sg.sg_vector_wrap(ctx, sg.SG_F32, n, big.data_ptr())
    kb = sg.sg_filter(ctx, [("x", 0), ("c", 0.0), ("gt",)], vb)
    sg.sg_flush(ctx)
    sg.sg_vector_release(kb)
    x = inputs.uniform_pm1(inputs.rng(n % 97), n)
    t = torch.from_numpy(x).cuda()
    v = sg.sg_vector_wrap(ctx, sg.SG_F32, n, t.data_ptr())
    pred = [("x", 0), ("c", 0.5), ("gt",)]
    k = sg.sg_filter(ctx, pred, v)
    rc = sg.sg_reduce(ctx, sg.SG_REDUCE_COUNT, k)
    rs = sg.sg_reduce(ctx, sg.SG_REDUCE_SUM, k)
    rm = sg.sg_reduce(ctx, sg.SG_REDUCE_MAX, k)
    kept = oracle.filter(pred, x)
    assert sg.sg_scalar_get(ctx, rc) == len(kept)
    assert sg.sg_vector_count(ctx, k) == len(kept)
    s = sg.sg_scalar_get(ctx, rs)
    assert abs(s - oracle.sum(kept)) <= 1e-5 * np.abs(kept.astype(np.float64)).sum() + 1e-30
    m = sg.sg_scalar_get(ctx, rm)
    assert (np.isnan(m) and len(kept) == 0) or m == oracle.max(kept)
    for h in (rc, rs, rm):
        sg.sg_scalar_release(h)
    for h in (k, v, vb):
        sg.sg_vector_release(h)


def test_filter_then_chain(env):
    """A filtered collection feeds further deferred operations."""
    sg, ctx, torch = env
    n = 300_007
    x = inputs.uniform_pm1(inputs.rng(9), n)
    t = torch.from_numpy(x).cuda()
    v = sg.sg_vector_wrap(ctx, sg.SG_F32, n, t.data_ptr())
    y = sg.sg_map(ctx, [("x", 0), ("c", 3.0), ("mul",)], v)
    k = sg.sg_filter(ctx, [("x", 0), ("c", 1.0), ("gt",)], y)
    s = sg.sg_reduce(ctx, sg.SG_REDUCE_MAX, k)
    m = sg.sg_vector_count(ctx, k)
    kept = oracle.filter([("x", 0), ("c", 1.0), ("gt",)],
                         oracle.map([("x", 0), ("c", 3.0), ("mul",)], x))
    assert m == len(kept)
    assert sg.sg_scalar_get(ctx, s) == oracle.max(kept)
    z = sg.sg_map(ctx, [("x", 0), ("neg",)], k)
    out = sg.sg_vector_read(ctx, z, np.empty(m, f32))
    assert np.array_equal(out, -kept)


def kernels_of(env, fn):
    """Names of the library kernels that ran during fn()."""
    sg, ctx, _ = env
    sg.sg_profile_enable(ctx, True)
    sg.sg_profile_report(ctx, reset=True)
    try:
        fn()
        return set(sg.sg_profile_report(ctx, reset=True))
    finally:
        sg.sg_profile_enable(ctx, False)


@pytest.mark.parametrize("codegen", ["specialize", "interpret"])
@pytest.mark.parametrize("n", [5, 4096, 8192, 8193, 3 * 8192, 12 * 4096 + 77, 700_001])
def test_filter_both_kernels(env, codegen, n):
    """The run-time specialised filter (one CTA per 8192-item tile) and the
    interpreting one (4096-item tiles) keep the same items in the same order
    as the oracle."""
    sg, ctx, _ = env
    sg.sg_set_codegen(ctx, sg.SG_CODEGEN_SPECIALIZE if codegen == "specialize"
                      else sg.SG_CODEGEN_INTERPRET)
    try:
        x = inputs.uniform_pm1(inputs.rng(3 * n + 1), n)
        pred = PREDS[2]
        box = {}
        names = kernels_of(env, lambda: box.update(got=run_filter(env, x, pred)[0]))
        assert ("filter_jit" if codegen == "specialize" else "filter") in names
        ref = oracle.filter(pred, x)
        assert np.array_equal(box["got"].view(np.uint32), ref.view(np.uint32))
    finally:
        sg.sg_set_codegen(ctx, sg.SG_CODEGEN_SPECIALIZE)


@pytest.mark.parametrize("n", [4096 * 9 + 3, 333_333])
def test_filter_unaligned_input(env, n):
    """An input that starts 4 bytes past a 16-byte boundary: every tile is
    loaded with 4-byte loads instead of 16-byte ones."""
    sg, ctx, torch = env
    x = inputs.uniform_pm1(inputs.rng(n), n + 1)
    t = torch.from_numpy(x).cuda()
    v = sg.sg_vector_wrap(ctx, sg.SG_F32, n, t.data_ptr() + 4)
    pred = PREDS[0]
    k = sg.sg_filter(ctx, pred, v)
    m = sg.sg_vector_count(ctx, k)
    got = sg.sg_vector_read(ctx, k, np.empty(m, f32))
    ref = oracle.filter(pred, x[1:])
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_filter_nan_and_signed_zero(env):
    """NaN items fail `x > c` and pass `x != x`; -0.0 and +0.0 are both kept by
    `x == 0` and keep their sign bits."""
    base = inputs.uniform_pm1(inputs.rng(77), 50_000)
    base[::7] = np.nan
    base[3::11] = -0.0
    base[5::13] = 0.0
    for pred in ([("x", 0), ("c", 0.25), ("gt",)], [("x", 0), ("x", 0), ("ne",)],
                 [("x", 0), ("c", 0.0), ("eq",)]):
        got, _ = run_filter(env, base, pred)
        ref = oracle.filter(pred, base)
        assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


# (filter predicate, postcondition on the kept items): one that holds, one
# that fails at the first kept item <= 0.5, one on output positions (fails
# at position 1000 when more than 1000 items are kept)
POSTS = [
    ([("x", 0), ("c", 0.25), ("gt",)], [("x", 0), ("c", 0.25), ("gt",)]),
    ([("x", 0), ("c", 0.25), ("gt",)], [("x", 0), ("c", 0.5), ("gt",)]),
    ([("x", 0), ("c", 0.0), ("lt",)], [("index",), ("c", 1000.0), ("lt",)]),
    # nothing kept: the postcondition holds on the empty result
    ([("x", 0), ("c", 2.0), ("gt",)], [("x", 0), ("c", 5.0), ("gt",)]),
]


@pytest.mark.parametrize("mode", ["folded", "unfused", "interpret"])
@pytest.mark.parametrize("n", [5, 4097, 300_007, (1 << 22) + 3])
@pytest.mark.parametrize("k", range(len(POSTS)))
def test_filter_postcondition_on_the_kept_items(env, mode, n, k):
    """`Result.for_all(p)` on a filter's result (Sec. 4) runs in the filter's
    flush: folded into the specialised filter (each kept item checked as it
    is written), or as a pass over the filter's count.  Either way the
    outcome, and the first violating position of the result, are the
    oracle's; when it holds the kept items are the oracle's, bit for bit."""
    sg, ctx, torch = env
    pred, post = POSTS[k]
    x = inputs.uniform_pm1(inputs.rng(n + 31 * k), n)
    ref = oracle.filter(pred, x)
    want = oracle.first_false(post, ref)
    t = torch.from_numpy(x).cuda()
    v = sg.sg_vector_wrap(ctx, sg.SG_F32, n, t.data_ptr())
    if mode == "unfused":
        sg.sg_set_fusion(ctx, sg.SG_FUSE_OFF)
    if mode == "interpret":
        sg.sg_set_codegen(ctx, sg.SG_CODEGEN_INTERPRET)
    try:
        kf = sg.sg_filter(ctx, pred, v)
        cid = sg.sg_ensure(ctx, kf, sg.contract(sg.SG_C_FOR_ALL, post))
        plan = sg.sg_plan_describe(ctx).splitlines()
        if mode == "folded":
            assert plan == ["filter n=%d for_all=1" % n], plan
        else:
            assert len(plan) == 2 and "(the filter's count)" in plan[1], plan
        if want < 0:
            m = sg.sg_vector_count(ctx, kf)
            out = sg.sg_vector_read(ctx, kf, np.empty(m, f32))
            assert m == len(ref)
            assert np.array_equal(out.view(np.uint32), ref.view(np.uint32))
        else:
            with pytest.raises(sg.SgError) as e:
                sg.sg_flush(ctx)
            assert e.value.status == sg.SG_ERR_POSTCONDITION
            viol = sg.sg_last_violation(ctx)
            assert viol.first_index == want and viol.contract_id == cid and viol.role == sg.SG_POST
        sg.sg_vector_release(kf)
    finally:
        sg.sg_set_fusion(ctx, sg.SG_FUSE_ON)
        sg.sg_set_codegen(ctx, sg.SG_CODEGEN_SPECIALIZE)
        sg.sg_vector_release(v)


def test_folded_postcondition_is_one_kernel(env):
    """With the postcondition folded in, the filter and its check are one
    kernel launch (after the first flush of the workload, which measures the
    filter's tiles)."""
    sg, ctx, torch = env
    n = 1 << 20
    x = inputs.uniform_pm1(inputs.rng(77), n)
    t = torch.from_numpy(x).cuda()
    v = sg.sg_vector_wrap(ctx, sg.SG_F32, n, t.data_ptr())
    pred = [("x", 0), ("c", 0.25), ("gt",)]
    for _ in range(2):
        k0 = sg.sg_kernel_count(ctx)
        kf = sg.sg_filter(ctx, pred, v)
        sg.sg_ensure(ctx, kf, sg.contract(sg.SG_C_FOR_ALL, pred))
        m = sg.sg_vector_count(ctx, kf)
        sg.sg_vector_release(kf)
    assert sg.sg_kernel_count(ctx) - k0 == 1
    assert m == len(oracle.filter(pred, x))
    sg.sg_vector_release(v)


@pytest.mark.parametrize("fuse", [True, False])
def test_filter_postcondition_nan_kept(env, fuse):
    """NaN items kept by the filter (x > 0.5 or x != x) fail `x > 0.5` (an
    IEEE comparison with NaN is false): the first NaN's position in the
    result is the violation, folded or not."""
    sg, ctx, torch = env
    n = 300_007
    x = inputs.uniform_pm1(inputs.rng(41), n)
    x[[1234, 5678, 200_001]] = np.nan
    pred = [("x", 0), ("c", 0.5), ("gt",), ("x", 0), ("x", 0), ("ne",), ("or",)]
    post = [("x", 0), ("c", 0.5), ("gt",)]
    ref = oracle.filter(pred, x)
    want = oracle.first_false(post, ref)
    assert want >= 0 and np.isnan(ref[want])
    t = torch.from_numpy(x).cuda()
    v = sg.sg_vector_wrap(ctx, sg.SG_F32, n, t.data_ptr())
    sg.sg_set_fusion(ctx, sg.SG_FUSE_ON if fuse else sg.SG_FUSE_OFF)
    try:
        kf = sg.sg_filter(ctx, pred, v)
        cid = sg.sg_ensure(ctx, kf, sg.contract(sg.SG_C_FOR_ALL, post))
        with pytest.raises(sg.SgError) as e:
            sg.sg_flush(ctx)
        assert e.value.status == sg.SG_ERR_POSTCONDITION
        viol = sg.sg_last_violation(ctx)
        assert viol.first_index == want and viol.contract_id == cid
        sg.sg_vector_release(kf)
    finally:
        sg.sg_set_fusion(ctx, sg.SG_FUSE_ON)
        sg.sg_vector_release(v)
