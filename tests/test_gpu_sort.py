"""GPU parity of the int32 sort and its postconditions (Listing 4:
Result.is_sorted; Result.count = a.count strengthened to a permutation
check), through the C ABI.  The output is unique, so it must be
bit-identical to the oracle's."""
import numpy as np
import pytest

import oracle
from paper_1410_6685_gb300 import inputs

pytestmark = pytest.mark.gpu

TILE = 6144   # keys per tile of the onesweep kernel


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_6685_gb300 import safegpu as sg
    ctx = sg.sg_init(0, torch.cuda.current_stream().cuda_stream)
    yield sg, ctx, torch
    sg.sg_destroy(ctx)


def run_sort(env, keys, flush_ok=True):
    sg, ctx, torch = env
    t = torch.from_numpy(np.ascontiguousarray(keys, dtype=np.int32)).cuda()
    v = sg.sg_vector_wrap(ctx, sg.SG_I32, len(keys), t.data_ptr())
    out = sg.sg_sort(ctx, v)
    if flush_ok:
        sg.sg_flush(ctx)
    return v, out, t


def read(env, h, n):
    sg, ctx, _ = env
    return sg.sg_vector_read(ctx, h, np.empty(n, np.int32))


@pytest.mark.parametrize("n", [1, 2, 3, 17, TILE - 1, TILE, TILE + 1, 3 * TILE + 17,
                               100_003, 1 << 20])
def test_sort_uniform_bit_exact(env, n):
    keys = inputs.sort_keys_uniform(n, seed=1000 + n)
    v, out, t = run_sort(env, keys)
    assert np.array_equal(read(env, out, n), oracle.sort_i32(keys))


@pytest.mark.parametrize("n", [5000, 1 << 20])
def test_sort_256_distinct_values(env, n):
    keys = inputs.sort_keys_distinct(n)
    v, out, t = run_sort(env, keys)
    got = read(env, out, n)
    assert np.array_equal(got, oracle.sort_i32(keys))


def test_sort_extremes_and_orders(env):
    base = np.array([2**31 - 1, -2**31, 0, -1, 1, 255, 256, -256, 65536, -65537], np.int32)
    for keys in (np.tile(base, 1000), np.sort(np.tile(base, 700)),
                 np.sort(np.tile(base, 900))[::-1].copy(), np.zeros(12345, np.int32),
                 np.full(9999, -7, np.int32)):
        v, out, t = run_sort(env, keys)
        assert np.array_equal(read(env, out, len(keys)), oracle.sort_i32(keys))


def test_sort_full_size_workload(env):
    """The sort workload at full size: 2^26 uniform int32 keys."""
    n = 1 << 26
    keys = inputs.sort_keys_uniform(n)
    v, out, t = run_sort(env, keys)
    got = read(env, out, n)
    assert oracle.first_unsorted_i32(got) == -1
    assert np.array_equal(got, oracle.sort_i32(keys))


def test_sort_full_size_256_distinct(env):
    """The workload's second variant at full size: 2^26 keys drawn from 256
    distinct values (long runs of equal digits in every pass).  Bit-exact
    against the oracle's sort."""
    n = 1 << 26
    keys = inputs.sort_keys_distinct(n)
    v, out, t = run_sort(env, keys)
    got = read(env, out, n)
    assert oracle.first_unsorted_i32(got) == -1
    assert np.array_equal(got, oracle.sort_i32(keys))


def test_sort_input_is_not_modified(env):
    keys = inputs.sort_keys_uniform(50_000, seed=3)
    v, out, t = run_sort(env, keys)
    assert np.array_equal(t.cpu().numpy(), keys)


def radix_intermediate(keys):
    """Keys after the first three 8-bit LSD passes: stably ordered by their
    low 24 bits (the definition of LSD radix sorting)."""
    low = keys.view(np.uint32) & np.uint32(0xFFFFFF)
    return keys[np.argsort(low, kind="stable")]


def last_pass(inter):
    """The last LSD pass: stable by the top byte, sign bit flipped."""
    top = (inter.view(np.uint32) >> np.uint32(24)) ^ np.uint32(0x80)
    return inter[np.argsort(top, kind="stable")]


@pytest.mark.parametrize("n,i,j", [(3 * TILE + 17, 5, 6), (3 * TILE + 17, 100, 3000),
                                   (1 << 20, 70000, 70001), (1 << 20, 12, 900000),
                                   (100_003, 0, 100_002)])
def test_fused_sortedness_catches_planted_swap(env, n, i, j):
    sg, ctx, torch = env
    keys = inputs.sort_keys_uniform(n, seed=77)
    inter = radix_intermediate(keys)
    bad = inter.copy()
    bad[i], bad[j] = bad[j], bad[i]
    expect_out = last_pass(bad)
    expect_first = oracle.first_unsorted_i32(expect_out)
    sg.sg_debug_inject_sort(ctx, sg.SG_INJECT_SWAP, i, j)
    v, out, t = run_sort(env, keys, flush_ok=False)
    if expect_first < 0:
        sg.sg_flush(ctx)
    else:
        with pytest.raises(sg.SgError) as e:
            sg.sg_flush(ctx)
        assert e.value.status == sg.SG_ERR_POSTCONDITION
        vio = sg.sg_last_violation(ctx)
        assert vio.kind == sg.SG_C_SORTED and vio.first_index == expect_first
        assert vio.contract_id == -1          # a built-in contract of sort
        with pytest.raises(sg.SgError) as e:
            read(env, out, n)
        assert e.value.status == sg.SG_ERR_POISONED


@pytest.mark.parametrize("n,i,val", [(3 * TILE + 17, 10, 123), (1 << 20, 500000, -2**31)])
def test_fused_permutation_catches_overwrite(env, n, i, val):
    sg, ctx, torch = env
    keys = inputs.sort_keys_uniform(n, seed=78)
    sg.sg_debug_inject_sort(ctx, sg.SG_INJECT_OVERWRITE, i, val)
    v, out, t = run_sort(env, keys, flush_ok=False)
    with pytest.raises(sg.SgError) as e:
        sg.sg_flush(ctx)
    assert e.value.status == sg.SG_ERR_POSTCONDITION
    vio = sg.sg_last_violation(ctx)
    bad = radix_intermediate(keys)
    bad[i] = val
    exp_first = oracle.first_unsorted_i32(last_pass(bad))
    if vio.kind == sg.SG_C_SORTED:
        assert vio.first_index == exp_first
    else:
        assert vio.kind == sg.SG_C_PERMUTATION and vio.first_index == -1 and exp_first == -1
    assert not oracle.same_multiset_i32(keys, last_pass(bad))


def test_unfused_strict_checks(env):
    """With fusion off the postconditions re-read the output (strict mode)."""
    sg, ctx, torch = env
    sg.sg_set_fusion(ctx, sg.SG_FUSE_OFF)
    try:
        n = 200_001
        keys = inputs.sort_keys_uniform(n, seed=9)
        v, out, t = run_sort(env, keys)
        assert np.array_equal(read(env, out, n), oracle.sort_i32(keys))
        # user contracts on arbitrary vectors
        bad = oracle.sort_i32(keys)
        bad[123], bad[124] = bad[124], bad[123]
        tb = torch.from_numpy(bad).cuda()
        vb = sg.sg_vector_wrap(ctx, sg.SG_I32, n, tb.data_ptr())
        sg.sg_ensure(ctx, vb, sg.contract(sg.SG_C_SORTED))
        sg.sg_ensure(ctx, vb, sg.contract(sg.SG_C_PERMUTATION, other=[v]))
        with pytest.raises(sg.SgError) as e:
            sg.sg_flush(ctx)
        vio = sg.sg_last_violation(ctx)
        assert vio.kind == sg.SG_C_SORTED and vio.first_index == oracle.first_unsorted_i32(bad)
        bad2 = oracle.sort_i32(keys)
        bad2[-1] = bad2[-1] ^ 1
        tb2 = torch.from_numpy(bad2).cuda()
        vb2 = sg.sg_vector_wrap(ctx, sg.SG_I32, n, tb2.data_ptr())
        sg.sg_ensure(ctx, vb2, sg.contract(sg.SG_C_PERMUTATION, other=[v]))
        with pytest.raises(sg.SgError) as e:
            sg.sg_flush(ctx)
        assert sg.sg_last_violation(ctx).kind == sg.SG_C_PERMUTATION
    finally:
        sg.sg_set_fusion(ctx, sg.SG_FUSE_ON)


def test_contracts_off_sort(env):
    sg, ctx, torch = env
    sg.sg_set_contract_mode(ctx, sg.SG_CONTRACTS_OFF)
    try:
        keys = inputs.sort_keys_uniform(70_000, seed=10)
        sg.sg_debug_inject_sort(ctx, sg.SG_INJECT_SWAP, 1, 60000)
        v, out, t = run_sort(env, keys)          # nothing is checked
        got = read(env, out, len(keys))
        bad = radix_intermediate(keys)
        bad[1], bad[60000] = bad[60000], bad[1]
        assert np.array_equal(got, last_pass(bad))
    finally:
        sg.sg_set_contract_mode(ctx, sg.SG_CONTRACTS_PRE_POST)


# ---- binary32 keys (Listing 4 sorts REAL_32), IEEE totalOrder ----

SPECIAL = np.array([0xFFC00005, 0xFFC00001, 0xFF800000, 0xC0200000, 0x80000001, 0x80000000,
                    0x00000000, 0x00000001, 0x3F800000, 0x7F800000, 0x7FC00001, 0x7FC00005],
                   dtype=np.uint32).view(np.float32)


def float_keys(n, seed):
    g = np.random.default_rng(seed)
    x = (g.standard_normal(n) * np.float32(1e3)).astype(np.float32)
    if n >= 64:
        idx = g.choice(n, min(n // 8, 4096), replace=False)
        x[idx] = SPECIAL[g.integers(0, len(SPECIAL), len(idx))]
    return x


def run_sort_f32(env, keys, flush_ok=True):
    sg, ctx, torch = env
    t = torch.from_numpy(np.ascontiguousarray(keys, dtype=np.float32)).cuda()
    v = sg.sg_vector_wrap(ctx, sg.SG_F32, len(keys), t.data_ptr())
    out = sg.sg_sort(ctx, v)
    if flush_ok:
        sg.sg_flush(ctx)
    return v, out, t


@pytest.mark.parametrize("n", [1, 2, 12, 100, TILE - 1, TILE + 1, 3 * TILE + 17, 1 << 20])
def test_sort_f32_total_order_bit_exact(env, n):
    keys = float_keys(n, 2000 + n) if n != 12 else SPECIAL[::-1].copy()
    v, out, t = run_sort_f32(env, keys)
    sg, ctx, _ = env
    got = sg.sg_vector_read(ctx, out, np.empty(n, np.float32))
    assert np.array_equal(got.view(np.uint32), oracle.sort_f32(keys).view(np.uint32))
    assert oracle.first_unsorted_f32(got) == -1


def test_sort_f32_full_size(env):
    """2^26 binary32 keys (N(0,1e3) with special values planted)."""
    n = 1 << 26
    keys = float_keys(n, 5)
    v, out, t = run_sort_f32(env, keys)
    sg, ctx, _ = env
    got = sg.sg_vector_read(ctx, out, np.empty(n, np.float32))
    assert np.array_equal(got.view(np.uint32), oracle.sort_f32(keys).view(np.uint32))


def test_sort_f32_fused_checks_catch_planted_swap(env):
    sg, ctx, _ = env
    n = 3 * TILE + 17
    keys = float_keys(n, 9)
    sg.sg_debug_inject_sort(ctx, sg.SG_INJECT_SWAP, 3, n - 2)
    v, out, t = run_sort_f32(env, keys, flush_ok=False)
    with pytest.raises(sg.SgError) as e:
        sg.sg_flush(ctx)
    assert e.value.status == sg.SG_ERR_POSTCONDITION
    assert sg.sg_last_violation(ctx).kind == sg.SG_C_SORTED


def test_sorted_contract_f32_ieee_comparison(env):
    """A user-attached sortedness contract on binary32 data uses the IEEE
    comparison: +0 before -0 and NaNs are not violations; 2 > 1 is."""
    sg, ctx, torch = env
    for data, first in [(np.array([1.0, 2.0, np.nan, 0.5, 3.0], np.float32), -1),
                        (np.array([0.0, -0.0, 1.0], np.float32), -1),
                        (np.array([0.0, 1.0, 2.0, 1.0, 5.0], np.float32), 2)]:
        assert oracle.first_unsorted_f32(data) == first
        t = torch.from_numpy(data).cuda()
        v = sg.sg_vector_wrap(ctx, sg.SG_F32, len(data), t.data_ptr())
        sg.sg_ensure(ctx, v, sg.contract(sg.SG_C_SORTED))
        if first < 0:
            sg.sg_flush(ctx)
        else:
            with pytest.raises(sg.SgError):
                sg.sg_flush(ctx)
            assert sg.sg_last_violation(ctx).first_index == first
        sg.sg_vector_release(v)
