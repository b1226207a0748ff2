"""GPU parity of Listing 3's postcondition Current = old Current (Sec. 4),
through the C ABI: sg_old keeps the target's fingerprint (equal, bit for
bit, to the oracle's), and an SG_C_UNCHANGED postcondition fails exactly
when the oracle finds a changed unit between the snapshot and the check --
an in-place for_each, or a write to the caller's buffer between flushes --
and holds for compwise_divide, which only reads Current."""
import numpy as np
import pytest

import oracle
from paper_1410_6685_gb300 import inputs

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


def fp_of(sg, ctx, old):
    f = sg.sg_vector_read(ctx, old, np.empty(2, np.int64))
    return int(f[0]) & ((1 << 64) - 1), int(f[1]) & ((1 << 64) - 1)


@pytest.mark.parametrize("dt", ["float32", "float64", "bfloat16", "float16", "int32"])
@pytest.mark.parametrize("n", [0, 1, 7, 4096 + 3, 1_000_003])
def test_fingerprint_matches_oracle(env, dt, n):
    sg, ctx, torch = env
    x = inputs.uniform_pm1(inputs.rng(n + 1), n)
    if dt == "int32":
        t = torch.from_numpy(x.view(np.int32)).cuda()
    else:
        t = torch.from_numpy(x).to(getattr(torch, dt)).cuda()
    old = sg.sg_old(ctx, sg.wrap_tensor(ctx, t))
    host = t.cpu()
    ref = host.view(torch.int16).numpy() if t.element_size() == 2 else host.numpy()
    assert fp_of(sg, ctx, old) == oracle.fingerprint_old(ref)
    # an unaligned view (offset by one element)
    if n > 1:
        old = sg.sg_old(ctx, sg.wrap_tensor(ctx, t[1:]))
        assert fp_of(sg, ctx, old) == oracle.fingerprint_old(ref[1:])


def unchanged(sg, x, old):
    return sg.contract(sg.SG_C_UNCHANGED, other=[old])


def test_compwise_divide_keeps_current(env):
    """Listing 3: Result := Current / other; ensure Current = old Current and
    Result * other = Current (the latter within two roundings)."""
    sg, ctx, torch = env
    n = 1 << 20
    a, b = inputs.vadd_inputs(n)
    b[b == 0] = 0.5
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    va, vb = sg.wrap_tensor(ctx, ta), sg.wrap_tensor(ctx, tb)
    old = sg.sg_old(ctx, va)
    r = sg.sg_zip(ctx, [("x", 0), ("x", 1), ("div",)], va, vb)
    sg.sg_ensure(ctx, va, unchanged(sg, va, old))
    assert "check_unchanged" in sg.sg_plan_describe(ctx)
    sg.sg_flush(ctx)
    got = sg.sg_vector_read(ctx, r, np.empty(n, np.float32))
    assert np.array_equal(got.view(np.uint32),
                          oracle.map([("x", 0), ("x", 1), ("div",)], a, b).view(np.uint32))


@pytest.mark.parametrize("f,changes", [
    ([("x", 0), ("c", 1.0), ("mul",)], False),      # x * 1 keeps every bit
    ([("x", 0), ("c", 0.0), ("add",)], True),       # -0 + 0 = +0 changes bits
    ([("x", 0), ("c", 1.0), ("add",)], True),
])
def test_in_place_write_between_old_and_check(env, f, changes):
    sg, ctx, torch = env
    n = 300_001
    x = inputs.uniform_pm1(inputs.rng(7), n)
    x[::1000] = -0.0
    t = torch.from_numpy(x).cuda()
    v = sg.wrap_tensor(ctx, t)
    old = sg.sg_old(ctx, v)
    sg.sg_for_each(ctx, f, v)
    sg.sg_ensure(ctx, v, unchanged(sg, v, old))
    after = oracle.map(f, x)
    expect = oracle.first_changed(x, after)
    assert (expect >= 0) == changes
    if changes:
        with pytest.raises(sg.SgError) as e:
            sg.sg_flush(ctx)
        assert e.value.status == sg.SG_ERR_POSTCONDITION
        vio = sg.sg_last_violation(ctx)
        assert vio.kind == sg.SG_C_UNCHANGED and vio.role == sg.SG_POST
        assert vio.first_index == -1
    else:
        sg.sg_flush(ctx)
    assert np.array_equal(t.cpu().numpy().view(np.uint32), after.view(np.uint32))


@pytest.mark.parametrize("k", [0, 12345, 299_999])
def test_caller_write_between_flushes(env, k):
    sg, ctx, torch = env
    n = 300_000
    x = inputs.uniform_pm1(inputs.rng(8), n)
    t = torch.from_numpy(x).cuda()
    v = sg.wrap_tensor(ctx, t)
    old = sg.sg_old(ctx, v)
    sg.sg_flush(ctx)
    t[k] = float(x[k]) + 1.0                       # the caller changes one item
    assert oracle.first_changed(x, t.cpu().numpy()) == k
    sg.sg_ensure(ctx, v, unchanged(sg, v, old))
    with pytest.raises(sg.SgError) as e:
        sg.sg_flush(ctx)
    assert e.value.status == sg.SG_ERR_POSTCONDITION
    assert sg.sg_last_violation(ctx).kind == sg.SG_C_UNCHANGED
    # restored: the postcondition holds again against the same snapshot
    t[k] = float(x[k])
    v2 = sg.wrap_tensor(ctx, t)
    sg.sg_ensure(ctx, v2, unchanged(sg, v2, old))
    sg.sg_flush(ctx)


def test_contracts_off_plans_no_check(env):
    sg, ctx, torch = env
    t = torch.zeros(1000, device="cuda")
    v = sg.wrap_tensor(ctx, t)
    old = sg.sg_old(ctx, v)
    sg.sg_set_contract_mode(ctx, sg.SG_CONTRACTS_OFF)
    try:
        sg.sg_ensure(ctx, v, unchanged(sg, v, old))
        assert "check_unchanged" not in sg.sg_plan_describe(ctx)
        sg.sg_flush(ctx)
    finally:
        sg.sg_set_contract_mode(ctx, sg.SG_CONTRACTS_PRE_POST)
