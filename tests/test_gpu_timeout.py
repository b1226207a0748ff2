"""Failure detection of the bounded device waits (the decoupled look-back of
the sort passes and of the filter): a tile that never publishes its
look-back word makes the waits of the tiles after it run out.  The fault is
planted from the host (sg_debug_lookback: a kernel argument names the tile
that publishes nothing, and a short poll limit); nothing traps, faults or
hangs.  The flush must come back with SG_ERR_TIMEOUT within a second or so,
and the same context must then give the oracle's results again."""
import time

import numpy as np
import pytest

import oracle
from paper_1410_6685_gb300 import inputs

pytestmark = pytest.mark.gpu

SHORT = 2000   # polls (about 2 ms of waiting with the 64 ns back-off)


@pytest.fixture(scope="module", params=["specialize", "interpret"])
def env(request):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_6685_gb300 import safegpu as sg
    ctx = sg.sg_init(0, torch.cuda.current_stream().cuda_stream)
    sg.sg_set_codegen(ctx, sg.SG_CODEGEN_SPECIALIZE if request.param == "specialize"
                      else sg.SG_CODEGEN_INTERPRET)
    yield sg, ctx, torch
    sg.sg_debug_lookback(ctx, 0, -1)
    sg.sg_destroy(ctx)


def _filter(sg, ctx, x, pred):
    v = sg.sg_vector_create(ctx, sg.SG_F32, len(x), x)
    k = sg.sg_filter(ctx, pred, v)
    try:
        m = sg.sg_vector_count(ctx, k)
        return sg.sg_vector_read(ctx, k, np.empty(m, np.float32))
    finally:
        sg.sg_vector_release(k)
        sg.sg_vector_release(v)


def _sort(sg, ctx, keys):
    v = sg.sg_vector_create(ctx, sg.SG_I32, len(keys), keys)
    s = sg.sg_sort(ctx, v)
    try:
        return sg.sg_vector_read(ctx, s, np.empty(len(keys), np.int32))
    finally:
        sg.sg_vector_release(s)
        sg.sg_vector_release(v)


@pytest.mark.parametrize("skip", [0, 5, 100])
def test_filter_wait_runs_out(env, skip):
    sg, ctx, _ = env
    n = 1 << 21
    x = inputs.uniform_pm1(inputs.rng(31), n)
    pred = [("x", 0), ("c", 0.25), ("gt",)]
    sg.sg_debug_lookback(ctx, SHORT, skip)
    t0 = time.time()
    try:
        with pytest.raises(sg.SgError) as e:
            _filter(sg, ctx, x, pred)
    finally:
        sg.sg_debug_lookback(ctx, 0, -1)
    assert e.value.status == sg.SG_ERR_TIMEOUT
    assert time.time() - t0 < 10.0
    # the context is usable: the same filter gives the oracle's items
    got = _filter(sg, ctx, x, pred)
    assert np.array_equal(got.view(np.uint32), oracle.filter(pred, x).view(np.uint32))


@pytest.mark.parametrize("contracts", [True, False])
@pytest.mark.parametrize("skip", [0, 7, 150])
def test_sort_wait_runs_out(env, skip, contracts):
    sg, ctx, _ = env
    n = 1 << 20     # 171 tiles per pass
    keys = inputs.sort_keys_uniform(n)
    if not contracts:
        sg.sg_set_contract_mode(ctx, sg.SG_CONTRACTS_OFF)
    sg.sg_debug_lookback(ctx, SHORT, skip)
    t0 = time.time()
    try:
        with pytest.raises(sg.SgError) as e:
            _sort(sg, ctx, keys)
    finally:
        sg.sg_debug_lookback(ctx, 0, -1)
        sg.sg_set_contract_mode(ctx, sg.SG_CONTRACTS_PRE_POST)
    assert e.value.status == sg.SG_ERR_TIMEOUT
    assert time.time() - t0 < 10.0
    got = _sort(sg, ctx, keys)
    assert np.array_equal(got, oracle.sort_i32(keys))


def test_default_limit_is_restored(env):
    """Without the switch no wait runs out at the full bandwidth size."""
    sg, ctx, _ = env
    keys = inputs.sort_keys_uniform(1 << 22)
    assert np.array_equal(_sort(sg, ctx, keys), oracle.sort_i32(keys))
