"""GPU tests of the asynchronous create / read forms (Sec. 3.1 copies to and
from the device at create and read, here enqueued on separate streams so
that one step's read overlaps the next step's create and compute), through
the C ABI: results equal the synchronous forms' and the oracle's, and the
ordering guarantees hold (later work waits for an in-flight read; a value
released at once is freed behind its read)."""
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


def pinned(torch, a):
    t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    return t, t.numpy()


def test_sort_pipeline_of_steps(env):
    """Four sort steps, each created and read asynchronously into its own
    pinned buffers (as the end-to-end benchmark does): every output is the
    oracle's sorted keys."""
    sg, ctx, torch = env
    n = 1 << 20
    keys = [inputs.sort_keys_uniform(n, seed=40 + i) for i in range(4)]
    hin = [pinned(torch, k) for k in keys]
    hout = [pinned(torch, np.zeros(n, np.int32)) for _ in range(4)]
    nxt = sg.sg_vector_create_async(ctx, sg.SG_I32, n, hin[0][1])
    for i in range(4):
        v = nxt
        if i + 1 < 4:   # the next input's copy overlaps this sort
            nxt = sg.sg_vector_create_async(ctx, sg.SG_I32, n, hin[i + 1][1])
        o = sg.sg_sort(ctx, v)
        sg.sg_vector_read_async(ctx, o, hout[i][1])
        sg.sg_vector_release(o)
        sg.sg_vector_release(v)
    sg.sg_sync(ctx)
    for i in range(4):
        assert np.array_equal(hout[i][1], oracle.sort_i32(keys[i]))


def test_create_async_then_synchronous_read(env):
    sg, ctx, torch = env
    x = np.random.default_rng(2).standard_normal(100_003).astype(np.float32)
    t, hx = pinned(torch, x)
    v = sg.sg_vector_create_async(ctx, sg.SG_F32, len(x), hx)
    y = sg.sg_map(ctx, [("x", 0), ("c", 2.0), ("mul",)], v)
    got = sg.sg_vector_read(ctx, y, np.empty(len(x), np.float32))
    assert np.array_equal(got, oracle.map([("x", 0), ("c", 2.0), ("mul",)], x))
    sg.sg_vector_release(y)
    sg.sg_vector_release(v)


def test_later_write_waits_for_inflight_read(env):
    """read_async, then an in-place update of the same vector: the
    asynchronous read sees the old values, a later read the new ones."""
    sg, ctx, torch = env
    n = 1 << 22
    x = np.arange(n, dtype=np.float32)
    t, hx = pinned(torch, x)
    v = sg.sg_vector_create_async(ctx, sg.SG_F32, n, hx)
    th, hout = pinned(torch, np.zeros(n, np.float32))
    sg.sg_vector_read_async(ctx, v, hout)
    sg.sg_for_each(ctx, [("x", 0), ("c", 1.0), ("add",)], v)
    after = sg.sg_vector_read(ctx, v, np.empty(n, np.float32))
    sg.sg_sync(ctx)
    assert np.array_equal(hout, x)
    assert np.array_equal(after, x + 1)
    sg.sg_vector_release(v)


def test_release_right_after_read_async(env):
    """A value released right after its asynchronous read is freed behind
    the copy: the data arrives intact even when new values are created at
    once (and may take the freed memory)."""
    sg, ctx, torch = env
    n = 1 << 22
    outs = []
    for i in range(3):
        x = np.full(n, float(i + 1), np.float32)
        t, hx = pinned(torch, x)
        v = sg.sg_vector_create_async(ctx, sg.SG_F32, n, hx)
        y = sg.sg_map(ctx, [("x", 0), ("c", 3.0), ("mul",)], v)
        th, hout = pinned(torch, np.zeros(n, np.float32))
        sg.sg_vector_read_async(ctx, y, hout)
        sg.sg_vector_release(y)
        sg.sg_vector_release(v)
        w = sg.sg_vector_create(ctx, sg.SG_F32, n, np.zeros(n, np.float32))
        outs.append((t, th, hout, w))
    sg.sg_sync(ctx)
    for i, (t, th, hout, w) in enumerate(outs):
        assert np.all(hout == 3.0 * (i + 1))
        sg.sg_vector_release(w)


def test_release_unused_async_create(env):
    """A vector created asynchronously and released before any use is freed
    behind its copy in; the memory is then safe to reuse."""
    sg, ctx, torch = env
    n = 1 << 22
    t, hx = pinned(torch, np.full(n, 7.0, np.float32))
    for _ in range(3):
        v = sg.sg_vector_create_async(ctx, sg.SG_F32, n, hx)
        sg.sg_vector_release(v)
    w = sg.sg_vector_create(ctx, sg.SG_F32, n, np.full(n, 2.0, np.float32))
    got = sg.sg_vector_read(ctx, w, np.empty(n, np.float32))
    sg.sg_sync(ctx)
    assert np.all(got == 2.0)
    sg.sg_vector_release(w)


def test_read_async_of_subset_and_parent(env):
    sg, ctx, torch = env
    x = np.arange(1000, dtype=np.float32)
    t, hx = pinned(torch, x)
    v = sg.sg_vector_create_async(ctx, sg.SG_F32, 1000, hx)
    s = sg.sg_subset(ctx, v, 100, 200)
    th, hout = pinned(torch, np.zeros(100, np.float32))
    sg.sg_vector_read_async(ctx, s, hout)
    sg.sg_for_each(ctx, [("x", 0), ("c", -1.0), ("mul",)], v)   # waits for the read
    got = sg.sg_vector_read(ctx, v, np.empty(1000, np.float32))
    sg.sg_sync(ctx)
    assert np.array_equal(hout, x[100:200])
    assert np.array_equal(got, -x)
    sg.sg_vector_release(s)
    sg.sg_vector_release(v)


def test_async_errors(env):
    sg, ctx, torch = env
    x = np.array([1.0, np.nan, 3.0], np.float32)
    t, hx = pinned(torch, x)
    v = sg.sg_vector_create_async(ctx, sg.SG_F32, 3, hx)
    sg.sg_require(ctx, v, sg.contract(sg.SG_C_FOR_ALL, [("x", 0), ("x", 0), ("eq",)]))
    y = sg.sg_map(ctx, [("x", 0), ("c", 1.0), ("add",)], v)
    with pytest.raises(sg.SgError) as e:
        sg.sg_vector_read_async(ctx, y, np.empty(3, np.float32))
    assert e.value.status == sg.SG_ERR_POISONED
    t2, hx2 = pinned(torch, np.ones(3, np.float32))
    w = sg.sg_vector_create_async(ctx, sg.SG_F32, 3, hx2)
    with pytest.raises(sg.SgError) as e:
        sg.sg_vector_read_async(ctx, w, np.empty(4, np.float32))
    assert e.value.status == sg.SG_ERR_SHAPE
    sg.sg_sync(ctx)
    for h in (y, v, w):
        sg.sg_vector_release(h)
