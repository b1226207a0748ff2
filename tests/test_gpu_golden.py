"""GPU parity on the fixtures in tests/golden/ (the paper's worked examples,
Sec. 3.1, Listings 3-5, Sec. 5): the library, through the C ABI, gives the
stored values bit for bit."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
f32 = np.float32


def load(name):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        return json.load(f)


def arr(v):
    return np.array([int(b, 16) for b in v["bits"]], dtype=np.uint32).view(f32)


def expr(d):
    return [tuple(o) for o in d["expr"]]


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_6685_gb300 import safegpu as sg
    ctx = sg.sg_init(0, torch.cuda.current_stream().cuda_stream)
    yield sg, ctx
    sg.sg_destroy(ctx)


def vec(sg, ctx, a):
    return sg.sg_vector_create(ctx, sg.SG_F32, len(a), np.ascontiguousarray(a, dtype=f32))


def read(sg, ctx, v):
    n = sg.sg_vector_count(ctx, v)
    return sg.sg_vector_read(ctx, v, np.empty(n, f32))


def bits_equal(a, b):
    return a.shape == b.shape and np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_filter_less_than_five(env):
    sg, ctx = env
    d = load("filter_less_than_five")
    v = vec(sg, ctx, arr(d["in"][0]))
    k = sg.sg_filter(ctx, expr(d), v)
    assert bits_equal(read(sg, ctx, k), arr(d["out"]))
    for h in (k, v):
        sg.sg_vector_release(h)


def test_for_each_double(env):
    sg, ctx = env
    d = load("for_each_double")
    v = vec(sg, ctx, arr(d["in"][0]))
    sg.sg_for_each(ctx, expr(d), v)
    assert bits_equal(read(sg, ctx, v), arr(d["out"]))
    sg.sg_vector_release(v)


def test_project_sqrt(env):
    sg, ctx = env
    d = load("project_sqrt")
    v = vec(sg, ctx, arr(d["in"][0]))
    y = sg.sg_map(ctx, expr(d), v)
    assert bits_equal(read(sg, ctx, y), arr(d["out"]))
    for h in (y, v):
        sg.sg_vector_release(h)


def test_dot_product(env):
    sg, ctx = env
    d = load("dot_product")
    a, b = vec(sg, ctx, arr(d["in"][0])), vec(sg, ctx, arr(d["in"][1]))
    t = sg.sg_zip(ctx, expr(d), a, b)
    s = sg.sg_reduce(ctx, sg.SG_REDUCE_SUM, t)
    assert sg.sg_scalar_get(ctx, s) == float(d["out"]["sum"])
    sg.sg_scalar_release(s)
    for h in (t, a, b):
        sg.sg_vector_release(h)


@pytest.mark.parametrize("name", ["compwise_divide", "axpy"])
def test_zip_examples(env, name):
    sg, ctx = env
    d = load(name)
    a, b = vec(sg, ctx, arr(d["in"][0])), vec(sg, ctx, arr(d["in"][1]))
    if "pre_on_second" in d:
        sg.sg_require(ctx, b, sg.contract(sg.SG_C_FOR_ALL, [tuple(o) for o in d["pre_on_second"]]))
    z = sg.sg_zip(ctx, expr(d), a, b)
    assert bits_equal(read(sg, ctx, z), arr(d["out"]))
    for h in (z, a, b):
        sg.sg_vector_release(h)


def test_quicksort(env):
    sg, ctx = env
    d = load("quicksort")
    v = vec(sg, ctx, arr(d["in"][0]))
    s = sg.sg_sort(ctx, v)
    sg.sg_ensure(ctx, s, sg.contract(sg.SG_C_SORTED))
    assert bits_equal(read(sg, ctx, s), arr(d["out"]))
    for h in (s, v):
        sg.sg_vector_release(h)
