"""The schedule chooser's decision families beyond the batched launch: the
stream pass's launch shape, the filter's tile, the product's tile form and
the fusion boundaries.

Every candidate must give the oracle's results (element-wise and filter
outputs bit-exact; sums within 1e-5; products within the normwise bound of
their operand precision), a sweep must report every candidate measured, a
pass that writes over its input must not be re-run by a sweep, and on
held-out workloads the learned choice's regret is compared with the plain
table's (sched_study)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

STREAM, FILTER, PRODUCT, FUSION = 1, 2, 3, 4


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


def bits(a):
    return np.asarray(a, np.float32).view(np.uint32)


MAP = [("x", 0), ("c", 2.0), ("mul",), ("c", 1.0), ("add",)]
PRED = [("x", 0), ("c", 0.25), ("gt",)]


@pytest.mark.parametrize("n", [5, 4099, (1 << 20) + 3])
def test_stream_every_candidate_exact(env, n):
    sg, ctx, torch = env
    x = np.random.default_rng(n).uniform(-1, 1, n).astype(np.float32)
    tx, vx = dev(env, x)
    want = oracle.map(MAP, x)
    want_sum = oracle.sum(x)
    sg.sg_sched_forget(ctx, STREAM)
    y = sg.sg_map(ctx, MAP, vx)
    s = sg.sg_reduce(ctx, sg.SG_REDUCE_SUM, vx)
    sg.sg_flush(ctx)
    rep = sg.sg_sched_last(ctx, STREAM)
    assert rep.family == STREAM and rep.ncand >= 1
    assert rep.chosen_index == rep.best_index
    assert all(rep.measured_us[i] > 0 for i in range(rep.ncand)) or rep.ncand == 1
    assert np.array_equal(bits(sg.sg_vector_read(ctx, y, np.empty(n, np.float32))), bits(want))
    sg.sg_vector_release(y)
    sg.sg_scalar_release(s)
    ncand = rep.ncand
    for i in range(ncand):
        sg.sg_sched_force(ctx, STREAM, i)
        try:
            y = sg.sg_map(ctx, MAP, vx)
            s = sg.sg_reduce(ctx, sg.SG_REDUCE_SUM, vx)
            got = sg.sg_scalar_get(ctx, s)
            r = sg.sg_sched_last(ctx, STREAM)
            assert r.chosen_index == i
            assert np.array_equal(bits(sg.sg_vector_read(ctx, y, np.empty(n, np.float32))),
                                  bits(want))
            assert abs(got - want_sum) <= 1e-5 * np.abs(x.astype(np.float64)).sum() + 1e-30
            sg.sg_vector_release(y)
            sg.sg_scalar_release(s)
        finally:
            sg.sg_sched_force(ctx, STREAM, -1)
    sg.sg_vector_release(vx)
    del tx


def test_stream_plain_choice_is_the_table(env):
    sg, ctx, torch = env
    n = 1 << 24
    x = np.random.default_rng(3).uniform(-1, 1, n).astype(np.float32)
    tx, vx = dev(env, x)
    sg.sg_sched_forget(ctx, STREAM)
    y = sg.sg_map(ctx, MAP, vx)
    sg.sg_flush(ctx)
    rep = sg.sg_sched_last(ctx, STREAM)
    d = rep.default_index
    assert rep.chunk[d] == 256 and rep.ctas_per_sm[d] == 8
    assert rep.ncand == 12   # no two candidates share a grid at this length
    sg.sg_vector_release(y)
    sg.sg_vector_release(vx)


def test_in_place_pass_is_not_swept(env):
    """x := 2x + 1 in place: a sweep would apply it once per run; the pass
    takes the plain table's choice unmeasured and applies it once."""
    sg, ctx, torch = env
    n = (1 << 20) + 1
    x = np.random.default_rng(9).uniform(-1, 1, n).astype(np.float32)
    tx, vx = dev(env, x)
    sg.sg_sched_forget(ctx, STREAM)
    sg.sg_for_each(ctx, MAP, vx)
    sg.sg_flush(ctx)
    rep = sg.sg_sched_last(ctx, STREAM)
    assert rep.chosen_index == rep.default_index
    assert all(rep.measured_us[i] == 0 for i in range(rep.ncand))
    got = sg.sg_vector_read(ctx, vx, np.empty(n, np.float32))
    assert np.array_equal(bits(got), bits(oracle.map(MAP, x)))
    sg.sg_vector_release(vx)


@pytest.mark.parametrize("n", [1, 2047, 2049, 4096 * 3 + 5, 8192 * 7, (1 << 22) + 9])
def test_filter_every_tile_exact(env, n):
    sg, ctx, torch = env
    x = np.random.default_rng(n + 1).uniform(-1, 1, n).astype(np.float32)
    tx, vx = dev(env, x)
    want = oracle.filter(PRED, x)
    sg.sg_sched_forget(ctx, FILTER)
    y = sg.sg_filter(ctx, PRED, vx)
    sg.sg_flush(ctx)
    rep = sg.sg_sched_last(ctx, FILTER)
    assert rep.ncand == 3 and list(rep.chunk[:3]) == [2048, 4096, 8192]
    assert rep.default_index == 2
    assert rep.chosen_index == rep.best_index
    assert all(rep.measured_us[i] > 0 for i in range(3))
    assert sg.sg_vector_count(ctx, y) == len(want)
    assert np.array_equal(bits(sg.sg_vector_read(ctx, y, np.empty(len(want), np.float32))),
                          bits(want))
    sg.sg_vector_release(y)
    for i in range(3):
        sg.sg_sched_force(ctx, FILTER, i)
        try:
            y = sg.sg_filter(ctx, PRED, vx)
            sg.sg_flush(ctx)
            assert sg.sg_sched_last(ctx, FILTER).chosen_index == i
            assert sg.sg_vector_count(ctx, y) == len(want)
            got = sg.sg_vector_read(ctx, y, np.empty(len(want), np.float32))
            assert np.array_equal(bits(got), bits(want))
            sg.sg_vector_release(y)
        finally:
            sg.sg_sched_force(ctx, FILTER, -1)
    sg.sg_vector_release(vx)


@pytest.mark.parametrize("shape", [(128, 256, 64), (384, 640, 192), (129, 257, 65),
                                   (1024, 384, 512)])
@pytest.mark.parametrize("prec", [1, 2])
def test_product_both_forms(env, shape, prec):
    sg, ctx, torch = env
    M, N, K = shape
    g = np.random.default_rng(M + 3 * N + 7 * K)
    A = g.standard_normal((M, K)).astype(np.float32)
    B = g.standard_normal((K, N)).astype(np.float32)
    ref = oracle.matmul_f64(A, B)
    ta, ma = dev(env, A)
    tb, mb = dev(env, B)
    sg.sg_sched_forget(ctx, PRODUCT)
    mc = sg.sg_matmul(ctx, ma, mb, prec)
    sg.sg_flush(ctx)
    rep = sg.sg_sched_last(ctx, PRODUCT)
    assert rep.ncand in (1, 2)
    if rep.ncand == 2:   # the pair first, then one CTA
        assert (rep.chunk[0], rep.ctas_per_sm[0], rep.chunk[1], rep.ctas_per_sm[1]) == (256, 2, 128, 1)
        assert rep.default_index == 0 and rep.chosen_index == rep.best_index
    tol = 8e-3 if prec == 1 else 2e-3
    outs = []
    for i in range(rep.ncand):
        sg.sg_sched_force(ctx, PRODUCT, i)
        try:
            mc2 = sg.sg_matmul(ctx, ma, mb, prec)
            C = sg.sg_matrix_read(ctx, mc2, np.empty((M, N), np.float32))
            assert sg.sg_sched_last(ctx, PRODUCT).chosen_index == i
            eta = np.linalg.norm(C.astype(np.float64) - ref) / np.linalg.norm(ref)
            assert eta <= tol, (i, eta)
            outs.append(C)
            sg.sg_matrix_release(mc2)
        finally:
            sg.sg_sched_force(ctx, PRODUCT, -1)
    sg.sg_matrix_release(mc)


@pytest.mark.parametrize("n", [3, 4099, (1 << 22) + 5])
def test_fusion_boundaries_both_plans_exact(env, n):
    """a * b range-checked and summed, the product released before the flush:
    the fused plan is one kernel, the unfused one a kernel per call (three);
    both give the oracle's results, and a sweep measures both."""
    sg, ctx, torch = env
    g = np.random.default_rng(n + 5)
    a = g.uniform(-1, 1, n).astype(np.float32)
    b = g.uniform(-1, 1, n).astype(np.float32)
    ta, va = dev(env, a)
    tb, vb = dev(env, b)
    prod = oracle.map([("x", 0), ("x", 1), ("mul",)], a, b)
    want_sum = oracle.sum(prod)
    bound = 1e-5 * np.abs(prod.astype(np.float64)).sum() + 1e-30

    def run():
        z = sg.sg_zip(ctx, [("x", 0), ("x", 1), ("mul",)], va, vb)
        f = sg.sg_for_all(ctx, [("x", 0), ("c", -2.0), ("gt",)], [z])
        s = sg.sg_reduce(ctx, sg.SG_REDUCE_SUM, z)
        sg.sg_vector_release(z)
        k0 = sg.sg_kernel_count(ctx)
        ok = sg.sg_scalar_get(ctx, f)
        got = sg.sg_scalar_get(ctx, s)
        k = sg.sg_kernel_count(ctx) - k0
        sg.sg_scalar_release(f)
        sg.sg_scalar_release(s)
        assert ok == 1.0 and abs(got - want_sum) <= bound
        return k

    sg.sg_sched_forget(ctx, -1)
    run()
    rep = sg.sg_sched_last(ctx, FUSION)
    assert rep.ncand == 2 and rep.default_index == 0
    assert (rep.chunk[0], rep.ctas_per_sm[0], rep.chunk[1], rep.ctas_per_sm[1]) == (1, 1, 3, 0)
    assert rep.measured_us[0] > 0 and rep.measured_us[1] > 0
    fused_wins = rep.measured_us[1] >= 0.97 * rep.measured_us[0]
    assert rep.chosen_index == (0 if fused_wins else 1)
    for i, kernels in ((0, 1), (1, 3)):
        sg.sg_sched_force(ctx, FUSION, i)
        try:
            assert run() == kernels
            assert sg.sg_sched_last(ctx, FUSION).chosen_index == i
        finally:
            sg.sg_sched_force(ctx, FUSION, -1)


def test_fusion_not_decided_when_off_or_in_place(env):
    sg, ctx, torch = env
    n = 1 << 16
    x = np.random.default_rng(1).uniform(-1, 1, n).astype(np.float32)
    tx, vx = dev(env, x)
    # in place: the flush is not measured (a re-run would apply it twice)
    sg.sg_sched_forget(ctx, -1)
    sg.sg_for_each(ctx, MAP, vx)
    s = sg.sg_reduce(ctx, sg.SG_REDUCE_SUM, vx)
    got = sg.sg_scalar_get(ctx, s)
    want = oracle.map(MAP, x)
    assert np.array_equal(bits(sg.sg_vector_read(ctx, vx, np.empty(n, np.float32))), bits(want))
    assert abs(got - oracle.sum(want)) <= 1e-5 * np.abs(want.astype(np.float64)).sum()
    sg.sg_scalar_release(s)
    # fusion off: one kernel per call, nothing decided
    sg.sg_set_fusion(ctx, sg.SG_FUSE_OFF)
    try:
        k0 = sg.sg_kernel_count(ctx)
        z = sg.sg_zip(ctx, [("x", 0), ("x", 0), ("mul",)], vx, vx)
        s = sg.sg_reduce(ctx, sg.SG_REDUCE_SUM, z)
        sg.sg_vector_release(z)
        sg.sg_scalar_get(ctx, s)
        assert sg.sg_kernel_count(ctx) - k0 >= 2
        sg.sg_scalar_release(s)
    finally:
        sg.sg_set_fusion(ctx, sg.SG_FUSE_ON)


def test_learned_families_against_the_plain_table(env):
    """Held-out regret of the learned choice and of the plain table, per
    family (sched_study: trained on 64 swept workloads per family, 24
    held-out ones, each timed by two independent sweeps).  The learned
    choice beats the plain table where the plain table can be beaten (launch
    shape, filter tile, product tile form) and does not lose to it on the
    fusion boundaries."""
    sg, ctx, torch = env
    from paper_1410_6685_gb300 import sched_study
    sctx = sg.sg_init(0, torch.cuda.current_stream().cuda_stream)
    try:
        res = sched_study.study(sg, sctx, torch, train=64, heldout=24)
    finally:
        sg.sg_destroy(sctx)
    print(res)
    for fam in ("stream", "filter", "product"):
        r = res[fam]
        assert r["learned_mean_regret"] < r["plain_mean_regret"], (fam, r)
        assert r["learned_median_regret"] <= r["plain_median_regret"], (fam, r)
    # the fused plan is the plain choice and mostly the fastest: the learned
    # choice must not lose to it
    r = res["fusion"]
    assert r["learned_mean_regret"] <= r["plain_mean_regret"], r
