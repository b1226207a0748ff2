"""CPU checks of the boundary: the library loads without a GPU, exports every
function include/safegpu.h declares, and the host planner (Sec. 5 optimizer)
makes the plans the paper describes, on a planning-only context (device -1).
No compute call is made."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "safegpu.h")


@pytest.fixture(scope="module")
def sg():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_6685_gb300 import safegpu
    return safegpu


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:sg_status|const char\*)\s+(sg_\w+)\s*\(", text, re.M)))


def test_every_declared_symbol_is_exported(sg):
    names = declared_functions()
    assert len(names) >= 40
    out = subprocess.run(["nm", "-D", "--defined-only", sg.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (sg_\w+)$", out, re.M))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert getattr(sg.lib, n) is not None


def test_no_cpu_fallback_symbols(sg):
    # the library links no oracle code
    out = subprocess.run(["nm", "-D", sg.LIB_PATH], capture_output=True, text=True).stdout
    assert "or_" + "map" not in out and "or_sort" not in out


def test_status_names(sg):
    for i, name in enumerate(sg.STATUS):
        assert sg.lib.sg_status_name(i).decode() == name


@pytest.fixture
def pctx(sg):
    ctx = sg.sg_init(-1)
    yield ctx
    sg.sg_destroy(ctx)


ADD = [("x", 0), ("x", 1), ("add",)]
MUL = [("x", 0), ("x", 1), ("mul",)]


def vec(sg, ctx, n, dt=None):
    return sg.sg_vector_create(ctx, sg.SG_F32 if dt is None else dt, n)


def lines(sg, ctx):
    return [l for l in sg.sg_plan_describe(ctx).splitlines() if l]


def test_dot_product_plans_to_one_kernel(sg, pctx):
    # Listing 5 / Fig. 2: compwise_multiply then sum -> one kernel, the
    # product is never stored
    a, b = vec(sg, pctx, 1000), vec(sg, pctx, 1000)
    t = sg.sg_zip(pctx, MUL, a, b)
    s = sg.sg_reduce(pctx, sg.SG_REDUCE_SUM, t)
    sg.sg_vector_release(t)
    L = lines(sg, pctx)
    assert len(L) == 1 and "store=0" in L[0] and "reduce=1" in L[0] and "in=2" in L[0], L
    sg.sg_scalar_release(s)


def test_axpy_rewrite_is_one_kernel(sg, pctx):
    # Fig. 3: smult then plus -> one kernel computing a*X[i] + Y[i]
    x, y = vec(sg, pctx, 4096), vec(sg, pctx, 4096)
    ax = sg.sg_map(pctx, [("c", 2.5), ("x", 0), ("mul",)], x)
    r = sg.sg_zip(pctx, ADD, ax, y)
    sg.sg_vector_release(ax)
    L = lines(sg, pctx)
    assert len(L) == 1 and "store=1" in L[0] and "in=2" in L[0], L
    sg.sg_set_fusion(pctx, sg.SG_FUSE_OFF)
    assert len(lines(sg, pctx)) == 2
    sg.sg_vector_release(r)


def test_vadd_sum_post_fused_and_unfused(sg, pctx):
    a, b = vec(sg, pctx, 1 << 20), vec(sg, pctx, 1 << 20)
    z = sg.sg_zip(pctx, ADD, a, b)
    sg.sg_ensure(pctx, z, sg.contract(sg.SG_C_FOR_ALL,
                                      [("x", 0), ("x", 1), ("x", 2), ("add",), ("eq",)],
                                      other=[a, b]))
    s = sg.sg_reduce(pctx, sg.SG_REDUCE_SUM, z)
    L = lines(sg, pctx)
    assert L == ["stream n=1048576 in=2 store=1 pred=1 reduce=1 ops=17"], L
    sg.sg_set_fusion(pctx, sg.SG_FUSE_OFF)
    L = lines(sg, pctx)
    assert len(L) == 3 and all(l.startswith("stream") for l in L), L
    sg.sg_scalar_release(s)


def test_filter_then_sum_becomes_masked_reduce(sg, pctx):
    x = vec(sg, pctx, 10000)
    y = sg.sg_map(pctx, [("x", 0), ("x", 0), ("c", 1.0), ("fma",)], x)
    k = sg.sg_filter(pctx, [("x", 0), ("c", 1.5), ("gt",)], y)
    sg.sg_vector_release(y)
    s = sg.sg_reduce(pctx, sg.SG_REDUCE_SUM, k)
    sg.sg_vector_release(k)
    L = lines(sg, pctx)
    assert len(L) == 1 and "reduce=1" in L[0] and "store=0" in L[0], L
    sg.sg_scalar_release(s)


def test_filter_postcondition_folded_into_the_filter(sg, pctx):
    """`Result.for_all(p)` (Sec. 4) on a queued filter's result runs in the
    same flush: folded into the specialised filter, which checks each kept
    item as it writes it, else as a pass over the filter's count."""
    if sg.sg_debug_jit_check_filter([("x", 0)])[0] != sg.SG_OK:
        pytest.skip("no NVRTC on this machine")
    x = vec(sg, pctx, 10000)
    pred = [("x", 0), ("c", 0.0), ("gt",)]
    post = sg.contract(sg.SG_C_FOR_ALL, [("x", 0), ("c", -1.0), ("gt",)])
    k = sg.sg_filter(pctx, pred, x)
    sg.sg_ensure(pctx, k, post)
    assert lines(sg, pctx) == ["filter n=10000 for_all=1"]
    sg.sg_set_fusion(pctx, sg.SG_FUSE_OFF)
    L = lines(sg, pctx)
    assert L[0] == "filter n=10000" and len(L) == 2, L
    assert L[1].startswith("stream n=10000 (the filter's count)") and "pred=1" in L[1], L
    sg.sg_set_fusion(pctx, sg.SG_FUSE_ON)
    sg.sg_set_codegen(pctx, sg.SG_CODEGEN_INTERPRET)
    L = lines(sg, pctx)
    assert L[0] == "filter n=10000" and len(L) == 2, L
    sg.sg_set_codegen(pctx, sg.SG_CODEGEN_SPECIALIZE)
    # exists, and a second filter's contract, are not folded into the first
    k2 = sg.sg_filter(pctx, pred, x)
    sg.sg_ensure(pctx, k2, sg.contract(sg.SG_C_EXISTS, [("x", 0), ("c", 0.5), ("gt",)]))
    L = lines(sg, pctx)
    assert L[0] == "filter n=10000 for_all=1" and L[1] == "filter n=10000", L
    assert L[2].startswith("stream n=10000 (the filter's count)") and len(L) == 3, L


def test_filter_kept_by_handle_is_compacted(sg, pctx):
    """A reduction of a kept filter result runs after the compaction, over
    the filter's count (read on the device), in a pass of its own."""
    x = vec(sg, pctx, 10000)
    k = sg.sg_filter(pctx, [("x", 0), ("c", 0.0), ("gt",)], x)
    s = sg.sg_reduce(pctx, sg.SG_REDUCE_SUM, k)
    s2 = sg.sg_reduce(pctx, sg.SG_REDUCE_MAX, k)
    L = lines(sg, pctx)
    assert L[0].startswith("filter n=10000") and len(L) == 3, L
    assert all(l.startswith("stream n=10000 (the filter's count)") for l in L[1:]), L
    sg.sg_scalar_release(s)
    sg.sg_scalar_release(s2)


def test_contract_mode_off_plans_no_check(sg, pctx):
    a = vec(sg, pctx, 100)
    sg.sg_set_contract_mode(pctx, sg.SG_CONTRACTS_OFF)
    sg.sg_require(pctx, a, sg.contract(sg.SG_C_FOR_ALL, [("x", 0), ("c", 0.0), ("ne",)]))
    assert lines(sg, pctx) == []
    sg.sg_set_contract_mode(pctx, sg.SG_CONTRACTS_PRE)
    sg.sg_ensure(pctx, a, sg.contract(sg.SG_C_FOR_ALL, [("x", 0), ("c", 0.0), ("ne",)]))
    assert lines(sg, pctx) == []
    sg.sg_require(pctx, a, sg.contract(sg.SG_C_FOR_ALL, [("x", 0), ("c", 0.0), ("ne",)]))
    assert len(lines(sg, pctx)) == 1


def test_sort_plans_fused_postconditions(sg, pctx):
    k = vec(sg, pctx, 1 << 20, sg.SG_I32)
    out = sg.sg_sort(pctx, k)
    assert lines(sg, pctx) == ["sort n=1048576 sorted=1 perm=1"]
    sg.sg_set_fusion(pctx, sg.SG_FUSE_OFF)
    assert lines(sg, pctx) == ["sort n=1048576 sorted=0 perm=0", "check_sorted n=1048576",
                               "check_perm n=1048576"]
    sg.sg_vector_release(out)


def test_scalar_contracts_on_host(sg, pctx):
    a, b = vec(sg, pctx, 10), vec(sg, pctx, 11)
    with pytest.raises(sg.SgError) as e:
        sg.sg_zip(pctx, ADD, a, b)
    assert e.value.status == sg.SG_ERR_SHAPE
    with pytest.raises(sg.SgError) as e:
        sg.sg_map(pctx, [("x", 0), ("add",)], a)
    assert e.value.status == sg.SG_ERR_INVALID_ARG
    with pytest.raises(sg.SgError) as e:
        sg.sg_map(pctx, [("x", 1)], a)
    assert e.value.status == sg.SG_ERR_INVALID_ARG
    i = vec(sg, pctx, 10, sg.SG_I32)
    with pytest.raises(sg.SgError) as e:
        sg.sg_map(pctx, [("x", 0)], i)
    assert e.value.status == sg.SG_ERR_DTYPE
    m1 = sg.sg_matrix_create(pctx, sg.SG_F32, 3, 4)
    m2 = sg.sg_matrix_create(pctx, sg.SG_F32, 5, 3)
    with pytest.raises(sg.SgError) as e:
        sg.sg_matmul(pctx, m1, m2)
    assert e.value.status == sg.SG_ERR_SHAPE


def test_planning_only_context_cannot_execute(sg, pctx):
    a = vec(sg, pctx, 10)
    s = sg.sg_reduce(pctx, sg.SG_REDUCE_SUM, a)
    with pytest.raises(sg.SgError) as e:
        sg.sg_flush(pctx)
    assert e.value.status == sg.SG_ERR_UNSUPPORTED


def test_async_transfers_on_a_planning_context(sg, pctx):
    """The asynchronous create / read need a device: a planning-only context
    refuses them with SG_ERR_UNSUPPORTED (nothing is enqueued) and sg_sync
    has nothing to wait for; bad arguments are rejected first."""
    import numpy as np
    host = np.zeros(16, np.float32)
    with pytest.raises(sg.SgError) as e:
        sg.sg_vector_create_async(pctx, sg.SG_F32, 16, host)
    assert e.value.status == sg.SG_ERR_UNSUPPORTED
    assert sg.lib.sg_vector_create_async(pctx, sg.SG_F32, -1, None, ctypes.byref(ctypes.c_void_p())) \
        == sg.SG_ERR_INVALID_ARG
    assert sg.lib.sg_vector_create_async(None, sg.SG_F32, 4, None, ctypes.byref(ctypes.c_void_p())) \
        == sg.SG_ERR_INVALID_ARG
    v = vec(sg, pctx, 16)
    with pytest.raises(sg.SgError) as e:
        sg.sg_vector_read_async(pctx, v, host)
    assert e.value.status == sg.SG_ERR_UNSUPPORTED
    with pytest.raises(sg.SgError) as e:
        sg.sg_vector_read_async(pctx, v, np.zeros(3, np.float32))
    assert e.value.status == sg.SG_ERR_SHAPE
    sg.sg_sync(pctx)
    assert sg.lib.sg_sync(None) == sg.SG_ERR_INVALID_ARG
    sg.sg_vector_release(v)


def test_portable_switch_arguments(sg, pctx):
    assert sg.lib.sg_debug_portable_kernels(None, 1) == sg.SG_ERR_INVALID_ARG
    sg.sg_debug_portable_kernels(pctx, True)
    sg.sg_debug_portable_kernels(pctx, False)


MALFORMED = [
    [("x", 0), ("gt",)],                                   # too few operands
    [("x", 0), ("x", 0)],                                  # two values left
    [("x", 1), ("c", 0.0), ("gt",)],                       # slot 1 of a one-input filter
    [("x", 0)] * 7 + [("add",)] * 6,                       # stack deeper than 6
]


@pytest.mark.parametrize("k", range(len(MALFORMED)))
def test_malformed_predicates_refused_alike(sg, pctx, k):
    """sg_filter and the allocation-free filter share one expression
    validator: every malformed predicate is refused by both, before any
    device work (the allocation-free call gets fake pointers here)."""
    pred = MALFORMED[k]
    v = vec(sg, pctx, 100)
    with pytest.raises(sg.SgError) as e1:
        sg.sg_filter(pctx, pred, v)
    with pytest.raises(sg.SgError) as e2:
        sg.sg_filter_noalloc(pred, 16, 100, 16, 16)
    assert e1.value.status == e2.value.status == sg.SG_ERR_INVALID_ARG
    sg.sg_vector_release(v)


def test_lookback_switch_arguments(sg, pctx):
    sg.sg_debug_lookback(pctx, 100, 3)
    sg.sg_debug_lookback(pctx, 0, -1)
    with pytest.raises(sg.SgError) as e:
        sg.sg_debug_lookback(pctx, 0, -2)
    assert e.value.status == sg.SG_ERR_INVALID_ARG


def test_schedule_family_arguments(sg, pctx):
    """The schedule chooser's per-family calls: nothing decided yet, bad
    families and indices refused, forgetting and forcing accepted."""
    for fam in (sg.SG_SCHED_BATCH, sg.SG_SCHED_STREAM, sg.SG_SCHED_FILTER, sg.SG_SCHED_PRODUCT,
                sg.SG_SCHED_FUSION):
        with pytest.raises(sg.SgError) as e:
            sg.sg_sched_last(pctx, fam)
        assert e.value.status == sg.SG_ERR_INVALID_ARG
        sg.sg_sched_forget(pctx, fam)
        sg.sg_sched_force(pctx, fam, 0)
        sg.sg_sched_force(pctx, fam, -1)
    sg.sg_sched_forget(pctx, -1)
    for bad in ((5, 0), (-1, 0), (0, -2), (0, sg.SG_SCHED_MAX_CANDIDATES)):
        with pytest.raises(sg.SgError) as e:
            sg.sg_sched_force(pctx, *bad)
        assert e.value.status == sg.SG_ERR_INVALID_ARG
    with pytest.raises(sg.SgError):
        sg.sg_sched_forget(pctx, 5)
    # an empty log trains nothing
    X, y, fam = sg.sg_sched_log(pctx)
    assert X.shape == (0, 12) and y.shape == (0,) and fam.shape == (0,)
