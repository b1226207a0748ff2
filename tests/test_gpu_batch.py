"""GPU parity of the batched collections (many collections of uneven size
through one persistent launch replayed from a CUDA graph), each running
map(x*x+1) -> require for_all(y >= 1) -> filter(y > 1.5) -> sum, through the
C ABI.  Kept counts and first-violation indices must be identical to the
oracle's; sums within 1e-5 relative or the kernel's binary32-pair bound."""
import numpy as np
import pytest

import oracle
from paper_1410_6685_gb300 import inputs

pytestmark = pytest.mark.gpu

MAP = [("x", 0), ("x", 0), ("c", 1.0), ("fma",)]
PRE = [("x", 0), ("c", 1.0), ("ge",)]
KEEP = [("x", 0), ("c", 1.5), ("gt",)]


@pytest.fixture(scope="module", params=["specialize", "interpret"])
def env(request):
    """Both forms of the batch kernel: the program compiled at run time into
    straight-line code, and the interpreting kernel."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_6685_gb300 import safegpu as sg
    ctx = sg.sg_init(0, torch.cuda.current_stream().cuda_stream)
    sg.sg_set_codegen(ctx, sg.SG_CODEGEN_SPECIALIZE if request.param == "specialize"
                      else sg.SG_CODEGEN_INTERPRET)
    yield sg, ctx, torch
    sg.sg_destroy(ctx)


def run(env, x, off, chain=None, expect_status=None):
    sg, ctx, torch = env
    nseg = len(off) - 1
    tx = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    to = torch.from_numpy(np.ascontiguousarray(off)).cuda()
    sums = torch.empty(nseg, dtype=torch.float64, device="cuda")
    fv = torch.empty(nseg, dtype=torch.int64, device="cuda")
    kept = torch.empty(nseg, dtype=torch.int64, device="cuda")
    ch = chain or sg.chain(MAP, PRE, KEEP)
    args = (ctx, ch, tx.data_ptr(), to.data_ptr(), nseg, sums.data_ptr(), fv.data_ptr(),
            kept.data_ptr())
    if expect_status is None:
        sg.sg_batch_run(*args)
    else:
        with pytest.raises(sg.SgError) as e:
            sg.sg_batch_run(*args)
        assert e.value.status == expect_status
    return sums.cpu().numpy(), fv.cpu().numpy(), kept.cpu().numpy(), (tx, to, sums, fv, kept, args)


def sums_ok(got, ref, x, off):
    for s in range(len(ref)):
        seg = x[off[s]:off[s + 1]].astype(np.float64)
        scale = np.abs(seg * seg + 1).sum() if len(seg) else 0.0
        assert abs(got[s] - ref[s]) <= max(1e-5 * abs(ref[s]), 2.0 ** -22 * scale), s


def test_small_ragged_batch(env):
    L = np.array([0, 1, 2, 3, 4, 5, 63, 64, 65, 1000, 16384, 16385, 40000, 7])
    off = inputs.batch_offsets(L)
    x = inputs.batch_data(int(off[-1]), seed=31)
    sums, fv, kept, _ = run(env, x, off)
    rs, rf, rk = oracle.batch_chain(MAP, PRE, KEEP, x, off)
    assert np.array_equal(kept, rk) and np.array_equal(fv, rf)
    sums_ok(sums, rs, x, off)


def test_precondition_violations_reported_per_collection(env):
    sg, ctx, _ = env
    L = np.array([100, 20000, 50000, 10, 33333])
    off = inputs.batch_offsets(L)
    x = inputs.batch_data(int(off[-1]), seed=32)
    plants = [(1, 19999), (1, 5), (2, 40000), (4, 0)]
    for s, k in plants:
        x[off[s] + k] = np.nan
    sums, fv, kept, _ = run(env, x, off, expect_status=sg.SG_ERR_PRECONDITION)
    rs, rf, rk = oracle.batch_chain(MAP, PRE, KEEP, x, off)
    assert list(rf) == [-1, 5, 40000, -1, 0]
    assert np.array_equal(fv, rf) and np.array_equal(kept, rk)


def test_contracts_off_skips_the_precondition(env):
    """Contract mode OFF (Sec. 6.3): the precondition is not evaluated, so
    the planted NaNs are not reported (every first index -1, no error); the
    kept counts and sums are the oracle's all the same.  Back in PRE_POST
    the same batch reports them again (a separately captured graph)."""
    sg, ctx, _ = env
    L = np.array([100, 20000, 50000, 10, 33333])
    off = inputs.batch_offsets(L)
    x = inputs.batch_data(int(off[-1]), seed=33)
    x[off[1] + 5] = np.nan
    x[off[4]] = np.nan
    sg.sg_set_contract_mode(ctx, sg.SG_CONTRACTS_OFF)
    try:
        sums, fv, kept, _ = run(env, x, off)
    finally:
        sg.sg_set_contract_mode(ctx, sg.SG_CONTRACTS_PRE_POST)
    rs, rf, rk = oracle.batch_chain(MAP, PRE, KEEP, x, off)
    assert list(fv) == [-1] * 5
    assert np.array_equal(kept, rk)
    for s in range(len(L)):     # a NaN is never kept (NaN > 1.5 is false)
        seg = x[off[s]:off[s + 1]].astype(np.float64)
        scale = np.nansum(np.abs(seg * seg + 1))
        assert abs(sums[s] - rs[s]) <= max(1e-5 * abs(rs[s]), 2.0 ** -22 * scale), s
    sums2, fv2, kept2, _ = run(env, x, off, expect_status=sg.SG_ERR_PRECONDITION)
    assert np.array_equal(fv2, rf) and list(rf) == [-1, 5, -1, -1, 0]


def test_graph_replay_is_deterministic(env):
    sg, ctx, _ = env
    L = inputs.batch_lengths(500, seed=40, hi_log2=16)
    off = inputs.batch_offsets(L)
    x = inputs.batch_data(int(off[-1]), seed=41)
    sums1, fv1, kept1, keep = run(env, x, off)
    tx, to, s_t, f_t, k_t, args = keep
    sg.sg_batch_run(*args)            # replay of the cached graph
    assert np.array_equal(s_t.cpu().numpy(), sums1)
    tx.mul_(-1.0)                     # new data under the same pointers
    sg.sg_batch_run(*args)
    assert np.array_equal(k_t.cpu().numpy(), kept1)     # x*x is unchanged by a sign flip
    rs, rf, rk = oracle.batch_chain(MAP, PRE, KEEP, -x, off)
    sums_ok(s_t.cpu().numpy(), rs, -x, off)


def test_other_chains(env):
    sg, _, _ = env
    L = np.array([5000, 1, 77777, 4096])
    off = inputs.batch_offsets(L)
    x = inputs.batch_data(int(off[-1]), seed=42) * np.float32(4)
    chains = [([("x", 0), ("abs",), ("sqrt",)], [("x", 0), ("c", 1.5), ("le",)],
               [("index",), ("c", 2.0), ("div",), ("dup",), ("c", 0.5), ("add",), ("c", 0.0),
                ("add",), ("swap",), ("sub",), ("c", 0.25), ("lt",)]),
              ([("x", 0), ("c", 0.5), ("sub",)], [("x", 0), ("x", 0), ("eq",)],
               [("x", 0), ("c", 0.0), ("lt",)])]
    for m, p, k in chains:
        sums, fv, kept, _ = run(env, x, off, chain=sg.chain(m, p, k),
                                expect_status=None if m[1][0] == "c" else sg.SG_ERR_PRECONDITION)
        rs, rf, rk = oracle.batch_chain(m, p, k, x, off)
        assert np.array_equal(kept, rk) and np.array_equal(fv, rf)


def test_full_size_workload_sampled(env):
    """10,000 collections, lengths log-uniform in [2^6, 2^20] (about 1.08e9
    elements); the oracle checks a seeded sample of 300 collections."""
    L = inputs.batch_lengths()
    off = inputs.batch_offsets(L)
    x = inputs.batch_data(int(off[-1]))
    sums, fv, kept, keep = run(env, x, off)
    del keep
    pick = np.random.default_rng(5).choice(len(L), 300, replace=False)
    for s in pick:
        o2 = np.array([0, L[s]], dtype=np.int64)
        rs, rf, rk = oracle.batch_chain(MAP, PRE, KEEP, x[off[s]:off[s + 1]], o2)
        assert kept[s] == rk[0] and fv[s] == rf[0]
        sums_ok([sums[s]], rs, x[off[s]:off[s + 1]], o2)
    assert np.all(fv == -1)
