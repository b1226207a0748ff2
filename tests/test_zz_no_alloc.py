"""GPU test of sg_filter_noalloc, the filter for callers that cannot allocate
device memory: a serving runtime that has reserved all of HBM in its own
pool, a latency-critical path that cannot take an allocation's
synchronisation, a plugin host that hands out only the input and output
buffers.  Its scratch is a fixed array in the library's device memory.

It is called through the C ABI on caller-owned buffers and must give, bit
for bit, what the oracle's filter gives and what the ordinary sg_filter
gives, on calls in a row -- each smaller than the one before, so that state
an earlier call leaves in the shared array would show -- with an empty
input, a whole number of tiles, a predicate deep enough for the second
kernel, and an unaligned input.  Once both kernels have been loaded, the
device's free memory must not change across the calls.  Collected last on
purpose: a failure here stops a -x run only after every other test has
run."""
import numpy as np
import pytest

import oracle
from paper_1410_6685_gb300 import inputs

pytestmark = pytest.mark.gpu

GT = [("x", 0), ("c", 0.25), ("gt",)]
ABS_LT = [("x", 0), ("abs",), ("c", 0.5), ("lt",)]
# stack depth 5 (the interpreting kernel's deeper instantiation):
# x > 0.5 * (x + x * 0.25)
DEEP = [("x", 0), ("c", 0.5), ("x", 0), ("x", 0), ("c", 0.25), ("mul",), ("add",), ("mul",),
        ("gt",)]

# (n, predicate, seed, offset of the input view in elements)
CALLS = [
    (1_000_003, GT, 101, 0),
    (300_001, ABS_LT, 102, 0),
    (200_003, GT, 104, 1),        # x[1:]: not 16-byte aligned
    (4096 * 37, DEEP, 103, 0),    # a whole number of 4096-item tiles
    (4097, DEEP, 105, 1),
    (0, GT, 106, 0),
]


def _env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_6685_gb300 import safegpu as sg
    return torch, sg


def _call(torch, sg, pred, tx, n, out, cnt, stream):
    xp = tx.data_ptr() if n else 0
    sg.sg_filter_noalloc(pred, xp, n, out.data_ptr(), cnt.data_ptr(), stream)
    return int(cnt.item())


def test_noalloc_filter_matches_oracle_and_filter_on_calls_in_a_row():
    torch, sg = _env()
    stream = torch.cuda.current_stream().cuda_stream
    nmax = max(c[0] for c in CALLS) + 1
    out = torch.empty(nmax, dtype=torch.float32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int64, device="cuda")
    data = {}
    for n, pred, seed, off in CALLS:
        x = inputs.uniform_pm1(inputs.rng(seed), n + off)
        data[seed] = (x, torch.from_numpy(x).cuda())

    # warm-up: one shallow and one deep predicate load both kernels (and
    # the array) before free memory is measured
    w = data[101][1]
    _call(torch, sg, GT, w, 1000, out, cnt, stream)
    _call(torch, sg, DEEP, w, 1000, out, cnt, stream)
    torch.cuda.synchronize()

    # the calls in a row, each with the free memory around it
    results = []
    for n, pred, seed, off in CALLS:
        tx = data[seed][1][off:]
        out.fill_(float("nan"))
        cnt.fill_(-7)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        m = _call(torch, sg, pred, tx, n, out, cnt, stream)
        free1 = torch.cuda.mem_get_info()[0]
        assert free1 == free0, "the call took device memory"
        results.append((m, out[:m].cpu().numpy().copy()))

    for (n, pred, seed, off), (m, got) in zip(CALLS, results):
        xs = data[seed][0][off:]
        ref = oracle.filter(pred, xs)
        assert m == len(ref)
        assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
        # and the ordinary entry point on the same input
        if n:
            tx = data[seed][1][off:]
            ctx = sg.sg_init(0, stream)
            try:
                v = sg.sg_vector_wrap(ctx, sg.SG_F32, n, tx.data_ptr())
                k = sg.sg_filter(ctx, pred, v)
                ref_m = sg.sg_vector_count(ctx, k)
                lib = sg.sg_vector_read(ctx, k, np.empty(ref_m, np.float32))
            finally:
                sg.sg_destroy(ctx)
            assert ref_m == m
            assert np.array_equal(lib.view(np.uint32), got.view(np.uint32))


def test_noalloc_filter_rejects_sizes_beyond_its_array():
    torch, sg = _env()
    with pytest.raises(sg.SgError) as e:
        sg.sg_filter_noalloc(GT, 16, sg.SG_FILTER_NOALLOC_MAX_N + 1, 16, 16)
    assert e.value.status == sg.SG_ERR_SHAPE
    # a malformed predicate is refused by the same validator sg_filter uses
    with pytest.raises(sg.SgError) as e:
        sg.sg_filter_noalloc([("x", 0), ("gt",)], 16, 16, 16, 16)
    assert e.value.status == sg.SG_ERR_INVALID_ARG
