"""GPU test of sg_filter_noalloc, the filter for callers that cannot allocate
device memory (its scratch is a fixed array in the library's device memory).
It is called through the C ABI on caller-owned buffers and must give exactly
what the ordinary sg_filter gives, on two calls in a row -- the second
smaller than the first, so that state the first call leaves in the shared
array would show.  Collected last on purpose: a failure here stops a -x run
only after every other test has run."""
import numpy as np
import pytest

from paper_1410_6685_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_noalloc_filter_matches_filter_on_two_calls():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_6685_gb300 import safegpu as sg

    stream = torch.cuda.current_stream().cuda_stream
    calls = [
        (1_000_003, [("x", 0), ("c", 0.25), ("gt",)], 101),
        (300_001, [("x", 0), ("abs",), ("c", 0.5), ("lt",)], 102),
    ]
    for n, pred, seed in calls:
        x = inputs.uniform_pm1(inputs.rng(seed), n)
        tx = torch.from_numpy(x).cuda()
        out = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
        cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda")
        sg.sg_filter_noalloc(pred, tx.data_ptr(), n, out.data_ptr(), cnt.data_ptr(), stream)
        m = int(cnt.item())

        ctx = sg.sg_init(0, stream)
        try:
            v = sg.sg_vector_wrap(ctx, sg.SG_F32, n, tx.data_ptr())
            k = sg.sg_filter(ctx, pred, v)
            ref_m = sg.sg_vector_count(ctx, k)
            ref = sg.sg_vector_read(ctx, k, np.empty(ref_m, np.float32))
        finally:
            sg.sg_destroy(ctx)
        assert m == ref_m
        got = out[:m].cpu().numpy()
        assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_noalloc_filter_rejects_sizes_beyond_its_array():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_6685_gb300 import safegpu as sg
    with pytest.raises(sg.SgError) as e:
        sg.sg_filter_noalloc([("x", 0), ("c", 0.0), ("gt",)], 16, sg.SG_FILTER_NOALLOC_MAX_N + 1,
                             16, 16)
    assert e.value.status == sg.SG_ERR_SHAPE
