"""CPU check of run-time specialisation (Sec. 5: the kernel template
instantiated and compiled per call): the specialised filter kernel of each
predicate below compiles with NVRTC for sm_103a.  Only the compiler runs,
so no GPU is needed.  A predicate whose kernel failed to compile would still
filter correctly, through the interpreting kernel, so only this check shows
such a failure."""
import pytest

PREDICATES = [
    [("x", 0), ("c", 0.25), ("gt",)],
    [("x", 0), ("c", 5.0), ("lt",)],
    [("x", 0), ("abs",), ("c", 0.5), ("lt",), ("x", 0), ("c", -0.9), ("lt",), ("or",)],
    [("index",), ("c", 3.0), ("div",), ("dup",), ("c", 0.5), ("add",), ("c", 0.0), ("add",),
     ("swap",), ("sub",), ("c", 0.4), ("gt",)],
    [("x", 0), ("x", 0), ("mul",), ("c", 0.5), ("gt",)],
    [("x", 0), ("x", 0), ("ne",)],
    [("x", 0), ("c", 0.0), ("eq",)],
    [("x", 0)],
    [("x", 0), ("sqrt",), ("c", 0.5), ("ge",), ("not",)],
    [("x", 0), ("c", 2.0), ("c", 1.0), ("fma",), ("x", 0), ("c", -1.0), ("max",), ("le",)],
    [("x", 0), ("c", 0.0), ("lt",), ("c", 1.0), ("c", 0.0), ("select",)],
    [("x", 0), ("c", -0.5), ("ge",), ("x", 0), ("c", 0.5), ("le",), ("and",), ("not",)],
]


@pytest.fixture(scope="module")
def sg():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_6685_gb300 import safegpu
    return safegpu


@pytest.mark.parametrize("k", range(len(PREDICATES)))
def test_specialised_filter_compiles(sg, k):
    st, log = sg.sg_debug_jit_check_filter(PREDICATES[k])
    if st == sg.SG_ERR_UNSUPPORTED and "NVRTC library not found" in log:
        pytest.skip("no NVRTC on this machine")
    assert st == sg.SG_OK, log


def test_malformed_predicate_rejected(sg):
    st, _ = sg.sg_debug_jit_check_filter([("x", 0), ("add",)])
    assert st == sg.SG_ERR_INVALID_ARG
    st, _ = sg.sg_debug_jit_check_filter([("x", 1), ("c", 0.0), ("gt",)])
    assert st == sg.SG_ERR_INVALID_ARG


POSTS = [
    [("x", 0), ("c", 0.25), ("gt",)],
    [("index",), ("c", 100.0), ("lt",)],
    [("x", 0), ("x", 0), ("eq",), ("x", 0), ("abs",), ("c", 2.0), ("le",), ("and",)],
]


@pytest.mark.parametrize("k", range(len(POSTS)))
def test_specialised_filter_with_folded_postcondition_compiles(sg, k):
    st, log = sg.sg_debug_jit_check_filter_post(PREDICATES[k], POSTS[k])
    if st == sg.SG_ERR_UNSUPPORTED and "NVRTC library not found" in log:
        pytest.skip("no NVRTC on this machine")
    assert st == sg.SG_OK, log


def test_folded_postcondition_size_limit(sg):
    # the two programs share the 48 constant slots: 46 operations together
    pred = [("x", 0), ("abs",)] + [("c", 1.0), ("add",)] * 10 + [("c", 0.0), ("gt",)]
    post = [("x", 0)] + [("c", 1.0), ("add",)] * 10 + [("c", 0.0), ("gt",)]
    assert (len(pred), len(post)) == (24, 23)
    st, log = sg.sg_debug_jit_check_filter_post(pred, post[:-4] + [("c", 0.0), ("gt",)])
    if st == sg.SG_ERR_UNSUPPORTED and "NVRTC library not found" in log:
        pytest.skip("no NVRTC on this machine")
    assert st == sg.SG_OK, log          # 24 + 21 operations fold
    st, log = sg.sg_debug_jit_check_filter_post(pred, post)
    if st == sg.SG_ERR_UNSUPPORTED and "NVRTC library not found" in log:
        pytest.skip("no NVRTC on this machine")
    assert st == sg.SG_ERR_UNSUPPORTED and "folded" in log, log
