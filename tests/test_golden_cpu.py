"""The fixtures in tests/golden/ (the paper's worked examples with small
inputs: Sec. 3.1 filter / for_each / project, Listing 3 compwise_divide,
Listing 4 quicksort, Listing 5 dot product, Sec. 5 aX + Y).  Their expected
values were written by tests/golden/make_golden.py from the oracle; here they
are checked against what each passage says the example computes, worked out
with plain numpy and Python, and the oracle is checked to reproduce them."""
import glob
import json
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")
f32 = np.float32


def load(name):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        return json.load(f)


def arr(v):
    return np.array([int(b, 16) for b in v["bits"]], dtype=np.uint32).view(f32)


def same_bits(a, b):
    return a.shape == b.shape and np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_every_fixture_cites_a_passage():
    files = sorted(glob.glob(os.path.join(GOLDEN, "*.json")))
    assert len(files) == 7
    for p in files:
        d = json.load(open(p))
        assert d["cite"].startswith(("Sec.", "Listing")), p
        for v in d["in"]:
            assert np.array_equal(arr(v), np.array([float(s) for s in v["decimal"]], dtype=f32))


def test_filter_less_than_five():
    d = load("filter_less_than_five")
    x = arr(d["in"][0])
    assert same_bits(arr(d["out"]), np.array([v for v in x if v < 5], dtype=f32))


def test_for_each_double():
    d = load("for_each_double")
    assert same_bits(arr(d["out"]), arr(d["in"][0]) * f32(2))


def test_project_sqrt():
    d = load("project_sqrt")
    assert same_bits(arr(d["out"]), np.sqrt(arr(d["in"][0])))


def test_dot_product_exact():
    d = load("dot_product")
    a, b = arr(d["in"][0]), arr(d["in"][1])
    exact = sum(int(p) * int(q) for p, q in zip(a, b))   # small integers: exact
    assert float(d["out"]["sum"]) == exact == 16


def test_compwise_divide_and_its_contracts():
    d = load("compwise_divide")
    a, b = arr(d["in"][0]), arr(d["in"][1])
    r = arr(d["out"])
    assert same_bits(r, a / b)                            # correctly rounded binary32
    assert d["pre_first_false"] == -1 and all(v != 0 for v in b)
    # Result * v2 = v1 within one rounding of the quotient and one of the product
    assert np.all(np.abs(r.astype(np.float64) * b - a) <= 2 * np.finfo(f32).eps * np.abs(a) + 1e-30)


def test_quicksort_postconditions():
    d = load("quicksort")
    x, out = arr(d["in"][0]), arr(d["out"])
    assert same_bits(out, np.array(sorted(x), dtype=f32))
    assert len(out) == len(x)
    first = next((i for i in range(len(x) - 1) if x[i] > x[i + 1]), -1)
    assert d["first_unsorted_of_input"] == first == 0


def test_axpy_two_roundings():
    d = load("axpy")
    xv, yv = arr(d["in"][0]), arr(d["in"][1])
    assert same_bits(arr(d["out"]), (f32(3) * xv) + yv)


def test_oracle_reproduces_the_fixtures():
    sys.path.insert(0, GOLDEN)
    import make_golden
    for fx in make_golden.fixtures():
        stored = load(fx["name"])
        assert json.loads(json.dumps(fx)) == stored, fx["name"]
