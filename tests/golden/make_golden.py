"""Writes the fixtures of this folder: the paper's worked examples with small
inputs chosen here.  The paper states what each example computes but prints
no data for it, so the expected values come from `oracle/` (this script
calls nothing else).  Each fixture cites the passage it restates.

    python tests/golden/make_golden.py

Float values are stored as the hex of their binary32 bit patterns (exact),
with a decimal copy for reading.
"""
import json
import os
import struct
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
import oracle  # noqa: E402

f32 = np.float32


def bits(a):
    a = np.ascontiguousarray(a, dtype=f32)
    return [format(struct.unpack("<I", struct.pack("<f", float(v)))[0], "08x") for v in a]


def vec(a):
    a = np.ascontiguousarray(a, dtype=f32)
    return {"bits": bits(a), "decimal": [repr(float(v)) for v in a]}


def fixtures():
    out = []
    # Sec. 3.1: c.filter (agent (a: INT) do Result := a < 5 end): the
    # elements less than five, in their order
    x = np.array([7, 3, 5, 1, 9, -2, 4, 5, 0, 12, -7, 4], dtype=f32)
    pred = [["x", 0], ["c", 5.0], ["lt"]]
    out.append({"name": "filter_less_than_five", "cite": "Sec. 3.1, the filter example (a < 5)",
                "op": "filter", "expr": pred, "in": [vec(x)],
                "out": vec(oracle.filter([tuple(o) for o in pred], x))})
    # Sec. 3.1: c.for_each (agent (a: INT) do a := a * 2 end): every element
    # doubled, in place
    x = np.array([1, -3, 0, 21, 1024, -6, 7, 2], dtype=f32)
    ex = [["x", 0], ["c", 2.0], ["mul"]]
    out.append({"name": "for_each_double", "cite": "Sec. 3.1, the for_each example (a := a * 2)",
                "op": "for_each", "expr": ex, "in": [vec(x)],
                "out": vec(oracle.map([tuple(o) for o in ex], x))})
    # Sec. 3.1: c.project (agent (a: INT): DOUBLE do Result := sqrt (a) end)
    # (binary32 here): the square root of each element, a new collection
    x = np.array([0, 1, 4, 9, 2, 16, 100, 3], dtype=f32)
    ex = [["x", 0], ["sqrt"]]
    out.append({"name": "project_sqrt", "cite": "Sec. 3.1, the project example (sqrt (a))",
                "op": "map", "expr": ex, "in": [vec(x)],
                "out": vec(oracle.map([tuple(o) for o in ex], x))})
    # Listing 5: a.compwise_multiply (b).sum, the dot product (one fused
    # kernel, Sec. 5)
    a = np.array([1, 2, 3, 4, 5, 6, 7, 8], dtype=f32)
    b = np.array([8, -7, 6, -5, 4, -3, 2, 1], dtype=f32)
    mul = [["x", 0], ["x", 1], ["mul"]]
    s = oracle.sum(oracle.map([tuple(o) for o in mul], a, b))
    out.append({"name": "dot_product", "cite": "Listing 5, dot product (compwise_multiply, sum)",
                "op": "zip_sum", "expr": mul, "in": [vec(a), vec(b)],
                "out": {"sum": repr(float(s))}})
    # Listing 3: v1.compwise_divide (v2), precondition v2.for_all (item /= 0),
    # postcondition: Result * v2 equals v1 (within rounding)
    a = np.array([1, -4, 9, 2.5, 0, 7, -1, 3], dtype=f32)
    b = np.array([2, 8, -3, 0.5, 5, 7, 4, 6], dtype=f32)
    div = [["x", 0], ["x", 1], ["div"]]
    pre = [["x", 0], ["c", 0.0], ["ne"]]
    out.append({"name": "compwise_divide", "cite": "Listing 3, compwise_divide and its contracts",
                "op": "zip", "expr": div, "pre_on_second": pre, "in": [vec(a), vec(b)],
                "out": vec(oracle.map([tuple(o) for o in div], a, b)),
                "pre_first_false": oracle.first_false([tuple(o) for o in pre], b)})
    # Listing 4: quicksort by three filters and two concatenations; its
    # postconditions: the result is sorted and has the input's count
    x = np.array([5, -1, 3, 3, 0, 8, -7, 2, 5, 1], dtype=f32)
    out.append({"name": "quicksort", "cite": "Listing 4, quicksort (is_sorted, count)",
                "op": "sort", "in": [vec(x)], "out": vec(oracle.sort_f32(x)),
                "first_unsorted_of_input": oracle.first_unsorted_f32(x)})
    # Sec. 5: aX + Y computed by adjusting the addition kernel (X[i] + Y[i]
    # becomes a*X[i] + Y[i]; a = 3 here)
    xv = np.array([1, 2, 3, 4, -1, -2, 0.5, 10], dtype=f32)
    yv = np.array([10, 20, 30, 40, 1, 2, 0.25, -30], dtype=f32)
    axpy = [["c", 3.0], ["x", 0], ["mul"], ["x", 1], ["add"]]
    out.append({"name": "axpy", "cite": "Sec. 5, the aX + Y rewrite (a = 3)",
                "op": "zip", "expr": axpy, "in": [vec(xv), vec(yv)],
                "out": vec(oracle.map([tuple(o) for o in axpy], xv, yv))})
    return out


def main():
    for fx in fixtures():
        path = os.path.join(HERE, fx["name"] + ".json")
        with open(path, "w") as f:
            # one key per line, compact values
            f.write("{\n" + ",\n".join(" %s: %s" % (json.dumps(k), json.dumps(v))
                                        for k, v in fx.items()) + "\n}\n")
        print("wrote", path)


if __name__ == "__main__":
    main()
