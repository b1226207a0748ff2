"""Run one named workload through the library and print per-kernel times.

A small command-line driver for measuring and profiling single kernels:

    python -m paper_1410_6685_gb300.workloads sort   [--n N] [--reps R] [--contracts on|off]
    python -m paper_1410_6685_gb300.workloads stream [--n N] [--reps R]
    python -m paper_1410_6685_gb300.workloads gemm   [--n N] [--reps R] [--prec 0|1|2]
    python -m paper_1410_6685_gb300.workloads solve  [--n N] [--reps R] [--prec 0|1|2]
    python -m paper_1410_6685_gb300.workloads batch  [--n collections] [--reps R]
    python -m paper_1410_6685_gb300.workloads filter [--n N] [--reps R]
    python -m paper_1410_6685_gb300.workloads transpose [--n N] [--reps R]

Each prints one JSON line: per kernel name, launches and mean milliseconds
(CUDA events bracketing each launch on the context's stream), plus the
workload's algorithmic bytes or flops per launch of its main kernel.
Inputs are the seeded synthetic workloads of `inputs`.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["sort", "stream", "gemm", "solve", "batch", "filter",
                                     "transpose"])
    ap.add_argument("--n", type=int, default=0)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--prec", type=int, default=1)
    ap.add_argument("--contracts", choices=["on", "off"], default="on",
                    help="off: contract mode SG_CONTRACTS_OFF (the unchecked schedule)")
    ap.add_argument("--post", action="store_true",
                    help="filter: also ensure Result.for_all(x > 0.25) on its result")
    a = ap.parse_args(argv)

    import torch
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    from paper_1410_6685_gb300 import build
    build.build()
    from paper_1410_6685_gb300 import inputs
    from paper_1410_6685_gb300 import safegpu as sg

    ctx = sg.sg_init(0, torch.cuda.current_stream().cuda_stream)
    if a.contracts == "off":
        sg.sg_set_contract_mode(ctx, sg.SG_CONTRACTS_OFF)
    keep = []
    out = {"case": a.case}

    def run(step):
        step()          # warm-up (and run-time specialisation, if any)
        sg.sg_profile_enable(ctx, True)
        sg.sg_profile_report(ctx, reset=True)
        for _ in range(a.reps):
            step()
        rep = sg.sg_profile_report(ctx, reset=True)
        sg.sg_profile_enable(ctx, False)
        return {k: (c, round(ms / c, 5)) for k, (c, ms) in rep.items()}

    if a.case == "sort":
        n = a.n or 1 << 26
        t = torch.from_numpy(inputs.sort_keys_uniform(n)).cuda()
        v = sg.sg_vector_wrap(ctx, sg.SG_I32, n, t.data_ptr())
        keep.append(t)

        def step():
            o = sg.sg_sort(ctx, v)
            sg.sg_flush(ctx)
            sg.sg_vector_release(o)
        out["kernels"] = run(step)
        out["bytes_per_onesweep_launch"] = 8 * n
    elif a.case in ("stream", "filter"):
        n = a.n or 1 << 28
        g = torch.Generator(device="cuda").manual_seed(0)
        x = torch.rand(n, device="cuda", generator=g) * 2 - 1
        y = torch.rand(n, device="cuda", generator=g) * 2 - 1
        vx, vy = sg.wrap_tensor(ctx, x), sg.wrap_tensor(ctx, y)
        keep += [x, y]
        if a.case == "stream":
            add = [("x", 0), ("x", 1), ("add",)]
            post = sg.contract(sg.SG_C_FOR_ALL, [("x", 0), ("x", 1), ("x", 2), ("add",), ("eq",)],
                               other=[vx, vy])

            def step():
                z = sg.sg_zip(ctx, add, vx, vy)
                sg.sg_ensure(ctx, z, post)
                s = sg.sg_reduce(ctx, sg.SG_REDUCE_SUM, z)
                sg.sg_scalar_get(ctx, s)
                sg.sg_vector_release(z)
                sg.sg_scalar_release(s)
            out["kernels"] = run(step)
            out["bytes_per_launch"] = 12 * n
        else:
            pred = [("x", 0), ("c", 0.25), ("gt",)]
            fpost = sg.contract(sg.SG_C_FOR_ALL, pred)

            def step():
                k = sg.sg_filter(ctx, pred, vx)
                if a.post:
                    sg.sg_ensure(ctx, k, fpost)
                sg.sg_vector_count(ctx, k)
                sg.sg_vector_release(k)
            out["kernels"] = run(step)
            out["bytes_per_launch"] = int(4 * n + 4 * n * 0.375)
    elif a.case == "gemm":
        n = a.n or 4096
        A = torch.randn(n, n, device="cuda")
        B = torch.randn(n, n, device="cuda")
        ma, mb = sg.wrap_tensor(ctx, A), sg.wrap_tensor(ctx, B)
        keep += [A, B]

        def step():
            c = sg.sg_matmul(ctx, ma, mb, a.prec)
            sg.sg_flush(ctx)
            sg.sg_matrix_release(c)
        out["kernels"] = run(step)
        out["flops_per_launch"] = 2 * n ** 3
    elif a.case == "solve":
        n = a.n or 2048
        A, b = inputs.gepp_inputs(n)
        ta, tb = torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda()
        ma, vb = sg.wrap_tensor(ctx, ta), sg.wrap_tensor(ctx, tb)
        keep += [ta, tb]
        o = sg.SgSolveOpts()
        o.precision, o.max_iter, o.refine_tol, o.residual_tol = a.prec, 30, 1e-14, 1e-12
        info_box = {}

        def step():
            x, info = sg.sg_solve(ctx, ma, vb, o)
            xs = sg.sg_vector_read(ctx, x, np.empty(n))
            sg.sg_vector_release(x)
            info_box.update(iterations=info.iterations, max_err=float(np.max(np.abs(xs - 1))))
        out["kernels"] = run(step)
        out.update(info_box)
    elif a.case == "batch":
        L = inputs.batch_lengths(a.n or 10000)
        off = inputs.batch_offsets(L)
        total = int(off[-1])
        g = torch.Generator(device="cuda").manual_seed(9)
        x = torch.rand(total, device="cuda", generator=g) * 2 - 1
        to = torch.from_numpy(off).cuda()
        nseg = len(L)
        outs = (torch.empty(nseg, dtype=torch.float64, device="cuda"),
                torch.empty(nseg, dtype=torch.int64, device="cuda"),
                torch.empty(nseg, dtype=torch.int64, device="cuda"))
        keep += [x, to, *outs]
        ch = sg.chain([("x", 0), ("x", 0), ("c", 1.0), ("fma",)], [("x", 0), ("c", 1.0), ("ge",)],
                      [("x", 0), ("c", 1.5), ("gt",)])

        def step():
            sg.sg_batch_run(ctx, ch, x.data_ptr(), to.data_ptr(), nseg,
                            *(t.data_ptr() for t in outs))
        out["kernels"] = run(step)
        out["bytes_per_launch"] = 4 * total + 24 * nseg
    elif a.case == "transpose":
        # Listing 1: transpose (materialised), then A^T x with the transpose
        # folded into the left product, then the right product A x
        n = a.n or 8192
        g = torch.Generator(device="cuda").manual_seed(12)
        A = torch.randn(n, n, device="cuda", generator=g)
        x = torch.randn(n, device="cuda", generator=g)
        mA, vx = sg.wrap_tensor(ctx, A), sg.wrap_tensor(ctx, x)
        keep += [A, x]

        def step():
            t = sg.sg_transpose(ctx, mA)
            sg.sg_flush(ctx)
            sg.sg_matrix_release(t)
            t = sg.sg_transpose(ctx, mA)
            y = sg.sg_matvec(ctx, t, vx)
            sg.sg_matrix_release(t)
            z = sg.sg_matvec(ctx, mA, vx)
            sg.sg_flush(ctx)
            sg.sg_vector_release(y)
            sg.sg_vector_release(z)
        out["kernels"] = run(step)
        out["bytes_per_transpose"] = 8 * n * n
        out["bytes_per_product"] = 4 * n * n
    torch.cuda.synchronize()
    sg.sg_destroy(ctx)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
