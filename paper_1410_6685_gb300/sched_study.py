"""Regret study of the schedule chooser's decision families.

For the stream pass's launch shape, the filter's tile, the product's tile
form and the fusion boundaries (sg_sched_family), sweeps of every candidate on training workloads fill
the context's timing log; sg_sched_train fits each family's 2x64 cost model
to it; then, on held-out workloads drawn from the same distribution with
another seed, the learned choice (predicted before the workload is measured)
and the plain table's choice are compared with the fastest candidate:

    regret(choice) = t(choice) / t(fastest) - 1,

t being the mean of two independent sweeps of the workload (the second after
sg_sched_forget), so that one noisy measurement does not decide.

Workloads (seeded, synthetic; uniform binary32 data in [-1, 1)):
  stream   one of four fused chains -- a + b summed; 2x + 1 stored; a
           for_all range check; a * b + c stored and summed -- over n
           elements, n = floor(2^u), u uniform in [10, 27]
  filter   one of three predicates (x > 0.25, x^2 < 0.04, x > -0.9: 37.5%,
           20% and 95% kept) over n elements, u uniform in [11, 27]
  product  C = A B in bf16 or fp16 with M, N, K each drawn from
           {128, 192, 256, 384, 512, 640, 768, 1024, 1536, 2048, 3072, 4096}
  fusion   one of three chains whose intermediates no handle keeps -- a + b
           summed; (2x + 1)^2 summed; a * b range-checked and summed -- over
           n elements, u uniform in [10, 27]: fused, one kernel; unfused, one
           kernel per call

    python -m paper_1410_6685_gb300.sched_study [--train T] [--heldout H]
"""
from __future__ import annotations

import json

import numpy as np

STREAM_CHAINS = 4
FILTER_PREDS = [
    [("x", 0), ("c", 0.25), ("gt",)],
    [("x", 0), ("x", 0), ("mul",), ("c", 0.04), ("lt",)],
    [("x", 0), ("c", -0.9), ("gt",)],
]
PRODUCT_DIMS = [128, 192, 256, 384, 512, 640, 768, 1024, 1536, 2048, 3072, 4096]
MAX_STREAM_N = 1 << 27


def draw(family, count, seed):
    """`count` workloads of `family`, seeded."""
    g = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        if family == "stream":
            out.append((int(g.integers(STREAM_CHAINS)), int(2.0 ** g.uniform(10, 27))))
        elif family == "fusion":
            out.append((4 + int(g.integers(3)), int(2.0 ** g.uniform(10, 27))))
        elif family == "filter":
            out.append((int(g.integers(len(FILTER_PREDS))), int(2.0 ** g.uniform(11, 27))))
        else:
            M, N, K = (int(g.choice(PRODUCT_DIMS)) for _ in range(3))
            out.append((M, N, K, 1 + int(g.integers(2))))
    return out


class Runner:
    """Runs one workload of a family through the library (one flush)."""

    def __init__(self, sg, ctx, torch):
        self.sg, self.ctx, self.torch = sg, ctx, torch
        self.vec = None
        self.mat = None

    def _vectors(self):
        if self.vec is None:
            t = self.torch
            g = t.Generator(device="cuda").manual_seed(41)
            self.vec = [t.rand(MAX_STREAM_N, device="cuda", generator=g) * 2 - 1
                        for _ in range(3)]
        return self.vec

    def _matrices(self):
        if self.mat is None:
            t = self.torch
            g = t.Generator(device="cuda").manual_seed(42)
            m = max(PRODUCT_DIMS)
            self.mat = [t.randn(m * m, device="cuda", generator=g) for _ in range(2)]
        return self.mat

    def stream(self, chain, n):
        sg, ctx = self.sg, self.ctx
        a, b, c = (sg.sg_vector_wrap(ctx, sg.SG_F32, n, v.data_ptr()) for v in self._vectors())
        rel = [a, b, c]
        if chain == 0:
            z = sg.sg_zip(ctx, [("x", 0), ("x", 1), ("add",)], a, b)
            s = sg.sg_reduce(ctx, sg.SG_REDUCE_SUM, z)
            sg.sg_scalar_get(ctx, s)
            sg.sg_scalar_release(s)
            rel.append(z)
        elif chain == 1:
            y = sg.sg_map(ctx, [("x", 0), ("c", 2.0), ("mul",), ("c", 1.0), ("add",)], a)
            sg.sg_flush(ctx)
            rel.append(y)
        elif chain == 2:
            f = sg.sg_for_all(ctx, [("x", 0), ("c", -2.0), ("gt",)], [a])
            sg.sg_scalar_get(ctx, f)
            sg.sg_scalar_release(f)
        elif chain == 3:
            y = sg.sg_mapn(ctx, [("x", 0), ("x", 1), ("mul",), ("x", 2), ("add",)], [a, b, c])
            s = sg.sg_reduce(ctx, sg.SG_REDUCE_SUM, y)
            sg.sg_scalar_get(ctx, s)
            sg.sg_scalar_release(s)
            rel.append(y)
        else:
            # the fusion family's chains: intermediates released before the
            # flush, so the fused plan stores nothing
            if chain == 4:
                z = sg.sg_zip(ctx, [("x", 0), ("x", 1), ("add",)], a, b)
                outs = [sg.sg_reduce(ctx, sg.SG_REDUCE_SUM, z)]
                mids = [z]
            elif chain == 5:
                y1 = sg.sg_map(ctx, [("x", 0), ("c", 2.0), ("mul",), ("c", 1.0), ("add",)], a)
                y2 = sg.sg_map(ctx, [("x", 0), ("x", 0), ("mul",)], y1)
                outs = [sg.sg_reduce(ctx, sg.SG_REDUCE_SUM, y2)]
                mids = [y1, y2]
            else:
                z = sg.sg_zip(ctx, [("x", 0), ("x", 1), ("mul",)], a, b)
                outs = [sg.sg_for_all(ctx, [("x", 0), ("c", -2.0), ("gt",)], [z]),
                        sg.sg_reduce(ctx, sg.SG_REDUCE_SUM, z)]
                mids = [z]
            for v in mids:
                sg.sg_vector_release(v)
            for o in outs:
                sg.sg_scalar_get(ctx, o)
                sg.sg_scalar_release(o)
        for v in rel:
            sg.sg_vector_release(v)

    def fusion(self, chain, n):
        self.stream(chain, n)

    def filter(self, pred, n):
        sg, ctx = self.sg, self.ctx
        x = sg.sg_vector_wrap(ctx, sg.SG_F32, n, self._vectors()[0].data_ptr())
        y = sg.sg_filter(ctx, FILTER_PREDS[pred], x)
        sg.sg_flush(ctx)
        sg.sg_vector_release(y)
        sg.sg_vector_release(x)

    def product(self, M, N, K, prec):
        sg, ctx = self.sg, self.ctx
        ta, tb = self._matrices()
        A = sg.sg_matrix_wrap(ctx, sg.SG_F32, M, K, ta.data_ptr())
        B = sg.sg_matrix_wrap(ctx, sg.SG_F32, K, N, tb.data_ptr())
        C = sg.sg_matmul(ctx, A, B, prec)
        sg.sg_flush(ctx)
        for m in (C, A, B):
            sg.sg_matrix_release(m)

    def run(self, family, w):
        getattr(self, family)(*w)


FAMILY_ID = {"stream": 1, "filter": 2, "product": 3, "fusion": 4}


def sweep(runner, family, w):
    """Measures every candidate of workload w twice; returns (mean times,
    plain index, learned index)."""
    sg, ctx = runner.sg, runner.ctx
    fid = FAMILY_ID[family]
    ts = []
    rep = None
    # a first run settles the other families' decisions in the same flush
    # (the fusion boundaries of a stream chain are measured on first sight)
    runner.run(family, w)
    for k in range(2):
        sg.sg_sched_forget(ctx, fid)
        runner.run(family, w)
        r = sg.sg_sched_last(ctx, fid)
        if k == 0:
            rep = r
        ts.append(np.array(r.measured_us[:r.ncand], dtype=np.float64))
    return (ts[0] + ts[1]) / 2, rep.default_index, rep.learned_index, rep


def study(sg, ctx, torch, families=("stream", "filter", "product", "fusion"), train=48, heldout=24,
          seed=5, epochs=400):
    """Trains on `train` swept workloads per family and reports the held-out
    regrets.  The context's scheduler is set to SG_SCHED_AUTOTUNE."""
    sg.sg_set_scheduler(ctx, sg.SG_SCHED_AUTOTUNE)
    runner = Runner(sg, ctx, torch)
    out = {}
    for fam in families:
        for w in draw(fam, train, seed):
            sg.sg_sched_forget(ctx, FAMILY_ID[fam])
            runner.run(fam, w)
    loss = sg.sg_sched_train(ctx, epochs=epochs, lr=3e-3, seed=7)
    for fam in families:
        rl, rp, changed = [], [], 0
        for w in draw(fam, heldout, seed + 1000):
            t, d, li, _ = sweep(runner, fam, w)
            best = t.min()
            rp.append(t[d] / best - 1)
            rl.append(t[li] / best - 1)
            changed += int(li != d)
        rl, rp = np.array(rl), np.array(rp)
        out[fam] = {
            "train": train, "heldout": heldout, "learned_differs": changed,
            "learned_mean_regret": round(float(rl.mean()), 4),
            "learned_median_regret": round(float(np.median(rl)), 4),
            "plain_mean_regret": round(float(rp.mean()), 4),
            "plain_median_regret": round(float(np.median(rp)), 4),
            "learned_worse": int((rl > rp + 1e-9).sum()),
            "learned_better": int((rl < rp - 1e-9).sum()),
        }
    out["train_loss"] = round(float(loss), 5)
    return out


def main(argv=None):
    import argparse
    import os
    import sys
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=48)
    ap.add_argument("--heldout", type=int, default=24)
    ap.add_argument("--families", default="stream,filter,product,fusion")
    ap.add_argument("--dump", default="", help="write every held-out sweep to this JSON file")
    a = ap.parse_args(argv)
    import torch
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    from paper_1410_6685_gb300 import build
    build.build()
    from paper_1410_6685_gb300 import safegpu as sg
    ctx = sg.sg_init(0, torch.cuda.current_stream().cuda_stream)
    fams = tuple(f for f in a.families.split(",") if f)
    res = study(sg, ctx, torch, fams, a.train, a.heldout)
    if a.dump:
        runner = Runner(sg, ctx, torch)
        rows = []
        for fam in fams:
            for w in draw(fam, a.heldout, 1005):
                t, d, li, r = sweep(runner, fam, w)
                rows.append({"family": fam, "w": list(w), "t": [round(x, 3) for x in t],
                             "chunk": list(r.chunk[:r.ncand]),
                             "ctas": list(r.ctas_per_sm[:r.ncand]), "plain": d, "learned": li})
        with open(a.dump, "w") as f:
            json.dump(rows, f)
    torch.cuda.synchronize()
    sg.sg_destroy(ctx)
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
