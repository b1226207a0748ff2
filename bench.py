#!/usr/bin/env python3
"""Benchmark of the contract-checked sort path on GB300.

A step is one pass of the hot path over one batch: sg_sort of 2^26 uniform
int32 keys (full signed range) with its built-in postconditions
(Result.is_sorted and Result is a permutation of the input, Listing 4 of the
paper) fused into the last radix pass, and the flush that reads the contract
verdict back.  `value` is whole-job GB/s counted as 36 bytes per key (the
algorithmic traffic of an 8-bit LSD onesweep sort: one histogram read plus
four read+write passes).  Inputs are resident in HBM and larger than L2
(268 MB > 126 MB), so no L2 flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 run under torch.distributed.run: each rank sorts its own keys (weak
scaling, no data-path collective; a barrier and a max over ranks frame the
timed region).  `--impl reference` times the CPU oracle on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_KEYS = 1 << 26
BYTES_PER_KEY = 36
METRIC = "fused collection+contract GB/s (% HBM peak); GEMM TFLOP/s; contract overhead %"
WORKLOAD = ("sort int32 n=2^26 uniform full range, postconditions sorted + permutation "
            "fused into the last onesweep pass")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [v for v in vis.split(",") if v.strip()]
        self.gpu = ids[local_rank] if local_rank < len(ids) and ids[local_rank].isdigit() \
            else str(local_rank)
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-i", self.gpu, "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [l.split(",") for l in self.f.read().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_step(keys):
    """The oracle's version of one step: sort, then both postconditions."""
    import oracle
    out = oracle.sort_i32(keys)
    ok_sorted = oracle.first_unsorted_i32(out) == -1
    ok_perm = oracle.same_multiset_i32(keys, out)
    assert ok_sorted and ok_perm
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_1410_6685_gb300 import inputs
    oracle.build()
    sample = 1 << 22
    keys = inputs.sort_keys_uniform(sample)
    for _ in range(args.warmup):
        oracle_step(keys)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(keys)
    dt = (time.perf_counter() - t0) / args.steps
    v = BYTES_PER_KEY * sample / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": sample, "bytes_per_key": BYTES_PER_KEY},
        "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": "2^22 uniform int32 keys per step: C qsort + is_sorted + "
                                   "multiset equality (the oracle as it stands)"},
        "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_KEYS)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
        return

    import numpy as np
    import torch
    import __graft_entry__
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    __graft_entry__.build()
    from paper_1410_6685_gb300 import inputs
    from paper_1410_6685_gb300 import safegpu as sg

    n = args.n
    stream = torch.cuda.current_stream()
    ctx = sg.sg_init(local, stream.cuda_stream)
    keys = inputs.sort_keys_uniform(n, seed=1 + rank)
    tk = torch.from_numpy(keys).cuda()
    vk = sg.sg_vector_wrap(ctx, sg.SG_I32, n, tk.data_ptr())

    def step():
        out = sg.sg_sort(ctx, vk)
        sg.sg_flush(ctx)
        sg.sg_vector_release(out)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def timed(k):
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1)
        if world > 1:
            import torch.distributed as dist
            t = torch.tensor([ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms / k

    for _ in range(args.warmup):
        step()
    # timed region (kernel tracing on: events bracket each launch on `stream`)
    clocks = Clocks(local)
    sg.sg_profile_enable(ctx, True)
    sg.sg_profile_report(ctx, reset=True)
    k0 = sg.sg_kernel_count(ctx)
    clocks.start()
    ms = timed(args.steps)
    clk = clocks.stop()
    launches = sg.sg_kernel_count(ctx) - k0
    prof = sg.sg_profile_report(ctx, reset=True)
    sg.sg_profile_enable(ctx, False)

    # contract overhead: the same steps with checking off
    sg.sg_set_contract_mode(ctx, sg.SG_CONTRACTS_OFF)
    for _ in range(2):
        step()
    ms_off = timed(args.steps)
    sg.sg_set_contract_mode(ctx, sg.SG_CONTRACTS_PRE_POST)

    # end to end through the C ABI with host buffers (pinned)
    hk = torch.from_numpy(keys).pin_memory()
    hout = torch.empty(n, dtype=torch.int32).pin_memory()
    hk_np, hout_np = hk.numpy(), hout.numpy()

    def e2e_step():
        v = sg.sg_vector_create(ctx, sg.SG_I32, n, hk_np)
        out = sg.sg_sort(ctx, v)
        sg.sg_vector_read(ctx, out, hout_np)
        sg.sg_vector_release(out)
        sg.sg_vector_release(v)

    e2e_step()
    ke = max(3, min(args.steps, 10))
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ke):
        e2e_step()
    torch.cuda.synchronize()
    t_e2e = (time.perf_counter() - t0) / ke
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([t_e2e], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_e2e = float(t.item())
    assert np.array_equal(hout_np[:1000], np.sort(keys)[:1000])

    if rank != 0:
        sg.sg_destroy(ctx)
        return

    peak, peak_kind = peaks()
    value = world * BYTES_PER_KEY * n / (ms / 1e3) / 1e9
    roof = None
    if "onesweep" in prof:
        cnt, tot = prof["onesweep"]
        dur = tot / cnt / 1e3
        achieved = 8.0 * n / dur / 1e9
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None,
                "kernel": "k_onesweep (passes 1-3; 8 bytes/key read+write)",
                "peak_kind": peak_kind + " hbm_gbs (copy bandwidth)"}
    cpu = None
    if world == 1:
        import oracle
        oracle.build()
        sample = 1 << 24
        sk = keys[:sample].copy()
        t0 = time.perf_counter()
        oracle_step(sk)
        dt = time.perf_counter() - t0
        cpu = {"value": round(BYTES_PER_KEY * sample / dt / 1e9, 4), "unit": "GB/s", "cores": 1,
               "kind": "oracle",
               "sample": "first 2^24 keys of the same workload, one step: C qsort + is_sorted + "
                         "multiset equality, single thread"}
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "bytes_per_key": BYTES_PER_KEY,
                   "l2": "inputs larger than L2 (268 MB keys vs 126 MB L2), no flush",
                   "contracts": "pre_post, fused", "parallelism": "replicas" if world > 1 else "1 GPU"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": round(world * BYTES_PER_KEY * n / t_e2e / 1e9, 2), "unit": "GB/s",
                "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 4 * n,
                "api": "sg_vector_create(host) -> sg_sort -> sg_vector_read(host), pinned"},
        "clocks": clk,
        "gpu_launches": launches,
        "extras": {
            "keys_per_s": round(world * n / (ms / 1e3), 1),
            "contract_overhead_pct": round((ms / ms_off - 1.0) * 100.0, 2),
            "ms_per_step_contracts_off": round(ms_off, 4),
            "per_kernel_ms": {k: round(v[1] / v[0], 5) for k, v in prof.items()},
            "per_kernel_launches": {k: v[0] for k, v in prof.items()},
        },
    }
    print(json.dumps(line), flush=True)
    sg.sg_destroy(ctx)


if __name__ == "__main__":
    main()
