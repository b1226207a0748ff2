#!/usr/bin/env python3
"""Benchmark of the contract-checked sort path on GB300.

A step is one pass of the hot path over one batch: sg_sort of 2^26 uniform
int32 keys (full signed range) with its built-in postconditions
(Result.is_sorted and Result is a permutation of the input, Listing 4 of the
paper) fused into the last radix pass, and the flush that reads the contract
results back.  `value` is whole-job GB/s counted as 36 bytes per key (the
algorithmic traffic of an 8-bit LSD onesweep sort: one histogram read plus
four read+write passes).  Inputs are resident in HBM and larger than L2
(268 MB > 126 MB), so no L2 flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 run under torch.distributed.run: each rank sorts its own keys (weak
scaling, no data-path collective; a barrier and a max over ranks frame the
timed region).  `--impl reference` times the CPU oracle on a bounded sample.

After the headline, rank 0 also reports the other parts of the metric under
`extras.secondary` (skip with --no-extras): the fused zip + for_all + sum
stream at n = 2^28 (GB/s, fraction of HBM, contract overhead), the bf16
tcgen05 GEMM at 8192^2 with its Freivalds postcondition (TFLOP/s, contract
overhead), GEPP at n = 8192 with refinement, the sort's second variant
(2^26 keys from 256 distinct values), the transpose of 8192^2 and the
transposed matrix-vector product of Listing 1, and the batch of 10,000
collections.
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


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one
# k_onesweep digit pass over 2^26 keys, from an ncu capture of the sort
# kernels, valid only for the kernel source it was taken on (its SHA-256
# prefix); for any other source the roofline reports no traffic.
ONESWEEP_TRAFFIC = {"k_sort.cu": "6b00e4b654c0ca82", "n": 1 << 26, "bytes": 269313280 + 222068736}


def onesweep_traffic(n):
    import hashlib
    path = os.path.join(ROOT, "paper_1410_6685_gb300", "csrc", "k_sort.cu")
    try:
        with open(path, "rb") as f:
            h = hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None
    if h != ONESWEEP_TRAFFIC["k_sort.cu"] or n != ONESWEEP_TRAFFIC["n"]:
        return None
    return ONESWEEP_TRAFFIC["bytes"]


def peaks():
    """(HBM GB/s, bf16 TFLOP/s burst, kind): the measured copy bandwidth and
    cuBLAS bf16 rate of this GPU model, else the fallback figures."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


def sustained_tc_peak():
    """bf16 TFLOP/s of a seconds-long cuBLAS loop (for kernels timed inside a
    long step), else the burst figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p.get("bf16_tflops_sustained", p["bf16_tflops"]))
    except Exception:
        return 1700.0


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, world, device):
    """The largest x over all ranks (the slowest rank sets the job's time);
    x itself with one rank.  device: where the process group's backend
    reduces ("cuda" for NCCL, "cpu" for gloo)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gbs(world, bytes_per_rank, seconds):
    """Whole-job throughput: every rank's bytes over the slowest rank's time
    (weak scaling: each rank sorts its own keys)."""
    return world * bytes_per_rank / seconds / 1e9


def rank_seed(rank):
    """Each replica sorts different keys: the workload's seed plus its rank."""
    return 1 + rank


class Clocks:
    """SM clock and clock-event reasons sampled during the timed region.

    NVML through ctypes every ~2 ms when libnvidia-ml is loadable (the timed
    region lasts milliseconds), else nvidia-smi every 200 ms from just before
    to just after the region."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank, torch=None):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [v for v in vis.split(",") if v.strip()]
        self.gpu = ids[local_rank] if local_rank < len(ids) and ids[local_rank].isdigit() \
            else str(local_rank)
        self.local_rank = local_rank
        self.torch = torch
        self.samples, self.mx, self.reasons = [], 0.0, set()
        self.nvml = self._nvml_handle()
        self.proc = self.f = self.thread = None
        self.running = False

    def _nvml_handle(self):
        try:
            import ctypes
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return None
            dev = ctypes.c_void_p()
            bus = None
            if self.torch is not None:
                pr = self.torch.cuda.get_device_properties(self.local_rank)
                if all(hasattr(pr, k) for k in ("pci_domain_id", "pci_bus_id", "pci_device_id")):
                    bus = "%08X:%02X:%02X.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
            if bus is not None:
                rc = lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(dev))
            else:
                rc = lib.nvmlDeviceGetHandleByIndex_v2(int(self.gpu), ctypes.byref(dev))
            if rc != 0:
                return None
            mx = ctypes.c_uint()
            if lib.nvmlDeviceGetMaxClockInfo(dev, 1, ctypes.byref(mx)) == 0:
                self.mx = float(mx.value)
            fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
            return (lib, dev, fn)
        except Exception:
            return None

    def _poll(self):
        import ctypes
        lib, dev, fn = self.nvml
        clk, rs = ctypes.c_uint(), ctypes.c_ulonglong()
        while self.running:
            if lib.nvmlDeviceGetClockInfo(dev, 1, ctypes.byref(clk)) == 0:
                self.samples.append(float(clk.value))
            if fn(dev, ctypes.byref(rs)) == 0:
                for bit, name in self.REASONS.items():
                    if rs.value & bit:
                        self.reasons.add(name)
            time.sleep(0.002)

    def start(self):
        if self.nvml:
            import threading
            self.running = True
            self.thread = threading.Thread(target=self._poll, daemon=True)
            self.thread.start()
            while not self.samples and self.thread.is_alive():
                time.sleep(0.001)
            return
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-i", self.gpu, "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
            t0 = time.time()
            while time.time() - t0 < 3.0 and os.path.getsize(self.f.name) == 0:
                time.sleep(0.02)
        except Exception:
            self.proc = None

    def stop(self):
        if self.thread is not None:
            time.sleep(0.004)
            self.running = False
            self.thread.join()
            if not self.samples:
                return None
            return {"sm_mhz": statistics.median(self.samples), "sm_max_mhz": self.mx,
                    "reasons": sorted(self.reasons), "samples": len(self.samples),
                    "source": "nvml"}
        if not self.proc:
            return None
        size0 = os.path.getsize(self.f.name)
        t0 = time.time()
        while time.time() - t0 < 1.0 and os.path.getsize(self.f.name) == size0:
            time.sleep(0.02)   # one sample after the region
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
                "samples": len(sm), "source": "nvidia-smi, 200 ms, from just before to just after"}


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
    sample = args.ref_sample
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
        "config": {"workload": WORKLOAD, "n": args.n, "bytes_per_key": BYTES_PER_KEY,
                   "sample_keys_per_step": sample},
        "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": "%d uniform int32 keys per step: C qsort + is_sorted + "
                                   "multiset equality (the oracle as it stands)" % sample},
        "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def time_steps(torch, stream, step, k):
    """Mean device milliseconds of `step` over k calls (CUDA events on `stream`)."""
    step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(k):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / k


def fusion_plan(sg, ctx):
    """The plan the last fusion-boundary decision ran: "fused" (Sec. 5's
    merges) or "unfused (autotuned)"."""
    try:
        r = sg.sg_sched_last(ctx, sg.SG_SCHED_FUSION)
    except sg.SgError:
        return "fused"
    return "fused" if r.chosen_index == 0 else "unfused (autotuned)"


def with_contracts_off(sg, ctx, fn):
    sg.sg_set_contract_mode(ctx, sg.SG_CONTRACTS_OFF)
    try:
        return fn()
    finally:
        sg.sg_set_contract_mode(ctx, sg.SG_CONTRACTS_PRE_POST)


def secondary_workloads(torch, sg, ctx, stream, k, hbm_peak, tc_peak):
    """The other rows of the metric, each on its own synthetic workload:
    the fused zip+reduce+for_all stream, the bf16 tensor-core GEMM with its
    Freivalds postcondition, GEPP with iterative refinement, the sort of keys
    from 256 distinct values, transpose and the folded A^T x of Listing 1,
    filter, and the batched chain with its learned schedule.  Every figure is device time from CUDA events; the overhead of
    contract checking is the ratio of the same steps with checking on and off."""
    import numpy as np
    from paper_1410_6685_gb300 import inputs
    out = {}
    g = torch.Generator(device="cuda")

    # 1. zip(+) -> ensure for_all(z = x + y) -> reduce(sum), n = 2^28, one fused pass
    n = 1 << 28
    g.manual_seed(0)
    x = torch.rand(n, device="cuda", generator=g) * 2 - 1
    y = torch.rand(n, device="cuda", generator=g) * 2 - 1
    vx, vy = sg.wrap_tensor(ctx, x), sg.wrap_tensor(ctx, y)
    add = [("x", 0), ("x", 1), ("add",)]
    post = sg.contract(sg.SG_C_FOR_ALL, [("x", 0), ("x", 1), ("x", 2), ("add",), ("eq",)],
                       other=[vx, vy])

    def s_stream():
        z = sg.sg_zip(ctx, add, vx, vy)
        sg.sg_ensure(ctx, z, post)
        r = sg.sg_reduce(ctx, sg.SG_REDUCE_SUM, z)
        sg.sg_scalar_get(ctx, r)
        sg.sg_vector_release(z)
        sg.sg_scalar_release(r)
    ms = time_steps(torch, stream, s_stream, k)
    plan = fusion_plan(sg, ctx)
    ms_off = with_contracts_off(sg, ctx, lambda: time_steps(torch, stream, s_stream, k))
    gbs = 12.0 * n / (ms / 1e3) / 1e9     # read x, y; write z
    out["stream_zip_sum_forall"] = {
        "n": n, "ms": round(ms, 4), "GBps": round(gbs, 1), "frac_hbm": round(gbs / hbm_peak, 4),
        "bytes_per_elem": 12, "contract_overhead_pct": round((ms / ms_off - 1) * 100, 2), "plan": plan}
    sg.sg_vector_release(vx)
    sg.sg_vector_release(vy)
    del x, y

    # 2. matmul 8192^2, bf16 operands on tcgen05, f32 accumulate, Freivalds (4 vectors)
    N = 8192
    g.manual_seed(4)
    A = torch.randn(N, N, device="cuda", generator=g)
    B = torch.randn(N, N, device="cuda", generator=g)
    ma, mb = sg.wrap_tensor(ctx, A), sg.wrap_tensor(ctx, B)

    def s_mm():
        c = sg.sg_matmul(ctx, ma, mb, sg.SG_PREC_BF16_TC)
        sg.sg_flush(ctx)
        sg.sg_matrix_release(c)
    sg.sg_profile_enable(ctx, True)
    sg.sg_profile_report(ctx, reset=True)
    ms = time_steps(torch, stream, s_mm, k)
    prof = sg.sg_profile_report(ctx, reset=True)
    sg.sg_profile_enable(ctx, False)
    ms_off = with_contracts_off(sg, ctx, lambda: time_steps(torch, stream, s_mm, k))
    kern = {kk: round(v[1] / v[0], 4) for kk, v in prof.items()}
    g_ms = kern.get("gemm_tc_bf16")
    out["gemm_bf16_8192"] = {
        "ms_step": round(ms, 4), "TFLOPs_step": round(2 * N ** 3 / (ms / 1e3) / 1e12, 1),
        "TFLOPs_gemm_kernel": round(2 * N ** 3 / (g_ms / 1e3) / 1e12, 1) if g_ms else None,
        "frac_tensor_gemm_kernel": round(2 * N ** 3 / (g_ms / 1e3) / 1e12 / tc_peak, 4)
        if g_ms else None,
        "per_kernel_ms": kern, "contract_overhead_pct": round((ms / ms_off - 1) * 100, 2)}
    sg.sg_matrix_release(ma)
    sg.sg_matrix_release(mb)
    del A, B

    # 3. GEPP n = 8192, bf16 trailing updates, binary64 refinement + residual check
    n = 8192
    An, bn = inputs.gepp_inputs(n)
    ta, tb = torch.from_numpy(An).cuda(), torch.from_numpy(bn).cuda()
    mA, vb = sg.wrap_tensor(ctx, ta), sg.wrap_tensor(ctx, tb)
    o = sg.SgSolveOpts()
    o.precision, o.max_iter, o.refine_tol, o.residual_tol = sg.SG_PREC_BF16_TC, 30, 1e-14, 1e-12
    info_box = {}

    def s_solve():
        xs, info = sg.sg_solve(ctx, mA, vb, o)
        info_box["it"] = info.iterations
        sg.sg_vector_release(xs)
    ms, kern = profiled(sg, ctx, lambda: time_steps(torch, stream, s_solve, 2))
    it_bf16 = info_box.get("it")
    # the plain form: every update in binary32 on the CUDA cores
    o.precision = sg.SG_PREC_F32_SIMT
    ms32, kern32 = profiled(sg, ctx, lambda: time_steps(torch, stream, s_solve, 2))
    fl = 2 / 3 * n ** 3
    f_ms, f32_ms = kern.get("lu_factor_graph"), kern32.get("lu_factor_graph")
    out["solve_gepp_8192"] = {"ms": round(ms, 3), "iterations": it_bf16,
                              "GFLOPs": round(fl / (ms / 1e3) / 1e9, 1),
                              "factor_ms": round(f_ms, 3) if f_ms else None,
                              "LU_TFLOPs": round(fl / (f_ms / 1e3) / 1e12, 2) if f_ms else None,
                              "LU_frac_of_sustained_bf16":
                                  round(fl / (f_ms / 1e3) / 1e12 / sustained_tc_peak(), 4)
                                  if f_ms else None,
                              "plain_f32_ms": round(ms32, 3),
                              "plain_f32_factor_ms": round(f32_ms, 3) if f32_ms else None,
                              "plain_f32_iterations": info_box.get("it"),
                              "speedup_mixed_over_plain": round(ms32 / ms, 3)}
    sg.sg_matrix_release(mA)
    sg.sg_vector_release(vb)
    del ta, tb

    # 3b. the sort's second variant: 2^26 keys from 256 distinct values
    nk = 1 << 26
    tk = torch.from_numpy(inputs.sort_keys_distinct(nk)).cuda()
    vk = sg.sg_vector_wrap(ctx, sg.SG_I32, nk, tk.data_ptr())

    def s_sort_distinct():
        o = sg.sg_sort(ctx, vk)
        sg.sg_flush(ctx)
        sg.sg_vector_release(o)
    ms_d = time_steps(torch, stream, s_sort_distinct, k)
    out["sort_256_distinct_2e26"] = {
        "ms": round(ms_d, 4), "GBps": round(36.0 * nk / (ms_d / 1e3) / 1e9, 1),
        "keys_per_s": round(nk / (ms_d / 1e3), 1), "bytes_per_key": 36}
    sg.sg_vector_release(vk)
    del tk

    # 4. Listing 1: transpose of 8192^2 (materialised), and A^T x with the
    #    transpose folded into the left product (A read once)
    n = 8192
    g.manual_seed(12)
    tA = torch.randn(n, n, device="cuda", generator=g)
    tx = torch.randn(n, device="cuda", generator=g)
    mA, vx = sg.wrap_tensor(ctx, tA), sg.wrap_tensor(ctx, tx)

    def s_transpose():
        t = sg.sg_transpose(ctx, mA)
        sg.sg_flush(ctx)
        sg.sg_matrix_release(t)

    def s_listing1():
        t = sg.sg_transpose(ctx, mA)
        y = sg.sg_matvec(ctx, t, vx)
        sg.sg_matrix_release(t)
        sg.sg_flush(ctx)
        sg.sg_vector_release(y)
    ms_t = time_steps(torch, stream, s_transpose, k)
    ms_l = time_steps(torch, stream, s_listing1, k)
    out["transpose_8192"] = {"ms": round(ms_t, 4), "GBps": round(8.0 * n * n / (ms_t / 1e3) / 1e9, 1),
                             "frac_hbm": round(8.0 * n * n / (ms_t / 1e3) / 1e9 / hbm_peak, 4),
                             "bytes_per_elem": 8}
    out["listing1_transpose_matvec_8192"] = {
        "ms": round(ms_l, 4), "GBps": round(4.0 * n * n / (ms_l / 1e3) / 1e9, 1),
        "frac_hbm": round(4.0 * n * n / (ms_l / 1e3) / 1e9 / hbm_peak, 4), "bytes_per_elem": 4,
        "plan": "transpose folded into x^T A (never materialised)"}
    sg.sg_matrix_release(mA)
    sg.sg_vector_release(vx)
    del tA, tx

    # 4b. filter x > 0.25 of 2^28 uniform [-1, 1) binary32 values (37.5% kept),
    #     with the count read back: one decoupled look-back compaction pass
    n = 1 << 28
    g.manual_seed(5)
    fx = torch.rand(n, device="cuda", generator=g) * 2 - 1
    vf = sg.wrap_tensor(ctx, fx)
    fcount = {}

    def s_filter():
        kf = sg.sg_filter(ctx, [("x", 0), ("c", 0.25), ("gt",)], vf)
        fcount["m"] = sg.sg_vector_count(ctx, kf)
        sg.sg_vector_release(kf)
    sg.sg_profile_enable(ctx, True)
    sg.sg_profile_report(ctx, reset=True)
    ms_f = time_steps(torch, stream, s_filter, k)
    prof = sg.sg_profile_report(ctx, reset=True)
    sg.sg_profile_enable(ctx, False)
    fk = "filter_jit" if "filter_jit" in prof else "filter"
    kf_ms = prof[fk][1] / prof[fk][0] if fk in prof else None
    fb = 4.0 * n + 4.0 * fcount["m"]      # read every item, write the kept ones
    out["filter_2e28"] = {
        "n": n, "kept": int(fcount["m"]), "ms_step": round(ms_f, 4),
        "GBps_step": round(fb / (ms_f / 1e3) / 1e9, 1),
        "kernel": fk, "kernel_ms": round(kf_ms, 4) if kf_ms else None,
        "frac_hbm_kernel": round(fb / (kf_ms / 1e3) / 1e9 / hbm_peak, 4) if kf_ms else None,
        "bytes": "4 per item + 4 per kept item"}
    sg.sg_vector_release(vf)
    del fx

    # 5. 10,000 collections (log-uniform lengths), map -> filter -> sum, one launch
    L = inputs.batch_lengths()
    off = inputs.batch_offsets(L)
    total = int(off[-1])
    g.manual_seed(9)
    xb = torch.rand(total, device="cuda", generator=g) * 2 - 1
    to = torch.from_numpy(off).cuda()
    nseg = len(L)
    outs = (torch.empty(nseg, dtype=torch.float64, device="cuda"),
            torch.empty(nseg, dtype=torch.int64, device="cuda"),
            torch.empty(nseg, dtype=torch.int64, device="cuda"))
    ch = sg.chain([("x", 0), ("x", 0), ("c", 1.0), ("fma",)], [("x", 0), ("c", 1.0), ("ge",)],
                  [("x", 0), ("c", 1.5), ("gt",)])

    def s_batch():
        sg.sg_batch_run(ctx, ch, xb.data_ptr(), to.data_ptr(), nseg, *(t.data_ptr() for t in outs))
    ms = time_steps(torch, stream, s_batch, k)
    gbs = (4.0 * total + 24 * nseg) / (ms / 1e3) / 1e9
    out["batch_10000"] = {"elements": total, "ms": round(ms, 4), "GBps": round(gbs, 1),
                          "frac_hbm": round(gbs / hbm_peak, 4)}

    # 6. schedule of that batch: the 2x64 MLP cost model, trained on the GPU on
    #    autotuner sweeps of 40 other synthetic batches of the family it serves
    #    (1,000-10,000 collections, log-uniform lengths, at most 4e8 elements;
    #    never this one), against the plain table and the autotuner's best
    rng = np.random.default_rng(12)
    sg.sg_set_scheduler(ctx, sg.SG_SCHED_AUTOTUNE)
    for _ in range(40):
        lo = int(rng.integers(6, 10))
        hi = int(rng.integers(14, 21))
        ns = int(rng.integers(1000, 10001))
        while ns * (2.0 ** hi - 2.0 ** lo) / ((hi - lo) * np.log(2)) > 4e8:
            ns = ns * 3 // 4
        ns = max(ns, 16)
        Ls = np.floor(2.0 ** (lo + (hi - lo) * rng.random(ns))).astype(np.int64)
        offs = inputs.batch_offsets(Ls)
        xs = torch.rand(max(int(offs[-1]), 1), device="cuda") * 2 - 1
        ts = torch.from_numpy(offs).cuda()
        os_ = (torch.empty(ns, dtype=torch.float64, device="cuda"),
               torch.empty(ns, dtype=torch.int64, device="cuda"),
               torch.empty(ns, dtype=torch.int64, device="cuda"))
        sg.sg_batch_run(ctx, ch, xs.data_ptr(), ts.data_ptr(), ns, *(t.data_ptr() for t in os_))
        del xs, ts, os_
    t0 = time.perf_counter()
    loss = sg.sg_sched_train(ctx, epochs=400, lr=3e-3, seed=7)
    t_train = time.perf_counter() - t0
    r = sg.sg_batch_report(ctx, ch, xb.data_ptr(), to.data_ptr(), nseg, *(t.data_ptr() for t in outs))
    t_us = np.array(r.measured_us[:r.ncand])
    best = float(t_us.min())
    out["batch_10000_schedule"] = {
        "candidates": int(r.ncand),
        "plain_table_ms": round(t_us[r.default_index] / 1e3, 4),
        "learned_ms": round(t_us[r.learned_index] / 1e3, 4),
        "autotuned_best_ms": round(best / 1e3, 4),
        "regret_plain": round(t_us[r.default_index] / best - 1, 4),
        "regret_learned": round(t_us[r.learned_index] / best - 1, 4),
        "learned_choice": {"chunk": int(r.chunk[r.learned_index]),
                           "ctas_per_sm": int(r.ctas_per_sm[r.learned_index])},
        "train_records": int(sg.sg_sched_log(ctx)[1].shape[0]), "train_loss": round(loss, 5),
        "train_s": round(t_train, 2)}

    # 7. the other decision families -- the stream pass's launch shape, the
    #    filter's tile, the product's tile form: held-out regret of the
    #    learned choice and of the plain table (sched_study: 40 swept training
    #    workloads per family, 16 held-out ones each timed by two sweeps), in
    #    a context of its own
    from paper_1410_6685_gb300 import sched_study
    sctx = sg.sg_init(torch.cuda.current_device(), stream.cuda_stream)
    try:
        t0 = time.perf_counter()
        fam = sched_study.study(sg, sctx, torch, train=40, heldout=16)
        fam["study_s"] = round(time.perf_counter() - t0, 1)
    finally:
        sg.sg_destroy(sctx)
    out["schedule_families"] = fam
    return out


def profiled(sg, ctx, fn):
    """Runs fn with per-kernel event tracing: (result, {kernel: mean ms})."""
    sg.sg_profile_enable(ctx, True)
    sg.sg_profile_report(ctx, reset=True)
    try:
        r = fn()
        prof = sg.sg_profile_report(ctx, reset=True)
    finally:
        sg.sg_profile_enable(ctx, False)
    return r, {kk: v[1] / v[0] for kk, v in prof.items()}


def cpu_time(fn, reps=1):
    """Seconds of one call of a CPU oracle function (best of reps)."""
    best = 1e300
    for _ in range(reps):
        t0 = time.perf_counter()
        fn()
        best = min(best, time.perf_counter() - t0)
    return best


def per_config_workloads(torch, sg, ctx, stream, k, hbm_peak, tc_peak, tc_sustained):
    """Every configuration of the benchmark plan as stated (vector add + sum
    at 2^20 on the plain unfused path; GEMM at N = 1024 / 4096 / 8192 in the
    three forms; GEPP + refinement at n = 2048 / 8192 in the three update
    precisions; the batched chain and the filter with and without their
    contracts), each with its contract overhead (the same steps with checking
    off) and the oracle timed on one host core on a stated sample."""
    import numpy as np
    import oracle
    from paper_1410_6685_gb300 import inputs
    oracle.build()
    res = {}

    # config 1: a + b, ensure for_all(z = a + b), sum; n = 2^20, plain unfused
    # path (one kernel per call; the postcondition re-reads a, b and z)
    n = 1 << 20
    a, b = inputs.vadd_inputs(n)
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    va, vb = sg.wrap_tensor(ctx, ta), sg.wrap_tensor(ctx, tb)
    add = [("x", 0), ("x", 1), ("add",)]
    post = sg.contract(sg.SG_C_FOR_ALL, [("x", 0), ("x", 1), ("x", 2), ("add",), ("eq",)],
                       other=[va, vb])

    def s_vadd():
        z = sg.sg_zip(ctx, add, va, vb)
        sg.sg_ensure(ctx, z, post)
        r = sg.sg_reduce(ctx, sg.SG_REDUCE_SUM, z)
        sg.sg_scalar_get(ctx, r)
        sg.sg_vector_release(z)
        sg.sg_scalar_release(r)
    row = {}
    for fusion, name in ((sg.SG_FUSE_OFF, "unfused"), (sg.SG_FUSE_ON, "fused")):
        sg.sg_set_fusion(ctx, fusion)
        try:
            ms = time_steps(torch, stream, s_vadd, 4 * k)
            plan = "unfused" if fusion == sg.SG_FUSE_OFF else fusion_plan(sg, ctx)
            ms_off = with_contracts_off(sg, ctx, lambda: time_steps(torch, stream, s_vadd, 4 * k))
        finally:
            sg.sg_set_fusion(ctx, sg.SG_FUSE_ON)
        row[name] = {"ms": round(ms, 4), "GBps_12B": round(12.0 * n / (ms / 1e3) / 1e9, 1),
                     "plan": plan, "ms_contracts_off": round(ms_off, 4),
                     "contract_overhead_pct": round((ms / ms_off - 1) * 100, 2)}
    t_cpu = cpu_time(lambda: (oracle.sum(oracle.map(add, a, b)),
                              oracle.first_false([("x", 0), ("x", 1), ("x", 2), ("add",), ("eq",)],
                                                 a, b, oracle.map(add, a, b))), 3)
    row["oracle"] = {"ms": round(t_cpu * 1e3, 3), "cores": 1,
                     "sample": "the same n = 2^20 (map, for_all, binary64 sum)"}
    row["note"] = "12.6 MB working set: L2-resident, launch-bound; HBM fractions are claimed at 2^28"
    res["1_vadd_sum_2e20"] = row
    sg.sg_vector_release(va)
    sg.sg_vector_release(vb)
    del ta, tb

    # config 2 (second variant): the oracle on keys from 256 distinct values
    ks = inputs.sort_keys_distinct(1 << 22)
    t_cpu = cpu_time(lambda: oracle_step(ks))
    res["2_sort_256_distinct_oracle"] = {
        "GBps": round(BYTES_PER_KEY * len(ks) / t_cpu / 1e9, 4), "cores": 1,
        "sample": "2^22 keys: C qsort + is_sorted + multiset equality"}

    # config 3: C = A B, N(0,1), N in {1024, 4096, 8192}, binary32 SIMT and
    # bf16 / fp16 operands on the tensor cores; built-in Freivalds check
    names = {sg.SG_PREC_F32_SIMT: ("f32_simt", "gemm_f32_simt"),
             sg.SG_PREC_BF16_TC: ("bf16_tc", "gemm_tc_bf16"),
             sg.SG_PREC_F16_TC: ("f16_tc", "gemm_tc_f16")}
    for N in (1024, 4096, 8192):
        A, B = inputs.matmul_inputs(N)
        tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        ma, mb = sg.wrap_tensor(ctx, tA), sg.wrap_tensor(ctx, tB)
        for prec, (pname, kname) in names.items():
            def s_mm():
                c = sg.sg_matmul(ctx, ma, mb, prec)
                sg.sg_flush(ctx)
                sg.sg_matrix_release(c)
            kk = k if N > 1024 else 4 * k
            ms, kern = profiled(sg, ctx, lambda: time_steps(torch, stream, s_mm, kk))
            ms_off = with_contracts_off(sg, ctx, lambda: time_steps(torch, stream, s_mm, kk))
            g_ms = kern.get(kname)
            fl = 2.0 * N ** 3
            ent = {"ms_step": round(ms, 4), "TFLOPs_step": round(fl / (ms / 1e3) / 1e12, 1),
                   "kernel_ms": round(g_ms, 4) if g_ms else None,
                   "TFLOPs_kernel": round(fl / (g_ms / 1e3) / 1e12, 1) if g_ms else None,
                   "ms_contracts_off": round(ms_off, 4),
                   "contract_overhead_pct": round((ms / ms_off - 1) * 100, 2),
                   "per_kernel_ms": {x: round(v, 4) for x, v in kern.items()}}
            if prec != sg.SG_PREC_F32_SIMT and g_ms:
                # fp16 and bf16 share the nominal dense rate: the measured bf16 peak
                ent["frac_tensor_kernel"] = round(fl / (g_ms / 1e3) / 1e12 / tc_peak, 4)
            res["3_gemm_%d_%s" % (N, pname)] = ent
        # the binary64 oracle on one core: the whole product at 1024, 16 rows above
        rows = np.arange(N) if N == 1024 else np.arange(16)
        t_cpu = cpu_time(lambda: oracle.matmul_rows_f64(A, B, rows))
        res["3_gemm_%d_oracle" % N] = {
            "GFLOPs": round(2.0 * len(rows) * N * N / t_cpu / 1e9, 3), "cores": 1,
            "sample": "%d of %d rows of C, binary64" % (len(rows), N)}
        sg.sg_matrix_release(ma)
        sg.sg_matrix_release(mb)
        del tA, tB

    # config 4: GEPP + binary64 refinement, diagonally dominant, b = A 1,
    # n in {2048, 8192}, trailing updates in binary32 / bf16 / fp16; the
    # residual postcondition on and off
    for n in (2048, 8192):
        An, bn = inputs.gepp_inputs(n)
        tA, tb = torch.from_numpy(An).cuda(), torch.from_numpy(bn).cuda()
        mA, vb = sg.wrap_tensor(ctx, tA), sg.wrap_tensor(ctx, tb)
        for prec, pname in ((sg.SG_PREC_F32_SIMT, "f32_simt"), (sg.SG_PREC_BF16_TC, "bf16_tc"),
                            (sg.SG_PREC_F16_TC, "f16_tc")):
            o = sg.SgSolveOpts()
            o.precision, o.max_iter, o.refine_tol, o.residual_tol = prec, 30, 1e-14, 1e-12
            box = {}

            def s_solve():
                xs, info = sg.sg_solve(ctx, mA, vb, o)
                box["it"] = info.iterations
                box["x"] = xs
            def s_solve_rel():
                s_solve()
                sg.sg_vector_release(box.pop("x"))
            kk = 3 if n > 2048 else 6
            ms, kern = profiled(sg, ctx, lambda: time_steps(torch, stream, s_solve_rel, kk))
            ms_off = with_contracts_off(sg, ctx, lambda: time_steps(torch, stream, s_solve_rel, kk))
            s_solve()
            xs = sg.sg_vector_read(ctx, box["x"], np.empty(n))
            sg.sg_vector_release(box.pop("x"))
            f_ms = kern.get("lu_factor_graph")
            fl = 2.0 / 3.0 * n ** 3
            res["4_solve_%d_%s" % (n, pname)] = {
                "ms": round(ms, 3), "iterations": box.get("it"),
                "max_abs_x_minus_1": float(np.max(np.abs(xs - 1.0))),
                "factor_ms": round(f_ms, 3) if f_ms else None,
                "LU_TFLOPs": round(fl / (f_ms / 1e3) / 1e12, 2) if f_ms else None,
                "LU_frac_of_sustained_bf16": round(fl / (f_ms / 1e3) / 1e12 / tc_sustained, 4)
                if f_ms else None,
                "ms_contracts_off": round(ms_off, 3),
                "contract_overhead_pct": round((ms / ms_off - 1) * 100, 2),
                "per_kernel_ms": {x: round(v, 4) for x, v in kern.items()}}
        sg.sg_matrix_release(mA)
        sg.sg_vector_release(vb)
        del tA, tb
    # the binary64 oracle (textbook GEPP + substitution) on one core at n = 1024
    A1, b1 = inputs.gepp_inputs(1024)
    t_cpu = cpu_time(lambda: oracle.solve(A1, b1))
    res["4_solve_oracle"] = {"GFLOPs": round(2.0 / 3.0 * 1024 ** 3 / t_cpu / 1e9, 3), "cores": 1,
                             "ms_n1024": round(t_cpu * 1e3, 1),
                             "sample": "n = 1024 (2048 and 8192 are pinned by x = 1)"}

    # config 5: the batched chain with its precondition and without (mode OFF)
    L = inputs.batch_lengths()
    off = inputs.batch_offsets(L)
    total = int(off[-1])
    g = torch.Generator(device="cuda").manual_seed(9)
    xb = torch.rand(total, device="cuda", generator=g) * 2 - 1
    to = torch.from_numpy(off).cuda()
    nseg = len(L)
    outs = (torch.empty(nseg, dtype=torch.float64, device="cuda"),
            torch.empty(nseg, dtype=torch.int64, device="cuda"),
            torch.empty(nseg, dtype=torch.int64, device="cuda"))
    mp = [("x", 0), ("x", 0), ("c", 1.0), ("fma",)]
    pre = [("x", 0), ("c", 1.0), ("ge",)]
    kp = [("x", 0), ("c", 1.5), ("gt",)]
    ch = sg.chain(mp, pre, kp)

    def s_batch():
        sg.sg_batch_run(ctx, ch, xb.data_ptr(), to.data_ptr(), nseg, *(t.data_ptr() for t in outs))
    ms = time_steps(torch, stream, s_batch, k)
    ms_off = with_contracts_off(sg, ctx, lambda: time_steps(torch, stream, s_batch, k))
    ns = 200
    xs = inputs.batch_data(int(off[ns]), seed=9)
    t_cpu = cpu_time(lambda: oracle.batch_chain(mp, pre, kp, xs, off[:ns + 1]))
    res["5_batch_10000"] = {
        "ms": round(ms, 4), "GBps": round((4.0 * total + 24 * nseg) / (ms / 1e3) / 1e9, 1),
        "ms_contracts_off": round(ms_off, 4),
        "contract_overhead_pct": round((ms / ms_off - 1) * 100, 2),
        "oracle": {"elements_per_s": round(int(off[ns]) / t_cpu, 1), "cores": 1,
                   "sample": "the first %d collections (%d elements)" % (ns, int(off[ns]))}}
    del xb, to, outs

    # the filter x > 0.25 of 2^28 items, and the same with the postcondition
    # Result.for_all(x > 0.25) on its output (one more pass over the kept items)
    n = 1 << 28
    g.manual_seed(5)
    fx = torch.rand(n, device="cuda", generator=g) * 2 - 1
    vf = sg.wrap_tensor(ctx, fx)
    pr = [("x", 0), ("c", 0.25), ("gt",)]
    fpost = sg.contract(sg.SG_C_FOR_ALL, pr)

    def s_filter():
        kf = sg.sg_filter(ctx, pr, vf)
        sg.sg_ensure(ctx, kf, fpost)
        sg.sg_vector_count(ctx, kf)
        sg.sg_flush(ctx)
        sg.sg_vector_release(kf)
    ms = time_steps(torch, stream, s_filter, k)
    ms_off = with_contracts_off(sg, ctx, lambda: time_steps(torch, stream, s_filter, k))
    xh = inputs.uniform_pm1(inputs.rng(5), 1 << 24)
    t_cpu = cpu_time(lambda: oracle.filter(pr, xh))
    res["filter_2e28_with_postcondition"] = {
        "ms": round(ms, 4), "ms_contracts_off": round(ms_off, 4),
        "contract_overhead_pct": round((ms / ms_off - 1) * 100, 2),
        "oracle": {"items_per_s": round((1 << 24) / t_cpu, 1), "cores": 1,
                   "sample": "2^24 items"}}
    sg.sg_vector_release(vf)
    del fx
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_KEYS)
    ap.add_argument("--ref-sample", type=int, default=1 << 22,
                    help="keys per step of the oracle in --impl reference")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the stream / GEMM / solve / batch figures")
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
    keys = inputs.sort_keys_uniform(n, seed=rank_seed(rank))
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
        ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
        return ms / k

    for _ in range(args.warmup):
        step()
    # timed region: the K steps, untraced
    clocks = Clocks(local, torch)
    k0 = sg.sg_kernel_count(ctx)
    clocks.start()
    ms = timed(args.steps)
    clk = clocks.stop()
    launches = sg.sg_kernel_count(ctx) - k0
    # the same K steps again with kernel tracing (CUDA events bracket each
    # launch on `stream`): the per-kernel durations of the roofline; tracing
    # adds its event records to the step, so the step time comes from the
    # untraced region above
    sg.sg_profile_enable(ctx, True)
    sg.sg_profile_report(ctx, reset=True)
    ms_traced = timed(args.steps)
    prof = sg.sg_profile_report(ctx, reset=True)
    sg.sg_profile_enable(ctx, False)

    # contract overhead: the same steps with checking off, untraced too
    sg.sg_set_contract_mode(ctx, sg.SG_CONTRACTS_OFF)
    for _ in range(2):
        step()
    ms_off = timed(args.steps)
    sg.sg_set_contract_mode(ctx, sg.SG_CONTRACTS_PRE_POST)

    # end to end through the C ABI with host buffers (pinned): every step
    # copies its keys in and its sorted keys out.  Pipelined: create and read
    # are the asynchronous forms, so one step's read overlaps the next step's
    # copy in and sort (two pinned buffers each way); the synchronous forms
    # are timed too.
    hk = [torch.from_numpy(keys).pin_memory() for _ in range(2)]
    hout = [torch.empty(n, dtype=torch.int32).pin_memory() for _ in range(2)]
    hk_np, hout_np = [t.numpy() for t in hk], [t.numpy() for t in hout]

    def e2e_pipeline(k):
        # step i's keys are copied in (asynchronously) before step i - 1's sort
        # is flushed, so the copies in both directions overlap the sorts
        nxt = sg.sg_vector_create_async(ctx, sg.SG_I32, n, hk_np[0])
        for i in range(k):
            v = nxt
            if i + 1 < k:
                nxt = sg.sg_vector_create_async(ctx, sg.SG_I32, n, hk_np[(i + 1) % 2])
            out = sg.sg_sort(ctx, v)
            sg.sg_vector_read_async(ctx, out, hout_np[i % 2])
            sg.sg_vector_release(out)
            sg.sg_vector_release(v)
        sg.sg_sync(ctx)

    def e2e_sync(k):
        for i in range(k):
            v = sg.sg_vector_create(ctx, sg.SG_I32, n, hk_np[0])
            out = sg.sg_sort(ctx, v)
            sg.sg_vector_read(ctx, out, hout_np[0])
            sg.sg_vector_release(out)
            sg.sg_vector_release(v)

    ke = max(3, min(args.steps, 10))

    def time_e2e(run):
        # the host links' copy engines and the memory pool settle over the
        # first steps: four warm-up steps, then the median of three runs of
        # ke steps (every run's time per step is reported)
        run(4)
        runs = []
        for _ in range(3):
            barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            run(ke)
            torch.cuda.synchronize()
            runs.append(max_over_ranks((time.perf_counter() - t0) / ke, world, "cuda"))
        return sorted(runs)[1], runs

    t_e2e, e2e_runs = time_e2e(e2e_pipeline)
    ref_sorted = np.sort(keys)
    for b in hout_np:
        assert np.array_equal(b, ref_sorted)
    t_e2e_sync, e2e_sync_runs = time_e2e(e2e_sync)
    assert np.array_equal(hout_np[0][:1000], ref_sorted[:1000])

    if rank != 0:
        sg.sg_destroy(ctx)
        return

    peak, tc_peak, peak_kind = peaks()
    value = job_gbs(world, BYTES_PER_KEY * n, ms / 1e3)
    roof = None
    if "onesweep" in prof:
        cnt, tot = prof["onesweep"]
        dur = tot / cnt / 1e3
        achieved = 8.0 * n / dur / 1e9
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": onesweep_traffic(n),
                "kernel": "k_onesweep (passes 1-3; 8 bytes/key read+write)",
                "peak_kind": peak_kind + " hbm_gbs (copy bandwidth)"}
    extras = None
    per_config = None
    if not args.no_extras:
        extras = secondary_workloads(torch, sg, ctx, stream, max(3, min(args.steps, 10)), peak,
                                     tc_peak)
        per_config = per_config_workloads(torch, sg, ctx, stream, max(3, min(args.steps, 10)),
                                          peak, tc_peak, sustained_tc_peak())
    cpu = None
    if world == 1:
        import oracle
        oracle.build()
        sample = min(n, 1 << 26)
        sk = keys[:sample].copy()
        t0 = time.perf_counter()
        oracle_step(sk)
        dt = time.perf_counter() - t0
        cpu = {"value": round(BYTES_PER_KEY * sample / dt / 1e9, 4), "unit": "GB/s", "cores": 1,
               "kind": "oracle",
               "sample": "first %d keys of the same workload, one step: C qsort + is_sorted + "
                         "multiset equality, single thread" % sample}
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "bytes_per_key": BYTES_PER_KEY,
                   "l2": "inputs larger than L2 (268 MB keys vs 126 MB L2), no flush",
                   "contracts": "pre_post, fused", "parallelism": "replicas" if world > 1 else "1 GPU",
                   "timing": "CUDA events around K untraced steps; the roofline's kernel "
                             "durations from K further steps with per-launch events"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": round(job_gbs(world, BYTES_PER_KEY * n, t_e2e), 2), "unit": "GB/s",
                "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 4 * n,
                "api": "sg_vector_create_async(pinned host) -> sg_sort -> "
                       "sg_vector_read_async(pinned host), sg_sync after the last step; each "
                       "step's copy in is enqueued before the previous step's sort, so the "
                       "copies in both directions overlap the sorts",
                "ms_per_step_runs": [round(t * 1e3, 3) for t in e2e_runs],
                "timing": "median of 3 runs of %d steps after 4 warm-up steps" % ke,
                "synchronous_value": round(job_gbs(world, BYTES_PER_KEY * n, t_e2e_sync), 2),
                "synchronous_ms_per_step_runs": [round(t * 1e3, 3) for t in e2e_sync_runs],
                "synchronous_api": "sg_vector_create(host) -> sg_sort -> sg_vector_read(host)"},
        "clocks": clk,
        "gpu_launches": launches,
        "extras": {
            "keys_per_s": round(world * n / (ms / 1e3), 1),
            "contract_overhead_pct": round((ms / ms_off - 1.0) * 100.0, 2),
            "ms_per_step_contracts_off": round(ms_off, 4),
            "ms_per_step_traced": round(ms_traced, 4),
            "per_kernel_ms": {k: round(v[1] / v[0], 5) for k, v in prof.items()},
            "per_kernel_launches": {k: v[0] for k, v in prof.items()},
            "secondary": extras,
            "per_config": per_config,
        },
    }
    print(json.dumps(line), flush=True)
    sg.sg_destroy(ctx)


if __name__ == "__main__":
    main()
