#!/usr/bin/env python3
"""Effective TFLOP/s (2 m n k / t) of the Strassen-Winograd product on one GB300, beside the
plain tensor-core GEMM of the same library and the FP64 CPU oracle.

Workload (default): one FP32 product C = A B, square n = 8192, A and B i.i.d. uniform[-1, 1]
(PCG64 seeds 0 and 1), TF32 leaves with FP32 accumulation.  A step is one whole product
through the C ABI (sw_smm): the operand-sum pass and the grouped leaf GEMM (CTA pairs, B read
N-major as stored) with the post-additions in its epilogue.  Inputs (256 MiB each) exceed the 129 MB L2, so no flush is
needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs its own product on its own GPU (replicas, weak scaling);
rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2309_00628_gb300 import inputs  # noqa: E402

TF32_OVER_BF16 = 1.1 / 2.25  # nominal dense TF32 : BF16 tensor rate of the GB300


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=8192)
    p.add_argument("--algo", choices=["winograd", "knuth", "strassen", "naive"], default="winograd")
    p.add_argument("--sched", choices=["fused", "two_temp", "in_place", "alloc"], default="fused")
    p.add_argument("--leaf", choices=["tf32", "bf16x3", "tf32x3", "f64", "f64wt"], default="tf32",
                   help="leaf precision of the profile case (the headline line is TF32; f64 / f64wt: an FP64 "
                        "product on uniform operands with the plain or the tile-step leaf)")
    p.add_argument("--cutoff", type=int, default=None,
                   help="recursion cutoff (default n / 2: one level); 0 = the library's autotuner")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU-oracle sample budget")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--no-extra", action="store_true",
                   help="skip the depth sweep, the split-BF16 line and the n = 16384 comparison")
    p.add_argument("--serve-rates", default="2,4,8", help="Poisson arrival rates (requests/s) of the serving sweep")
    p.add_argument("--serve-requests", type=int, default=40, help="requests per rate")
    p.add_argument("--serve-share", type=int, default=16, help="SMs of the resident leaf-GEMM loop")
    p.add_argument("--sweep", action="store_true", help="print plain and L = 1..3 timings, no JSON line")
    p.add_argument("--profile-case", action="store_true",
                   help="only --warmup products plus one more of the chosen variant (for ncu captures)")
    p.add_argument("--profile-batched", type=int, default=0, metavar="COUNT",
                   help="only the first COUNT products of the batched workload: one tuning call, then "
                        "--warmup + 1 more batched calls (for ncu captures)")
    p.add_argument("--batched-cutoff", type=int, default=0,
                   help="cutoff of the --profile-batched calls (0: the autotuner; 1073741824: no recursion, "
                        "the default grouped-launch form, no tuning launches)")
    return p.parse_args()


# ---------------------------------------------------------------- helpers
def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5], f[6], f[7], f[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[2 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def traffic_from_profiles(kernel_file: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it matches the current kernel."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"{workload}.md")
    src = os.path.join(ROOT, "paper_2309_00628_gb300", "csrc", kernel_file)
    try:
        text = open(path).read()
        sha = hashlib.sha1(open(src, "rb").read()).hexdigest()[:12]
    except OSError:
        return None
    m = re.search(r"kernel_source_sha1:\s*([0-9a-f]+)", text)
    t = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m or not t or m.group(1) != sha:
        return None
    return float(t.group(1))


def replica_throughput(times_ms, units_per_rank: float, dist=None, device=None):
    """Whole-job throughput of independent replicas: every rank's timed region is reduced to the
    slowest rank's (max over ranks), and the units all ranks processed are divided by that time.
    Returns (max times in ms, units per second for each time)."""
    import torch
    t = torch.tensor([float(x) for x in times_ms], dtype=torch.float64, device=device)
    world = 1
    if dist is not None and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        world = dist.get_world_size()
    mx = [float(x) for x in t.cpu()]
    return mx, [units_per_rank * world / (x / 1e3) for x in mx]


def workload_config(args, L: int) -> dict:
    """The bench line's `config`: the same for our arm and the reference (oracle) arm."""
    n = args.n
    return {"workload": f"single FP32 product n={n}, uniform[-1,1], {args.algo} {args.sched} "
                        f"L={L}, TF32 leaves, FP32 accumulation",
            "n": n, "depth": L, "algo": args.algo, "schedule": args.sched,
            "l2": "inputs 256 MiB each exceed the 129 MB L2; no flush"}


def leaf_flops(n: int, L: int) -> float:
    return 2.0 * (n >> L) ** 3 * 7 ** L


SIZE_CLASSES = ("order <= 1024", "order 2048", "order >= 4096")


def size_class(m: int, n: int, k: int) -> str:
    """Serving size class of a request by the geometric mean of its dimensions."""
    g = (float(m) * n * k) ** (1.0 / 3.0)
    return SIZE_CLASSES[0] if g <= 1448 else SIZE_CLASSES[1] if g <= 2896 else SIZE_CLASSES[2]


def latency_summary(lat):
    """Count, p50 and p99 (ms) of a list of latencies in seconds (None fields when empty)."""
    if not lat:
        return {"requests": 0, "p50_ms": None, "p99_ms": None}
    ls = sorted(lat)
    return {"requests": len(ls), "p50_ms": 1e3 * statistics.median(ls),
            "p99_ms": 1e3 * ls[min(len(ls) - 1, int(math.ceil(0.99 * len(ls))) - 1)]}


def serving_bench(h, swmm, torch, rates, count, share, seed=3):
    """Poisson arrivals of the FP32 / FP64 serving mix through sw_server_*; per rate: achieved
    throughput, p50 / p99 latency (submit to completion, host clock), Freivalds error; once: the
    largest difference of a served result from the same request run alone."""
    import ctypes
    import threading
    reqs = inputs.serving_requests(count, seed)
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    bufs = []
    for (m, n, k, eb) in reqs:
        dt = torch.float32 if eb == 4 else torch.float64
        A = torch.rand((m, k), generator=g, device="cuda", dtype=dt) * 2 - 1
        B = torch.rand((k, n), generator=g, device="cuda", dtype=dt) * 2 - 1
        C = torch.empty((m, n), device="cuda", dtype=dt)
        var = swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_FUSED
        bufs.append((A, B, C, swmm.request(A, B, C, 0, var), var))
    torch.cuda.synchronize()
    flops = sum(2.0 * m * n * k for (m, n, k, _) in reqs)
    cfg = swmm.sw_server_cfg(share, 64, 60 << 30, 20000)
    swmm.check(h, swmm.sw_server_start(h, cfg))
    try:
        ts = []  # warm-up: every request once (module loads, tensor-map encoders, first launches)
        for b in bufs:
            st, t = swmm.sw_server_submit(h, b[3])
            swmm.check(h, st)
            ts.append(t)
        for t in ts:
            swmm.check(h, swmm.sw_server_wait(h, t, -1))
        rows = []
        for rate in rates:
            arr = np.cumsum(np.random.Generator(np.random.PCG64(seed)).exponential(1.0 / rate, count))
            lat = [0.0] * count
            out = {}
            lock = threading.Lock()
            t0 = time.perf_counter()

            def submitter():
                for i in range(count):
                    d = t0 + arr[i] - time.perf_counter()
                    if d > 0:
                        time.sleep(d)
                    ts_ = time.perf_counter()
                    st_, t_ = swmm.sw_server_submit(h, bufs[i][3])
                    with lock:
                        out[t_] = (i, ts_, st_)

            th = threading.Thread(target=submitter)
            th.start()
            done, t_last = 0, t0
            while done < count:
                with lock:
                    pend = list(out.items())
                for t_, (i, ts_, st_) in pend:
                    if st_ != swmm.SW_OK:
                        raise RuntimeError(f"submit failed: {swmm.sw_last_error(h)}")
                    st_ = swmm.sw_server_wait(h, t_, 0)
                    if st_ == swmm.SW_ETIMEOUT:
                        continue
                    swmm.check(h, st_)
                    t_last = time.perf_counter()
                    lat[i] = t_last - ts_
                    with lock:
                        del out[t_]
                    done += 1
                time.sleep(50e-6)
            th.join()
            span = t_last - (t0 + arr[0])
            ls = sorted(lat)
            rows.append({"rate_per_s": rate, "requests": count, "achieved_req_per_s": count / span,
                         "eff_tflops": flops / span / 1e12, "p50_ms": 1e3 * statistics.median(ls),
                         "p99_ms": 1e3 * ls[min(count - 1, int(math.ceil(0.99 * count)) - 1)],
                         "max_ms": 1e3 * ls[-1],
                         "by_dtype": {name: latency_summary([lat[i] for i, r in enumerate(reqs) if r[3] == eb])
                                      for name, eb in (("fp32", 4), ("fp64", 8))},
                         "by_size": {name: latency_summary([lat[i] for i, r in enumerate(reqs)
                                                            if size_class(*r[:3]) == name])
                                     for name in SIZE_CLASSES}})
        # accuracy of the last rate's results: Freivalds with random signs, normalised like the
        # element-wise metric; then each request alone (sw_smm / sw_dmm) against its served result
        gx = torch.Generator(device="cuda")
        gx.manual_seed(seed + 1)
        worst = {4: 0.0, 8: 0.0}
        solo_diff = {4: 0.0, 8: 0.0}
        for (m, n, k, eb), (A, B, C, r, var) in zip(reqs, bufs):
            x = (torch.randint(0, 2, (n, 1), generator=gx, device="cuda").double() * 2 - 1)
            Ad, Bd = A.double(), B.double()
            scale = math.sqrt(n) * k * float(Ad.abs().max()) * float(Bd.abs().max())
            res = float((C.double() @ x - Ad @ (Bd @ x)).abs().max()) / scale
            worst[eb] = max(worst[eb], res)
            S = torch.empty_like(C)
            fn = swmm.sw_smm if eb == 4 else swmm.sw_dmm
            pp = lambda t: ctypes.c_void_p(t.data_ptr())
            swmm.check(h, fn(h, pp(A), k, pp(B), n, pp(S), n, m, n, k, 0, var, None))
            swmm.check(h, swmm.sw_sync(h, None))
            d = float((S.double() - C.double()).abs().max()) / (k * float(Ad.abs().max()) * float(Bd.abs().max()))
            solo_diff[eb] = max(solo_diff[eb], d)
    finally:
        swmm.sw_server_stop(h)
    n64 = sum(1 for r in reqs if r[3] == 8)
    return {"workload": f"{count} requests per rate, Poisson arrivals (seed {seed}); FP32 (TF32 leaves) / FP64 "
                        f"50/50 ({count - n64}/{n64}); order s in {{512..8192}}, square or aspect <= 8:1; "
                        f"Winograd FUSED, library cutoff; uniform[-1,1]",
            "sm_share": share, "budget_gb": 60, "flops_per_pass": flops, "rates": rows,
            "freivalds_err": {"fp32": worst[4], "fp64": worst[8],
                              "metric": "max|C x - A (B x)| / (sqrt(n) k max|A| max|B|), x random signs"},
            "mix_vs_solo": {"fp32": solo_diff[4], "fp64": solo_diff[8],
                            "metric": "max|C_served - C_alone| / (k max|A| max|B|)"}}


# ---------------------------------------------------------------- reference arm: the CPU oracle
def run_reference(args, rank: int):
    if rank != 0:
        return
    import oracle
    n = args.n
    if args.cutoff is None:
        args.cutoff = n // 2
    L = 0 if args.algo == "naive" else oracle.depth(n, n, n, args.cutoff if args.cutoff > 0 else 8192)
    A, B = inputs.pair(n, n, n, "uniform", seed=0, dtype=np.float32)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    threads = oracle.max_threads()
    t0 = time.perf_counter()
    oracle.naive_mt(A64[:threads], B64, threads)
    rate = 2.0 * threads * n * n / max(time.perf_counter() - t0, 1e-6)
    budget = max(2.0, min(args.cpu_seconds, 150.0 / max(args.steps + args.warmup, 1)))
    rows = int(max(threads, min(n, rate * budget / (2.0 * n * n))))
    rng = np.random.Generator(np.random.PCG64(7))
    times = []
    for i in range(args.warmup + args.steps):
        sel = rng.choice(n, rows, replace=False)
        t0 = time.perf_counter()
        oracle.naive_mt(A64[sel], B64, threads)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = 2.0 * rows * n * n * len(times) / tot / 1e12
    line = {
        "impl": "reference", "metric": "effective TFLOP/s (2mnk/t), Winograd vs plain GEMM, same error",
        "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, L),
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": threads, "kind": "oracle",
                         "sample": f"{rows} of {n} rows of C = A B per step (the FP64 oracle's naive product, "
                                   f"Alg. 1, OpenMP over rows; the same product in exact arithmetic)"},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    from paper_2309_00628_gb300 import swmm

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", rank=rank, world_size=world)
    swmm.load(build_if_missing=True)
    h = swmm.sw_create(0)
    stream = torch.cuda.current_stream()
    sp = swmm._stream_ptr(stream)
    n = args.n
    algo = {"winograd": swmm.SW_ALGO_WINOGRAD, "knuth": swmm.SW_ALGO_WINOGRAD_KNUTH, "strassen": swmm.SW_ALGO_STRASSEN,
            "naive": swmm.SW_ALGO_NAIVE}[args.algo]
    sched = {"fused": swmm.SW_SCHED_FUSED, "two_temp": swmm.SW_SCHED_TWO_TEMP, "in_place": swmm.SW_SCHED_IN_PLACE,
             "alloc": swmm.SW_SCHED_ALLOC}[args.sched]
    variant = algo | sched | swmm.SW_LEAF_TF32
    if args.cutoff is None:
        args.cutoff = n // 2
    st, L = swmm.sw_mm_depth(n, n, n, args.cutoff, variant, 4)
    swmm.check(h, st)

    A, B = inputs.pair(n, n, n, "uniform", seed=0, dtype=np.float32)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.empty((n, n), dtype=torch.float32, device="cuda")
    p = lambda t: __import__("ctypes").c_void_p(t.data_ptr())

    def product(v, cutoff):
        swmm.check(h, swmm.sw_smm(h, p(dA), n, p(dB), n, p(dC), n, n, n, n, cutoff, v, sp))

    def timed(v, cutoff, steps, warmup, clocks=None, profile=False):
        for _ in range(warmup):
            product(v, cutoff)
        swmm.check(h, swmm.sw_sync(h, sp))
        if profile:
            swmm.sw_profile(h, True)
            swmm.sw_profile_read(h)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
            time.sleep(0.3)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        ev[0].record(stream)
        for i in range(steps):
            product(v, cutoff)
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        clk = clocks.stop() if clocks else None
        swmm.check(h, swmm.sw_sync(h, sp))
        prof = None
        if profile:
            _, prof = swmm.sw_profile_read(h)
            swmm.sw_profile(h, False)
        per = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
        total = ev[0].elapsed_time(ev[steps])
        return total, per, clk, prof

    if args.profile_batched:
        shapes = inputs.batched_shapes(512, seed=2)[:args.profile_batched]
        g = torch.Generator(device="cuda")
        g.manual_seed(2)
        keep, probs = [], []
        for (m, nn, k) in shapes:
            tA = torch.rand((m, k), generator=g, device="cuda") * 2 - 1
            tB = torch.rand((k, nn), generator=g, device="cuda") * 2 - 1
            tC = torch.empty((m, nn), device="cuda")
            keep.append((tA, tB, tC))
            probs.append(swmm.sw_problem(tA.data_ptr(), k, tB.data_ptr(), nn, tC.data_ptr(), nn, m, nn, k))
        arr = (swmm.sw_problem * len(probs))(*probs)
        vb = swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_FUSED
        for _ in range(args.warmup + 2):  # cutoff 0: the first call tunes (5 candidates, 2 timed runs each)
            swmm.check(h, swmm.sw_mm_batched(h, len(probs), arr, args.batched_cutoff, vb, sp))
        swmm.check(h, swmm.sw_sync(h, sp))
        if rank == 0:
            tune = swmm.sw_last_tuning(h)
            print(json.dumps({"profile_batched": len(probs), "autotuner": tune[1] if tune[0] == swmm.SW_OK else None}),
                  flush=True)
        swmm.sw_destroy(h)
        return

    if args.profile_case:
        if args.leaf in ("f64", "f64wt"):
            A8, B8 = dA.double(), dB.double()
            C8 = torch.empty((n, n), dtype=torch.float64, device="cuda")
            v8 = variant | (swmm.SW_LEAF_F64_WTILE if args.leaf == "f64wt" else 0)
            for _ in range(args.warmup + 1):
                swmm.check(h, swmm.sw_dmm(h, p(A8), n, p(B8), n, p(C8), n, n, n, n, args.cutoff, v8, sp))
            L = swmm.sw_mm_depth(n, n, n, args.cutoff, v8, 8)[1]
        else:
            leafbits = {"tf32": swmm.SW_LEAF_TF32, "bf16x3": swmm.SW_LEAF_BF16X3,
                        "tf32x3": swmm.SW_LEAF_TF32X3}[args.leaf]
            for _ in range(args.warmup + 1):
                product(variant | leafbits, args.cutoff)
        swmm.check(h, swmm.sw_sync(h, sp))
        if rank == 0:
            print(json.dumps({"profile_case": args.algo, "schedule": args.sched, "leaf": args.leaf, "n": n, "depth": L}),
                  flush=True)
        swmm.sw_destroy(h)
        return

    if args.sweep:
        rows = []
        BF = swmm.SW_LEAF_BF16X3
        for name, v, c in [("plain", swmm.SW_ALGO_NAIVE, 0)] + [
                (f"{a}-L{l}", alg | swmm.SW_SCHED_FUSED, n >> l)
                for a, alg in (("winograd", swmm.SW_ALGO_WINOGRAD), ("strassen", swmm.SW_ALGO_STRASSEN))
                for l in (1, 2, 3)] + [("plain-bf16x3", swmm.SW_ALGO_NAIVE | BF, 0),
                                      ("winograd-L1-bf16x3", swmm.SW_ALGO_WINOGRAD | BF, n >> 1),
                                      ("winograd-L2-two_temp-bf16x3", swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_TWO_TEMP | BF,
                                       n >> 2)]:
            tot, per, _, prof = timed(v, c, max(args.steps // 4, 10), args.warmup, profile=True)
            ms = tot / max(args.steps // 4, 10)
            g = prof["gemm_bf16x3"] if v & BF else prof["gemm_tf32"]
            row = {"variant": name, "ms": round(ms, 4), "eff_tflops": round(2 * n ** 3 / ms / 1e9, 1),
                   "gemm_ms_per_launch": round(g[1] / max(g[0], 1), 4),
                   "kernels": {k: [a, round(b, 3)] for k, a, b in ((k, *prof[k]) for k in prof) if a}}
            rows.append(row)
            if rank == 0:
                print(json.dumps(row), flush=True)
        return

    K, W = args.steps, max(args.warmup, 3)
    clocks = ClockSampler(local)
    # the headline: K whole products, nothing but the product in the timed region
    total, per, clk, _ = timed(variant, args.cutoff, K, W, clocks=clocks)
    # plain tensor-core GEMM of the same library, same size, same timing
    total0, per0, _, _ = timed(swmm.SW_ALGO_NAIVE, 0, K, W)
    # per-kernel durations (roofline, launch counts): the same step again with every launch of the
    # library bracketed by CUDA events on its own stream (the events cost some time per launch,
    # so this pass is kept out of the headline)
    Kp = max(K // 4, 10)
    _, _, _, prof = timed(variant, args.cutoff, Kp, W, profile=True)
    flop = 2.0 * n ** 3
    (total, total0), (rate, rate0) = replica_throughput([total, total0], flop * K, dist, device="cuda")
    value, value0 = rate / 1e12, rate0 / 1e12

    # dominant kernel: the grouped TF32 leaf GEMM
    gl, gms = prof["gemm_tf32"]
    launches = int(round(sum(v[0] for k, v in prof.items()) * K / Kp))
    achieved = leaf_flops(n, L) / (gms / gl / 1e3) / 1e12 if gl else None
    pk = peaks()
    peak, peak_src = (pk["bf16_tflops"] * TF32_OVER_BF16, "of measured (bf16 burst x nominal TF32/BF16)") \
        if pk else (1900.0 * TF32_OVER_BF16, "of fallback")

    # end to end: host operands, copies inside the timed region (rank-local)
    e2e = None
    if not args.no_e2e:
        hA = torch.from_numpy(A).pin_memory()
        hB = torch.from_numpy(B).pin_memory()
        hC = torch.empty((n, n), dtype=torch.float32).pin_memory()
        ke = max(min(K // 4, 50), 5)
        for i in range(W + ke):
            if i == W:
                t0 = time.perf_counter()
            swmm.check(h, swmm.sw_smm_host(h, p(hA), n, p(hB), n, p(hC), n, n, n, n, args.cutoff, variant, sp))
        te = time.perf_counter() - t0
        e2e = {"value": flop * ke * world / te / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": 2 * n * n * 4,
               "d2h_bytes_per_step": n * n * 4}

    # batched workload: 512 uneven FP32 products (m, n, k log-uniform in [96, 3000]) in one grouped
    # launch, replayed through its CUDA graph
    batched = None
    if not args.no_batched:
        shapes = inputs.batched_shapes(512, seed=2)
        g = torch.Generator(device="cuda")
        g.manual_seed(2)
        keep, probs = [], []
        for (m, nn, k) in shapes:
            tA = torch.rand((m, k), generator=g, device="cuda") * 2 - 1
            tB = torch.rand((k, nn), generator=g, device="cuda") * 2 - 1
            tC = torch.empty((m, nn), device="cuda")
            keep.append((tA, tB, tC))
            probs.append(swmm.sw_problem(tA.data_ptr(), k, tB.data_ptr(), nn, tC.data_ptr(), nn, m, nn, k))
        arr = (swmm.sw_problem * len(probs))(*probs)
        vb = swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_FUSED
        for _ in range(W):
            swmm.check(h, swmm.sw_mm_batched(h, len(probs), arr, 0, vb, sp))
        swmm.check(h, swmm.sw_sync(h, sp))
        kb = max(min(K // 4, 50), 5)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(kb):
            swmm.check(h, swmm.sw_mm_batched(h, len(probs), arr, 0, vb, sp))
        e1.record(stream)
        swmm.check(h, swmm.sw_sync(h, sp))
        tb = e0.elapsed_time(e1) / kb
        fl = sum(2.0 * m * nn * k for (m, nn, k) in shapes)
        _, btune = swmm.sw_last_tuning(h)
        batched = {"value": fl / (tb / 1e3) / 1e12, "unit": "TFLOP/s", "ms_per_step": tb, "problems": len(shapes),
                   "workload": "512 FP32 products, m,n,k log-uniform [96,3000], uniform[-1,1], one grouped "
                               "launch (CUDA graph replay), tile shape and cutoff chosen by the autotuner",
                   "autotuner": btune}
        del keep

    serving = None
    if not args.no_serving and world == 1:
        rates = [float(x) for x in args.serve_rates.split(",") if x]
        serving = serving_bench(h, swmm, torch, rates, args.serve_requests, args.serve_share)

    # CPU oracle on this machine: timed sample rows, also the reference for the error report
    cpu = None
    err = {}
    if rank == 0:
        import oracle
        threads = oracle.max_threads()
        A64, B64 = A.astype(np.float64), B.astype(np.float64)
        t0 = time.perf_counter()
        oracle.naive_mt(A64[:threads], B64, threads)
        rate = 2.0 * threads * n * n / max(time.perf_counter() - t0, 1e-6)
        rows = int(max(threads, min(n, rate * args.cpu_seconds / (2.0 * n * n))))
        sel = np.sort(np.random.Generator(np.random.PCG64(7)).choice(n, rows, replace=False))
        t0 = time.perf_counter()
        R = oracle.naive_mt(A64[sel], B64, threads)
        tc = time.perf_counter() - t0
        cpu = {"value": 2.0 * rows * n * n / tc / 1e12, "unit": "TFLOP/s", "cores": threads, "kind": "oracle",
               "sample": f"{rows} random rows of the n={n} product (Alg. 1, FP64, OpenMP over rows), {tc:.1f} s"}
        amax, bmax = float(np.max(np.abs(A))), float(np.max(np.abs(B)))
        idx = torch.from_numpy(sel).cuda()

        def row_err(v, c):
            product(v, c)
            swmm.check(h, swmm.sw_sync(h, sp))
            Cr = dC[idx].double().cpu().numpy()
            return float(np.max(np.abs(Cr - R)) / (n * amax * bmax))

        for name, v, c in (("winograd", variant, args.cutoff), ("plain", swmm.SW_ALGO_NAIVE, 0)):
            err[name] = row_err(v, c)

    # error and time against recursion depth (same inputs, same oracle rows), the FP32-accuracy
    # split-BF16 leaves, and the n = 16384 comparison of plain and Winograd
    extra = None
    if rank == 0 and not args.no_extra:
        ks = max(K // 8, 10)
        BF = swmm.SW_LEAF_BF16X3
        depth_rows = []
        for lab, v, c in [("plain L0", swmm.SW_ALGO_NAIVE, 0)] + [
                (f"winograd L{l}", swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_FUSED, n >> l) for l in (1, 2, 3)] + [
                (f"strassen L{l}", swmm.SW_ALGO_STRASSEN | swmm.SW_SCHED_FUSED, n >> l) for l in (1, 2)] + [
                (f"winograd-knuth L{l}", swmm.SW_ALGO_WINOGRAD_KNUTH | swmm.SW_SCHED_FUSED, n >> l) for l in (1, 2)]:
            tot, _, _, _ = timed(v, c, ks, W)
            depth_rows.append({"variant": lab, "ms": tot / ks, "eff_tflops": flop / (tot / ks / 1e3) / 1e12,
                               "err": row_err(v, c)})
        # context: the vendor library's TF32 GEMM on the same operands (not part of the method)
        tf32_prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = True
        with torch.cuda.stream(stream):
            for _ in range(W):
                torch.matmul(dA, dB, out=dC)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(ks):
                torch.matmul(dA, dB, out=dC)
            e1.record(stream)
        stream.synchronize()
        torch.backends.cuda.matmul.allow_tf32 = tf32_prev
        ms_lib = e0.elapsed_time(e1) / ks
        err_lib = float(np.max(np.abs(dC[idx].double().cpu().numpy() - R)) / (n * amax * bmax))
        depth_rows.append({"variant": "cublas tf32 (torch, context)", "ms": ms_lib,
                           "eff_tflops": flop / (ms_lib / 1e3) / 1e12, "err": err_lib})
        # the same sweep at n = 4096 (config 2's smaller size): its own seeded inputs and oracle rows
        n5 = n // 2
        A5, B5 = inputs.pair(n5, n5, n5, "uniform", seed=0, dtype=np.float32)
        dA5, dB5 = torch.from_numpy(A5).cuda(), torch.from_numpy(B5).cuda()
        dC5 = torch.empty((n5, n5), dtype=torch.float32, device="cuda")
        sel5 = np.sort(np.random.Generator(np.random.PCG64(10)).choice(n5, 16, replace=False))
        R5 = oracle.naive_mt(A5[sel5].astype(np.float64), B5.astype(np.float64), oracle.max_threads())
        scale5 = n5 * float(np.max(np.abs(A5))) * float(np.max(np.abs(B5)))
        idx5 = torch.from_numpy(sel5).cuda()
        depth_rows5 = []
        for lab, v, c in [("plain L0", swmm.SW_ALGO_NAIVE, 0)] + [
                (f"winograd L{l}", swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_FUSED, n5 >> l) for l in (1, 2, 3)]:
            run5 = lambda: swmm.check(h, swmm.sw_smm(h, p(dA5), n5, p(dB5), n5, p(dC5), n5, n5, n5, n5, c, v, sp))
            for _ in range(W):
                run5()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(ks):
                run5()
            e1.record(stream)
            swmm.check(h, swmm.sw_sync(h, sp))
            ms5 = e0.elapsed_time(e1) / ks
            err5 = float(np.max(np.abs(dC5[idx5].double().cpu().numpy() - R5)) / scale5)
            depth_rows5.append({"variant": lab, "ms": ms5, "eff_tflops": 2.0 * n5 ** 3 / (ms5 / 1e3) / 1e12,
                                "err": err5})
        del dA5, dB5, dC5
        bf_rows = []
        X3 = swmm.SW_LEAF_TF32X3
        for lab, v, c in (("plain L0", swmm.SW_ALGO_NAIVE | BF, 0),
                          ("winograd L1", swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_FUSED | BF, n >> 1),
                          ("tf32x3 plain L0", swmm.SW_ALGO_NAIVE | X3, 0),
                          ("tf32x3 winograd L1", swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_FUSED | X3, n >> 1)):
            tot, _, _, _ = timed(v, c, ks, W)
            bf_rows.append({"variant": lab, "ms": tot / ks, "eff_tflops": flop / (tot / ks / 1e3) / 1e12,
                            "err": row_err(v, c)})
        # n = 16384: device-generated uniform[-1, 1] operands (seeded), 1 GiB each
        n2 = 2 * n
        g2 = torch.Generator(device="cuda")
        g2.manual_seed(11)
        A2 = torch.rand((n2, n2), generator=g2, device="cuda") * 2 - 1
        B2 = torch.rand((n2, n2), generator=g2, device="cuda") * 2 - 1
        C2 = torch.empty((n2, n2), device="cuda")
        big = []
        for lab, v, c in (("plain L0", swmm.SW_ALGO_NAIVE, 0),
                          ("winograd L1", swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_FUSED, n2 >> 1),
                          ("winograd L2", swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_FUSED, n2 >> 2)):
            for _ in range(W):
                swmm.check(h, swmm.sw_smm(h, p(A2), n2, p(B2), n2, p(C2), n2, n2, n2, n2, c, v, sp))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            kb2 = 10
            e0.record(stream)
            for _ in range(kb2):
                swmm.check(h, swmm.sw_smm(h, p(A2), n2, p(B2), n2, p(C2), n2, n2, n2, n2, c, v, sp))
            e1.record(stream)
            swmm.check(h, swmm.sw_sync(h, sp))
            ms2 = e0.elapsed_time(e1) / kb2
            big.append({"variant": lab, "ms": ms2, "eff_tflops": 2.0 * n2 ** 3 / (ms2 / 1e3) / 1e12})
        # the FP32-accuracy configuration: n = 16384, normal(0, 1), split-BF16 leaves; the
        # low-allocation schedule (Table 2) beside FUSED and the plain product, error on 16
        # sampled rows of the FP64 oracle
        A2.normal_(0.0, 1.0, generator=g2)
        B2.normal_(0.0, 1.0, generator=g2)
        import oracle
        sel2 = np.sort(np.random.Generator(np.random.PCG64(8)).choice(n2, 16, replace=False))
        A2h, B2h = A2.double().cpu().numpy(), B2.double().cpu().numpy()
        R2 = oracle.naive_mt(A2h[sel2], B2h, oracle.max_threads())
        scale2 = n2 * float(np.max(np.abs(A2h))) * float(np.max(np.abs(B2h)))
        idx2 = torch.from_numpy(sel2).cuda()
        cfg3 = []
        for lab, v, c in (("plain", swmm.SW_ALGO_NAIVE | BF, 0),
                          ("two_temp L1", swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_TWO_TEMP | BF, n2 >> 1),
                          ("two_temp L2", swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_TWO_TEMP | BF, n2 >> 2),
                          ("fused L1", swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_FUSED | BF, n2 >> 1),
                          ("tf32x3 plain", swmm.SW_ALGO_NAIVE | X3, 0),
                          ("tf32x3 two_temp L1", swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_TWO_TEMP | X3, n2 >> 1)):
            for _ in range(2):
                swmm.check(h, swmm.sw_smm(h, p(A2), n2, p(B2), n2, p(C2), n2, n2, n2, n2, c, v, sp))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                swmm.check(h, swmm.sw_smm(h, p(A2), n2, p(B2), n2, p(C2), n2, n2, n2, n2, c, v, sp))
            e1.record(stream)
            swmm.check(h, swmm.sw_sync(h, sp))
            ms3 = e0.elapsed_time(e1) / 3
            err3 = float(np.max(np.abs(C2[idx2].double().cpu().numpy() - R2)) / scale2)
            st3, ws3 = swmm.sw_mm_workspace_size(n2, n2, n2, c, v, 4)
            cfg3.append({"variant": lab, "ms": ms3, "eff_tflops": 2.0 * n2 ** 3 / (ms3 / 1e3) / 1e12, "err": err3,
                         "workspace_bytes": ws3 if st3 == swmm.SW_OK else None})
        del A2, B2, C2
        # FP64 (FP64-ALU bound on this part): n = 4096 uniform[-1, 1], the plain SIMT product, Winograd
        # depth 3 with plain FP64 leaves and with the Winograd-step leaf tiles; cuBLAS DGEMM (torch)
        # as context; error on 8 sampled rows of the FP64 oracle
        n4 = n // 2
        g4 = torch.Generator(device="cuda")
        g4.manual_seed(12)
        A4 = torch.rand((n4, n4), generator=g4, device="cuda", dtype=torch.float64) * 2 - 1
        B4 = torch.rand((n4, n4), generator=g4, device="cuda", dtype=torch.float64) * 2 - 1
        C4 = torch.empty((n4, n4), device="cuda", dtype=torch.float64)
        sel4 = np.sort(np.random.Generator(np.random.PCG64(9)).choice(n4, 8, replace=False))
        A4h, B4h = A4.cpu().numpy(), B4.cpu().numpy()
        R4 = oracle.naive_mt(A4h[sel4], B4h, oracle.max_threads())
        scale4 = n4 * float(np.max(np.abs(A4h))) * float(np.max(np.abs(B4h)))
        idx4 = torch.from_numpy(sel4).cuda()
        fp64 = []
        for lab, v, c in (("plain (SIMT leaf)", swmm.SW_ALGO_NAIVE, 0),
                          ("tile step only (depth 0)", swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_FUSED |
                           swmm.SW_LEAF_F64_WTILE, 1 << 30),
                          ("winograd L3", swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_FUSED, n4 >> 3),
                          ("winograd L3 + tile step", swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_FUSED |
                           swmm.SW_LEAF_F64_WTILE, n4 >> 3),
                          ("winograd L5 (2 Table 2 levels over a fused L3)", swmm.SW_ALGO_WINOGRAD |
                           swmm.SW_SCHED_FUSED, n4 >> 5),
                          ("winograd L5 + tile step", swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_FUSED |
                           swmm.SW_LEAF_F64_WTILE, n4 >> 5),
                          ("cublas dgemm (torch, context)", None, 0)):
            def run4():
                if v is None:
                    torch.matmul(A4, B4, out=C4)
                else:
                    swmm.check(h, swmm.sw_dmm(h, p(A4), n4, p(B4), n4, p(C4), n4, n4, n4, n4, c, v, sp))
            run4()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                run4()
            e1.record(stream)
            swmm.check(h, swmm.sw_sync(h, sp))
            ms4 = e0.elapsed_time(e1) / 3
            err4 = float(np.max(np.abs(C4[idx4].cpu().numpy() - R4)) / scale4)
            fp64.append({"variant": lab, "depth": swmm.sw_mm_depth(n4, n4, n4, c, v, 8)[1] if v is not None else 0,
                         "ms": ms4, "eff_tflops": 2.0 * n4 ** 3 / (ms4 / 1e3) / 1e12, "err": err4})
        del A4, B4, C4
        # FP64 ALU roofline of the two leaf kernels (depth 0: one launch per product); the peak is
        # the FP64 units' nominal rate, about 2 FP64 FMAs per clock per SM x 152 SMs x 2.07 GHz
        fp64_peak = 1.25
        fp64_roof = {"bound": "alu", "peak": fp64_peak, "unit": "TFLOP/s", "peak_source": "nominal FP64 rate",
                     "plain_leaf": {"achieved": fp64[0]["eff_tflops"], "frac": fp64[0]["eff_tflops"] / fp64_peak},
                     "tile_step_leaf": {"achieved": fp64[1]["eff_tflops"] * 7 / 8,
                                        "frac": fp64[1]["eff_tflops"] * 7 / 8 / fp64_peak,
                                        "note": "executed FMAs: 7/8 of 2n^3 (tile sums not counted)"}}
        # peak workspace of each schedule for the n = 16384 split-BF16 configuration (depth 2)
        ws = {}
        for lab, sc in (("alloc", swmm.SW_SCHED_ALLOC), ("two_temp", swmm.SW_SCHED_TWO_TEMP),
                        ("in_place", swmm.SW_SCHED_IN_PLACE), ("fused", swmm.SW_SCHED_FUSED)):
            st_, b_ = swmm.sw_mm_workspace_size(16384, 16384, 16384, 4096, swmm.SW_ALGO_WINOGRAD | sc | BF, 4)
            ws[lab] = b_ if st_ == swmm.SW_OK else None
        # the autotuner's own pick for this product (cutoff 0: candidate depths timed on first use)
        product(swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_FUSED, 0)
        swmm.check(h, swmm.sw_sync(h, sp))
        _, tune = swmm.sw_last_tuning(h)
        tot, _, _, _ = timed(swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_FUSED, 0, ks, W)
        tuned = {"cutoff": tune["cutoff"], "depth": swmm.sw_mm_depth(n, n, n, tune["cutoff"], variant, 4)[1],
                 "candidates": tune["candidates"], "ms": tot / ks, "eff_tflops": flop / (tot / ks / 1e3) / 1e12}
        # Winograd and the plain product in alternating blocks (the power cap drifts over a long
        # timed region, so back-to-back blocks compare the two under the same conditions)
        alt = {"winograd_ms": [], "plain_ms": []}
        for _ in range(5):
            for key, v, c in (("winograd_ms", variant, args.cutoff), ("plain_ms", swmm.SW_ALGO_NAIVE, 0)):
                tot, _, _, _ = timed(v, c, 20, 2)
                alt[key].append(tot / 20)
        alt["speedup_per_round"] = [p_ / w_ for w_, p_ in zip(alt["winograd_ms"], alt["plain_ms"])]
        alt["speedup"] = sum(alt["plain_ms"]) / sum(alt["winograd_ms"])
        extra = {"autotuned_winograd_n8192": tuned, "alternating_vs_plain_n8192": alt,
                 "depth_sweep_n8192_tf32": depth_rows, "depth_sweep_n4096_tf32": depth_rows5,
                 "fp32_accuracy_leaves_n8192": bf_rows,
                 "n16384_tf32": big,
                 "fp32_accuracy_n16384_normal_bf16x3": cfg3,
                 "workspace_bytes_n16384_L2_bf16x3": ws,
                 "fp64_n4096": fp64,
                 "fp64_roofline": fp64_roof,
                 "err_metric": "max|C - C_oracle| / (n max|A| max|B|) on the sampled oracle rows"}

    if rank == 0:
        traffic = traffic_from_profiles("gemm_tc.cu", f"gemm_tf32_winograd_n{n}_L{L}")
        lat = sorted(per)
        line = {
            "metric": "effective TFLOP/s (2mnk/t), Winograd vs plain GEMM, same error",
            "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": total / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "tf32", "data": "synthetic",
            "config": workload_config(args, L),
            "p50_ms": statistics.median(lat), "p99_ms": lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)],
            "plain_gemm": {"value": value0, "unit": "TFLOP/s", "ms_per_step": total0 / K,
                           "p50_ms": statistics.median(per0)},
            "speedup_vs_plain": value / value0,
            "error": {"winograd": err.get("winograd"), "plain": err.get("plain"),
                      "metric": "max|C - C_oracle| / (n max|A| max|B|) on the sampled rows"},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                         "kernel": "gemm_tf32_kernel (grouped leaf GEMM)", "peak_source": peak_src,
                         "algorithmic_flops_per_launch": leaf_flops(n, L),
                         "avg_launch_ms": gms / gl if gl else None},
            "kernels_in_step": {k: {"launches_per_step": v[0] / Kp, "ms_per_step": v[1] / Kp}
                                for k, v in prof.items() if v[0]},
            "profiled_steps": Kp,
            "gpu_launches": launches,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "batched": batched,
            "serving": serving,
            "extra": extra,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    swmm.sw_destroy(h)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
