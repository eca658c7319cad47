#!/usr/bin/env python
"""Throughput of the TCTF2R completion loop on one or more GB300s.

Workload: the plain FP32 method on the 144 x 288 x 168 synthetic traffic
tensor (144 OD pairs x 288 five-minute slots x 168 days), tubal rank 8,
weights mu = 1e-3, rho1 = 1e-3, rho2 = 1e-1, Bernoulli masks at 10/20/40/60%
observed (one resident instance per ratio).  One step = 100 iterations of the
TCTF2R Algorithm on one instance; steps cycle through the four instances.
L2 is flushed (512 MiB write) before every timed step.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the same workload instead (bounded samples on the host cores).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as wl  # noqa: E402

OBSERVED = (0.1, 0.2, 0.4, 0.6)
WEIGHTS = {"mu": 1e-3, "rho1": 1e-3, "rho2": 1e-1}
METRIC = "completion iters/s (TCTF2R, 144x288x168 r=8 FP32, 100 iters per completion)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--iters", type=int, default=100, help="iterations per step (one completion)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-nmse", action="store_true")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_config(iters):
    w = wl.c2(0.2)
    return {"workload": "144x288x168 traffic tensor (OD x 5-min slots x days), tubal rank 8, FP32",
            "n1": w.n1, "n2": w.n2, "n3": w.n3, "r": w.r, "observed": list(OBSERVED),
            "iters_per_step": iters, "weights": WEIGHTS, "step": "exact (unit) steps",
            "l2": "flushed before every timed step (512 MiB write)"}


def cpu_cores():
    try:
        from threadpoolctl import threadpool_info
        n = max((d.get("num_threads", 1) for d in threadpool_info()), default=1)
        return int(n)
    except Exception:
        return len(os.sched_getaffinity(0))


def oracle_rate(inst, w, n_iter):
    """Oracle iterations/s on a bounded sample: n_iter iterations of the C2
    instance (the initial DFT is outside the timed part)."""
    from oracle import method as O
    t0 = time.perf_counter()
    O.tctf2r(inst["G"], inst["mask"], w.r, WEIGHTS["mu"], WEIGHTS["rho1"], WEIGHTS["rho2"], inst["Y0"], iters=0)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    O.tctf2r(inst["G"], inst["mask"], w.r, WEIGHTS["mu"], WEIGHTS["rho1"], WEIGHTS["rho2"], inst["Y0"], iters=n_iter)
    t = time.perf_counter() - t0 - t_setup
    return n_iter / max(t, 1e-9), t


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    w = wl.c2(0.2)
    inst = wl.as_precision(wl.generate(w), np.float32)
    for _ in range(args.warmup):
        oracle_rate(inst, w, 1)
    times = []
    for _ in range(args.steps):
        _, t = oracle_rate(inst, w, 1)
        times.append(t)
    total = sum(times)
    value = args.steps / total
    cores = cpu_cores()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(1),
            "cpu_baseline": {"value": value, "unit": "iters/s", "cores": cores, "kind": "oracle",
                             "sample": "1 TCTF2R iteration of the 144x288x168 instance (20% observed) per step"},
            "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def src_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2005_09838_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic():
    """Per-launch DRAM bytes of the slab kernel from the committed ncu summary,
    if it was taken on the current sources."""
    path = os.path.join(ROOT, "profiles", "slab_kernel_traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    if d.get("src_sha") != src_hash():
        return None
    return d.get("dram_bytes_per_launch")


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_2005_09838_gb300 import build as _b
    _b.build()
    from paper_2005_09838_gb300 import tc

    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    # resident inputs: one instance per observed ratio (distinct seeds per rank)
    ctxs, insts = [], []
    for q in OBSERVED:
        w = wl.c2(q)
        w = wl.Workload(w.name, w.n1, w.n2, w.n3, w.r, w.period, w.observed, w.iters, w.seed + 7919 * rank)
        inst = wl.as_precision(wl.generate(w), np.float32)
        insts.append((w, inst))
        g = torch.from_numpy(wl.to_colmajor(inst["G"], np.float32)).to(dev)
        m = torch.from_numpy(wl.to_colmajor(inst["mask"], np.uint8)).to(dev)
        y = torch.from_numpy(wl.to_colmajor(inst["Y0"], np.float32)).to(dev)
        p = tc.make_params(w.n1, w.n2, w.n3, w.r, WEIGHTS["mu"], WEIGHTS["rho1"], WEIGHTS["rho2"], tc.TC_FP32)
        torch.cuda.synchronize()
        ctxs.append(tc.Completion(p, g, m, y, on_device=True, stream=sptr))
        del g, m, y
    w0 = insts[0][0]
    N = w0.N
    S = w0.S
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def step(i):
        ctxs[i % len(ctxs)].iterate(args.iters)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    t_wall0 = time.perf_counter()
    step_ms = []
    with ClockSampler(torch.cuda.current_device()) as clk:
        for i in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(i)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    t_wall = time.perf_counter() - t_wall0
    total_ms = sum(step_ms)
    if ws > 1:
        tt = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(tt.item())
    iters_total = args.iters * args.steps * ws
    value = iters_total / (total_ms / 1e3)

    # ---- per-kernel device times (CUDA events inside the library) ------------------
    prof = ctxs[1].profile(20)  # qcon, xstep, ystep, slab in ms
    names = ("qcon", "xstep", "ystep", "slab")
    s = 4
    n1, n2, r = w0.n1, w0.n2, w0.r
    rt = 2 * s * n1 * n2 * S           # one pass over a half spectrum of the slab (R~ or Z~)
    fx, fy = 2 * s * r * n1 * S, 2 * s * r * n2 * S
    ag = 16 * S * ((n2 + 31) // 32) * (r * (r + 1) // 2)   # FP64 tile Grams of Y~
    maskb = 4 * n1 * n2 * ((w0.n3 + 31) // 32)              # mask words
    alg = {"qcon": rt + fy + fx,                 # R~, Y~ in; Q out
           "xstep": 3 * fx + ag,                 # X~, Q in; X~' out; tile Grams in
           "ystep": 2 * rt + fx + 2 * fy + ag,   # R~, X~', Y~ in; Y~', Z~, tile Grams out
           "slab": s * N + maskb + 2 * rt}       # G, mask, Z~ in; R~ out
    dom = names[int(np.argmax(prof))]
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    achieved = alg[dom] / (prof[names.index(dom)] * 1e-3) / 1e9
    traffic = ncu_traffic() if dom == "slab" else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": dom, "peak_source": peak_src,
                "algorithmic_bytes_per_launch": alg[dom],
                "kernel_ms": {n: v for n, v in zip(names, prof)},
                "iteration_alg_bytes": sum(alg.values()),
                "iteration_ms_sum_of_kernels": sum(prof)}

    # ---- recovery accuracy: FP32 vs the FP64 GPU path, 100 iterations, 20% mask ---------
    nmse = None
    if not args.no_nmse and rank == 0:
        from paper_2005_09838_gb300 import api
        wq, inst = insts[1]
        res = {}
        for prec in ("fp32", "fp64"):
            o = api.complete(inst["G"], inst["mask"], inst["Y0"], wq.r, args.iters, WEIGHTS["mu"], WEIGHTS["rho1"],
                             WEIGHTS["rho2"], prec, objective=False)
            res[prec] = wl.nmse(inst["M"], o["W"], inst["mask"])
        nmse = {"observed": wq.observed, "fp32": res["fp32"], "fp64": res["fp64"],
                "abs_diff": abs(res["fp32"] - res["fp64"])}

    # ---- end to end through the C ABI with host buffers ------------------------------------
    e2e = None
    if not args.no_e2e:
        wq, inst = insts[1]
        g = torch.from_numpy(wl.to_colmajor(inst["G"], np.float32)).pin_memory()
        m = torch.from_numpy(wl.to_colmajor(inst["mask"], np.uint8)).pin_memory()
        y = torch.from_numpy(wl.to_colmajor(inst["Y0"], np.float32)).pin_memory()
        wout = torch.empty(N, dtype=torch.float32).pin_memory()
        p = tc.make_params(wq.n1, wq.n2, wq.n3, wq.r, WEIGHTS["mu"], WEIGHTS["rho1"], WEIGHTS["rho2"], tc.TC_FP32)

        def e2e_step():
            with tc.Completion(p, g, m, y, on_device=False, stream=sptr) as c:
                c.iterate(args.iters)
                c.result(wout)

        e2e_step()
        torch.cuda.synchronize()
        ts = []
        for _ in range(max(2, min(args.steps, 5))):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_step()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        e2e = {"value": args.iters / statistics.mean(ts), "unit": "iters/s",
               "h2d_bytes_per_step": g.numel() * 4 + m.numel() + y.numel() * 4,
               "d2h_bytes_per_step": wout.numel() * 4,
               "note": "tc_init from pinned host buffers + 100 iterations + tc_result to host + tc_free"}

    # ---- CPU baseline: the FP64 oracle on a bounded sample ---------------------------------
    cpu = None
    if not args.no_cpu_baseline and rank == 0 and ws == 1:
        wq, inst = insts[1]
        n_it = 3
        rate, t = oracle_rate(inst, wq, n_it)
        cpu = {"value": rate, "unit": "iters/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": f"{n_it} TCTF2R iterations of the 144x288x168 instance (20% observed), {t:.1f} s"}

    clocks = clk.summary()
    if rank == 0:
        cfg = workload_config(args.iters)
        cfg["parallelism"] = f"replicas x{ws} (independent completions per GPU)"
        cfg["entries_per_s"] = value * N
        cfg["wall_s_timed_region"] = t_wall
        line = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": 4 * args.iters * args.steps, "clocks": clocks, "nmse": nmse}
        print(json.dumps(line), flush=True)
    for c in ctxs:
        c.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
