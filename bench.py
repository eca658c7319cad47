#!/usr/bin/env python
"""Throughput of the TCTF2R completion loop on one or more GB300s.

Workload: the plain FP32 method on the 144 x 288 x 168 synthetic traffic
tensor (144 OD pairs x 288 five-minute slots x 168 days), tubal rank 8,
weights mu = 1e-3, rho1 = 1e-3, rho2 = 1e-1, Bernoulli masks at 10/20/40/60%
observed (inputs resident on the device).  One step = one completion: 100
iterations of the TCTF2R Algorithm from the initial point, on a context
initialised before the timed region; steps cycle through the four ratios.
L2 is flushed (512 MiB write) before every timed step.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the same workload instead (bounded samples on the host cores).
On one GPU the default line also carries, under ``forms``, shorter
measurements of the precision form, the batched form and the differentiation
form (529 x 288 x 168, r = 16, block gradient descent); ``--no-forms`` skips them.

The first two forms also have JSON lines of their own:
``--form precision``: the 529 x 96 x 112 tensor (529 OD pairs x 96
fifteen-minute slots x 112 days), tubal rank 32, 30% observed; the precision
form (TF32 / BF16 tensor-core contractions, FP64-storage solves) against the
plain FP32 path on the same resident instance, 30 iterations per step, with
the recovery NMSE of each against the FP64 path.
``--form batched``: 64 seeded instances with n1 in [64, 1024], n2 in
[96, 288], n3 in [28, 168], r in [4, 32], 10-60% observed, advanced together
by one graph launch per iteration (tc_batch_*), TF32 tensor-core
contractions where r > 16; compared with the same contexts iterated one after
the other and with the plain FP32 batch.
"""
from __future__ import annotations

import argparse
import hashlib
import json
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
    ap.add_argument("--form", default="plain", choices=["plain", "precision", "batched"])
    ap.add_argument("--no-forms", action="store_true", help="skip the precision / batched / differentiation "
                    "measurements nested in the default line")
    ap.add_argument("--precision-forms", default="", help="with --form precision: comma-separated subset of "
                    "fp32, tf32, bf16, tf32_single_pass, bf16_single_pass (default all)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_workloads(rank):
    """The bench instances of one rank: one per observed ratio, seeds distinct
    per rank (each rank completes its own tensors; no data is exchanged)."""
    out = []
    for q in OBSERVED:
        w = wl.c2(q)
        out.append(wl.Workload(w.name, w.n1, w.n2, w.n3, w.r, w.period, w.observed, w.iters,
                               w.seed + 7919 * rank))
    return out


def job_throughput(local_ms, units_per_rank, ws, device):
    """Whole-job rate: the slowest rank's time (all-reduce MAX over ranks when
    ws > 1) and the units all ranks processed over it.  Returns (ms, units/s)."""
    total_ms = float(local_ms)
    if ws > 1:
        import torch
        tt = torch.tensor([total_ms], device=device, dtype=torch.float64)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(tt.item())
    return total_ms, units_per_rank * ws / (total_ms / 1e3)


def workload_config(iters):
    w = wl.c2(0.2)
    return {"workload": "144x288x168 traffic tensor (OD x 5-min slots x days), tubal rank 8, FP32",
            "n1": w.n1, "n2": w.n2, "n3": w.n3, "r": w.r, "observed": list(OBSERVED),
            "iters_per_step": iters, "weights": WEIGHTS, "step": "exact (unit) steps",
            "completion": "one completion per step from the initial point, context initialised before timing",
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


SLAB_SOURCES = ("k_slab_f.cuh", "k_slab.cuh", "fft_reg.cuh", "tc_common.cuh", "tc_kernels.cuh", "tc_f32_168.cu")


def src_hash():
    """Hash of the sources the 168-point slab kernel is compiled from."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2005_09838_gb300", "csrc")
    for f in SLAB_SOURCES:
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


def iteration_bytes(w, s=4):
    """Algorithmic bytes of one iteration: the observed tensor (s N), the mask
    (N bits) and three passes over the half spectrum of the residual (read by
    the X-step contraction, read by the Y-step contraction, written by the
    fused transform / W-step / residual step)."""
    return s * w.N + w.N / 8 + 3 * (2 * s * w.n1 * w.n2 * w.S)


def algorithmic_bytes(w, s=4):
    """Algorithmic bytes per launch of each kernel of the iteration, by the
    steps it carries: Q = R~Y~^H one read of R~ (plus the factors), the X-step
    the factors and the tile Grams, the Y-step one read of R~ (plus the
    factors), the slab kernel G, the mask bits and one write of R~.  Their sum
    is iteration_bytes plus the factor traffic."""
    n1, n2, r, S = w.n1, w.n2, w.r, w.S
    rt = 2 * s * n1 * n2 * S
    fx, fy = 2 * s * r * n1 * S, 2 * s * r * n2 * S
    ag = 16 * S * ((n2 + 31) // 32) * (r * (r + 1) // 2)
    return {"qcon": rt + fy + fx, "xstep": 3 * fx + ag, "ystep": rt + fx + 2 * fy + ag,
            "slab": s * w.N + w.N / 8 + rt}


def design_bytes(w, s=4):
    """Bytes each kernel of this design moves, including the spectrum Z~ that
    the Y-step writes and the slab kernel reads back (a design choice: the
    synthesis Z~ = X~Y~ could run inside the slab kernel instead) and the mask
    as 32-bit row words."""
    n1, n2, r, S = w.n1, w.n2, w.r, w.S
    rt = 2 * s * n1 * n2 * S
    fx, fy = 2 * s * r * n1 * S, 2 * s * r * n2 * S
    ag = 16 * S * ((n2 + 31) // 32) * (r * (r + 1) // 2)
    maskb = 4 * n1 * w.n3 * ((n2 + 31) // 32)
    return {"qcon": rt + fy + fx, "xstep": 3 * fx + ag, "ystep": 2 * rt + fx + 2 * fy + ag,
            "slab": s * w.N + maskb + 2 * rt}


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
    insts, dev_in = [], []
    for w in rank_workloads(rank):
        inst = wl.as_precision(wl.generate(w), np.float32)
        insts.append((w, inst))
        dev_in.append((torch.from_numpy(wl.to_colmajor(inst["G"], np.float32)).to(dev),
                       torch.from_numpy(wl.to_colmajor(inst["mask"], np.uint8)).to(dev),
                       torch.from_numpy(wl.to_colmajor(inst["Y0"], np.float32)).to(dev)))
    w0 = insts[0][0]
    N = w0.N
    S = w0.S
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def context(q):
        w = insts[q][0]
        p = tc.make_params(w.n1, w.n2, w.n3, w.r, WEIGHTS["mu"], WEIGHTS["rho1"], WEIGHTS["rho2"], tc.TC_FP32)
        torch.cuda.synchronize()
        return tc.Completion(p, *dev_in[q], on_device=True, stream=sptr)

    # one fresh context per step, initialised outside the timed region
    ctxs = [context(i % len(OBSERVED)) for i in range(args.warmup + args.steps)]

    def step(i):
        ctxs[i].iterate(args.iters)

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
            step(args.warmup + i)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    t_wall = time.perf_counter() - t_wall0
    total_ms, value = job_throughput(sum(step_ms), args.iters * args.steps, ws, dev)

    # ---- per-kernel device times (CUDA events inside the library), averaged over one
    # completion (100 iterations) of a fresh context ------------------------------------
    for c in ctxs:
        c.close()
    pc = context(1)
    prof = pc.profile(args.iters)  # qcon, xstep, ystep, slab in ms
    pc.close()
    ctxs = []
    names = ("qcon", "xstep", "ystep", "slab")
    alg, design = algorithmic_bytes(w0), design_bytes(w0)
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
    b_iter = iteration_bytes(w0)
    it_ms = total_ms / (args.iters * args.steps)  # device time per iteration of the timed region
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": dom, "peak_source": peak_src,
                "algorithmic_bytes_per_launch": alg[dom],
                "design_bytes_per_launch": design[dom],
                "kernel_ms": {n: v for n, v in zip(names, prof)},
                "iteration_alg_bytes": b_iter,
                "iteration_ms": it_ms,
                "iteration_frac": b_iter / (it_ms * 1e-3) / 1e9 / peak,
                "iteration_design_bytes": sum(design.values()),
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
    # ---- the precision, batched and differentiation forms (one GPU only) -----------------
    forms = None
    if not args.no_forms and rank == 0 and ws == 1:
        forms = {}
        small = max(2, min(args.steps, 3))
        try:
            forms["precision"] = precision_form(torch, dev, stream, flush, small, 2, names=("fp32", "tf32", "bf16"))
        except Exception as exc:  # reported, not hidden: the headline line still prints
            forms["precision"] = {"error": repr(exc)}
        try:
            forms["batched"] = batched_form(torch, dev, stream, flush, small, 1)
        except Exception as exc:
            forms["batched"] = {"error": repr(exc)}
        try:
            forms["differentiation"] = grad_form(torch, dev, small)
        except Exception as exc:
            forms["differentiation"] = {"error": repr(exc)}
    if rank == 0:
        cfg = workload_config(args.iters)
        cfg["parallelism"] = f"replicas x{ws} (independent completions per GPU)"
        cfg["entries_per_s"] = value * N
        cfg["wall_s_timed_region"] = t_wall
        line = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": 5 * args.iters * args.steps, "clocks": clocks, "nmse": nmse, "forms": forms}
        print(json.dumps(line), flush=True)
    for c in ctxs:
        c.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------------------
# precision form
# ---------------------------------------------------------------------------
def _resident(tc, torch, dev, w, inst, prec, flags, sptr):
    g = torch.from_numpy(wl.to_colmajor(inst["G"], np.float32 if prec != tc.TC_FP64 else np.float64)).to(dev)
    m = torch.from_numpy(wl.to_colmajor(inst["mask"], np.uint8)).to(dev)
    y = torch.from_numpy(wl.to_colmajor(inst["Y0"], np.float32 if prec != tc.TC_FP64 else np.float64)).to(dev)
    p = tc.make_params(w.n1, w.n2, w.n3, w.r, WEIGHTS["mu"], WEIGHTS["rho1"], WEIGHTS["rho2"], prec, flags=flags)
    torch.cuda.synchronize()
    return tc.Completion(p, g, m, y, on_device=True, stream=sptr)


def _timed(torch, stream, flush, fn, steps, warmup):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return sum(ms)


def precision_form(torch, dev, stream, flush, steps, warmup, names=None, with_nmse=True):
    """The precision form on the 529 x 96 x 112 workload (r = 32, 30% observed):
    completions of 30 iterations per step on resident inputs, per form; recovery
    NMSE of each against the FP64 path after the same iterations."""
    from paper_2005_09838_gb300 import tc, api
    sptr = stream.cuda_stream
    w = wl.c3(0.3)
    iters = w.iters
    inst = wl.as_precision(wl.generate(w), np.float32)
    forms = {"fp32": (tc.TC_FP32, 0), "tf32": (tc.TC_TF32, 0), "bf16": (tc.TC_BF16, 0),
             "tf32_single_pass": (tc.TC_TF32, tc.TC_FLAG_SINGLE_PASS),
             "bf16_single_pass": (tc.TC_BF16, tc.TC_FLAG_SINGLE_PASS)}
    if names:
        forms = {k: v for k, v in forms.items() if k in names}
    rates, kern = {}, {}
    for name, (prec, fl) in forms.items():
        # one completion (30 iterations from the initial point) per step, each on a
        # context initialised before the timed region
        cs = [_resident(tc, torch, dev, w, inst, prec, fl, sptr) for _ in range(warmup + steps)]
        it = iter(cs)
        ms = _timed(torch, stream, flush, lambda: next(it).iterate(iters, count=False), steps, warmup)
        rates[name] = iters * steps / (ms / 1e3)
        kern[name] = dict(zip(("qcon", "xstep", "ystep", "slab"), cs[0].profile(10)))
        for c in cs:
            c.close()
    nmse = {}
    if with_nmse:
        for name in ["fp64"] + [n for n in ("fp32", "tf32", "bf16") if n in forms]:
            o = api.complete(inst["G"], inst["mask"], inst["Y0"], w.r, iters, *WEIGHTS.values(), name,
                             objective=False)
            nmse[name] = wl.nmse(inst["M"], o["W"], inst["mask"])
    return {"workload": "529x96x112 traffic tensor (OD x 15-min slots x days), tubal rank 32, 30% observed",
            "iters_per_step": iters, "iters_per_s": rates,
            "speedup_vs_fp32": {k: v / rates["fp32"] for k, v in rates.items()} if "fp32" in rates else None,
            "kernel_ms_after_30_iters": kern, "nmse": nmse,
            "nmse_abs_diff_vs_fp64": {k: abs(v - nmse["fp64"]) for k, v in nmse.items()} if nmse else None,
            "entries_per_s": {k: v * w.N for k, v in rates.items()}}


def run_precision(args):
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    from paper_2005_09838_gb300 import build as _b
    _b.build()
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    with ClockSampler(0) as clk:
        names = [n for n in args.precision_forms.split(",") if n] or None
        res = precision_form(torch, dev, stream, flush, args.steps, args.warmup, names=names,
                             with_nmse=not args.no_nmse)
    rates = res["iters_per_s"]
    w = wl.c3(0.3)
    line = {"metric": "completion iters/s, precision form (TF32 tensor-core contractions, FP64-storage solves) "
                      "vs plain FP32, 529x96x112 r=32",
            "value": rates["tf32"], "unit": "iters/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": w.iters * 1e3 / rates["tf32"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "tf32 (split operands) / f32", "data": "synthetic",
            "config": {"workload": res["workload"], "iters_per_step": w.iters, "weights": WEIGHTS,
                       "l2": "flushed before every timed step", "entries_per_s": rates["tf32"] * w.N},
            "forms_iters_per_s": rates, "speedup_vs_fp32": res["speedup_vs_fp32"],
            "kernel_ms_after_30_iters": res["kernel_ms_after_30_iters"], "nmse": res["nmse"],
            "nmse_abs_diff_vs_fp64": res["nmse_abs_diff_vs_fp64"], "gpu_launches_per_iter": 10,  # qcon_tc, xbg, xbc, xg, xc, dcon_tc, ystep, zsyn_tc, slab; xa on a branch
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def grad_form(torch, dev, steps):
    """The differentiation form on the 529 x 288 x 168 workload (r = 16, 20%
    observed, rho1 = 1e-3, FP32): device time of one loss-and-gradient
    evaluation through torch.autograd at the seeded initial factors, and of one
    block step of block gradient descent (gradient plus backtracking
    evaluations)."""
    from paper_2005_09838_gb300 import autograd as ag
    w = wl.c4(0.2)
    inst = wl.as_precision(wl.generate(w), np.float32)
    rng = np.random.default_rng(w.seed + 17)
    X = torch.tensor(rng.standard_normal((w.n1, w.r, w.n3)), dtype=torch.float32, device=dev)
    Y = torch.tensor(inst["Y0"], dtype=torch.float32, device=dev)
    g = ag.grad_context(inst["G"], inst["mask"], w.r, 1e-3, dtype=torch.float32)
    Xr, Yr = X.clone().requires_grad_(True), Y.clone().requires_grad_(True)

    def evaluate():
        Xr.grad = None
        Yr.grad = None
        ag.factor_loss(Xr, Yr, g).backward()

    for _ in range(2):
        evaluate()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        evaluate()
    torch.cuda.synchronize()
    t_eval = (time.perf_counter() - t0) / steps
    Xf, Yf = np.fft.fft(X.cpu().numpy(), axis=2), np.fft.fft(inst["Y0"], axis=2)
    Ly = max(np.linalg.norm(Yf[:, :, k] @ Yf[:, :, k].conj().T, 2) for k in range(w.n3))
    Lx = max(np.linalg.norm(Xf[:, :, k].conj().T @ Xf[:, :, k], 2) for k in range(w.n3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, _, hist = ag.block_gradient_descent(g, X, Y, steps, 1.0 / Ly, 1.0 / Lx)
    torch.cuda.synchronize()
    t_bgd = (time.perf_counter() - t0) / (2 * steps)
    g.close()
    return {"workload": "529x288x168 traffic tensor, tubal rank 16, 20% observed, rho1 = 1e-3, FP32",
            "ms_per_loss_and_gradient": 1e3 * t_eval, "ms_per_block_step": 1e3 * t_bgd,
            "loss_first": hist[0], "loss_last": hist[-1], "block_steps": 2 * steps,
            "entries_per_s_loss_and_gradient": w.N / t_eval}


# ---------------------------------------------------------------------------
# batched form
# ---------------------------------------------------------------------------
BATCH = 64


def batch_workloads():
    rng = np.random.default_rng(2005_09838 + 5000)
    out = []
    for q in range(BATCH):
        n1, n2, n3 = int(rng.integers(64, 1025)), int(rng.integers(96, 289)), int(rng.integers(28, 169))
        r = int(rng.integers(4, 33))
        obs = float(rng.uniform(0.1, 0.6))
        out.append(wl.custom(n1, n2, n3, r, obs, seed=2005_09838 + 5000 + q, period=n2,
                             name=f"batch {q}: {n1}x{n2}x{n3} r={r}"))
    return out


NMSE_SAMPLE = range(0, BATCH, 8)  # instances whose recovery NMSE is compared (every eighth)


def _gen32_m(args):
    w, want_m = args
    inst = wl.as_precision(wl.generate(w), np.float32)
    m = inst["M"].astype(np.float32) if want_m else None
    return (wl.to_colmajor(inst["G"], np.float32), wl.to_colmajor(inst["mask"], np.uint8),
            wl.to_colmajor(inst["Y0"], np.float32), m, inst["mask"] if want_m else None)


def batched_form(torch, dev, stream, flush, steps, warmup):
    """The batched form: 64 seeded instances advanced together by one graph
    launch per iteration (mixed: TF32 tensor-core contractions where r > 16;
    fp32: plain FP32), against the same contexts iterated one after the other,
    and the recovery NMSE of every eighth instance (mixed against fp32, after
    the same iterations)."""
    import multiprocessing as mp
    from paper_2005_09838_gb300 import tc
    ws = batch_workloads()
    with mp.get_context("spawn").Pool(min(len(os.sched_getaffinity(0)), 32)) as pool:
        data = pool.map(_gen32_m, [(w, q in NMSE_SAMPLE) for q, w in enumerate(ws)])
    sptr = stream.cuda_stream
    iters = 10
    entries = sum(w.N for w in ws)

    def contexts(mixed):
        cs = []
        for w, (g, m, y, _, _) in zip(ws, data):
            prec = tc.TC_TF32 if (mixed and w.r > 16) else tc.TC_FP32
            p = tc.make_params(w.n1, w.n2, w.n3, w.r, WEIGHTS["mu"], WEIGHTS["rho1"], WEIGHTS["rho2"], prec)
            cs.append(tc.Completion(p, torch.from_numpy(g).to(dev), torch.from_numpy(m).to(dev),
                                    torch.from_numpy(y).to(dev), on_device=True, stream=sptr))
            torch.cuda.synchronize()
        return cs

    res, nmse = {}, {}
    for label, mixed in (("mixed", True), ("fp32", False)):
        cs = contexts(mixed)
        with tc.Batch(cs, stream=sptr) as B:
            B.iterate(2 * 4)  # tuning trials (two per candidate branch count), real iterations
            n0, _ = B.launches()
            ms = _timed(torch, stream, flush, lambda: B.iterate(iters), steps, warmup)
            n1, loop = B.launches()
            res[f"batch_{label}"] = BATCH * iters * steps / (ms / 1e3)
            res[f"branches_{label}"] = B.branches()
            res[f"graph_launches_per_call_{label}"] = (n1 - n0) / (steps + warmup)
            res[f"device_loop_{label}"] = loop
        tiles = {}
        for c in cs:
            tiles[str(c.tile())] = tiles.get(str(c.tile()), 0) + 1
        res[f"transform_tiles_{label}"] = tiles
        ms = _timed(torch, stream, flush, lambda: [c.iterate(iters, count=False) for c in cs], steps, warmup)
        res[f"sequential_{label}"] = BATCH * iters * steps / (ms / 1e3)
        for q in NMSE_SAMPLE:
            W, _, _ = cs[q].result_numpy()
            w = ws[q]
            Mq, maskq = data[q][3], data[q][4]
            nmse.setdefault(q, {})[label] = wl.nmse(Mq.astype(np.float64),
                                                    wl.from_colmajor(W, (w.n1, w.n2, w.n3)).astype(np.float64),
                                                    maskq)
        for c in cs:
            c.close()
        torch.cuda.synchronize()
    diffs = [abs(v["mixed"] - v["fp32"]) for v in nmse.values()]
    return {"workload": "64 traffic tensors, n1 64-1024, n2 96-288, n3 28-168, r 4-32, 10-60% observed",
            "instances": [w.name for w in ws], "iters_per_step": iters, "entries_total": entries,
            "instance_iters_per_s": res,
            "speedup_batched_mixed_vs_sequential_fp32": res["batch_mixed"] / res["sequential_fp32"],
            "speedup_batched_mixed_vs_batched_fp32": res["batch_mixed"] / res["batch_fp32"],
            "nmse_sample": {ws[q].name: v for q, v in nmse.items()},
            "nmse_max_abs_diff_mixed_vs_fp32": max(diffs),
            "iterations_per_instance_at_nmse": 8 + 2 * (warmup + steps) * iters}


def run_batched(args):
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    from paper_2005_09838_gb300 import build as _b
    _b.build()
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    with ClockSampler(0) as clk:
        res = batched_form(torch, dev, stream, flush, args.steps, args.warmup)
    value = res["instance_iters_per_s"]["batch_mixed"]
    line = {"metric": "instance-iterations/s, batched form (64 heterogeneous completions, one graph launch per "
                      "iteration, TF32 tensor cores where r > 16)",
            "value": value, "unit": "instance-iters/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": BATCH * res["iters_per_step"] * 1e3 / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "tf32 (split operands, r > 16) / f32",
            "data": "synthetic",
            "config": {"workload": res["workload"], "instances": res["instances"],
                       "iters_per_step": res["iters_per_step"], "entries_total": res["entries_total"],
                       "entries_per_s": value * res["entries_total"] / BATCH,
                       "l2": "flushed before every timed step"},
            "rates": res["instance_iters_per_s"], "speedup_vs_sequential_fp32":
                res["speedup_batched_mixed_vs_sequential_fp32"],
            "speedup_vs_batched_fp32": res["speedup_batched_mixed_vs_batched_fp32"],
            "nmse_max_abs_diff_mixed_vs_fp32": res["nmse_max_abs_diff_mixed_vs_fp32"], "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.form == "precision":
        run_precision(args)
    elif args.form == "batched":
        run_batched(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
