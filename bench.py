"""Benchmark: one EDA pass (build, block-Lanczos solve to rel-res 1e-6, recovery, projection).

A step is the whole hot path on one synthetic problem shaped like the largest face workload that fits
one GPU: 256x256 images, 200 classes of 10 images (d = 65536, n = 2000, t = 199, block size 32,
tau = 20), inputs resident in HBM (1.05 GB of samples: larger than the 129 MB L2, which is also flushed
by a 256 MB write before every step, outside the timed events). The solver is FP64 throughout; by
default (--prec tc) its products with [H_W H_B] and with the Krylov basis run as FP64-accurate
tensor-core products (error-free splitting into bf16 digit planes), --prec f64 keeps them on the FP64
pipe. The plain FP64 solver is timed beside it ("fp64_plain"), and the d = 4096, k = 40 workload (64x64
images) under "small_config".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference] [--workload NAME]

Prints one JSON line. Under torchrun each rank solves its own random split (weak scaling, no
collective on the data path); rank 0 prints the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1512_06500_gb300 import synth  # noqa: E402

METRIC = "EDA solve time to t Ritz pairs @rel-res 1e-6; exp-apply GB/s vs HBM peak"
NOMINAL_FP64_TFLOPS = 1.25          # GB300 FP64 (non-tensor), profiling recipe
HEADLINE = "d65536_k200"
SMALL = "d4096_k40"
# DRAM bytes (read + write) of one launch of the Gram SYRK kernel, k_gemm_tn_partial<32, double, SYRK>,
# per workload, from ncu captures (profiles/); None until captured for the current kernel
GRAM_TRAFFIC_BYTES = {}
# DRAM bytes (read + write) per launch of k_oz_gemm with a narrow operand, averaged over those launches of
# one timed step of the workload, from an ncu capture of the same command (profiles/); absent until captured
# for the current kernel
OZ_TRAFFIC_BYTES = {"d65536_k200": 599.07e6}
FALLBACK_HBM_GBS = 6800.0           # profiling recipe fallback when no measured peaks exist
FALLBACK_BF16_TFLOPS = 1900.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default=HEADLINE, choices=list(synth.CONFIGS) + ["batched64"])
    ap.add_argument("--small-steps", type=int, default=20, help="steps of the d4096_k40 leg (0: skip it)")
    ap.add_argument("--prec", default="tc", choices=["tc", "f64", "bf16"],
                    help="tc: FP64 solver whose sweeps over [H_W H_B], Grams and recovery run as FP64-accurate "
                         "tensor-core products (error-free splitting); f64: plain FP64 throughout; bf16: bf16 "
                         "sweeps on the tensor cores with FP64 small steps and refinement (the batched "
                         "workload's own precision; at tau = 20 and d = 65536 it does not converge)")
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="steps of the plain FP64 comparison leg on the same workload (0: skip it)")
    ap.add_argument("--direct-steps", type=int, default=2,
                    help="timed calls of the exact solve in span([H_W H_B]) (eda_solve_direct) beside the Krylov "
                         "solve on one handle of the workload (0: skip it)")
    ap.add_argument("--workers", type=int, default=32, help="host workers of the batched solve")
    ap.add_argument("--m-form", type=int, default=1, choices=[0, 1],
                    help="FP64 M-apply: 0 = the three products one after another, 1 = their composed form")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-exp-apply", action="store_true", help="skip the bf16 tensor-core exp-apply leg")
    ap.add_argument("--exp-apply-reps", type=int, default=30)
    ap.add_argument("--profile-exp-apply", default=None, metavar="D,K,NJ,B",
                    help="profiling driver: build a bf16 handle on a d x (K*NJ) Gaussian-cluster problem "
                         "and run three W exp-applies of width B, nothing else")
    ap.add_argument("--profile-timed", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    ap.add_argument("--profile-build", default=None, metavar="WORKLOAD",
                    help="profiling driver: one FP64 build of the named workload (its first split-K launch is "
                         "the Gram SYRK G_W = H_W^T H_W), nothing else")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            j = json.load(fh)
        return dict(hbm=float(j.get("hbm_gbs", FALLBACK_HBM_GBS)), bf16=float(j.get("bf16_tflops", FALLBACK_BF16_TFLOPS)),
                    bf16_sustained=float(j.get("bf16_tflops_sustained", FALLBACK_BF16_TFLOPS)), source="measured")
    return dict(hbm=FALLBACK_HBM_GBS, bf16=FALLBACK_BF16_TFLOPS, bf16_sustained=FALLBACK_BF16_TFLOPS, source="fallback")


# ---------------------------------------------------------------- clocks during the timed region

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload_config(args, name=None):
    name = name or args.workload
    if name == "batched64":
        return {"workload": "batched64: 64 independent problems, d in {1024, 4096, 16384}, k ~ U[10, 100], "
                            f"n_j ~ U[3, 10] per class, t = k - 1, tau = {synth.BATCHED['tau']}, tol={args.tol}",
                "l2": "flushed (256 MB write) before every step",
                "precision": {"tc": "FP64 solver with FP64-accurate tensor-core products (7 bf16 digit planes, exact "
                                    "integer accumulation)",
                              "bf16": "bf16 sweeps on the tensor cores (FP32 accumulation), FP64 Grams, small steps "
                                      "and refinement to tol",
                              }.get(getattr(args, "prec", "f64"), "plain FP64 sweeps and small steps")
                             + "; block size tuned per problem shape",
                "m_form": ["three products one after another", "composed form I + Z C Z^T"][args.m_form],
                "workers": args.workers}
    c = synth.CONFIGS[name]
    return {"workload": f"{name}: d={c['d']}, k={c['k']}, n_j={c['n_j']} (n={c['k'] * c['n_j']}), "
                        f"t={c['t']}, b={c['b']}, tau={c['tau']}, tol={args.tol}",
            "l2": "flushed (256 MB write) before every step; the samples (d n 8 bytes) are read from HBM",
            "precision": ("FP64 solver; the products with [H_W H_B], the Krylov basis and the n x n Grams (Grams, "
                          "M-apply sweeps, reorthogonalisation, Ritz vectors, K_W, recovery, projection) as "
                          "FP64-accurate tensor-core products: operands split exactly into 7 bf16 digit planes, exact "
                          "integer accumulation" if getattr(args, "prec", "f64") == "tc" else
                          ("bf16 sweeps on the tensor cores (FP32 accumulation), FP64 Grams, small steps and "
                           "refinement to tol" if getattr(args, "prec", "f64") == "bf16" else
                           "plain FP64 sweeps and small steps")),
            "m_form": ["three products one after another", "composed form I + Z C Z^T"][args.m_form]}


# ---------------------------------------------------------------- CPU oracle leg

def oracle_step(p, c, tol):
    import oracle as O
    sol = O.eda(p.X, p.labels, p.k, c["t"], tau=c["tau"], tier="projected")
    Ptr = O.project(sol["V"], p.X)
    Pte = O.project(sol["V"], p.Xtest)
    O.nn_classify(Ptr, p.labels, Pte)
    return sol


def oracle_problem(p, tau):
    """One batched problem through the oracle (projected exact FP64 route + 1-NN)."""
    import oracle as O
    sol = O.eda(p.X, p.labels, p.k, p.k - 1, tau=tau, tier="projected")
    O.nn_classify(O.project(sol["V"], p.X), p.labels, O.project(sol["V"], p.Xtest))
    return sol


def cpu_baseline_batched(ps, budget_s=20.0):
    """The oracle on a bounded sample of the batch (largest problems of each d first), scaled to one
    batch by the sample's share of the batch's estimated cost (d n^2 + d (n + k) k)."""
    def cost(p):
        return p.d * p.n * p.n + p.d * (p.n + p.k) * p.k
    order = sorted(range(len(ps)), key=lambda i: ps[i].d)
    picked, t0 = [], time.perf_counter()
    for i in order[:: max(1, len(order) // 8)]:
        oracle_problem(ps[i], synth.BATCHED["tau"])
        picked.append(i)
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    share = sum(cost(ps[i]) for i in picked) / sum(cost(p) for p in ps)
    return {"value": dt / share * 1e3, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{len(picked)} of the 64 problems (projected exact FP64 route + 1-NN) in {dt:.1f} s, "
                      f"scaled by their share {share:.3f} of the batch's d n^2 + d (n + k) k cost; numpy threads default"}


def cpu_baseline(p, c, tol, budget_s=12.0, max_reps=30):
    """The oracle as it stands, timed on the host cores on repeated solves of the same workload."""
    t0 = time.perf_counter()
    reps = 0
    while reps < max_reps and (reps == 0 or time.perf_counter() - t0 < budget_s):
        oracle_step(p, c, tol)
        reps += 1
    dt = (time.perf_counter() - t0) / reps
    return {"value": dt * 1e3, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{reps} full solves of the {p.name} workload (projected exact FP64 route + 1-NN), "
                      f"numpy threads default"}


# ---------------------------------------------------------------- multi-rank helpers (no collective on the data path)

def rank_problem(workload, rank):
    """The independent problem a rank solves: its own random split (weak scaling)."""
    return synth.config_problem(workload, split=rank)


def rank_batch_seed(rank):
    """Seed of the 64-problem batch a rank solves (every rank its own batch)."""
    return synth.BATCHED["seed"] + 1000 * rank


def max_over_ranks(value, device):
    """The maximum of a per-rank time over all ranks (the value itself on one process)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- bf16 tensor-core exp-apply leg

EXP_APPLY_WORKLOADS = ("d16384_k100", "d65536_k200")


def exp_apply_bytes(d, m, b, one_pass=False):
    """Algorithmic bytes of one exp-apply on the tensor cores, X (FP32) read twice and Y written once, plus:
    four-launch form Y = X + (H K)(H^T X): a sweep over bf16 H and one over bf16 H K (2 bytes each);
    one-pass form Y = X + sigma B (B^T X): bf16 B read once (it stays in shared memory for the second sweep)."""
    return (1 if one_pass else 2) * 2 * d * m + 3 * 4 * d * b


def exp_apply_leg(dev, flush, reps):
    """Cold-L2 timing of the Theorem 3.1 product exp(-c^2 H_W H_W^T / 2) X with bf16 H_W on the
    tensor cores, on the W factor of the mixed-precision workloads; CUDA events on the launching
    stream, the L2 flushed (256 MB write) before every call. Both forms where the one-pass form applies
    (the factor resident in shared memory: one launch), else the four-launch form alone."""
    import torch
    from paper_1512_06500_gb300 import eda

    pk = peaks()
    out = {}
    stream = torch.cuda.current_stream()
    for name in EXP_APPLY_WORKLOADS:
        c = synth.CONFIGS[name]
        p = synth.config_problem(name)
        X = torch.from_numpy(p.X).to(dev)
        lab = torch.from_numpy(p.labels).to(dev)
        b = c["b"]
        gen = torch.Generator(device=dev)
        gen.manual_seed(7)
        Xb = torch.randn(b, p.d, dtype=torch.float32, device=dev, generator=gen)
        Y = torch.empty_like(Xb)
        res = {}
        for form, fused in (("one_pass", 0), ("four_launch", -1)):
            h = eda.build(X, lab, p.k, eda.config(prec=eda.EDA_BF16, block_b=b, tau=c["tau"], tc_fused=fused))
            alpha = -0.5 * h.c2
            for _ in range(3):
                h.apply_exp(eda.OP_SW, Xb, alpha=alpha, out=Y)
            launches0 = eda.kernel_launches()
            ev = []
            for _ in range(reps):
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                e = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                h.apply_exp(eda.OP_SW, Xb, alpha=alpha, out=Y)
                e.record(stream)
                ev.append((a, e))
            torch.cuda.synchronize()
            per_call = (eda.kernel_launches() - launches0) / reps
            h.close()
            one = per_call == 1 or (b > 32 and per_call == (b + 31) // 32)
            if form == "one_pass" and not one:
                continue   # the factor does not fit: the default is the four-launch form
            us = sorted(a.elapsed_time(e) * 1e3 for a, e in ev)
            med = us[len(us) // 2]
            nbytes = exp_apply_bytes(p.d, p.n, b, one_pass=(form == "one_pass"))
            gbs = nbytes / med / 1e3
            res[form] = {"us_median": med, "us_min": us[0], "algorithmic_bytes": nbytes, "achieved_gbs": gbs,
                         "frac": gbs / pk["hbm"], "kernels_per_call": per_call}
        del X
        best = res.get("one_pass") or res["four_launch"]
        out[name] = dict({"d": p.d, "m": p.n, "b": b, "form": "one_pass" if "one_pass" in res else "four_launch",
                          "peak_gbs": pk["hbm"], "peak_source": pk["source"], "l2": "flushed before every call",
                          "two_pass_bytes": exp_apply_bytes(p.d, p.n, b)}, **best)
        if "one_pass" in res:
            out[name]["four_launch"] = res["four_launch"]
            out[name]["speedup_over_four_launch"] = res["four_launch"]["us_median"] / res["one_pass"]["us_median"]
        del p
    return out


def profile_exp_apply(spec):
    """Small fixed case for ncu: three W exp-applies, no timing."""
    import torch
    from paper_1512_06500_gb300 import build_lib, eda

    build_lib.build()
    d, k, nj, b = (int(v) for v in spec.split(","))
    p = synth.gaussian_clusters(d=d, k=k, n_per_class=nj, seed=3)
    X = torch.from_numpy(p.X).cuda()
    lab = torch.from_numpy(p.labels).cuda()
    h = eda.build(X, lab, p.k, eda.config(prec=eda.EDA_BF16, block_b=min(b, 16), tau=20.0))
    del X
    Xb = torch.randn(b, p.d, dtype=torch.float32, device="cuda")
    Y = torch.empty_like(Xb)
    for _ in range(3):
        h.apply_exp(eda.OP_SW, Xb, alpha=-0.5 * h.c2, out=Y)
    torch.cuda.synchronize()
    print(json.dumps({"mode": "profile-exp-apply", "d": d, "m": p.n, "b": b,
                      "checksum": float(Y.double().abs().sum().item())}))
    h.close()


# ---------------------------------------------------------------- GPU leg

def run_gpu_batched(args, rank, world, local_rank):
    """64 independent problems per step through eda_solve_batched (weak scaling: each rank its own batch)."""
    import torch
    from paper_1512_06500_gb300 import build_lib, eda

    build_lib.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    ps = synth.batched_problems(synth.BATCHED["count"], seed=rank_batch_seed(rank))
    Xs = [torch.from_numpy(p.X).to(dev) for p in ps]
    labs = [torch.from_numpy(p.labels).to(dev) for p in ps]
    probs = [dict(X=X, labels=lab, k=p.k, t=p.k - 1, tol=args.tol) for X, lab, p in zip(Xs, labs, ps)]
    cfg = eda.config(prec=PRECS[args.prec], block_b=0, tau=synth.BATCHED["tau"], m_form=args.m_form)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(pr=probs):
        res, code = eda.solve_batched(pr, cfg, workers=args.workers)
        if code != 0:
            raise RuntimeError(f"batched solve failed: {[r['status'] for r in res]}")
        return res

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    eda.profile_reset()
    eda.profile_enable(True)
    launches0 = eda.kernel_launches()
    clocks = ClockSampler(local_rank)
    clocks.start()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        res = step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    eda.profile_enable(False)
    launches = eda.kernel_launches() - launches0
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    ms = max_over_ranks(ms, dev)
    tri_ms, tri_calls = eda.profile_read("tridiag")
    tri_flops, _ = eda.profile_work("tridiag")
    breakdown = {r: eda.profile_read(r)[0] / args.steps
                 for r in ("gram", "symeig", "tridiag", "bisect", "invit", "backtransform", "m_apply", "exp_apply_w",
                           "exp_apply_b", "rr", "reorth")}
    ew = [eda.profile_read(r) for r in ("exp_apply_w", "exp_apply_b")]
    ewk = [eda.profile_work(r) for r in ("exp_apply_w", "exp_apply_b")]
    exp_ms = sum(v[0] for v in ew)
    exp_flops = sum(v[0] for v in ewk)
    exp_bytes = sum(v[1] for v in ewk)
    pk = peaks()
    tri_tf = tri_flops / (tri_ms / 1e3) / 1e12 if tri_ms > 0 else float("nan")
    rr = dict(regions={r: eda.profile_read(r) for r in REGIONS},
              work={r: eda.profile_work(r) for r in ("gram", "tn_f64", "nn_f64", "oz_gemm", "oz_kernel", "oz_tiled")})
    roofline = roofline_of("batched64", rr, args.steps, args.prec, pk)
    if args.prec == "tc" and ms > 0:
        # the problems run concurrently on many streams, so an event pair around one launch also spans other
        # problems' kernels: the rate is taken over the whole step instead (a lower bound for the kernel)
        oz_bytes = rr["work"]["oz_kernel"][1] / args.steps
        roofline["achieved"] = oz_bytes / (ms / 1e3) / 1e9
        roofline["frac"] = roofline["achieved"] / roofline["peak"]
        roofline["note"] = ("achieved = the narrow split products' algorithmic bytes per step / the whole step's "
                            "time (launches of 64 problems overlap on many streams): a lower bound")
        roofline.pop("avg_launch_us", None)
    tridiag = {
        "kernel": "k_tridiag_res / k_tridiag_cluster / k_tridiag: Householder tridiagonalisation (4/3 n^3 flops) of the FP64 "
                  "Grams and Rayleigh-Ritz matrices, summed over concurrent problems",
        "bound": "alu", "achieved": tri_tf, "peak": NOMINAL_FP64_TFLOPS, "unit": "TFLOP/s",
        "frac": tri_tf / NOMINAL_FP64_TFLOPS, "traffic": None,
        "peak_source": "nominal FP64 rate of the profiling recipe (own probe measured 1.19 TFLOP/s)",
        "note": "achieved = algorithmic flops / summed per-launch durations (launches overlap across streams)",
        "calls": tri_calls,
    }
    exp_apply_fp64 = {"calls": sum(v[1] for v in ew), "summed_ms_per_step": exp_ms / args.steps,
                      "achieved_tflops_per_launch": exp_flops / (exp_ms / 1e3) / 1e12 if exp_ms > 0 else None,
                      "algorithmic_gb_per_step": exp_bytes / args.steps / 1e9}
    # end to end: samples and labels from pinned host memory, V and lambda back to the host
    Xh = [torch.from_numpy(p.X).pin_memory() for p in ps]
    labh = [torch.from_numpy(p.labels).pin_memory() for p in ps]

    def e2e_step():
        pr = [dict(X=x.to(dev, non_blocking=True), labels=l.to(dev, non_blocking=True), k=p.k, t=p.k - 1,
                   tol=args.tol) for x, l, p in zip(Xh, labh, ps)]
        res = step(pr)
        out = [(r["V"].to("cpu", non_blocking=True), r["lam"].to("cpu", non_blocking=True)) for r in res]
        torch.cuda.current_stream().synchronize()
        return out

    e2e_step()
    e2e_ms = []
    for _ in range(max(2, args.steps // 2)):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e2e_step()
        b.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    h2d = sum(x.numel() * 8 + l.numel() * 4 for x, l in zip(Xh, labh))
    d2h = sum((p.k - 1) * (p.d + 1) * 8 for p in ps)
    e2e_v = sum(e2e_ms) / len(e2e_ms)
    e2e_v = max_over_ranks(e2e_v, dev)
    line = {
        "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (64 seeded Gaussian-cluster problems of uneven size; stand in for random training "
                "splits and class subsets of face sets)",
        "config": dict(workload_config(args), problems_per_s=1e3 * world * len(ps) / ms),
        "clocks": clk, "gpu_launches": launches,
        "e2e": {"value": e2e_v, "unit": "ms", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "roofline": roofline, "tridiag": tridiag, "exp_apply_fp64": exp_apply_fp64,
        "breakdown_ms_per_step_summed_over_streams": breakdown,
        "solve_info": {"mapplies_total": sum(r["info"]["mapplies"] for r in res),
                       "max_relres_est": max(r["info"]["max_relres_est"] for r in res)},
    }
    return line, ps


PRECS = {"tc": 4, "f64": 0, "bf16": 2}   # eda_prec codes: EDA_F64_TC, EDA_F64, EDA_BF16


def time_workload(name, steps, warmup, m_form, tol, dev, flush, rank, world, e2e=True, prec="tc",
                  profile_timed=False):
    """W untimed and K timed steps of one workload (build, solve, recovery, projection of the held-out
    set) with CUDA events on the launching stream, the L2 flushed before every step; optional end-to-end
    steps from pinned host buffers. Returns the per-step ms (max over ranks), the region timers read
    inside the timed region, the solve infos, the launch count and the end-to-end figures."""
    import torch
    from paper_1512_06500_gb300 import eda

    c = synth.CONFIGS[name]
    p = rank_problem(name, rank)
    X = torch.from_numpy(p.X).to(dev)
    lab = torch.from_numpy(p.labels).to(dev)
    Xt = torch.from_numpy(p.Xtest).to(dev)
    cfg = eda.config(prec=PRECS[prec], block_b=c["b"], tau=c["tau"], check_every=1, m_form=m_form)
    stream = torch.cuda.current_stream()

    def step():
        h = eda.build(X, lab, p.k, cfg)
        V, lam, _, info, code = h.solve(c["t"], tol)
        h.project(V, Xt)
        h.close()
        if code != 0:
            raise RuntimeError(f"{name}: solve did not converge: {info}")
        return info

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    eda.profile_reset()
    eda.profile_enable(True)
    launches0 = eda.kernel_launches()
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    wall0 = time.perf_counter()
    infos = []
    if profile_timed:
        torch.cuda.profiler.start()
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        infos.append(step())
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if profile_timed:
        torch.cuda.profiler.stop()
    wall = time.perf_counter() - wall0
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    eda.profile_enable(False)
    launches = eda.kernel_launches() - launches0
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / steps, dev)
    regions = {r: eda.profile_read(r) for r in REGIONS}
    work = {r: eda.profile_work(r) for r in ("gram", "tn_f64", "nn_f64", "oz_gemm", "oz_kernel", "oz_tiled", "m_apply_composed",
                                             "exp_apply_w", "tridiag")}
    out = dict(p=p, c=c, ms=ms, regions=regions, work=work, infos=infos, launches=launches, clocks=clk,
               wall=wall)
    if not e2e:
        return out
    # end to end through the public API: samples, labels and the held-out set from pinned host memory,
    # V, lambda and the projected held-out set back to pinned host memory, inside the timed region
    Xh = torch.from_numpy(p.X).pin_memory()
    labh = torch.from_numpy(p.labels).pin_memory()
    Xth = torch.from_numpy(p.Xtest).pin_memory()
    Vh = torch.empty((c["t"], p.d), dtype=torch.float64).pin_memory()
    lamh = torch.empty(c["t"], dtype=torch.float64).pin_memory()
    Ph = torch.empty((p.Xtest.shape[0], c["t"]), dtype=torch.float64).pin_memory()
    del X, Xt

    def e2e_step():
        Xd = Xh.to(dev, non_blocking=True)
        labd = labh.to(dev, non_blocking=True)
        Xtd = Xth.to(dev, non_blocking=True)
        h = eda.build(Xd, labd, p.k, cfg)
        V, lam, _, info, code = h.solve(c["t"], tol)
        P = h.project(V, Xtd)
        Vh.copy_(V, non_blocking=True)
        lamh.copy_(lam, non_blocking=True)
        Ph.copy_(P, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        h.close()
        if code != 0:
            raise RuntimeError(f"{name}: solve did not converge: {info}")

    e2e_steps = max(2, steps // 4)
    for _ in range(2):
        e2e_step()
    e2e_ms = []
    for _ in range(e2e_steps):
        flush.zero_()
        a, bb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e2e_step()
        bb.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(a.elapsed_time(bb))
    h2d = Xh.numel() * 8 + labh.numel() * 4 + Xth.numel() * 8
    d2h = Vh.numel() * 8 + lamh.numel() * 8 + Ph.numel() * 8
    out["e2e"] = {"value": max_over_ranks(sum(e2e_ms) / len(e2e_ms), dev), "unit": "ms",
                  "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
    return out


REGIONS = ("gram", "tn_f64", "nn_f64", "oz_gemm", "oz_kernel", "oz_tiled", "cluster_orth", "exp_apply_w", "exp_apply_b", "m_apply", "m_apply_composed",
           "tridiag", "bisect", "invit", "backtransform", "symeig", "lanczos", "phi_squaring", "rr", "reorth",
           "refine")


def direct_leg(name, prec, tol, steps, dev):
    """The exact solve in span([H_W H_B]) (eda_solve_direct) and the Krylov solve (eda_solve) timed on one
    handle of the workload (build excluded), with the largest relative difference of their eigenvalues."""
    import torch
    from paper_1512_06500_gb300 import eda

    c = synth.CONFIGS[name]
    p = synth.config_problem(name)
    cfg = eda.config(prec=PRECS[prec], block_b=c["b"], tau=c["tau"], check_every=1, m_form=1)
    out = {"workload": name, "unit": "ms"}
    with eda.build(torch.from_numpy(p.X).to(dev), torch.from_numpy(p.labels).to(dev), p.k, cfg) as h:
        for key, call in (("direct_ms", lambda: h.solve_direct(c["t"])[:2]),
                          ("krylov_ms", lambda: h.solve(c["t"], tol)[:2])):
            res = call()   # warm-up
            ts = []
            for _ in range(steps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                res = call()
                b.record()
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            out[key] = sum(ts) / len(ts)
            out["lam_" + key] = res[1].cpu().numpy()
    lam_d, lam_k = out.pop("lam_direct_ms"), out.pop("lam_krylov_ms")
    out["max_rel_diff_lambda"] = float(max(abs(lam_d / lam_k - 1.0)))
    out["note"] = ("eda_solve_direct: Cholesky of the Gram of n - 1 independent columns of [H_W H_B], the t largest "
                   "eigenpairs of the (n - 1)-dimensional projected matrix, recovery and orth in coordinates, one "
                   "pass over [H_W H_B]; eda_solve: block Lanczos to rel-res " + str(tol))
    return out


def rate(flops, ms):
    return flops / (ms / 1e3) / 1e12 if ms > 0 else float("nan")


def _all_launches(r, steps):
    tn_ms, tn_calls = r["regions"]["tn_f64"]
    nn_ms, nn_calls = r["regions"]["nn_f64"]
    oz_ms, oz_calls = r["regions"]["oz_kernel"]
    oz_flops, oz_bytes = r["work"]["oz_kernel"]
    return {
        "tn_f64": {"kernel": "k_gemm_tn_partial<*, double> (every FP64 split-K A^T B product of the step)",
                   "achieved_tflops": rate(r["work"]["tn_f64"][0], tn_ms), "launches": tn_calls,
                   "ms_per_step": tn_ms / steps},
        "nn_f64": {"kernel": "k_gemm_nn<*, double> (every FP64 tall A B product of the step)",
                   "achieved_tflops": rate(r["work"]["nn_f64"][0], nn_ms), "launches": nn_calls,
                   "ms_per_step": nn_ms / steps},
        "oz_kernel": {"kernel": "k_oz_gemm<narrow B> (tensor-core digit-plane products with a narrow operand of "
                                "<= 32 columns; the split of the narrow operand and the K-split reduction excluded)",
                      "achieved_gbs": oz_bytes / (oz_ms / 1e3) / 1e9 if oz_ms > 0 else None,
                      "tensor_tflops_bf16": rate(oz_flops, oz_ms) if oz_ms > 0 else None,
                      "launches": oz_calls, "ms_per_step": oz_ms / steps},
        "oz_tiled": {"kernel": "k_oz_gemm<tiled B> (both operands split: the Gram Z^T Z, the squaring's n x n "
                               "products); tensor-bound",
                     "tensor_tflops_bf16": rate(r["work"]["oz_tiled"][0], r["regions"]["oz_tiled"][0])
                     if r["regions"]["oz_tiled"][0] > 0 else None,
                     "peak_tflops_bf16": peaks()["bf16"],
                     "launches": r["regions"]["oz_tiled"][1], "ms_per_step": r["regions"]["oz_tiled"][0] / steps},
    }


def roofline_of(name, r, steps, prec, pk):
    """The dominant kernel of the step, on its launches inside the timed region (CUDA events around each
    launch, averaged).

    prec tc: k_oz_gemm, the FP64-accurate tensor-core product (largest share of the ncu launch list of
    the tensor-core step). Per launch it must read the seven bf16 digit planes of its split operand
    (14 M K bytes: Z^T or Z for the Grams and sweeps, the Krylov basis for its products) and of the
    narrow operand (14 K p) and write the M x p result (8 M p); its 28 digit-plane MMAs per 64 values of
    K (2 x 28 x 128 x 32 x 64 flops per 14 x 128 x 64 bytes of A: 128 flops per byte) sit below the bf16
    ridge point of 1866 TFLOP/s / 6768 GB/s = 276 flops per byte, so it is HBM-bound.

    prec f64: k_gemm_tn_partial<32, double, SYRK> + its split reduction on its largest launch, the Gram
    SYRK G_W = H_W^T H_W of the build, d n (n + 1) flops (one triangle), timed as the library's "gram"
    region. FP64-ALU bound: its flops per byte of H_W (n / 8) are far above GB300's FP64 ridge point."""
    if prec == "tc":
        ms, calls = r["regions"]["oz_kernel"]
        flops, nbytes = r["work"]["oz_kernel"]
        ach = nbytes / (ms / 1e3) / 1e9 if ms > 0 else float("nan")
        return {
            "kernel": "k_oz_gemm: FP64-accurate tensor-core product (7 bf16 digit planes per operand, tcgen05.mma "
                      "M=128 N=32 K=16 into tensor memory, exact integer folding), every Gram, sweep and basis "
                      "product of the step",
            "bound": "hbm", "achieved": ach, "peak": pk["hbm"], "unit": "GB/s", "frac": ach / pk["hbm"],
            "traffic": OZ_TRAFFIC_BYTES.get(name),
            "algorithmic_bytes_per_launch": nbytes / max(calls, 1),
            "avg_launch_us": ms * 1e3 / max(calls, 1), "launches": calls,
            "tensor_tflops_bf16": rate(flops, ms),
            "peak_source": f"{pk['source']} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
                           if pk["source"] == "measured" else "profiling recipe fallback",
            "all_launches": _all_launches(r, steps),
        }
    g_ms, g_calls = r["regions"]["gram"]
    g_flops, g_bytes = r["work"]["gram"]
    ach = rate(g_flops, g_ms)
    return {
        "kernel": "k_gemm_tn_partial<32, double, SYRK> + split reduction: FP64 Gram G_W = H_W^T H_W, "
                  "d n (n + 1) flops per launch",
        "bound": "alu", "achieved": ach, "peak": NOMINAL_FP64_TFLOPS, "unit": "TFLOP/s",
        "frac": ach / NOMINAL_FP64_TFLOPS,
        "traffic": GRAM_TRAFFIC_BYTES.get(name),
        "algorithmic_bytes_per_launch": g_bytes / max(g_calls, 1),
        "flops_per_launch": g_flops / max(g_calls, 1), "avg_launch_us": g_ms * 1e3 / max(g_calls, 1),
        "launches": g_calls,
        "peak_source": "nominal FP64 (non-tensor) rate of the profiling recipe; MEASURED_PEAKS.json has no FP64 "
                       "figure (own dependent-chain probe: 1.06-1.19 TFLOP/s attainable)",
        "all_launches": _all_launches(r, steps),
    }


def run_gpu(args, rank, world, local_rank):
    import torch
    from paper_1512_06500_gb300 import build_lib, eda

    build_lib.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    r = time_workload(args.workload, args.steps, args.warmup, args.m_form, args.tol, dev, flush, rank, world,
                      prec=args.prec, profile_timed=args.profile_timed)
    p, c = r["p"], r["c"]
    ms = r["ms"]
    regions = r["regions"]
    pk = peaks()
    roofline = roofline_of(args.workload, r, args.steps, args.prec, pk)
    tri_ms, tri_calls = regions["tridiag"]
    tri_flops, _ = r["work"]["tridiag"]
    latency_bound = {
        "kernel": "k_tridiag_res / k_tridiag_cluster / k_tridiag: Householder tridiagonalisation (4/3 n^3 flops) of the Rayleigh-Ritz "
                  "matrices (and of a Gram taking the eigensolver route)",
        "achieved_tflops": rate(tri_flops, tri_ms) if tri_ms > 0 else None,
        "avg_call_us": tri_ms * 1e3 / max(tri_calls, 1), "calls": tri_calls,
        "note": "latency-bound: n dependent column steps, each a chain of FP64 instructions (64 cycles per warp "
                "instruction on an SM sub-partition) and grid or cluster barriers",
    }
    region = "m_apply_composed" if args.m_form == 1 else "exp_apply_w"
    ew_ms, ew_calls = regions[region]
    ew_flops, ew_bytes = r["work"][region]
    ew_s = ew_ms / 1e3 if ew_ms > 0 else float("nan")
    if args.prec == "tc":
        # the sweeps read the seven bf16 digit planes of Z (14 bytes per entry) once each: HBM-bound
        m_apply = {
            "kernel": "composed M-apply on the tensor cores: M X = X + Z C Z^T X, Z = [H_W H_B], both sweeps "
                      "FP64-accurate digit-plane products (k_oz_gemm), C applied in FP64",
            "bound": "hbm", "achieved_gbs": ew_bytes / ew_s / 1e9, "peak_gbs": pk["hbm"],
            "frac": ew_bytes / ew_s / 1e9 / pk["hbm"], "peak_source": pk["source"],
            "fp64_equivalent_tflops": ew_flops / ew_s / 1e12,
            "avg_call_us": ew_ms * 1e3 / max(ew_calls, 1), "calls": ew_calls,
        }
    else:
        m_apply = {
            "kernel": ("composed M-apply (FP64): M X = X + Z C Z^T X, Z = [H_W H_B]" if args.m_form == 1
                       else "exp_apply (H_W, FP64 sweeps): Y = X + H_W K (H_W^T X)"),
            "bound": "alu",
            "achieved_tflops": ew_flops / ew_s / 1e12, "peak_tflops": NOMINAL_FP64_TFLOPS,
            "frac": ew_flops / ew_s / 1e12 / NOMINAL_FP64_TFLOPS,
            "achieved_gbs": ew_bytes / ew_s / 1e9, "hbm_peak_gbs": pk["hbm"], "hbm_peak_source": pk["source"],
            "avg_call_us": ew_ms * 1e3 / max(ew_calls, 1), "calls": ew_calls,
        }
    small = None
    if args.small_steps > 0 and args.workload != SMALL and rank == 0:
        rs = time_workload(SMALL, args.small_steps, 5, args.m_form, args.tol, dev, flush, rank, 1, prec=args.prec)
        small = {"workload": workload_config(args, SMALL)["workload"], "ms_per_step": rs["ms"], "unit": "ms",
                 "e2e_ms": rs["e2e"]["value"], "gpu_launches_per_step": rs["launches"] / args.small_steps,
                 "roofline": roofline_of(SMALL, rs, args.small_steps, args.prec, pk),
                 "solve_info": {kk: rs["infos"][-1][kk] for kk in ("iters", "mapplies", "checks", "basis_cols",
                                                                   "refills", "max_relres_est")}}
    fp64_leg = None
    if args.prec != "f64" and args.fp64_steps > 0 and rank == 0:
        # the plain FP64 GPU solver on the same workload, for the speedup at equal accuracy (both forms meet
        # the same oracle parity bars in the GPU tests)
        rf = time_workload(args.workload, args.fp64_steps, 1, args.m_form, args.tol, dev, flush, rank, 1, e2e=False,
                           prec="f64")
        fp64_leg = {"ms_per_step": rf["ms"], "speedup_of_tc_over_fp64": rf["ms"] / ms,
                    "breakdown_ms_per_step": {k: v[0] / args.fp64_steps for k, v in rf["regions"].items()},
                    "solve_info": {kk: rf["infos"][-1][kk] for kk in ("iters", "mapplies", "checks", "basis_cols",
                                                                     "refills", "refine_iters")}}
    direct = None
    if args.direct_steps > 0 and rank == 0 and args.workload != "batched64":
        direct = direct_leg(args.workload, args.prec, args.tol, args.direct_steps, dev)
    exp_leg = None
    if not args.no_exp_apply and rank == 0:
        exp_leg = exp_apply_leg(dev, flush, args.exp_apply_reps)
    line = {
        "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": ("synthetic (seeded low-rank smooth images plus noise; stands in for 256x256 face sets)"
                 if c["gen"] == "lowrank" else
                 "synthetic (seeded Gaussian class clusters clipped to [0, 1]; stands in for face sets)"),
        "config": dict(workload_config(args), solves_per_s=1e3 * world / ms),
        "clocks": r["clocks"], "gpu_launches": r["launches"],
        "e2e": r["e2e"],
        "roofline": roofline,
        "tridiag": latency_bound,
        "m_apply": m_apply,
        "exp_apply_bf16": exp_leg,
        "small_config": small,
        "fp64_plain": fp64_leg,
        "direct_solve": direct,
        "breakdown_ms_per_step": {k: v[0] / args.steps for k, v in regions.items()},
        "solve_info": {kk: r["infos"][-1][kk] for kk in ("iters", "mapplies", "checks", "basis_cols", "refills",
                                                         "refine_iters", "max_relres_est")},
        "wall_s": r["wall"],
    }
    return line, p, c


def profile_build(name, prec="f64"):
    """Small driver for ncu: one build of the named workload (FP64, or the tensor-core FP64 mode whose Grams
    are k_oz_gemm launches), nothing else."""
    import torch
    from paper_1512_06500_gb300 import build_lib, eda

    build_lib.build()
    c = synth.CONFIGS[name]
    p = synth.config_problem(name)
    X = torch.from_numpy(p.X).cuda()
    lab = torch.from_numpy(p.labels).cuda()
    h = eda.build(X, lab, p.k, eda.config(prec=PRECS[prec], block_b=c["b"], tau=c["tau"], m_form=1))
    torch.cuda.synchronize()
    print(json.dumps({"mode": "profile-build", "workload": name, "prec": prec, "c2": h.c2}))
    h.close()


def main():
    args = parse()
    if args.profile_exp_apply:
        profile_exp_apply(args.profile_exp_apply)
        return
    if args.profile_build:
        profile_build(args.profile_build, args.prec)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        if args.workload == "batched64":
            ps = synth.batched_problems(synth.BATCHED["count"], seed=synth.BATCHED["seed"])
            cb = cpu_baseline_batched(ps, budget_s=max(5.0, 60.0 / max(1, args.steps)))
            v = cb["value"]
            line = {"metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus, "steps": args.steps,
                    "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False, "scaling": "weak",
                    "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
                    "config": workload_config(args), "cpu_baseline": cb,
                    "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
            print(json.dumps(line))
            return
        c = synth.CONFIGS[args.workload]
        p = synth.config_problem(args.workload)
        for _ in range(args.warmup):
            oracle_step(p, c, args.tol)
        times = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            oracle_step(p, c, args.tol)
            times.append(time.perf_counter() - t0)
        v = 1e3 * sum(times) / len(times)
        line = {"metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
                "config": workload_config(args),
                "cpu_baseline": {"value": v, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
                                 "sample": f"{args.steps} full oracle solves of {args.workload}"},
                "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    if args.workload == "batched64":
        line, ps = run_gpu_batched(args, rank, world, local_rank)
        if rank == 0:
            if not args.no_cpu_baseline:
                line["cpu_baseline"] = cpu_baseline_batched(ps)
            print(json.dumps(line))
    else:
        line, p, c = run_gpu(args, rank, world, local_rank)
        if rank == 0:
            if not args.no_cpu_baseline:
                line["cpu_baseline"] = cpu_baseline(p, c, args.tol)
            print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
