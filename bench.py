#!/usr/bin/env python
"""Benchmark of the GB300 phylogenetic likelihood + gradient path.

One step = one pass of the whole hot path on one batch of synthetic input
(GTR+Gamma4, 512 taxa, 100,000 patterns, FP32 partials): device model set-up
and FP64 eigensystem, transition matrices and their derivatives, post-order
pruning with rescaling, root log-likelihood, fused pre-order pass with the
branch-length gradient. The metric counts post-order (pattern, internal
node) partials updates per second of that whole step.

  python bench.py [--gpus N --steps K --warmup W]      # this library
  python bench.py --impl reference                      # FP64 CPU oracle
Under torchrun (N > 1) each rank evaluates its own block of patterns (weak
scaling, no collective on the data path); rank 0 prints the JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pattern-node partials/s (4 & 61 states), grad evals/s; serving p50/p99 latency"
UNIT = "pattern-node/s"
DEFAULT_WORKLOAD = "gtr_512x100k"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--taxa", type=int, default=0, help="override the workload's taxa")
    ap.add_argument("--patterns", type=int, default=0, help="override the workload's patterns")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=0,
                    help="patterns in the oracle sample (0: sized to ~15 s)")
    ap.add_argument("--no-codon", action="store_true", help="skip the codon tensor-core line")
    ap.add_argument("--codon-only", action="store_true", help="only the codon line (profiling)")
    ap.add_argument("--codon-taxa", type=int, default=0)
    ap.add_argument("--codon-patterns", type=int, default=0)
    ap.add_argument("--serving", action="store_true",
                    help="continuous-batching serving run instead of the step benchmark")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--chains", type=int, default=128)
    ap.add_argument("--loads", default="0.5,0.8,1.2",
                    help="offered loads as fractions of the measured capacity")
    ap.add_argument("--baseline-seconds", type=float, default=60.0,
                    help="time budget of the one-at-a-time FP64 baseline")
    ap.add_argument("--adjoint-probe", default=None, metavar="WORKLOAD:PREC[:TAXA:PATTERNS]",
                    help="two forward + adjoint evaluations of one workload (a small launch "
                         "sequence for profiling the adjoint kernels)")
    ap.add_argument("--phylogeo", action="store_true",
                    help="one pattern, 64 states, 1,024 taxa: stored vs on-the-fly matrices")
    ap.add_argument("--autograd", action="store_true",
                    help="forward + backward through the autograd Function (GTR 1,024 x 50,000 "
                         "and GY94 64 x 5,000) in each precision against FP64")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# oracle timing: one thread, and every allowed host core (pattern chunks in
# spawned worker processes, one BLAS thread each)
# ---------------------------------------------------------------------------

def _oracle_step(w, Q, pi, tips, wt):
    from oracle import gradient as og, pruning as op
    op.loglik_chunked(w.tree, Q, pi, w.rates, w.cat_weights, wt, tips)
    og.branch_gradient(w.tree, Q, pi, w.rates, w.cat_weights, wt, tips)


def _oracle_worker(workload, lo, sample, steps, barrier, out):
    """One worker: logL + branch gradient of the FP64 oracle on patterns
    [lo, lo + sample) of the workload, ``steps`` times; every step starts at
    a barrier shared with the other workers, so a step's wall time is the
    latest end minus the common start."""
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    import numpy as np

    import synth
    from oracle import model as om
    w = synth.workload(workload)
    hi = min(lo + sample, w.n_patterns)
    tips = np.ascontiguousarray(w.tips[:, lo:hi])
    wt = w.pattern_weights[lo:hi]
    Q, pi, _ = om.build(w.model, w.params, w.freqs)
    res = []
    for _ in range(steps):
        barrier.wait()
        t0 = time.time()
        _oracle_step(w, Q, pi, tips, wt)
        res.append((t0, time.time()))
    out.put((hi - lo, w.tree.n_tips - 1, res))


def run_oracle(workload: str, sample: int, steps: int, cores: int) -> dict:
    """Time the oracle on ``cores`` worker processes (spawned, so no GPU
    state is inherited), each on its own ``sample`` consecutive patterns.
    Returns per-step wall times, units per step and the worker count."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    saved = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS",
                                             "MKL_NUM_THREADS", "CUDA_VISIBLE_DEVICES")}
    os.environ.update(OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1",
                      CUDA_VISIBLE_DEVICES="")
    try:
        barrier, out = ctx.Barrier(cores), ctx.Queue()
        procs = [ctx.Process(target=_oracle_worker,
                             args=(workload, i * sample, sample, steps, barrier, out))
                 for i in range(cores)]
        for pr in procs:
            pr.start()
        got = [out.get() for _ in procs]
        for pr in procs:
            pr.join()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    units = sum(g[0] for g in got) * got[0][1]
    walls = [max(g[2][s][1] for g in got) - min(g[2][s][0] for g in got) for s in range(steps)]
    return {"walls": walls, "units": units, "patterns": sum(g[0] for g in got), "workers": cores,
            "internal_nodes": got[0][1]}


def host_cores() -> tuple[int, int]:
    """(cores this process may run on, cores of the host)."""
    try:
        allowed = len(os.sched_getaffinity(0))
    except AttributeError:
        allowed = os.cpu_count() or 1
    return allowed, os.cpu_count() or allowed


def cpu_baseline(workload: str, sample: int) -> dict:
    """The oracle on one core and on every allowed core, each leg about
    10-15 s of CPU work: single-thread on the first ``sample`` patterns;
    all cores on ``sample`` patterns per core (consecutive chunks)."""
    allowed, total = host_cores()
    if sample <= 0:
        probe = run_oracle(workload, 500, 1, 1)
        per = probe["walls"][0] / 500
        sample = int(max(500, min(100_000 // max(1, allowed), 12.0 / max(per, 1e-9))))
        sample = (sample // 500) * 500
    one = run_oracle(workload, sample, 1, 1)
    v1 = one["units"] / one["walls"][0]
    par = run_oracle(workload, sample, 1, allowed) if allowed > 1 else one
    vn = par["units"] / par["walls"][0]
    return {"value": vn, "unit": UNIT, "cores": par["workers"], "kind": "oracle",
            "host_cores": total, "affinity_cores": allowed,
            "sample": f"{par['patterns']} patterns of {workload} ({sample} per worker process, "
                      f"{par['workers']} processes, one BLAS thread each), logL + branch gradient, "
                      f"FP64 numpy/scipy, {par['walls'][0]:.1f} s wall",
            "single_thread": {"value": v1, "cores": 1,
                              "sample": f"first {one['patterns']} patterns, "
                                        f"{one['walls'][0]:.1f} s"}}


def reference_arm(args) -> None:
    """The FP64 CPU oracle as it stands, same workload and metric, on every
    allowed host core (one worker process per core, each on its own chunk
    of patterns; every step is all workers' chunks)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    allowed, total = host_cores()
    sample = args.cpu_sample or 300
    r = run_oracle(args.workload, sample, args.warmup + args.steps, allowed)
    t = statistics.median(r["walls"][args.warmup:])
    value = r["units"] / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "sample_patterns": r["patterns"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": r["workers"],
                             "kind": "oracle", "host_cores": total, "affinity_cores": allowed,
                             "sample": f"{r['patterns']} patterns of {args.workload} per step "
                                       f"({sample} per worker process, {r['workers']} processes), "
                                       "logL + branch gradient, FP64 numpy/scipy"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, enabled: bool, device_id: str | None):
        self.proc = None
        self.path = None
        if not enabled:
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if device_id:
            cmd += ["-i", device_id]
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def device_id_for_smi() -> str | None:
    import torch
    try:
        u = str(torch.cuda.get_device_properties(0).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        return vis.split(",")[0] if vis else None


def peaks() -> tuple[float, str]:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def tf32_peak() -> tuple[float, str]:
    """Dense TF32 tensor peak: the measured BF16 burst figure times the
    nominal TF32:BF16 ratio (1:2)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return 0.5 * float(json.load(f)["bf16_tflops"]), "measured bf16 x 1/2"
    except (OSError, KeyError, ValueError):
        return 0.5 * 1900.0, "fallback bf16 x 1/2"


def codon_line(steps: int, warmup: int, taxa: int = 0, patterns: int = 0,
               prec: str = "tf32") -> dict:
    """GY94 128 taxa x 20,000 patterns on the tensor-core path (TF32;
    "tf32x2": matrices split into two TF32 terms; "tf32x3": FP32 partials
    split on chip as well, three products): one step = model + eigensystem,
    P and dP/dt, post-order, root logL, pre-order gradient. Algorithmic
    FLOPs count the contractions of internal children only (padded 64 x 64
    per category): post 1, gradient 3 per child; the split modes issue 2 or
    3 products for each ("issued"). Algorithmic bytes of the post-order
    pass: each internal child's partials read once, every internal node's
    partials and exponents written once, tip states read once. The step's
    gradient comes back under "_grad" (for the error columns)."""
    import numpy as np
    import torch

    import synth
    from paper_2606_27607_gb300 import TreeLikelihood
    over = {}
    if taxa:
        over["n_tips"] = taxa
    if patterns:
        over["n_patterns"] = patterns
    w = synth.workload("gy94_128x20k", **over)
    N, P = w.tree.n_tips, w.n_patterns
    stream = torch.cuda.current_stream()
    tl = TreeLikelihood(N, P, 61, 4, prec, stream=stream.cuda_stream)
    inst = tl.inst
    tl.set_tips(w.tips)
    tl.set_model("gy94", w.params, w.freqs)
    tl.set_rates(w.rates, w.cat_weights)
    tl.set_tree(w.tree.children, w.tree.edge_len)
    nn = tl.nn
    v = np.arange(nn - 1, dtype=np.int32)
    dp = (nn + v).astype(np.int32)
    lengths = np.ascontiguousarray(w.tree.edge_len[: nn - 1])
    d_out = torch.zeros(1 + nn, dtype=torch.float64, device="cuda")
    ev = {"post": [], "pre": []}

    def step(timed):
        inst.set_model_async(0, "gy94", w.params, w.freqs)
        inst.update_matrices(0, v, lengths, dp)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        e3 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        inst.update_partials(tl._post)
        e1.record(stream)
        inst.root_loglik_dev(nn - 1, 0, d_out.data_ptr())
        e2.record(stream)
        inst.pre_order_gradient_dev(tl._pre, nn, 0, d_out.data_ptr() + 8)
        e3.record(stream)
        if timed:
            ev["post"].append((e0, e1))
            ev["pre"].append((e2, e3))

    for _ in range(max(3, warmup)):
        step(False)
    torch.cuda.synchronize()
    inst.sync()
    n0 = inst.launch_count()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        step(True)
    b.record(stream)
    torch.cuda.synchronize()
    inst.sync()
    ms = a.elapsed_time(b) / steps
    k_ms = {k: statistics.mean(x.elapsed_time(y) for x, y in ev[k]) for k in ev}
    n_int_children = N - 2
    mult = {"tf32x2": 2, "tf32x3": 3}.get(prec, 1)
    f_post = n_int_children * 4 * 2 * 64 * 64 * P
    f_pre = 3 * f_post
    peak, src = tf32_peak()
    hbm, hsrc = peaks()
    ppad = (P + 127) // 128 * 128
    b_post = ppad * (n_int_children * 4 * 256 + (N - 1) * (4 * 256 + 4) + N)
    logl = float(d_out[0].item())
    grad = d_out[1:].cpu().numpy().copy()
    tl.close()
    how = {"tf32x2": " (P = P_hi + P_lo, two products)",
           "tf32x3": " (FP32 partials split on chip, P = P_hi + P_lo, three products)"}
    return {"workload": f"gy94_{N}x{P}",
            "precision": f"{prec} tcgen05" + how.get(prec, "") + ", fp32 accumulate",
            "value": P * (N - 1) / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "grad_evals_per_s": 1e3 / ms, "logL": logl, "_grad": grad,
            "kernels": {k: {"ms": k_ms[k],
                            "TFLOP/s": (f_post if k == "post" else f_pre) / (k_ms[k] * 1e-3) / 1e12,
                            "issued TFLOP/s": mult * (f_post if k == "post" else f_pre)
                                              / (k_ms[k] * 1e-3) / 1e12}
                        for k in k_ms},
            "hbm": {"kernel": "k_tc<post>", "algorithmic_bytes": b_post,
                    "achieved": b_post / (k_ms["post"] * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                    "frac": b_post / (k_ms["post"] * 1e-3) / 1e9 / hbm, "peak_source": hsrc},
            "roofline": {"bound": "tensor",
                         "kernel": ("k_tc_fused (subtree-fused post-order, tcgen05 kind::tf32)"
                                    if prec in ("tf32", "tf32x2") and
                                    os.environ.get("TL_TC_FUSED", "1") != "0"
                                    else "k_tc<post> (tcgen05 kind::tf32)"),
                         "achieved": f_post / (k_ms["post"] * 1e-3) / 1e12, "peak": peak,
                         "unit": "TFLOP/s",
                         "frac": f_post / (k_ms["post"] * 1e-3) / 1e12 / peak,
                         "peak_source": src}}


def per_component_err(g, ref) -> float:
    """max_i |g_i - ref_i| / max(|ref_i|, 1e-3 max_j |ref_j|)."""
    import numpy as np
    g, ref = np.asarray(g, float), np.asarray(ref, float)
    scale = float(np.max(np.abs(ref))) if ref.size else 0.0
    return float(np.max(np.abs(g - ref) / np.maximum(np.abs(ref), max(1e-3 * scale, 1e-300))))


def c64_taxa(line: dict) -> int:
    return int(line["workload"].split("_")[1].split("x")[0])


def traffic_for(kernel: str, per_launch_units: float) -> float | None:
    """ncu DRAM bytes of one launch, scaled from the capture recorded under
    profiles/ by the (pattern, internal node) units one launch processes, if
    the kernel source is unchanged since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    src = os.path.join(ROOT, "paper_2606_27607_gb300", "csrc", "tl_nuc.cu")
    try:
        rec = json.load(open(path))[kernel]
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if rec.get("source_sha256_16") != h:
            return None
        return rec["bytes_per_pattern_node"] * per_launch_units
    except (OSError, KeyError, ValueError):
        return None


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

# ---------------------------------------------------------------------------
# serving: continuous batching over many chains
# ---------------------------------------------------------------------------

def _pct(x, q):
    import numpy as np
    return float(np.percentile(np.asarray(x), q)) if len(x) else None


def serving_line(args) -> dict:
    """Poisson arrivals from many chains (taxa 16-1,024 and patterns
    100-200,000 log-uniform, 30% GY94 codon, half with gradients) through
    the continuous-batching server: capacity from a closed-loop pass, then
    p50/p99 latency at each offered load; next to the same requests served
    one at a time in FP64 (no batching) within a time budget."""
    import numpy as np
    import torch

    import synth
    from paper_2606_27607_gb300 import TreeLikelihood, build
    from paper_2606_27607_gb300.serve import Server, run_open_loop
    build.build()
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    chains, reqs, gaps = synth.serving_stream(args.requests, args.chains)
    t_gen = time.perf_counter() - t0
    work = [(chains[r.chain].tree.n_tips - 1) * chains[r.chain].n_patterns for r in reqs]
    server = Server()
    for w in chains:
        server.add_chain(w)
    resident = server.preload()
    clocks = Clocks(not args.no_clocks, device_id_for_smi())

    def summarise(futs, span, offered=None):
        ok = [i for i, f in enumerate(futs) if f.exception() is None]
        lat = [futs[i].result().latency for i in ok]
        gsz = [futs[i].result().group_size for i in ok]
        return {"offered_req_per_s": offered, "completed": len(ok),
                "rejected": len(futs) - len(ok), "seconds": span,
                "req_per_s": len(ok) / span,
                "pattern_node_per_s": sum(work[i] for i in ok) / span,
                "p50_s": _pct(lat, 50), "p99_s": _pct(lat, 99), "max_s": max(lat) if lat else None,
                "mean_group": float(np.mean(gsz)) if gsz else None}

    # warm-up (first launches, pinned staging), then capacity: every request
    # present at time 0
    warm = [server.submit(r) for r in reqs[:32]]
    server.drain()
    del warm
    t1 = time.perf_counter()
    futs, span = run_open_loop(server, reqs, np.zeros(len(reqs)))
    cap = summarise(futs, span)
    served = [f.result().logl if f.exception() is None else None for f in futs]
    capacity = cap["req_per_s"]
    loads = []
    for f in [float(x) for x in args.loads.split(",") if x]:
        arrivals = np.cumsum(gaps) / (f * capacity)
        futs, span = run_open_loop(server, reqs, arrivals)
        loads.append(dict(load=f, **summarise(futs, span, f * capacity)))
    t_serve = time.perf_counter() - t1
    clk = clocks.stop()
    stats = dict(server.stats)
    budget_gb = server.budget / 1e9
    n_codon = sum(chains[r.chain].n_states == 61 for r in reqs)
    server.close()
    del server
    torch.cuda.empty_cache()

    # one request at a time, FP64, no batching (codon through the FP64
    # generic path), in arrival order until the time budget is spent
    base_lat, base_work, base_err = [], 0, []
    cache: dict = {}
    tb = time.perf_counter()
    for i, r in enumerate(reqs):
        if time.perf_counter() - tb > args.baseline_seconds:
            break
        w = chains[r.chain]
        tl = cache.get(r.chain)
        if tl is None:
            for k in list(cache):
                cache.pop(k).close()
            torch.cuda.empty_cache()
            try:
                tl = TreeLikelihood(w.tree.n_tips, w.n_patterns, w.n_states, 4, "f64")
            except Exception:
                continue
            tl.inst.set_tip_states_all(w.tips)
            tl.set_rates(w.rates, w.cat_weights)
            tl.set_pattern_weights(w.pattern_weights)
            tl.set_model(w.model, w.params, w.freqs)
            cache[r.chain] = tl
        ts = time.perf_counter()
        tl.set_model(w.model, r.params, w.freqs)
        tl.set_tree(w.tree.children, r.edge_len)
        if r.gradient:
            l64, _ = tl.gradient()
        else:
            l64 = tl.loglik()
        base_lat.append(time.perf_counter() - ts)
        if served[i] is not None:
            base_err.append(abs(served[i] - l64) / abs(l64))
        base_work += (w.tree.n_tips - 1) * w.n_patterns
    for tl in cache.values():
        tl.close()
    t_base = sum(base_lat)
    baseline = {"kind": "fp64 one request at a time, no batching", "requests": len(base_lat),
                "req_per_s": len(base_lat) / t_base if t_base else None,
                "pattern_node_per_s": base_work / t_base if t_base else None,
                "p50_service_s": _pct(base_lat, 50), "p99_service_s": _pct(base_lat, 99),
                # the served logL (FP32 / split TF32, batched) of the same
                # requests against this FP64 evaluation
                "served_vs_fp64_rel_err_max": max(base_err) if base_err else None,
                "served_vs_fp64_rel_err_p99": _pct(base_err, 99)}
    return {"metric": "serving requests/s and p50/p99 latency (s) at offered load",
            "value": capacity, "unit": "requests/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": "f32 (4-state), tf32x3 (codon)", "data": "synthetic",
            "config": {"workload": "serving", "requests": len(reqs), "chains": len(chains),
                       "codon_requests": int(n_codon),
                       "gradient_requests": int(sum(r.gradient for r in reqs)),
                       "taxa": [16, 1024], "patterns": [100, 200000],
                       "resident_at_start": resident, "memory_budget_gb": budget_gb},
            "capacity": cap, "loads": loads, "server_stats": stats,
            "baseline_fp64_one_at_a_time": baseline, "clocks": clk,
            "generate_s": t_gen, "serve_s": t_serve}


def autograd_line(args) -> dict:
    """logL and its gradient (every branch length and every substitution
    parameter) through the torch.autograd Function, one forward + backward
    per evaluation (host-synchronous: the loss comes back as a number), on
    GTR+G4 1,024 taxa x 50,000 patterns (FP32, FP64), GY94 64 taxa x 5,000
    patterns (TF32, split TF32, FP64 generic) and the same GY94 with a random
    effect on each of its 263 non-zero rate pairs (265 parameters). The
    backward is one pre-order pass plus the adjoint pass. Latency per
    evaluation and the error of each precision against the FP64 GPU path;
    then, per workload, the backward's substitution gradient by three
    methods: the exact adjoint, the first-order approximation of the
    matrix-exponential derivative, and one pre-order pass per parameter
    (not available for the 263 random effects), with time and error."""
    import numpy as np
    import torch

    import synth
    from paper_2606_27607_gb300 import LogLikelihood, TreeLikelihood, build
    build.build()
    torch.cuda.set_device(0)
    out, methods = {}, {}
    eps = synth.random_effects()
    for name, base, precs, model in (("gtr_1024x50k", "gtr_1024x50k", ("f64", "f32"), "gtr"),
                                     ("gy94_64x5k", "gy94_64x5k", ("f64", "tf32", "tf32x2", "tf32x3"),
                                      "gy94"),
                                     ("gy94re_64x5k", "gy94_64x5k", ("f64", "tf32x3"), "gy94re")):
        w = synth.workload(base)
        params = np.r_[w.params, eps] if model == "gy94re" else np.asarray(w.params, float)
        res, ref = {}, None
        for prec in precs:
            tl = TreeLikelihood(w.tree.n_tips, w.n_patterns, w.n_states, 4, prec)
            tl.set_tips(w.tips)
            tl.set_model(model, params, w.freqs)
            tl.set_rates(w.rates, w.cat_weights)
            tl.set_pattern_weights(w.pattern_weights)
            tl.set_tree(w.tree.children, w.tree.edge_len)
            lat = []
            n_it = max(3, min(args.steps, 20))
            for it in range(3 + n_it):
                t = torch.tensor(w.tree.edge_len[:-1], dtype=torch.float64, requires_grad=True)
                th = torch.tensor(params, dtype=torch.float64, requires_grad=True)
                t0 = time.perf_counter()
                y = LogLikelihood.apply(t, th, tl, model, w.freqs)
                y.backward()
                gt, gk = t.grad.numpy().copy(), th.grad.numpy().copy()
                if it >= 3:
                    lat.append(time.perf_counter() - t0)
            r = {"evals_per_s": len(lat) / sum(lat), "p50_ms": 1e3 * _pct(lat, 50),
                 "p99_ms": 1e3 * _pct(lat, 99), "logL": float(y.detach()), "n_params": len(params)}
            if prec == "f64":
                ref = (float(y.detach()), gt, gk)
            else:
                r["rel_err_logL"] = abs(float(y.detach()) - ref[0]) / abs(ref[0])
                r["rel_err_grad_t"] = float(np.linalg.norm(gt - ref[1]) / np.linalg.norm(ref[1]))
                r["rel_err_grad_theta"] = float(np.max(np.abs(gk - ref[2])) /
                                                np.max(np.abs(ref[2])))
                r["grad_err_per_component_t"] = per_component_err(gt, ref[1])
                r["grad_err_per_component_theta"] = per_component_err(gk, ref[2])
            res[prec] = r
            if prec == precs[-1]:
                # the substitution gradient of the backward by three methods
                m = {}
                tl.loglik()

                def timed(f, n=5):
                    f()
                    torch.cuda.synchronize()
                    t1 = time.perf_counter()
                    for _ in range(n):
                        val = f()
                    torch.cuda.synchronize()
                    return 1e3 * (time.perf_counter() - t1) / n, val

                ms, (_, _, g_ex) = timed(lambda: tl.adjoint())
                m["adjoint_exact"] = {"backward_ms": ms, "rel_err_theta_vs_f64": float(
                    np.max(np.abs(g_ex - ref[2])) / np.max(np.abs(ref[2])))}
                ms, (_, _, g_fo) = timed(lambda: tl.adjoint(first_order=True))
                m["adjoint_first_order"] = {"backward_ms": ms, "rel_err_theta_vs_f64": float(
                    np.max(np.abs(g_fo - ref[2])) / np.max(np.abs(ref[2])))}
                if model != "gy94re":
                    ms, g_pp = timed(lambda: tl.subst_gradient(), 2)
                    m["pre_order_pass_per_parameter"] = {
                        "backward_ms": ms, "passes": len(params),
                        "rel_err_theta_vs_f64": float(np.max(np.abs(g_pp - ref[2])) /
                                                      np.max(np.abs(ref[2])))}
                methods[f"{name}/{prec}"] = m
            tl.close()
        out[name] = res
    return {"metric": "autograd forward+backward evaluations/s and latency", "unit": "evals/s",
            "n_gpus": 1, "data": "synthetic", "config": {"workload": "autograd"},
            "results": out, "substitution_gradient_methods": methods}


def phylogeo_line(args) -> dict:
    """One site pattern on 64 states (a discrete-location model), 1,024 taxa,
    FP64: logL with the transition matrices formed and stored (S^3 per edge
    and category, then pruning) against forming them on the fly inside
    pruning from the eigensystem (two S^2 products per edge and category).
    Both from the same eigensystem and partials buffers."""
    import numpy as np
    import torch

    import synth
    from paper_2606_27607_gb300 import TreeLikelihood, build, tree
    build.build()
    torch.cuda.set_device(0)
    w = synth.workload("geo64_1024x1")
    tl = TreeLikelihood(w.tree.n_tips, w.n_patterns, w.n_states, 4, "f64")
    tl.set_tips(w.tips)
    tl.set_model(w.model, w.params, w.freqs)
    tl.set_rates(w.rates, w.cat_weights)
    tl.set_tree(w.tree.children, w.tree.edge_len)
    ops = tree.eig_ops(w.tree.children, w.tree.n_tips, w.tree.edge_len)

    def stored():
        return tl.loglik()

    def fly():
        tl.inst.update_partials_eigen(ops)
        return tl.inst.root_loglik(tl.nn - 1, 0)

    res = {}
    for name, f in (("stored_matrices", stored), ("on_the_fly", fly)):
        for _ in range(3):
            val = f()
        lat = []
        for _ in range(max(5, min(args.steps, 50))):
            t0 = time.perf_counter()
            val = f()
            lat.append(time.perf_counter() - t0)
        res[name] = {"ms": 1e3 * _pct(lat, 50), "logL": val}
    tl.close()
    res["speedup"] = res["stored_matrices"]["ms"] / res["on_the_fly"]["ms"]
    res["rel_diff_logL"] = abs(res["on_the_fly"]["logL"] - res["stored_matrices"]["logL"]) / abs(
        res["stored_matrices"]["logL"])
    return {"metric": "single-pattern logL latency (host-synchronous)", "unit": "ms",
            "n_gpus": 1, "data": "synthetic", "dtype": "f64",
            "config": {"workload": "geo64_1024x1", "taxa": 1024, "states": 64, "patterns": 1},
            "results": res}


def adjoint_probe(spec: str) -> dict:
    """Forward pass and reverse-mode adjoint of one workload, twice."""
    import torch

    import synth
    from paper_2606_27607_gb300 import TreeLikelihood, build
    build.build()
    torch.cuda.set_device(0)
    parts = spec.split(":")
    kw = {} if len(parts) < 4 else dict(n_tips=int(parts[2]), n_patterns=int(parts[3]))
    w = synth.workload(parts[0], **kw)
    tl = TreeLikelihood(w.tree.n_tips, w.n_patterns, w.n_states, 4, parts[1])
    tl.set_tips(w.tips)
    tl.set_model(w.model, w.params, w.freqs)
    tl.set_rates(w.rates, w.cat_weights)
    tl.set_pattern_weights(w.pattern_weights)
    tl.set_tree(w.tree.children, w.tree.edge_len)
    for _ in range(2):
        logl = tl.loglik()
        g, _, th = tl.adjoint()
    torch.cuda.synchronize()
    tl.close()
    return {"workload": spec, "logL": logl, "dlogL_dtheta": [float(x) for x in th]}


def main() -> None:
    args = parse()
    if args.adjoint_probe:
        print(json.dumps(adjoint_probe(args.adjoint_probe)), flush=True)
        return
    if getattr(args, "phylogeo", False):
        print(json.dumps(phylogeo_line(args)), flush=True)
        return
    if args.autograd:
        print(json.dumps(autograd_line(args)), flush=True)
        return
    if args.serving:
        print(json.dumps(serving_line(args)), flush=True)
        return
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.taxa or args.patterns:
        args.no_cpu_baseline = True
    if args.codon_only:
        import torch

        from paper_2606_27607_gb300 import build
        build.build()
        torch.cuda.set_device(0)
        line = codon_line(args.steps, args.warmup, args.codon_taxa, args.codon_patterns,
                          os.environ.get("TL_CODON_PREC", "tf32"))
        line.pop("_grad", None)
        print(json.dumps(line))
        return

    import numpy as np
    import torch

    import synth
    from paper_2606_27607_gb300 import TreeLikelihood, build
    build.build()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    over = {}
    if args.taxa:
        over["n_tips"] = args.taxa
    if args.patterns:
        over["n_patterns"] = args.patterns
    w = synth.workload(args.workload, **over)
    N, P, S = w.tree.n_tips, w.n_patterns, w.n_states
    R = len(w.rates)
    stream = torch.cuda.current_stream()
    tl = TreeLikelihood(N, P, S, R, "f32", stream=stream.cuda_stream)
    inst = tl.inst
    tl.set_tips(w.tips)
    tl.set_model(w.model, w.params, w.freqs)
    tl.set_rates(w.rates, w.cat_weights)
    tl.set_pattern_weights(w.pattern_weights)
    tl.set_tree(w.tree.children, w.tree.edge_len)
    nn = tl.nn
    v = np.arange(nn - 1, dtype=np.int32)
    dp = (nn + v).astype(np.int32)
    lengths = np.ascontiguousarray(w.tree.edge_len[: nn - 1])
    d_out = torch.zeros(1 + nn, dtype=torch.float64, device="cuda")
    post, pre = tl._post, tl._pre

    ev = {k: [] for k in ("post", "pre")}

    def step(timed: bool) -> None:
        inst.set_model_async(0, w.model, w.params, w.freqs)            # a1
        inst.update_matrices(0, v, lengths, dp)                        # a2, a6
        if timed:
            e0 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        inst.update_partials(post)                                     # a3, a4
        if timed:
            e1 = torch.cuda.Event(enable_timing=True)
            e1.record(stream)
            ev["post"].append((e0, e1))
        inst.root_loglik_dev(nn - 1, 0, d_out.data_ptr())              # a5
        if timed:
            e2 = torch.cuda.Event(enable_timing=True)
            e2.record(stream)
        inst.pre_order_gradient_dev(pre, nn, 0, d_out.data_ptr() + 8)  # a7, a8
        if timed:
            e3 = torch.cuda.Event(enable_timing=True)
            e3.record(stream)
            ev["pre"].append((e2, e3))

    clocks = Clocks(not args.no_clocks and rank == 0, device_id_for_smi() if rank == 0 else None)
    t_w = time.perf_counter()
    n_w = 0
    while n_w < max(3, args.warmup) or (not args.no_clocks and time.perf_counter() - t_w < 1.0):
        step(False)
        n_w += 1
        if n_w % 50 == 0:
            torch.cuda.synchronize()
    torch.cuda.synchronize()
    inst.sync()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    n0 = inst.launch_count()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(args.steps):
        step(True)
    end.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = (inst.launch_count() - n0) // max(1, args.steps)
    clk = clocks.stop()
    inst.sync()
    ms = start.elapsed_time(end) / args.steps
    t_max = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    ms = float(t_max.item())
    logl = float(d_out[0].item())
    k_ms = {k: statistics.mean(a.elapsed_time(b) for a, b in ev[k]) for k in ev}

    # e2e: the public API with host buffers; tips, weights and parameters go
    # host -> device every step, logL and gradient come back
    e2e = None
    if not args.no_e2e:
        # Each step's tip states come from page-locked host memory (two
        # buffers, as a producer filling the next batch would use) through
        # the asynchronous double-buffered upload: step k queues its
        # kernels, then the upload of step k + 1's tips (it overlaps step k's
        # kernels), then reads its logL and gradient back to the host.
        tips_h = [torch.from_numpy(np.ascontiguousarray(w.tips)).pin_memory() for _ in range(2)]
        tips_np = [t.numpy() for t in tips_h]
        wts = np.ascontiguousarray(w.pattern_weights)
        d_res = torch.zeros(1 + nn, dtype=torch.float64, device="cuda")
        h_res = torch.zeros(1 + nn, dtype=torch.float64).pin_memory()
        nstep = [0]

        def e2e_step():
            k = nstep[0]
            nstep[0] += 1
            inst.set_pattern_weights(wts)
            inst.set_model_async(0, w.model, w.params, w.freqs)
            inst.update_matrices(0, v, lengths, dp)
            inst.update_partials(post)
            inst.root_loglik_dev(nn - 1, 0, d_res.data_ptr())
            inst.pre_order_gradient_dev(pre, nn, 0, d_res.data_ptr() + 8)
            inst.set_tip_states_all_async(tips_np[(k + 1) % 2])
            h_res.copy_(d_res, non_blocking=True)
            torch.cuda.current_stream().synchronize()
            return float(h_res[0]), h_res[1:].numpy()

        inst.set_tip_states_all_async(tips_np[0])
        for _ in range(3):
            e2e_step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        ke = max(3, args.steps // 2)
        for _ in range(ke):
            e2e_step()
        torch.cuda.synchronize()
        t_e2e = (time.perf_counter() - t0) / ke
        te = torch.tensor([t_e2e], dtype=torch.float64, device="cuda")
        if dist:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        t_e2e = float(te.item())
        # tips (one upload per step, for the next step) + padded weights +
        # model parameters + (rates, branch lengths); op lists and matrix
        # indices are unchanged between steps and stay resident (the library
        # skips identical uploads)
        h2d = (N * P + 8 * ((P + 31) // 32 * 32) + 8 * (len(w.params) + np.size(w.freqs))
               + 8 * (R + nn - 1))
        e2e = {"value": world * P * (N - 1) / t_e2e, "unit": UNIT, "ms_per_step": 1e3 * t_e2e,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(8 + 8 * nn)}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel. Algorithmic bytes per unit (pattern x
    # internal node) of the plain level-by-level formulation: post-order
    # 131 B (an internal child's 64 B partial read, a tip's state byte, the
    # 64 B partial and 2 B exponent written), pre-order and gradient 193 B
    # per parent (q 64 B read, the children's partials 65 B, q 64 B
    # written). The fused tile walks move less (children handed over on
    # chip, q never stored): their compulsory bytes are in "compulsory".
    hbm, src = peaks()
    RS = R * 4 * 4  # bytes of one pattern's FP32 partial, all categories
    alg = {"post": 131 * P * (N - 1), "pre": 193 * P * (N - 1)}
    comp = {"post": P * ((N - 1) * (RS + 4) + N * 1),
            "pre": P * ((N - 2) * RS + N * 1) + 8 * (2 * N - 2) * ((P + 31) // 32)}
    dom = max(k_ms, key=k_ms.get)
    ach = alg[dom] / (k_ms[dom] * 1e-3) / 1e9
    lpp = int(os.environ.get("TL_NUC_LANES", "1"))
    lpp = lpp if lpp in (1, 2, 4) else 1
    if dom == "pre":
        lpp = max(lpp, int(os.environ.get("TL_PRE_LANES", "0") or 0))
        lpp = lpp if lpp in (1, 2, 4) else 1
    kname = f"k_{dom}4<float,{lpp},{4 // lpp},4>"
    traffic = traffic_for(kname, P * (N - 1))
    roof = {"bound": "hbm", "kernel": kname, "achieved": ach, "peak": hbm, "unit": "GB/s",
            "frac": ach / hbm, "peak_source": src, "traffic": traffic,
            "algorithmic_bytes": alg[dom], "ms": k_ms[dom],
            "bytes_per_unit": {"post": 131, "pre": 193, "units": P * (N - 1)},
            "other": {k: {"ms": k_ms[k], "GB/s": alg[k] / (k_ms[k] * 1e-3) / 1e9,
                          "frac": alg[k] / (k_ms[k] * 1e-3) / 1e9 / hbm,
                          "compulsory_bytes": comp[k],
                          "compulsory_frac": comp[k] / (k_ms[k] * 1e-3) / 1e9 / hbm}
                      for k in k_ms}}

    codon = codon_split = codon_x3 = codon64 = fp64 = None
    if not args.no_codon and world == 1:
        try:
            codon = codon_line(max(5, args.steps // 20), 3)
            codon_split = codon_line(max(5, args.steps // 20), 3, prec="tf32x2")
            codon_x3 = codon_line(max(5, args.steps // 20), 3, prec="tf32x3")
            # the same split-matrix step with the level-by-level post-order
            # kernels instead of the subtree-fused one
            os.environ["TL_TC_FUSED"] = "0"
            try:
                lvl = codon_line(max(5, args.steps // 20), 3, prec="tf32x2")
            finally:
                os.environ.pop("TL_TC_FUSED", None)
            lvl.pop("_grad", None)
            codon_split["level_by_level"] = {"ms_per_step": lvl["ms_per_step"],
                                             "post_ms": lvl["kernels"]["post"]["ms"],
                                             "logL": lvl["logL"]}
        except Exception as exc:  # reported, not fatal
            codon = {"error": str(exc)[:300]}
        try:
            c64 = codon_line(3, 1, prec="f64")
            g64 = c64.pop("_grad")[: 2 * c64_taxa(c64) - 2]
            codon64 = {"ms_per_step": c64["ms_per_step"], "value": c64["value"],
                       "logL": c64["logL"], "path": "FP64 generic kernels, one tree at a time",
                       "speedup_tf32": c64["ms_per_step"] / codon["ms_per_step"]}
            for name, line_ in (("tf32", codon), ("tf32x2", codon_split), ("tf32x3", codon_x3)):
                gq = line_.pop("_grad")[: len(g64)]
                codon64[f"rel_err_logL_{name}"] = abs(line_["logL"] - c64["logL"]) / abs(c64["logL"])
                codon64[f"grad_err_per_component_{name}"] = per_component_err(gq, g64)
        except Exception as exc:  # reported, not fatal
            codon64 = {"error": str(exc)[:300]}
        for line_ in (codon, codon_split, codon_x3):
            if isinstance(line_, dict):
                line_.pop("_grad", None)
    if world == 1 and not args.taxa and not args.patterns:
        # the same step on the FP64 four-state kernels (the plain FP64 path)
        tl64 = TreeLikelihood(N, P, S, R, "f64", stream=stream.cuda_stream)
        tl64.set_tips(w.tips)
        tl64.set_model(w.model, w.params, w.freqs)
        tl64.set_rates(w.rates, w.cat_weights)
        tl64.set_pattern_weights(w.pattern_weights)
        tl64.set_tree(w.tree.children, w.tree.edge_len)
        d64 = torch.zeros(1 + nn, dtype=torch.float64, device="cuda")
        i64 = tl64.inst

        def step64():
            i64.set_model_async(0, w.model, w.params, w.freqs)
            i64.update_matrices(0, v, lengths, dp)
            i64.update_partials(tl64._post)
            i64.root_loglik_dev(nn - 1, 0, d64.data_ptr())
            i64.pre_order_gradient_dev(tl64._pre, nn, 0, d64.data_ptr() + 8)

        for _ in range(3):
            step64()
        torch.cuda.synchronize()
        a64, b64 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k64 = max(3, args.steps // 20)
        a64.record(stream)
        for _ in range(k64):
            step64()
        b64.record(stream)
        torch.cuda.synchronize()
        ms64 = a64.elapsed_time(b64) / k64
        l64 = float(d64[0].item())
        g32 = d_out[1:].cpu().numpy()
        g64 = d64[1:].cpu().numpy()
        fp64 = {"ms_per_step": ms64, "value": P * (N - 1) / (ms64 * 1e-3), "logL": l64,
                "path": "FP64 four-state kernels, one tree at a time",
                "speedup_fp32": ms64 / ms, "rel_err_logL_fp32": abs(logl - l64) / abs(l64),
                "rel_err_grad_fp32": float(np.linalg.norm(g32 - g64) / np.linalg.norm(g64)),
                "grad_err_per_component_fp32": per_component_err(g32[: nn - 1], g64[: nn - 1])}
        tl64.close()

    cpu = None
    if not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline(args.workload, args.cpu_sample)
        except Exception as exc:  # reported, not fatal
            cpu = {"error": str(exc)[:200]}

    value = world * P * (N - 1) / (ms * 1e-3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "model": w.model.upper() + "+G4",
                       "n_taxa": N, "n_patterns": P, "n_states": S, "n_categories": R,
                       "precision": "f32 partials, f64 eigensystem/reductions",
                       "step": "model+eigen, P and dP/dt, post-order, root logL, "
                               "pre-order gradient",
                       "l2": "no flush: partials working set "
                             f"{(N - 1) * P * RS / 1e9:.1f} GB > 129 MB L2",
                       "parallelism": f"patterns, weak x{world}"},
            "grad_evals_per_s": world * 1e3 / ms, "logL": logl, "clocks": clk, "e2e": e2e,
            "gpu_launches": int(launches) * args.steps, "gpu_launches_per_step": int(launches),
            "roofline": roof, "cpu_baseline": cpu, "fp64": fp64, "codon": codon,
            "codon_split": codon_split, "codon_x3": codon_x3, "codon_fp64": codon64}
    print(json.dumps(line), flush=True)
    tl.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
