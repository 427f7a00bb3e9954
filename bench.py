#!/usr/bin/env python
"""Throughput of the SCSC code update (Eq. 3 by proximal gradient with
randomized code-coordinate subsampling) on GB300.

One step = one scsc_code_step call over one batch: draw M^t, pack the warm
start on the sampled set, the step-size power iteration, n_iters proximal-
gradient iterations (masked synthesis, residual, adjoint at the sampled
coordinates, soft threshold), up-projection to dense codes (Eq. 4).
Metric: Gpix.filter/s = sum_n H_n W_n * K * n_iters / step time.

Default workload: 64 images 256x256 of the blob generator, K = 100 filters
11x11, p = 1/4, lambda = 1, 100 iterations per step, BF16 tensor path.
Multi-GPU: each rank processes its own batch (different image ids), no
collective on the data path; value = all ranks' work / max time.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores.
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

WORKLOADS = {
    # name: (H list builder, K, p, n_iters)
    "c3": dict(n=64, H=256, W=256, K=100, p=(1, 4), n_iters=100,
               desc="64 x 256x256 blob images, K=100 11x11, p=1/4, lambda=1, 100 PG its/step"),
    "c1": dict(n=1, H=100, W=100, K=16, p=(1, 2), n_iters=20,
               desc="1 x 100x100 blob image, K=16 11x11, p=1/2, lambda=1, 20 PG its/step"),
    "prof": dict(n=8, H=256, W=256, K=100, p=(1, 4), n_iters=4,
                 desc="8 x 256x256 blob images, K=100 11x11, p=1/4, lambda=1, 4 PG its/step "
                      "(small case for profiler captures)"),
    "c5": dict(n=512, H=None, W=None, K=100, p=(1, 4), n_iters=20,
               desc="512 blob images, H,W uniform in {64..512}, K=100 11x11, p=1/4, 20 PG its/step"),
    # inpainting (Sec. 4.3): ten 256x256 images, 50% of the pixels observed at
    # random, lambda = 0.4, 50 iterations, every code coordinate (p = 1)
    "inpaint": dict(n=10, H=256, W=256, K=100, p=(1, 1), n_iters=50, lam=0.4, observed=0.5,
                    desc="inpainting: 10 x 256x256 blob images, 50% pixels observed, K=100 11x11, "
                         "lambda=0.4, p=1, 50 PG its/step"),
    # the paper's ADMM code solver (Sec. 3.2) on its fruit-set shape: ten
    # 100x100 images, K=100, p=0.1, 10 ADMM iterations (20 CG steps each)
    "admm": dict(n=10, H=100, W=100, K=100, p=(1, 10), n_iters=10, solver="admm", cg_iters=20,
                 desc="ADMM code step: 10 x 100x100 blob images, K=100 11x11, p=1/10, lambda=1, "
                      "10 ADMM its x 20 CG steps/step (plain FP32 operators)"),
    # safe screening (Sec. 5) on the 64 x 256^2 batch: the duality-gap sphere
    # test before PG iterations 0, 25, 50 and 75 of each step
    "screen": dict(n=64, H=256, W=256, K=100, p=(1, 4), n_iters=100, solver="screen",
                   screen_every=25,
                   desc="screened code step: 64 x 256x256 blob images, K=100 11x11, p=1/4, "
                        "lambda=1, 100 PG its/step, gap-safe test every 25 its"),
}


def make_inputs(wl, rank):
    from paper_1909_00145_gb300 import inputs as I
    if wl["H"] is None:
        H, W = I.uneven_sizes(1000 + rank, wl["n"])
    else:
        H = np.full(wl["n"], wl["H"], dtype=np.int32)
        W = np.full(wl["n"], wl["W"], dtype=np.int32)
    ids = np.arange(wl["n"], dtype=np.int64) + rank * wl["n"]
    x = I.images(10 + rank, H, W)
    d = I.filters(7, wl["K"], 11)
    return H, W, ids, x, d


def reduce_over_ranks(v: float, op: str, device) -> float:
    """max or sum of a per-rank scalar over the ranks of the process group
    (the value itself with one rank or none)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return v
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def make_observed(wl, rank, H, W):
    """Observation mask of an inpainting workload (None for the others)."""
    from paper_1909_00145_gb300 import inputs as I
    if "observed" not in wl:
        return None
    return I.observed_pixels(20 + rank, int(np.dot(H.astype(np.int64), W)), wl["observed"])


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
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
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p["bf16_tflops"]), float(p.get("bf16_tflops_sustained",
                                                                        p["bf16_tflops"])), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, 1900.0, 1700.0, "fallback"


def source_code_sha1(text: str) -> str:
    """SHA-1 of a C++ source with its comments and whitespace runs removed:
    unchanged as long as the code itself is."""
    import hashlib
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    text = re.sub(r"\s+", " ", text).strip()
    return hashlib.sha1(text.encode()).hexdigest()


def measured_traffic(kernel: str, npx: int):
    """DRAM bytes per launch of `kernel` from the committed ncu counters of the
    small profiling workload, scaled by pixels; None if the kernel source's
    code has changed since the counters were taken."""
    names = {"adj_tc": ("tc_kernels_prof_workload_counters.json", "adj2_kernel"),
             "synth_tc": ("tc_kernels_prof_workload_counters.json", "syn2_kernel"),
             "fused": ("fused_kernel_prof_workload_counters.json", "fused_kernel")}
    try:
        fname, kname = names[kernel]
        with open(os.path.join(ROOT, "profiles", fname)) as f:
            c = json.load(f)
        with open(os.path.join(ROOT, c["source"])) as f:
            if source_code_sha1(f.read()) != c["source_code_sha1"]:
                return None
        k = c["kernels"][kname]
        return k["dram_bytes_per_launch"] * npx / c["workload_pixels"]
    except (OSError, KeyError, ValueError):
        return None


def launches_per_step(wl, path: str, n_iters: int, n_images: int, per_image: bool) -> int:
    """Kernels the library launches in one step of workload `wl` (counted from
    the host orchestration).  Proximal gradient: mask 1; step size: stencils
    2, power iteration 3 + 50 * 3 + 3; then per call on the active set
    plain: apply-mask 1 + per iteration synthesis and adjoint (one launch per
    image with per_image) and the observed-pixel mask when there is one;
    tensor: filter images 1, segment counts 1, scan 3, pack 1, A tiles 1,
    per iteration synthesis and adjoint (plus the residual pass with an
    observation mask), unpack 1.  Screening adds 7 per test (apply-mask, tap
    norms, synthesis, adjoint, statistics, per-image finish, test).  ADMM:
    mask 1, init 1, A^T x 1, per iteration rhs 1, QP 3, CG init 1, dots 2,
    per CG step QP 3 + dots 2 + update 2, shrink 1; final 1."""
    obs = "observed" in wl

    def pg(n):
        if path == "fp32":
            per_it = 2 * (n_images if per_image else 1) + (1 if obs else 0)
            return 1 + per_it * n
        return 1 + 1 + 3 + 1 + 1 + (3 if obs else 2) * n + 1

    if wl.get("solver") == "admm":
        return 1 + 2 + n_iters * (1 + 3 + 1 + 2 + 7 * wl["cg_iters"] + 1) + 1
    base = 1 + 2 + (3 + 50 * 3 + 3)
    if wl.get("solver") == "screen":
        e = wl["screen_every"]
        return base + sum(7 + pg(min(e, n_iters - i)) for i in range(0, n_iters, e))
    return base + pg(n_iters)


def cpu_baseline(wl, budget_s=20.0):
    """Time the FP64 oracle's proximal-gradient iterations on one image of the
    workload on the host cores (bounded sample)."""
    from oracle import reference as R
    H, W, ids, x, d = make_inputs(dict(wl, n=1), 0)
    cfg = R.Config(K=wl["K"], s=11, lam=wl.get("lam", 1.0), p_num=wl["p"][0], p_den=wl["p"][1],
                   seed=0)
    b = R.Batch(H=H[:1], W=W[:1], ids=ids[:1])
    z = np.zeros(int(H[0]) * int(W[0]) * wl["K"])
    obs = make_observed(dict(wl, n=1), 0, H[:1], W[:1])
    step = 1.0 / 200.0  # fixed step: the sample times the PG iterations only

    def run(n):
        if wl.get("solver") == "admm":
            m = R.mask_image(cfg, 1, int(ids[0]), int(H[0]), int(W[0])).ravel()
            R.admm_image(cfg, d, x, z, m, int(H[0]), int(W[0]), n, cg_iters=wl["cg_iters"])
        elif wl.get("solver") == "screen":
            R.code_step_screened(cfg, b, x, d, z, 1, n, wl["screen_every"], step=step)
        elif obs is None:
            R.code_step(cfg, b, x, d, z, 1, n, step=step)
        else:
            R.code_step_observed(cfg, b, x, d, z, obs, 1, n, step=step)
    t0 = time.perf_counter()
    run(1)
    one = time.perf_counter() - t0
    iters = max(1, int(budget_s / max(one, 1e-3)))
    t0 = time.perf_counter()
    run(iters)
    el = time.perf_counter() - t0
    pf = int(H[0]) * int(W[0]) * wl["K"] * iters
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    what = (f"{iters} ADMM iterations x {wl['cg_iters']} CG steps" if wl.get("solver") == "admm"
            else f"{iters} PG iterations, a screening test every {wl['screen_every']}"
            if wl.get("solver") == "screen" else f"{iters} PG iterations")
    return {"value": pf / el / 1e9, "unit": "Gpix*filter/s", "cores": cores, "kind": "oracle",
            "sample": f"1 image {int(H[0])}x{int(W[0])} of the workload, K={wl['K']}, "
                      f"{what} (FP64, adjoint at the sampled coordinates, OpenMP), {el:.1f} s"}


def run_reference(args, wl):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import reference as R
    H, W, ids, x, d = make_inputs(dict(wl, n=1), 0)
    cfg = R.Config(K=wl["K"], s=11, lam=wl.get("lam", 1.0), p_num=wl["p"][0], p_den=wl["p"][1],
                   seed=0)
    b = R.Batch(H=H[:1], W=W[:1], ids=ids[:1])
    z = np.zeros(int(H[0]) * int(W[0]) * wl["K"])
    obs = make_observed(dict(wl, n=1), 0, H[:1], W[:1])
    step = 1.0 / 200.0

    def run(z, n):
        if wl.get("solver") == "admm":
            m = R.mask_image(cfg, 1, int(ids[0]), int(H[0]), int(W[0])).ravel()
            return R.admm_image(cfg, d, x, z, m, int(H[0]), int(W[0]), n,
                                cg_iters=wl["cg_iters"])
        if wl.get("solver") == "screen":
            return R.code_step_screened(cfg, b, x, d, z, 1, n, wl["screen_every"], step=step)[0]
        if obs is None:
            return R.code_step(cfg, b, x, d, z, 1, n, step=step)
        return R.code_step_observed(cfg, b, x, d, z, obs, 1, n, step=step)
    t0 = time.perf_counter()
    run(z, 1)
    one = time.perf_counter() - t0
    per_step = max(1, int(4.0 / max(one, 1e-3)))
    for i in range(args.warmup):
        z = run(z, per_step)
    t0 = time.perf_counter()
    for i in range(args.steps):
        z = run(z, per_step)
    el = time.perf_counter() - t0
    pf = int(H[0]) * int(W[0]) * wl["K"] * per_step * args.steps
    val = pf / el / 1e9
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"impl": "reference", "metric": "code-update Gpix*filter/s", "value": val,
           "unit": "Gpix*filter/s", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": wl["desc"]},
           "cpu_baseline": {"value": val, "unit": "Gpix*filter/s", "cores": cores, "kind": "oracle",
                            "sample": f"1 image {int(H[0])}x{int(W[0])}, {per_step} PG its per step"},
           "e2e": {"value": val, "unit": "Gpix*filter/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def accuracy_report(n_images=4):
    """Errors of the BF16 and plain-FP32 paths against the FP64 oracle on the
    first images of the 64 x 256^2 workload: one outer iteration (100 PG
    iterations with the computed step) and one batch dictionary step; codes
    and filters as relative L2 errors, the objective (Eq. 1) after each step
    as a relative error.  One JSON line."""
    import time
    import torch
    from oracle import reference as R
    from paper_1909_00145_gb300 import scsc
    wl = dict(WORKLOADS["c3"], n=n_images)
    H, W, ids, x, d = make_inputs(wl, 0)
    K, n_iters = wl["K"], wl["n_iters"]
    cfg = R.Config(K=K, s=11, lam=1.0, p_num=wl["p"][0], p_den=wl["p"][1], seed=0)
    rb = R.Batch(H=H, W=W, ids=ids)
    t0 = time.perf_counter()
    zo = R.code_step(cfg, rb, x, d, np.zeros(rb.total_pixels * K), 1, n_iters)
    fzo = R.objective(cfg, rb, x, zo, d)
    do = R.dict_step_batch(cfg, rb, x, zo, d)
    fdo = R.objective(cfg, rb, x, zo, do)
    oracle_s = time.perf_counter() - t0

    def rel(a, b):
        a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    out = {}
    for prec in ["bf16", "fp32"]:
        ctx = scsc.Context(K, 11, 1.0, wl["p"], seed=0, prec=prec, stream=torch.cuda.Stream())
        batch = scsc.Batch(H, W, ids)
        xt = torch.from_numpy(x).cuda()
        dt = torch.from_numpy(np.ascontiguousarray(d)).cuda()
        z = torch.zeros(batch.total_pixels * K, device="cuda")
        torch.cuda.synchronize()
        with torch.cuda.stream(ctx.stream):
            ctx.code_step(batch, xt, dt, z, 1, n_iters)
            fz = ctx.objective(batch, xt, z, dt)
            ctx.dict_step(batch, xt, z, dt, scsc.SCSC_DICT_BATCH, 1)
            fd = ctx.objective(batch, xt, z, dt)
            ctx.sync()
        out[prec] = {"codes_rel_l2": rel(z.cpu().numpy(), zo),
                     "objective_after_codes_rel": abs(fz - fzo) / abs(fzo),
                     "filters_rel_l2": rel(dt.cpu().numpy(), do),
                     "objective_after_dict_rel": abs(fd - fdo) / abs(fdo)}
        ctx.close()
    print(json.dumps({"accuracy": out, "reference": "FP64 oracle",
                      "workload": f"{n_images} x 256x256 of the 64-image workload, K=100, p=1/4, "
                                  f"100 PG its + 1 batch dictionary step",
                      "oracle_seconds": oracle_s}), flush=True)


def dict_report(steps=5):
    """Time the dictionary steps (Eq. 5: simultaneous projected gradient, and
    the Gauss-Seidel pass over the filters) on the 64 x 256^2 workload with
    the codes of one code step; one JSON line."""
    import torch
    from paper_1909_00145_gb300 import scsc
    wl = WORKLOADS["c3"]
    H, W, ids, x_np, d_np = make_inputs(wl, 0)
    K = wl["K"]
    stream = torch.cuda.Stream()
    ctx = scsc.Context(K, 11, 1.0, wl["p"], seed=0, prec="bf16", stream=stream)
    batch = scsc.Batch(H, W, ids)
    x = torch.from_numpy(x_np).cuda()
    d0 = torch.from_numpy(d_np).cuda().contiguous()
    z = torch.zeros(batch.total_pixels * K, device="cuda")
    out = {"workload": "dictionary steps on " + wl["desc"], "n_gpus": 1, "steps": steps}
    with torch.cuda.stream(stream):
        ctx.code_step(batch, x, d0, z, 1, wl["n_iters"])
        for name, mode in [("jacobi", scsc.SCSC_DICT_BATCH), ("gauss_seidel", scsc.SCSC_DICT_BATCH_GS)]:
            d = d0.clone()
            ctx.dict_step(batch, x, z, d, mode, 1)  # warm-up
            ctx.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                ctx.dict_step(batch, x, z, d, mode, 1)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / steps
            f = ctx.objective(batch, x, z, d)
            out[name] = {"ms_per_step": ms, "objective_after": f}
        out["objective_before"] = ctx.objective(batch, x, z, d0)
    print(json.dumps(out), flush=True)


def online_profile_step():
    """One tensor code step of the online workload's first mini-batch (50 x
    100x100 images, K = 400 11x11, p = 1/10, 4 PG iterations), every kernel
    launched directly (no graph, no variant timing): a small case for ncu
    captures of the single-stage kernels."""
    import torch
    from paper_1909_00145_gb300 import inputs as I
    from paper_1909_00145_gb300 import scsc
    K, s, eta, side = 400, 11, 50, 100
    stream = torch.cuda.Stream()
    H = np.full(eta, side, dtype=np.int32)
    W = np.full(eta, side, dtype=np.int32)
    d = torch.from_numpy(I.filters(7, K, s)).cuda().contiguous()
    ctx = scsc.Context(K, s, 1.0, (1, 10), seed=0, prec="bf16", stream=stream,
                       flags=scsc.SCSC_FLAG_NO_GRAPH | scsc.SCSC_FLAG_NO_AUTOTUNE)
    with torch.cuda.stream(stream):
        batch = scsc.Batch(H, W, np.arange(eta))
        x = torch.from_numpy(I.images(5001, H, W)).cuda()
        z = torch.zeros(eta * side * side * K, device="cuda")
        ctx.code_step(batch, x, d, z, 1, 4)
        stream.synchronize()
    print(json.dumps({"online_profile_step": "ok", "l1": float(z.abs().sum())}), flush=True)


def online_report(prec="bf16", batches=4):
    """The online workload of Alg. 2 at its stated size, on a prefix of the
    stream: mini-batches of eta = 50 new 100x100 images, K = 400 filters of
    11x11, p = 1/10, lambda = 1, 20 PG iterations per mini-batch, each
    followed by the online dictionary step (Eq. 7 surrogate update, Eq. 8
    projected-gradient step with its power iteration on the 48,400 x 48,400
    surrogate).  The code step runs on `prec`: the tensor path (its
    single-stage kernels at this K) or the plain FP32 path.  One warm-up
    mini-batch, then `batches` timed ones; one JSON line with the code-update
    throughput and the dictionary step's time."""
    import torch
    from paper_1909_00145_gb300 import inputs as I
    from paper_1909_00145_gb300 import scsc
    K, s, eta, side, n_iters, p = 400, 11, 50, 100, 20, (1, 10)
    stream = torch.cuda.Stream()
    ctx = scsc.Context(K, s, 1.0, p, seed=0, prec=prec, stream=stream)
    H = np.full(eta, side, dtype=np.int32)
    W = np.full(eta, side, dtype=np.int32)
    d = torch.from_numpy(I.filters(7, K, s)).cuda().contiguous()
    npx = eta * side * side
    code_ms, dict_ms, dens = [], [], []
    with torch.cuda.stream(stream):
        for t in range(1, batches + 2):
            ids = np.arange(eta, dtype=np.int64) + (t - 1) * eta  # the stream's next images
            batch = scsc.Batch(H, W, ids)
            x = torch.from_numpy(I.images(5000 + t, H, W)).cuda()
            z = torch.zeros(npx * K, device="cuda")
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            ctx.code_step(batch, x, d, z, t, n_iters)
            e[1].record(stream)
            # the surrogate update runs on the nonzero codes below a density of
            # 1/16; denser codes would take the dense (K s^2)^2-per-pixel GEMM,
            # hours at this K, so the run stops instead
            frac = float((z != 0).float().mean())
            if frac * 16 > 1:
                print(json.dumps({"online": "stopped", "nonzero_code_fraction": frac}), flush=True)
                return
            ctx.dict_step(batch, x, z, d, scsc.SCSC_DICT_ONLINE, t)
            e[2].record(stream)
            e[2].synchronize()
            if t > 1:
                code_ms.append(e[0].elapsed_time(e[1]))
                dict_ms.append(e[1].elapsed_time(e[2]))
                dens.append(frac)
        f = ctx.objective(batch, x, z, d)
    cm, dm = float(np.mean(code_ms)), float(np.mean(dict_ms))
    print(json.dumps({
        "metric": "code-update Gpix*filter/s", "value": npx * K * n_iters / (cm * 1e-3) / 1e9,
        "unit": "Gpix*filter/s", "n_gpus": 1, "steps": batches, "warmup": 1,
        "higher_is_better": True, "dtype": prec, "data": "synthetic",
        "config": {"workload": f"online (Alg. 2): mini-batches of {eta} x {side}x{side} blob images, "
                               f"K={K} {s}x{s}, p=1/10, lambda=1, {n_iters} PG its per mini-batch, "
                               "then the online dictionary step"},
        "code_step_ms_per_batch": cm, "dict_step_ms_per_batch": dm,
        "mini_batches_per_s": 1e3 / (cm + dm), "nonzero_code_fraction": float(np.mean(dens)),
        "surrogate_bytes": (K * s * s) ** 2 * 4, "objective_last_batch": f}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default="bf16", choices=["bf16", "fp32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--per-image", action="store_true",
                    help="plain path: launch the kernels once per image (batched-launch baseline)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="tensor path: always use the pipelined kernels (for profiler captures)")
    ap.add_argument("--no-graph", action="store_true",
                    help="tensor path: launch iterations directly instead of replaying a graph")
    ap.add_argument("--accuracy", action="store_true",
                    help="print the BF16 / FP32 errors against the FP64 oracle on 4 images and exit")
    ap.add_argument("--dict", action="store_true",
                    help="time the Jacobi and Gauss-Seidel dictionary steps and exit")
    ap.add_argument("--online", action="store_true",
                    help="time the online workload at K=400 (Alg. 2 prefix) and exit")
    ap.add_argument("--online-profile", action="store_true",
                    help="run one K=400 tensor code step (small case for ncu captures) and exit")
    args = ap.parse_args()
    if args.online_profile:
        online_profile_step()
        return
    if args.online:
        online_report(args.prec)
        return
    if args.accuracy:
        accuracy_report()
        return
    if args.dict:
        dict_report()
        return
    if args.warmup < 3:
        args.warmup = 3
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl)
        return

    import torch
    import torch.distributed as dist
    from paper_1909_00145_gb300 import scsc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    H, W, ids, x_np, d_np = make_inputs(wl, rank)
    K, n_iters = wl["K"], wl["n_iters"]
    batch = scsc.Batch(H, W, ids)
    npx = batch.total_pixels
    stream = torch.cuda.Stream()
    x = torch.from_numpy(x_np).cuda()
    d = torch.from_numpy(d_np).cuda().contiguous()
    z = torch.zeros(npx * K, dtype=torch.float32, device="cuda")
    flags = (scsc.SCSC_FLAG_PER_IMAGE if args.per_image else 0) | \
        (scsc.SCSC_FLAG_NO_GRAPH if args.no_graph else 0) | \
        (scsc.SCSC_FLAG_NO_AUTOTUNE if args.no_autotune else 0)
    lam = wl.get("lam", 1.0)
    ctx = scsc.Context(K, 11, lam, wl["p"], seed=0, prec=args.prec, stream=stream, flags=flags)
    obs_np = make_observed(wl, rank, H, W)
    obs = torch.from_numpy(obs_np).cuda() if obs_np is not None else None
    screen_stats = {}  # screened workload: the last call's t, mean gap and survivors

    def code_step(c, x_, d_, z_, t, o=None):
        """One code step of the workload (inpainting: observed pixels only;
        the ADMM workload: the ADMM solver)."""
        if wl.get("solver") == "admm":
            c.code_step_admm(batch, x_, d_, z_, t, n_iters, wl["cg_iters"])
        elif wl.get("solver") == "screen":
            gaps, kept = c.code_step_screened(batch, x_, d_, z_, t, n_iters, wl["screen_every"])
            screen_stats.update(t=t, gap_mean=float(np.mean(gaps)), active=int(kept.sum()))
        elif obs is None:
            c.code_step(batch, x_, d_, z_, t, n_iters)
        else:
            c.code_step_observed(batch, x_, d_, z_, obs if o is None else o, t, n_iters)

    def barrier():
        if world > 1:
            dist.barrier()

    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            code_step(ctx, x, d, z, 1 + i)
        ctx.sync()
        z_warm = z.clone()
        sampler = ClockSampler(local)
        barrier()
        torch.cuda.synchronize()
        sampler.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(args.steps):
            code_step(ctx, x, d, z, 100 + i)
        e1.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        ctx.sync()
        barrier()
    # each rank runs its own batch (its own image ids; C5's sizes differ per
    # rank): the job's units are summed, its time is the slowest rank's
    ms = reduce_over_ranks(e0.elapsed_time(e1), "max", "cuda")
    per_step_ms = ms / args.steps
    units = reduce_over_ranks(float(npx * K * n_iters * args.steps), "sum", "cuda")
    value = units / (ms / 1e3) / 1e9

    # per-kernel device times: the same steps again with CUDA events around
    # every launch of the library (direct launches, no graph replay)
    kt = {}
    prof_steps = min(args.steps, 3)
    with torch.cuda.stream(stream):
        scsc.scsc_diag_profile(ctx, True)
        for i in range(prof_steps):
            code_step(ctx, x, d, z, 100 + i)
        ctx.sync()
        for name in ["fused", "synth_tc", "adj_tc", "finalize_r", "synth_fp32", "adjoint_fp32",
                     "pack", "unpack", "power", "mask", "screen"]:
            tot, n = scsc.scsc_diag_kernel_time(ctx, name)
            if n:
                kt[name] = (tot, n)
        scsc.scsc_diag_profile(ctx, False)

    # accuracy of this path against the plain FP32 path: one code step from
    # the same warm state, relative difference of the Eq. 1 objectives
    rel_err = None
    if args.prec != "fp32":
        with torch.cuda.stream(stream):
            ref = scsc.Context(K, 11, lam, wl["p"], seed=0, prec="fp32", stream=stream)
            za, zb = z_warm.clone(), z_warm.clone()
            code_step(ctx, x, d, za, 500)
            code_step(ref, x, d, zb, 500)
            if obs is None:
                fa = ctx.objective(batch, x, za, d)
                fb = ref.objective(batch, x, zb, d)
            else:
                fa = ctx.objective_observed(batch, x, za, d, obs)
                fb = ref.objective_observed(batch, x, zb, d, obs)
            rel_err = abs(fa - fb) / abs(fb)
            ref.close()
            del za, zb
    del z_warm

    dom = max(kt, key=lambda k: kt[k][0]) if kt else None
    hbm, bf16, bf16s, src = peaks()
    sampled = float(wl["p"][0]) / wl["p"][1] * npx * K  # expected sampled coordinates
    kw = (K + 31) // 32
    roof = None
    if dom is not None:
        # one launch covers the whole batch, or one image with --per-image:
        # time the kernel per PG iteration of the batch
        per_iter = len(H) if args.per_image else 1
        n_launch = kt[dom][1] / per_iter
        if dom == "fused":
            # one synthesis-only launch per step, then one per PG iteration:
            # its time is charged to the iterations
            n_launch -= prof_steps
        avg_s = kt[dom][0] / n_launch / 1e3
        # algorithmic bytes per launch (stated per kernel in the design notes)
        bytes_per_launch = {
            # the metric's algorithmic bytes per PG iteration (per pix*filter:
            # BF16 packed codes read and written 2 p b_z, one mask bit, the
            # image amortised over K, i.e. 2 p 2 + 1/8 + 4/K)
            "fused": 4 * sampled + npx * K / 8 + 4 * npx,
            # packed r+w, mask, and the residual: r itself with an observation
            # mask, else the synthesis output and the image it is formed from
            "adj_tc": 8 * sampled + 4 * kw * npx + (4 if obs is not None else 8) * npx,
            "synth_tc": 4 * sampled + 4 * kw * npx + 4 * npx,     # packed read, mask, xhat write
            "adjoint_fp32": 8 * sampled + 4 * kw * npx + 4 * npx,
            "synth_fp32": 4 * npx * K + 8 * npx,
        }.get(dom)
        if bytes_per_launch is not None:
            ach = bytes_per_launch / avg_s / 1e9
            roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm, "unit": "GB/s",
                    "frac": ach / hbm, "traffic": measured_traffic(dom, npx),
                    "algorithmic_bytes": bytes_per_launch, "peak_source": src,
                    "avg_ms_per_iteration": avg_s * 1e3}

    # end to end through the public API with host buffers: the library's
    # host-buffer entry (pinned memory; copies overlapped with the compute in
    # chunks of the batch) for the PG workloads, else device copies around the
    # device entry
    xh = torch.from_numpy(x_np).pin_memory()
    dh = torch.from_numpy(d_np).contiguous().pin_memory()
    zh = torch.zeros(npx * K, dtype=torch.float32).pin_memory()
    oh = torch.from_numpy(obs_np).pin_memory() if obs is not None else None
    host_entry = obs is None and wl.get("solver") is None
    with torch.cuda.stream(stream):
        xd, dd, zd = torch.empty_like(x), torch.empty_like(d), torch.empty_like(z)
        od = torch.empty_like(obs) if obs is not None else None
        if host_entry:  # warm-up: the chunks' kernel variant and graphs
            ctx.code_step_host(batch, xh, dh, zh, 199, n_iters)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for i in range(args.e2e_steps):
            if host_entry:  # z_host: the previous step's codes in, this step's out
                ctx.code_step_host(batch, xh, dh, zh, 200 + i, n_iters)
                continue
            xd.copy_(xh, non_blocking=True)
            dd.copy_(dh, non_blocking=True)
            zd.copy_(zh, non_blocking=True)
            if od is not None:
                od.copy_(oh, non_blocking=True)
            code_step(ctx, xd, dd, zd, 200 + i, od)
            zh.copy_(zd, non_blocking=True)
            stream.synchronize()
        e2e_s = time.perf_counter() - t0
    e2e_s = reduce_over_ranks(e2e_s, "max", "cuda")
    e2e_units = reduce_over_ranks(float(npx * K * n_iters * args.e2e_steps), "sum", "cuda")
    e2e_val = e2e_units / e2e_s / 1e9
    h2d = x.numel() * 4 + d.numel() * 4 + z.numel() * 4 + (obs.numel() if obs is not None else 0)
    d2h = z.numel() * 4

    if rank == 0:
        out = {"metric": "code-update Gpix*filter/s", "value": value, "unit": "Gpix*filter/s",
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": per_step_ms, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
               "config": {"workload": wl["desc"], "images_per_gpu": int(len(H)),
                          "pixels_per_gpu": npx, "K": K, "p": f"{wl['p'][0]}/{wl['p'][1]}",
                          "n_iters": n_iters, "lambda": lam, "path": args.prec,
                          **({"observed_fraction": wl["observed"]} if "observed" in wl else {}),
                          "launches": "per image" if args.per_image else "batched",
                          "graph": not args.no_graph,
                          "l2": "inputs larger than L2 (dense codes %.2f GB)" % (npx * K * 4 / 1e9)},
               "clocks": clocks,
               "roofline": roof,
               "kernels_ms_per_step": {k: v[0] / prof_steps for k, v in kt.items()},
               "rel_obj_err_vs_fp32": rel_err,
               "e2e": {"value": e2e_val, "unit": "Gpix*filter/s", "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h},
               "gpu_launches": launches_per_step(wl, args.prec, n_iters, len(H),
                                                 args.per_image) * args.steps}
        if screen_stats:
            with torch.cuda.stream(stream):
                bits = ctx.mask(batch, screen_stats["t"]).cpu().numpy()
            sampled = int(np.unpackbits(bits.view(np.uint8)).sum())
            out["screening"] = {"sampled_coordinates": sampled,
                                "active_after_last_test": screen_stats["active"],
                                "mean_gap_at_last_test": screen_stats["gap_mean"]}
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(wl)
        print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
