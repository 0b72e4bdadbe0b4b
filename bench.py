#!/usr/bin/env python
"""Throughput of the differential-BEM Levenberg-Marquardt hot path on GB300.

One step = one LM iteration of the mixed-precision path (panelize, boundary
right-hand side and solve, evaluation + residual + loss at every sample,
adjoint gradient, Gauss-Newton matrix, damped KKT solve, trial evaluation)
on the 32-curve / 2,048-panel / 1,048,576-sample workload.  Prints one JSON
line.  `--impl reference` times the FP64 CPU oracle instead (rank 0 only).

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torch.distributed.run, one independent replica per GPU (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gen  # noqa: E402

METRIC = ("LM iters/s & sample×panel evals/s (fwd+adjoint), mixed vs FP64 GPU at "
          "≤1e-4 RMSE")
UNIT = "LM iter/s"
CFG = 2            # the configuration the metric is quoted on
L2_FLUSH_BYTES = 256 << 20
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")


# regularisers of the 500-handle segment workload: length above twice the
# initial 1/20 of the width, snapping within 1% of the width, no sparsity
SEG_REG = dict(len_weight=1.0, len_max=0.1, snap_weight=1.0, snap_radius=0.01, snap_alpha=0.5)


def workload_desc(sc, cfg=CFG):
    noise = ("lognormal noise with 1% fireflies" if sc.noise.get("noise") == "lognormal"
             else "Gaussian noise")
    return (f"cfg{cfg}: {sc.n_curves} cubic Bezier curves x {int(sc.panels_per_curve[0])} panels "
            f"({sc.n_panels} panels), {sc.W}x{sc.W} px x {sc.spp} spp ({sc.n_samples} samples), "
            f"1024 boundary segments, {noise}")


def make_inputs(rank: int, cfg: int = CFG):
    sc = gen.make_scene(cfg)
    seed = sc.seed + 7919 * rank        # independent sample set per replica
    xy = gen.make_samples(sc.W, sc.spp, seed, dtype=np.float32)
    truth = gen.analytic_truth(xy, sc.seed)
    target = gen.add_noise(truth, sc.noise, seed).astype(np.float32)
    return sc, xy, target


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic work per unit, counted from the source formulas (FP32 flops:
# add/mul = 1, FMA = 2, one special-function op = 1; compares, selects and
# min/max are not counted)

# handle pair of the evaluation: rounded frame 9, h^2 1, h', q1, q2, t1 t2 8, atan2(h'L, h'^2 + t1 t2) 22 (octant reduction, one
# reciprocal, degree-7 minimax polynomial), S from t2 log q2 - t1 log q1 9 (two
# logarithms, one product, three multiply-adds), Dl 2, 3-channel accumulation 12
FLOP_FWD_HANDLE = 9 + 1 + 8 + 22 + 9 + 2 + 12
# boundary pair: vertex offset 2, cross 3, dot 3, atan2 20, 3-channel accumulation 6
FLOP_FWD_BOUND = 2 + 3 + 3 + 20 + 6
# F-row pair: frame 10, values and frame partials of both layers 57 (both
# logarithms taken directly), chain rule to both endpoints for Dl and S 43,
# jump columns 16, 3 channels x 2 coordinates x (combine 7 + four Bernstein
# accumulations 8) 90
FLOP_FROWS_PAIR = 10 + 57 + 43 + 16 + 90
# FP32 lanes x 2 flops per FMA x SMs x max SM clock (GB300: 128, 152, 2070 MHz)
FP32_PEAK_TFLOPS = 128 * 2 * 152 * 2.070e9 / 1e12


def step_work(name, n, P, Nb, nc):
    """(flops of one LM step's launches of `name`, bound) for the modelled
    kernels; for k_field the flops of one launch (every launch evaluates all
    samples, and the step has one or two of them)."""
    if name == "k_field":            # one evaluation of every sample (per launch)
        return n * (P * FLOP_FWD_HANDLE + Nb * FLOP_FWD_BOUND), "alu_per_launch"
    if name == "k_field_bnd":        # boundary term of every sample, in chunks
        return float(n) * Nb * FLOP_FWD_BOUND, "alu"
    if name == "k_frows":            # all samples, plus the 3 Nb boundary Gauss points
        return float(n + 3 * Nb) * P * FLOP_FROWS_PAIR, "alu"
    if name == "tc_jrows":           # J^T = M_c^T Phi^T (+ F^T) for 3 channels
        return 2.0 * 3 * nc * Nb * n, "tensor"
    if name == "tc_syrk":            # 3 symmetric rank-n updates of order nc
        return 3.0 * nc * (nc + 1) * n, "tensor"
    return None, None


def read_peaks():
    try:
        with open(PEAKS) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def kernel_traffic(name, cfg=CFG):
    """DRAM bytes per launch from the committed ncu summary, or None when the
    kernel's sources have changed since the counters were taken or the
    counters were taken on another configuration."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
            rec = json.load(f).get(name)
        if not rec or rec.get("config") != cfg:
            return None
        h = hashlib.sha256()
        for src in rec["sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
        return rec["bytes_per_launch"] if h.hexdigest() == rec["sha256"] else None
    except (OSError, ValueError, KeyError):
        return None


def rooflines(prof, steps, n, P, Nb, nc, cfg=CFG):
    peaks, src = read_peaks()
    out = []
    for name, (ms, cnt) in prof.items():
        work, bound = step_work(name, n, P, Nb, nc)
        if work is None or not cnt:
            continue
        if bound == "alu_per_launch":
            per_launch, bound = work, "alu"
        else:
            per_launch = work * steps / cnt
        ach = per_launch / (ms / cnt / 1e3) / 1e12
        if bound == "alu":
            peak, psrc = FP32_PEAK_TFLOPS, "FP32: 128 lanes x 2 x 152 SMs x 2070 MHz (derived)"
        else:
            peak = peaks["bf16_tflops_sustained"]
            psrc = f"bf16 dense, sustained ({src})"
        out.append({"bound": bound, "kernel": name, "achieved": ach, "peak": peak,
                    "unit": "TFLOP/s", "frac": ach / peak, "traffic": kernel_traffic(name, cfg),
                    "flops_per_launch": per_launch, "peak_source": psrc,
                    "share_ms": ms})
    out.sort(key=lambda r: -r.pop("share_ms"))
    return out


# ---------------------------------------------------------------------------

def oracle_rate(sc, xy, target, n_sub: int, steps: int, warmup: int = 0) -> dict:
    """The oracle as it stands, timed on bounded samples of the same workload.

    One LM step costs a + b n on n samples (a: boundary Jacobian and other
    per-iteration work, b: per-sample evaluation and Jacobian rows).  One step
    on n_sub/2 samples and `steps` steps on n_sub samples fit a and b; the full
    workload's time per iteration is a + b S.
    """
    import oracle
    mean = np.minimum(target, 1.0).mean(0)
    o = oracle.Oracle.from_scene(sc, mean_color=mean)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(xy.shape[0], n_sub, replace=False))
    x, t = xy[idx].astype(np.float64), target[idx].astype(np.float64)
    th, lam = sc.theta_init.copy(), 1e-3
    for _ in range(warmup):
        res = o.lm_step(th, x, t, lam)
        th, lam = res["theta"], res["lambda_next"]
    h = n_sub // 2
    t0 = time.perf_counter()
    o.lm_step(th, x[:h], t[:h], lam)
    t_half = time.perf_counter() - t0
    t0 = time.perf_counter()
    for _ in range(max(steps, 1)):
        res = o.lm_step(th, x, t, lam)
        th, lam = res["theta"], res["lambda_next"]
    t_full = (time.perf_counter() - t0) / max(steps, 1)
    b = max((t_full - t_half) / (n_sub - h), t_full / n_sub * 0.5)
    a = max(t_full - b * n_sub, 0.0)
    per_iter = a + b * xy.shape[0]
    return {"value": 1.0 / per_iter, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": (f"FP64 oracle LM steps on {h} and {n_sub} of {xy.shape[0]} samples "
                       f"({t_half:.2f} s, {t_full:.2f} s); per-iteration time a + b S with "
                       f"a = {a:.2f} s, b = {b * 1e3:.3f} ms/sample"),
            "ms_per_step": per_iter * 1e3}


def cpu_baseline(sc, xy, target, n_sub: int) -> dict:
    r = oracle_rate(sc, xy, target, n_sub, steps=1)
    r.pop("ms_per_step")
    return r


def run_reference(args, rank, world):
    if rank != 0:
        return
    sc, xy, target = make_inputs(0)
    r = oracle_rate(sc, xy, target, args.cpu_samples, steps=args.steps, warmup=args.warmup)
    v = r["value"]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_desc(sc)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_quadrants(bg, quads, flush, stream, n):
    """Four quadrant subdomains stepped together by one bem_batch_lm call."""
    import torch
    bq = bg.BEMBatch([q[0] for q in quads])
    lq = [1e-3, 1e-2, 1e-1, 1.0]
    bq.lm_step([q[1] for q in quads], [q[2] for q in quads], lq)
    torch.cuda.synchronize()
    e0q, e1q = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    qms = 0.0
    for _ in range(2):
        flush.zero_()
        e0q.record(stream)
        bq.lm_step([q[1] for q in quads], [q[2] for q in quads], lq)
        e1q.record(stream)
        torch.cuda.synchronize()
        qms += e0q.elapsed_time(e1q) / 2
    bq.close()
    return {"subdomains": 4, "boundary": "each quadrant a square subdomain, 128 segments "
            "per edge", "curves_per_subdomain": 8, "samples": n, "lm_trials": 4,
            "ms_per_step": qms}


def run_ours(args, rank, world, dist):
    import torch
    import paper_2602_05492_gb300 as bg
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = args.config
    sc, xy, target = make_inputs(rank, cfg)
    if args.samples:                     # profiling aid: leading part of the workload
        xy, target = xy[:args.samples].copy(), target[:args.samples].copy()
    n = xy.shape[0]
    jm = {"bf16": bg.BEM_JTJ_BF16, "3xtf32": bg.BEM_JTJ_3XTF32}[args.jtj]
    # config 4 states its FP64 near field: sample-panel distance < 2 panel lengths
    nf = 2.0 if cfg == 4 else 0.5
    m = bg.BEM(precision=bg.BEM_MIXED, device=local, jtj_mode=jm, near_factor=nf)
    xt = torch.from_numpy(xy).to(dev)
    tt = torch.from_numpy(target).to(dev)
    m.setup(sc.n_curves, sc.panels_per_curve, sc.closed, sc.theta_init, np.zeros(3))
    mean = m.sample_mean(tt)
    m.set_mean_color(mean)
    m.factor()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    lam = [1e-3]

    def step():
        r = m.lm_step(xt, tt, lam)
        lam[0] = r["lambda_next"]
        return r

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = m.launch_count()
    m.profile(True)
    clocks.start()
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()                              # evict L2 between steps
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    prof = m.profile_read()
    m.profile(False)
    launches = m.launch_count() - launches0
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)
    if dist is not None:
        tt_ = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(tt_, op=dist.ReduceOp.MAX)
        total_ms = float(tt_.item())
        dist.barrier()
    value = world * args.steps / (total_ms / 1e3)

    if rank != 0:
        return
    # ---- per-kernel live timing -> roofline of the dominant modelled kernel
    P, Nb, nc = sc.n_panels, 1024, 16 * sc.n_curves
    roofs = rooflines(prof, args.steps, n, P, Nb, nc, cfg)
    roof = roofs[0] if roofs else None
    kernels = {k: {"ms_per_launch": v[0] / max(v[1], 1), "launches": v[1],
                   "share": v[0] / total_ms} for k, v in sorted(prof.items())}

    # ---- sample x panel throughput, forward and adjoint, measured separately
    out = torch.empty((n, 3), dtype=torch.float32, device=dev)
    res = torch.empty((n, 3), dtype=torch.float32, device=dev)
    m.loss(xt, tt, res)
    reps = 3
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4 * reps)]
    fwd_ms = adj_ms = 0.0
    for r in range(reps):
        flush.zero_()
        ev[4 * r].record(stream)
        m.eval(xt, out)
        ev[4 * r + 1].record(stream)
        flush.zero_()
        ev[4 * r + 2].record(stream)
        g = m.vjp(xt, res)
        ev[4 * r + 3].record(stream)
    torch.cuda.synchronize()
    for r in range(reps):
        fwd_ms += ev[4 * r].elapsed_time(ev[4 * r + 1]) / reps
        adj_ms += ev[4 * r + 2].elapsed_time(ev[4 * r + 3]) / reps
    pairs = n * (P + Nb)
    pairs_per_s = 2 * pairs / ((fwd_ms + adj_ms) / 1e3)

    # ---- M_H = M_J / 4: H from every fourth sample (lm_step_split)
    xh = xt[::4].contiguous()
    m.set_params(sc.theta_init)
    lam_s = [1e-3]
    r_ = m.lm_step_split(xt, tt, xh, lam_s)
    lam_s[0] = r_["lambda_next"]
    torch.cuda.synchronize()
    e0s, e1s = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sms = 0.0
    for _ in range(2):
        flush.zero_()
        e0s.record(stream)
        r_ = m.lm_step_split(xt, tt, xh, lam_s)
        e1s.record(stream)
        torch.cuda.synchronize()
        lam_s[0] = r_["lambda_next"]
        sms += e0s.elapsed_time(e1s) / 2
    split_h = {"hessian_samples": int(xh.shape[0]), "gradient_samples": n, "ms_per_step": sms,
               "lm_iters_per_s": 1e3 / sms, "note": "H from every fourth sample, g by the adjoint"}
    del xh

    # ---- four subdomains (the quadrants, Sec. 4.2), 8 curves and the samples
    # of each quadrant, stepped together by one bem_batch_lm call (left out
    # with --samples, whose leading samples do not reach every quadrant)
    quads = []
    for qi in range(4 if not args.samples else 0):
        x0, y0 = 0.5 * (qi % 2), 0.5 * (qi // 2)
        poly = [(x0, y0), (x0 + 0.5, y0), (x0 + 0.5, y0 + 0.5), (x0, y0 + 0.5)]
        sel = ((xy[:, 0] >= x0) & (xy[:, 0] < x0 + 0.5) & (xy[:, 1] >= y0) & (xy[:, 1] < y0 + 0.5))
        th = sc.theta_init.reshape(sc.n_curves, 4, 8)[8 * qi:8 * qi + 8].copy()
        th[:, :, 0:2] = np.array([x0, y0]) + 0.05 + 0.4 * th[:, :, 0:2]
        mq = bg.BEM(precision=bg.BEM_MIXED, device=local, segs_per_side=128)
        tq = torch.from_numpy(np.ascontiguousarray(target[sel])).to(dev)
        qmean = np.minimum(target[sel], 1.0).mean(0)
        mq.setup(8, sc.panels_per_curve[:8], sc.closed[8 * qi:8 * qi + 8], th.reshape(-1), qmean)
        mq.set_boundary(poly, 128)
        mq.factor()
        quads.append((mq, torch.from_numpy(np.ascontiguousarray(xy[sel])).to(dev), tq))
    subdomains = run_quadrants(bg, quads, flush, stream, n) if quads else None
    for q in quads:
        q[0].close()
    del quads

    # ---- the paper's own parametrisation: 500 segment handles (Sec. 4.2) on
    # the same sample count, with the length and snapping regularisers on and
    # sparsity off (the paper's default, Sec. 4.4)
    ss = gen.make_segment_scene("seg500")
    xs = gen.make_samples(ss.W, ss.spp, ss.seed, dtype=np.float32)
    ts = gen.add_noise(gen.analytic_truth(xs, ss.seed), ss.noise, ss.seed).astype(np.float32)
    xst, tst = torch.from_numpy(xs).to(dev), torch.from_numpy(ts).to(dev)
    ms_ = bg.BEM(precision=bg.BEM_MIXED, device=local, jtj_mode=jm, near_factor=nf)
    ms_.setup_segments(ss.n_handles, ss.theta_init, np.minimum(ts, 1.0).mean(0))
    ms_.factor()
    ms_.set_regularizers(**SEG_REG)
    lseg = [1e-3]
    r_ = ms_.lm_step(xst, tst, lseg)
    lseg[0] = r_["lambda_next"]
    torch.cuda.synchronize()
    e0g, e1g = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gms = 0.0
    ms_.profile(True)
    for _ in range(3):
        flush.zero_()
        e0g.record(stream)
        r_ = ms_.lm_step(xst, tst, lseg)
        e1g.record(stream)
        torch.cuda.synchronize()
        lseg[0] = r_["lambda_next"]
        gms += e0g.elapsed_time(e1g) / 3
    gprof = ms_.profile_read()
    ms_.profile(False)
    segments = {"handles": ss.n_handles, "n_theta": 10 * ss.n_handles,
                "samples": int(xs.shape[0]), "regularisers": SEG_REG, "ms_per_step": gms,
                "lm_iters_per_s": 1e3 / gms,
                "kernel_share": {k: round(v[0] / (3 * gms), 4) for k, v in sorted(gprof.items())
                                 if v[0] / (3 * gms) >= 0.005},
                "workload": "500 random segment handles (length 0.025-0.1), 256^2 px x 16 spp, "
                            "lognormal noise with 1% fireflies"}
    ms_.close()
    del xst, tst

    # ---- output rendering: the colour field on a 1024 x 1024 pixel grid
    img = torch.empty((1024, 1024, 3), dtype=torch.float32, device=dev)
    m.render(1024, 1024, img)
    e0r, e1r = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0r.record(stream)
    for _ in range(3):
        m.render(1024, 1024, img)
    e1r.record(stream)
    torch.cuda.synchronize()
    rms = e0r.elapsed_time(e1r) / 3
    render = {"pixels": 1024 * 1024, "ms": rms, "mpix_per_s": 1024 * 1024 / rms / 1e3}
    del img

    # ---- FP64 GPU path: one LM iteration (after one warm-up iteration); at
    # config 4 its cost a + b S is fitted from steps on two sample subsets
    fp64 = None
    accuracy = None
    if args.fp64_steps > 0:
        n64 = n if (cfg != 4 or args.fp64_samples <= 0) else min(n, args.fp64_samples)
        m64 = bg.BEM(precision=bg.BEM_FP64, device=local)
        x64, t64 = xt[:n64].double(), tt[:n64].double()
        m64.setup(sc.n_curves, sc.panels_per_curve, sc.closed, sc.theta_init, mean)
        m64.factor()
        u64 = m64.eval(x64)
        m.set_params(sc.theta_init)
        u32 = m.eval(xt[:n64]).double()
        rmse = float(torch.sqrt(torch.mean((u32 - u64) ** 2)).item())
        r64 = torch.empty((n64, 3), dtype=torch.float64, device=dev)
        m64.loss(x64, t64, r64)
        g64 = m64.vjp(x64, r64)
        r32 = torch.empty((n64, 3), dtype=torch.float32, device=dev)
        m.loss(xt[:n64], tt[:n64], r32)
        g32 = m.vjp(xt[:n64], r32)
        gerr = float((torch.linalg.norm(g32 - g64) / torch.linalg.norm(g64)).item())
        del u64, u32, r64, r32
        m64.lm_step(x64, t64, [1e-3])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        def t64_step(k):
            tot = 0.0
            for _ in range(args.fp64_steps):
                m64.set_params(sc.theta_init)
                flush.zero_()
                e0.record(stream)
                m64.lm_step(x64[:k], t64[:k], [1e-3])
                e1.record(stream)
                torch.cuda.synchronize()
                tot += e0.elapsed_time(e1) / args.fp64_steps
            return tot

        if n64 == n:
            t64_ms = t64_step(n64)
            timed = f"{args.fp64_steps} full FP64 LM iteration(s) after one warm-up"
        else:
            th, tf = t64_step(n64 // 2), t64_step(n64)
            b = (tf - th) / (n64 - n64 // 2)
            t64_ms = tf + b * (n - n64)
            timed = (f"FP64 LM iterations on {n64 // 2} and {n64} of {n} samples "
                     f"({th:.0f} ms, {tf:.0f} ms), extrapolated linearly in samples")
        fp64 = {"lm_iters_per_s": 1e3 / t64_ms, "ms_per_iter": t64_ms,
                "mixed_over_fp64": (value / world) / (1e3 / t64_ms), "timed": timed}
        accuracy = {"colour_rmse_mixed_vs_fp64_gpu": rmse, "grad_rel_err_mixed_vs_fp64_gpu": gerr,
                    "at": f"theta_init, {'all' if n64 == n else n64} samples"}
        m64.close()

    # ---- end to end through the public API with host buffers
    xy_h = torch.from_numpy(xy).pin_memory()
    t_h = torch.from_numpy(target).pin_memory()
    xe = torch.empty_like(xt)
    te = torch.empty_like(tt)
    m.set_params(sc.theta_init)
    lam_e = [1e-3]
    torch.cuda.synchronize()
    e_steps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(e_steps):
        xe.copy_(xy_h, non_blocking=True)
        te.copy_(t_h, non_blocking=True)
        r = m.lm_step(xe, te, lam_e)          # returns losses to the host
        lam_e[0] = r["lambda_next"]
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e_steps
    e2e = {"value": 1.0 / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(xy.nbytes + target.nbytes),
           "d2h_bytes_per_step": 8 * 3}

    cpu = None
    if world == 1 and not args.no_cpu_baseline and cfg == CFG:
        cpu = cpu_baseline(sc, xy, target, n_sub=args.cpu_samples)
        cpu.pop("seconds_per_sample_step", None)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": workload_desc(sc, cfg), "near_factor": nf,
                       "precision": "mixed (f32 pairs, f64 near field and refined solves)", "jtj": args.jtj, "lm_trials_per_step": 1,
                       "l2": "flushed between timed steps (256 MiB write)",
                       "wall_s_timed_region": t_wall},
            "pairs_per_s": {"value": pairs_per_s, "unit": "sample x panel evals/s (fwd+adjoint)",
                            "fwd_ms": fwd_ms, "adj_ms": adj_ms, "pairs_per_pass": pairs},
            "fp64_gpu": fp64, "accuracy": accuracy, "render_1024x1024": render,
            "lm_step_split_hessian": split_h, "subdomains_batched": subdomains,
            "segments_500": segments,
            "kernels": kernels,
            "roofline": roof, "rooflines_other": roofs[1:], "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": int(launches)}
    print(json.dumps(line), flush=True)


def run_batch(args, rank, world):
    """Config 5: uneven scenes with 4 damping trials each, stepped by one
    bem_batch_lm call per LM iteration, against stepping the same scenes one
    at a time with lm_step (same trials).  Unit: scene LM iterations/s."""
    import torch
    import paper_2602_05492_gb300 as bg
    if rank != 0:
        return
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    lams = [1e-3, 1e-2, 1e-1, 1.0]
    scenes = gen.batch_scenes(args.scenes)
    data = []
    for k, sc in enumerate(scenes):
        xy = gen.make_samples(sc.W, sc.spp, sc.seed, dtype=np.float32)
        tgt = gen.add_noise(gen.analytic_truth(xy, sc.seed), sc.noise, sc.seed).astype(np.float32)
        data.append((torch.from_numpy(xy).to(dev), torch.from_numpy(tgt).to(dev),
                     np.minimum(tgt, 1.0).mean(0).astype(np.float64)))

    def contexts():
        ms = []
        for sc, (x, t, mean) in zip(scenes, data):
            m = bg.BEM(precision=bg.BEM_MIXED)
            m.setup(sc.n_curves, sc.panels_per_curve, sc.closed, sc.theta_init, mean)
            m.factor()
            ms.append(m)
        return ms

    xs = [d[0] for d in data]
    ts = [d[1] for d in data]
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    # batched
    mb = contexts()
    b = bg.BEMBatch(mb)
    for _ in range(max(args.warmup, 0)):
        b.lm_step(xs, ts, lams)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    tb = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0.record(stream)
        b.lm_step(xs, ts, lams)
        e1.record(stream)
        torch.cuda.synchronize()
        tb += e0.elapsed_time(e1)
    clk = clocks.stop()
    shape = b.tile_shape()
    b.close()
    for m in mb:
        m.close()
    # one scene at a time
    ms = contexts()
    for _ in range(max(args.warmup, 0)):
        for m, x, t in zip(ms, xs, ts):
            m.lm_step(x, t, lams)
    torch.cuda.synchronize()
    tsq = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0.record(stream)
        for m, x, t in zip(ms, xs, ts):
            m.lm_step(x, t, lams)
        e1.record(stream)
        torch.cuda.synchronize()
        tsq += e0.elapsed_time(e1)
    for m in ms:
        m.close()
    S = len(scenes)
    nsamp = int(sum(x.shape[0] for x in xs))
    npan = int(sum(sc.n_panels for sc in scenes))
    value = S * args.steps / (tb / 1e3)
    seq = S * args.steps / (tsq / 1e3)
    line = {"metric": "scene LM iterations/s, 4 damping trials per scene (batched)",
            "value": value, "unit": "scene LM iter/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tb / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"cfg5: {S} scenes, panels log-uniform in [256, 4096] "
                                   f"(64 per curve, {npan} in all), 128^2..512^2 px at "
                                   f"4..32 spp ({nsamp} samples in all), lambda in {lams}",
                       "l2": "flushed between timed steps (256 MiB write)",
                       "tile_shape": {"points_per_tile": shape[0], "ctas_per_sm": shape[1]}},
            "one_at_a_time": {"value": seq, "unit": "scene LM iter/s",
                              "ms_per_step": tsq / args.steps},
            "batched_over_one_at_a_time": value / seq, "clocks": clk}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--cpu-samples", type=int, default=4096)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--jtj", default="bf16", choices=["bf16", "3xtf32"],
                    help="tensor-core scheme of the J^T J contraction")
    ap.add_argument("--config", type=int, default=CFG, choices=[2, 4, 5],
                    help="2: the metric's configuration (default); 4: 67M samples, 8,192 "
                         "panels; 5: batched uneven scenes against one at a time")
    ap.add_argument("--scenes", type=int, default=64, help="config 5: number of scenes")
    ap.add_argument("--fp64-samples", type=int, default=1 << 20,
                    help="config 4: samples of the FP64 GPU comparison (0 = all)")
    ap.add_argument("--samples", type=int, default=0,
                    help="profiling aid: time only the first N samples of the workload")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        backend = "nccl" if (args.impl == "ours" and torch.cuda.is_available()) else "gloo"
        tdist.init_process_group(backend=backend)
        dist = tdist
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.config == 5:
        run_batch(args, rank, world)
    else:
        run_ours(args, rank, world, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
