#!/usr/bin/env python
"""Throughput of the differential-BEM Levenberg-Marquardt hot path on GB300.

One step = one LM iteration of the mixed-precision path (panelize, boundary
right-hand side and solve, residual + loss at every sample, gradient,
Gauss-Newton matrix, damped KKT solve, trial evaluation) on the workload the
throughput target is stated on: 128 cubic Bezier curves x 64 panels (8,192
panels), 1024 x 1024 px x 64 spp (67,108,864 samples), FP64 near field within
2 panel lengths.  Prints one JSON line.  `--impl reference` times the FP64
CPU oracle on the same workload instead (rank 0 only).

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torch.distributed.run, one independent replica per GPU (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gen  # noqa: E402

METRIC = ("LM iters/s & sample×panel evals/s (fwd+adjoint), mixed vs FP64 GPU at "
          "≤1e-4 RMSE")
UNIT = "LM iter/s"
CFG = 4            # 1024^2 px x 64 spp, 8,192 panels: the configuration of the throughput target
L2_FLUSH_BYTES = 256 << 20
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")


# regularisers of the 500-handle segment workload: length above twice the
# initial 1/20 of the width, snapping within 1% of the width, no sparsity
SEG_REG = dict(len_weight=1.0, len_max=0.1, snap_weight=1.0, snap_radius=0.01, snap_alpha=0.5)


def near_factor(cfg):
    # config 4 states its FP64 near field: sample-panel distance < 2 panel lengths
    return 2.0 if cfg == 4 else 0.5


def workload_desc(sc, cfg=CFG):
    noise = ("lognormal noise with 1% fireflies" if sc.noise.get("noise") == "lognormal"
             else "Gaussian noise")
    return (f"cfg{cfg}: {sc.n_curves} cubic Bezier curves x {int(sc.panels_per_curve[0])} panels "
            f"({sc.n_panels} panels), {sc.W}x{sc.W} px x {sc.spp} spp ({sc.n_samples} samples), "
            f"1024 boundary segments, {noise}")


def bench_config(sc, cfg, jtj="bf16"):
    """The `config` object of both arms' JSON lines (identical for the same workload)."""
    return {"workload": workload_desc(sc, cfg), "near_factor": near_factor(cfg),
            "precision": "mixed (f32 pairs, f64 near field and refined solves)", "jtj": jtj,
            "lm_trials_per_step": 1,
            "l2": "flushed between timed steps (256 MiB write); inputs larger than L2"}


def make_inputs(rank: int, cfg: int = CFG):
    sc = gen.make_scene(cfg)
    seed = sc.seed + 7919 * rank        # independent sample set per replica
    xy = gen.make_samples(sc.W, sc.spp, seed, dtype=np.float32)
    truth = gen.analytic_truth(xy, sc.seed)
    target = gen.add_noise(truth, sc.noise, seed).astype(np.float32)
    return sc, xy, target


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


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
# algorithmic work per unit, counted from the source formulas.  FP32 flops:
# add/mul = 1, FMA = 2 (compares, selects, min/max not counted).  Each
# transcendental of the method (log, atan2, sqrt or rsqrt, rcp) is one
# special-function op, whatever its implementation costs (atan2 has no
# hardware instruction and runs as a polynomial).

# handle pair of the evaluation: rounded frame 9, h^2 1, h'^2, h', t1 t2, q1, q2 7,
# atan2 arguments 2, t2 log q2 - t1 log q1 3, Sh 4, Dh 2, 3-channel
# accumulation 12; special ops as the method states them: 2 logs, atan2, the
# square root h' and the reciprocal in h/h' (the kernels form h' and 1/h'
# from one reciprocal square root)
FWD_HANDLE = (9 + 1 + 7 + 2 + 3 + 4 + 2 + 12, 5)        # (flops, special ops)
# boundary pair: vertex offset 2, cross 3, dot 3, 3-channel accumulation 6 (+ atan2)
FWD_BOUND = (2 + 3 + 3 + 6, 1)
# F-row pair: frame 9, h^2 1, values and frame partials of both layers 31 (+
# sqrt and reciprocal of h', atan2, 2 logs, 2 rcp), chain rule to both
# endpoints for Dl and S 42, jump columns 16, 3 channels x 2 coordinates x
# (combine 7 + four Bernstein accumulations 8) 90
FROWS_PAIR = (9 + 1 + 31 + 42 + 16 + 90, 7)


def step_work(name, n, P, Nb, nc):
    """((flops, special ops) of one LM step's launches of `name`, bound) for
    the modelled kernels; for k_field the work of one launch (every launch
    evaluates all samples)."""
    if name == "k_field":            # one evaluation of every sample (per launch)
        return (n * (P * FWD_HANDLE[0] + Nb * FWD_BOUND[0]),
                n * (P * FWD_HANDLE[1] + Nb * FWD_BOUND[1])), "alu_per_launch"
    if name == "k_field_bnd":        # boundary term of every sample, in chunks
        return (float(n) * Nb * FWD_BOUND[0], float(n) * Nb * FWD_BOUND[1]), "alu"
    if name == "k_frows":            # all samples, plus the 3 Nb boundary Gauss points
        u = float(n + 3 * Nb) * P
        return (u * FROWS_PAIR[0], u * FROWS_PAIR[1]), "alu"
    # J rows: the position columns of each channel and the jump columns once
    # (they are the same in every channel): 3 (nc/2) + nc/2 = 2 nc rows for
    # Bezier curves (nc = 16 C: 8 C position, 8 C jump columns per channel)
    rows, jump = 3 * (nc // 2) + nc // 2, nc // 2
    if name == "tc_jrows":           # J^T = M^T Phi^T (+ F^T) over those rows
        return 2.0 * rows * Nb * n, "tensor"
    if name == "tc_syrk":            # 3 symmetric rank-n updates of order nc, the
        # jump-jump block (the same in every channel) once
        return (3.0 * nc * (nc + 1) - 2.0 * jump * (jump + 1)) * n, "tensor"
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


def measure_pipes(m):
    """Measured pipe peaks of this GPU (bem_pipe_peak) with the clocks seen
    while the probes ran: FP32 FMA (TFLOP/s, 2 flops per FMA) and the MUFU
    rate of the slowest of lg2 / rcp / rsqrt (special ops per second)."""
    clk = ClockSampler(m.device)
    clk.start()
    fma = m.pipe_peak(0, 20) * 2.0
    mufu = {nm: m.pipe_peak(k, 20) for k, nm in ((1, "lg2"), (2, "rcp"), (3, "rsqrt"))}
    c = clk.stop()
    return {"fp32_tflops": fma / 1e12, "mufu_gops": {k: v / 1e9 for k, v in mufu.items()},
            "sfu_gops": min(mufu.values()) / 1e9, "clocks": c,
            "how": "bem_pipe_peak: 4 CTAs x 256 threads per SM, 8 independent chains per "
                   "thread, median of 20 launches of about 30 ms"}


def rooflines(prof, steps, n, P, Nb, nc, pipes, cfg=CFG, jtj="bf16"):
    """One entry per modelled kernel.  ALU kernels: the FP32/SFU roofline of
    two pipes that run side by side, t_roof = max(flops / FP32 peak, special
    ops / SFU peak), peaks measured by bem_pipe_peak; `bound` names the
    binding pipe and `frac` = t_roof / measured time.  `fp32_only` gives the
    FP32-peak fraction with each special op counted as one flop.  Tensor
    kernels: flops against the measured sustained bf16 rate; the compensated
    schemes count their three products per block, 3xtf32 against the bf16
    rate times the nominal tf32/bf16 ratio (1.1 / 2.25 PFLOP/s)."""
    peaks, src = read_peaks()
    out = []
    fp32 = pipes["fp32_tflops"] * 1e12
    sfu = pipes["sfu_gops"] * 1e9
    for name, (ms, cnt) in prof.items():
        work, bound = step_work(name, n, P, Nb, nc)
        if work is None or not cnt:
            continue
        t = ms / cnt / 1e3                      # seconds per launch
        if bound in ("alu", "alu_per_launch"):
            F, T = work if bound == "alu_per_launch" else (w * steps / cnt for w in work)
            t_fp, t_sf = F / fp32, T / sfu
            if t_sf > t_fp:
                rec = {"bound": "sfu", "achieved": T / t / 1e9, "peak": pipes["sfu_gops"],
                       "unit": "Gop/s (special functions)"}
            else:
                rec = {"bound": "fp32", "achieved": F / t / 1e12, "peak": pipes["fp32_tflops"],
                       "unit": "TFLOP/s"}
            rec.update({"kernel": name, "frac": max(t_fp, t_sf) / t,
                        "traffic": kernel_traffic(name, cfg), "flops_per_launch": F,
                        "special_ops_per_launch": T,
                        "fp32_pipe_frac": t_fp / t, "sfu_pipe_frac": t_sf / t,
                        "fp32_only": {"achieved": (F + T) / t / 1e12, "peak": pipes["fp32_tflops"],
                                      "frac": (F + T) / t / fp32},
                        "peak_source": "measured by bem_pipe_peak in this run"})
        else:
            products = 1 if jtj == "bf16" else 3
            per_launch = work * steps / cnt * products
            ach = per_launch / t / 1e12
            peak = peaks["bf16_tflops_sustained"]
            psrc = f"bf16 dense, sustained ({src}, MEASURED_PEAKS.json)"
            if jtj == "3xtf32":
                peak *= 1.1 / 2.25
                psrc = f"tf32: bf16 dense sustained ({src}) x nominal tf32/bf16 1.1/2.25"
            rec = {"bound": "tensor", "kernel": name, "achieved": ach, "peak": peak,
                   "unit": "TFLOP/s", "frac": ach / peak,
                   "traffic": kernel_traffic(name, cfg) if jtj == "bf16" else None,
                   "flops_per_launch": per_launch, "products_per_block": products,
                   "peak_source": psrc}
        rec["share_ms"] = ms
        out.append(rec)
    out.sort(key=lambda r: -r.pop("share_ms"))
    return out


# ---------------------------------------------------------------------------
# the oracle, timed as it stands on the host cores

def _oracle_fixed(o, th, x0, t0):
    """The part of the oracle's LM iteration (Oracle.lm_step) that does not
    depend on the number of samples: boundary values and boundary Jacobian
    (the stacked right-hand sides) at theta, the damped KKT solve of order
    n_theta, and the trial's boundary values.  Returns its seconds and the
    state the per-sample part needs."""
    import oracle
    c0 = time.perf_counter()
    ub = o.boundary_values(th)
    Mb = o.boundary_jac(th)
    t_bnd = time.perf_counter() - c0
    # H and g of a small sample set stand in for the full sums (same size;
    # their cost belongs to the per-sample part and is not counted here)
    r = o.eval(th, x0, ub) - np.minimum(t0, 1.0)
    J = o.jac(th, x0, Mb)
    g = np.einsum("sct,sc->t", J, r) / x0.shape[0]
    Jf = J.reshape(-1, o.geo.n_theta)
    H = Jf.T @ Jf / x0.shape[0]
    c1 = time.perf_counter()
    delta = o.solve_step(th, H, g, 1e-3)
    th1 = oracle.project_compat(o.geo, th + delta)
    ub1 = o.boundary_values(th1)
    t_solve = time.perf_counter() - c1
    return t_bnd + t_solve, dict(th=th, ub=ub, Mb=Mb, th1=th1, ub1=ub1)


def _oracle_per_sample(o, st, x, t):
    """The oracle's per-sample work of one LM iteration on the points x:
    colour and residual at theta, J rows (handle part + boundary part), their
    contributions to g and H, and the colour at the trial theta (its loss).
    Returns seconds."""
    c0 = time.perf_counter()
    nt = o.geo.n_theta
    r = o.eval(st["th"], x, st["ub"]) - np.minimum(t, 1.0)
    J = o.jac(st["th"], x, st["Mb"])
    g = np.einsum("sct,sc->t", J, r)
    Jf = J.reshape(-1, nt)
    H = Jf.T @ Jf
    u1 = o.eval(st["th1"], x, st["ub1"])
    L1 = 0.5 * float(np.sum((u1 - np.minimum(t, 1.0)) ** 2))
    assert np.isfinite(L1) and np.isfinite(g).all() and np.isfinite(H).all()
    return time.perf_counter() - c0


def oracle_rate(sc, xy, target, steps: int, warmup: int, n_step: int = 64, one_thread=True) -> dict:
    """The oracle's LM iteration timed in its two parts on the host cores:
    the fixed part once (after the warm-up of the per-sample part), the
    per-sample part on `steps` seeded subsets of n_step samples after
    `warmup` untimed ones.  One iteration on the S samples of the workload
    costs a + b S (extrapolated).  With one_thread, the per-sample part is
    also timed in a child process limited to one thread."""
    import oracle
    mean = np.minimum(target, 1.0).mean(0)
    o = oracle.Oracle.from_scene(sc, mean_color=mean)
    rng = np.random.default_rng(0)
    S = xy.shape[0]

    def subset():
        idx = np.sort(rng.choice(S, n_step, replace=False))
        return xy[idx].astype(np.float64), target[idx].astype(np.float64)

    x0, t0 = subset()
    a, st = _oracle_fixed(o, sc.theta_init, x0, t0)
    for _ in range(max(warmup, 0)):
        _oracle_per_sample(o, st, *subset())
    per = [_oracle_per_sample(o, st, *subset()) / n_step for _ in range(max(steps, 1))]
    b = statistics.mean(per)
    per_iter = a + b * S
    out = {"value": 1.0 / per_iter, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "cpu_model": cpu_model(),
           "sample": (f"FP64 oracle LM iteration in two parts: the fixed part (boundary values, "
                      f"boundary Jacobian, damped solve of order {o.geo.n_theta}, trial boundary "
                      f"values) once, {a:.1f} s; the per-sample part (colour, J rows, g and H "
                      f"sums, trial colour) on {max(steps, 1)} seeded subsets of {n_step} of "
                      f"the {S} samples, b = {b * 1e3:.3f} ms/sample; one iteration a + b S "
                      f"= {per_iter:.4g} s (extrapolated)"),
           "fixed_s": a, "per_sample_s": b, "ms_per_step": per_iter * 1e3}
    if one_thread:
        out["one_thread"] = oracle_one_thread(o, st, sc, xy, target, S)
    return out


def oracle_one_thread(o, st, sc, xy, target, S, n_step=16):
    """Per-sample part of the oracle's iteration in a child process with one
    thread (OpenMP and BLAS); the fixed part is not repeated there (at
    millions of samples it is a negligible share of a + b S)."""
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "state.npz")
        rng = np.random.default_rng(1)
        idx = np.sort(rng.choice(xy.shape[0], 3 * n_step, replace=False))
        np.savez(path, x=xy[idx].astype(np.float64), t=target[idx].astype(np.float64),
                 mean=o.mean, **st)
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
                   MKL_NUM_THREADS="1")
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-probe", path,
                            "--config", str(_cfg_of(sc))], env=env, capture_output=True,
                           text=True, timeout=600)
    if r.returncode != 0:
        return {"error": r.stderr.strip().splitlines()[-1] if r.stderr.strip() else "failed"}
    b1 = json.loads(r.stdout.strip().splitlines()[-1])["per_sample_s"]
    return {"cores": 1, "per_sample_s": b1, "iters_per_s": 1.0 / (b1 * S),
            "sample": f"per-sample part on {2 * n_step} samples after {n_step} untimed, one "
                      f"thread; iterations/s = 1 / (b S), the fixed part left out"}


def _cfg_of(sc):
    from gen import scenes
    return next(k for k, v in scenes.CONFIGS.items() if v["seed"] == sc.seed)


def oracle_probe(path, cfg):
    """Child process of oracle_one_thread: the per-sample part with the
    threads the environment allows."""
    import oracle
    z = np.load(path)
    sc = gen.make_scene(cfg)
    o = oracle.Oracle.from_scene(sc, mean_color=z["mean"])
    st = {k: z[k] for k in ("th", "ub", "Mb", "th1", "ub1")}
    x, t = z["x"], z["t"]
    n = x.shape[0] // 3
    _oracle_per_sample(o, st, x[:n], t[:n])
    dt = _oracle_per_sample(o, st, x[n:], t[n:])
    print(json.dumps({"per_sample_s": dt / (x.shape[0] - n), "threads": oracle.num_threads()}))


def run_reference(args, rank, world):
    if rank != 0:
        return
    sc, xy, target = make_inputs(0, args.config)
    r = oracle_rate(sc, xy, target, steps=args.steps, warmup=args.warmup, one_thread=False)
    v = r["value"]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": bench_config(sc, args.config, args.jtj),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                             "cpu_model": r["cpu_model"], "sample": r["sample"]},
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


def _timed(step, K, flush, stream):
    """K steps, each after an L2 flush, bracketed by CUDA events on the
    launching stream; per-step milliseconds."""
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    for k in range(K):
        flush.zero_()                              # evict L2 between steps
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize()
    return [s.elapsed_time(e) for s, e in zip(starts, ends)]


def config2_extras(bg, dev, flush, stream, local, jm, rank):
    """Secondary measurements on the 1,048,576-sample / 2,048-panel workload:
    a 50-iteration fit from theta_init, its full LM step, H from every fourth
    sample, four quadrant subdomains, the paper's 500 segment handles, and a
    1024 x 1024 rendering."""
    import torch
    sc2, xy2, tg2 = make_inputs(rank, 2)
    n2 = xy2.shape[0]
    x2, t2 = torch.from_numpy(xy2).to(dev), torch.from_numpy(tg2).to(dev)
    m2 = bg.BEM(precision=bg.BEM_MIXED, device=local, jtj_mode=jm, near_factor=near_factor(2))
    m2.setup(sc2.n_curves, sc2.panels_per_curve, sc2.closed, sc2.theta_init, np.zeros(3))
    m2.set_mean_color(m2.sample_mean(t2))
    m2.factor()
    out = {"workload": workload_desc(sc2, 2)}

    # the fit the workload is specified with: 50 LM iterations from
    # theta_init, each damping from the previous proposal (losses read back
    # by every iteration; no flush between them)
    loss0 = loss_end = None
    acc = 0
    lam_f = 1e-3
    e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e_a.record(stream)
    for k in range(50):
        r = m2.lm_step(x2, t2, [lam_f])
        loss0 = r["loss_before"] if k == 0 else loss0
        acc += int(r["accepted"])
        lam_f = r["lambda_next"]
        loss_end = r["loss_after"] if r["accepted"] else r["loss_before"]
    e_b.record(stream)
    torch.cuda.synchronize()
    out["fit_50"] = {"iterations": 50, "accepted": acc, "loss_init": loss0, "loss_end": loss_end,
                     "ms": e_a.elapsed_time(e_b)}
    m2.set_params(sc2.theta_init)
    lam = [1e-3]

    def step2():
        r = m2.lm_step(x2, t2, lam)
        lam[0] = r["lambda_next"]

    for _ in range(3):
        step2()
    torch.cuda.synchronize()
    ms = _timed(step2, 10, flush, stream)
    out["lm_step"] = {"ms_per_step": sum(ms) / len(ms), "lm_iters_per_s": 1e3 * len(ms) / sum(ms)}

    # the same step with the Gauss-Newton matrix in the two compensated schemes
    for name, mode in (("lm_step_bf16x3", bg.BEM_JTJ_BF16X3), ("lm_step_3xtf32", bg.BEM_JTJ_3XTF32)):
        mj = bg.BEM(precision=bg.BEM_MIXED, device=local, jtj_mode=mode, near_factor=near_factor(2))
        mj.setup(sc2.n_curves, sc2.panels_per_curve, sc2.closed, sc2.theta_init, np.zeros(3))
        mj.set_mean_color(mj.sample_mean(t2))
        mj.factor()
        lam_j = [1e-3]

        def step_j():
            r = mj.lm_step(x2, t2, lam_j)
            lam_j[0] = r["lambda_next"]

        for _ in range(2):
            step_j()
        torch.cuda.synchronize()
        ms = _timed(step_j, 5, flush, stream)
        out[name] = {"ms_per_step": sum(ms) / len(ms), "lm_iters_per_s": 1e3 * len(ms) / sum(ms)}
        mj.close()

    # M_H = M_J / 4: H from every fourth sample (lm_step_split)
    xh = x2[::4].contiguous()
    m2.set_params(sc2.theta_init)
    lam_s = [1e-3]

    def split_step():
        r = m2.lm_step_split(x2, t2, xh, lam_s)
        lam_s[0] = r["lambda_next"]

    split_step()
    torch.cuda.synchronize()
    ms = _timed(split_step, 2, flush, stream)
    out["lm_step_split_hessian"] = {
        "hessian_samples": int(xh.shape[0]), "gradient_samples": n2,
        "ms_per_step": sum(ms) / 2, "lm_iters_per_s": 2e3 / sum(ms),
        "note": "H from every fourth sample, g by the adjoint"}
    del xh

    # four subdomains (the quadrants, Sec. 4.2), 8 curves and the samples of
    # each quadrant, stepped together by one bem_batch_lm call
    quads = []
    for qi in range(4):
        x0, y0 = 0.5 * (qi % 2), 0.5 * (qi // 2)
        poly = [(x0, y0), (x0 + 0.5, y0), (x0 + 0.5, y0 + 0.5), (x0, y0 + 0.5)]
        sel = ((xy2[:, 0] >= x0) & (xy2[:, 0] < x0 + 0.5) & (xy2[:, 1] >= y0) &
               (xy2[:, 1] < y0 + 0.5))
        th = sc2.theta_init.reshape(sc2.n_curves, 4, 8)[8 * qi:8 * qi + 8].copy()
        th[:, :, 0:2] = np.array([x0, y0]) + 0.05 + 0.4 * th[:, :, 0:2]
        mq = bg.BEM(precision=bg.BEM_MIXED, device=local, segs_per_side=128)
        tq = torch.from_numpy(np.ascontiguousarray(tg2[sel])).to(dev)
        qmean = np.minimum(tg2[sel], 1.0).mean(0)
        mq.setup(8, sc2.panels_per_curve[:8], sc2.closed[8 * qi:8 * qi + 8], th.reshape(-1), qmean)
        mq.set_boundary(poly, 128)
        mq.factor()
        quads.append((mq, torch.from_numpy(np.ascontiguousarray(xy2[sel])).to(dev), tq))
    out["subdomains_batched"] = run_quadrants(bg, quads, flush, stream, n2)
    for q in quads:
        q[0].close()
    del quads

    # output rendering: the colour field on a 1024 x 1024 pixel grid
    img = torch.empty((1024, 1024, 3), dtype=torch.float32, device=dev)
    m2.render(1024, 1024, img)
    e0r, e1r = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0r.record(stream)
    for _ in range(3):
        m2.render(1024, 1024, img)
    e1r.record(stream)
    torch.cuda.synchronize()
    rms = e0r.elapsed_time(e1r) / 3
    out["render_1024x1024"] = {"pixels": 1024 * 1024, "ms": rms, "mpix_per_s": 1024 * 1024 / rms / 1e3}
    del img
    m2.close()
    del x2, t2

    # the paper's own parametrisation: 500 segment handles (Sec. 4.2) on the
    # same sample count, with the length and snapping regularisers on and
    # sparsity off (the paper's default, Sec. 4.4)
    ss = gen.make_segment_scene("seg500")
    xs = gen.make_samples(ss.W, ss.spp, ss.seed, dtype=np.float32)
    ts = gen.add_noise(gen.analytic_truth(xs, ss.seed), ss.noise, ss.seed).astype(np.float32)
    xst, tst = torch.from_numpy(xs).to(dev), torch.from_numpy(ts).to(dev)
    ms_ = bg.BEM(precision=bg.BEM_MIXED, device=local, jtj_mode=jm, near_factor=near_factor(2))
    ms_.setup_segments(ss.n_handles, ss.theta_init, np.minimum(ts, 1.0).mean(0))
    ms_.factor()
    ms_.set_regularizers(**SEG_REG)
    lseg = [1e-3]

    def seg_step():
        r = ms_.lm_step(xst, tst, lseg)
        lseg[0] = r["lambda_next"]

    seg_step()
    torch.cuda.synchronize()
    ms_.profile(True)
    ms = _timed(seg_step, 3, flush, stream)
    gprof = ms_.profile_read()
    ms_.profile(False)
    gms = sum(ms) / 3
    out["segments_500"] = {
        "handles": ss.n_handles, "n_theta": 10 * ss.n_handles, "samples": int(xs.shape[0]),
        "regularisers": SEG_REG, "ms_per_step": gms, "lm_iters_per_s": 1e3 / gms,
        "kernel_share": {k: round(v[0] / (3 * gms), 4) for k, v in sorted(gprof.items())
                         if v[0] / (3 * gms) >= 0.005},
        "workload": "500 random segment handles (length 0.025-0.1), 256^2 px x 16 spp, "
                    "lognormal noise with 1% fireflies"}
    ms_.close()
    return out


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
    jm = {"bf16": bg.BEM_JTJ_BF16, "bf16x3": bg.BEM_JTJ_BF16X3, "3xtf32": bg.BEM_JTJ_3XTF32}[args.jtj]
    nf = near_factor(cfg)
    m = bg.BEM(precision=bg.BEM_MIXED, device=local, jtj_mode=jm, near_factor=nf)
    xt = torch.from_numpy(xy).to(dev)
    tt = torch.from_numpy(target).to(dev)
    m.setup(sc.n_curves, sc.panels_per_curve, sc.closed, sc.theta_init, np.zeros(3))
    mean = m.sample_mean(tt)
    m.set_mean_color(mean)
    m.factor()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    pipes = measure_pipes(m)
    lam = [1e-3]

    def step():
        r = m.lm_step(xt, tt, lam)
        lam[0] = r["lambda_next"]
        return r

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = m.launch_count()
    m.profile(True)
    clocks.start()
    t_wall0 = time.perf_counter()
    step_ms = _timed(step, args.steps, flush, stream)
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    prof = m.profile_read()
    launches = m.launch_count() - launches0
    total_ms = sum(step_ms)
    if dist is not None:
        tt_ = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(tt_, op=dist.ReduceOp.MAX)
        total_ms = float(tt_.item())
        dist.barrier()
    value = world * args.steps / (total_ms / 1e3)

    # ---- end to end through the public API with host buffers: the same
    # start (theta_init, lambda 1e-3), warm-up, steps, L2 flush and event
    # profiler as the device-timed run; every step is one lm_step_host call
    # on pinned host memory, which copies the inputs in (chunk by chunk,
    # alongside the Gauss-Newton pass) and reads the losses back
    xy_h = torch.from_numpy(xy).pin_memory()
    t_h = torch.from_numpy(target).pin_memory()
    m.set_params(sc.theta_init)
    lam_e = [1e-3]

    def e2e_step():
        r = m.lm_step_host(xy_h, t_h, lam_e)
        lam_e[0] = r["lambda_next"]

    for _ in range(max(args.warmup, 0)):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        c0 = time.perf_counter()
        e2e_step()
        torch.cuda.synchronize()
        e2e_s += time.perf_counter() - c0
    m.profile(False)
    e2e = {"value": world * args.steps / e2e_s if dist is None else args.steps / e2e_s * world,
           "unit": UNIT, "h2d_bytes_per_step": int(xy.nbytes + target.nbytes),
           "d2h_bytes_per_step": 8 * 3, "steps": args.steps, "warmup": args.warmup,
           "timer": "host clock around each lm_step_host call (its copies from pinned host "
                    "memory, the step, its host read-back)"}
    del xy_h, t_h

    if rank != 0:
        return
    # ---- per-kernel live timing -> roofline of the dominant modelled kernel
    P, Nb, nc = sc.n_panels, 1024, 16 * sc.n_curves
    roofs = rooflines(prof, args.steps, n, P, Nb, nc, pipes, cfg, args.jtj)
    roof = roofs[0] if roofs else None
    kernels = {k: {"ms_per_launch": v[0] / max(v[1], 1), "launches": v[1],
                   "share": v[0] / total_ms} for k, v in sorted(prof.items())}

    # ---- sample x panel throughput, forward and adjoint, measured separately
    m.set_params(sc.theta_init)
    out = torch.empty((n, 3), dtype=torch.float32, device=dev)
    res = torch.empty((n, 3), dtype=torch.float32, device=dev)
    m.loss(xt, tt, res)
    reps = 1 if n > (1 << 22) else 3
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4 * reps)]
    fwd_ms = adj_ms = 0.0
    for r in range(reps):
        flush.zero_()
        ev[4 * r].record(stream)
        m.eval(xt, out)
        ev[4 * r + 1].record(stream)
        flush.zero_()
        ev[4 * r + 2].record(stream)
        m.vjp(xt, res)
        ev[4 * r + 3].record(stream)
    torch.cuda.synchronize()
    for r in range(reps):
        fwd_ms += ev[4 * r].elapsed_time(ev[4 * r + 1]) / reps
        adj_ms += ev[4 * r + 2].elapsed_time(ev[4 * r + 3]) / reps
    pairs = n * (P + Nb)
    pairs_per_s = 2 * pairs / ((fwd_ms + adj_ms) / 1e3)
    del out, res

    # ---- the same LM step with the compensated bf16 Gauss-Newton matrix
    # (every operand split into two bf16 parts, three products), device time
    comp = None
    if cfg == 4 and args.jtj == "bf16" and not args.samples and not args.no_extras:
        mc = bg.BEM(precision=bg.BEM_MIXED, device=local, jtj_mode=bg.BEM_JTJ_BF16X3, near_factor=nf)
        mc.setup(sc.n_curves, sc.panels_per_curve, sc.closed, sc.theta_init, mean)
        mc.factor()
        lam_c = [1e-3]

        def step_c():
            r = mc.lm_step(xt, tt, lam_c)
            lam_c[0] = r["lambda_next"]

        step_c()
        torch.cuda.synchronize()
        ms_c = _timed(step_c, 3, flush, stream)
        comp = {"jtj": "bf16x3", "ms_per_step": sum(ms_c) / len(ms_c),
                "lm_iters_per_s": 1e3 * len(ms_c) / sum(ms_c), "steps": len(ms_c), "warmup": 1,
                "note": "the benched workload with the Gauss-Newton matrix in compensated bf16"}
        mc.close()

    # ---- FP64 GPU path: LM iterations on two leading sample sets (fitted
    # a + b S when they are smaller than the workload), colour and gradient
    # error of the mixed path against it
    fp64 = None
    accuracy = None
    if args.fp64_steps > 0:
        n64 = n if args.fp64_samples <= 0 else min(n, args.fp64_samples)
        m64 = bg.BEM(precision=bg.BEM_FP64, device=local)
        x64, t64 = xt[:n64].double(), tt[:n64].double()
        m64.setup(sc.n_curves, sc.panels_per_curve, sc.closed, sc.theta_init, mean)
        m64.factor()
        u64 = m64.eval(x64)
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
        m64.lm_step(x64[:n64 // 2], t64[:n64 // 2], [1e-3])
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
            th_, tf = t64_step(n64 // 2), t64_step(n64)
            b = (tf - th_) / (n64 - n64 // 2)
            t64_ms = tf + b * (n - n64)
            timed = (f"FP64 LM iterations on {n64 // 2} and {n64} of {n} samples "
                     f"({th_:.0f} ms, {tf:.0f} ms), extrapolated linearly in samples")
        fp64 = {"lm_iters_per_s": 1e3 / t64_ms, "ms_per_iter": t64_ms,
                "mixed_over_fp64": (value / world) / (1e3 / t64_ms), "timed": timed}
        accuracy = {"colour_rmse_mixed_vs_fp64_gpu": rmse, "grad_rel_err_mixed_vs_fp64_gpu": gerr,
                    "at": f"theta_init, {'all' if n64 == n else n64} samples"}
        m64.close()
        del x64, t64
    m.close()
    del xt, tt

    extras = None
    if cfg == 4 and not args.samples and not args.no_extras:
        extras = config2_extras(bg, dev, flush, stream, local, jm, rank)

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        r = oracle_rate(sc, xy, target, steps=args.cpu_steps, warmup=1)
        cpu = {k: r[k] for k in ("value", "unit", "cores", "kind", "cpu_model", "sample",
                                 "one_thread")}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": bench_config(sc, cfg, args.jtj),
            "wall_s_timed_region": t_wall,
            "pairs_per_s": {"value": pairs_per_s, "unit": "sample x panel evals/s (fwd+adjoint)",
                            "fwd_ms": fwd_ms, "adj_ms": adj_ms, "pairs_per_pass": pairs},
            "fp64_gpu": fp64, "accuracy": accuracy, "compensated_bf16": comp, "config2": extras,
            "pipe_peaks": pipes,
            "kernels": kernels,
            "roofline": roof, "rooflines_other": roofs[1:], "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clk, "gpu_launches": int(launches)}
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
    def kernel_totals(ms, steps, total_ms):
        tot = {}
        for m in ms:
            for k, (t, c) in m.profile_read().items():
                a = tot.setdefault(k, [0.0, 0])
                a[0] += t
                a[1] += c
            m.profile(False)
        out = {k: {"ms_per_step": v[0] / steps, "launches_per_step": v[1] / steps}
               for k, v in sorted(tot.items(), key=lambda kv: -kv[1][0])}
        out["_outside_kernels_ms_per_step"] = (total_ms - sum(v[0] for v in tot.values())) / steps
        return out

    # batched
    mb = contexts()
    b = bg.BEMBatch(mb)
    for _ in range(max(args.warmup, 0)):
        b.lm_step(xs, ts, lams)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    tb = 0.0
    for m in mb:
        m.profile(True)
    for _ in range(args.steps):
        flush.zero_()
        e0.record(stream)
        b.lm_step(xs, ts, lams)
        e1.record(stream)
        torch.cuda.synchronize()
        tb += e0.elapsed_time(e1)
    clk = clocks.stop()
    kb = kernel_totals(mb, args.steps, tb)
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
    for m in ms:
        m.profile(True)
    for _ in range(args.steps):
        flush.zero_()
        e0.record(stream)
        for m, x, t in zip(ms, xs, ts):
            m.lm_step(x, t, lams)
        e1.record(stream)
        torch.cuda.synchronize()
        tsq += e0.elapsed_time(e1)
    ks = kernel_totals(ms, args.steps, tsq)
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
            "batched_over_one_at_a_time": value / seq, "clocks": clk,
            "kernels_batched": kb, "kernels_one_at_a_time": ks,
            "kernels_note": "event times per kernel name; in the batched call the scenes' "
                            "Gauss-Newton passes and trial setups (damped solves, trial "
                            "geometry) run on one stream per scene, several at once, so those "
                            "kernels' times overlap and their sum exceeds the wall time they "
                            "take"}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--cpu-steps", type=int, default=8,
                    help="seeded 64-sample subsets of the oracle's per-sample part")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="leave out the secondary measurements on the 1M-sample workload")
    ap.add_argument("--oracle-probe", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--jtj", default="bf16", choices=["bf16", "bf16x3", "3xtf32"],
                    help="tensor-core scheme of the J^T J contraction")
    ap.add_argument("--config", type=int, default=CFG, choices=[2, 4, 5],
                    help="4: 67M samples, 8,192 panels (default); 2: 1M samples, 2,048 "
                         "panels; 5: batched uneven scenes against one at a time")
    ap.add_argument("--scenes", type=int, default=64, help="config 5: number of scenes")
    ap.add_argument("--fp64-samples", type=int, default=1 << 20,
                    help="config 4: samples of the FP64 GPU comparison (0 = all)")
    ap.add_argument("--samples", type=int, default=0,
                    help="profiling aid: time only the first N samples of the workload")
    args = ap.parse_args()
    if args.oracle_probe:
        oracle_probe(args.oracle_probe, args.config)
        return
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
