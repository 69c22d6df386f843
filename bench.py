#!/usr/bin/env python
"""Benchmark of the DomDec hot path on one GB300 (or N independent replicas).

Headline workload (``lognormal1024``): 1024 x 1024 grids, mu and nu seeded
log-normal random fields (correlation length 0.05) of masses 1.0 / 1.2,
squared-Euclidean cost, lam = 1, eps-scaling to (2/1024)^2 (global Sinkhorn
warm start from eps = 1 down to 2 (2/1024)^2, then DomDec at (2/1024)^2),
basic cells 16 x 16, FP32 cell Sinkhorn, FP64 score and step size, staggered
strategy (swift on each sub-batch, no leniency), cell tolerance 2e-5.

One step = one DomDec sweep over one partition (all four staggered
sub-batches: nu_{-J} gather, cell Sinkhorn, GetWeights, mixing and box
refresh, arena compaction).  Metric: cell-iterations per second (one X-half
plus one Y-half on one composite cell).  L2 is flushed (256 MB write) between
timed steps, outside the timed events.

The same JSON line also carries: the roofline of the cell kernel (exp terms
of its log-sum-exp passes against the MUFU ex2 rate measured on this GPU by
domdec_probe_peaks), the GB/s of the decision / mixing / compaction kernels,
an end-to-end number through the C ABI with host buffers (domdec_reset from
pinned host memory + sweeps + score and marginals back), the FP64 CPU oracle
on a bounded sample, and every other configuration of the benchmark plan:
blobs256 at lam = 0.1, 1, 10, mix32 (FP64, DomDec against global Sinkhorn to a
relative primal-dual gap of 1e-6), the time to a relative gap of 1e-5 on
blobs256 (the paper's pipeline first), batch64 (64 problems in one
persistent launch), grad512 (the backward pass) and the FP32-vs-FP64 error of
each result.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

# every FP64 oracle process of the CPU baseline runs single-threaded: keep BLAS to one thread
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to stated primal-dual gap and cell-iters/s vs full Sinkhorn on one GB300"
UNIT = "cell-iters/s"
GAP_TARGET = 1e-5
# dram read + write bytes of one cell-kernel launch (main grid, one staggered
# sub-batch) from an ncu capture of the current kernel in this configuration
# (profiles/cell_solve_lognormal1024.md); a size without an entry: not captured
# since the kernel last changed (reported as null)
CELL_KERNEL_DRAM_BYTES = {1024: 53298176 + 8162304}


def peaks_file():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def aggregate_ranks(units, ms, world, device):
    """Whole-job figures of N replicas: units summed over ranks, time = the
    slowest rank's (max).  world == 1: the local values."""
    if world <= 1:
        return float(units), float(ms)
    import torch
    import torch.distributed as dist
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u[0]), float(t[0])


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self):
        self.proc = None
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            dev = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0"
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={dev}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        rows = [r.split(",") for r in out.strip().splitlines() if r.strip()]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "samples": len(sm), "reasons": sorted(reasons)}


def to_dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel().copy()).cuda()


def warm_start(dd, torch, mu_d, nu_d, N, eps, lam, precision=None, err=2e-5 / 4, maxit=4000):
    """Global separable Sinkhorn from eps = 1 down to 2 eps at a quarter of the
    cell tolerance (Section 5.3 warm start).  Returns (alpha, beta, seconds, iterations)."""
    a = torch.empty(N * N, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    it, gap, P, D, rc = dd.domdec_full_sinkhorn(mu_d, nu_d, N, 2 * eps, lam, eps_start=1.0,
                                                variant=dd.SINKHORN_SEPARABLE,
                                                precision=dd.MIXED if precision is None else precision,
                                                maxit=maxit, err=err, check_every=10, alpha=a, beta=b)
    torch.cuda.synchronize()
    return a, b, time.perf_counter() - t0, it


def timed_sweeps(dd, torch, g, steps, warmup, flush, sample_clocks=False):
    """warmup untimed sweeps, then `steps` sweeps timed one by one with CUDA events
    on the current stream (L2 flushed before each, outside the events).
    Returns a dict of the timed region's figures."""
    g.iterate(warmup)
    g.sync()
    g.kernel_times(reset=True)
    st0 = g.stats()
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    sampler = ClockSampler() if sample_clocks else None
    torch.cuda.synchronize()
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        g.iterate(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    rc = g.sync()
    t_ms = sum(a.elapsed_time(b) for a, b in ev)
    st1 = g.stats()
    kms, kn = g.kernel_times(reset=True)
    d = {k: st1[k] - st0[k] for k in ("cell_iters", "cell_solves", "lse_terms", "box_points", "maxit_cells",
                                      "greedy_steps", "safe_steps")}
    d.update(ms=t_ms, kms=kms, kn=kn, clocks=clocks, box_entries=st1["box_entries"], rc=rc,
             max_ny=st1["max_ny"])
    return d


def roofline_of(d, pk, N, peaks_meas):
    """Cell kernel against the measured MUFU ex2 rate; the other sweep kernels
    against the measured HBM copy bandwidth (algorithmic bytes per launch)."""
    k1_s = d["kms"][0] / 1e3
    achieved = d["lse_terms"] / k1_s / 1e12 if k1_s > 0 else 0.0
    peak = peaks_meas["ex2_per_s"] / 1e12
    hbm = float(pk.get("hbm_gbs", 6800.0))
    n = N * N
    nsub = max(int(d["kn"][1]), 1)
    # decide: P_X, mu, P_Y, nu, dP_Y read per pixel (8 B each), log nu where dP_Y != 0
    dec_bytes = 5 * 8 * n
    # apply: per Y-box point of the solved cells, per quadrant: old value, new value read,
    # mixed value written (8 B each), plus dP_Y zeroed; P_X / P_Xnew mixed on the cells' pixels
    pts = d["box_points"] / nsub
    app_bytes = 4 * 3 * 8 * pts + 8 * pts + 3 * 8 * n / 4
    # compaction: every live box entry read and written once per sweep
    nsw = max(int(d["kn"][3]), 1)
    cmp_bytes = 16 * d["box_entries"]

    def gbs(b, ms, k):
        return b / (ms / k / 1e3) / 1e9 if ms > 0 else 0.0

    return {"bound": "alu", "kernel": "k_cell_solve<float>", "achieved": achieved, "peak": peak,
            "unit": "Tex2/s", "frac": achieved / peak if peak > 0 else 0.0,
            "traffic": CELL_KERNEL_DRAM_BYTES.get(N),
            "peak_source": ("measured on this GPU (domdec_probe_peaks: ex2.approx.ftz.f32 chains on all "
                            f"{peaks_meas['sms']} SMs): {peaks_meas['ex2_per_sm_clk']:.1f} ex2/SM/clk at "
                            f"{peaks_meas['ex2_sm_mhz']:.0f} MHz"),
            "kernel_share": float(d["kms"][0] / max(d["kms"].sum(), 1e-12)),
            "kernel_ms": {"cell_solve": float(d["kms"][0]), "decide": float(d["kms"][1]),
                          "apply": float(d["kms"][2]), "compact": float(d["kms"][3])},
            "launches": {"cell_solve": int(d["kn"][0]), "decide": int(d["kn"][1]), "apply": int(d["kn"][2]),
                         "compact": int(d["kn"][3])},
            "hbm_kernels": {"peak_gb_s": hbm,
                            "decide": {"bytes_per_launch": dec_bytes, "gb_s": gbs(dec_bytes, d["kms"][1], nsub)},
                            "apply": {"bytes_per_launch": app_bytes, "gb_s": gbs(app_bytes, d["kms"][2], nsub)},
                            "compact": {"bytes_per_launch": cmp_bytes,
                                        "gb_s": gbs(cmp_bytes, d["kms"][3], nsw)}}}


def sweep_config(dd, torch, name, lam, steps, warmup, flush, peaks_meas, pk, precision="fp32", cell_ctas=0):
    """Warm start + timed sweeps of one workload at one lam (the throughput
    figures of one configuration)."""
    from paper_2410_08859_gb300 import inputs
    mu, nu, spec = inputs.workload(name)
    N, s, eps = spec["N"], spec["s"], spec["eps"]
    mu_d, nu_d = to_dev(torch, mu), to_dev(torch, nu)
    a0, b0, t_w, it_w = warm_start(dd, torch, mu_d, nu_d, N, eps, lam)
    g = dd.DomDec(mu_d, nu_d, eps, lam, s, alpha0=a0, beta0=b0, eps_init=2 * eps, precision=precision,
                  tau=0.0, err=2e-5, profile=1, cell_ctas=cell_ctas)
    tuned = g.autotune() if cell_ctas == 0 else None
    d = timed_sweeps(dd, torch, g, steps, warmup, flush)
    cert = g.pd_gap()
    g.close()
    rl = roofline_of(d, pk, N, peaks_meas)
    return {"value": d["cell_iters"] / (d["ms"] / 1e3), "unit": UNIT, "ms_per_sweep": d["ms"] / steps,
            "mufu_frac": rl["frac"], "cell_kernel_share": rl["kernel_share"],
            "mean_iters_per_solve": d["cell_iters"] / max(d["cell_solves"], 1), "max_ny": d["max_ny"],
            "autotuned": None if tuned is None else {"cluster_ctas": tuned[0], "split": tuned[1]},
            "warm_start_s": t_w, "warm_start_iters": it_w, "rel_gap_after": float(cert[2])}


def domdec_to_gap(dd, torch, mu_d, nu_d, N, s, eps, lam, a0, b0, t_warm, target, max_sweeps=60, fast=False,
                  precision="fp32", err=1e-7, maxit=1000):
    """DomDec from a warm start until the certificate's relative gap reaches
    `target`.  fast = False: the paper's pipeline (plain cells, staggered swift);
    fast = True: the extension of this library (translation step in the cells,
    GetWeights_line on each staggered sub-batch; not in the paper)."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = dd.DomDec(mu_d, nu_d, eps, lam, s, alpha0=a0, beta0=b0, eps_init=2 * eps, precision=precision,
                  tau=0.0, err=err, maxit=300 if fast else maxit, profile=1,
                  cell_ti=1 if fast else 0, strategy="staggered_line" if fast else "staggered")
    sweeps, rel = 0, float("inf")
    while sweeps < max_sweeps:
        g.iterate(2)
        sweeps += 2
        rel = g.pd_gap()[2]
        if rel <= target:
            break
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    st = g.stats()
    kms, _ = g.kernel_times(reset=True)
    g.close()
    return {"s": t + t_warm, "warm_start_s": t_warm, "sweeps_s": t, "gap": rel, "sweeps": sweeps,
            "cell_iters": st["cell_iters"], "cell_kernel_ms": float(kms[0]),
            "cell_iters_per_s": st["cell_iters"] / max(kms[0] / 1e3, 1e-12), "lse_terms": int(st["lse_terms"])}


def sinkhorn_to_gap(dd, torch, mu_d, nu_d, N, eps, lam, variant, precision, target, max_rounds=6, maxit=3000,
                    err0=2e-5):
    """Global Sinkhorn with eps-scaling from 1 to eps, tightening the PD
    tolerance until the relative gap (E - D)/|D| <= target.
    Returns (seconds, gap, iterations)."""
    b = torch.zeros(N * N, dtype=torch.float64, device="cuda")
    a = torch.empty_like(b)
    err = err0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    it, gap, P, D, rc = dd.domdec_full_sinkhorn(mu_d, nu_d, N, eps, lam, eps_start=1.0, variant=variant,
                                                precision=precision, maxit=maxit, err=err, check_every=10,
                                                beta_in=b, alpha=a, beta=b)
    tot = it
    rel = (P - D) / abs(D)
    rounds = 0
    while not rel <= target and rounds < max_rounds:
        err /= 4
        it, gap, P, D, rc = dd.domdec_full_sinkhorn(mu_d, nu_d, N, eps, lam, variant=variant,
                                                    precision=precision, maxit=maxit, err=err,
                                                    check_every=10, beta_in=b.clone(), alpha=a, beta=b)
        tot += it
        rel = (P - D) / abs(D)
        rounds += 1
    torch.cuda.synchronize()
    return time.perf_counter() - t0, rel, tot


def time_to_gap_blobs256(dd, torch, mu, nu, spec, lam):
    """Time to a relative primal-dual gap of 1e-5 on blobs256, all from eps = 1
    on the same GPU: DomDec as in the paper (headline), the library's extension
    (labelled), global separable FP64 Sinkhorn (with and without the
    translation step) and the dense FP32 Sinkhorn of the plain method."""
    N, s, eps = spec["N"], spec["s"], spec["eps"]
    mu_d, nu_d = to_dev(torch, mu), to_dev(torch, nu)
    a0, b0, t_w, it_w = warm_start(dd, torch, mu_d, nu_d, N, eps, lam)
    paper = domdec_to_gap(dd, torch, mu_d, nu_d, N, s, eps, lam, a0, b0, t_w, GAP_TARGET)
    paper.update(what="warm start (global separable Sinkhorn, eps 1 -> 2 eps, PD/lam <= 5e-6 |mu|); "
                      "plain cell Sinkhorn (tolerance 1e-7, at most 1000 iterations); staggered swift "
                      "(Section 5.3)", warm_start_iters=it_w)
    a_f, b_f, t_wf, it_wf = warm_start(dd, torch, mu_d, nu_d, N, eps, lam, err=2e-5)
    ext = domdec_to_gap(dd, torch, mu_d, nu_d, N, s, eps, lam, a_f, b_f, t_wf, GAP_TARGET, fast=True)
    ext.update(what="not in the paper: looser warm start (2e-5); cells with the translation step (at most 300 "
                    "iterations); GetWeights_line per staggered sub-batch", warm_start_iters=it_wf)
    t_sep, g_sep, i_sep = sinkhorn_to_gap(dd, torch, mu_d, nu_d, N, eps, lam, dd.SINKHORN_SEPARABLE, dd.FP64,
                                          GAP_TARGET)
    t_ti, g_ti, i_ti = sinkhorn_to_gap(dd, torch, mu_d, nu_d, N, eps, lam,
                                       dd.SINKHORN_SEPARABLE | dd.SINKHORN_TI, dd.FP64, GAP_TARGET)
    t_den, g_den, i_den = sinkhorn_to_gap(dd, torch, mu_d, nu_d, N, eps, lam, dd.SINKHORN_DENSE, dd.FP32,
                                          GAP_TARGET, max_rounds=0, maxit=100)
    return {"target_rel_gap": GAP_TARGET, "workload": "blobs256", "lam": lam,
            "domdec_paper_pipeline": paper, "domdec_extension_pipeline": ext,
            "sinkhorn_separable_fp64": {"s": t_sep, "gap": g_sep, "iters": i_sep},
            "sinkhorn_separable_fp64_translation": {"s": t_ti, "gap": g_ti, "iters": i_ti,
                                                    "what": "not in the paper (translation step)"},
            "sinkhorn_dense_fp32": {"s": t_den, "gap": g_den, "iters": i_den,
                                    "what": "plain method, eps-scaling stages capped at 100 iterations"}}


def mix32_fp64(dd, torch):
    """Config 1: 32 x 32 Gaussian mixtures, FP64, pi0 = mu x nu; DomDec and the
    global separable Sinkhorn to a relative primal-dual gap of 1e-6."""
    from paper_2410_08859_gb300 import inputs
    mu, nu, spec = inputs.workload("mix32")
    N, s, eps, lam = spec["N"], spec["s"], spec["eps"], spec["lam"]
    mu_d, nu_d = to_dev(torch, mu), to_dev(torch, nu)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = dd.DomDec(mu_d, nu_d, eps, lam, s, precision="fp64", tau=0.0, err=1e-8, maxit=5000)
    sweeps, rel = 0, float("inf")
    while sweeps < 120:
        g.iterate(2)
        sweeps += 2
        rel = g.pd_gap()[2]
        if rel <= 1e-6:
            break
    torch.cuda.synchronize()
    t_dd = time.perf_counter() - t0
    its = g.stats()["cell_iters"]
    g.close()
    t_sk, g_sk, i_sk = sinkhorn_to_gap(dd, torch, mu_d, nu_d, N, eps, lam, dd.SINKHORN_SEPARABLE, dd.FP64, 1e-6,
                                       max_rounds=8, maxit=20000, err0=1e-6)
    return {"N": N, "s": s, "eps": eps, "lam": lam, "precision": "fp64", "target_rel_gap": 1e-6,
            "domdec": {"s": t_dd, "gap": rel, "sweeps": sweeps, "cell_iters": its},
            "sinkhorn_separable_fp64": {"s": t_sk, "gap": g_sk, "iters": i_sk}}


def fp32_vs_fp64(dd, torch, name, lam, sweeps=4):
    """The same sweeps from the same warm start with FP32 and with FP64 cell
    arithmetic: relative difference of the tracked score, L1 differences of
    P_X and P_Y relative to the mass, max difference of alpha relative to its
    magnitude, and whether the step-size decisions agree."""
    from paper_2410_08859_gb300 import inputs
    mu, nu, spec = inputs.workload(name)
    N, s, eps = spec["N"], spec["s"], spec["eps"]
    mu_d, nu_d = to_dev(torch, mu), to_dev(torch, nu)
    a0, b0, _, _ = warm_start(dd, torch, mu_d, nu_d, N, eps, lam)
    res = {}
    for prec in ("fp32", "fp64"):
        g = dd.DomDec(mu_d, nu_d, eps, lam, s, alpha0=a0, beta0=b0, eps_init=2 * eps, precision=prec, tau=0.0,
                      err=2e-5)
        g.iterate(sweeps)
        g.sync()
        res[prec] = (g.score()[0], *g.marginals(), g.duals(), g.decisions()[:, 3], g.pd_gap()[2])
        g.close()
    s32, s64 = res["fp32"], res["fp64"]
    mass = float(mu.sum())
    return {"workload": name, "lam": lam, "sweeps": sweeps,
            "score_rel": abs(s32[0] - s64[0]) / abs(s64[0]),
            "PX_l1_rel": float(np.abs(s32[1] - s64[1]).sum() / mass),
            "PY_l1_rel": float(np.abs(s32[2] - s64[2]).sum() / mass),
            "alpha_max_rel": float(np.abs(s32[3] - s64[3]).max() / (1 + np.abs(s64[3]).max())),
            "decisions_equal": bool(np.array_equal(s32[4], s64[4])),
            "rel_gap_fp32": float(s32[5]), "rel_gap_fp64": float(s64[5])}


def run_batch(dd, torch, steps, warmup, peaks_meas):
    """Many-instance batching (config 4): 64 independent problems (sides from
    {64, 128, 256, 512}, eps = (2/n)^2, lam in {0.5, 1, 5}) swept together in
    one persistent launch per staggered sub-batch, each warm-started by
    global Sinkhorn (float, 2e-5) down to 2 eps; against the same problems
    swept one after another with single handles."""
    from paper_2410_08859_gb300 import inputs
    probs = inputs.batch_instances(64)
    t0 = time.perf_counter()
    handles_b, handles_s = [], []
    for p in probs:
        N = p["N"]
        mu_d, nu_d = to_dev(torch, p["mu"]), to_dev(torch, p["nu"])
        a, b, _, _ = warm_start(dd, torch, mu_d, nu_d, N, p["eps"], p["lam"], precision=dd.FP32, err=2e-5,
                                maxit=1000)
        for lst in (handles_b, handles_s):
            lst.append(dd.DomDec(mu_d, nu_d, p["eps"], p["lam"], 8, alpha0=a, beta0=b, eps_init=2 * p["eps"],
                                 precision="fp32", tau=0.0, err=2e-5, spill_slots=32))
    torch.cuda.synchronize()
    t_warm = time.perf_counter() - t0
    B = dd.DomDecBatch(handles_b)
    chosen_c, chosen_f = B.autotune()
    B.iterate(warmup)
    B.sync()
    it0 = sum(h.stats()["cell_iters"] for h in handles_b)
    lt0 = sum(h.stats()["lse_terms"] for h in handles_b)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    B.iterate(steps)
    e1.record()
    torch.cuda.synchronize()
    B.sync()
    t_b = e0.elapsed_time(e1)
    it_b = sum(h.stats()["cell_iters"] for h in handles_b) - it0
    lt_b = sum(h.stats()["lse_terms"] for h in handles_b) - lt0
    for h in handles_s:
        h.iterate(warmup)
        h.sync()
    it0 = sum(h.stats()["cell_iters"] for h in handles_s)
    torch.cuda.synchronize()
    e0.record()
    for h in handles_s:
        h.iterate(steps)
    e1.record()
    torch.cuda.synchronize()
    for h in handles_s:
        h.sync()
    t_s = e0.elapsed_time(e1)
    it_s = sum(h.stats()["cell_iters"] for h in handles_s) - it0
    B.close()
    for h in handles_b + handles_s:
        h.close()
    peak = peaks_meas["ex2_per_s"] / 1e12
    return {"value": it_b / (t_b / 1000.0), "unit": UNIT, "ms_per_sweep": t_b / steps, "instances": len(probs),
            "sides": sorted(set(p["N"] for p in probs)),
            "autotuned": {"cluster_ctas": chosen_c, "split_factor_mean_works_per_cta": chosen_f},
            "sequential_single_handles": {"value": it_s / (t_s / 1000.0), "ms_per_sweep": t_s / steps},
            "batch_speedup": (it_b / t_b) / max(it_s / t_s, 1e-30),
            # exp terms of all cell iterations over the whole sweep time (decide, apply and
            # compaction included): a lower bound of the cell kernel's own fraction
            "mufu_frac_whole_sweep": (lt_b / (t_b / 1e3)) / 1e12 / peak, "warm_start_s": t_warm}


def run_grad(dd, torch, steps, warmup):
    """Differentiation (config 5): 512 x 512, eps = (2/512)^2, lam = 1, blob
    mixtures of masses 1.0 / 1.1; DomDec (FP32 cells) to a relative PD gap of
    1e-6, then the backward pass (beta_star by one global Y-half, adjoint
    kernels for d/dmu, d/dnu, d/dx) timed per call, FP32 and FP64 summation."""
    from paper_2410_08859_gb300 import autograd as ag
    from paper_2410_08859_gb300 import inputs
    N, s = 512, 8
    mu, nu = inputs.mixture_blobs(N=N, seed=5000, mass_ratio=1.1)
    eps, lam = (2.0 / N) ** 2, 1.0
    mu_d, nu_d = to_dev(torch, mu), to_dev(torch, nu)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g, info = ag.solve(mu_d, nu_d, eps, lam, s=s, gap=1e-6, precision="fp32")
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t0
    n = N * N
    bufs = {p: (torch.empty(n, dtype=torch.float64, device="cuda"), torch.empty(n, dtype=torch.float64, device="cuda"),
                torch.empty(2 * n, dtype=torch.float64, device="cuda")) for p in (dd.FP32, dd.FP64)}
    times = {}
    for p in (dd.FP32, dd.FP64):
        for _ in range(warmup):
            g.gradients(p, *bufs[p])
        ts = []
        for _ in range(steps):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            g.gradients(p, *bufs[p])
            ts.append(time.perf_counter() - t1)
        times[p] = 1000 * float(np.median(ts))
    a = torch.empty(n, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    dd.domdec_duals(g.h, a)
    g.gradients(dd.FP64, beta=b)
    adj = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for p in (dd.FP32, dd.FP64):
        for _ in range(warmup):
            dd.domdec_uot_gradients(mu_d, nu_d, a, b, N, eps, lam, p, *bufs[p])
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            dd.domdec_uot_gradients(mu_d, nu_d, a, b, N, eps, lam, p, *bufs[p])
        e1.record()
        torch.cuda.synchronize()
        adj[p] = e0.elapsed_time(e1) / steps
    errs = {}
    for k, name in enumerate(("mu", "nu", "x")):
        ref = bufs[dd.FP64][k]
        errs[name] = float((bufs[dd.FP32][k] - ref).abs().max() / ref.abs().max())
    g.close()
    return {"backward_ms": times[dd.FP32], "backward_fp64_ms": times[dd.FP64],
            "adjoint_only_ms": {"fp32": adj[dd.FP32], "fp64": adj[dd.FP64]}, "fp32_vs_fp64_rel_err": errs,
            "solve": {"seconds": t_solve, "sweeps": info["sweeps"], "rel_gap": info["rel_gap"]},
            "N": N, "eps": eps, "lam": lam, "masses": [1.0, 1.1]}


def e2e_reset(dd, torch, mu, nu, a0, b0, spec, lam, steps=3, sweeps=8):
    """End to end through the C ABI with host buffers: every step loads the
    problem from pinned host memory into one reused handle (domdec_reset: mu,
    nu and the warm-start duals), runs `sweeps` sweeps and reads the tracked
    score and both plan marginals back to pinned host memory."""
    N, s, eps = spec["N"], spec["s"], spec["eps"]
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64).ravel().copy()).pin_memory()
    mu_h, nu_h, a_h, b_h = pin(mu), pin(nu), a0.cpu().pin_memory(), b0.cpu().pin_memory()
    PX = torch.empty(N * N, dtype=torch.float64).pin_memory()
    PY = torch.empty_like(PX)
    g = dd.DomDec(mu_h, nu_h, eps, lam, s, alpha0=a_h, beta0=b_h, eps_init=2 * eps, precision="fp32", tau=0.0,
                  err=2e-5)
    g.iterate(1)
    g.sync()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    its = 0
    for _ in range(steps):
        g.reset(mu_h, nu_h, alpha0=a_h, beta0=b_h, eps_init=2 * eps)
        g.iterate(sweeps)
        g.score()
        dd.domdec_plan_marginals(g.h, PX, PY)
        its += g.stats()["cell_iters"]
    te = time.perf_counter() - t0
    g.close()
    return {"value": its / te, "unit": UNIT, "cell_iters": its, "seconds": te, "h2d_bytes_per_step": 4 * N * N * 8,
            "d2h_bytes_per_step": 2 * N * N * 8 + 6 * 8,
            "step": f"domdec_reset from pinned host mu, nu, alpha0, beta0 + {sweeps} sweeps + score + "
                    "P_X, P_Y to pinned host memory, one reused handle"}


def oracle_sample(max_seconds=20.0, sweeps=None, maxit=None):
    """The FP64 oracle on a bounded sample of the headline workload: a
    log-normal field (correlation length 0.05, masses 1.0 / 1.2) on a 32 x 32
    grid, eps = (2/32)^2 (4 pixels^2, as the workload's (2/1024)^2), lam = 1,
    s = 8, pi0 = mu x nu, staggered, cell tolerance 2e-5; whole sweeps are timed
    until max_seconds.  Returns (cell-iters/s, description, cell-iters, seconds)."""
    from oracle import domdec as odd
    from paper_2410_08859_gb300 import inputs
    N, s = 32, 8
    mu, nu = inputs.lognormal_field(N=N, seed=3100)
    mu, nu = mu.ravel(), nu.ravel()
    geo = odd.Geometry(N, s)
    st = odd.init_product(geo, mu, nu, (2.0 / N) ** 2, 1.0)
    t0 = time.perf_counter()
    its, k = 0, 0
    while True:
        lg = odd.sweep(st, "AB"[k % 2], "staggered", tau=0.0, err=2e-5, maxit=maxit or 2000)
        its += sum(sum(r["iters"]) for r in lg)
        k += 1
        el = time.perf_counter() - t0
        if (sweeps is not None and k >= sweeps) or (sweeps is None and el >= max_seconds):
            break
    desc = (f"oracle (NumPy FP64, 1 thread) DomDec sweeps on a log-normal 32x32 sample of the workload "
            f"(eps = 4 pixels^2 as the workload, lam=1, s=8: composite cells 16x16, pi0=mu x nu); "
            f"{k} sweeps, {its} cell-iterations in {el:.1f} s")
    return its / el, desc, its, el


def _oracle_worker(max_seconds):
    return oracle_sample(max_seconds=max_seconds)[:3]


def oracle_sample_all_cores(max_seconds=15.0):
    """oracle_sample in one single-threaded process per host core, all at once
    (spawned: this process holds a CUDA context).  Returns (summed
    cell-iters/s, processes, description)."""
    import multiprocessing as mp
    n = max(1, os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(n) as pool:
        res = pool.map(_oracle_worker, [max_seconds] * n, chunksize=1)
    rate = sum(r[0] for r in res)
    desc = (f"{n} processes (one per host core), each the 1-thread oracle on the same 32x32 sample for "
            f"{max_seconds:.0f} s; summed rate ({sum(r[2] for r in res)} cell-iterations)")
    return rate, n, desc


def _oracle_sweep_worker(_):
    return oracle_sample(sweeps=1, maxit=200)[2]


def run_reference(args, rank, world):
    """The oracle as it stands on every host core: each step runs one oracle
    sweep of the 32 x 32 sample in each of os.cpu_count() single-threaded
    processes at once (spawned, started before the timed steps)."""
    if rank != 0:
        return
    import multiprocessing as mp
    n = max(1, os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(n) as pool:
        for _ in range(args.warmup):
            pool.map(_oracle_sweep_worker, range(n), chunksize=1)
        t_all, its_all = 0.0, 0
        for _ in range(args.steps):
            t0 = time.perf_counter()
            its_all += sum(pool.map(_oracle_sweep_worker, range(n), chunksize=1))
            t_all += time.perf_counter() - t0
    value = its_all / t_all
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * t_all / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": "lognormal1024 (oracle sample: log-normal 32x32 grid, eps = 4 pixels^2, "
                                   "s = 8)", "lam": 1.0},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": n, "kind": "oracle",
                             "sample": f"per step one oracle sweep (cell maxit 200) on a log-normal 32x32 sample, "
                                       f"s=8, in each of {n} single-threaded processes (one per host core) at once"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--lam", type=float, default=1.0)
    ap.add_argument("--workload", default="lognormal1024", choices=["blobs256", "lognormal1024"])
    ap.add_argument("--no-extras", action="store_true",
                    help="headline line only: no other configurations, e2e or CPU baseline")
    ap.add_argument("--extras", default="all",
                    help="comma list of extras: configs,ttg,mix32,batch64,grad512,fp32fp64,e2e,cpu (default all)")
    ap.add_argument("--cell-ctas", type=int, default=0, choices=[0, 1, 2, 4, 8],
                    help="CTAs per cell of the timed sweeps (domdec_params.cell_ctas)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_2410_08859_gb300 import domdec as dd
    from paper_2410_08859_gb300 import inputs
    dd.lib()
    t_start = time.perf_counter()

    pk, pk_kind = peaks_file()
    peaks_meas = dd.domdec_probe_peaks(20000)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    # ---- headline: the contract's largest single-GPU configuration
    mu, nu, spec = inputs.workload(args.workload, instance=rank)
    N, s, eps, lam = spec["N"], spec["s"], spec["eps"], args.lam
    mu_d, nu_d = to_dev(torch, mu), to_dev(torch, nu)
    a0, b0, t_warm, it_warm = warm_start(dd, torch, mu_d, nu_d, N, eps, lam)
    g = dd.DomDec(mu_d, nu_d, eps, lam, s, alpha0=a0, beta0=b0, eps_init=2 * eps, precision="fp32",
                  tau=0.0, err=2e-5, profile=1, cell_ctas=args.cell_ctas)
    # the cell launch's cluster size and split threshold, chosen on this GPU (untimed sweeps)
    tuned = g.autotune() if args.cell_ctas == 0 else None
    if world > 1:
        dist.barrier()
    d = timed_sweeps(dd, torch, g, args.steps, args.warmup, flush, sample_clocks=(rank == 0))
    if world > 1:
        dist.barrier()
    cert = g.pd_gap()
    g.close()
    iters_all, t_max = aggregate_ranks(float(d["cell_iters"]), d["ms"], world, "cuda")
    value = iters_all / (t_max / 1000.0)
    # kernels of the timed region: per sweep one ordering kernel, per sub-batch the cell solve,
    # decision and mixing kernels, three compaction kernels (one timed class)
    launches = int(d["kn"][0] + d["kn"][1] + d["kn"][2] + 4 * d["kn"][3])
    # end to end through the C ABI with host buffers, on every rank: summed work over the
    # slowest rank's time, like the device figure
    e2e = None
    if not args.no_extras and (args.extras == "all" or "e2e" in args.extras.split(",")):
        e2e = e2e_reset(dd, torch, mu, nu, a0, b0, spec, lam)
        its_e, ms_e = aggregate_ranks(float(e2e["cell_iters"]), 1000.0 * e2e["seconds"], world, "cuda")
        e2e.update(value=its_e / (ms_e / 1000.0), cell_iters=int(its_e), seconds=ms_e / 1000.0)
    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    roofline = roofline_of(d, pk, N, peaks_meas)

    extras, cpu = {}, None
    # the other configurations and the CPU baseline at N = 1 only (under torchrun the other
    # ranks' GPUs would wait meanwhile)
    want = set() if args.no_extras or world > 1 else set(args.extras.split(",")) if args.extras != "all" else \
        {"configs", "ttg", "mix32", "batch64", "grad512", "fp32fp64", "cpu"}
    configs = {}
    if "configs" in want:
        configs["blobs256"] = {f"lam={lm:g}": sweep_config(dd, torch, "blobs256", lm, args.steps, args.warmup,
                                                             flush, peaks_meas, pk)
                               for lm in (0.1, 1.0, 10.0)}
    if "mix32" in want:
        configs["mix32"] = mix32_fp64(dd, torch)
    if "batch64" in want:
        configs["batch64"] = run_batch(dd, torch, 4, 2, peaks_meas)
    if "grad512" in want:
        configs["grad512"] = run_grad(dd, torch, 10, 3)
    if configs:
        extras["configs"] = configs
    if "ttg" in want:
        bm, bn, bspec = inputs.workload("blobs256")
        extras["time_to_gap"] = time_to_gap_blobs256(dd, torch, bm, bn, bspec, 1.0)
    if "fp32fp64" in want:
        extras["fp32_vs_fp64"] = [fp32_vs_fp64(dd, torch, "blobs256", 1.0), fp32_vs_fp64(dd, torch, "mix32", 1.0)]
    if "cpu" in want:
        v1, desc1, its, el = oracle_sample(max_seconds=10.0)
        cpu = {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc1,
               "host_cores": os.cpu_count()}
        try:
            va, nproc, desca = oracle_sample_all_cores(max_seconds=10.0)
            cpu.update(value=va, cores=nproc, sample=desca,
                       one_core={"value": v1, "cores": 1, "sample": desc1})
        except Exception as e:  # the one-core figure stands
            cpu["all_cores_error"] = repr(e)[:200]

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "N": N, "basic_cell": s, "eps": eps, "lam": lam,
                       "eps_scaling": "1 -> 2 eps by global Sinkhorn (warm start), DomDec at eps",
                       "strategy": "staggered", "tau": 0.0, "err": 2e-5, "precision": "fp32 cell / fp64 score",
                       "cell_ctas": args.cell_ctas,
                       "autotuned": None if tuned is None else {"cluster_ctas": tuned[0], "split": tuned[1]},
                       "l2": "flushed (256 MB write) between timed steps",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": d["clocks"],
            "gpu_launches": launches, "cell_iters_timed": int(iters_all),
            "mean_iters_per_solve": d["cell_iters"] / max(d["cell_solves"], 1), "max_ny": d["max_ny"],
            "warm_start": {"s": t_warm, "iters": it_warm},
            "final_rel_gap_after_timed_sweeps": float(cert[2]),
            "peaks_measured": peaks_meas, "peaks_file": pk_kind, "bench_wall_s": None}
    line.update(extras)
    line["bench_wall_s"] = time.perf_counter() - t_start
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
