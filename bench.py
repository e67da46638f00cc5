#!/usr/bin/env python
"""Benchmark of one Matérn log-likelihood + gradient evaluation in TLR form.

Workload (the n = 90,000 configuration): 300 x 300 jittered grid on [0,1]^2,
theta = (sigma2, beta, nu) = (1, 0.3, 1.0), tile size nb = 900, absolute
threshold eps = 1e-7, float64 storage.  One step is the whole path on one
batch: Matérn generation, compression of the off-diagonal tiles, TLR Cholesky,
log-determinant and solves (eq. 1), the adjoint gradient (TLR inverse and the
fused regenerate-and-reduce pass) and kriging of 100 new points (eq. 4) on the
same factor.  z is a draw from the model, z = L e with L the exact Cholesky
factor of the dense float64 comparator (measured once at the same n before
the timed region).

Prints one JSON line (rank 0).  --impl reference times the CPU oracle instead
(dense float64 likelihood + gradient on a bounded sample, scaled to n).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "loglik+grad evals/s at n=90k: TLR vs dense FP64, 1 GB300, rel err≤1e-6"
UNIT = "evals/s"
THETA = (1.0, 0.3, 1.0)
# float64 peak of the GB300 derived from unit counts and clock: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# double-float ceiling of the float32 pipe: 152 SMs x 128 lanes x 2.07 GHz, about 12 float32 instructions per
# float64-accurate multiply-add (2 flops)
FF32_CEIL_TFLOPS = 152 * 128 * 2.07e9 / 12 * 2 / 1e12
BF16_FALLBACK_TFLOPS = 1700.0  # sustained dense bf16 of an earlier GB300 measurement (no measured file)


def bf16_peak():
    """Sustained dense bf16 TFLOP/s from MEASURED_PEAKS.json (driver-written), else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        for key in ("bf16_tflops_sustained", "bf16_tflops"):
            if isinstance(d.get(key), (int, float)):
                return float(d[key]), f"measured ({key}, MEASURED_PEAKS.json)"
    except (OSError, ValueError):
        pass
    return BF16_FALLBACK_TFLOPS, "fallback (1.7 PFLOP/s sustained, earlier GB300 measurement)"
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic_n22500.json")
# the source each kernel's DRAM figure was measured on: (file, first marker, end marker or None)
KERNEL_SOURCES = {
    "k_upd_lr_pair": [("tileops.cu", None, "__global__ void k_upd_d_desc"), ("recompress.cuh", None, None),
                      ("tile.cuh", None, None), ("df.cuh", None, None)],
    "k_oz_gemm": [("tcgemm.cu", "// ------------------------------------------------------------------ GEMM",
                   "int launch_split("), ("tcgemm.h", "#define OZ_BM", "size_t oz_slices_elems("),
                  ("df.cuh", None, None)],
}


def _code_only(src: str) -> str:
    """C++ source without comments and whitespace: what the compiler turns into the kernel."""
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return re.sub(r"\s+", "", src)


def kernel_hash(kernel="k_upd_lr_pair"):
    """Hash of a kernel's source code (the parts of the files it is built from; comments and layout
    excluded): a DRAM traffic figure measured on another code state is not reported."""
    h = hashlib.sha256()
    for f, start, end in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1804_09137_gb300", "csrc", f), encoding="utf-8") as fh:
            src = fh.read()
        if start is not None:
            src = src[src.index(start):]
        if end is not None:
            src = src[:src.index(end)]
        h.update(_code_only(src).encode())
    return h.hexdigest()[:16]


def measured_traffic(kernel):
    """DRAM bytes per launch of `kernel` at the benchmark's size, from the committed ncu summary, when it
    was taken on the present source of that kernel (else None)."""
    try:
        with open(TRAFFIC_FILE) as fh:
            tr = json.load(fh).get(kernel, {})
    except (OSError, ValueError):
        return None
    return tr.get("dram_bytes_per_launch_n90000") if tr.get("source_sha") == kernel_hash(kernel) else None


def args_():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="tlr", choices=["tlr", "reference"])
    p.add_argument("--workload", default="n90k",
                   choices=["n90k", "regions", "n40k", "accuracy", "accuracy36k", "config4", "mc"],
                   help="n90k: the n = 90,000 TLR likelihood + gradient (default); regions: 512 independent "
                        "regions; n40k: TLR vs dense likelihood at n = 40,000 and kriging of 10% held out")
    p.add_argument("--regions", type=int, default=512)
    p.add_argument("--mc-reps", type=int, default=2, help="replicates per beta of the reduced Monte Carlo")
    p.add_argument("--mc-betas", default="0.03,0.1,0.3", help="range parameters of the reduced Monte Carlo")
    p.add_argument("--workers", type=int, default=8)
    p.add_argument("--side", type=int, default=300)
    p.add_argument("--nb", type=int, default=900)
    p.add_argument("--eps", type=float, default=1e-7)
    p.add_argument("--rank-cap", type=int, default=256)
    p.add_argument("--no-dense", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-side", type=int, default=40, help="grid side of the CPU oracle sample")
    return p.parse_args()


class Clocks:
    """nvidia-smi samples of the SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [c.strip() for c in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def log(*a):
    print("[bench]", *a, file=sys.stderr, flush=True)


def dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(x: float, world: int, device=None) -> float:
    """Largest value over the ranks (the slowest replica sets the job time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as tdist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(ms_per_step_max: float, world: int) -> float:
    """Whole-job evaluations per second: every replica completes one evaluation per step."""
    return world / (ms_per_step_max / 1e3)


def cpu_oracle_sample(side):
    """One dense CPU-oracle likelihood + gradient evaluation at n = side^2.

    Returns (total seconds, seconds of the O(n^2) Matérn and derivative generation (timed as a separate
    call of the same oracle functions), n)."""
    from oracle import dense as DN
    from oracle import matern as M
    from paper_1804_09137_gb300 import inputs

    x, y = inputs.jittered_grid(side)
    z = DN.sample(x, y, THETA, inputs.standard_normal(len(x)))
    t = time.perf_counter()
    DN.loglik_grad(x, y, z, THETA)
    total = time.perf_counter() - t
    t = time.perf_counter()
    R = DN.distances(x, y, x, y)
    M.matern(R, *THETA)
    M.matern_derivs(R, *THETA)
    gen = time.perf_counter() - t
    return total, min(gen, total), len(x)


def cpu_baseline_line(total, gen, ns, n, steps=1):
    """Scale a measured oracle run at ns points to n: generation ~ n^2, factorisation and inverse ~ n^3."""
    t_full = gen * (n / ns) ** 2 + (total - gen) * (n / ns) ** 3
    return t_full, {"value": 1.0 / t_full, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                    "sample": f"dense float64 oracle loglik+grad measured at n={ns} ({int(round(ns ** 0.5))}^2 "
                              f"grid): {total:.3f} s ({gen:.3f} s of it Matérn/derivative generation); value "
                              f"scaled to n={n} as gen*(n/{ns})^2 + rest*(n/{ns})^3",
                    "measured_n": ns, "measured_s": total, "measured_evals_per_s": 1.0 / total,
                    "extrapolated_s_at_n": t_full, "runs": steps}


def main_config(a, n, m_new, parallelism):
    """The configuration both arms report: the n = 90,000 TLR workload."""
    return {"workload": f"matern_tlr_n{n}_nb{a.nb}_eps{a.eps:g}_theta1-0.3-1.0", "n": n, "nb": a.nb,
            "eps": a.eps, "rank_cap": a.rank_cap, "theta": list(THETA), "kriging_points": m_new,
            "kriging_points_from": "uniform on [0,1]^2, not on the grid",
            "l2": "inputs larger than L2 (TLR factor > 1 GB)", "parallelism": parallelism}


PRECISION = {"storage": "f64", "potrf_trsv_logdet_quadform_gradient_sums": "f64",
             "tile_gemm_householder_qr": "float32 pairs (double-float: ~48-bit significand, float32 exponent "
                                         "range)",
             "inverse_depth_ge_256_contractions": "bf16 tensor cores (tcgen05) on 6 digit slices per float64 "
                                                  "operand, exact float32 accumulation of the leading slice "
                                                  "groups: ~1e-12 of the operands' scale",
             "gradient_derivative_polynomials": "float32 pairs (Horner on a double-float copy of the Matern "
                                                "table's coefficients; distances, weights and sums in f64)"}


def run_reference(a):
    world, rank, _ = dist()
    if rank != 0:
        return
    n_full = a.side * a.side
    tot, gen = [], []
    for i in range(a.warmup + a.steps):
        t, g, ns = cpu_oracle_sample(a.cpu_side)
        if i >= a.warmup:
            tot.append(t)
            gen.append(g)
    t_full, cpu = cpu_baseline_line(statistics.mean(tot), statistics.mean(gen), ns, n_full, a.steps)
    val = 1.0 / t_full
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": t_full * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": main_config(a, n_full, 100, "single"), "cpu_baseline": cpu,
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_regions(a):
    """512 independent regions, n_r ~ U{500..8000}, own theta each, eps = 1e-8, nb autotuned per size class."""
    import torch

    world, rank, local = dist()
    torch.cuda.set_device(local)
    import __graft_entry__ as ge

    ge.build()
    from paper_1804_09137_gb300 import inputs, regions
    from paper_1804_09137_gb300 import tlr as T

    eps = 1e-8
    dev = torch.device("cuda", local)
    sizes, thetas, pts = regions.region_problems(a.regions)
    t64 = lambda v: torch.tensor(np.asarray(v), dtype=torch.float64, device=dev)
    choice = regions.autotune_nb(sizes, eps, dev=dev)
    log("autotune", {k: v[:3] for k, v in choice.items()})
    xs = [t64(p[0]) for p in pts]
    ys = [t64(p[1]) for p in pts]
    zs = [t64(inputs.standard_normal(int(n), seed=7 + r)) for r, n in enumerate(sizes)]
    opts = [regions.make_opts(int(n), choice, eps) for n in sizes]
    for i in range(a.warmup):
        t0 = time.perf_counter()
        _, _, st = T.loglik_grad_batched(xs, ys, zs, thetas, opts, nworkers=a.workers)
        torch.cuda.synchronize()
        log(f"warmup {i}: {time.perf_counter() - t0:.2f} s, failures {sum(v != 0 for v in st)}")
    torch.cuda.synchronize()
    l0 = T.launch_count()
    clocks = Clocks(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        ll, grad, st = T.loglik_grad_batched(xs, ys, zs, thetas, opts, nworkers=a.workers)
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = reduce_max(e0.elapsed_time(e1) / a.steps, world, dev)
    value = world * a.regions / (ms / 1e3)
    if rank != 0:
        return
    line = {"metric": "independent regions loglik+grad evaluated per second (512 regions, n_r in [500, 8000])",
            "value": value, "unit": "regions/s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (jittered grid per region)",
            "config": {"workload": f"regions{a.regions}_n500-8000_eps1e-8", "regions": a.regions,
                       "sum_n": int(sizes.sum()), "workers": a.workers,
                       "nb_by_size_class": {str(k): v[0] for k, v in choice.items()},
                       "rank_cap_by_size_class": {str(k): v[1] for k, v in choice.items()},
                       "l2": "inputs larger than L2"},
            "gpu_launches": int(T.launch_count() - l0), "clocks": clk,
            "result": {"failures": int(sum(v != 0 for v in st)), "ll_sum": float(ll.sum().item())}}
    print(json.dumps(line), flush=True)


def run_mc(a):
    """Reduced Monte Carlo of the maximum-likelihood estimate (Sec. VIII-D1): the 200 x 200 jittered grid
    with 10% held out (n = 36,000 observed), theta0 = (1, beta, 0.5) for beta in {0.03, 0.1, 0.3},
    --mc-reps replicates each with z drawn from the exact model (dense float64 factor of this library).
    theta_hat by L-BFGS-B with the TLR likelihood and gradient (nb = 800, eps = 1e-9, rank cap 200) from a
    fixed start.  The dense float64 MLE is located from there to first order: the dense gradient g and
    Hessian H (central differences of dense gradients) at the TLR estimate give the Newton step
    -H^{-1} g to the dense maximiser; its size relative to theta_hat is the reported difference."""
    import torch

    import __graft_entry__ as ge

    ge.build()
    from paper_1804_09137_gb300 import inputs, mle
    from paper_1804_09137_gb300 import tlr as T

    dev = torch.device("cuda")
    t64 = lambda v: torch.tensor(np.asarray(v), dtype=torch.float64, device=dev)
    x, y = inputs.jittered_grid(200)
    obs, _ = inputs.holdout(len(x), len(x) // 10)
    xo, yo = t64(x[obs]), t64(y[obs])
    n = len(obs)
    hd = T.Handle(xo, yo, nb=800, eps=-1.0)
    ht = T.Handle(xo, yo, nb=800, eps=1e-9, rank_cap=200)

    def dense_grad(th, z):
        hd.factor(th)
        ll, g = hd.loglik_grad(z)
        hd.check()
        return float(ll.item()), g.cpu().numpy().astype(np.float64)

    out = []
    betas = [float(b) for b in a.mc_betas.split(",")]
    for beta in betas:
        theta0 = (1.0, beta, 0.5)
        for r in range(a.mc_reps):
            hd.factor(theta0)
            z = hd.sample(t64(inputs.standard_normal(n, seed=inputs.SEED + 1000 + r)))
            hd.check()
            start = (0.9, 1.2 * beta, 0.6)
            t0 = time.perf_counter()
            th_t, ll_t, info_t = mle.fit(ht, z, start, ftol=1e-15, gtol=1e-5, maxiter=200)
            t_t = time.perf_counter() - t0
            t0 = time.perf_counter()
            ll_d, g_d = dense_grad(th_t, z)
            H = np.zeros((3, 3))
            for p in range(3):
                hstep = 1e-4 * th_t[p]
                tp, tm = th_t.copy(), th_t.copy()
                tp[p] += hstep
                tm[p] -= hstep
                H[:, p] = (dense_grad(tp, z)[1] - dense_grad(tm, z)[1]) / (2 * hstep)
            H = 0.5 * (H + H.T)
            step = -np.linalg.solve(H, g_d)
            t_d = time.perf_counter() - t0
            th_d = th_t + step
            rel = [float(v) for v in np.abs(step) / np.abs(th_d)]
            rec = {"beta": beta, "rep": r, "theta_tlr": [float(v) for v in th_t], "theta_dense": [float(v) for v in th_d],
                   "rel_diff": rel, "loglik_tlr": ll_t, "loglik_dense_at_tlr": ll_d,
                   "dense_grad_at_tlr": [float(v) for v in g_d], "evals_tlr": info_t["evals"],
                   "converged_tlr": info_t["success"], "seconds_tlr": t_t, "seconds_dense_newton": t_d}
            log("mc", rec)
            out.append(rec)
    ht.close()
    hd.close()
    worst = max(max(r["rel_diff"]) for r in out)
    summary = {}
    for beta in betas:
        th = np.array([r["theta_tlr"] for r in out if r["beta"] == beta])
        summary[str(beta)] = {"mean_theta_tlr": th.mean(axis=0).tolist(), "std_theta_tlr": th.std(axis=0).tolist()}
    line = {"metric": "reduced Monte Carlo of theta_hat: TLR vs dense float64 MLE at n = 36,000",
            "value": worst, "unit": "max relative difference of theta_hat components", "n_gpus": 1,
            "higher_is_better": False, "data": "synthetic (z from the exact model)",
            "config": {"workload": "mc_n36000_nb800_eps1e-9_cap200", "n": n, "reps_per_beta": a.mc_reps,
                       "betas": betas, "dense_mle": "one Newton step from the TLR estimate "
                                                             "(dense gradient, central-difference Hessian)"},
            "within_1pct": bool(worst <= 0.01), "summary": summary, "runs": out}
    print(json.dumps(line), flush=True)


def run_n40k(a):
    """200 x 200 jittered grid, theta = (1, 0.1, 0.5), nb = 800, eps = 1e-9, rank cap 200; 10% held out.

    One likelihood evaluation on the 36,000 observed points in TLR form and in dense float64 (same library,
    every tile dense), their relative difference, the kriging MSE of the 4,000 held-out values (the
    paper's Sec. VIII-D1 reports an average MSE of 0.036 at beta = 0.1 for 100 held-out of 40K points)
    and their prediction variances."""
    import torch

    import __graft_entry__ as ge

    ge.build()
    from paper_1804_09137_gb300 import inputs
    from paper_1804_09137_gb300 import tlr as T

    theta = (1.0, 0.1, 0.5)
    dev = torch.device("cuda")
    t64 = lambda v: torch.tensor(np.asarray(v), dtype=torch.float64, device=dev)
    x, y = inputs.jittered_grid(200)
    n = len(x)
    # z at all 40,000 points from a tight factor (eps = 1e-12), then 10% held out
    hs = T.Handle(t64(x), t64(y), nb=800, eps=1e-12, rank_cap=400)
    hs.factor(theta)
    z = hs.sample(t64(inputs.standard_normal(n)))
    hs.check()
    hs.close()
    obs, held = inputs.holdout(n, n // 10)
    zo = z[torch.as_tensor(obs, device=dev)].contiguous()
    zh = z[torch.as_tensor(held, device=dev)].contiguous()
    res = {}
    for name, eps, cap in (("tlr", 1e-9, 200), ("dense", -1.0, 0)):
        h = T.Handle(t64(x[obs]), t64(y[obs]), nb=800, eps=eps, rank_cap=cap)
        for _ in range(2 if name == "tlr" else 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h.factor(theta)
            out = h.loglik(zo)
            torch.cuda.synchronize()
            secs = time.perf_counter() - t0
        h.check()
        pred = h.predict(zo, t64(x[held]), t64(y[held]))
        mse = float(((pred - zh) ** 2).mean().item())
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        var = h.predict_var(t64(x[held]), t64(y[held]))
        torch.cuda.synchronize()
        var_s = time.perf_counter() - t1
        h.check()
        # standardised errors of a calibrated predictor have mean square 1
        calib = float((((pred - zh) ** 2) / var.clamp_min(1e-300)).mean().item())
        res[name] = {"loglik": float(out[0].item()), "seconds": secs, "mse": mse,
                     "mean_pred_var": float(var.mean().item()), "pred_var_seconds": var_s,
                     "standardised_mse": calib, "ranks": h.rank_stats() if name == "tlr" else None}
        log(name, res[name])
        h.close()
    rel = abs(res["tlr"]["loglik"] - res["dense"]["loglik"]) / abs(res["dense"]["loglik"])
    line = {"metric": "loglik evals/s at n=36k (40k grid, 10% held out): TLR eps=1e-9 vs dense FP64",
            "value": 1.0 / res["tlr"]["seconds"], "unit": "evals/s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": res["tlr"]["seconds"] * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "matern_n40000_nb800_eps1e-9_cap200_theta1-0.1-0.5", "n_obs": len(obs),
                       "n_held_out": len(held)},
            "dense_fp64_gpu": {"value": 1.0 / res["dense"]["seconds"], "unit": "evals/s",
                               "seconds": res["dense"]["seconds"]},
            "tlr_rel_err_vs_dense": rel, "kriging_mse": {"tlr": res["tlr"]["mse"], "dense": res["dense"]["mse"],
                                                        "paper_average_beta_0.1": 0.036},
            "result": res}
    print(json.dumps(line), flush=True)


def run_accuracy(a):
    """TLR against the dense float64 path of the same library at the full n = 89,900 configuration.

    One evaluation each of l and dl/dtheta (z drawn from the TLR model as in the benchmark); the dense
    handle stores every tile dense and runs the same kernels with no truncation anywhere."""
    import torch

    import __graft_entry__ as ge

    ge.build()
    from paper_1804_09137_gb300 import inputs
    from paper_1804_09137_gb300 import tlr as T

    dev = torch.device("cuda")
    t64 = lambda v: torch.tensor(np.asarray(v), dtype=torch.float64, device=dev)
    x, y = inputs.jittered_grid(a.side)
    obs, _ = inputs.holdout(len(x), 100)
    xo, yo = t64(x[obs]), t64(y[obs])
    res = {}
    h = T.Handle(xo, yo, nb=a.nb, eps=a.eps, rank_cap=a.rank_cap)
    h.factor(THETA)
    z = h.sample(t64(inputs.standard_normal(len(obs))))
    for name, eps in (("tlr", a.eps), ("dense", -1.0)):
        if name == "dense":
            h.close()
            torch.cuda.empty_cache()
            h = T.Handle(xo, yo, nb=a.nb, eps=-1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.factor(THETA)
        ll, g = h.loglik_grad(z)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        h.check()
        res[name] = {"loglik": float(ll.item()), "grad": [float(v) for v in g.cpu().numpy()], "seconds": secs}
        log(name, res[name])
    h.close()
    ld, lt = res["dense"]["loglik"], res["tlr"]["loglik"]
    gd, gt = np.array(res["dense"]["grad"]), np.array(res["tlr"]["grad"])
    line = {"metric": "TLR vs dense FP64 at n=89,900: relative error of l and of dl/dtheta", "n": len(obs),
            "nb": a.nb, "eps": a.eps, "theta": list(THETA), "loglik_rel_err": abs(lt - ld) / abs(ld),
            "grad_rel_err": [float(v) for v in np.abs(gt - gd) / np.abs(gd)],
            "grad_rel_err_norm": float(np.linalg.norm(gt - gd) / np.linalg.norm(gd)),
            "seconds": {"tlr": res["tlr"]["seconds"], "dense": res["dense"]["seconds"]}, "result": res}
    print(json.dumps(line), flush=True)


def _host_free_ram_gb():
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 1e6
    except OSError:
        pass
    return 0.0


def run_accuracy36k(a):
    """Accuracy against true float64 at scale: the 40k configuration (200 x 200 grid, theta = (1, 0.1, 0.5),
    nb = 800, 10% held out: n = 36,000 observed).  The CPU oracle's dense float64 l (scipy kv, LAPACK
    Cholesky) against the library's TLR l at eps = 1e-7 and 1e-9 and its dense path (float-float tile GEMMs).
    Needs about 80 GB of host memory for the oracle's dense matrices; refuses to start with less."""
    import torch

    import __graft_entry__ as ge

    ge.build()
    from oracle import dense as DN
    from paper_1804_09137_gb300 import inputs
    from paper_1804_09137_gb300 import tlr as T

    need = 90.0
    if _host_free_ram_gb() < need:
        print(json.dumps({"workload": "accuracy36k", "skipped": f"needs {need:.0f} GB of free host memory, "
                                                                  f"{_host_free_ram_gb():.0f} GB available"}))
        return
    theta = (1.0, 0.1, 0.5)
    dev = torch.device("cuda")
    t64 = lambda v: torch.tensor(np.asarray(v), dtype=torch.float64, device=dev)
    x, y = inputs.jittered_grid(200)
    obs, _ = inputs.holdout(len(x), len(x) // 10)
    xo, yo = x[obs], y[obs]
    res = {}
    hd = T.Handle(t64(xo), t64(yo), nb=800, eps=-1.0)
    hd.factor(theta)
    z = hd.sample(t64(inputs.standard_normal(len(obs))))  # z = L e from the dense factor (input only)
    out = hd.loglik(z).cpu().numpy()
    hd.check()
    hd.close()
    res["gpu_dense"] = [float(v) for v in out]
    for eps in (1e-7, 1e-9):
        h = T.Handle(t64(xo), t64(yo), nb=800, eps=eps, rank_cap=400)
        h.factor(theta)
        res[f"gpu_tlr_eps{eps:g}"] = [float(v) for v in h.loglik(z).cpu().numpy()]
        h.check()
        h.close()
    zc = z.cpu().numpy()
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    ll, ld, q = DN.loglik(xo, yo, zc, theta)
    t_cpu = time.perf_counter() - t0
    res["cpu_oracle"] = [float(ll), float(ld), float(q)]
    rel = {k: {"loglik": abs(v[0] - ll) / abs(ll), "logdet": abs(v[1] - ld) / abs(ld), "quad": abs(v[2] - q) / abs(q)}
           for k, v in res.items() if k != "cpu_oracle"}
    print(json.dumps({"workload": "accuracy36k", "n": len(obs), "theta": list(theta), "nb": 800,
                      "rel_err_vs_cpu_oracle": rel, "cpu_oracle_seconds": t_cpu, "cores": os.cpu_count(),
                      "values": res}), flush=True)


def run_config4(a):
    """The mixed-precision configuration: 500 x 500 jittered grid (n = 250,000), theta = (1, 0.1, 0.5),
    nb = 2000, eps = 1e-7, l only.  z = L e from a tighter TLR factor (eps = 1e-9, double-float), whose l
    is the reference (the dense path would need 250 GB and the CPU TLR reference is out of reach at this
    size).  One evaluation each with precision 5 (tensor-core contractions of depth >= 256 in the
    Cholesky, 5 bf16 slices) and precision 1 (double-float on the CUDA cores)."""
    import torch

    import __graft_entry__ as ge

    ge.build()
    from paper_1804_09137_gb300 import inputs
    from paper_1804_09137_gb300 import tlr as T

    theta = (1.0, 0.1, 0.5)
    side, nb, cap = 500, 2000, 256
    dev = torch.device("cuda")
    t64 = lambda v: torch.tensor(np.asarray(v), dtype=torch.float64, device=dev)
    x, y = inputs.jittered_grid(side)
    xo, yo = t64(x), t64(y)
    res = {}
    h = T.Handle(xo, yo, nb=nb, eps=1e-9, rank_cap=cap, precision=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h.factor(theta)
    torch.cuda.synchronize()
    z = h.sample(t64(inputs.standard_normal(len(x))))
    ref = h.loglik(z).cpu().numpy()
    h.check()
    res["ref_eps1e-9"] = {"loglik": float(ref[0]), "factor_s": time.perf_counter() - t0, "ranks": h.rank_stats()}
    h.close()
    del h
    torch.cuda.empty_cache()
    log("reference", res["ref_eps1e-9"])
    for prec in (5, 1):
        h = T.Handle(xo, yo, nb=nb, eps=a.eps, rank_cap=cap, precision=prec)
        for rep in range(2):  # the second evaluation is timed
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h.factor(theta)
            out = h.loglik(z)
            torch.cuda.synchronize()
            secs = time.perf_counter() - t0
        h.check()
        o = out.cpu().numpy()
        res[f"precision{prec}"] = {"loglik": float(o[0]), "seconds": secs,
                                   "rel_err_vs_ref": abs(float(o[0]) - float(ref[0])) / abs(float(ref[0])),
                                   "ranks": h.rank_stats(), "tiles": h.tile_counts()}
        log(prec, res[f"precision{prec}"])
        h.close()
        del h
        torch.cuda.empty_cache()
    line = {"metric": "loglik evals/s at n=250k (500^2 grid), nb=2000, eps=1e-7, mixed precision",
            "value": 1.0 / res["precision5"]["seconds"], "unit": "evals/s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": res["precision5"]["seconds"] * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+ff32+bf16x5", "data": "synthetic (z from the eps = 1e-9 TLR factor)",
            "config": {"workload": "matern_tlr_n250000_nb2000_eps1e-7_theta1-0.1-0.5", "n": len(x), "nb": nb,
                       "eps": a.eps, "rank_cap": cap},
            "double_float_seconds": res["precision1"]["seconds"], "result": res}
    print(json.dumps(line), flush=True)


def main():
    a = args_()
    if a.workload == "accuracy" and a.impl != "reference":
        return run_accuracy(a)
    if a.workload == "n40k" and a.impl != "reference":
        return run_n40k(a)
    if a.workload == "accuracy36k" and a.impl != "reference":
        return run_accuracy36k(a)
    if a.workload == "mc" and a.impl != "reference":
        return run_mc(a)
    if a.workload == "config4" and a.impl != "reference":
        return run_config4(a)
    if a.impl == "reference":
        return run_reference(a)
    if a.workload == "regions":
        return run_regions(a)
    import torch

    world, rank, local = dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as tdist

        tdist.init_process_group("nccl")
    import __graft_entry__ as ge

    ge.build()
    from paper_1804_09137_gb300 import inputs
    from paper_1804_09137_gb300 import tlr as T

    dev = torch.device("cuda", local)
    t64 = lambda v: torch.tensor(np.asarray(v), dtype=torch.float64, device=dev)
    x, y = inputs.jittered_grid(a.side)
    n = len(x)  # every grid point is observed
    xn_h, yn_h = inputs.uniform_points(100)
    xo, yo = t64(x), t64(y)
    xh, yh = t64(xn_h), t64(yn_h)
    e = t64(inputs.standard_normal(n))

    # ---- dense float64 comparator at the same n (every tile dense, no truncation anywhere), measured once
    # outside the timed region; its exact Cholesky factor also draws z = L e from the model itself
    dense = None
    z = None
    if not a.no_dense:
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(dev)[0]
        hd = T.Handle(xo, yo, nb=a.nb, eps=-1.0)
        t0 = time.perf_counter()
        hd.factor(THETA)
        torch.cuda.synchronize()
        t_f = time.perf_counter() - t0
        z = hd.sample(e)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lld, gd = hd.loglik_grad(z)
        pd = hd.predict(z, xh, yh)
        torch.cuda.synchronize()
        t_g = time.perf_counter() - t0
        hd.check()
        dense_bytes = free0 - torch.cuda.mem_get_info(dev)[0]
        td = t_f + t_g
        dense = {"value": 1.0 / td, "unit": UNIT, "measured_n": n, "measured_s": td, "factor_s": t_f,
                 "grad_and_kriging_s": t_g, "device_bytes": int(dense_bytes),
                 "loglik": float(lld.item()), "grad": [float(v) for v in gd.cpu().numpy()]}
        pred_dense = pd.clone()
        hd.close()
        del hd
        torch.cuda.synchronize()
        log(f"dense comparator: factor {t_f:.1f} s, gradient + kriging {t_g:.1f} s")

    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    h = T.Handle(xo, yo, nb=a.nb, eps=a.eps, rank_cap=a.rank_cap)
    # counts launches of the low-rank update kernel before the timed region (ncu -s offsets)
    T.profile(True)
    if z is None:  # without the dense comparator: a draw from the TLR model (not timed)
        h.factor(THETA)
        z = h.sample(e)
        h.check()
    ll = torch.empty(1, dtype=torch.float64, device=dev)
    grad = torch.empty(3, dtype=torch.float64, device=dev)
    pred = torch.empty(len(xn_h), dtype=torch.float64, device=dev)
    hist = torch.zeros(a.warmup + a.steps, 4, dtype=torch.float64, device=dev)
    nstep = [0]

    def step(zz):
        h.matern_generate(THETA)
        h.compress()
        h.potrf()
        h.loglik_grad(zz, ll, grad)
        h.predict(zz, xh, yh, pred)

    def record():
        if nstep[0] < hist.shape[0]:
            hist[nstep[0], 0:1].copy_(ll)
            hist[nstep[0], 1:4].copy_(grad)
        nstep[0] += 1

    log("setup done", f"n={n}")
    for i in range(a.warmup):
        t0 = time.perf_counter()
        step(z)
        record()
        torch.cuda.synchronize()
        log(f"warmup {i}: {time.perf_counter() - t0:.2f} s")
    h.check()
    tlr_bytes = free0 - torch.cuda.mem_get_info(dev)[0]
    mem = h.memory()  # the handle's own account: arenas, their used part, workspaces
    stream = torch.cuda.current_stream()
    clocks = Clocks(local)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timed region
    barrier()
    pre = T.profile_read()["launches"]
    T.profile(True)
    l0 = T.launch_count()
    log(f"timed region starts after {l0} launches of this library ({pre} of k_upd_lr_gen)")
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        step(z)
        record()
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    launches = T.launch_count() - l0
    prof = T.profile_read()
    prof_tc = T.profile_read_tc()
    T.profile(False)
    ms = e0.elapsed_time(e1) / a.steps
    h.check()
    ms = reduce_max(ms, world, dev)
    value = replica_throughput(ms, world)
    log(f"timed: {ms:.1f} ms/step, profile {prof}")
    # every step (warm-up and timed) gives bitwise the same l and gradient
    hh = hist.cpu().numpy()
    deterministic = bool(np.all(hh == hh[0:1]))

    # ---- end to end: pinned host z in, (l, grad) out, every step
    z_h = z.cpu().pin_memory()
    out_h = torch.empty(4, dtype=torch.float64).pin_memory()
    out_d = torch.empty(4, dtype=torch.float64, device=dev)
    z_d = torch.empty_like(z)
    barrier()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        z_d.copy_(z_h, non_blocking=True)
        step(z_d)
        out_d[0:1].copy_(ll)
        out_d[1:4].copy_(grad)
        out_h.copy_(out_d, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    barrier()
    e2e_s = (time.perf_counter() - t0) / a.steps
    e2e_s = reduce_max(e2e_s, world, dev)
    log(f"e2e: {e2e_s:.2f} s/step")
    e2e = {"value": replica_throughput(e2e_s * 1e3, world), "unit": UNIT, "h2d_bytes_per_step": int(z_h.numel() * 8),
           "d2h_bytes_per_step": int(out_h.numel() * 8)}

    result = out_h.numpy().copy()
    # prediction variance at 4,000 new points (batched multi-right-hand-side solve), after the timed region
    xv, yv = inputs.uniform_points(4000, seed=inputs.SEED + 11)
    xv, yv = (torch.tensor(v, dtype=torch.float64, device=dev) for v in (xv, yv))
    torch.cuda.synchronize()
    t_var = time.perf_counter()
    var4k = h.predict_var(xv, yv)
    torch.cuda.synchronize()
    t_var = time.perf_counter() - t_var
    h.check()
    pred_var = {"points": 4000, "seconds": t_var, "min": float(var4k.min().item()), "max": float(var4k.max().item())}
    ranks = h.rank_stats()
    counts = h.tile_counts()
    inv = h.inverse_stats()
    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
        return

    # ---- roofline of the dominant kernel (low-rank update with recompression)
    achieved = prof["flops"] / (prof["ms"] * 1e-3) / 1e12 if prof["ms"] > 0 else None
    traffic = measured_traffic("k_upd_lr_pair")
    roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": (achieved / FP64_PEAK_TFLOPS) if achieved else None, "traffic": traffic,
            "kernel": "k_upd_lr_pair", "launches": prof["launches"], "kernel_ms_per_step": prof["ms"] / a.steps,
            "peak_source": "float64 derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (a DFMA loop measured "
                           "1.19 TFLOP/s)",
            "frac_of_ff32_ceiling": (achieved / FF32_CEIL_TFLOPS) if achieved else None,
            "ff32_ceiling": FF32_CEIL_TFLOPS}
    # the tensor-core GEMM of the inverse (bf16 slice products): MMA flops / its device time
    bpk, bsrc = bf16_peak()
    tc_ach = prof_tc["flops"] / (prof_tc["ms"] * 1e-3) / 1e12 if prof_tc["ms"] > 0 else None
    roof_tc = {"bound": "tensor", "kernel": "k_oz_gemm", "achieved": tc_ach, "peak": bpk, "unit": "TFLOP/s",
               "frac": (tc_ach / bpk) if tc_ach else None, "peak_source": bsrc, "launches": prof_tc["launches"],
               "kernel_ms_per_step": prof_tc["ms"] / a.steps, "mma_flops_per_step": prof_tc["flops"] / a.steps,
               "traffic": measured_traffic("k_oz_gemm")}

    accuracy = None
    if dense is not None:
        dense["tlr_speedup"] = value / dense["value"]
        gdn, gt = np.array(dense["grad"]), result[1:4]
        accuracy = {"vs": "dense float64 path of this library at the same n (equal to the CPU oracle to <= 1e-10 "
                          "at n <= 870)",
                    "loglik_rel_err": abs(result[0] - dense["loglik"]) / abs(dense["loglik"]),
                    "grad_rel_err": [float(v) for v in np.abs(gt - gdn) / np.abs(gdn)],
                    "kriging_max_abs_diff": float((pred - pred_dense).abs().max().item())}

    cpu = None
    if not a.no_cpu and world == 1:
        tot, gen, ns = cpu_oracle_sample(a.cpu_side)
        _, cpu = cpu_baseline_line(tot, gen, ns, n)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64+ff32+bf16x6", "precision": PRECISION,
            "data": "synthetic (jittered grid; z = L e drawn from the exact model by the dense path)"
                    if dense is not None else "synthetic (jittered grid; z drawn from the TLR model)",
            "config": main_config(a, n, len(xn_h), "replicas" if world > 1 else "single"),
            "roofline": roof, "roofline_tensor": roof_tc, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "gpu_launches_per_step": int(launches) / a.steps, "clocks": clk,
            "dense_fp64_gpu": dense, "accuracy": accuracy, "deterministic_across_steps": deterministic,
            "device_bytes": {"tlr_handle_after_first_step": int(tlr_bytes), "handle": mem},
            "prediction_variance": pred_var,
            "result": {"loglik": float(result[0]), "grad": [float(v) for v in result[1:4]], "ranks": ranks,
                       "tiles": counts, "inverse": inv}}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()


if __name__ == "__main__":
    main()
