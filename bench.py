#!/usr/bin/env python
"""Throughput of the BPMF Gibbs sampler: rows sampled per second per iteration.

One step is one Gibbs iteration of Algorithm 1 over the whole workload:
hyperparameters of the users, every user row, hyperparameters of the movies,
every movie row, then the test predictions and RMSE.  rows/s = (M + N) per
iteration / iteration time.

Default workload: Netflix-shaped synthetic ratings (480,189 x 17,770, 100M
ratings, 10% held out, power-law degrees, K = 100), generated on the device
from a seed.  The timed region starts with every input resident in HBM.  Its
working set per iteration (two compressed copies of 90M ratings, 1.4 GB, plus
the factors) is far larger than the 129 MB L2, so no flush is needed.

Reported beside the main value: the plain FP32 GPU form on the same workload,
an end-to-end number through the C ABI from pinned host buffers (bpmf_init,
the iterations, copies of the result), the roofline of the dominant kernel,
and the FP64 CPU oracle on a bounded sample of the workload.

--impl reference runs the CPU oracle (the reference arm) on bounded samples.
Multi-GPU (torchrun): every rank runs an independent replica; no collective
touches the data path (rows of a job never leave their GPU).
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "rows sampled/s per Gibbs sweep"
UNIT = "rows/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP32_LANES_PER_SM = 128  # FP32 FMA lanes per Blackwell SM (2 flop each per clock)
# DRAM bytes per launch of the dominant kernel from one ncu capture, with the
# case and kernel version they were taken on; keyed by (workload, side,
# heavy kernel, consumer warps).  A capture of a smaller case is scaled to the
# full launch by ratings (the per-rating index and value reads dominate).
TRAFFIC = {
    ("netflix", 0, 1, 6): (
        849.56e6 + 183.31e6,
        "ncu dram__bytes_read + dram__bytes_write of the users launch with this schedule (six "
        "consumers), captured on this full-size workload (1-pass metrics; "
        "profiles/dram_netflix_k100_fullsize.md)"),
}


def fp32_peak_from(sms, sm_mhz):
    """FP32 CUDA-core peak in TFLOP/s from unit counts: SMs x 128 lanes x 2 flop x clock."""
    return sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def fp32_peak_tflops(sm_mhz):
    """The same for this device's SM count."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    return fp32_peak_from(sms, sm_mhz), sms


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="netflix")
    p.add_argument("--relabel", choices=["none", "degree"], default="none",
                   help="degree: renumber the rows (users) in descending degree order before "
                        "the sampler sees them, so that the most-rated users' factor rows are "
                        "contiguous (the locality reordering of paper Sec. IV-B, measured)")
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--autotune", type=int, default=1, choices=[0, 1])
    p.add_argument("--heavy", type=int, default=0, choices=[0, 1, 2],
                   help="heavy-row kernel: 0 tuned, 1 persistent, 2 one CTA per row")
    p.add_argument("--thresholds", default=None,
                   help="schedule for both sides instead of the autotuner's, as printed under "
                        "bins.thresholds_tiny_light_hub: 'users;movies', five integers each, "
                        "e.g. --thresholds=-1,0,1099511627776,1,6;-1,0,1099511627776,1,2")
    p.add_argument("--serving-jobs", type=int, default=256)
    p.add_argument("--serving-iters", type=int, default=50)
    p.add_argument("--path", default="mixed", choices=["mixed", "binned", "plain"],
                   help="execution path of the main arm")
    p.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle work")
    p.add_argument("--no-cpu-full", action="store_true",
                   help="skip the fully timed oracle iteration of the CPU baseline")
    return p.parse_args()


# ------------------------------------------------------------------ dist --

def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks --

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)

    def summary(self):
        sm, mx, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power)}


# ------------------------------------------------------------- workload --

def load_workload(name, seed, device):
    """A named recipe of synth, or "powerlaw:M:N:nnz:K:row_expo:col_expo"."""
    import synth
    if name.startswith("powerlaw:"):
        M, N, nnz, K = (int(x) for x in name.split(":")[1:5])
        re_, ce = (float(x) for x in name.split(":")[5:7])
        return synth.powerlaw(M, N, nnz, K, re_, ce, seed=seed, alpha=2.0, device=device,
                              name=name)
    cache = os.environ.get("BPMF_SYNTH_CACHE", "/tmp/bpmf_synth_cache")
    return synth.make(name, seed=seed, device=device, cache_dir=cache)


def relabel_by_degree(ds):
    """The same ratings with the rows renumbered in descending degree order
    (ties by id): row i becomes its rank.  Test rows follow the training
    rows' numbering."""
    import dataclasses
    deg = np.bincount(ds.train_row, minlength=ds.M)
    order = np.argsort(-deg, kind="stable")
    new = np.empty(ds.M, np.int32)
    new[order] = np.arange(ds.M, dtype=np.int32)
    return dataclasses.replace(ds, train_row=new[ds.train_row], test_row=new[ds.test_row],
                               name=ds.name + " (rows in degree order)")


def algorithmic_work(ds, K):
    """Work of one half-sweep per side (the unit counts of the row update):
    Gram + right-hand side flops (nnz (K(K+1) + 2K)), Cholesky + solve flops
    (R (K^3/3 + 3K^2)) and bytes (ratings 8 B each, the other side's factors
    once, this side's factors written and its row pointers)."""
    nnz = ds.nnz
    out = {}
    for side, (R, C) in enumerate(((ds.M, ds.N), (ds.N, ds.M))):
        f_gram = nnz * (K * (K + 1) + 2 * K)
        f_chol = R * (K ** 3 / 3 + 3 * K ** 2)
        nbytes = nnz * 8 + C * 4 * K + R * (4 * K + 8)
        out[side] = (f_gram, f_chol, nbytes)
    return out


def measured_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "of measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, \
            "of fallback"


# ------------------------------------------------------------- GPU arms --

def device_arm(bp, ds, path, steps, warmup, world, stream, autotune=1, heavy=0, schedule=None):
    """Steady-state iterations with every input already in HBM."""
    import torch
    dev = torch.device("cuda")
    t = {k: torch.from_numpy(getattr(ds, k)).to(dev) for k in
         ("train_row", "train_col", "train_val", "test_row", "test_col", "test_val")}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = bp.Sampler(ds.M, ds.N, t["train_row"], t["train_col"], t["train_val"], K=ds.K,
                   alpha=ds.alpha, seed=0, path=path, stream=stream, autotune=autotune,
                   heavy_kernel=heavy)
    if schedule is not None:
        for side in (0, 1):
            s.set_thresholds(side, schedule[side])
    s.set_test(t["test_row"], t["test_col"], t["test_val"])
    torch.cuda.synchronize()
    init_s = time.perf_counter() - t0
    for _ in range(warmup):
        s.step()
    s.set_timing(True)
    barrier(world)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        s.step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = ev0.elapsed_time(ev1) / steps
    phase_ms, phase_cnt, kernels = s.timing()
    rmse = s.test_rmse()
    info = [s.sweep_info(0), s.sweep_info(1)]
    thresholds = [s.thresholds(0), s.thresholds(1)]
    s.close()
    del t
    torch.cuda.empty_cache()
    return dict(ms=ms, init_s=init_s, phase_ms=phase_ms, phase_cnt=phase_cnt, kernels=kernels,
                rmse=rmse, info=info, thresholds=thresholds)


def serving_arm(bp, n_jobs, iterations, seed=0):
    """The serving stream: independent jobs submitted at their Poisson arrival
    times to the continuous-batching server; latency = completion - arrival."""
    import synth
    import torch
    specs = synth.serving_stream(n_jobs, 20.0, seed)
    t0 = time.perf_counter()
    jobs = [synth.serving_job(sp, "cuda") for sp in specs]
    gen_s = time.perf_counter() - t0
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    with bp.Server() as srv:
        start = time.perf_counter()
        ids = []
        for sp, ds in zip(specs, jobs):
            delay = start + sp["arrival_s"] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            ids.append(srv.submit(ds.M, ds.N, ds.train_row, ds.train_col, ds.train_val, ds.K,
                                  iterations, test=(ds.test_row, ds.test_col, ds.test_val),
                                  alpha=ds.alpha, seed=sp["seed"], path=bp.PATH_MIXED))
        res = [srv.result(j)[0] for j in ids]
        st = srv.stats()
    ok = [r for r in res if r.status == 0]
    lat = sorted((r.t_end - r.t_submit) * 1e3 for r in ok)
    q = lambda f: lat[min(len(lat) - 1, int(math.ceil(f * len(lat))) - 1)] if lat else None
    span = max(r.t_end for r in ok) - min(r.t_submit for r in ok) if ok else float("nan")
    rows = sum((ds.M + ds.N) * r.iterations for ds, r in zip(jobs, res) if r.status == 0)
    return {"jobs": n_jobs, "completed": len(ok), "iterations": iterations,
            "rate_per_s": 20.0, "p50_ms": q(0.50), "p99_ms": q(0.99),
            "mean_ms": statistics.mean(lat) if lat else None,
            "rows_per_s": rows / span if ok else None, "makespan_s": span,
            "peak_resident": st["peak_resident"], "budget_gb": st["budget"] / 1e9,
            "peak_budgeted_gb": st["peak_bytes"] / 1e9, "generate_s": gen_s,
            "workload": "256 jobs, Poisson 20/s, rows log-U[1k,200k], cols log-U[1k,50k], "
                        "ratings log-U[10k,5M], K in {16,32,64}, mixed path"}


def e2e_arm(bp, ds, path, steps, stream, autotune=1):
    """A whole job through the C ABI from pinned host buffers: bpmf_init (H2D of
    the ratings, structure build), bpmf_set_test, `steps` iterations, then the
    factors and the RMSE back to the host."""
    import torch
    pin = {k: torch.from_numpy(getattr(ds, k)).pin_memory() for k in
           ("train_row", "train_col", "train_val", "test_row", "test_col", "test_val")}
    host = {k: v.numpy() for k, v in pin.items()}
    U = torch.empty((ds.M, ds.K), dtype=torch.float32).pin_memory().numpy()
    V = torch.empty((ds.N, ds.K), dtype=torch.float32).pin_memory().numpy()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    s = bp.Sampler(ds.M, ds.N, host["train_row"], host["train_col"], host["train_val"], K=ds.K,
                   alpha=ds.alpha, seed=1, path=path, stream=stream, autotune=autotune)
    s.set_test(host["test_row"], host["test_col"], host["test_val"])
    for _ in range(steps):
        s.step()
    s.get_state(U=U, V=V)
    rmse = s.test_rmse()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    s.close()
    h2d = sum(host[k].nbytes for k in host)
    d2h = U.nbytes + V.nbytes + 16
    return dict(ms=ms, rmse=rmse, h2d=h2d / steps, d2h=d2h / steps)


# ----------------------------------------------------------- CPU oracle --

def cpu_oracle_rate(ds, K, budget_s, seed=0):
    """Oracle rows/s on a bounded sample of one iteration of the workload.

    The oracle's hyper draw runs on every row of each side; the row draws run
    on uniform random samples of users and movies, sized to stay within the
    budget; predictions on a sample of the test set.  Each part is scaled by
    its sampling fraction to one full iteration."""
    import oracle
    rng = np.random.default_rng(seed)
    mu = oracle.mean(ds.train_val)
    csr = oracle.build_compressed(ds.M, ds.train_row, ds.train_col, ds.train_val, mu)
    csc = oracle.build_compressed(ds.N, ds.train_col, ds.train_row, ds.train_val, mu)
    U = rng.normal(size=(ds.M, K)) * 0.3
    V = rng.normal(size=(ds.N, K)) * 0.3
    prior = dict(mu0=np.zeros(K), beta0=2.0, nu0=float(K), W0=np.eye(K))
    parts = {}
    t_iter = 0.0
    rows_done = 0
    for side, (X, Xo, (ptr, idx, val)) in enumerate(((U, V, csr), (V, U, csc))):
        t0 = time.perf_counter()
        Lam, m = oracle.sample_hyper(X, prior, 0, 0, side)
        th = time.perf_counter() - t0
        R = X.shape[0]
        deg = np.diff(ptr)
        avg_cost = float(np.mean(deg)) * K * K + K ** 3 / 3.0
        # size the sample to about a third of the budget per side
        n = 16
        while True:
            sub = rng.choice(R, size=min(n, R), replace=False)
            Xs = X.copy() if side == 0 else X.copy()
            t0 = time.perf_counter()
            oracle.sweep(side, ptr, idx, val, Xo, Lam, m, ds.alpha, 0, 0, Xs, subset=sub)
            ts = time.perf_counter() - t0
            if ts > budget_s / 3 or n >= R:
                break
            n = int(min(R, n * max(2.0, 0.8 * (budget_s / 3) / max(ts, 1e-4))))
        per_row = ts / len(sub)
        parts[side] = dict(hyper_s=th, rows=len(sub), sweep_s=ts, est_sweep_s=per_row * R,
                           sampled_mean_degree=float(np.mean(deg[sub])), mean_degree=float(np.mean(deg)))
        t_iter += th + per_row * R
        rows_done += len(sub)
    nt = len(ds.test_row)
    ns = min(nt, 1_000_000)
    sel = rng.choice(nt, size=ns, replace=False)
    t0 = time.perf_counter()
    oracle.predict(ds.test_row[sel], ds.test_col[sel], U, V, mu)
    tp = (time.perf_counter() - t0) * nt / ns
    t_iter += tp
    rate = (ds.M + ds.N) / t_iter
    sample = (f"hyper draws on all rows; row draws on {parts[0]['rows']} random users and "
              f"{parts[1]['rows']} random movies; predictions on {ns} test pairs; scaled to one "
              f"iteration ({t_iter:.1f} s estimated)")
    return rate, sample, oracle.max_threads(), parts


def cpu_oracle_full_iteration(ds, K, seed=0):
    """One whole Gibbs iteration of the oracle, timed: hyperparameters and every
    row of the users, the same for the movies, then every test prediction
    (Algorithm 1's loop body, as oracle.Chain runs it)."""
    import oracle
    rng = np.random.default_rng(seed)
    mu = oracle.mean(ds.train_val)
    csr = oracle.build_compressed(ds.M, ds.train_row, ds.train_col, ds.train_val, mu)
    csc = oracle.build_compressed(ds.N, ds.train_col, ds.train_row, ds.train_val, mu)
    U = rng.normal(size=(ds.M, K)) * 0.3
    V = rng.normal(size=(ds.N, K)) * 0.3
    prior = dict(mu0=np.zeros(K), beta0=2.0, nu0=float(K), W0=np.eye(K))
    t0 = time.perf_counter()
    for side, (X, Xo, (ptr, idx, val)) in enumerate(((U, V, csr), (V, U, csc))):
        Lam, m = oracle.sample_hyper(X, prior, 0, 0, side)
        oracle.sweep(side, ptr, idx, val, Xo, Lam, m, ds.alpha, 0, 0, X)
    oracle.predict(ds.test_row, ds.test_col, U, V, mu)
    return time.perf_counter() - t0


# ----------------------------------------------------------------- main --

def main():
    args = parse()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    import torch
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        return reference_arm(args, world, rank)
    import paper_1705_04159_gb300 as bp
    bp.build()
    bp.lib()
    stream = torch.cuda.current_stream()
    ds = load_workload(args.workload, args.seed, "cuda")
    if args.relabel == "degree":
        ds = relabel_by_degree(ds)
    K = ds.K
    work = algorithmic_work(ds, K)
    main_path = {"mixed": bp.PATH_MIXED, "binned": bp.PATH_BINNED, "plain": bp.PATH_PLAIN}[args.path]
    schedule = None
    if args.thresholds:
        schedule = [tuple(int(x) for x in part.split(",")) for part in args.thresholds.split(";")]
        if len(schedule) != 2 or any(len(t) != 5 for t in schedule):
            raise SystemExit("--thresholds: 'users;movies', five integers each")

    with ClockSampler(local) as clk:
        mixed = device_arm(bp, ds, main_path, args.steps, args.warmup, world, stream,
                           autotune=args.autotune, heavy=args.heavy, schedule=schedule)
    clocks = clk.summary()
    ms = max_over_ranks(world, mixed["ms"])
    rows = ds.M + ds.N
    value = world * rows / (ms / 1e3)

    plain = None
    if not args.no_plain:
        # the same iteration count as the main arm, so that the test RMSEs compare
        p = device_arm(bp, ds, bp.PATH_PLAIN, args.steps, args.warmup, world, stream)
        pm = max_over_ranks(world, p["ms"])
        plain = {"value": world * rows / (pm / 1e3), "ms_per_step": pm,
                 "rows_users_ms": p["phase_ms"]["rows_users"] / max(1, p["phase_cnt"]["rows_users"]),
                 "rows_movies_ms": p["phase_ms"]["rows_movies"] / max(1, p["phase_cnt"]["rows_movies"]),
                 "rmse_mean": p["rmse"][1]}

    e2e = None
    if not args.no_e2e:
        e = e2e_arm(bp, ds, main_path, args.steps, stream, args.autotune)
        em = max_over_ranks(world, e["ms"])
        e2e = {"value": world * rows * args.steps / (em / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(e["h2d"]), "d2h_bytes_per_step": int(e["d2h"]),
               "job_ms": em, "iterations": args.steps}

    # dominant kernel: the row-update phase with the larger time per launch
    ph, pc = mixed["phase_ms"], mixed["phase_cnt"]
    per = {k: ph[k] / max(1, pc[k]) for k in ph}
    dom = max(("rows_users", "rows_movies"), key=lambda k: per[k])
    side = 0 if dom == "rows_users" else 1
    # the relevant bound: the slowest of the tensor-core Gram (bf16 peak), the
    # FP32 Cholesky and solves (FP32 peak) and the algorithmic bytes (HBM) when
    # most of the side's rows take a tensor-core kernel (heavy bin, kernel 1 or
    # 2); otherwise Gram and factorisations on the FP32 lanes.  Split-precision
    # and padding work not counted.
    peaks, peak_src = measured_peaks()
    f_gram, f_chol, nbytes = work[side]
    t_ms = per[dom]
    sm_mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
    fp32_peak, n_sms = fp32_peak_tflops(sm_mhz)
    bins = mixed["info"][side][0]
    tensor_gram = (args.path == "mixed" and mixed["thresholds"][side][3] in (1, 2)
                   and 2 * int(bins[2]) > int(sum(bins)))
    if tensor_gram:
        # the Gram on the tensor cores (bf16), the factorisations on the FP32 lanes
        terms = {"tensor": f_gram / (peaks["bf16_tflops"] * 1e12) * 1e3,
                 "alu": f_chol / (fp32_peak * 1e12) * 1e3,
                 "hbm": nbytes / (peaks["hbm_gbs"] * 1e9) * 1e3}
    else:
        # the FP32 paths run the Gram and the factorisations on the FP32 lanes
        terms = {"alu": (f_gram + f_chol) / (fp32_peak * 1e12) * 1e3,
                 "hbm": nbytes / (peaks["hbm_gbs"] * 1e9) * 1e3}
    bound = max(terms, key=terms.get)
    if bound == "hbm":
        achieved, peak, unit = nbytes / (t_ms / 1e3) / 1e9, peaks["hbm_gbs"], "GB/s"
    elif bound == "tensor":
        achieved, peak, unit = f_gram / (t_ms / 1e3) / 1e12, peaks["bf16_tflops"], "TFLOP/s"
    else:
        flops = f_chol if tensor_gram else f_gram + f_chol
        achieved, peak, unit = flops / (t_ms / 1e3) / 1e12, fp32_peak, "TFLOP/s"
    key = (args.workload, side, mixed["thresholds"][side][3], mixed["thresholds"][side][4])
    traffic, traffic_note = TRAFFIC.get(key, (None, "no ncu capture of this kernel version"))
    roofline = {"kernel": f"row update, {'users' if side == 0 else 'movies'} side"
                          f" ({'tensor-core Gram' if tensor_gram else 'FP32 Gram'})",
                "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "traffic": traffic, "traffic_note": traffic_note,
                "peak_note": (f"alu: FP32 CUDA-core peak from unit counts ({n_sms} SMs x "
                              f"{FP32_LANES_PER_SM} lanes x 2 flop x {sm_mhz:.0f} MHz, the median "
                              f"SM clock sampled under load); tensor and hbm {peak_src} "
                              f"(bf16 burst, copy)"),
                "roofline_ms": terms, "ms_per_launch": t_ms,
                "gram_flops_per_launch": f_gram, "chol_flops_per_launch": f_chol,
                "algorithmic_bytes_per_launch": nbytes}

    serving = None
    if not args.no_serving:
        serving = serving_arm(bp, args.serving_jobs, args.serving_iters, seed=args.seed)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, sample, cores, parts = cpu_oracle_rate(ds, K, args.cpu_budget)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
        if not args.no_cpu_full:
            t_full = cpu_oracle_full_iteration(ds, K)
            cpu["full_iteration"] = {"s": t_full, "value": (ds.M + ds.N) / t_full,
                                     "what": "one whole iteration timed: both hyper draws, every "
                                             "row of both sides, every test prediction"}
            cpu["value"] = (ds.M + ds.N) / t_full
            cpu["sample"] = ("one whole iteration of the workload, timed (the bounded-sample "
                             f"estimate beside it: {rate:.4g} rows/s from {sample})")

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": ("f32 (Gram of heavy rows: bf16 hi/lo split, 3 tensor-core products, f32 "
                      "accumulation; Cholesky and solves f32; FP64 redo of flagged rows)"
                      if args.path == "mixed" else "f32"),
            "data": f"synthetic (seeded {ds.name}-shaped ratings generated on the device)",
            "config": {"workload": f"{ds.name}: {ds.M}x{ds.N}, {ds.nnz} train + "
                                   f"{len(ds.test_row)} test ratings, K={K}",
                       "path": args.path, "global_batch": rows, "parallelism": f"replicas{world}",
                       "l2": "no flush: per-iteration working set > 1.4 GB vs 129 MB L2"},
            "clocks": clocks, "gpu_launches": int(mixed["kernels"]),
            "phase_ms_per_step": {k: v / args.steps for k, v in ph.items()},
            "init_s": mixed["init_s"], "rmse": {"sample": mixed["rmse"][0], "mean": mixed["rmse"][1]},
            "bins": {"users": mixed["info"][0][0].tolist(), "movies": mixed["info"][1][0].tolist(),
                     "fp64_rows": [mixed["info"][0][1], mixed["info"][1][1]],
                     "thresholds_tiny_light_hub": mixed["thresholds"],
                     "autotune": ("set by --thresholds" if schedule is not None else
                                  "on: timed at the first init (init_s), reused from the "
                                  "process cache by the e2e job" if args.autotune else "off")},
            "plain_fp32": plain, "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu,
            "serving": serving,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


class OracleSteps:
    """Bounded steps of the oracle on one workload.  A step draws both sides'
    hyperparameters from all their rows, redraws n_users random users and
    n_movies random movies, and predicts n_test random test pairs; it counts
    the rows it redrew.  The compressed structure is built once, outside the
    steps (it is the initialisation, not part of an iteration)."""

    def __init__(self, ds, K):
        import oracle
        self.o, self.ds, self.K = oracle, ds, K
        self.mu = oracle.mean(ds.train_val)
        self.csr = oracle.build_compressed(ds.M, ds.train_row, ds.train_col, ds.train_val,
                                           self.mu)
        self.csc = oracle.build_compressed(ds.N, ds.train_col, ds.train_row, ds.train_val,
                                           self.mu)
        rng = np.random.default_rng(1)
        self.U = rng.normal(size=(ds.M, K)) * 0.3
        self.V = rng.normal(size=(ds.N, K)) * 0.3
        self.prior = dict(mu0=np.zeros(K), beta0=2.0, nu0=float(K), W0=np.eye(K))

    def sizes(self, frac):
        """Row and test-pair counts of a step covering `frac` of an iteration."""
        ds = self.ds
        return (max(1, int(ds.M * frac)), max(1, int(ds.N * frac)),
                max(1, int(len(ds.test_row) * frac)) if len(ds.test_row) else 0)

    def step(self, frac, seed):
        """(seconds, rows redrawn) of one step covering `frac` of an iteration."""
        o, ds = self.o, self.ds
        n_u, n_v, n_t = self.sizes(frac)
        rng = np.random.default_rng(seed)
        subs = (rng.choice(ds.M, size=n_u, replace=False),
                rng.choice(ds.N, size=n_v, replace=False))
        tsel = rng.choice(len(ds.test_row), size=n_t, replace=False) if n_t else None
        t0 = time.perf_counter()
        for side, (X, Xo, (ptr, idx, val)) in enumerate(((self.U, self.V, self.csr),
                                                         (self.V, self.U, self.csc))):
            Lam, m = o.sample_hyper(X, self.prior, 0, seed, side)
            o.sweep(side, ptr, idx, val, Xo, Lam, m, ds.alpha, 0, seed, X, subset=subs[side])
        if n_t:
            o.predict(ds.test_row[tsel], ds.test_col[tsel], self.U, self.V, self.mu)
        return time.perf_counter() - t0, n_u + n_v


def reference_arm(args, world, rank):
    """The FP64 CPU oracle as the reference arm.  Every step is a bounded
    sample of one iteration of the workload (OracleSteps), timed as it runs:
    ms_per_step is the measured time of a step and value the rows it redrew
    per second, so ms_per_step x steps is the timed part of the run."""
    if rank != 0:
        return
    ds = load_workload(args.workload, args.seed, "cuda" if _cuda() else "cpu")
    K = ds.K
    steps = OracleSteps(ds, K)
    # the fraction of an iteration one step covers: about --cpu-budget seconds
    # (less when many steps are asked for, so that the run stays within a few
    # minutes), sized from a short calibration step
    per_step = min(args.cpu_budget, max(2.0, 150.0 / max(1, args.steps)))
    f = min(1.0, 200.0 / max(1, ds.M + ds.N))
    t, _ = steps.step(f, seed=997)
    f = min(1.0, f * max(1.0, per_step / max(t, 1e-3)))
    for w in range(args.warmup):
        steps.step(f, seed=1000 + w)
    times, rows = [], 0
    t0 = time.perf_counter()
    for k in range(args.steps):
        dt, n = steps.step(f, seed=k)
        times.append(dt)
        rows += n
    elapsed = time.perf_counter() - t0
    value = rows / sum(times)
    n_u, n_v, n_t = steps.sizes(f)
    import oracle
    sample = (f"each step: hyper draws of both sides on all rows, row draws of {n_u} random users "
              f"and {n_v} random movies, predictions of {n_t} random test pairs "
              f"({f:.3%} of an iteration's rows); value = rows redrawn / step seconds")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": f"synthetic (seeded {ds.name}-shaped ratings)",
            "config": {"workload": f"{ds.name}: {ds.M}x{ds.N}, {ds.nnz} train ratings, K={K}",
                       "global_batch": n_u + n_v, "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": elapsed}
    print(json.dumps(line))


def _cuda():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


if __name__ == "__main__":
    main()
