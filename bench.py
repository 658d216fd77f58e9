#!/usr/bin/env python
"""Benchmark of the truncated-Newton EOT solver on one GB300.

Workload (a synthetic stand-in for the paper's upsampled-MNIST problems, Sec. 4.1,
Table 1): a 64 x 64 grid, n = m = 4096, two Gaussian-mixture histograms with 10%
of the bins zeroed, squared-Euclidean grid cost with max 1 stored as FP32 in HBM
(64 MiB), gamma annealed from 2^4 to 2^14 (Alg. 1 with adaptive q), mixed
precision, solved until the marginal L1 error of the output is <= 1e-6.

One step = one full eot_solve (every row of the hot path: exponent formation,
exp, row and column sweeps, HVP assembly, PCG, Jacobi diagonal, the NewtonSolve
outer test and the LSE sweeps). value = mean time per solve (time-to-1e-6).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --impl reference the FP64 numpy oracle is timed on the host cores instead
(see cpu_sample below); it never touches the GPU.
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
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time-to-1e-6 marginal L1 error, mixed vs plain FP32 on 1 GB300; P-entries/s"
GAMMA_I, GAMMA_F, TOL = 16.0, 16384.0, 1e-6
N = 4096
WORKLOAD = "grid64x64_sqeuclid_f32_n4096_gamma2^14"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2


def bench_config(args, world):
    """The workload both arms report on (identical keys in both lines)."""
    return {"workload": WORKLOAD, "n": N, "m": N, "gamma_i": GAMMA_I, "gamma_f": GAMMA_F, "tol": TOL,
            "cost": args.cost, "parallelism": "replicas" if world > 1 else "single",
            "l2": "flushed between steps (512 MiB write)"}


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle as it stands, timed on a bounded sample
# ---------------------------------------------------------------------------

def oracle_ops_of_workload():
    """The oracle's own operation counts on this workload, from its recorded run
    (tests/golden/grid4096_oracle_trace.json, written by calling oracle/ only). In
    the oracle every stage makes a column and a row LSE update, every Newton step
    forms the plan once and makes a row LSE update, every line-search trial a
    column LSE, every ChiSinkhorn iteration two LSE updates; the outer tests of
    NewtonSolve and d_v are matrix-vector products on the stored plan, as are the
    CG steps."""
    tr = json.load(open(os.path.join(ROOT, "tests", "golden", "grid4096_oracle_trace.json")))
    t = tr["sqeuclid"]
    lse_like = 2 * t["stages"] + 2 * t["newton_steps"] + t["ls_trials"] + 2 * t["sinkhorn_iters"]
    cg_like = t["cg_iters"] + 2 * t["newton_steps"]
    return {"lse_like": lse_like, "cg_like": cg_like, "recorded_seconds": t.get("oracle_seconds"),
            "source": "tests/golden/grid4096_oracle_trace.json"}


def oracle_sample(seconds):
    """Times the oracle's two primitive operations on the full-size workload with
    numpy's default threading (BLAS on every host core; numpy's elementwise exp
    is single-threaded): one O(n^2) log-sum-exp update (plan formation and a
    reduction, as in each of the oracle's LSE updates) and one CG step on a stored
    plan (F_r(rho) applied: two matrix-vector products). Returns seconds per op."""
    import numpy as np

    import workloads as W
    from oracle import eot_oracle as O

    p = W.grid_problem_4096(0, "sqeuclid")
    C = p["C"].astype(np.float64)
    g = GAMMA_F
    u = np.log(p["r"] + 1e-9)
    v = np.log(p["c"] + 1e-9) - O.lse_c(u[:, None] - g * C)
    t0 = time.perf_counter()
    k_lse = 0
    while time.perf_counter() - t0 < seconds / 2 or k_lse < 2:
        O.log_row_sum(u, v, g, C)
        k_lse += 1
    t_lse = (time.perf_counter() - t0) / k_lse
    P = O.plan(u, v, g, C)
    x = np.random.default_rng(0).normal(size=N)
    t1 = time.perf_counter()
    k_cg = 0
    while time.perf_counter() - t1 < seconds / 2 or k_cg < 2:
        O.F_r_apply(P, 0.9, x)
        k_cg += 1
    t_cg = (time.perf_counter() - t1) / k_cg
    return {"t_lse": t_lse, "t_cg": t_cg, "k_lse": k_lse, "k_cg": k_cg,
            "wall": time.perf_counter() - t0}


def oracle_estimate(sample, ops):
    """The oracle's time for one solve of the workload: its recorded operation
    counts priced at the sampled per-operation times."""
    return ops["lse_like"] * sample["t_lse"] + ops["cg_like"] * sample["t_cg"]


def cpu_cores():
    return os.cpu_count() or 1


def cpu_sample_text(sample, ops):
    return ("oracle log_row_sum x%d (%.4f s each) and F_r_apply x%d (%.5f s each) at n = 4096, "
            "BLAS on %d host threads; one solve = the oracle's recorded %d LSE updates and %d "
            "CG-step products (%s) at those times"
            % (sample["k_lse"], sample["t_lse"], sample["k_cg"], sample["t_cg"], cpu_cores(),
               ops["lse_like"], ops["cg_like"], ops["source"]))


def oracle_full_solve_seconds():
    """One complete oracle solve of the workload (measured, not estimated)."""
    import numpy as np

    import workloads as W
    from oracle import eot_oracle as O
    p = W.grid_problem_4096(0, "sqeuclid")
    C = p["C"].astype(np.float64)
    t0 = time.perf_counter()
    res = O.mdot(C, p["r"], p["c"], gamma_i=GAMMA_I, gamma_f=GAMMA_F, tol_final=TOL)
    return time.perf_counter() - t0, res


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def max_over_ranks(value, world, device=None):
    """The job's time is the slowest rank's: MAX all-reduce of one float over the
    process group (identity for a single process)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def replica_seed(rank):
    """Replicas only: every rank solves its own problem of the workload, seeded by its rank."""
    return rank


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def traffic_record():
    """DRAM bytes per launch of the CG sweeps from the committed ncu summary, valid
    only while the sweep source is unchanged (hash recorded with the numbers)."""
    path = os.path.join(ROOT, "profiles", "cg_sweeps_grid4096_traffic.txt")
    try:
        rec = {"dram_bytes_per_launch": {}}
        for line in open(path):
            parts = line.split()
            if len(parts) == 2 and not line.startswith("#"):
                if parts[0] == "sweep_cuh_sha256_16":
                    rec[parts[0]] = parts[1]
                else:
                    rec["dram_bytes_per_launch"][parts[0]] = int(parts[1])
    except Exception:
        return None
    h = hashlib.sha256(open(os.path.join(ROOT, "paper_2504_02067_gb300", "csrc", "sweep.cuh"),
                            "rb").read()).hexdigest()[:16]
    return rec if rec.get("sweep_cuh_sha256_16") == h else None


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def roofline_at_scale(h, E, dev, flush, peak, side=128):
    """The same CG sweep kernels on a 128 x 128 grid (n = m = 16384, 1 GiB FP32
    squared-Euclidean cost made on the device, larger than L2): one pass per
    launch from HBM, each launch timed alone after the L2 overwrite."""
    import torch
    n = side * side
    g = torch.arange(side, dtype=torch.float32, device=dev) / (side - 1)
    px = g.repeat_interleave(side)
    py = g.repeat(side)
    C = ((px[:, None] - px[None, :]) ** 2 + (py[:, None] - py[None, :]) ** 2) * 0.5
    w = torch.full((n,), 1.0 / n, dtype=torch.float64, device=dev)
    prob = E.Problem(C, w, w, precision="mixed")
    gen = torch.Generator(device="cpu").manual_seed(0)
    u = (torch.full((n,), -math.log(n), dtype=torch.float64)
         + 0.1 * torch.randn(n, generator=gen, dtype=torch.float64)).to(dev)
    v = torch.full((n,), -math.log(n), dtype=torch.float64, device=dev)
    nbytes = n * n * 4
    out = {"workload": "grid128x128_sqeuclid_f32_n16384_gamma2^10", "bytes_per_launch": nbytes}
    for kind, name in ((0, "cg_col_sweep"), (1, "cg_row_sweep")):
        ms = h.eot_sweep_bench(prob, u, v, 1024.0, kind, 5, flush=flush)
        gbs = nbytes / (ms * 1e-3) / 1e9
        out[name] = {"us": round(ms * 1e3, 2), "achieved": round(gbs, 1), "frac": round(gbs / peak, 4)}
    del C
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# sub-records of the other workloads (driver-visible: they ride on the default
# run's JSON line; each takes seconds)
# ---------------------------------------------------------------------------

MUFU_PER_CLK_SM = 16     # ex2 results per clock per SM (4 per SM sub-partition)
FP32_LANES_SM = 128      # FP32 lanes per SM
SM_MAX_GHZ = 2.07


def _event_time(fn, stream=None):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3, out


def _solve_record(h, E, prob, prm, n, m, warm=1, reps=1):
    import torch
    u = torch.empty(n, dtype=torch.float64, device="cuda")
    v = torch.empty(m, dtype=torch.float64, device="cuda")
    for _ in range(warm):
        h.eot_solve(prob, prm, u, v)
    ts = []
    for _ in range(reps):
        t, st = _event_time(lambda: h.eot_solve(prob, prm, u, v).as_dict())
        ts.append(t)
    sec = statistics.mean(ts)
    return {"seconds": round(sec, 5), "marg_err_l1": st["marg_err_l1"], "reached_tol": st["marg_err_l1"] <= TOL,
            "stages": st["stages"], "newton_steps": st["newton_steps"], "cg_iters": st["cg_iters"],
            "sweeps_total": st["sweeps_total"],
            "p_entries_per_s": round(st["sweeps_total"] * n * m / sec, 1)}, u, v


def record_cfg1_fp64(E, dev):
    """28 x 28 grid (n = m = 784), 3-Gaussian histograms, squared-Euclidean cost,
    FP64 throughout (the paper's precision), gamma 2^4 -> 2^12, tol 1e-6."""
    import torch
    import workloads as W
    p = W.grid_problem_784(0)
    h = E.Handle(0, 784, 784)
    try:
        prob = E.Problem(torch.from_numpy(p["C"]).to(dev), torch.from_numpy(p["r"]).to(dev),
                         torch.from_numpy(p["c"]).to(dev), precision="fp64")
        prm = E.default_params(gamma_i=16.0, gamma_f=4096.0, tol_final=TOL)
        rec, _, _ = _solve_record(h, E, prob, prm, 784, 784, warm=1, reps=3)
    finally:
        h.close()
    rec["workload"] = "grid28x28_sqeuclid_f64_n784_gamma2^12"
    return rec


def record_cfg2_breadth(E, dev):
    """The 64 x 64 grid workload with both costs (squared Euclidean and L1) and
    seeds 0, 1, 2, mixed precision, gamma 2^4 -> 2^14, tol 1e-6."""
    import torch
    import workloads as W
    h = E.Handle(0, N, N)
    out = []
    try:
        prm = E.default_params(gamma_i=GAMMA_I, gamma_f=GAMMA_F, tol_final=TOL)
        for kind in ("sqeuclid", "l1"):
            for seed in (0, 1, 2):
                p = W.grid_problem_4096(seed, kind)
                prob = E.Problem(torch.from_numpy(p["C"]).to(dev), torch.from_numpy(p["r"]).to(dev),
                                 torch.from_numpy(p["c"]).to(dev), precision="mixed")
                rec, _, _ = _solve_record(h, E, prob, prm, N, N, warm=1, reps=1)
                rec.update({"cost": kind, "seed": seed})
                out.append(rec)
    finally:
        h.close()
    return {"workload": "grid64x64_f32_n4096_gamma2^14 (3 seeds x 2 costs)", "solves": out,
            "all_reached": all(r["reached_tol"] for r in out)}


def record_next3(E, dev, alg2_seconds, alg2_sweeps):
    """The full-system NewtonSolve (PCG on the (n + m) discounted Hessian, one
    two-sided sweep per iteration) on the headline workload, measured against
    Alg. 2's reduced system (the headline solve)."""
    import torch
    import workloads as W
    p = W.grid_problem_4096(0, "sqeuclid")
    h = E.Handle(0, N, N)
    try:
        prob = E.Problem(torch.from_numpy(p["C"]).to(dev), torch.from_numpy(p["r"]).to(dev),
                         torch.from_numpy(p["c"]).to(dev), precision="mixed")
        prm = E.default_params(gamma_i=GAMMA_I, gamma_f=GAMMA_F, tol_final=TOL, newton_system=E.NEWTON_FULL)
        rec, _, _ = _solve_record(h, E, prob, prm, N, N, warm=1, reps=2)
    finally:
        h.close()
    rec.update({"system": "full (n + m) discounted Hessian", "vs_alg2_time": round(rec["seconds"] / alg2_seconds, 4),
                "vs_alg2_sweeps": round(rec["sweeps_total"] / alg2_sweeps, 4)})
    return rec


def record_d64(E, dev, peaks):
    """n = m = 16384 points in d = 64 (8-component mixtures), gamma 2^4 -> 2^10,
    tol 1e-6: the mixed path (tensor-core sweeps) against the plain FP32 comparator
    on the same points. The comparator runs with max_newton = 10 per stage (a
    bound on the benchmark's wall time); when a cap stops it, its floor is the
    marginal L1 error of the last iterate, evaluated by eot_marginals on the mixed
    path (accurate to about 1e-7)."""
    import numpy as np
    import torch
    import workloads as W
    p = W.gmm_problem_d64(0)
    n = p["X"].shape[0]
    X, Y = torch.from_numpy(p["X"]).to(dev), torch.from_numpy(p["Y"]).to(dev)
    r, c = torch.from_numpy(p["r"]).to(dev), torch.from_numpy(p["c"]).to(dev)
    gf = 1024.0
    h = E.Handle(0, n, n, 64)
    out = {"workload": "gmm8_d64_n16384_gamma2^10", "n": n, "d": 64, "gamma_f": gf, "tol": TOL}
    try:
        prob = E.Problem(X=X, Y=Y, r=r, c=c, precision="mixed", cost_scale=0.0)
        prm = E.default_params(gamma_i=16.0, gamma_f=gf, tol_final=TOL)
        mixed, u, v = _solve_record(h, E, prob, prm, n, n, warm=1, reps=2)
        out["mixed"] = mixed
        # sweep rates of the tensor-core kernels at the solution
        rates = {}
        for kind, name in ((0, "cg_col_sweep"), (1, "cg_row_sweep"), (3, "row_lse_sweep")):
            ms = h.eot_sweep_bench(prob, u, v, gf, kind, 5)
            rates[name] = {"ms": round(ms, 4), "p_entries_per_s": round(n * n / (ms * 1e-3), 1)}
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        bf16 = (peaks or {}).get("bf16_tflops", 1900.0) * 1e12
        flop_per_entry = 15 * 2 * 64           # 15 digit-slice BF16 MMAs of K = 64 per entry
        fp32_issue = sms * FP32_LANES_SM * SM_MAX_GHZ * 1e9
        ex2 = sms * MUFU_PER_CLK_SM * SM_MAX_GHZ * 1e9
        best = max(rates["cg_col_sweep"]["p_entries_per_s"], rates["cg_row_sweep"]["p_entries_per_s"])
        out["tc_sweeps"] = rates
        out["tc_roofline"] = {
            "bound": "tensor", "kernel": "tc_sweep_kernel (CG halves)", "achieved_entries_per_s": best,
            "frac": round(best / (bf16 / flop_per_entry), 4),
            "peak_tensor_entries_per_s": round(bf16 / flop_per_entry, 1),
            "peak_ex2_entries_per_s": round(ex2, 1),
            "fp32_issue_per_s": round(fp32_issue, 1),
            "frac_of_tensor": round(best / (bf16 / flop_per_entry), 4),
            "frac_of_ex2": round(best / ex2, 4),
            "peak_source": "tensor: measured bf16 burst (MEASURED_PEAKS.json) / %d flop per entry; ex2 and "
                           "FP32 issue: %d SMs x %d ex2 / %d lanes per clock x %.2f GHz" %
                           (flop_per_entry, sms, MUFU_PER_CLK_SM, FP32_LANES_SM, SM_MAX_GHZ)}
        # the plain FP32 comparator on the same points
        probp = E.Problem(X=X, Y=Y, r=r, c=c, precision="plain_fp32", cost_scale=0.0)
        prmp = E.default_params(gamma_i=16.0, gamma_f=gf, tol_final=TOL, max_newton=10)
        up = torch.empty(n, dtype=torch.float64, device=dev)
        vp = torch.empty(n, dtype=torch.float64, device=dev)
        t0 = time.perf_counter()
        try:
            stp = h.eot_solve(probp, prmp, up, vp).as_dict()
            status = "EOT_OK"
        except E.EotError as ex:
            stp, status = getattr(ex, "stats", None), str(ex).split(":")[0]
        torch.cuda.synchronize()
        tp = time.perf_counter() - t0
        g_last = stp["final_gamma"] if stp else float(np.float32(gf))
        rr, cc, _, _, _ = h.marginals(prob, up, vp, g_last)
        floor = float((rr - r).abs().sum() + (cc - c).abs().sum())
        out["plain_fp32"] = {"status": status, "seconds": round(tp, 3), "stopped_at_gamma": g_last,
                             "marg_err_l1_last_iterate": floor,
                             "reached_tol": status == "EOT_OK" and floor <= TOL, "max_newton": 10,
                             "stats": ({k: stp[k] for k in ("stages", "newton_steps", "cg_iters", "grad_l1")}
                                       if stp else None)}
        out["mixed_faster_to_1e-6"] = bool(mixed["reached_tol"] and not out["plain_fp32"]["reached_tol"])
    finally:
        h.close()
    return out


def record_batch256(E, dev):
    """256 point problems (n = m uniform in [256, 4096], uniform points in the unit
    square, Dirichlet(1) weights), gamma 2^4 -> 2^12, mixed, tol 1e-6, one
    eot_solve_batched launch (autotuned on the first call)."""
    import numpy as np
    import torch
    import workloads as W
    sizes = W.batch_sizes(0)
    ps = [W.uniform_points_problem(1000 + k, int(nk)) for k, nk in enumerate(sizes)]
    devs = [{k: torch.from_numpy(p[k]).to(dev) for k in ("X", "Y", "r", "c")} for p in ps]
    probs = [E.Problem(X=d["X"], Y=d["Y"], r=d["r"], c=d["c"], precision="mixed", cost_scale=0.0) for d in devs]
    us = [torch.empty(int(nk), dtype=torch.float64, device=dev) for nk in sizes]
    vs = [torch.empty(int(nk), dtype=torch.float64, device=dev) for nk in sizes]
    h = E.Handle(0, 64, 64)
    try:
        prm = E.default_params(gamma_i=16.0, gamma_f=4096.0, tol_final=TOL)
        t_first = time.perf_counter()
        h.eot_solve_batched(probs, prm, us, vs)
        t_first = time.perf_counter() - t_first
        sec, (st, stats) = _event_time(lambda: h.eot_solve_batched(probs, prm, us, vs))
        G, ro, groups = h.batch_last_config()
    finally:
        h.close()
    entries = sum(sm["sweeps_total"] * int(nk) * int(nk) for sm, nk in zip(stats, sizes))
    return {"workload": "batch256_uniform2d_n256-4096_gamma2^12", "seconds": round(sec, 4),
            "all_ok": all(x == 0 for x in st), "max_marg_err_l1": max(sm["marg_err_l1"] for sm in stats),
            "p_entries_per_s": round(entries / sec, 1), "first_call_incl_autotune_s": round(t_first, 3),
            "sum_n2": int(np.sum(sizes.astype(np.int64) ** 2)),
            "batch_config": {"ctas_per_group": G, "elements_per_thread": ro, "groups": groups}}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2504_02067_gb300 as E
    import workloads as W

    E.build()
    dev = torch.device("cuda", local)
    p = W.grid_problem_4096(replica_seed(rank), args.cost)
    C_h = torch.from_numpy(p["C"]).pin_memory()
    r_h = torch.from_numpy(p["r"]).pin_memory()
    c_h = torch.from_numpy(p["c"]).pin_memory()
    C, r, c = C_h.to(dev), r_h.to(dev), c_h.to(dev)
    h = E.Handle(local, N, N)
    prm = E.default_params(gamma_i=GAMMA_I, gamma_f=GAMMA_F, tol_final=TOL)
    prob = E.Problem(C, r, c, precision="mixed")
    u = torch.empty(N, dtype=torch.float64, device=dev)
    v = torch.empty(N, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        h.eot_solve(prob, prm, u, v)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timed region ----
    sampler = ClockSampler(local)
    barrier()
    launches0 = h.launches()
    sampler.start()
    times, stats = [], []
    for _ in range(args.steps):
        flush.zero_()  # evict the 64 MiB cost from L2 between steps (not timed)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = h.eot_solve(prob, prm, u, v)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        stats.append(st.as_dict())
    barrier()
    clocks = sampler.stop()
    launches = h.launches() - launches0
    total = max_over_ranks(sum(times), world, dev)
    sec = total / args.steps
    last = stats[-1]
    sweeps = last["sweeps_total"]
    p_entries_per_s = sweeps * N * N / (sum(times) / args.steps)

    # ---- end to end through the public API, host buffers ----
    u_h = torch.empty(N, dtype=torch.float64).pin_memory()
    v_h = torch.empty(N, dtype=torch.float64).pin_memory()
    barrier()
    e_times = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        C.copy_(C_h, non_blocking=True)
        r.copy_(r_h, non_blocking=True)
        c.copy_(c_h, non_blocking=True)
        h.eot_solve(prob, prm, u, v)
        u_h.copy_(u, non_blocking=True)
        v_h.copy_(v, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e_times.append(e0.elapsed_time(e1) / 1e3)
    e2e = max_over_ranks(sum(e_times) / len(e_times), world, dev)

    # ---- roofline of the dominant kernels (CG column / row halves) ----
    # ms_hbm: each launch timed alone right after a 512 MiB overwrite (the cost
    # comes from HBM); ms_l2warm: back-to-back launches (the cost stays in L2, as
    # inside a solve)
    bytes_per_launch = N * N * 4  # the FP32 cost streamed once per sweep (vectors are O(n))
    kern = {}
    for kind, name in ((0, "cg_col_sweep"), (1, "cg_row_sweep")):
        cold = h.eot_sweep_bench(prob, u, v, GAMMA_F, kind, 10, flush=flush)
        warm = h.eot_sweep_bench(prob, u, v, GAMMA_F, kind, 50)
        kern[name] = {"ms_hbm": cold, "ms_l2warm": warm}
    dom = max(kern, key=lambda k: kern[k]["ms_l2warm"])
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    ach = bytes_per_launch / (kern[dom]["ms_hbm"] * 1e-3) / 1e9
    tr = traffic_record()
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(ach, 1), "peak": peak,
                "unit": "GB/s", "frac": round(ach / peak, 4),
                "traffic": tr["dram_bytes_per_launch"].get(dom) if tr else None,
                "peak_source": "measured" if peaks else "fallback",
                "algorithmic_bytes_per_launch": bytes_per_launch,
                "achieved_l2warm": round(bytes_per_launch / (kern[dom]["ms_l2warm"] * 1e-3) / 1e9, 1),
                "sweeps_us": {k: {kk: round(vv * 1e3, 2) for kk, vv in d.items()} for k, d in kern.items()},
                "at_scale": roofline_at_scale(h, E, dev, flush, peak)}

    # ---- plain FP32 comparator (same workload, same tolerance) ----
    # When a cap stops it, eot_solve leaves its last iterate in (u, v): its marginal
    # L1 error, evaluated on the mixed path (about 1e-7 accurate), is the floor.
    plain = None
    if not args.no_plain:
        prob_p = E.Problem(C, r, c, precision="plain_fp32")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            stp = h.eot_solve(prob_p, prm, u, v).as_dict()
            status = "EOT_OK"
        except E.EotError as ex:
            stp, status = getattr(ex, "stats", None), str(ex)[:160]
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        g_last = stp["final_gamma"] if stp else GAMMA_F
        rr, cc, _, _, _ = h.marginals(prob, u, v, g_last)
        floor = float((rr - r).abs().sum() + (cc - c).abs().sum())
        plain = {"seconds": round(secs, 3), "status": status, "stopped_at_gamma": g_last,
                 "marg_err_l1_last_iterate": floor, "reached": status == "EOT_OK" and floor <= TOL,
                 "note": "marginal L1 error of the last iterate at the temperature of the stage it stopped in"}

    # ---- Round (Alg. 1's closing step) of the last solve's plan ----
    h.eot_solve(prob, prm, u, v)
    flush.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rcost, rcorr = h.eot_round(prob, u, v, GAMMA_F)
    e1.record(stream)
    e1.synchronize()
    rounded = {"transport_cost": rcost, "correction_l1": rcorr,
               "ms": round(e0.elapsed_time(e1), 3)}

    # ---- MDOT-Sinkhorn on the same problem (Sec. 4's comparison method) ----
    mdot_sk = None
    if not args.no_sinkhorn:
        prm_sk = E.default_params(gamma_i=GAMMA_I, gamma_f=GAMMA_F, tol_final=TOL,
                                  projector=E.PROJECT_SINKHORN)
        h.eot_solve(prob, prm_sk, u, v)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sk = h.eot_solve(prob, prm_sk, u, v).as_dict()
        e1.record(stream)
        e1.synchronize()
        sk_sec = e0.elapsed_time(e1) / 1e3
        mdot_sk = {"seconds": round(sk_sec, 5), "marg_err_l1": sk["marg_err_l1"],
                   "reached_tol": sk["marg_err_l1"] <= TOL, "stages": sk["stages"],
                   "sinkhorn_iters": sk["sinkhorn_iters"], "sweeps_total": sk["sweeps_total"],
                   "newton_over_sinkhorn_time": round(sec / sk_sec, 4),
                   "newton_over_sinkhorn_sweeps": round(sweeps / sk["sweeps_total"], 4)}
        # plain Sinkhorn at gamma_f (MDOT-Sinkhorn with gamma_i = gamma_f, Sec. 4),
        # capped at 200000 iterations
        prm_pl = E.default_params(gamma_i=GAMMA_F, gamma_f=GAMMA_F, tol_final=TOL,
                                  projector=E.PROJECT_SINKHORN, max_sinkhorn=200000)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        try:
            pl = h.eot_solve(prob, prm_pl, u, v).as_dict()
            e1.record(stream)
            e1.synchronize()
            mdot_sk["plain_sinkhorn_gamma_f"] = {
                "seconds": round(e0.elapsed_time(e1) / 1e3, 4), "sinkhorn_iters": pl["sinkhorn_iters"],
                "marg_err_l1": pl["marg_err_l1"], "reached_tol": pl["marg_err_l1"] <= TOL}
        except E.EotError as ex:
            e1.record(stream)
            e1.synchronize()
            mdot_sk["plain_sinkhorn_gamma_f"] = {
                "seconds": round(e0.elapsed_time(e1) / 1e3, 4), "reached_tol": False,
                "error": str(ex)[:120]}

    extra = {}
    if not args.no_extra and world == 1:
        for key, fn in (("cfg1_fp64", lambda: record_cfg1_fp64(E, dev)),
                        ("cfg2_breadth", lambda: record_cfg2_breadth(E, dev)),
                        ("next3_full_system", lambda: record_next3(E, dev, sec, sweeps)),
                        ("d64", lambda: record_d64(E, dev, measured_peaks())),
                        ("batch256", lambda: record_batch256(E, dev))):
            try:
                extra[key] = fn()
            except Exception as ex:  # a sub-record never hides the headline line
                extra[key] = {"error": str(ex)[:200]}
            torch.cuda.empty_cache()

    result = None
    if rank == 0:
        # Table 1's shape (operations per subroutine) and Fig. 1's (delta_min and q per
        # stage) from the solver's own counters, on this synthetic workload
        fixed = last["sweeps_cg"] + last["sweeps_newton"] + last["sweeps_linesearch"] + \
            last["sweeps_sinkhorn"] + last["sweeps_stage"]
        op_breakdown = {
            "unit": "O(nm) sweeps (fused passes over the implicit plan)",
            "newton_solve": last["sweeps_cg"] + last["sweeps_newton"], "of_which_cg": last["sweeps_cg"],
            "line_search": last["sweeps_linesearch"], "chi_sinkhorn": last["sweeps_sinkhorn"],
            "stage_fixes": last["sweeps_stage"], "final_evaluation": last["sweeps_total"] - fixed,
            "total": last["sweeps_total"],
            "paper_table1_adaptive": {"NewtonSolve": 1831, "Line Search": 24, "ChiSinkhorn": 8,
                                      "Mirror Descent": 23, "Total": 2795,
                                      "context": "primitive O(n^2) operations, upsampled MNIST n = 4096, "
                                                 "L1 cost, gamma 2^5 -> 2^18, FP64, RTX 2080 Ti"}}
        stage_trace = {"columns": ["gamma", "delta_min", "q_next", "newton_steps", "cg_iters", "sweeps"],
                       "rows": [[rc["gamma"], rc["delta_min"] if math.isfinite(rc["delta_min"]) else None,
                                 rc["q_next"], rc["newton_steps"], rc["cg_iters"], rc["sweeps"]]
                                for rc in last.get("stage_records", [])]}
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            ops = oracle_ops_of_workload()
            smp = oracle_sample(args.cpu_seconds)
            cpu = {"value": round(oracle_estimate(smp, ops), 3), "unit": "s", "cores": cpu_cores(),
                   "kind": "oracle", "sample": cpu_sample_text(smp, ops),
                   "sample_wall_s": round(smp["wall"], 2)}
        result = {
            "metric": METRIC, "value": round(sec, 5), "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(sec * 1e3, 3),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 exp/sums on f64 potentials (mixed)", "data": "synthetic",
            "config": bench_config(args, world),
            "marg_err_l1": last["marg_err_l1"], "reached_tol": last["marg_err_l1"] <= TOL,
            "p_entries_per_s": round(p_entries_per_s, 1), "sweeps_per_solve": sweeps,
            "solve_stats": {k: last[k] for k in ("stages", "newton_steps", "cg_iters", "cg_solves",
                                                 "ls_trials", "sinkhorn_iters", "curvature_stops",
                                                 "sweeps_cg", "sweeps_total", "final_rho")},
            "e2e": {"value": round(e2e, 5), "unit": "s",
                    "h2d_bytes_per_step": int(C_h.numel() * 4 + r_h.numel() * 8 + c_h.numel() * 8),
                    "d2h_bytes_per_step": int(2 * N * 8)},
            "op_breakdown": op_breakdown, "stage_trace": stage_trace,
            "gpu_launches": int(launches), "roofline": roofline, "cpu_baseline": cpu,
            "plain_fp32": plain, "rounded": rounded, "mdot_sinkhorn": mdot_sk, "clocks": clocks,
            **extra,
        }
        print(json.dumps(result), flush=True)
    h.close()
    if world > 1:
        dist.destroy_process_group()
    return result


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------

def run_reference(args):
    """The reference arm: the oracle (the paper ships no code), as it stands, on the
    host cores. Each step is one bounded sample of the workload (the oracle's LSE
    update and CG step timed for --cpu-seconds / 2 s each, as in the GPU arm's
    cpu_baseline); value = the oracle's time for one whole solve, its recorded
    operation counts priced at the step's per-operation times, averaged over the
    timed steps. ms_per_step is the wall time of one sample step. With --cpu-full
    each step is instead one complete oracle solve (about two minutes)."""
    rank, world, _ = env_rank()
    if rank != 0:
        return None
    ops = oracle_ops_of_workload()
    per = max(2.0, args.cpu_seconds / 2)
    vals, walls, last = [], [], None
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        if args.cpu_full:
            sec, _ = oracle_full_solve_seconds()
            est = sec
        else:
            last = oracle_sample(per)
            est = oracle_estimate(last, ops)
        if k >= args.warmup:
            vals.append(est)
            walls.append(time.perf_counter() - t0)
    v = statistics.mean(vals)
    sample = ("per step: one complete oracle solve" if args.cpu_full else cpu_sample_text(last, ops))
    out = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(1e3 * statistics.mean(walls), 1), "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": bench_config(args, world),
           "value_is": ("mean measured oracle solve time" if args.cpu_full else
                        "oracle solve time estimated per step from a bounded sample; ms_per_step is "
                        "the sample's wall time"),
           "cpu_baseline": {"value": round(v, 3), "unit": "s", "cores": cpu_cores(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(v, 3), "unit": "s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return out


# ---------------------------------------------------------------------------
# further workloads (parity-test configurations; each prints its own JSON line)
# ---------------------------------------------------------------------------


def _gpu_props(dev):
    import torch
    pr = torch.cuda.get_device_properties(dev)
    return pr.multi_processor_count


def _point_problem_tensors(p, dev):
    import torch
    hs = {k: torch.from_numpy(p[k]).pin_memory() for k in ("X", "Y", "r", "c")}
    ds = {k: v.to(dev) for k, v in hs.items()}
    return hs, ds


def _sweep_rates(h, E, prob, u, v, gamma, n, m, sms, kinds=((0, "cg_col_sweep"), (1, "cg_row_sweep"),
                                                             (3, "row_lse_sweep")), iters=3):
    out = {}
    for kind, name in kinds:
        ms = h.eot_sweep_bench(prob, u, v, gamma, kind, iters)
        ent = n * m / (ms * 1e-3)
        out[name] = {"ms": round(ms, 3), "p_entries_per_s": round(ent, 1),
                     "ex2_frac_of_mufu_peak": round(ent / (sms * MUFU_PER_CLK_SM * 2.07e9), 4)}
    return out


def run_batch256(args):
    """256 point problems (n = m uniform in [256, 4096], points uniform in the unit
    square, Dirichlet(1) weights, squared-Euclidean cost normalised per problem),
    gamma 2^4 -> 2^12, mixed precision, tol 1e-6, one eot_solve_batched call per
    step. value = seconds for the whole batch."""
    import numpy as np
    import torch

    import paper_2504_02067_gb300 as E
    import workloads as W
    E.build()
    dev = torch.device("cuda", 0)
    sizes = W.batch_sizes(0)
    ps = [W.uniform_points_problem(1000 + k, int(nk)) for k, nk in enumerate(sizes)]
    host, devs = zip(*[_point_problem_tensors(p, dev) for p in ps])
    probs = [E.Problem(X=d["X"], Y=d["Y"], r=d["r"], c=d["c"], precision="mixed", cost_scale=0.0)
             for d in devs]
    us = [torch.empty(int(nk), dtype=torch.float64, device=dev) for nk in sizes]
    vs = [torch.empty(int(nk), dtype=torch.float64, device=dev) for nk in sizes]
    h = E.Handle(0, 64, 64)
    prm = E.default_params(gamma_i=16.0, gamma_f=4096.0, tol_final=TOL)
    t0 = time.perf_counter()
    for _ in range(args.warmup):
        st, stats = h.eot_solve_batched(probs, prm, us, vs)
    tune_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(0)
    torch.cuda.synchronize()
    l0 = h.launches()
    sampler.start()
    times = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, stats = h.eot_solve_batched(probs, prm, us, vs)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    clocks = sampler.stop()
    launches = h.launches() - l0
    sec = sum(times) / len(times)
    entries = sum(s["sweeps_total"] * int(nk) * int(nk) for s, nk in zip(stats, sizes))
    # end to end: inputs from pinned host memory, potentials back
    uh = [torch.empty(int(nk), dtype=torch.float64).pin_memory() for nk in sizes]
    vh = [torch.empty(int(nk), dtype=torch.float64).pin_memory() for nk in sizes]
    e_times = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for hh, dd in zip(host, devs):
            for k in ("X", "Y", "r", "c"):
                dd[k].copy_(hh[k], non_blocking=True)
        h.eot_solve_batched(probs, prm, us, vs)
        for a, b in zip(uh + vh, us + vs):
            a.copy_(b, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e_times.append(e0.elapsed_time(e1) / 1e3)
    h2d = sum(sum(t.numel() * t.element_size() for t in hh.values()) for hh in host)
    d2h = sum(t.numel() * 8 for t in uh + vh)
    G, ro, groups = h.batch_last_config()
    cpu = None
    if not args.no_cpu_baseline:
        # the oracle's full solve of the smallest problems, scaled by sum n_k m_k
        from oracle import eot_oracle as O
        order = np.argsort(sizes)
        t0 = time.perf_counter()
        done, work = 0, 0
        while done < 3 and time.perf_counter() - t0 < args.cpu_seconds:
            p = ps[order[done]]
            C64 = O.sqeuclid_scale(p["X"], p["Y"]) * O.sqeuclid(p["X"], p["Y"])
            O.mdot(C64, p["r"], p["c"], gamma_i=16.0, gamma_f=4096.0, tol_final=TOL)
            work += int(sizes[order[done]]) ** 2
            done += 1
        dt = time.perf_counter() - t0
        total_work = int(np.sum(sizes.astype(np.int64) ** 2))
        cpu = {"value": round(dt * total_work / work, 1), "unit": "s", "cores": os.cpu_count(),
               "kind": "oracle",
               "sample": "oracle MDOT of the %d smallest problems (n = %s) in %.1f s, scaled by "
                         "sum n_k^2 of the batch" % (done, [int(sizes[i]) for i in order[:done]], dt)}
    out = {"metric": METRIC, "value": round(sec, 4), "unit": "s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(sec * 1e3, 2), "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32 exp/sums on f64 potentials (mixed)",
           "data": "synthetic",
           "config": {"workload": "batch256_uniform2d_n256-4096_gamma2^12", "problems": len(ps),
                      "sum_n2": int(np.sum(sizes.astype(np.int64) ** 2)), "gamma_f": 4096.0,
                      "tol": TOL, "parallelism": "single", "l2": "inputs < L2; not flushed"},
           "all_ok": all(x == 0 for x in st), "max_marg_err_l1": max(s["marg_err_l1"] for s in stats),
           "p_entries_per_s": round(entries / sec, 1), "first_call_incl_autotune_s": round(tune_s, 3),
           "batch_config": {"ctas_per_group": G, "elements_per_thread": ro, "groups": groups},
           "e2e": {"value": round(sum(e_times) / len(e_times), 4), "unit": "s",
                   "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
           "gpu_launches": int(launches), "cpu_baseline": cpu, "clocks": clocks}
    print(json.dumps(out), flush=True)
    h.close()
    return out


def run_points_workload(args, kind):
    """d64: n = m = 16384 points in d = 64 (8-component Gaussian mixtures), gamma
    2^4 -> 2^10, mixed, tol 1e-6: one solve per step plus sweep rates.
    colour: n = m = 2^20 RGB points (d = 3, 16-component mixtures), sweep rates of
    the CG halves and the row LSE at gamma 2^10 (a full solve is out of the bench's
    time budget)."""
    import numpy as np
    import torch

    import paper_2504_02067_gb300 as E
    import workloads as W
    E.build()
    dev = torch.device("cuda", 0)
    sms = _gpu_props(dev)
    p = W.gmm_problem_d64(0) if kind == "d64" else W.colour_problem(0)
    n = p["X"].shape[0]
    hs, ds = _point_problem_tensors(p, dev)
    h = E.Handle(0, 64, 64)
    prob = E.Problem(X=ds["X"], Y=ds["Y"], r=ds["r"], c=ds["c"], precision="mixed", cost_scale=0.0)
    gf = 1024.0
    rng = np.random.default_rng(0)
    u = torch.from_numpy(np.full(n, -np.log(n)) + rng.normal(0, 0.1, n)).to(dev)
    v = torch.from_numpy(np.full(n, -np.log(n))).to(dev)
    rates = _sweep_rates(h, E, prob, u, v, gf, n, n, sms, iters=2 if kind == "colour" else 5)
    out = {"metric": METRIC, "unit": "s", "n_gpus": 1, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32 exp/sums on f64 potentials (mixed)", "data": "synthetic",
           "sweeps": rates}
    if kind == "d64":
        prm = E.default_params(gamma_i=16.0, gamma_f=gf, tol_final=TOL)
        uu = torch.empty(n, dtype=torch.float64, device=dev)
        vv = torch.empty(n, dtype=torch.float64, device=dev)
        for _ in range(min(args.warmup, 1)):
            h.eot_solve(prob, prm, uu, vv)
        sampler = ClockSampler(0)
        sampler.start()
        times = []
        for _ in range(max(1, min(args.steps, 2))):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st = h.eot_solve(prob, prm, uu, vv).as_dict()
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        out["clocks"] = sampler.stop()
        sec = sum(times) / len(times)
        out.update({"value": round(sec, 3), "ms_per_step": round(sec * 1e3, 1), "steps": len(times),
                    "marg_err_l1": st["marg_err_l1"],
                    "solve_stats": {k: st[k] for k in ("stages", "newton_steps", "cg_iters", "ls_trials",
                                                       "sweeps_total")},
                    "p_entries_per_s": round(st["sweeps_total"] * n * n / sec, 1),
                    "config": {"workload": "gmm8_d64_n16384_gamma2^10", "n": n, "d": 64,
                               "gamma_f": gf, "tol": TOL}})
    elif args.solve:
        # the paper's colour-transfer regime (Fig. 3): solve to its eps_d at gamma_f =
        # 2^10 (eps_d = min(H(r), H(c)) / gamma_f^1.5, about 4.2e-4 for uniform weights
        # on 2^20 points; tol_final = 1e-3 makes the last stage's tolerance eps_d)
        # under a wall-clock budget
        prm = E.default_params(gamma_i=16.0, gamma_f=gf, tol_final=1e-3, max_seconds=args.max_seconds)
        uu = torch.empty(n, dtype=torch.float64, device=dev)
        vv = torch.empty(n, dtype=torch.float64, device=dev)
        eps_d = float(np.log(n)) / gf ** 1.5
        sampler = ClockSampler(0)
        sampler.start()
        t0 = time.perf_counter()
        try:
            st = h.eot_solve(prob, prm, uu, vv).as_dict()
            status = "EOT_OK"
        except E.EotError as ex:
            st, status = getattr(ex, "stats", None), str(ex)[:200]
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        out["clocks"] = sampler.stop()
        g_last = st["final_gamma"] if st else gf
        rr, cc, _, _, _ = h.marginals(prob, uu, vv, g_last)
        err = float((rr - ds["r"]).abs().sum() + (cc - ds["c"]).abs().sum())
        out.update({"value": round(sec, 2) if status == "EOT_OK" else None, "ms_per_step": round(sec * 1e3, 1),
                    "status": status, "max_seconds": args.max_seconds, "eps_d_paper": eps_d,
                    "reached_eps_d": status == "EOT_OK" and err <= 1.5 * eps_d,
                    "stopped_at_gamma": g_last, "marg_err_l1": err,
                    "solve_stats": ({k: st[k] for k in ("stages", "newton_steps", "cg_iters", "ls_trials",
                                                        "sinkhorn_iters", "sweeps_total", "grad_l1")} if st else None),
                    "config": {"workload": "rgb_gmm16_d3_n2^20_gamma2^10", "n": n, "d": 3, "gamma_f": gf,
                               "tol": "eps_d of the paper (Sec. 2.2 / Fig. 3)"}})
    else:
        out.update({"value": None, "config": {"workload": "rgb_gmm16_d3_n2^20_gamma2^10", "n": n,
                                               "d": 3, "gamma": gf}})
    print(json.dumps(out), flush=True)
    h.close()
    return out


def run_profile_points(args):
    """A few launches of one point sweep kernel (for ncu) on the d = 64 workload
    (n = m = 16384, gamma 2^10, mixed): set-up launches first, then
    `args.profile_iters` launches of kind args.profile_points."""
    import numpy as np
    import torch

    import paper_2504_02067_gb300 as E
    import workloads as W
    E.build()
    dev = torch.device("cuda", 0)
    p = W.gmm_problem_d64(0)
    n = p["X"].shape[0]
    X, Y = torch.from_numpy(p["X"]).to(dev), torch.from_numpy(p["Y"]).to(dev)
    r, c = torch.from_numpy(p["r"]).to(dev), torch.from_numpy(p["c"]).to(dev)
    h = E.Handle(0, 64, 64)
    prob = E.Problem(X=X, Y=Y, r=r, c=c, precision="mixed", cost_scale=0.0)
    rng = np.random.default_rng(0)
    u = torch.from_numpy(np.full(n, -np.log(n)) + rng.normal(0, 0.1, n)).to(dev)
    v = torch.from_numpy(np.full(n, -np.log(n))).to(dev)
    ms = h.eot_sweep_bench(prob, u, v, 1024.0, args.profile_points, args.profile_iters)
    print(json.dumps({"kind": args.profile_points, "iters": args.profile_iters, "ms_per_launch": ms}))
    h.close()


def run_profile_sweep(args):
    """A few launches of one sweep kernel on the full-size workload (for ncu):
    the set-up launches come first (one row LSE, the Newton-step column and row
    sweeps, the d_v column sweep), then `args.profile_iters` timed launches."""
    import numpy as np
    import torch

    import paper_2504_02067_gb300 as E
    import workloads as W

    E.build()
    dev = torch.device("cuda", 0)
    p = W.grid_problem_4096(0, args.cost)
    C = torch.from_numpy(p["C"]).to(dev)
    r = torch.from_numpy(p["r"]).to(dev)
    c = torch.from_numpy(p["c"]).to(dev)
    h = E.Handle(0, N, N)
    prob = E.Problem(C, r, c, precision="mixed")
    rng = np.random.default_rng(0)
    u = torch.from_numpy(np.log(p["r"] + 1e-6) + rng.normal(0, 1, N)).to(dev)
    v = torch.from_numpy(np.log(p["c"] + 1e-6)).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev) if args.profile_cold else None
    ms = h.eot_sweep_bench(prob, u, v, GAMMA_F, args.profile_sweep, args.profile_iters, flush=flush)
    print(json.dumps({"kind": args.profile_sweep, "iters": args.profile_iters, "cold": bool(args.profile_cold),
                      "ms_per_launch": ms}))
    h.close()


def run_profile_solve(args):
    """One solve for a profiler's launch list: a warm-up solve, then one solve
    between cudaProfilerStart and Stop (capture with ncu --profile-from-start
    off). `grid4096`: the headline 64 x 64 grid workload (mixed precision);
    `grid784`: the 28 x 28 grid in FP64, gamma 2^4 -> 2^12 (the FP64 record).
    Kernels inside CUDA graphs with conditional nodes are not listed by ncu, so
    run it with EOT_GRAPH=0: the same kernels in the same order, launched
    directly."""
    import torch

    import paper_2504_02067_gb300 as E
    import workloads as W

    E.build()
    dev = torch.device("cuda", 0)
    small = args.profile_solve == "grid784"
    nn = 784 if small else N
    p = W.grid_problem_784(0) if small else W.grid_problem_4096(0, args.cost)
    C = torch.from_numpy(p["C"]).to(dev)
    r = torch.from_numpy(p["r"]).to(dev)
    c = torch.from_numpy(p["c"]).to(dev)
    h = E.Handle(0, nn, nn)
    prob = E.Problem(C, r, c, precision="fp64" if small else "mixed")
    prm = E.default_params(gamma_i=GAMMA_I, gamma_f=4096.0 if small else GAMMA_F, tol_final=TOL)
    u = torch.empty(nn, dtype=torch.float64, device=dev)
    v = torch.empty(nn, dtype=torch.float64, device=dev)
    h.eot_solve(prob, prm, u, v)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    flush.zero_()
    torch.cuda.synchronize()
    l0 = h.launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()
    e0.record()
    st = h.eot_solve(prob, prm, u, v).as_dict()
    e1.record()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"workload": args.profile_solve, "graph": os.environ.get("EOT_GRAPH", "1") != "0",
                      "ms": round(e0.elapsed_time(e1), 3),
                      "launches": h.launches() - l0, "cg_iters": st["cg_iters"],
                      "sweeps": st["sweeps_total"]}))
    h.close()


def run_profile_batch(args):
    """One eot_solve_batched launch on the first `args.profile_batch` problems of
    the batch256 workload, between cudaProfilerStart and Stop, after a warm-up
    launch that autotunes the configuration (for ncu --profile-from-start off)."""
    import torch

    import paper_2504_02067_gb300 as E
    import workloads as W

    E.build()
    dev = torch.device("cuda", 0)
    sizes = W.batch_sizes(0)[: args.profile_batch]
    ps = [W.uniform_points_problem(1000 + k, int(nk)) for k, nk in enumerate(sizes)]
    devs = [{k: torch.from_numpy(p[k]).to(dev) for k in ("X", "Y", "r", "c")} for p in ps]
    probs = [E.Problem(X=d["X"], Y=d["Y"], r=d["r"], c=d["c"], precision="mixed", cost_scale=0.0) for d in devs]
    us = [torch.empty(int(nk), dtype=torch.float64, device=dev) for nk in sizes]
    vs = [torch.empty(int(nk), dtype=torch.float64, device=dev) for nk in sizes]
    h = E.Handle(0, 64, 64)
    prm = E.default_params(gamma_i=16.0, gamma_f=4096.0, tol_final=TOL)
    h.eot_solve_batched(probs, prm, us, vs)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()
    e0.record()
    st, stats = h.eot_solve_batched(probs, prm, us, vs)
    e1.record()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    G, ro, groups = h.batch_last_config()
    print(json.dumps({"problems": len(sizes), "sizes": [int(x) for x in sizes], "ms": round(e0.elapsed_time(e1), 3),
                      "all_ok": all(x == 0 for x in st), "config": [G, ro, groups],
                      "sweeps": sum(sm["sweeps_total"] for sm in stats)}))
    h.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cost", default="sqeuclid", choices=["sqeuclid", "l1"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--cpu-full", action="store_true",
                    help="--impl reference: each step is one complete oracle solve (about two minutes)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the sub-records of the other workloads (config 1, config 2 breadth, d = 64, batch)")
    ap.add_argument("--no-sinkhorn", action="store_true",
                    help="skip the MDOT-Sinkhorn comparison solve on the headline workload")
    ap.add_argument("--profile-sweep", type=int, default=-1,
                    help="run only eot_sweep_bench of this kind (0 CG column, 1 CG row, 2 HVP, 3 row LSE)")
    ap.add_argument("--profile-iters", type=int, default=3)
    ap.add_argument("--profile-cold", action="store_true",
                    help="with --profile-sweep: time each launch alone after an L2 overwrite")
    ap.add_argument("--profile-solve", nargs="?", const="grid4096", default=None, choices=["grid4096", "grid784"],
                    help="one solve between profiler start and stop (for ncu)")
    ap.add_argument("--profile-batch", type=int, default=0,
                    help="one eot_solve_batched launch on the first K batch256 problems (for ncu)")
    ap.add_argument("--profile-points", type=int, default=-1,
                    help="run only eot_sweep_bench of this kind on the d = 64 point workload")
    ap.add_argument("--solve", action="store_true", help="--workload colour: a full solve to the paper's eps_d")
    ap.add_argument("--max-seconds", type=float, default=900.0, help="wall-clock budget of --workload colour --solve")
    ap.add_argument("--workload", default="grid4096", choices=["grid4096", "batch256", "d64", "colour"],
                    help="grid4096 = the headline line; the others print their own lines")
    args = ap.parse_args()
    if args.profile_sweep >= 0:
        run_profile_sweep(args)
        return
    if args.profile_solve:
        run_profile_solve(args)
        return
    if args.profile_batch > 0:
        run_profile_batch(args)
        return
    if args.profile_points >= 0:
        run_profile_points(args)
        return
    if args.workload != "grid4096" and args.impl == "ours":
        if args.workload == "batch256":
            run_batch256(args)
        else:
            run_points_workload(args, args.workload)
        return
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
