#!/usr/bin/env python
"""Benchmark of the GB300 sequential posterior simulator.

Metric: M-phase particle x observation likelihood evaluations per second.  One
step is one whole simulator run (Algorithm 2: prior draws -> C, S, M cycles ->
log marginal likelihood).  Default workload: the largest one-GPU shape, EGARCH
with K = 3 factors and I = 4 mixture components (23 parameters, Table 1),
T = 20000 synthetic daily returns with heavy-tailed mixture shocks, J = 128
groups x N = 8192 particles (about 1M), FP32 recursion with FP64 accumulators,
random-walk Metropolis adapted toward 0.25 acceptance, power tempering; its
`equal_nse` entry compares FP32 random-walk and FP32 MALA runs at equal log-ML
NSE.  `--workload egarch22_T5000` runs Section 5's own J = 64 x N = 1024,
K = 2, I = 2, T = 5000 shape.
`value` = sum over steps of the M-phase evaluations / summed step time, with
the observations and prior draws resident in HBM; `e2e` repeats the run through
the public API from host buffers (context creation, host->device copies of
observations and prior draws, and the read-back of the result inside the timed
region).  Each step's device time is bracketed by CUDA events on the run's
stream; L2 is flushed between steps by writing a 256 MB buffer.

`--impl reference` times the FP64 CPU oracle on the host cores instead (bounded
sample: random-walk Metropolis iterations over a subsample of particles per
step).  `--peaks` prints the measured ALU pipe rates (smc_peaks) and exits.
Multi-GPU: independent replicas, one per rank (the path has no exchange step).
"""
from __future__ import annotations

import argparse
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

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
SM_COUNT_GB300 = 152
# ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of the current
# mutation kernel, by (workload, particles per thread, threads per block): the
# mean of two launches of the second cycle's M phase at the full size, captured
# with --metrics dram__bytes_read.sum,dram__bytes_write.sum (one pass;
# profiles/k_mutate_x2_egarch34_T20000.md).  Shapes without a capture of the
# current kernel report null.
MUTATE_TRAFFIC = {("egarch34_T20000", 2, 128): 1.153083008e9, ("egarch22_T5000", 1, 224): 8.935808e6}
SM_MAX_MHZ_FALLBACK = 2070.0
# Acceptance target of the MALA runs: 0.574, the asymptotically optimal rate of
# Langevin proposals (Roberts and Rosenthal, 1998); the random walk keeps the
# paper's 0.25.  Measured on K=2, I=2, T=5000, 262,144 particles (3 seeds):
# run time x NSE^2 0.000475 against 0.000620 with a target of 0.5.
MALA_TARGET = 0.574
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="egarch34_T20000")
    ap.add_argument("--peaks", action="store_true", help="print the measured ALU pipe rates and exit")
    ap.add_argument("--precision", action="store_true",
                    help="print the FP32 path's measured error against FP64 for each result and exit")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cycles", type=int, default=0, help="cap on cycles per run (0 = full run; profiling only)")
    ap.add_argument("--no-equal-nse", action="store_true")
    ap.add_argument("--launch-shape", default="", help="PPT,THREADS: fixed mutation launch shape instead of autotuning")
    ap.add_argument("--equal-nse-seeds", type=int, default=3)
    ap.add_argument("--particles", default="", help="J,N: override the workload's groups x particles (profiling only)")
    ap.add_argument("--tempering", default="power", choices=["power", "data"],
                    help="C phase: power tempering (default) or the paper's data tempering")
    return ap.parse_args()


# ----------------------------------------------------------------- roofline
def alu_ops_per_eval(K, I, gamma):
    """Algorithmic per-observation work of the FP32 recursion (one particle):
    FP32 lane operations and SFU (MUFU) operations.  See the roofline section of
    the design notes for the derivation."""
    fp32 = 1 + (3 if gamma else 2) * K + K + 1 + 2
    fp32 += {1: 1, 2: 8}.get(I, 5 * I)
    mufu = 1 + {1: 0, 2: 1}.get(I, I)
    return fp32, mufu


def mala_ops_per_eval(K, I, gamma):
    """Algorithmic per-observation work of one MALA likelihood-and-gradient
    evaluation: the forward recursion (as the random walk's), the state-only
    recomputation of the reverse sweep's segment, and the adjoint step of the
    reverse sweep (the formulas of the adjoint kernel's header: per mixture
    component the responsibility, its three parameter adjoints and the shock's
    adjoint term; per factor the shock coefficient, the state adjoint and three
    parameter adjoints)."""
    fp32, mufu = alu_ops_per_eval(K, I, gamma)
    fp32 += 1 + (3 if gamma else 2) * K + (K - 1) + 4
    mufu += 1
    fp32 += (18 * I if I >= 2 else 1) + 7 * K + 4
    mufu += I + 1 if I >= 2 else 0
    return fp32, mufu


NOMINAL_RATES = {"ffma": 128.0, "ffma2": 128.0, "ex2": 32.0, "issue": 4.0}


def alu_peak_evals(K, I, gamma, sms, mhz, paired=False, mala=False, rates=None):
    """Evaluations/s bound at the given SM clock from the FP32 pipe, the SFU
    (ex2/lg2) and instruction issue.  `rates` are per SM and clock: lane
    operations of FFMA ("ffma"), of the paired FFMA2 ("ffma2") and of MUFU.EX2
    ("ex2"), and warp instructions issued ("issue"); by default the nominal
    128 / 128 / 32 lanes and 4 warp instructions (4 schedulers x 32 lanes, each
    instruction once), else the measured rates of smc_peaks.  With paired FP32
    instructions (two particles per thread) an FP32 instruction carries two
    lanes' work, so issue counts fp32/2 + mufu per evaluation while the FP32
    pipe (at the FFMA2 rate) still bounds fp32."""
    r = dict(NOMINAL_RATES)
    if rates:
        r.update({k: v for k, v in rates.items() if k in r and v})
    fp32, mufu = (mala_ops_per_eval if mala else alu_ops_per_eval)(K, I, gamma)
    limits = {"issue": 32.0 * r["issue"] / ((fp32 / 2.0 if paired else fp32) + mufu),
              "fp32": (r["ffma2"] if paired else r["ffma"]) / fp32, "mufu": r["ex2"] / mufu}
    pipe = min(limits, key=limits.get)
    return sms * mhz * 1e6 * limits[pipe], pipe


def sm_max_mhz():
    try:
        with open(MEASURED_PEAKS) as f:
            return float(json.load(f).get("sm_max_mhz", SM_MAX_MHZ_FALLBACK)), "of measured"
    except Exception:
        return SM_MAX_MHZ_FALLBACK, "of fallback"


# ------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling during the timed region (read-only queries)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.proc:
            return out
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
            os.unlink(self.path)
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for name, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(name)
            except Exception:
                continue
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), reasons=sorted(reasons),
                       samples=len(sm))
        return out


# ------------------------------------------------------------ distributed
def combine_ranks(seconds, evals, world, device="cpu"):
    """Whole-job figures of N independent replicas: the slowest rank's timed
    seconds and the evaluations of all ranks (the process group must be up
    when world > 1; NCCL on the GPUs, gloo in the CPU test)."""
    if world <= 1:
        return seconds, evals
    import torch
    import torch.distributed as dist
    tt = torch.tensor([seconds], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    ee = torch.tensor([evals], device=device, dtype=torch.float64)
    dist.all_reduce(ee, op=dist.ReduceOp.SUM)
    return float(tt.item()), float(ee.item())


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# -------------------------------------------------------------- CPU oracle
def host_cpu():
    """CPU model of the host (read-only, /proc/cpuinfo or lscpu)."""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        d = {a.strip(): b.strip() for a, b in (l.split(":", 1) for l in out.splitlines() if ":" in l)}
        return " ".join(x for x in (d.get("Vendor ID"), d.get("Model name")) if x) or "unknown"
    except Exception:
        return "unknown"


def cpu_oracle_rate(w, y, budget_s=12.0, sample=256, threads=None):
    """The FP64 oracle's M-phase rate (one random-walk Metropolis iteration over
    `sample` posterior-like particles x all T observations per call), on
    `threads` host threads (default: every core), repeated for about
    `budget_s` seconds."""
    import numpy as np
    import oracle as O
    from paper_1304_4334_gb300 import inputs as I

    spec = O.ModelSpec(K=w.K, I=w.I, gamma=w.gamma)
    th = I.posterior_cloud(I.theta_of_truth(w.truth, I_model=w.I, gamma=w.gamma), sample, 0.02, seed=5)
    cores = threads or os.cpu_count() or 1
    ll, st = O.loglik(spec, y, th, with_state=True, nthreads=cores)
    lp = O.logprior(spec, th)
    _, V = O.mean_cov(th)
    Lm, _ = O.cholesky(0.09 * V)
    evals, t0, it = 0.0, time.perf_counter(), 0
    while True:
        th, ll, lp, st, _, _ = O.mutate_rw(spec, y, th, ll, lp, st, Lm, 1.0, 7, 1, it, nthreads=cores)
        it += 1
        evals += sample * len(y)
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    return {"value": evals / el, "unit": "particle*obs lik evals/s", "cores": cores, "kind": "oracle",
            "cpu": host_cpu(),
            "sample": f"{it} random-walk Metropolis iterations x {sample} particles x T={len(y)} "
                      f"({w.name}), FP64 C oracle, {cores} OpenMP thread{'s' if cores > 1 else ''}, {el:.1f} s"}


def cpu_oracle_full_run(threads=None):
    """The FP64 oracle's whole adaptive run on the small EGARCH(1,1) workload
    (K = 1, I = 1, no leverage, T = 500, J = 4 x N = 256, FP64 random walk,
    10 Metropolis iterations per M phase), timed on the host cores."""
    import oracle as O
    from paper_1304_4334_gb300 import inputs as I

    w = I.WORKLOADS["egarch11_T500"]
    y = w.data()
    spec = O.ModelSpec(K=1, I=1, gamma=False)
    th0 = I.draw_prior(*O.table1_prior(1, 1, False), w.P, seed=w.prior_seed)
    cores = threads or os.cpu_count() or 1
    t0 = time.perf_counter()
    r = O.smc_run(spec, y, th0, w.J, w.N, rbar=w.rbar, kappa=w.kappa, seed=7, nthreads=cores)
    el = time.perf_counter() - t0
    return {"workload": w.name, "seconds": el, "cores": cores, "cycles": r["cycles"],
            "metropolis_steps": r["metropolis_steps"], "log_ml": r["log_ml"], "nse": r["log_ml_nse"],
            "value": r["evals"] / el, "unit": "particle*obs lik evals/s"}


def cpu_baseline_leg(w, y):
    """The oracle on the host cores: M-phase rate with every core (OpenMP over
    particles; the headline) and with one thread, plus the small workload's
    whole run in both modes."""
    cpu = cpu_oracle_rate(w, y)
    one = cpu_oracle_rate(w, y, budget_s=6.0, sample=64, threads=1)
    cpu["single_thread"] = {"value": one["value"], "sample": one["sample"]}
    cpu["full_run_egarch11_T500"] = {"all_cores": cpu_oracle_full_run(),
                                     "single_thread": cpu_oracle_full_run(threads=1)}
    return cpu


def run_reference(args, world, rank):
    if rank != 0:
        return
    from paper_1304_4334_gb300 import inputs as I
    import oracle
    oracle.build()
    w = I.WORKLOADS[args.workload]
    y = w.data()
    for _ in range(args.warmup):
        cpu_oracle_rate(w, y, budget_s=0.5, sample=64)
    vals = []
    t0 = time.perf_counter()
    last = None
    for _ in range(args.steps):
        last = cpu_oracle_rate(w, y, budget_s=4.0, sample=256)
        vals.append(last["value"])
    total = time.perf_counter() - t0
    value = statistics.mean(vals)
    line = {"metric": "M-phase particle*obs lik evals/s", "value": value,
            "unit": "particle*obs lik evals/s", "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "K": w.K, "I": w.I, "T": w.T,
                                            "J": w.J, "N": w.N, "sampler": "rw"},
            "cpu_baseline": {"value": value, "unit": "particle*obs lik evals/s", "cores": last["cores"],
                             "kind": "oracle", "sample": last["sample"]},
            "e2e": {"value": value, "unit": "particle*obs lik evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------- wall time at equal NSE
def equal_nse_comparison(S, w, y, th0, stream, seeds, shape=None, fp64_seeds=None):
    """The paper's efficiency measure, precision / time = 1 / (NSE^2 t)
    (Section 5.2, Table 3), for the log marginal likelihood: whole runs of
    several forms on the same GPU, same data and prior draws.  At T = 5000 the
    reference is the plain FP64 random-walk form, against the FP32 random-walk
    and FP32 MALA forms; at 1M particles x T = 20000 (where an FP64 run would
    take hours) the FP32 random walk is the reference for FP32 MALA.  Reported
    per form: mean run time, mean NSE^2, and the wall time it needs to reach
    the reference form's NSE (t * NSE^2 / NSE_ref^2), relative to that form.
    shape: the random-walk runs' mutation launch shape (the benchmark's
    autotuned one); fp64_seeds: fewer seeds for the slow FP64 form."""
    import torch
    m = S.model_egarch(w.K, w.I, w.gamma)
    forms = [("fp64_rw", S.FP64, S.RW, 0.25), ("fp32_rw", S.FP32, S.RW, 0.25),
             ("fp32_mala", S.FP32, S.MALA, MALA_TARGET)]
    if w.T > 10000:
        forms = forms[1:]
    out = {}
    for name, prec, mut, target in forms:
        ts, nse2, lml = [], [], []
        nseeds = fp64_seeds if (prec == S.FP64 and fp64_seeds) else seeds
        for k in range(nseeds):
            cfg = S.config_default(J=w.J, N=w.N, precision=prec, mutation=mut, acc_target=target,
                                   rbar=w.rbar, kappa=w.kappa, seed=500 + k)
            ctx = S.init(m, cfg, y, th0, stream=stream.cuda_stream)
            if shape and mut == S.RW and prec == S.FP32:
                ctx.set_launch_shape(shape[0], shape[1])
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.run()
            lm, nse, _ = ctx.log_ml()
            e1.record(stream)
            torch.cuda.synchronize()
            ctx.close()
            ts.append(e0.elapsed_time(e1) / 1e3)
            nse2.append(nse * nse)
            lml.append(lm)
        out[name] = {"seconds": statistics.mean(ts), "nse2": statistics.mean(nse2),
                     "log_ml": statistics.mean(lml), "runs": nseeds}
    ref = out[forms[0][0]]
    for v in out.values():
        v["wall_time_at_ref_nse_rel"] = (v["seconds"] * v["nse2"] / ref["nse2"]) / ref["seconds"]
        v["precision_per_second"] = 1.0 / (v["nse2"] * v["seconds"])
    return out


# ---------------------------------------------------- FP32 error per result
def _err_stats(x, ref):
    import numpy as np
    ok = np.isfinite(ref) & (ref > -1e7)
    ab = np.abs(x[ok] - ref[ok])
    rel = ab / np.abs(ref[ok])
    return {"n": int(ok.sum()), "rel_max": float(rel.max()), "rel_median": float(np.median(rel)),
            "abs_max": float(ab.max()), "abs_median": float(np.median(ab)),
            "share_rel_le_1e-4": float((rel <= 1e-4).mean())}


def precision_report(S, I, P=2048, seeds=2):
    """The FP32 path's error against FP64, per result (the FP32 mode of the
    precision contract: recursion in FP32, log likelihood, log weights and
    estimators in FP64), on the two FP32 workload shapes:
    - log likelihood of P particles over the full series, from the stand-alone
      likelihood kernel (which carries 1 - alpha) and from the mutation kernel
      (a zero-step random-walk iteration from a log likelihood of -inf accepts
      theta itself and stores its log likelihood), against the FP64 oracle:
      posterior-like particles (theta_true + N(0, 0.05^2)) and raw prior draws;
    - whole runs (J = 64 x N = 256) in FP32 and in FP64 on the GPU from the same
      prior draws and seed: log ML difference (absolute and in units of the FP64
      run's NSE) and the largest posterior-mean difference over the parameters
      (in units of the FP64 run's NSE of that mean)."""
    import numpy as np
    import torch
    import oracle as O
    out = {"what": "FP32 path vs FP64 per result", "shapes": {}}
    cores = os.cpu_count() or 1
    for name in ("egarch22_T5000", "egarch34_T20000"):
        w = I.WORKLOADS[name]
        y = w.data()
        spec = O.ModelSpec(K=w.K, I=w.I, gamma=w.gamma)
        m = S.model_egarch(w.K, w.I, w.gamma)
        mean, sd, lo = S.model_prior(m)
        yd = torch.as_tensor(y, dtype=torch.float32, device="cuda")
        rec = {"K": w.K, "I": w.I, "T": w.T}
        clouds = {"posterior_like": I.posterior_cloud(I.theta_of_truth(w.truth, I_model=w.I, gamma=w.gamma),
                                                      P, 0.05, seed=3),
                  "prior_draws": I.draw_prior(mean, sd, lo, P, seed=w.prior_seed + 99)}
        for cname, th in clouds.items():
            ll_o = O.loglik(spec, y, th, nthreads=cores)
            theta = torch.as_tensor(np.ascontiguousarray(th.T), device="cuda")
            ll = torch.empty(P, dtype=torch.float64, device="cuda")
            S.loglik(m, S.FP32, yd, theta, ll)
            llm = torch.full((P,), -math.inf, dtype=torch.float64, device="cuda")
            lpm = torch.as_tensor(O.logprior(spec, th), device="cuda")
            tm = theta.clone()
            S.mutate_rw(m, S.FP32, yd, tm, llm, lpm, None,
                        torch.zeros((spec.d, spec.d), dtype=torch.float64, device="cuda"), 1.0, 5, 1, 0)
            torch.cuda.synchronize()
            rec[f"loglik_{cname}"] = {"likelihood_kernel": _err_stats(ll.cpu().numpy(), ll_o),
                                      "mutation_kernel": _err_stats(llm.cpu().numpy(), ll_o)}
        runs = []
        J, N = 64, 256
        for k in range(seeds):
            th0 = I.draw_prior(mean, sd, lo, J * N, seed=w.prior_seed + 500 + k)
            res = {}
            for prec in (S.FP64, S.FP32):
                ctx = S.init(m, S.config_default(J=J, N=N, precision=prec, seed=77 + k), y, th0)
                t0 = time.perf_counter()
                ctx.run()
                lml = ctx.log_ml()
                el = time.perf_counter() - t0
                res[prec] = (lml, ctx.moments(), el)
                ctx.close()
            (l64, n64, _), m64, t64 = res[S.FP64]
            (l32, n32, _), m32, t32 = res[S.FP32]
            dm = np.abs(m32[:, 0] - m64[:, 0]) / m64[:, 2]
            runs.append({"log_ml_fp64": l64, "nse_fp64": n64, "log_ml_fp32": l32, "nse_fp32": n32,
                         "log_ml_diff": l32 - l64, "log_ml_diff_in_nse": (l32 - l64) / n64,
                         "max_mean_diff_in_nse": float(dm.max()), "seconds_fp64": t64, "seconds_fp32": t32})
        rec["runs_same_seed_J64_N256"] = runs
        out["shapes"][name] = rec
    out["log_ml_over_seeds"] = log_ml_bias_over_seeds(S, I)
    return out


def log_ml_bias_over_seeds(S, I, n=10):
    """FP32 - FP64 log ML over n prior-draw seeds (K=2, I=2, T=5000,
    J=64 x N=256): FP64 runs, FP32 runs with independent random numbers and
    FP32 runs with the FP64 runs' seeds; mean difference with its standard
    error from the seeds, and each form's seed-to-seed s.d. beside its mean
    NSE."""
    import numpy as np
    w = I.WORKLOADS["egarch22_T5000"]
    y = w.data()
    m = S.model_egarch(2, 2, True)
    mean, sd, lo = S.model_prior(m)
    J, N = 64, 256
    res = {"f64": [], "f32": [], "f32_same": []}
    for k in range(n):
        th0 = I.draw_prior(mean, sd, lo, J * N, seed=900 + k)
        for prec, key, seed in ((S.FP64, "f64", 11 + k), (S.FP32, "f32", 5011 + k), (S.FP32, "f32_same", 11 + k)):
            ctx = S.init(m, S.config_default(J=J, N=N, precision=prec, seed=seed), y, th0)
            ctx.run()
            res[key].append(ctx.log_ml()[:2])
            ctx.close()
    out = {"seeds": n}
    for key, v in res.items():
        a = np.array(v)
        out[key] = {"mean_log_ml": float(a[:, 0].mean()), "sd_over_seeds": float(a[:, 0].std(ddof=1)),
                    "mean_nse": float(a[:, 1].mean())}
    for key in ("f32", "f32_same"):
        dlt = np.array(res[key])[:, 0] - np.array(res["f64"])[:, 0]
        out[f"{key}_minus_f64"] = {"mean": float(dlt.mean()), "se": float(dlt.std(ddof=1) / np.sqrt(n))}
    return out


def batched_equal_nse(S, I, stream, n=8):
    """The FP32 + adjoint + batched form against the plain FP64 random walk,
    at equal log-ML NSE (the precision / time measure of Section 5.2): the
    first n datasets of the 32-dataset batch (T ~ U{500..10000}, K ~ U{1,2,3},
    I ~ U{1..4}, J = 16 x N = 1024 each) run (a) as one batch with FP32 MALA,
    (b) as one batch with the FP32 random walk and (c) one at a time with the
    FP64 random walk, from the same prior draws.  A batch's time to reach, for
    every dataset, the NSE of the FP64 run is its run time x the largest ratio
    NSE_batch^2 / NSE_fp64^2 over the datasets (NSE^2 falls as 1 / particles);
    'mean' uses the mean ratio instead.  Reported relative to the summed FP64
    run times."""
    import numpy as np
    import torch
    ws = I.batched_workloads(n=32, seed=40, J=16, N=1024)[:n]
    models, ys, ths = [], [], []
    for w in ws:
        m = S.model_egarch(w.K, w.I, True)
        mean, sd, lo = S.model_prior(m)
        models.append(m)
        ys.append(w.data())
        ths.append(I.draw_prior(mean, sd, lo, w.P, seed=w.prior_seed))
    th_dev = [torch.as_tensor(np.ascontiguousarray(t.T), device="cuda") for t in ths]

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, r

    out = {"datasets": n, "T": [w.T for w in ws], "KI": [[w.K, w.I] for w in ws]}
    for name, mut, target in (("fp32_mala_batched", S.MALA, MALA_TARGET), ("fp32_rw_batched", S.RW, 0.25)):
        cfgs = [S.config_default(J=w.J, N=w.N, precision=S.FP32, seed=300 + k, mutation=mut, acc_target=target)
                for k, w in enumerate(ws)]
        b = S.Batch(models, cfgs, ys, ths, stream=stream.cuda_stream)
        b.autotune(iters=1)
        b.reset(th_dev, 300)
        b.run()                                   # warm-up run
        t, _ = timed(lambda: (b.reset(th_dev, 300), b.run()))
        nse = [b.member(i).log_ml()[1] for i in range(n)]
        lml = [b.member(i).log_ml()[0] for i in range(n)]
        b.close()
        out[name] = {"seconds": t, "nse": nse, "log_ml": lml}
    t64, n64, l64 = [], [], []
    for k, w in enumerate(ws):
        cfg = S.config_default(J=w.J, N=w.N, precision=S.FP64, seed=300 + k)
        ctx = S.init(models[k], cfg, ys[k], ths[k], stream=stream.cuda_stream)
        t, _ = timed(lambda: ctx.run())
        lm, nse, _ = ctx.log_ml()
        ctx.close()
        t64.append(t)
        n64.append(nse)
        l64.append(lm)
    ref = sum(t64)
    out["fp64_rw_one_at_a_time"] = {"seconds": ref, "nse": n64, "log_ml": l64}
    for name in ("fp32_mala_batched", "fp32_rw_batched"):
        r = np.square(out[name]["nse"]) / np.square(n64)
        out[name]["wall_time_at_fp64_nse_rel_worst"] = out[name]["seconds"] * float(r.max()) / ref
        out[name]["wall_time_at_fp64_nse_rel_mean"] = out[name]["seconds"] * float(r.mean()) / ref
    return out


# ------------------------------------------------------------------ our arm
def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import numpy as np
    import torch

    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1304_4334_gb300 import inputs as I
    from paper_1304_4334_gb300 import smc as S

    if args.peaks:
        if rank == 0:
            print(json.dumps({"peaks": S.peaks(), "unit": "lane operations per SM and clock "
                              "(issue: warp instructions per SM and clock)"}), flush=True)
        return
    if args.precision:
        if rank == 0:
            print(json.dumps(precision_report(S, I)), flush=True)
        return
    if args.workload in ("batched32", "batched32_mala"):
        return run_batched(args, world, rank, local, mala=args.workload == "batched32_mala")
    w = I.WORKLOADS[args.workload]
    if args.particles:
        import dataclasses
        J_, N_ = (int(v) for v in args.particles.split(","))
        w = dataclasses.replace(w, J=J_, N=N_)
    y = w.data()
    m = S.model_egarch(w.K, w.I, w.gamma)
    mean, sd, lo = S.model_prior(m)
    th0 = I.draw_prior(mean, sd, lo, w.P, seed=w.prior_seed + 1000 * rank)
    prec = S.FP32 if w.precision == "f32" else S.FP64
    mala = w.mutation == "mala"
    cfg = S.config_default(J=w.J, N=w.N, precision=prec, rbar=w.rbar, kappa=w.kappa, seed=1 + rank,
                           mutation=S.MALA if mala else S.RW, acc_target=MALA_TARGET if mala else 0.25,
                           tempering=S.POWER if args.tempering == "power" else S.DATA)
    stream = torch.cuda.Stream()
    th0_dev = torch.as_tensor(np.ascontiguousarray(th0.T), device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        ctx = S.init(m, cfg, y, th0, stream=stream.cuda_stream)
    if args.launch_shape:
        ppt, thr = (int(v) for v in args.launch_shape.split(","))
        ctx.set_launch_shape(ppt, thr)
        shape = (ppt, thr, None)
    else:
        shape = ctx.autotune(iters=2) if not mala else (1, 128, None)
    seed_of = lambda k: 1 + rank + 7919 * k
    # ALU pipe rates of this device (a few ms of microbenchmark kernels)
    rates = {k: v for k, v in S.peaks(stream.cuda_stream).items() if k != "sms"}

    def one_run(k):
        ctx.reset(th0_dev, seed_of(k), theta0_on_device=True)
        ctx.run(args.cycles)
        lml = ctx.log_ml()
        return ctx.totals(), lml

    for k in range(args.warmup):
        one_run(k)
    torch.cuda.synchronize()

    # events around the first mutation launch of every M phase only: an event
    # recorded between two kernels linked by programmatic dependent launch
    # serialises them, so timing every launch would slow the step it measures
    # data tempering: every launch is timed (their lengths t_l differ), which
    # gives up the programmatic dependent launches' overlap
    ctx.profile(2 if args.tempering == "power" else 1)
    ctx.mutate_time(reset=True)
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = S.launch_count()
    clocks.start()
    ev = []
    evals_total, cycles, msteps = 0.0, [], []
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        (cyc, ms, evl), lml = one_run(args.warmup + k)
        e1.record(stream)
        ev.append((e0, e1))
        evals_total += evl
        cycles.append(cyc)
        msteps.append(ms)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    launches = S.launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_total = sum(step_ms) / 1e3
    mut_ms, mut_n = ctx.mutate_time(reset=True)
    t_total, evals_all = combine_ranks(t_total, evals_total, world, device="cuda")
    value = evals_all / t_total

    # ---- end to end through the public API from host buffers ----
    e2e = None
    if not args.no_e2e:
        e2e_time, e2e_evals, h2d, d2h = 0.0, 0.0, 0, 0
        # the initial particles live in pinned host memory (a view of it is
        # what smc_init copies from)
        th0_host = torch.from_numpy(np.ascontiguousarray(th0)).pin_memory().numpy()
        for k in range(args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            c2 = S.init(m, cfg, y, th0_host, stream=stream.cuda_stream)
            c2.set_launch_shape(shape[0], shape[1])
            c2.run(args.cycles)
            c2.log_ml()
            cyc2, ms2, evl2 = c2.totals()
            hb, db = c2.transfer_bytes()
            c2.close()
            e2e_time += time.perf_counter() - t0
            e2e_evals += evl2
            h2d, d2h = hb, db
        e2e = {"value": e2e_evals / e2e_time, "unit": "particle*obs lik evals/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    # ---- roofline of the dominant kernel (fused RW mutate) ----
    # DRAM bytes (read + write) of one mutate launch from an ncu capture of the
    # same kernel, workload and launch shape (profiles/); None where no capture
    # of the current kernel exists.
    traffic = MUTATE_TRAFFIC.get((args.workload, shape[0], shape[1])) if not mala else None
    mhz, src = sm_max_mhz()
    paired = shape[0] == 2
    # MALA's bound counts its forward, recomputation and reverse sweep per
    # evaluation (mala_ops_per_eval).  The pipe rates per SM and clock are
    # those the microbenchmark measured on this device before the timed region
    # (smc_peaks), at the maximum SM clock; the nominal rates give a second bound.
    peak, pipe = alu_peak_evals(w.K, w.I, w.gamma, SM_COUNT_GB300, mhz, paired, mala, rates=rates)
    peak_nom, pipe_nom = alu_peak_evals(w.K, w.I, w.gamma, SM_COUNT_GB300, mhz, paired, mala)
    avg_launch_s = (mut_ms / mut_n) / 1e3 if mut_n else float("nan")
    if args.tempering == "power":
        achieved = w.P * w.T / avg_launch_s if mut_n else float("nan")
    else:   # every launch timed: all M-phase evaluations over their summed time
        achieved = evals_total / (mut_ms / 1e3) if mut_n else float("nan")
    fp32_ops, mufu_ops = (mala_ops_per_eval if mala else alu_ops_per_eval)(w.K, w.I, w.gamma)
    roof = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Geval/s",
            "frac": achieved / peak, "traffic": traffic,
            "traffic_unit": "DRAM bytes read + written per launch (ncu); the kernel is ALU-bound: "
                            "traffic / launch time is under 1% of the HBM bandwidth",
            "pipe": pipe,
            "peak_source": (f"pipe rates measured by smc_peaks on this device x {src} SM clock "
                            f"{mhz:.0f} MHz x {SM_COUNT_GB300} SMs"),
            "measured_rates": rates, "peak_nominal": peak_nom / 1e9, "pipe_nominal": pipe_nom,
            "frac_nominal": achieved / peak_nom,
            "ops_per_eval": {"fp32": fp32_ops, "mufu": mufu_ops},
            "kernel": (f"k_mutate_mala<GradEgarch<float,{w.K},{w.I}>>" if mala
                       else f"k_mutate_x2<{w.K},{w.I}>" if paired
                       else f"k_mutate<PolicyEgarchF32<{w.K},{w.I}>>"), "avg_launch_ms": avg_launch_s * 1e3,
            "launches": int(sum(msteps)), "timed_launches": mut_n,
            "timed": ("first mutation launch of every M phase (CUDA events)" if args.tempering == "power"
                      else "every mutation launch (CUDA events)"),
            "share_of_step": avg_launch_s * sum(msteps) / t_total if t_total and mut_n else None,
            "launch_shape": {"particles_per_thread": shape[0], "threads_per_block": shape[1],
                             "autotune_ms_per_iteration": shape[2]}}
    if clk.get("sm_mhz"):
        roof["frac_at_median_clock"] = achieved / alu_peak_evals(w.K, w.I, w.gamma, SM_COUNT_GB300, clk["sm_mhz"],
                                                                 paired, mala, rates=rates)[0]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_leg(w, y)
    eq = None
    if (rank == 0 and not args.no_equal_nse and args.cycles == 0 and args.tempering == "power"
            and w.name in ("egarch22_T5000", "egarch34_T20000")):
        eq = equal_nse_comparison(S, w, y, th0, stream, args.equal_nse_seeds, shape=shape)
        eq["batched"] = batched_equal_nse(S, I, stream)
        # MALA at the K=2, I=2, T=5000 shape with J = 64 x N = 4096 particles,
        # against the FP32 and the (one-seed) FP64 random walk
        w3 = I.WORKLOADS["egarch22_T5000_mala"]
        y3 = w3.data()
        m3 = S.model_egarch(w3.K, w3.I, w3.gamma)
        th3 = I.draw_prior(*S.model_prior(m3), w3.P, seed=w3.prior_seed)
        eq["egarch22_T5000_J64xN4096"] = equal_nse_comparison(S, w3, y3, th3, stream, args.equal_nse_seeds,
                                                              fp64_seeds=1)

    if rank == 0:
        line = {"metric": "M-phase particle*obs lik evals/s", "value": value,
                "unit": "particle*obs lik evals/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": w.precision,
                "data": "synthetic",
                "config": {"workload": w.name, "K": w.K, "I": w.I, "T": w.T, "J": w.J, "N": w.N,
                           "precision": ("fp32 recursion, fp64 accumulators" if w.precision == "f32"
                                         else "fp64 throughout"), "tempering": args.tempering,
                           "sampler": w.mutation, "stop_rule": f"deterministic Rbar={w.rbar} kappa={w.kappa}",
                           "cycles_per_run": cycles, "metropolis_steps_per_run": msteps,
                           "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}"},
                "clocks": {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
                "e2e": e2e, "gpu_launches": int(launches), "roofline": roof, "cpu_baseline": cpu,
                "equal_nse": eq, "wall_s": wall}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def run_batched(args, world, rank, local, mala=False):
    """32 datasets (T ~ U{500..10000}, K ~ U{1,2,3}, I ~ U{1..4}), J=16 x N=1024
    each, advanced together: one persistent M-phase kernel per Metropolis
    iteration, replayed from a captured CUDA graph; tile size autotuned.
    mala=True: the same batch with the MALA mutation (FP32 + adjoint +
    batched); the metric then counts each likelihood-and-gradient evaluation
    once."""
    import numpy as np
    import torch
    from paper_1304_4334_gb300 import inputs as I
    from paper_1304_4334_gb300 import smc as S

    ws = I.batched_workloads(n=32, seed=40 + rank, J=16, N=1024)
    models, cfgs, ys, ths = [], [], [], []
    for k, w in enumerate(ws):
        m = S.model_egarch(w.K, w.I, True)
        mean, sd, lo = S.model_prior(m)
        models.append(m)
        cfgs.append(S.config_default(J=w.J, N=w.N, precision=S.FP32, seed=100 + k,
                                     mutation=S.MALA if mala else S.RW, acc_target=MALA_TARGET if mala else 0.25))
        ys.append(w.data())
        ths.append(I.draw_prior(mean, sd, lo, w.P, seed=w.prior_seed))
    stream = torch.cuda.Stream()
    th_dev = [torch.as_tensor(np.ascontiguousarray(t.T), device="cuda") for t in ths]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    b = S.Batch(models, cfgs, ys, ths, stream=stream.cuda_stream)
    tune_ms = b.autotune(iters=2)

    def one(k):
        b.reset(th_dev, 1000 + 7919 * k)
        b.run(args.cycles)
        return b.totals()

    for k in range(args.warmup):
        one(k)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    launches0 = S.launch_count()
    clocks.start()
    evals, times, cyc = 0.0, [], []
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e, ms, cy = one(args.warmup + k)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        evals += e
        cyc.append(cy)
    clk = clocks.stop()
    launches = S.launch_count() - launches0
    t = sum(times)
    if rank == 0:
        line = {"metric": "M-phase particle*obs lik evals/s", "value": evals / t,
                "unit": "particle*obs lik evals/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "batched32_mala" if mala else "batched32", "datasets": 32, "J": 16, "N": 1024,
                           "sampler": "mala" if mala else "rw",
                           "T": [w.T for w in ws], "KI": [[w.K, w.I] for w in ws],
                           "tile": b.tile, "autotune_ms_per_iteration": tune_ms,
                           "cycles_per_run": cyc, "l2": "flushed between steps (256 MB write)"},
                "clocks": {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
                "gpu_launches": int(launches)}
        print(json.dumps(line), flush=True)
    b.close()


if __name__ == "__main__":
    main()
