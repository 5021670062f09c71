"""Benchmark: seconds to RMSE <= eps on E[outflux] with FMG-MLMC on one GB300.

Workload (default): five MLMC levels 16x16 .. 256x256, 128 KL modes of the
exponential covariance (sigma^2 = 1, lambda = 0.3), Case II boundary data
(p = 1 west, 0 east), FMG from 4x4 with 2 V(2,2) cycles per stage, MC points,
sample sizes from the optimal rule for RMSE 1e-3.  One step = one complete
mlmc_estimate call (points, KL synthesis, FMG solves, level sums, controller
rounds) from an empty estimator to RMSE <= eps; the KL basis is resident in
HBM before the timed region.  L2 is flushed (a 512 MiB write) between steps.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
a bounded sample of the same workload instead.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="fmg_mlmc5")
    ap.add_argument("--eps", type=float, default=None)
    ap.add_argument("--qmc", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0,
                    help="budget of the oracle's bounded timing sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--form", default="mixed_surrogate_batched",
                    choices=["mixed_surrogate", "mixed_surrogate_batched", "mixed", "fp64_converged",
                             "fp64_fmg2"])
    ap.add_argument("--no-standard-leg", action="store_true",
                    help="skip the FMG-MLMC vs standard-MLMC cost comparison")
    ap.add_argument("--no-uneven-leg", action="store_true",
                    help="skip the uneven-batch leg (4096 samples over 64x64 .. 1024x1024)")
    ap.add_argument("--only-chosen", action="store_true", help="skip timing the other forms")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--no-qmc-leg", action="store_true", help="skip timing the randomized-QMC estimator")
    ap.add_argument("--no-c5-leg", action="store_true",
                    help="skip the large high-contrast case (6 levels 64x64 .. 2048x2048, 1024 modes, "
                         "sigma^2 = 2, lambda = 0.1, RMSE 5e-4) in the chosen form and in plain FP64 "
                         "(run on one GPU only)")
    ap.add_argument("--c5-steps", type=int, default=1, help="timed estimates per form in the large case")
    ap.add_argument("--train-epochs", type=int, default=None,
                    help="epochs of the surrogate's training inside each step (default: SURROGATE_TRAIN)")
    ap.add_argument("--train-n", type=int, default=None,
                    help="training pairs of the surrogate (level-0 solves) inside each step (default: SURROGATE_TRAIN)")
    ap.add_argument("--surrogate-cost", type=float, default=None,
                    help="cost of an S sample relative to a level-0 sample in the allocation (default: SURROGATE_COST)")
    ap.add_argument("--train-tol", type=float, default=None,
                    help="tolerance of the training pairs' level-0 solves (default: SURROGATE_TRAIN)")
    ap.add_argument("--train-batch", type=int, default=None,
                    help="minibatch of the surrogate's training (default: SURROGATE_TRAIN)")
    ap.add_argument("--train-lr", type=float, default=None,
                    help="peak Adam learning rate of the surrogate's training (default: SURROGATE_TRAIN)")
    ap.add_argument("--ir-cycles", type=int, default=None,
                    help="FP32 V-cycles per FP64 residual test in the mixed forms (default: MIXED_IR_CYCLES)")
    ap.add_argument("--detail-out", default=None,
                    help="write the full record (every leg, every kernel family) to this JSON file")
    ap.add_argument("--kernel-case", default=None, choices=sorted(KERNEL_CASES),
                    help="run one small isolated kernel case (for a profiler) instead of the benchmark")
    return ap.parse_args()


METRIC = "seconds to RMSE<=1e-3 on E[outflux], plain FP64 vs chosen form; smoother HBM GB/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p["hbm_gbs"], p.get("bf16_tflops"), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ oracle
def oracle_params(converged):
    from oracle import lib as olib
    return olib.params(converged=converged, tol=SOLVE_TOL, max_cycles=300)


def oracle_level_seconds(wl, budget_s, converged):
    """Seconds per sample of the oracle on each level, on all host cores,
    from a bounded sample (about budget_s seconds in total)."""
    from oracle import kl as okl
    from oracle import mlmc as omlmc
    cores = os.cpu_count() or 1
    basis = okl.KLBasis(wl.n_ref, wl.M, wl.sigma2, wl.lam, q=32 if wl.M <= 128 else 0)
    s = omlmc.FMGSampler(wl.levels, basis, seed=wl.seed, prm=oracle_params(converged), nthreads=cores)
    per = []
    share = budget_s / len(wl.levels)
    counts = []
    for l, n in enumerate(wl.levels):
        k = max(cores, 16)
        t0 = time.perf_counter()
        s(l, 0, k)
        dt = time.perf_counter() - t0
        # grow the sample to about `share` seconds (at most 64x the first)
        k2 = int(min(64 * k, max(k, k * share / max(dt, 1e-6))))
        t0 = time.perf_counter()
        s(l, k, k2)
        dt = time.perf_counter() - t0
        per.append(dt / k2)
        counts.append(k2)
    return np.array(per), cores, counts


def oracle_level_seconds_1core(wl, budget_s, converged):
    """Seconds per sample of the oracle on one host core, per level, from a
    bounded sample (about budget_s seconds in total)."""
    from oracle import kl as okl
    from oracle import mlmc as omlmc
    basis = okl.KLBasis(wl.n_ref, wl.M, wl.sigma2, wl.lam, q=32 if wl.M <= 128 else 0)
    s = omlmc.FMGSampler(wl.levels, basis, seed=wl.seed, prm=oracle_params(converged), nthreads=1)
    per, counts = [], []
    share = budget_s / len(wl.levels)
    for l in range(len(wl.levels)):
        k = 2
        t0 = time.perf_counter()
        s(l, 0, k)
        dt = time.perf_counter() - t0
        k2 = int(min(256, max(2, k * share / max(dt, 1e-6))))
        t0 = time.perf_counter()
        s(l, k, k2)
        per.append((time.perf_counter() - t0) / k2)
        counts.append(k2)
    return np.array(per), counts


def oracle_surrogate_seconds(M, budget_s=4.0):
    """Seconds of the oracle network (FP64, numpy) per S evaluation and per
    training step (batch 256: loss, gradients, Adam), from a bounded sample."""
    from oracle import mlp as omlp
    r = W.rng(tag=900)
    params = omlp.init_params(M, lambda n: r.uniform(size=n))
    X = r.standard_normal((8192, M))
    t0 = time.perf_counter()
    omlp.forward(params, X, rounding=True)
    per_eval = (time.perf_counter() - t0) / len(X)
    opt = omlp.Adam(params, lr=1e-3)
    t = r.standard_normal(256)
    k, t0 = 0, time.perf_counter()
    while k < 4 or (time.perf_counter() - t0 < budget_s / 2 and k < 64):
        _, g = omlp.mse_loss_and_grad(params, X[:256], t, rounding=True)
        params = opt.step(params, g)
        k += 1
    per_step = (time.perf_counter() - t0) / k
    return per_eval, per_step, k


# ------------------------------------------------------------------ native
def flush_l2(buf):
    buf.fill_(1.0)


# refined stages stop at ||b - A p|| <= 1e-12 ||b|| or an outflux change of at
# most 1e-10 |Q| between tests: per-sample outflux within 1e-8 of the fully
# converged FP64 solution on every grid up to 1024 x 1024
SOLVE_TOL, SOLVE_QTOL = 1e-12, 1e-10

FORMS = {
    # the mixed form plus the surrogate control-variate level below 16x16; the
    # network is trained inside every timed step on level-0 samples the
    # solver produces (training data, training and estimate all timed)
    "mixed_surrogate": dict(precision=1, converged=True, surrogate=True),
    # the same, each round's solves of all levels as one uneven batch (one CUDA graph)
    "mixed_surrogate_batched": dict(precision=1, converged=True, surrogate=True, batched=True),
    # FP32 smoothing/transfers/coarsest solve inside FP64 iterative refinement
    # of the stages giving Q^c and Q^f (stopping rule above)
    "mixed": dict(precision=1, converged=True, surrogate=False),
    # the same converged solves, every step in FP64
    "fp64_converged": dict(precision=0, converged=True, surrogate=False),
    # the paper's fixed schedule: 2 V(2,2) cycles per FMG stage, FP64
    "fp64_fmg2": dict(precision=0, converged=False, surrogate=False),
}

# surrogate training: 20480 (xi, Q_0) pairs, batch 1024, 20 epochs (400 steps),
# Adam 4e-3 cosine.  Measured on GB300 (headline form, 6 FP32 V-cycles per
# test, seconds per estimate): 12 epochs 0.1322 (corr 0.9969), 16 epochs
# 0.1316 (0.9979), 20 epochs 0.1312 (0.9983), 24 epochs 0.1325 (0.9987);
# pairs x epochs 10240 x 30 0.1316, 14336 x 20 0.1291, 28672 x 14 0.1261
# against 0.1257 for 20480 x 20.  The pairs' level-0 solves stop at 1e-6
# (residual and outflux change): 0.1226 against 0.1244 at the estimator's
# 1e-12 / 1e-10, with the same fit (corr 0.99835)
SURROGATE_TRAIN = dict(n_train=20480, epochs=20, lr=4e-3, seed=7, batch=1024, target_tol=1e-6)
# kernels in one captured training step (batch gather, three forward GEMMs,
# output layer with its gradient, five backward GEMMs, four row sums, Adam)
TRAIN_STEP_KERNELS = 15


# cost of one S-level sample relative to one level-0 sample in the optimal
# allocation: 0.027, the ratio surrogate_cost() below measured on GB300 with
# earlier inference kernels (it now measures about 0.006, reported beside the
# estimate).  A fixed ratio keeps the schedule independent of timing; with
# the S level beside the solves the choice barely matters (seconds per
# estimate on GB300: 0.027 0.1225, 0.015 0.1218, 0.008 0.1222, 0.005 0.1222)
SURROGATE_COST = 0.027


def surrogate_cost(torch, ctx):
    """Device seconds of one S-level sample over one level-0 sample."""
    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b)
    sums = ctx.new_sums()
    ns, n0 = 1 << 20, 1 << 16
    t_s = timed(lambda: ctx.surrogate_eval_mc(12, 0, ns)) / ns
    t_0 = timed(lambda: ctx.mlmc_sample_level(0, 0, n0, sums=sums[0])) / n0
    return t_s / t_0


# FP32 V-cycles per FP64 residual test in the mixed forms' refinement loops:
# measured on GB300 (headline form, 12 training epochs, seconds per
# estimate) 0.1368 with 3, 0.1336-0.1342 with 4, 0.1337 with 5, 0.1322-0.1324
# with 6; with 16 epochs 0.1316 with 6 and 0.1401 with 8 (fewer FP64
# residual tests against FP32 cycles spent on samples already converged)
MIXED_IR_CYCLES = 6
IR_CYCLES = [MIXED_IR_CYCLES]


def make_ctx(fm, wl, rank, form):
    f = FORMS[form]
    return fm.Context(len(wl.levels), wl.levels[0], wl.M, sigma2=wl.sigma2, lam=wl.lam, pW=wl.pW,
                      pE=wl.pE, nu0=wl.nu0, nu1=wl.nu1, nu2=wl.nu2, n_coarsest=wl.n0,
                      n_shifts=wl.n_shifts, seed=wl.seed + 7919 * rank, precision=f["precision"],
                      converged=f["converged"], tol=SOLVE_TOL, qtol=SOLVE_QTOL, max_cycles=200,
                      ir_cycles=IR_CYCLES[0] if f["precision"] == 1 else 0)


# DRAM read + write of one FP32 strip call (two red-black sweeps) per cell:
# ncu's dram__bytes_read.sum + dram__bytes_write.sum of one k_rbgs_strip
# launch over 64 Mi cells (1024 samples of 256 x 256, synthetic operands)
# was 1.72 GB, i.e. 25.6 B per cell against the kernel's 24 algorithmic
# bytes per cell (read p, b, D, Te, Tn once, write p once)
STRIP_DRAM_BYTES_PER_CELL_F32 = 1.72e9 / (64 << 20)
STRIP_ALG_BYTES_PER_CELL_F32 = 24.0

# FP64 rate of GB300 (nominal, TFLOP/s): the denominator of the FP64 part of
# the resident kernel's ALU view
FP64_PEAK_TFLOPS = 1.25

# randomized QMC (Algorithm 2): 32 points per shift and level to start, 16 digital shifts
QMC_PILOT = 32


def time_estimates(torch, ctx, eps, args, wl, steps, warmup, flush, profile=False, clocks=None,
                   dist=None, form="mixed", qmc=None):
    sur = FORMS[form]["surrogate"]
    cost = measured = None
    if sur:
        ctx.surrogate_train(**SURROGATE_TRAIN)
        # the allocation uses the fixed ratio so that the sample schedule does
        # not depend on timing (a profiler slows the two legs differently);
        # the live ratio is reported beside it
        measured = surrogate_cost(torch, ctx)
        cost = SURROGATE_COST

    qmc = args.qmc if qmc is None else qmc
    n_pilot = wl.n_pilot if not qmc else QMC_PILOT

    batched = FORMS[form].get("batched", False)

    def estimate():
        if not sur:
            return ctx.mlmc_estimate(eps, qmc=qmc, n_pilot=n_pilot, batched=batched)
        # the training steps run on the network's stream beside the estimate's
        # first round (its solves need no network); the surrogate level and
        # level 0 wait for the last step on the device
        ctx.surrogate_train(**SURROGATE_TRAIN, async_run=True)
        r = ctx.mlmc_estimate(eps, qmc=qmc, n_pilot=n_pilot, surrogate=True, surrogate_cost=cost,
                              batched=batched)
        r["train"] = ctx.surrogate_train_finish()
        r["surrogate_cost"] = cost
        r["surrogate_cost_measured"] = measured
        return r

    for _ in range(warmup):
        estimate()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    if profile:
        ctx.profile_begin()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    times, results = [], []
    for _ in range(steps):
        flush_l2(flush)
        torch.cuda.synchronize()
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record()
        r = estimate()
        stop.record()
        torch.cuda.synchronize()
        times.append(start.elapsed_time(stop) / 1e3)
        results.append(r)
    prof = ctx.profile_end() if profile else None
    clk = clocks.stop() if clocks else None
    return times, results, prof, clk


def _case_resident(torch, fm, level, S):
    """S level-`level` samples of the five-level workload in the mixed
    converged form, solved three times on the resident schedule."""
    wl = W.WORKLOADS["fmg_mlmc5"]
    ctx = make_ctx(fm, wl, 0, "mixed")
    ctx.kl_basis_build(q=wl.kl_q)
    K = ctx.kl_field_batch(level, ctx.mc_points(level, 0, S))
    for _ in range(3):
        qf, qc, _ = ctx.fmg_solve_batch(K, kernel=2)
    torch.cuda.synchronize()
    ctx.sync()
    print("kernel case: %d samples of %dx%d, mean Q^f %.6f" % (S, K.shape[-1], K.shape[-1], float(qf.mean())))
    ctx.close()


def _case_levelwise(torch, fm, level, S):
    """S level-`level` samples of the five-level workload in the mixed
    converged form, solved three times on the level-wise schedule."""
    wl = W.WORKLOADS["fmg_mlmc5"]
    ctx = make_ctx(fm, wl, 0, "mixed")
    ctx.kl_basis_build(q=wl.kl_q)
    K = ctx.kl_field_batch(level, ctx.mc_points(level, 0, S))
    for _ in range(3):
        qf, qc, _ = ctx.fmg_solve_batch(K, kernel=1)
    torch.cuda.synchronize()
    ctx.sync()
    print("kernel case: %d samples of %dx%d, mean Q^f %.6f" % (S, K.shape[-1], K.shape[-1], float(qf.mean())))
    ctx.close()


def _case_surrogate_mc(torch, fm, n):
    """S for n MC samples by the fused inference kernel (a network of the
    five-level workload's size with seeded random parameters), three times."""
    wl = W.WORKLOADS["fmg_mlmc5"]
    ctx = make_ctx(fm, wl, 0, "mixed_surrogate")
    ctx.kl_basis_build(q=wl.kl_q)
    r = np.random.default_rng(5)
    ctx.surrogate_set_params((r.random(ctx.surrogate_param_count()) - 0.5).astype(np.float32) * 0.1, mu=1.0, sd=0.5)
    for k in range(3):
        s = ctx.surrogate_eval_mc(12, k * n, n)
    torch.cuda.synchronize()
    ctx.sync()
    print("kernel case: %d surrogate evaluations, mean %.6f" % (n, float(s.mean())))
    ctx.close()


# one small isolated launch pattern per case, for a profiler (-k/-c select it)
KERNEL_CASES = {
    "surrogate_mc_fused": lambda torch, fm: _case_surrogate_mc(torch, fm, 1 << 20),
    "fmg_levelwise_mixed256": lambda torch, fm: _case_levelwise(torch, fm, 4, 300),
    "fmg_resident_mixed16": lambda torch, fm: _case_resident(torch, fm, 0, 65536),
    "fmg_resident_mixed32": lambda torch, fm: _case_resident(torch, fm, 1, 16384),
    "fmg_resident_mixed64": lambda torch, fm: _case_resident(torch, fm, 2, 4096),
}


UNEVEN_COUNTS = [3075, 769, 192, 48, 12]   # 4096 samples, N_l ~ 4^-l (optimal ratio for beta ~ 2)


def uneven_leg(torch, fm, flush):
    """4096 samples over 64x64 .. 1024x1024 (256 KL modes, tensor-core BF16x3
    fields): the FP32-smoothing / FP64-refinement solves level after level
    (one fmg_solve_batch per grid) against one uneven batch (one CUDA graph),
    both after autotuning the smoother launch shapes."""
    wl = W.WORKLOADS["batched4096"]
    c = fm.Context(len(wl.levels), wl.levels[0], wl.M, sigma2=wl.sigma2, lam=wl.lam, pW=wl.pW, pE=wl.pE,
                   n_shifts=wl.n_shifts, seed=wl.seed, precision=1, converged=True, tol=SOLVE_TOL,
                   qtol=SOLVE_QTOL, max_cycles=200)
    t0 = time.perf_counter()
    c.kl_basis_build(q=wl.kl_q)
    basis_s = time.perf_counter() - t0
    Ks = []
    for l, cnt in enumerate(UNEVEN_COUNTS):
        xi = c.mc_points(l, 0, cnt)
        Ks.append(c.kl_field_batch(l, xi))
    tune = c.autotune(n_min=8, n_max=wl.levels[-1])
    torch.cuda.synchronize()

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush_l2(flush)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            out = fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b) / 1e3)
        return float(np.median(ts)), out

    t_seq, seq = timed(lambda: [c.fmg_solve_batch(K) for K in Ks])
    t_unv, unv = timed(lambda: c.solve_uneven(Ks))
    same = all(torch.equal(a[0], b[0]) for a, b in zip(seq, unv))
    n_total = sum(UNEVEN_COUNTS)
    out = {"workload": wl.name, "levels": wl.levels, "counts": UNEVEN_COUNTS, "kl_modes": wl.M,
           "kl": "tcgen05 BF16x3 (field error <= 5e-5)", "form": "FP32 smoothing, FP64 refinement (tol %g, "
           "outflux change %g)" % (SOLVE_TOL, SOLVE_QTOL), "seconds_per_level_calls": t_seq, "seconds_uneven_graph": t_unv,
           "samples_per_s_per_level_calls": n_total / t_seq, "samples_per_s_uneven_graph": n_total / t_unv,
           "speedup": t_seq / t_unv, "identical_results": bool(same), "graph": c.uneven_stats(),
           "kl_basis_build_s": basis_s,
           "autotune": [{k: e[k] for k in ("n", "tile", "threads", "ms_best", "ms_default")} for e in tune]}
    c.close()
    return out


# the large case's own settings of the chosen form, measured on GB300: 12
# training epochs and 4 FP32 V-cycles per FP64 test take 7.11 s per estimate,
# the five-level workload's 20 epochs and 6 cycles 7.65 s
C5_TRAIN = dict(SURROGATE_TRAIN, epochs=12)
C5_IR_CYCLES = 4


def c5_leg(torch, fm, flush, steps):
    """The large high-contrast case: six levels 64x64 .. 2048x2048, Matern
    nu = 1/2 with sigma^2 = 2 and lambda = 0.1, 1024 KL modes, RMSE 5e-4.
    Chosen form: randomized QMC (16 shifted Sobol' point sets), the surrogate
    level below 64x64, FP32 V-cycles in FP64 refinement, each round's solves
    as one uneven batch, and the energy-optimal correction step (the plain
    V-cycle diverges on some fields of this contrast).  Beside it the plain
    FP64 form: every step in FP64, converged stages, energy step, the same
    QMC estimator without the surrogate.  The KL basis (Nystrom, q = 96,
    interpolated on the tensor cores) is built once, outside the timed
    region, and handed to the second context."""
    wl = W.WORKLOADS["contrast6"]
    out = {"workload": wl.name, "levels": wl.levels, "kl_modes": wl.M, "sigma2": wl.sigma2, "lambda": wl.lam,
           "eps": wl.eps, "sampler": "qmc", "shifts": wl.n_shifts}

    def make(precision):
        return fm.Context(len(wl.levels), wl.levels[0], wl.M, sigma2=wl.sigma2, lam=wl.lam, n_shifts=wl.n_shifts,
                          seed=wl.seed, precision=precision, converged=True, tol=SOLVE_TOL, qtol=SOLVE_QTOL,
                          max_cycles=300, energy_step=True, ir_cycles=C5_IR_CYCLES if precision == 1 else 0)

    c = make(1)
    t0 = time.perf_counter()
    theta, captured = c.kl_basis_build(q=96)
    torch.cuda.synchronize()
    out["kl_basis_build_s"] = time.perf_counter() - t0
    out["captured_variance"] = captured

    def run(ctx, sur, batched, warmup=1):
        ts, rs = [], []
        for step in range(steps + warmup):   # the first `warmup` are not timed
            flush_l2(flush)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            if sur:
                ctx.surrogate_train(**C5_TRAIN, async_run=True)
                r = ctx.mlmc_estimate(wl.eps, qmc=True, n_pilot=QMC_PILOT, surrogate=True,
                                      surrogate_cost=SURROGATE_COST, batched=batched)
                r["train_corr"] = ctx.surrogate_train_finish()["corr"]
            else:
                r = ctx.mlmc_estimate(wl.eps, qmc=True, n_pilot=QMC_PILOT, batched=batched)
            b.record()
            torch.cuda.synchronize()
            if step >= warmup:
                ts.append(a.elapsed_time(b) / 1e3)
                rs.append(r)
        r = rs[-1]
        return {"value": float(np.mean(ts)), "unit": "s", "estimate": float(r["estimate"]),
                "rmse_estimate": float(np.sqrt(r["var_estimator"])), "N_per_level_per_shift": [int(x) for x in r["N"]],
                "rounds": int(r["rounds"]), "N_s_per_shift": int(r.get("N_s", 0)),
                "train_corr": r.get("train_corr")}

    out["chosen"] = run(c, True, True)
    B = c.kl_basis_get()
    c.close()
    c2 = make(0)
    c2.kl_basis_set(B)
    del B
    torch.cuda.empty_cache()
    # the plain form's estimate takes about 40 s: timed on its first call
    # (no warm-up; its set-up is a few allocations against that time)
    out["plain_fp64"] = run(c2, False, False, warmup=0)
    c2.close()
    out["speedup_vs_plain_fp64"] = out["plain_fp64"]["value"] / out["chosen"]["value"]
    out["difference_in_sigmas"] = abs(out["chosen"]["estimate"] - out["plain_fp64"]["estimate"]) / np.hypot(
        out["chosen"]["rmse_estimate"], out["plain_fp64"]["rmse_estimate"])
    return out


def standard_mlmc_leg(torch, ctx, wl, N, flush, samples=1000):
    """The paper's cost claim (Sec. 1): FMG-MLMC takes Q^c_l from the FMG
    hierarchy of the level-l solve, where standard MLMC solves the coarse
    problem of the same sample again.  With nested field points that coarse
    problem is the level-(l-1) field of the same xi, so its solve is timed
    here on the same samples, and its outflux checked against the by-product.
    Standard MLMC's two solves give one QoI each, so both run without the
    Q^c output (the solver then leaves their coarse stages unrefined); the
    FMG-MLMC solve of level l >= 1 refines its coarse stage for Q^c.  The
    saving is 1 - (FMG-MLMC solver time) / (standard MLMC solver time) at the
    estimate's N_l (level 0: one solve without Q^c in either)."""
    out = {"levels": [], "samples": samples}
    t_f, t_fs, t_c, q_diff, k_diff = [], [], [], [], [0.0]

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        flush_l2(flush)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        r = fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3, r

    for l in range(len(wl.levels)):
        xi = ctx.mc_points(l, 0, samples)
        Kf = ctx.kl_field_batch(l, xi)
        ts, _ = timed(lambda: ctx.fmg_solve_batch(Kf, want_qc=False))
        t_fs.append(ts / samples)
        if l == 0:
            t_f.append(ts / samples)
            t_c.append(0.0)
            q_diff.append(0.0)
            continue
        tf, (qf, qc, _) = timed(lambda: ctx.fmg_solve_batch(Kf))
        t_f.append(tf / samples)
        Kc = ctx.kl_field_batch(l - 1, xi)
        inj = Kf[:, ::2, ::2]
        k_diff.append(float(((Kc - inj).abs() / inj.abs()).max()))
        tc, (qc_std, _, _) = timed(lambda: ctx.fmg_solve_batch(Kc, want_qc=False))
        t_c.append(tc / samples)
        q_diff.append(float(((qc_std - qc).abs() / qc.abs()).max()))
    N = np.asarray(N, float)
    fmg_cost = float(np.sum(N * np.array(t_f)))
    std_cost = float(np.sum(N * (np.array(t_fs) + np.array(t_c))))
    out["levels"] = [{"n": n, "fmg_us_per_sample": 1e6 * a, "standard_fine_us_per_sample": 1e6 * b,
                      "standard_coarse_us_per_sample": 1e6 * c, "max_rel_diff_field": k, "max_rel_diff_qc": d}
                     for n, a, b, c, k, d in zip(wl.levels, t_f, t_fs, t_c, k_diff, q_diff)]
    out["saving_of_fmg_mlmc"] = 1.0 - fmg_cost / std_cost
    out["note"] = ("solver time weighted by the chosen form's N_l; the standard path's coarse field (the "
                   "level-(l-1) field of the same xi) against the injected fine field, and its separately "
                   "converged outflux against the FMG by-product")
    return out


def run_native(args, wl, eps):
    import torch
    import torch.distributed as dist

    import paper_1910_04727_gb300 as fm

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    fm.load_library()
    n_ref = wl.n_ref
    flush = torch.empty(512 << 20 >> 2, dtype=torch.float32, device="cuda")

    # replicas: each rank runs its own estimate with its own seed; the KL
    # basis is built once on the GPU and installed in every form's context
    ctx = make_ctx(fm, wl, rank, args.form)
    theta, captured = ctx.kl_basis_build(q=wl.kl_q)
    B_dev = ctx.kl_basis_get()
    # smoother launch shapes: the built-in defaults, which are fm_autotune's
    # choices measured on GB300 (the uneven-batch leg tunes live); a fixed
    # table keeps the schedule the same under a profiler

    clocks = ClockSampler(local)
    times, results, _, clk = time_estimates(torch, ctx, eps, args, wl, args.steps, args.warmup, flush,
                                            profile=False, clocks=clocks,
                                            dist=dist if world > 1 else None, form=args.form)
    t_total = float(np.sum(times))
    if world > 1:
        t = torch.tensor([t_total], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_total = float(t.item())
        dist.barrier()

    # kernel families of the same schedule: one more step with a CUDA event
    # pair around every launch (kept out of the timed steps above).  A batched
    # form's rounds run as one CUDA graph, timed as a whole; its kernels are
    # profiled in the per-level form of the same samples (the same kernels on
    # the same samples, one level after another instead of concurrently)
    prof_form = args.form[:-len("_batched")] if args.form.endswith("_batched") else args.form
    _, prof_results, prof, _ = time_estimates(torch, ctx, eps, args, wl, 1, 0, flush, profile=True,
                                              form=prof_form)
    same_schedule = [int(x) for x in prof_results[-1]["N"]] == [int(x) for x in results[-1]["N"]]

    # the other forms of the same estimate, timed the same way
    others = {}
    for form in FORMS:
        if form == args.form or args.only_chosen:
            continue
        c2 = make_ctx(fm, wl, rank, form)
        c2.kl_basis_set(B_dev)
        ts, rs, _, _ = time_estimates(torch, c2, eps, args, wl, max(1, min(args.steps, 3)), 1, flush,
                                      form=form)
        others[form] = {"value": float(np.mean(ts)), "unit": "s",
                        "estimate": float(np.mean([r["estimate"] for r in rs])),
                        "var_estimator": float(np.mean([r["var_estimator"] for r in rs])),
                        "N_per_level": [int(x) for x in rs[-1]["N"]],
                        "V_per_level": [float(x) for x in rs[-1]["V"]],
                        "level_seconds": [float(x) for x in rs[-1]["level_seconds"]]}
        c2.close()

    uneven = None if args.no_uneven_leg else uneven_leg(torch, fm, flush)
    c5 = None
    if not args.no_c5_leg and world == 1:
        try:
            c5 = c5_leg(torch, fm, flush, args.c5_steps)
        except Exception as e:   # reported in the record; the headline stands
            c5 = {"error": "%s: %s" % (type(e).__name__, e)}
            torch.cuda.synchronize()
    # FMG-MLMC against standard MLMC in the chosen form and in the paper's
    # fixed FP64 schedule (where the coarse stage is a plain FMG stage)
    standard = None
    if not args.no_standard_leg:
        standard = standard_mlmc_leg(torch, ctx, wl, results[-1]["N"], flush)
        c2 = make_ctx(fm, wl, rank, "fp64_fmg2")
        c2.kl_basis_set(B_dev)
        n_fixed = others["fp64_fmg2"]["N_per_level"] if "fp64_fmg2" in others else results[-1]["N"]
        standard["fixed_schedule"] = standard_mlmc_leg(torch, c2, wl, n_fixed, flush)
        c2.close()

    # the randomized-QMC estimator (16 shifted Sobol' point sets, doubling rule)
    # in the chosen form and in the plain FP64 form, timed the same way
    qmc_forms = {}
    for form in ([] if (args.qmc or args.no_qmc_leg) else [args.form, "fp64_converged"]):
        c2 = make_ctx(fm, wl, rank, form)
        c2.kl_basis_set(B_dev)
        ts, rs, _, _ = time_estimates(torch, c2, eps, args, wl, max(1, min(args.steps, 2)), 1, flush,
                                      form=form, qmc=True)
        qmc_forms[form] = {"value": float(np.mean(ts)), "unit": "s",
                           "estimate": float(np.mean([r["estimate"] for r in rs])),
                           "rmse_estimate": float(np.sqrt(np.mean([r["var_estimator"] for r in rs]))),
                           "N_per_level_per_shift": [int(x) for x in rs[-1]["N"]],
                           "shifts": wl.n_shifts, "rounds": int(rs[-1]["rounds"])}
        if FORMS[form]["surrogate"]:
            qmc_forms[form]["N_s_per_shift"] = int(rs[-1]["N_s"])
        c2.close()

    # end to end through the public API from pinned host memory: basis upload,
    # estimate, result read-back
    B_host = torch.empty((n_ref * n_ref, wl.M), dtype=torch.float64).pin_memory()
    ctx.kl_basis_get(B_host)
    ctx2 = make_ctx(fm, wl, rank, args.form)
    e2e_times, rounds = [], []
    sur = FORMS[args.form]["surrogate"]
    batched = FORMS[args.form].get("batched", False)
    for _ in range(0 if args.no_e2e else max(1, min(args.steps, 3))):
        flush_l2(flush)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx2.kl_basis_set_host_ptr(B_host.data_ptr())
        if sur:
            ctx2.surrogate_train(**SURROGATE_TRAIN, async_run=True)
            r = ctx2.mlmc_estimate(eps, qmc=args.qmc, n_pilot=wl.n_pilot, surrogate=True,
                                   surrogate_cost=results[-1]["surrogate_cost"], batched=batched)
            ctx2.surrogate_train_finish()
        else:
            r = ctx2.mlmc_estimate(eps, qmc=args.qmc, n_pilot=wl.n_pilot, batched=batched)
        e2e_times.append(time.perf_counter() - t0)
        rounds.append(r["rounds"])
    ctx2.close()
    h2d = B_host.numel() * 8
    d2h = int(np.mean(rounds) if rounds else 0) * len(wl.levels) * (wl.n_shifts if args.qmc else 1) * 128

    hbm, bf16, src = peaks()
    clk_mhz = (clk or {}).get("sm_mhz") or 2070.0
    peak_fp32_tf = 152 * 128 * 2 * clk_mhz * 1e6 / 1e12
    # dominant kernel family by event-timed device time in the profiled step
    # (the training graph is a whole replay loop, not one kernel)
    fam, st = max(((k, v) for k, v in prof.items() if k != "mlp_train_graph"), key=lambda kv: kv[1]["ms"])
    ach = st["bytes"] / (st["ms"] / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel": fam, "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(ach / hbm, 4), "traffic": None,
            "peak_source": src + " copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
            "launches": st["launches"], "avg_launch_ms": round(st["ms"] / st["launches"], 4)}
    if fam == "fmg_resident":
        # the whole FMG of a sample in shared memory.  achieved = the byte
        # model of the level-wise kernels (16 B a cell per FP32 sweep, 13 B
        # residual + restriction, 9 B correction, 20 B per FP64 residual test;
        # 310 B per finest cell for a fixed FMG with nu0 = 2) for the cycles
        # the kernel ran, over its event time.  Its own DRAM traffic is only K
        # in and the QoIs out.  The ALU view beside it: FP32 flops against
        # the FP32 FMA lanes, FP64 flops against GB300's FP64 rate.
        f64 = st.get("flops_fp64", 0.0)
        f32 = st["flops"] - f64
        sec = st["ms"] / 1e3
        roof["bytes_model"] = "streaming byte model of the level-wise kernels (310 B per finest cell for FMG nu0=2)"
        roof["alu"] = {"fp32_tflops": round(f32 / sec / 1e12, 3), "fp32_peak": round(peak_fp32_tf, 1),
                       "fp64_tflops": round(f64 / sec / 1e12, 4), "fp64_peak": FP64_PEAK_TFLOPS,
                       "fp64_frac": round(f64 / sec / 1e12 / FP64_PEAK_TFLOPS, 4)}
    # the HBM-bound kernels of the level-wise solves, beside the dominant one:
    # achieved = algorithmic bytes / event time over the profiled step
    hbm_kernels = {}
    for k in ("rbgs_strip", "residual_restrict", "rbgs_smoother", "rbgs_tile"):
        if k not in prof or prof[k]["ms"] <= 0:
            continue
        v = prof[k]
        a = v["bytes"] / (v["ms"] / 1e3) / 1e9
        e = {"achieved": round(a, 1), "frac": round(a / hbm, 4), "launches": v["launches"],
             "avg_launch_ms": round(v["ms"] / v["launches"], 4)}
        if k == "rbgs_strip" and FORMS[args.form]["precision"] == 1:
            e["traffic"] = round(v["bytes"] / v["launches"] * STRIP_DRAM_BYTES_PER_CELL_F32
                                 / STRIP_ALG_BYTES_PER_CELL_F32, 1)
            if fam == k:
                # DRAM bytes per average launch: the ncu-measured bytes per
                # cell of a 256 x 256 strip call times the launch's cells
                roof["traffic"] = e["traffic"]
                roof["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one 64 Mi-cell "
                                          "strip call (25.6 B per cell), scaled to the average launch's cells")
        hbm_kernels[k] = e
    families = {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                    "GBps": round(v["bytes"] / max(v["ms"], 1e-9) / 1e6, 1),
                    "TFLOPs": round(v["flops"] / max(v["ms"], 1e-9) / 1e9, 3)} for k, v in prof.items()}
    # kernels of the profiled step: every timed launch, with each replay of
    # the training graph counted as its 15 kernels
    launches_per_step = int(sum(v["launches"] for v in prof.values()))
    if "mlp_train_graph" in prof:
        t = SURROGATE_TRAIN
        replays = (t["n_train"] // t["batch"]) * t["epochs"]
        launches_per_step += replays * TRAIN_STEP_KERNELS - prof["mlp_train_graph"]["launches"]

    ests = [r["estimate"] for r in results]
    value = t_total / args.steps
    # per-level rates: a batched form solves all levels of a round in one
    # graph, so its rates come from the per-level form of the same samples
    level_seconds, level_source = results[-1]["level_seconds"], args.form
    if FORMS[args.form].get("batched") and prof_form in others:
        level_seconds, level_source = others[prof_form]["level_seconds"], prof_form + " (per-level calls)"
    fp64_fmg2 = others.get("fp64_fmg2", {}).get("value")
    fp64_conv = others.get("fp64_converged", {}).get("value")
    out = {
        "metric": METRIC,
        "value": value,
        "unit": "s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * value,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("f32+f64" if FORMS[args.form]["precision"] == 1 else "f64") + ("+bf16" if sur else ""),
        "data": "synthetic (seeded Philox KL coefficients, KL basis built on the GPU)",
        "plain_fp64_fmg2_s": fp64_fmg2,
        "plain_fp64_converged_s": fp64_conv,
        "speedup_vs_fp64_fmg2": (fp64_fmg2 / value) if fp64_fmg2 else None,
        "speedup_vs_fp64_converged": (fp64_conv / value) if fp64_conv else None,
        "config": {"workload": wl.name, "levels": wl.levels, "kl_modes": wl.M, "sigma2": wl.sigma2,
                   "lambda": wl.lam, "eps": eps, "sampler": "qmc" if args.qmc else "mc",
                   "form": args.form, "tol": SOLVE_TOL, "qtol": SOLVE_QTOL,
                   "l2": "flushed between steps (512 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roof,
        "smoother_hbm": hbm_kernels,
        "e2e": {"value": float(np.mean(e2e_times)) if e2e_times else None, "unit": "s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "estimate": float(np.mean(ests)),
        "rmse_estimate": float(np.sqrt(np.mean([r["var_estimator"] for r in results]))),
        "N_per_level": [int(x) for x in results[-1]["N"]],
        "samples_per_s_per_level": [round(float(n / t), 1) if t > 0 else None for n, t in
                                    zip(results[-1]["N"], level_seconds)],
        "samples_per_s_source": level_source,
    }
    detail = {"other_forms": others, "qmc": qmc_forms, "uneven_batch": uneven, "fmg_vs_standard_mlmc": standard,
              "large_high_contrast": c5,
              "kernel_families": families, "profiled_step_same_schedule": same_schedule,
              "captured_variance": captured, "step_seconds": times}
    if sur:
        r = results[-1]
        sr = {"train": {k: (float(v) if isinstance(v, float) else v) for k, v in r["train"].items()},
              "surrogate_cost": r["surrogate_cost"], "surrogate_cost_measured": r["surrogate_cost_measured"],
              "N_s": int(r["N_s"]), "mean_s": r["mean_s"],
              "var_s": r["var_s"], "var_q0_minus_s": float(r["V"][0]),
              "seconds_s_level": r["seconds_s"]}
        plain = others.get("mixed")
        if plain:
            sr["var_q0"] = plain["V_per_level"][0]
            sr["variance_reduction_level0"] = plain["V_per_level"][0] / max(float(r["V"][0]), 1e-300)
            sr["plain_estimate"] = plain["estimate"]
            sr["difference_in_sigmas"] = abs(out["estimate"] - plain["estimate"]) / np.sqrt(
                np.mean([x["var_estimator"] for x in results]) + plain["var_estimator"])
        detail["surrogate"] = sr
        out["surrogate"] = {"N_s": sr["N_s"], "variance_reduction_level0": sr.get("variance_reduction_level0"),
                            "difference_in_sigmas": sr.get("difference_in_sigmas"),
                            "train_corr": sr["train"].get("corr")}
    if uneven:
        out["uneven_batch"] = {"samples": sum(UNEVEN_COUNTS), "seconds_uneven_graph": uneven["seconds_uneven_graph"],
                               "seconds_per_level_calls": uneven["seconds_per_level_calls"],
                               "identical_results": uneven["identical_results"]}
    if standard:
        out["fmg_vs_standard_mlmc_saving"] = {"chosen_form": standard["saving_of_fmg_mlmc"],
                                              "fp64_fixed_schedule": standard["fixed_schedule"]["saving_of_fmg_mlmc"]}
    if c5 and "error" in c5:
        out["large_high_contrast"] = c5
    elif c5:
        out["large_high_contrast"] = {"chosen_s": c5["chosen"]["value"], "plain_fp64_s": c5["plain_fp64"]["value"],
                                      "speedup": c5["speedup_vs_plain_fp64"], "eps": c5["eps"],
                                      "rmse": c5["chosen"]["rmse_estimate"],
                                      "rmse_plain_fp64": c5["plain_fp64"]["rmse_estimate"]}
    if qmc_forms:
        # the randomized-QMC estimator of the same workload (16 shifts)
        out["qmc_s"] = {f: round(v["value"], 4) for f, v in qmc_forms.items()}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        conv = FORMS[args.form]["converged"]
        per, cores, counts = oracle_level_seconds(wl, args.cpu_seconds, conv)
        per1, counts1 = oracle_level_seconds_1core(wl, args.cpu_seconds / 2, conv)
        N = results[-1]["N"]
        t_cpu = float(np.sum(per * N))
        t_cpu1 = float(np.sum(per1 * N))
        sample = ("oracle FMG-MLMC samples per level %s (%s) timed on %d threads, %s on 1 thread; seconds "
                  "per sample x the GPU run's N_l (extrapolated)" % (
                      counts, "FP64 V-cycles to %g" % SOLVE_TOL if conv else "2 V(2,2) per stage", cores, counts1))
        if sur:
            r = results[-1]
            pe, ps, ks = oracle_surrogate_seconds(wl.M)
            steps = int(r["train"]["steps"])
            extra = pe * (r["N_s"] + r["N"][0]) + ps * steps
            t_cpu += per[0] * SURROGATE_TRAIN["n_train"] + extra
            t_cpu1 += per1[0] * SURROGATE_TRAIN["n_train"] + extra
            sample += ("; surrogate: %d training pairs at the level-0 rate, %d timed oracle training steps "
                       "extrapolated to %d, 8192 timed oracle evaluations extrapolated to N_S + N_0"
                       % (SURROGATE_TRAIN["n_train"], ks, steps))
        out["cpu_baseline"] = {"value": t_cpu, "unit": "s", "cores": cores, "kind": "oracle",
                               "value_1core": t_cpu1, "sample": sample}
    if args.detail_out and rank == 0:
        with open(args.detail_out, "w") as f:
            json.dump(dict(out, **detail), f, indent=1)
    if rank == 0:
        print(json.dumps(out))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def run_reference(args, wl, eps):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # the oracle's time to RMSE: per-level seconds per sample x the optimal
    # N_l of the target eps, N_l from the oracle's own pilot variances
    from oracle import mlmc as omlmc
    from oracle import kl as okl
    times = []
    budget = max(5.0, min(args.cpu_seconds, 60.0 / max(1, args.steps + args.warmup)))
    cores = os.cpu_count() or 1
    basis = okl.KLBasis(wl.n_ref, wl.M, wl.sigma2, wl.lam, q=32 if wl.M <= 128 else 0)
    conv = FORMS[args.form]["converged"]
    s = omlmc.FMGSampler(wl.levels, basis, seed=wl.seed, prm=oracle_params(conv), nthreads=cores)
    cost = omlmc.cost_model(np.array(wl.levels) ** 2)
    V = None
    for step in range(args.warmup + args.steps):
        per, var = [], []
        for l in range(len(wl.levels)):
            k = max(cores, int(64 / (1 << l)))
            t0 = time.perf_counter()
            y = s(l, step * 4096, k)[0]
            per.append((time.perf_counter() - t0) / k)
            var.append(np.var(y, ddof=1))
        V = np.array(var) if V is None else 0.5 * (V + np.array(var))
        N = omlmc.optimal_samples(V, cost, eps)
        if step >= args.warmup:
            times.append(float(np.sum(np.array(per) * N)))
    value = float(np.mean(times))
    out = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * value, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": wl.name, "levels": wl.levels, "kl_modes": wl.M, "eps": eps,
                      "sampler": "mc", "form": args.form,
                      "implementation": "FP64 CPU oracle, plain FMG-MLMC (no surrogate level)"},
           "cpu_baseline": {"value": value, "unit": "s", "cores": cores, "kind": "oracle",
                            "sample": "per step: a bounded batch per level timed on %d threads, "
                                      "extrapolated to the optimal N_l of eps" % cores},
           "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    global SURROGATE_COST
    args = parse()
    if args.ir_cycles is not None:
        IR_CYCLES[0] = args.ir_cycles
    if args.train_epochs is not None:
        SURROGATE_TRAIN["epochs"] = args.train_epochs
    if args.train_n is not None:
        SURROGATE_TRAIN["n_train"] = args.train_n
    if args.surrogate_cost is not None:
        SURROGATE_COST = args.surrogate_cost
    if args.train_tol is not None:
        SURROGATE_TRAIN["target_tol"] = args.train_tol
    if args.train_batch is not None:
        SURROGATE_TRAIN["batch"] = args.train_batch
    if args.train_lr is not None:
        SURROGATE_TRAIN["lr"] = args.train_lr
    if args.kernel_case:
        import torch
        import paper_1910_04727_gb300 as fm
        torch.cuda.set_device(0)
        KERNEL_CASES[args.kernel_case](torch, fm)
        return
    wl = W.WORKLOADS[args.workload]
    eps = args.eps if args.eps is not None else wl.eps
    if args.impl == "reference":
        run_reference(args, wl, eps)
    else:
        run_native(args, wl, eps)


if __name__ == "__main__":
    main()
