#!/usr/bin/env python3
"""Benchmark of the structured random phase-retrieval hot path on GB300.

One step = one whole solve of the paper's pipeline (Sec. IV-A) for a batch of
B independent problems: spectral initialisation by power iteration (Eq. 3-4)
followed by gradient descent (Eq. 2), every iteration one application of A and
one of A^H through the CUDA library. Workload: B = 64 signals, n = 2^14
(128 x 128 image-like signals, amplitude U[0, 1] times a random phase),
alpha = 4 (m = 2^16), L = 2, noiseless y, 100 power iterations + 500 GD steps.

Prints ONE JSON line (rank 0). `value` counts problem-iterations per second
(one iteration = one forward + adjoint pair on one problem), summed over all
ranks; each rank solves its own batch (weak scaling, no collective on the
data path).

--impl reference times the FP64 CPU oracle instead (the reference arm of this
comparison), on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GD iters/sec (fwd+adj) & HBM GB/s vs peak; speedup over dense i.i.d. at equal error"
UNIT = "problem-iters/s"
# GD step mu_t = MU0 * (1 - exp(-(t+1)/TAU0)) * m / sum(y). MU0 sits below the
# linear stability limit 2 sum(y) / (m lambda_max(J)) of GD at the solution
# (J: the linearised gradient map) for every problem of the headline batch
# (smallest limit 0.117) and for L >= 2 at alpha >= 4; a larger step leaves
# some problems in a limit cycle at the solution.
MU0, TAU0 = 0.1, 100.0
WORKLOAD = dict(name="structured-L2-n16384-m65536-B64-sp100-gd500", n=2 ** 14, m=2 ** 16, L=2, B=64,
                spectral_iters=100, gd_iters=500, weight="optimal", lam=-1.0, mu0=MU0, tau0=TAU0,
                seed=20240905)
FLUSH_BYTES = 512 << 20  # > 129 MB L2: written between timed steps
# Ragged batch: 256 independent problems, n = 2^k (k uniform in 10..16), alpha
# in {2, 4, 8}, L in {1, 2, 3}, own phase seeds, Poisson measurements at a mean
# of 100 photons per measurement; one autotuned ragged handle, the solve
# replayed as a CUDA graph with one branch per shape bucket.
RAGGED = dict(count=256, k_lo=10, k_hi=16, alphas=(2, 4, 8), Ls=(1, 2, 3), photons=100.0, spectral_iters=100,
              gd_iters=500, mu0=MU0, tau0=TAU0, seed=20240905, parity_sp=10, parity_gd=20)
# Structured (L = 2) against dense i.i.d. at equal recovery error (Sec. IV): both
# models solve the same B signals from their own noiseless y with the same
# spectral initialisation and step rule; each runs the fewest GD iterations (a
# multiple of GD_STEP) that bring the batch's median relative error to TARGET,
# and the speedup is the ratio of the two solve times.
DENSE_CMP = dict(n=4096, m=16384, L=2, B=64, spectral_iters=100, weight="optimal", lam=-1.0, mu0=MU0,
                 tau0=TAU0, target=1e-3, gd_step=50, gd_max=2000, seed=77)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-dense", action="store_true", help="skip the dense i.i.d. comparison")
    ap.add_argument("--no-graph", action="store_true", help="launch directly instead of replaying a CUDA graph")
    ap.add_argument("--no-library", action="store_true", help="skip the cuFFT pipeline comparison")
    ap.add_argument("--no-ragged", action="store_true", help="skip the ragged-batch workload")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the radix-3 and differentiable-operator workloads")
    ap.add_argument("--only", choices=sorted(EXTRA_LEGS),
                    help="run only this extra workload and print its JSON (for profiling one leg)")
    return ap.parse_args()


def max_over_ranks_of(torch, v: float, world: int, device) -> float:
    """The largest of every rank's v (the job's time is its slowest rank's)."""
    if world == 1:
        return v
    t = torch.tensor([v], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_throughput(world: int, B: int, iters: int, ms_step: float) -> float:
    """Problem-iterations per second of all ranks: each rank solves its own batch
    of B problems (weak scaling), the step time is the maximum over ranks."""
    return world * B * iters / (ms_step / 1e3)


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- oracle leg
def oracle_sample(W, power_iters: int, gd_iters: int, seed: int):
    """Times the FP64 oracle on one problem of the workload's shape; returns
    (problem-iterations per second, seconds)."""
    import oracle as O
    import synthetic as S
    n, m, L = W["n"], W["m"], W["L"]
    theta = S.phases(seed, L, m)
    fwd, adj = O.structured_ops(theta, n, m)
    x = S.signal_amplitude_phase(seed, 1, n)
    y = np.abs(fwd(x)) ** 2
    v0 = S.start_vector(seed, 1, n)
    t0 = time.perf_counter()
    x0 = O.spectral_init(y, v0, fwd, adj, power_iters, mode=W["weight"], lam=W["lam"])
    O.gradient_descent(x0, y, fwd, adj, gd_iters, mu0=W["mu0"], tau0=W["tau0"])
    dt = time.perf_counter() - t0
    return (power_iters + gd_iters) / dt, dt


def _oracle_worker(task):
    W, sp, gd, seed = task
    return oracle_sample(W, sp, gd, seed)[1]


def oracle_solve(W, b: int, seed: int, perturb: bool = False):
    """The FP64 oracle's whole solve of problem b of the workload's batch (the
    same signal, start vector and phases the GPU run uses; y = |A x|^2 computed
    by the oracle itself): (final iterate, its relative error up to a global
    phase, the spectral start's relative error). With perturb, the start vector
    is first multiplied entry by entry by 1 + 6e-8 (g1 + i g2), g ~ N(0, 1)
    (seeded): a change at the FP32 rounding level, which measures how strongly
    the problem's trajectory amplifies such changes."""
    import oracle as O
    import synthetic as S
    n, m, L, B = W["n"], W["m"], W["L"], W["B"]
    theta = S.phases(seed, L, m)
    fwd, adj = O.structured_ops(theta, n, m)
    x = S.signal_amplitude_phase(seed, B, n)[b:b + 1]
    y = np.abs(fwd(x)) ** 2
    v0 = S.start_vector(seed, B, n)[b:b + 1]
    if perturb:
        rng = np.random.default_rng(seed + b)
        v0 = v0 * (1 + 6e-8 * (rng.standard_normal(v0.shape) + 1j * rng.standard_normal(v0.shape)))
    x0 = O.spectral_init(y, v0, fwd, adj, W["spectral_iters"], mode=W["weight"], lam=W["lam"])
    xT, _ = O.gradient_descent(x0, y, fwd, adj, W["gd_iters"], mu0=W["mu0"], tau0=W["tau0"])
    return (xT[0], float(O.relative_error_global_phase(xT, x)[0]),
            float(O.relative_error_global_phase(x0, x)[0]))


def _oracle_solve_worker(task):
    return oracle_solve(*task)


def oracle_ragged_solve(n: int, m: int, L: int, seed: int, sp: int, gd: int, mu0: float, tau0: float):
    """The FP64 oracle's short noiseless solve of one problem of the ragged
    workload (its signal, start vector and phases; the oracle forms y itself)."""
    import oracle as O
    import synthetic as S
    theta = S.phases(seed, L, m)
    fwd, adj = O.structured_ops(theta, n, m)
    x = S.signal_gaussian(seed, 1, n)
    y = np.abs(fwd(x)) ** 2
    x0 = O.spectral_init(y, S.start_vector(seed, 1, n), fwd, adj, sp, mode="optimal", lam=-1.0)
    xT, _ = O.gradient_descent(x0, y, fwd, adj, gd, mu0=mu0, tau0=tau0)
    return xT[0]


def _oracle_ragged_worker(task):
    return oracle_ragged_solve(*task)


def oracle_leg_solve(t):
    """The FP64 oracle's whole solve of problem 0 of a bench leg from the same
    signal, start vector and phases as the GPU run (the oracle forms its own
    y): t = (kind, n, m, L, seed, sp, gd, signal), kind "1d" (signal_gaussian)
    or "2d" (t[1] = h = w image side, t[2] = grid side S, phase images of
    seed). Returns the final iterate."""
    import oracle as O
    import synthetic as S
    kind, n, m, L, seed, sp, gd, B = t
    if kind == "2d":
        h, S_ = n, m
        fwd, adj = O.structured_ops_2d(S.phases(seed, L, S_ * S_), h, h, S_)
        x = S.phase_image_ellipses(seed, B, h, h)[:1]
        v0 = S.start_vector(seed, B, h * h)[:1]
    else:
        fwd, adj = O.structured_ops(S.phases(seed, L, m), n, m)
        x = S.signal_gaussian(seed, B, n)[:1]
        v0 = S.start_vector(seed, B, n)[:1]
    y = np.abs(fwd(x)) ** 2
    x0 = O.spectral_init(y, v0, fwd, adj, sp, mode="optimal", lam=-1.0)
    xT, _ = O.gradient_descent(x0, y, fwd, adj, gd, mu0=MU0, tau0=TAU0)
    return xT[0]


def _oracle_leg_worker(task):
    return oracle_leg_solve(task)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """The FP64 oracle on every host core: one independent problem of the
    workload per core (the batch is data-parallel), in `spawn` worker processes
    (safe after CUDA use). A round's throughput is the problem-iterations of all
    workers over the slowest worker's solve time (their solves run concurrently;
    input generation is outside the timed part, as for the GPU arm)."""

    def __init__(self, cores: int):
        import multiprocessing as mp
        self.cores = cores
        self.pool = mp.get_context("spawn").Pool(cores)

    def round(self, W, sp, gd, seed0):
        dts = self.pool.map(_oracle_worker, [(W, sp, gd, seed0 + k) for k in range(self.cores)])
        dt = max(dts)
        return self.cores * (sp + gd) / dt, dt

    def ragged_solves(self, tasks):
        return self.pool.map(_oracle_ragged_worker, tasks)

    def leg_solves(self, tasks):
        return self.pool.map(_oracle_leg_worker, tasks)

    def solves(self, W, problems, seed):
        """Each problem solved as given and with its start vector perturbed."""
        return self.pool.map(_oracle_solve_worker, [(W, b, seed, pert) for b in problems for pert in (False, True)])

    def close(self):
        self.pool.close()
        self.pool.join()


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    W = WORKLOAD
    sp, gd = 2, 20  # bounded sample per step: one problem per core, 22 iterations
    pool = OraclePool(host_cores())
    for _ in range(max(1, args.warmup)):
        pool.round(W, sp, gd, W["seed"])
    total = 0.0
    for k in range(args.steps):
        _, dt = pool.round(W, sp, gd, W["seed"] + 100 * k)
        total += dt
    pool.close()
    value = args.steps * pool.cores * (sp + gd) / total
    sample = (f"{pool.cores} problems in parallel (one per host core; n={W['n']}, m={W['m']}, L={W['L']}) x "
              f"{sp} power + {gd} GD iterations per step, numpy FP64")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(W, world),
            "cpu_baseline": {"kind": "oracle", "cores": pool.cores, "sample": sample, "value": value, "unit": UNIT},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def config_dict(W, world):
    return {"workload": W["name"], "n": W["n"], "m": W["m"], "alpha": W["m"] / W["n"], "L": W["L"],
            "batch_per_gpu": W["B"], "global_batch": W["B"] * world, "spectral_iters": W["spectral_iters"],
            "gd_iters": W["gd_iters"], "spectral_weight": f"{W['weight']}(lambda={W['lam']})", "mu0": W["mu0"], "tau0": W["tau0"],
            "signal": "amplitude U[0,1] x random phase, seeded Philox", "y": "noiseless |Ax|^2",
            "l2": "flushed between timed steps (512 MiB write)",
            "parallelism": f"replicas x{world} (independent batches per GPU)"}


# ------------------------------------------------------------------ our leg
def algorithmic_mid_bytes(W, own_phases: bool = False):
    """Compulsory HBM bytes of one middle pass, averaged over the 2L-1 middle
    passes of one iteration: each reads and writes the batch's exchange buffer
    (8 B per complex element each way); the diagonal passes read the phases
    theta_l (4 B per entry: one table for the batch, or one per problem with
    own_phases); the epilogue pass reads y (4 B per element)."""
    m, B, L = W["m"], W["B"], W["L"]
    n_mid = 2 * L - 1
    diag = n_mid - 1
    tables = B if own_phases else 1
    total = n_mid * 16 * m * B + diag * 4 * m * tables + 4 * m * B
    return total / n_mid


def iteration_bytes(W, own_phases: bool = False):
    """Compulsory bytes of one iteration (all 2L+1 passes) for the batch: the
    first and last passes also read D_1 (8 B per entry)."""
    m, n, B, L = W["m"], W["n"], W["B"], W["L"]
    tables = B if own_phases else 1
    first = 8 * n * B + 8 * m * tables + 8 * m * B    # read x, D_1, write exchange
    mids = algorithmic_mid_bytes(W, own_phases) * (2 * L - 1)
    last = 8 * m * B + 8 * m * tables + 16 * n * B     # read exchange, D_1, read+write x
    return first + mids + last


def traffic_from_profile(name: str):
    """dram bytes per launch recorded by an ncu summary under profiles/, if the
    pass kernels' sources have not changed since (hash recorded in the summary)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", name)
    csrc = os.path.join(ROOT, "paper_2409_05734_gb300", "csrc")
    if not os.path.exists(path):
        return None
    h = hashlib.sha256()
    for f in ("passes.cuh", "sr_device.cuh", "sr_tma.cuh"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    want = h.hexdigest()[:16]
    vals = {}
    for line in open(path):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].rsplit(":", 1)  # keys may hold a colon ("sha256[:16]")
            vals[k.strip()] = v.strip()
    if vals.get("kernel sources sha256[:16]") != want:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def lib_metrics(x, x_true):
    """Cosine similarity (Eq. 6) and relative error up to a global phase per
    problem, computed by the library (sr_metrics), as float64 numpy arrays."""
    from paper_2409_05734_gb300 import metrics
    cos, err = metrics(x.contiguous(), x_true.contiguous())
    return cos.cpu().numpy().astype(np.float64), err.cpu().numpy().astype(np.float64)


def median_rel_err(torch, x, x_true):
    return float(np.median(lib_metrics(x, x_true)[1]))


def quantiles(v):
    """10 / 50 / 90 % quantiles of the finite entries (the paper reports its
    repetitions by 10 and 90 % quantiles around the median, Sec. IV)."""
    v = np.asarray(v, dtype=np.float64)
    v = v[np.isfinite(v)]
    if not v.size:
        return None
    q = np.quantile(v, [0.1, 0.5, 0.9])
    return {"q10": float(q[0]), "median": float(q[1]), "q90": float(q[2])}


def dense_comparison(torch, dev, flush, reps: int = 3):
    """Solve time of the structured model against the dense i.i.d. model (tcgen05
    GEMMs, BF16 matrix, and the same matrix in TF32) at equal median recovery
    error; see DENSE_CMP."""
    from paper_2409_05734_gb300 import DenseModel, Plan
    import synthetic as S
    C = DENSE_CMP
    n, m, B = C["n"], C["m"], C["B"]
    x_true = torch.from_numpy(S.signal_amplitude_phase(C["seed"], B, n)).to(torch.complex64).to(dev)
    v0 = torch.from_numpy(S.start_vector(C["seed"], B, n)).to(torch.complex64).to(dev)
    rng = np.random.default_rng(C["seed"])
    a = rng.standard_normal((m, n, 2), dtype=np.float32) * np.float32(1.0 / np.sqrt(2.0 * m))
    dense = DenseModel(a.view(np.complex64)[..., 0])
    dense_tf32 = DenseModel(a.view(np.complex64)[..., 0], format="tf32")
    del a
    plan = Plan(n, m, C["L"], C["seed"])
    plan.reserve(B)
    models = {"structured": plan, "dense": dense, "dense_tf32": dense_tf32}
    peaks = {}
    pth = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pth):
        peaks = json.load(open(pth))
    out = {}
    for name, mod in models.items():
        y = (mod.forward(x_true).abs() ** 2).contiguous()
        x = torch.empty_like(v0)

        def solve(T):
            mod.spectral_init(y, v0, C["spectral_iters"], weight=C["weight"], lam=C["lam"], out=x)
            if T:
                mod.gd_solve(y, x, T, mu0=C["mu0"], tau0=C["tau0"])

        T, err = None, None
        for t in range(C["gd_step"], C["gd_max"] + 1, C["gd_step"]):
            solve(t)
            err = median_rel_err(torch, x, x_true)
            if err <= C["target"]:
                T = t
                break
        mod.check()
        rec = {"gd_iters_to_target": T, "median_rel_err": err}
        if T is not None:
            times = []
            for r in range(reps + 1):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                solve(T)
                e1.record()
                torch.cuda.synchronize()
                if r:
                    times.append(e0.elapsed_time(e1))
            ms = statistics.median(times)
            rec.update({"solve_ms": ms, "ms_per_iteration": ms / (C["spectral_iters"] + T)})
        if name != "structured":
            # roofline of the dense GD iteration (two tcgen05 GEMMs with fused epilogues)
            it = 50
            mod.gd_solve(y, x, it, mu0=C["mu0"], tau0=C["tau0"])
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            mod.gd_solve(y, x, it, mu0=C["mu0"], tau0=C["tau0"])
            e1.record()
            torch.cuda.synchronize()
            t_it = e0.elapsed_time(e1) / 1e3 / it
            tf32 = name == "dense_tf32"
            tflops = 2 * 16 * m * n * B / t_it / 1e12   # executed: real GEMMs K = 2n, N = 2B, high + low
            gbs = 2 * (8 if tf32 else 4) * m * n / t_it / 1e9  # the matrix, read once per product
            # TF32 dense peak: the measured BF16 peak x the nominal TF32 / BF16 ratio (1.1 / 2.25 PFLOP/s)
            peak = peaks.get("bf16_tflops_sustained")
            if peak is not None and tf32:
                peak = peak * 1.1 / 2.25
            rec["gemm_roofline"] = {"ms_per_gd_iteration": t_it * 1e3, "tensor_tflops": tflops,
                                    "tensor_peak_tflops": peak,
                                    "tensor_peak_kind": ("measured bf16 sustained x nominal tf32/bf16 (1.1/2.25)"
                                                         if tf32 else "measured bf16 sustained"),
                                    "tensor_frac": tflops / peak if peak else None,
                                    "hbm_gbs": gbs, "hbm_frac": gbs / peaks["hbm_gbs"] if "hbm_gbs" in peaks else None}
        out[name] = rec
    dense.close()
    dense_tf32.close()
    del dense, dense_tf32
    s, d, d32 = out["structured"], out["dense"], out["dense_tf32"]
    speedup = d["solve_ms"] / s["solve_ms"] if "solve_ms" in s and "solve_ms" in d else None
    per_iter = d["ms_per_iteration"] / s["ms_per_iteration"] if speedup else None
    speedup32 = d32["solve_ms"] / s["solve_ms"] if "solve_ms" in s and "solve_ms" in d32 else None
    # A stronger dense bound: the same two real GEMMs per iteration (BF16 matrix, the
    # vector's high and low parts as 4B columns, FP32 accumulation) timed in cuBLAS
    # (torch.matmul), with every other step of the iteration taken as free.
    bounds = {}
    for fmt, rec in (("bf16", d), ("tf32", d32)):
        gemm_us = cublas_dense_gemm_us(torch, dev, n, m, B, fmt=fmt)
        if rec.get("gd_iters_to_target") is not None and "solve_ms" in s:
            iters = C["spectral_iters"] + rec["gd_iters_to_target"]
            bound_ms = iters * (gemm_us["forward"] + gemm_us["adjoint"]) / 1e3
            bounds[fmt] = {"cublas_gemm_us": gemm_us, "dense_solve_ms_lower_bound": bound_ms,
                           "speedup_at_equal_error": bound_ms / s["solve_ms"]}
    return {"workload": f"n={n}, m={m} (alpha={m // n}), B={B}, structured L={C['L']} vs dense i.i.d. CN(0,1/m) "
                        f"(BF16 entries, and the same matrix in TF32); {C['spectral_iters']} power iterations + GD "
                        f"to median relative error <= {C['target']}",
            "speedup_at_equal_error_vs_cublas_gemm_bound": bounds.get("bf16", {}).get("speedup_at_equal_error"),
            "speedup_at_equal_error": speedup, "speedup_at_equal_error_tf32": speedup32,
            "speedup_per_iteration": per_iter, "vs_cublas_gemm_bound": bounds.get("bf16"),
            "vs_cublas_gemm_bound_tf32": bounds.get("tf32"), **out}


def cublas_dense_gemm_us(torch, dev, n, m, B, reps=20, fmt="bf16"):
    """Device time (us) of the dense model's forward ([m, 2n] x [2n, 4B]) and adjoint
    ([2n, m] x [m, 4B]) real GEMMs in cuBLAS with FP32 accumulation: BF16 inputs, or
    FP32 inputs on the TF32 tensor cores (fmt = "tf32")."""
    g = torch.Generator(device=dev).manual_seed(0)
    prev = torch.backends.cuda.matmul.allow_bf16_reduced_precision_reduction
    prev32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_bf16_reduced_precision_reduction = False  # FP32 split-K reductions
    torch.backends.cuda.matmul.allow_tf32 = True
    cast = (lambda t: t.bfloat16()) if fmt == "bf16" else (lambda t: t)
    out = {}
    for name, (M, K) in (("forward", (m, 2 * n)), ("adjoint", (2 * n, m))):
        a = cast(torch.randn(M, K, device=dev, generator=g))
        b = cast(torch.randn(K, 4 * B, device=dev, generator=g))
        for _ in range(3):
            torch.matmul(a, b)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        out[name] = e0.elapsed_time(e1) / reps * 1e3
        del a, b
    torch.backends.cuda.matmul.allow_bf16_reduced_precision_reduction = prev
    torch.backends.cuda.matmul.allow_tf32 = prev32
    return out


def cufft_pipeline(torch, plan, W, y, x_true, fused_ms_per_iter, iters=20):
    """Informative: the same GD iteration composed from library calls (cuFFT via
    torch.fft, elementwise torch kernels), unfused, on the same batch."""
    n, m, L = W["n"], W["m"], W["L"]
    dev = y.device
    D = torch.exp(1j * torch.from_numpy(plan.phases)).to(torch.complex64).to(dev)  # [L][m]
    sumy = y.sum(dim=1, keepdim=True)
    mu = W["mu0"] * m / sumy

    def fwd(x):
        v = torch.zeros((x.shape[0], m), dtype=torch.complex64, device=dev)
        v[:, :n] = x
        for l in range(L):
            v = torch.fft.fft(D[l] * v, norm="ortho")
        return v

    def adj(w):
        v = w
        for l in reversed(range(L)):
            v = torch.conj(D[l]) * torch.fft.ifft(v, norm="ortho")
        return v[:, :n]

    def gd_iter(x):
        z = fwd(x)
        r = z.real ** 2 + z.imag ** 2 - y
        return x - mu * (2 * adj(r * z))

    x = x_true * 0.9
    for _ in range(3):
        x = gd_iter(x)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(iters):
        x = gd_iter(x)
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / iters
    return {"pipeline": "torch.fft (cuFFT) + torch elementwise kernels, unfused, same B, n, m, L",
            "ms_per_gd_iteration": t, "fused_ms_per_iteration": fused_ms_per_iter,
            "speedup_of_fused": t / fused_ms_per_iter}


def timed_graph(torch, fn, flush, reps=3):
    """Median device time (ms) of fn captured as a CUDA graph and replayed, L2
    flushed before each replay."""
    fn()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    g.replay()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def radix3_workload(torch, dev, flush):
    """The oversampling ratios 1.5, 3 and 6 of the recovery sweep (m = 3 * 2^a):
    n = 2^16, L = 2, B = 32 noiseless problems (the sweep's trials per cell),
    20 power + 100 GD iterations."""
    from paper_2409_05734_gb300 import Plan
    import synthetic as S
    out, parity = {}, []
    n, L, B, sp, gd = 2 ** 16, 2, 32, 20, 100
    for alpha, m in ((1.5, 3 * 2 ** 15), (3, 3 * 2 ** 16), (6, 3 * 2 ** 17)):
        plan = Plan(n, m, L, 31)
        plan.reserve(B)
        plan.autotune(B)
        x_true = torch.from_numpy(S.signal_gaussian(31, B, n)).to(torch.complex64).to(dev)
        y = (plan.forward(x_true).abs() ** 2).contiguous()
        v0 = torch.from_numpy(S.start_vector(31, B, n)).to(torch.complex64).to(dev)
        x = torch.empty_like(v0)

        def solve():
            plan.spectral_init(y, v0, sp, weight="optimal", out=x)
            plan.gd_solve(y, x, gd, mu0=MU0, tau0=TAU0)

        ms = timed_graph(torch, solve, flush)
        parity.append({"leg": f"alpha={alpha}", "task": ("1d", n, m, L, 31, sp, gd, B),
                       "x_gpu": x[0].cpu().numpy().astype(np.complex128)})
        it = sp + gd
        W = dict(n=n, m=m, L=L, B=B)
        out[f"alpha={alpha}"] = {"m": m, "split": list(plan.tuning[:2]), "ms_per_solve": ms,
                                 "problem_iters_per_s": B * it / (ms / 1e3),
                                 "algorithmic_gbs": iteration_bytes(W) * it / (ms / 1e3) / 1e9}
        plan.check()
        del plan
    return {"workload": f"n = 2^16, L = {L}, B = {B}, x ~ CN(0, I), noiseless, {sp} power + {gd} GD iterations; "
                        "m = 3 * 2^a runs on the four-step passes with radix-3 lines (192, 384 or 768 points: a radix-3 step inside the line FFT); autotuned split and grid",
            **out, "_parity_inputs": parity}


def two_d_workload(torch, dev, flush):
    """The 2D model the experiments of Sec. IV run: B = 64 phantom-like 128 x 128
    phase images zero-padded to 256 x 256 (alpha = 4), L = 2, noiseless, 100 power
    + 500 GD iterations (the headline's solve), graph-replayed; and L = 3, whose
    odd layer count leaves the forward on the transposed grid."""
    from paper_2409_05734_gb300 import Plan2D
    import synthetic as S
    out, parity = {}, []
    h = w = 128
    S_, B, sp, gd = 256, 64, 100, 500
    x_np = S.phase_image_ellipses(20240905, B, h, w)
    x_true = torch.from_numpy(x_np).to(torch.complex64).to(dev)
    for L in (2, 3):
        plan = Plan2D(h, w, S_, L, 20240905)
        plan.reserve(B)
        y = (plan.forward(x_true).abs() ** 2).contiguous()
        v0 = torch.from_numpy(S.start_vector(20240905, B, h * w)).to(torch.complex64).to(dev)
        x = torch.empty_like(v0)

        def solve():
            plan.spectral_init(y, v0, sp, weight="optimal", out=x)
            plan.gd_solve(y, x, gd, mu0=MU0, tau0=TAU0)

        ms = timed_graph(torch, solve, flush)
        parity.append({"leg": f"L={L}", "task": ("2d", h, S_, L, 20240905, sp, gd, B),
                       "x_gpu": x[0].cpu().numpy().astype(np.complex128)})
        it = sp + gd
        W = dict(n=h * w, m=S_ * S_, L=L, B=B)
        out[f"L={L}"] = {"ms_per_solve": ms, "problem_iters_per_s": B * it / (ms / 1e3),
                         "algorithmic_gbs": iteration_bytes(W) * it / (ms / 1e3) / 1e9,
                         "median_rel_err_global_phase": median_rel_err(torch, x, x_true)}
        plan.check()
        del plan
    return {"workload": f"B = {B} phantom-like phase images {h} x {w} (Philox ellipses, phase in [-pi/2, pi/2)) "
                        f"in a {S_} x {S_} grid (alpha = 4), 2D unitary DFTs, noiseless, {sp} power (optimal "
                        f"weights) + {gd} GD iterations, graph-replayed", **out, "_parity_inputs": parity}


def forward_time_vs_size(torch, dev, flush, reps: int = 5):
    """Forward time against image size at alpha = 1 (Sec. IV-C, Fig. 4): the 2D
    structured model (L = 2, S x S images, no padding) for S = 16 .. 4096 and the
    dense i.i.d. model (n = m = S^2, BF16 matrix) while it fits comfortably
    (S <= 128: 1 GiB), both on batches of 8 images (the dense kernel's
    smallest batch). Median of `reps` event-timed calls, L2 flushed before each."""
    from paper_2409_05734_gb300 import DenseModel, Plan2D
    B = 8
    gen = torch.Generator(device=dev).manual_seed(5)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    rows = []
    for k in range(4, 13):
        S_ = 1 << k
        n = S_ * S_
        x = torch.randn((B, n), dtype=torch.complex64, device=dev, generator=gen)
        plan = Plan2D(S_, S_, S_, 2, 7)
        plan.reserve(B)
        z = torch.empty((B, n), dtype=torch.complex64, device=dev)
        row = {"S": S_, "pixels": n, "structured_ms": timed(lambda: plan.forward(x, out=z))}
        plan.check()
        del plan
        if S_ <= 128:
            rng = np.random.default_rng(S_)
            a = rng.standard_normal((n, n, 2), dtype=np.float32) * np.float32(1.0 / np.sqrt(2.0 * n))
            dense = DenseModel(a.view(np.complex64)[..., 0])
            del a
            row["dense_ms"] = timed(lambda: dense.forward(x))
            dense.check()
            del dense
        rows.append(row)
        del x, z
        torch.cuda.empty_cache()
    return {"workload": f"alpha = 1, B = {B} images per forward, structured 2D model L = 2 (S x S) "
                        "against the dense i.i.d. model (BF16, n = m = S^2, S <= 128)", "rows": rows}


# The bounded subsample of the sweep that the default bench runs (about 20 s):
# config 5's n and step rule, fewer trials, cells and iterations.
SWEEP_BOUNDED = dict(n=2 ** 16, alphas=(2, 3, 4, 6, 8), Ls=(1, 2, 3), snrs=(None, 30), seeds=16,
                     spectral_iters=300, gd_iters=1000, mu0=MU0, tau0=TAU0, weight="optimal", lam=-1.0, tol=1e-3,
                     base_seed=20240905)
# The full sweep: run on demand (`--only sweep`, a few minutes of GPU time).
SWEEP = dict(n=2 ** 16, alphas=(1, 1.5, 2, 3, 4, 6, 8), Ls=(1, 2, 3, 4), snrs=(None, 40, 30, 20), seeds=32,
             spectral_iters=1000, gd_iters=3000, mu0=MU0, tau0=TAU0, weight="optimal", lam=-1.0, tol=1e-3,
             base_seed=20240905)


def robustness_sweep(torch, dev, flush, C=None, dense=True):
    """The robustness sweep: n = 2^16 complex Gaussian signals, L in {1..4},
    alpha in {1, 1.5, 2, 3, 4, 6, 8}, Gaussian noise on y at SNR 40 / 30 / 20 dB
    (and noiseless), 32 independent trials per cell (each problem of the batch
    has its own phases), spectral initialisation + GD; success = relative error
    below 1e-3 up to a global phase. Event-timed solves, L2 flushed before each."""
    import math
    from paper_2409_05734_gb300 import Plan
    C = C or SWEEP
    n, B, sp, gd = C["n"], C["seeds"], C["spectral_iters"], C["gd_iters"]
    gen = torch.Generator(device=dev)
    succ, med, qs = {}, {}, {}
    total_ms, total_iters = 0.0, 0
    for L in C["Ls"]:
        for alpha in C["alphas"]:
            m = int(round(alpha * n))
            cell = C["base_seed"] + 100000 * L + int(10 * alpha) * 1000
            plan = Plan(n, m, L, cell)
            plan.set_batch_seeds([cell + b for b in range(B)])
            plan.reserve(B)
            gen.manual_seed(cell)
            x_true = torch.randn((B, n), dtype=torch.complex64, device=dev, generator=gen)
            v0 = torch.randn((B, n), dtype=torch.complex64, device=dev, generator=gen)
            y0 = plan.forward(x_true).abs() ** 2
            for snr in C["snrs"]:
                y = y0
                if snr is not None:  # SNR = ||y0||^2 / E||noise||^2, noise ~ N(0, sigma^2) per entry
                    sigma = torch.linalg.vector_norm(y0, dim=1, keepdim=True) / math.sqrt(m * 10 ** (snr / 10))
                    y = y0 + sigma * torch.randn(y0.shape, device=dev, generator=gen)
                y = y.contiguous()
                x = torch.empty_like(v0)
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                plan.spectral_init(y, v0, sp, weight=C["weight"], lam=C["lam"], out=x)
                plan.gd_solve(y, x, gd, mu0=C["mu0"], tau0=C["tau0"])
                e1.record()
                torch.cuda.synchronize()
                total_ms += e0.elapsed_time(e1)
                total_iters += B * (sp + gd)
                err = lib_metrics(x, x_true)[1]
                key = f"L={L} " + ("noiseless" if snr is None else f"{snr}dB")
                ok = np.isfinite(err) & (err < C["tol"])
                succ.setdefault(key, []).append(round(float(np.mean(ok)), 4))
                med.setdefault(key, []).append(float(np.median(np.where(np.isfinite(err), err, np.inf))))
                qs.setdefault(key, []).append(quantiles(err))
            plan.check()
            del plan
    out = {"workload": f"n = {n} complex Gaussian signals, {B} trials per cell with their own phases, "
                       f"alpha {list(C['alphas'])}, L {list(C['Ls'])}, Gaussian noise on y at SNR "
                       f"{[s for s in C['snrs'] if s is not None]} dB and noiseless, {sp} power (optimal weights) "
                       f"+ {gd} GD iterations; success = relative error < {C['tol']} up to a global phase",
           "alphas": list(C["alphas"]), "success_rate": succ, "median_rel_err": med,
           "rel_err_quantiles": qs, "solve_ms_total": total_ms,
           "problem_iters_per_s": total_iters / (total_ms / 1e3)}
    if not dense:
        return out
    # the dense i.i.d. model at n = 4096 (one CN(0, 1/m) matrix per alpha, rounded
    # to BF16 by the model; the 32 trials share it), same protocol and noise
    from paper_2409_05734_gb300 import DenseModel
    nd = 4096
    dsucc, dmed = {}, {}
    for alpha in C["alphas"]:
        m = int(round(alpha * nd))
        rng = np.random.default_rng(C["base_seed"] + int(10 * alpha))
        a = rng.standard_normal((m, nd, 2), dtype=np.float32) * np.float32(1.0 / np.sqrt(2.0 * m))
        dense = DenseModel(a.view(np.complex64)[..., 0])
        del a
        gen.manual_seed(C["base_seed"] + int(10 * alpha))
        x_true = torch.randn((B, nd), dtype=torch.complex64, device=dev, generator=gen)
        v0 = torch.randn((B, nd), dtype=torch.complex64, device=dev, generator=gen)
        y0 = dense.forward(x_true).abs() ** 2
        for snr in C["snrs"]:
            y = y0
            if snr is not None:
                sigma = torch.linalg.vector_norm(y0, dim=1, keepdim=True) / math.sqrt(m * 10 ** (snr / 10))
                y = y0 + sigma * torch.randn(y0.shape, device=dev, generator=gen)
            y = y.contiguous()
            x = dense.spectral_init(y, v0, sp, weight=C["weight"], lam=C["lam"])
            dense.gd_solve(y, x, gd, mu0=C["mu0"], tau0=C["tau0"])
            err = lib_metrics(x, x_true)[1]
            key = "noiseless" if snr is None else f"{snr}dB"
            ok = np.isfinite(err) & (err < C["tol"])
            dsucc.setdefault(key, []).append(round(float(np.mean(ok)), 4))
            dmed.setdefault(key, []).append(float(np.median(np.where(np.isfinite(err), err, np.inf))))
        dense.check()
        del dense
    out["dense_iid_n4096"] = {"success_rate": dsucc, "median_rel_err": dmed}
    return out


def small_m_workload(torch, dev, flush):
    """Short transforms, which run as whole solves inside one CTA per problem
    (m <= 4096): B = 64, n = m / 4, L = 2, noiseless, 100 power + 500 GD
    iterations, graph-replayed, for m = 256, 1024 and 4096."""
    from paper_2409_05734_gb300 import Plan
    import synthetic as S
    out, parity = {}, []
    B, L, sp, gd = 64, 2, 100, 500
    for m in (256, 1024, 4096):
        n = m // 4
        plan = Plan(n, m, L, 41)
        plan.reserve(B)
        x_true = torch.from_numpy(S.signal_gaussian(41, B, n)).to(torch.complex64).to(dev)
        y = (plan.forward(x_true).abs() ** 2).contiguous()
        v0 = torch.from_numpy(S.start_vector(41, B, n)).to(torch.complex64).to(dev)
        x = torch.empty_like(v0)

        def solve():
            plan.spectral_init(y, v0, sp, weight="optimal", out=x)
            plan.gd_solve(y, x, gd, mu0=MU0, tau0=TAU0)

        ms = timed_graph(torch, solve, flush)
        parity.append({"leg": f"m={m}", "task": ("1d", n, m, L, 41, sp, gd, B),
                       "x_gpu": x[0].cpu().numpy().astype(np.complex128)})
        out[f"m={m}"] = {"n": n, "ms_per_solve": ms, "problem_iters_per_s": B * (sp + gd) / (ms / 1e3),
                         "median_rel_err_global_phase": median_rel_err(torch, x, x_true)}
        plan.check()
        del plan
    return {"workload": f"B = {B}, n = m / 4, L = {L}, x ~ CN(0, I), noiseless, {sp} power + {gd} GD iterations, "
                        "one launch per call (whole solves in one CTA per problem)", **out, "_parity_inputs": parity}


def layers_experiment(torch, dev, flush, sp=1000, B=32):
    """The layer experiment (Sec. IV-B, Fig. 5): spectral initialisation alone
    (1000 power iterations, optimal weights) on n = 4096 complex Gaussian
    signals and on phantom-like phase images (64 x 64), 32 trials per cell, alpha in {2, 3, 4, 6}, for structured models
    with L = 1, 2, 3 (own phases per trial), the one-layer model with an extra
    FFT (A = F D_1 F U: L = 2 with theta_1 = 0; one operator for all trials),
    a random unitary model (the first n columns of a Haar unitary m x m
    matrix, by QR of a complex Gaussian matrix with the diagonal phases of R
    divided out; run by the dense model, which rounds it to BF16) and the
    i.i.d. Gaussian model. Median cosine similarity (Eq. 6)."""
    from paper_2409_05734_gb300 import DenseModel, Plan
    import synthetic as S
    n = 4096
    alphas = (2, 3, 4, 6)
    gen = torch.Generator(device=dev)
    out, out_img, q_out, q_img = {}, {}, {}, {}
    # phantom-like phase images (64 x 64, flattened), the paper's signal class
    x_img = torch.from_numpy(S.phase_image_ellipses(20240905, B, 64, 64)).to(torch.complex64).to(dev)

    def cos_sim(x, x_true):
        return lib_metrics(x, x_true)[0]

    for alpha in alphas:
        m = alpha * n
        seed = 20240905 + 100 * alpha
        gen.manual_seed(seed)
        x_true = torch.randn((B, n), dtype=torch.complex64, device=dev, generator=gen)
        v0 = torch.randn((B, n), dtype=torch.complex64, device=dev, generator=gen)
        models = []
        for L in (1, 2, 3):
            plan = Plan(n, m, L, seed + L)
            plan.set_batch_seeds([seed + 1000 * L + b for b in range(B)])
            models.append((f"structured L={L}", plan))
        extra = Plan(n, m, 2, seed + 7)
        th = extra.phases
        th[0] = 0.0
        extra.set_phases(th)
        models.append(("one layer + extra FFT", extra))
        gq = torch.Generator(device=dev).manual_seed(seed + 11)
        G = torch.randn((m, n), dtype=torch.complex128, device=dev, generator=gq)
        Q, R = torch.linalg.qr(G)
        d = torch.diagonal(R)
        Q = Q * (d / d.abs()).unsqueeze(0)  # Haar: G = (Q P)(P^H R) with P^H R of positive diagonal
        models.append(("random unitary", DenseModel(Q.to(torch.complex64).cpu().numpy())))
        del G, Q, R
        rng = np.random.default_rng(seed + 13)
        a = rng.standard_normal((m, n, 2), dtype=np.float32) * np.float32(1.0 / np.sqrt(2.0 * m))
        models.append(("i.i.d. Gaussian", DenseModel(a.view(np.complex64)[..., 0])))
        del a
        for name, mod in models:
            for sig, res, qres in ((x_true, out, q_out), (x_img, out_img, q_img)):
                y = (mod.forward(sig).abs() ** 2).contiguous()
                x = mod.spectral_init(y, v0, sp, weight="optimal", lam=-1.0)
                mod.check()
                c = cos_sim(x, sig)
                res.setdefault(name, []).append(round(float(np.median(c)), 4))
                qres.setdefault(name, []).append(quantiles(c))
        del models
        torch.cuda.empty_cache()
    return {"workload": f"n = {n}, {B} trials, alpha {list(alphas)}, spectral initialisation alone ({sp} power "
                        f"iterations, optimal weights, lambda = -1), noiseless; complex Gaussian signals and "
                        f"phantom-like 64 x 64 phase images",
            "alphas": list(alphas), "median_cosine_similarity": out,
            "median_cosine_similarity_phase_images": out_img,
            "cosine_similarity_quantiles": q_out, "cosine_similarity_quantiles_phase_images": q_img}


def autograd_workload(torch, dev, flush):
    """Forward and backward of the differentiable operator (x, theta) -> z = A x at
    B = 8, n = 2^20, m = 2^22, L = 2, driven by a loss on |z|^2."""
    from paper_2409_05734_gb300 import Plan, structured_random
    import synthetic as S
    B, n, m, L = 8, 2 ** 20, 2 ** 22, 2
    plan = Plan(n, m, L, 11)
    plan.reserve(B)
    theta = torch.tensor(S.phases(11, L, m).astype(np.float32), device=dev, requires_grad=True)
    x = torch.from_numpy(S.signal_gaussian(11, B, n)).to(torch.complex64).to(dev).requires_grad_(True)
    wgt = torch.rand((B, m), device=dev, generator=torch.Generator(device=dev).manual_seed(3))

    def step():
        theta.grad = None
        x.grad = None
        z = structured_random(x, theta, plan)
        torch.sum(wgt * (z.real ** 2 + z.imag ** 2)).backward()

    step()
    torch.cuda.synchronize()
    ts = []
    for _ in range(3):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    plan.check()
    ms = statistics.median(ts)
    # compulsory bytes per problem: forward 56m + 8n (L = 2 DFTs through the
    # exchange buffers, x read, z written); backward about 100m (G_z read, the
    # h chain, the recomputed layer input, both theta-gradient reductions)
    nbytes = B * (56 * m + 8 * n + 100 * m)
    return {"workload": f"B = {B}, n = 2^20, m = 2^22, L = {L}: z = A x by the autograd function, "
                        "loss sum(w |z|^2), backward to x and theta (direct launches)",
            "ms_per_forward_backward": ms, "problems_per_s": B / (ms / 1e3),
            "algorithmic_gbs": nbytes / (ms / 1e3) / 1e9}


def ragged_workload(torch, dev, flush, reps: int = 3):
    """The ragged batch of RAGGED: problem-iterations per second of the whole
    graph-captured solve, its algorithmic HBM bytes per second, and accuracy."""
    from paper_2409_05734_gb300 import Ragged, _lib
    import synthetic as S
    R = RAGGED
    rng = np.random.default_rng(R["seed"])
    count = R["count"]
    n = (2 ** rng.integers(R["k_lo"], R["k_hi"] + 1, count)).astype(np.int64)
    alpha = rng.choice(R["alphas"], count)
    m = (n * alpha).astype(np.int64)
    L = rng.choice(R["Ls"], count).astype(np.int32)
    seeds = R["seed"] + 1000 * np.arange(count, dtype=np.uint64)
    rg = Ragged(n, m, L, seeds, autotune=True)
    x_true = torch.from_numpy(rg.pack([S.signal_gaussian(int(seeds[i]), 1, int(n[i]))[0] for i in range(count)],
                                      "x")).to(torch.complex64).to(dev)
    v0 = torch.from_numpy(rg.pack([S.start_vector(int(seeds[i]), 1, int(n[i]))[0] for i in range(count)],
                                  "x")).to(torch.complex64).to(dev)
    inten = rg.forward(x_true).abs() ** 2
    # Poisson counts at a mean of `photons` per measurement: gamma_i = photons m_i / sum|A x_i|^2
    gamma = torch.empty_like(inten)
    for i in range(count):
        sl = slice(int(rg.y_off[i]), int(rg.y_off[i] + m[i]))
        gamma[sl] = R["photons"] * float(m[i]) / float(inten[sl].sum())
    g = torch.Generator(device=dev).manual_seed(R["seed"])
    y = (torch.poisson(gamma * inten, generator=g) / gamma).contiguous()
    x = torch.empty_like(v0)

    def solve():
        rg.spectral_init(y, v0, R["spectral_iters"], weight="optimal", out=x)
        rg.gd_solve(y, x, R["gd_iters"], mu0=R["mu0"], tau0=R["tau0"])

    solve()
    torch.cuda.synchronize()
    lib = _lib.load()
    graph = torch.cuda.CUDAGraph()
    l0 = lib.sr_kernel_launches()
    with torch.cuda.graph(graph):
        solve()
    launches = lib.sr_kernel_launches() - l0
    graph.replay()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        graph.replay()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    rg.check()
    ms = statistics.median(times)
    iters = R["spectral_iters"] + R["gd_iters"]
    # every problem has its own phases (per-problem tables)
    nbytes = sum(iteration_bytes(dict(n=int(n[i]), m=int(m[i]), L=int(L[i]), B=1), own_phases=True)
                 for i in range(count))
    errs = np.array([lib_metrics(x[rg.x_off[i]:rg.x_off[i] + n[i]].view(1, -1),
                                 x_true[rg.x_off[i]:rg.x_off[i] + n[i]].view(1, -1))[1][0] for i in range(count)])
    fin = np.isfinite(errs)
    by_alpha = {int(a): float(np.median(errs[(alpha == a) & fin])) if np.any((alpha == a) & fin) else None
                for a in R["alphas"]}
    by_L = {int(l): {"median_rel_err": float(np.median(errs[(L == l) & fin])) if np.any((L == l) & fin) else None,
                     "diverged": int(np.sum((L == l) & ~fin)), "problems": int(np.sum(L == l))} for l in R["Ls"]}
    # a short noiseless solve of every problem (y = |A x|^2), whose sampled
    # problems -- one of each length -- the cpu_baseline leg re-solves with the
    # FP64 oracle (the Poisson draws of the timed workload come from torch and
    # have no oracle counterpart)
    y0 = (inten * 1.0).contiguous()
    xs = torch.empty_like(v0)
    rg.spectral_init(y0, v0, R["parity_sp"], weight="optimal", out=xs)
    rg.gd_solve(y0, xs, R["parity_gd"], mu0=R["mu0"], tau0=R["tau0"])
    rg.check()
    sampled = [int(np.flatnonzero(m == mv)[0]) for mv in sorted(set(m.tolist()))]
    xsh = xs.cpu().numpy()
    parity_inputs = [{"i": i, "n": int(n[i]), "m": int(m[i]), "L": int(L[i]), "seed": int(seeds[i]),
                      "x_gpu": xsh[rg.x_off[i]:rg.x_off[i] + n[i]].astype(np.complex128)} for i in sampled]
    return {"_parity_inputs": parity_inputs,
            "workload": f"{count} problems: n = 2^k, k ~ U{{{R['k_lo']}..{R['k_hi']}}}, alpha ~ U{list(R['alphas'])}, "
                        f"L ~ U{list(R['Ls'])}, own phases; Poisson y at {R['photons']:.0f} photons/measurement; "
                        f"{R['spectral_iters']} power (optimal weight, lambda = -1) + {R['gd_iters']} GD iterations "
                        f"(mu0 = {R['mu0']}, tau0 = {R['tau0']:.0f}); autotuned; CUDA graph",
            "buckets": rg.buckets, "total_m": int(m.sum()), "ms_per_solve": ms,
            "problem_iters_per_s": count * iters / (ms / 1e3),
            "algorithmic_gbs": nbytes * iters / (ms / 1e3) / 1e9, "gpu_launches_per_solve": int(launches),
            "median_rel_err_global_phase": float(np.median(errs[fin])) if np.any(fin) else None,
            "median_rel_err_by_alpha": by_alpha, "by_L": by_L, "diverged": int(np.sum(~fin)),
            "note": "throughput leg: Poisson y at 100 photons, alpha down to 2 and L = 1 lie outside the regime "
                    "where the paper reports recovery (alpha near 3 for L = 2, one layer far worse), so these "
                    "errors are reported, not targeted; oracle_parity checks the arithmetic on every length",
            "frac_rel_err_below_0.1": float(np.mean(errs[fin] < 1e-1)) if np.any(fin) else 0.0}


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU (the product path has no CPU fallback)")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    from paper_2409_05734_gb300 import Plan, buildlib, _lib
    import synthetic as S
    buildlib.build()
    lib = _lib.load()
    W = WORKLOAD
    n, m, L, B = W["n"], W["m"], W["L"], W["B"]
    seed = W["seed"] + 1000 * rank
    plan = Plan(n, m, L, seed)
    plan.reserve(B)
    dev = torch.device("cuda", local)
    x_true = torch.from_numpy(S.signal_amplitude_phase(seed, B, n)).to(torch.complex64).to(dev)
    y = (plan.forward(x_true).abs() ** 2).contiguous()
    v0 = torch.from_numpy(S.start_vector(seed, B, n)).to(torch.complex64).to(dev)
    x = torch.empty_like(v0)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step(y_in, v_in, x_out):
        plan.spectral_init(y_in, v_in, W["spectral_iters"], weight=W["weight"], lam=W["lam"], out=x_out)
        plan.gd_solve(y_in, x_out, W["gd_iters"], mu0=W["mu0"], tau0=W["tau0"])

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    def max_over_ranks(v):
        return max_over_ranks_of(torch, v, world, dev)

    # One step (the whole solve) is captured once as a CUDA graph and replayed:
    # the library makes no allocation and no host synchronisation inside a solve
    # once the workspace is reserved.
    y_d, v0_d, x_d = y.clone(), v0.clone(), torch.empty_like(x)
    for _ in range(args.warmup):
        flush.zero_()
        step(y_d, v0_d, x_d)
    torch.cuda.synchronize()
    if args.no_graph:
        def run():
            step(y_d, v0_d, x_d)
        launches0 = lib.sr_kernel_launches()
        run()
        launches_per_step = lib.sr_kernel_launches() - launches0
    else:
        graph = torch.cuda.CUDAGraph()
        launches0 = lib.sr_kernel_launches()
        with torch.cuda.graph(graph):
            step(y_d, v0_d, x_d)
        launches_per_step = lib.sr_kernel_launches() - launches0
        run = graph.replay
        for _ in range(args.warmup):
            flush.zero_()
            run()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    evs = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run()
        e1.record(stream)
        evs.append((e0, e1))
    barrier()
    launches = launches_per_step * args.steps
    clk = clocks.stop()
    x.copy_(x_d)
    ms_local = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    ms_step = max_over_ranks(ms_local)
    iters = W["spectral_iters"] + W["gd_iters"]
    value = whole_job_throughput(world, B, iters, ms_step)

    # accuracy of the solve (relative error up to a global phase, cosine
    # similarity of Eq. 6), computed by the library's metrics kernel
    cos, rel_err = lib_metrics(x, x_true)

    # end to end through the public API with host buffers: pinned H2D of y and v0,
    # the solve, D2H of the estimate, every step
    y_h = y.cpu().pin_memory()
    v0_h = v0.cpu().pin_memory()
    x_h = torch.empty(x.shape, dtype=x.dtype).pin_memory()
    for _ in range(args.warmup):
        y_d.copy_(y_h, non_blocking=True)
        v0_d.copy_(v0_h, non_blocking=True)
        run()
        x_h.copy_(x_d, non_blocking=True)
    barrier()
    evs = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        y_d.copy_(y_h, non_blocking=True)
        v0_d.copy_(v0_h, non_blocking=True)
        run()
        x_h.copy_(x_d, non_blocking=True)
        e1.record(stream)
        evs.append((e0, e1))
    barrier()
    e2e_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs) / args.steps)
    e2e = {"value": world * B * iters / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
           "h2d_bytes_per_step": y.numel() * 4 + v0.numel() * 8, "d2h_bytes_per_step": x.numel() * 8}

    # roofline of the dominant kernel: one extra step with per-pass event timing
    flush.zero_()
    torch.cuda.synchronize()
    _lib.check(lib.sr_plan_set_timing(plan._h, 1), "sr_plan_set_timing")
    step(y, v0, x)
    import ctypes as C
    ms3 = (C.c_double * 3)()
    cnt3 = (C.c_int64 * 3)()
    _lib.check(lib.sr_plan_get_timing(plan._h, ms3, cnt3), "sr_plan_get_timing")
    lib.sr_plan_set_timing(plan._h, 0)
    pass_ms = {k: (ms3[i] / cnt3[i] if cnt3[i] else None) for i, k in enumerate(("first", "mid", "last"))}
    share_mid = ms3[1] / max(1e-9, ms3[0] + ms3[1] + ms3[2])
    peak, peak_kind = measured_peaks()
    mid_bytes = algorithmic_mid_bytes(W)
    # The middle pass's average duration inside the timed region: the timed
    # steps' event time times the middle passes' share of the pass time (from
    # the instrumented step), over the middle-pass launches of a step. Events
    # around each launch (pass_avg_ms) also time each launch's start-up, which
    # the graph replay of the timed region overlaps with the previous kernel.
    n_mid = iters * (2 * L - 1)
    mid_ms_timed = ms_step * share_mid / n_mid
    achieved = mid_bytes / (mid_ms_timed / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": "k_mid (middle four-step pass, lines of 256)", "achieved": achieved,
                "peak": peak, "peak_kind": peak_kind + " hbm_gbs (copy, burst)", "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic_from_profile("k_mid_256_structured_B64_n16384_m65536.md"),
                "algorithmic_bytes_per_launch": mid_bytes, "avg_launch_ms": mid_ms_timed,
                "avg_launch_ms_method": "timed-region event time x middle-pass share of pass time / middle launches",
                "avg_launch_ms_events_per_launch": pass_ms["mid"],
                "frac_events_per_launch": mid_bytes / (pass_ms["mid"] / 1e3) / 1e9 / peak,
                "share_of_pass_time": share_mid, "pass_avg_ms": pass_ms,
                "iteration_gbs": iteration_bytes(W) / (ms_step / 1e3 / iters) / 1e9}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded Philox signals; y = |Ax|^2 on device)",
            "config": config_dict(W, world), "roofline": roofline, "e2e": e2e,
            "gpu_launches": int(launches), "clocks": clk,
            "accuracy": {"median_rel_err_global_phase": float(np.median(rel_err)),
                         "rel_err_global_phase_quantiles": quantiles(rel_err),
                         "median_cosine_similarity": float(np.median(cos))},
            "launch": "direct launches" if args.no_graph else "CUDA graph replay of the whole solve"}
    if rank == 0 and not args.no_library:
        line["library_comparison"] = cufft_pipeline(torch, plan, W, y, x_true, ms_step / iters)
    if rank == 0 and not args.no_dense:
        line["dense_iid_comparison"] = dense_comparison(torch, dev, flush)
    if rank == 0 and not args.no_extra:
        line["radix3_batch"] = radix3_workload(torch, dev, flush)
        line["two_dimensional"] = two_d_workload(torch, dev, flush)
        line["forward_time_vs_size"] = forward_time_vs_size(torch, dev, flush)
        line["small_m"] = small_m_workload(torch, dev, flush)
        line["differentiable_operator"] = autograd_workload(torch, dev, flush)
        line["robustness_sweep_bounded"] = robustness_sweep(torch, dev, flush, SWEEP_BOUNDED, dense=False)
        line["layer_experiment_bounded"] = layers_experiment(torch, dev, flush, sp=300, B=16)
    # problem 0 of each of these legs is re-solved by the oracle below
    leg_parity = {k: line[k].pop("_parity_inputs") for k in ("radix3_batch", "two_dimensional", "small_m")
                  if k in line}
    ragged_parity = None
    if rank == 0 and not args.no_ragged:
        line["ragged_batch"] = ragged_workload(torch, dev, flush)
        ragged_parity = line["ragged_batch"].pop("_parity_inputs")
    if rank == 0 and not args.no_cpu_baseline:
        sp, gd = 20, 200
        pool = OraclePool(host_cores())
        pool.round(W, 1, 1, W["seed"])  # worker start-up and imports outside the timed round
        v, dt = pool.round(W, sp, gd, W["seed"])
        # parity of the headline solve: the oracle's whole solve (its own y,
        # the same x, v0 and phases) of sampled problems of the batch against
        # the GPU's final iterates of the timed solve, next to the oracle's own
        # spread under an FP32-level change of the start vector
        t0 = time.perf_counter()
        sampled = (0, 9, 21, 30, 42, 51, 59, 63)
        res = pool.solves(W, sampled, seed)
        t_par = time.perf_counter() - t0
        for leg, items in leg_parity.items():
            xos = pool.leg_solves([q["task"] for q in items])
            rows = [{"case": q["leg"], "rel_diff_vs_oracle": float(np.linalg.norm(q["x_gpu"] - xo) / np.linalg.norm(xo))}
                    for q, xo in zip(items, xos)]
            line[leg]["oracle_parity"] = {
                "what": "final iterate of problem 0 of the timed solve against the FP64 oracle's solve from the "
                        "same signal, start vector and phases (the oracle forms its own y); "
                        "rel_diff = ||x_gpu - x_oracle|| / ||x_oracle||",
                "cases": rows, "max_rel_diff_vs_oracle": max(r["rel_diff_vs_oracle"] for r in rows)}
        if ragged_parity:
            R = RAGGED
            rres = pool.ragged_solves([(q["n"], q["m"], q["L"], q["seed"], R["parity_sp"], R["parity_gd"], R["mu0"],
                                        R["tau0"]) for q in ragged_parity])
            rows = [{"problem": q["i"], "n": q["n"], "m": q["m"], "L": q["L"],
                     "rel_diff_vs_oracle": float(np.linalg.norm(q["x_gpu"] - xo) / np.linalg.norm(xo))}
                    for q, xo in zip(ragged_parity, rres)]
            line["ragged_batch"]["oracle_parity"] = {
                "what": f"a noiseless solve of all {R['count']} problems ({R['parity_sp']} power + {R['parity_gd']} "
                        "GD iterations, same step rule) on the GPU; one problem of each length m re-solved by the "
                        "FP64 oracle from the same signal, start vector and phases (the oracle forms its own y); "
                        "rel_diff = ||x_gpu - x_oracle|| / ||x_oracle||",
                "problems": rows, "max_rel_diff_vs_oracle": max(r["rel_diff_vs_oracle"] for r in rows)}
        pool.close()
        xg = x.cpu().numpy().astype(np.complex128)
        per = []
        for k, b in enumerate(sampled):
            (xo, eo, e0o), (xp, ep, _) = res[2 * k], res[2 * k + 1]
            per.append({"problem": b, "rel_diff_vs_oracle": float(np.linalg.norm(xg[b] - xo) / np.linalg.norm(xo)),
                        "rel_err_gpu": float(rel_err[b]), "rel_err_oracle": eo,
                        "abs_diff_rel_err": float(abs(rel_err[b] - eo)),
                        "oracle_spectral_start_rel_err": e0o,
                        "oracle_self_spread": float(np.linalg.norm(xp - xo) / np.linalg.norm(xo)),
                        "oracle_rel_err_perturbed": ep})
        line["oracle_parity"] = {
            "what": f"final iterate of the whole solve ({W['spectral_iters']} power + {W['gd_iters']} GD "
                    "iterations) against the FP64 oracle on the same signal, start vector and phases (the oracle "
                    "forms its own y); rel_diff = ||x_gpu - x_oracle|| / ||x_oracle|| and the difference of the "
                    "two reconstruction errors up to a global phase. oracle_self_spread is the oracle's own "
                    "change when its start vector moves by 6e-8 relative (FP32 rounding level); the step "
                    f"mu0 = {W['mu0']} lies below every problem's stability limit of GD at the solution, so such "
                    "changes are damped",
            "problems": per, "max_rel_diff_vs_oracle": max(p["rel_diff_vs_oracle"] for p in per),
            "max_abs_diff_rel_err": max(p["abs_diff_rel_err"] for p in per),
            "target_abs_diff_rel_err": 1e-4, "oracle_wall_s": t_par}
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
                                "sample": f"{pool.cores} problems of the workload in parallel (one per host core), "
                                          f"{sp} power + {gd} GD iterations each, numpy FP64 (pocketfft), "
                                          f"{dt:.1f} s (slowest core)"}
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


EXTRA_LEGS = {
    "radix3": "radix3_workload",
    "two_d": "two_d_workload",
    "forward_curve": "forward_time_vs_size",
    "autograd": "autograd_workload",
    "sweep": "robustness_sweep",
    "small": "small_m_workload",
    "layers": "layers_experiment",
    "ragged": "ragged_workload",
    "dense": "dense_comparison",
}


def run_only(args):
    """One extra workload on its own (rank 0, one GPU): its JSON object."""
    import torch
    from paper_2409_05734_gb300 import buildlib
    buildlib.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    out = globals()[EXTRA_LEGS[args.only]](torch, dev, flush)
    out.pop("_parity_inputs", None)
    print(json.dumps({"only": args.only, **out}))
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        return run_only(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
