"""Benchmark: ADMM iterations per second of block-splitting ADMM over implicit
random Fourier features, on the TIMIT-shaped multiclass workload:

  n = 200,000 rows, d = 440, m = 147 (+-1 one-hot), sigma = 10, D = 16,384,
  4 row blocks x 4 column blocks of 50,000 x 4,096, squared loss + l2,
  lambda = 1e-5, rho = 1 (sum-scaled), synthetic Gaussian-mixture data.

A step is one ADMM iteration: both regeneration passes over every block of Z,
the cached projections of all 16 blocks, the proxes, exchange, averaging and
dual updates.  Set-up (Philox draw, Gram matrices, FP64 Cholesky, inverses) is
done before the timed region.  Every input of the timed region (X split,
V_ij, W'_ij, the factors) is larger than the 129 MB L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec split_bf16|fp32|cached_z]
                  [--loss squared|hinge|multinomial|crammer_singer|l1] [--block-fraction P]
  python bench.py --impl reference ...   # the FP64 oracle on the host cores

--loss swaps the loss of the same workload; --block-fraction P < 1 runs the stochastic
variant (each block takes part in an iteration's graph projection with probability P).

One JSON line on rank 0.  With N > 1 (torchrun), each rank solves its own
replica of the workload (the method keeps every block on one GPU) and the value
is the total iterations per second of all ranks ("replicas only", weak scaling).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="multiclass-200k-d440-D16384-m147-4x4", n=200_000, d=440, m=147, sigma=10.0, D=16384, R=4,
                C=4, loss="squared", reg="l2", lam=1e-5, rho=1.0, data_seed=1, philox_seed=2)
METRIC = "ADMM iter/s"
TRAFFIC_200K = {"pass1": 1.654e9, "pass2": 1.219e9}     # kernel -> DRAM bytes per launch (see run_ours)
TRAFFIC_CZ_200K = {"pass1": 14.35e9, "pass2": 14.08e9}   # the cached-Z streamed passes, likewise


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p["hbm_gbs"], p["bf16_tflops"], p["bf16_tflops_sustained"], "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


class Clocks:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def make_data(w, n=None):
    import synth
    n = n or w["n"]
    if w.get("feature_map", "fourier") == "laplace":   # the Laplace map takes histograms
        return synth.histograms(n=n, d=w["d"], m=w["m"], seed=w["data_seed"])
    return synth.multiclass(n=n, d=w["d"], m=w["m"], seed=w["data_seed"])


def solver_kw(w, prec):
    return dict(loss=w["loss"], reg=w["reg"], lam=w["lam"], sigma=w["sigma"], rho=w["rho"], D=w["D"], R=w["R"],
                C=w["C"], seed=w["philox_seed"], m=w["m"], prec=prec, feature_map=w.get("feature_map", "fourier"),
                degree=w.get("degree", 2), coef0=w.get("coef0", 1.0))


def flops_per_iter(w, prec):
    """Algorithmic work of one iteration.  Useful FP32-equivalent flops: two
    regenerations of X.G (2 n d D each) and two chained products (2 n D m each),
    the s_j x s_j x m product with the cached inverse per block.  Executed BF16 tensor flops of
    the split path: 3 products for X.G and 3 for each chained product at m_pad."""
    n, d, D, m, R, C = w["n"], w["d"], w["D"], w["m"], w["R"], w["C"]
    mpad = -(-m // 16) * 16
    dpad = -(-d // 64) * 64
    s = D // C
    useful = 2 * (2 * n * d * D) + 2 * (2 * n * D * m) + R * C * 2 * s * s * m
    pass_tc = 3 * 2 * n * dpad * D + 3 * 2 * n * D * mpad       # one pass, executed on tensor cores
    pass_simt = 2 * n * dpad * D + 2 * n * D * mpad              # one pass, FP32 FMA
    pass_cached = 3 * 2 * n * D * mpad                           # one streamed pass (Z stored)
    return useful, {"split_bf16": pass_tc, "fp32": pass_simt, "cached_z": pass_cached}[prec]


def bytes_per_cached_pass(w):
    """Algorithmic HBM bytes of one streamed pass of the cached-Z precision: Z (or Z^T)
    as a hi/lo BF16 pair (4 n D), the n x m_pad chained operand or result of all C
    column blocks (4 C n m_pad), and the D x m_pad operand or result of all R row
    blocks (4 R D m_pad)."""
    n, D, m, R, C = w["n"], w["D"], w["m"], w["R"], w["C"]
    mpad = -(-m // 16) * 16
    return 4 * n * D + 4 * C * n * mpad + 4 * R * D * mpad


def max_over_ranks(ms, dist, device):
    """The slowest rank's time: every rank's timed region ends at the same barrier, so the
    job's time is the maximum (all_reduce MAX; NCCL on the GPU, gloo in the CPU tests)."""
    import torch
    if dist is None:
        return ms
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(steps, world, ms):
    """Whole-job iterations per second: every rank runs `steps` iterations of its own replica
    of the workload (weak scaling, no data-path collective)."""
    return steps * world / (ms * 1e-3)


def new_solver(rff, w, prec, stream):
    s = rff.Solver(stream=stream.cuda_stream, **solver_kw(w, prec))
    if w.get("block_fraction", 1.0) < 1.0:
        s.set_block_fraction(w["block_fraction"])
    return s


def active_fraction(rff, w, k0, k1):
    """Fraction of blocks active over iterations [k0, k1) of the stochastic variant: the
    library's own Philox words at counters (block, k, 2, 0), thresholded as the solver does."""
    import numpy as np
    import torch
    p = w.get("block_fraction", 1.0)
    if p >= 1.0:
        return 1.0
    nb = w["R"] * w["C"]
    k = np.repeat(np.arange(k0, k1, dtype=np.uint32), nb)
    b = np.tile(np.arange(nb, dtype=np.uint32), k1 - k0)
    ctr = np.stack([b, k, np.full_like(b, 2), np.zeros_like(b)], axis=1)
    dctr = torch.from_numpy(ctr.view(np.int32)).cuda()
    out = torch.zeros_like(dctr)
    rff.rff_philox4x32_10(dctr, w["philox_seed"], out)
    w0 = out.cpu().numpy().view(np.uint32)[:, 0]
    return float(np.mean((w0 >> 8) < np.uint32(int(np.floor(p * 2.0 ** 24)))))


def measure(rff, w, X, Y, prec, steps, warmup, stream):
    """warmup untimed iterations (the first call also builds the factors), then steps
    iterations timed with CUDA events on the solver's stream; returns the device ms,
    the phase profile, the consensus weights and the clock record."""
    import torch
    s = new_solver(rff, w, prec, stream)
    s.set_data(X, Y)
    s.solve(warmup, stats=False)
    s.profiling(True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(torch.cuda.current_device()) as clk:
        e0.record(stream)
        s.solve(steps, stats=False)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = s.profile()
    W = s.weights()
    s.close()
    return ms, prof, W, clk


def run_ours(args, rank, world):
    import numpy as np
    import torch

    import paper_1409_0940_gb300 as rff

    w = workload(args)
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    X, Y = make_data(w)
    stream = torch.cuda.Stream()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    ms, prof, W_main, clk = measure(rff, w, X, Y, args.prec, args.steps, args.warmup, stream)
    if dist:
        dist.barrier()
        ms = max_over_ranks(ms, dist, "cuda")

    # end to end through the public API with host buffers: set_data (H2D of X, Y from pinned
    # host memory), set-up, K iterations, weights back to pinned host memory (D2H)
    e2e = None
    if not args.no_e2e:
        Xp, Yp = torch.from_numpy(X).pin_memory(), torch.from_numpy(Y).pin_memory()
        Wh = torch.empty((w["D"], w["m"]), dtype=torch.float32).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = new_solver(rff, w, args.prec, stream)
        s2.set_data(Xp, Yp)
        s2.solve(args.steps, stats=False)
        s2.weights(Wh)
        e2e_s = time.perf_counter() - t0
        s2.close()
        e2e = {"value": args.steps / e2e_s, "unit": "iter/s", "h2d_bytes_per_step": (X.nbytes + Y.nbytes) // args.steps,
               "d2h_bytes_per_step": Wh.numel() * 4 // args.steps,
               "note": "set_data + set-up + K iterations + get_weights, pinned host buffers"}

    # the other precisions on the same workload and iteration count: speed, and the
    # relative difference of the consensus weights (all three approximate the same
    # FP64 iterate; the oracle parity itself is in the tests)
    compare = None
    if not args.no_compare and rank == 0:
        compare = {}
        Ws = {args.prec: W_main}
        for prec in ("split_bf16", "cached_z", "fp32"):
            if prec == "split_bf16" and w["feature_map"] == "laplace":
                continue                      # the implicit split precision takes the Fourier map only
            if prec != "cached_z" and w["feature_map"] == "tensorsketch":
                continue                      # sketches are formed once: cached-Z precision only
            if prec == args.prec:
                compare[prec] = {"iter_per_s": args.steps / (ms * 1e-3)}
                continue
            k = args.steps if prec != "fp32" else max(1, min(args.steps, 5))
            # same total iteration count as the main run: the untimed part makes up the rest
            ms_p, _, W_p, _ = measure(rff, w, X, Y, prec, k, args.warmup + args.steps - k, stream)
            Ws[prec] = W_p
            compare[prec] = {"iter_per_s": k / (ms_p * 1e-3)}
        ref = Ws["fp32"].astype(np.float64)
        for prec, Wp in Ws.items():
            compare[prec]["rel_diff_vs_fp32"] = float(np.linalg.norm(Wp - ref) / np.linalg.norm(ref))
        compare["iterations"] = args.warmup + args.steps

    useful, exec_pass = flops_per_iter(w, args.prec)
    # the stochastic variant's passes do the work of its active blocks alone
    act = active_fraction(rff, w, args.warmup, args.warmup + args.steps)
    exec_pass *= act
    hbm, bf16, bf16_sus, src = peaks()
    # dominant kernel: the larger of the two fused passes
    ph = "ms_pass2" if prof["ms_pass2"] >= prof["ms_pass1"] else "ms_pass1"
    per_launch_ms = prof[ph] / max(prof["iters"], 1)
    achieved = exec_pass / (per_launch_ms * 1e-3) / 1e12
    if args.prec == "split_bf16":
        # DRAM bytes per launch from an ncu capture of the current k_regen_tc at n = 100k, scaled
        # to the 200k-row workload by rows (profiles/k_regen_tc_multiclass_100k.md); None while
        # the kernel has changed since the last capture
        traffic = TRAFFIC_200K.get(ph[3:]) if not args.n and act == 1.0 else None
        roof = {"bound": "tensor", "achieved": achieved, "peak": bf16_sus, "unit": "TFLOP/s",
                "frac": achieved / bf16_sus, "traffic": traffic, "kernel": ph[3:],
                "peak_source": src + " sustained bf16"}
    elif args.prec == "cached_z":
        # the streamed pass reads Z once: HBM-bound (the tensor work, 3 x 2 n D m_pad, would take
        # slightly less time at the sustained BF16 peak)
        gbs = bytes_per_cached_pass(w) * act / (per_launch_ms * 1e-3) / 1e9
        # DRAM bytes per launch from an ncu capture at n = 100k scaled by rows
        # (profiles/k_split_gemm_cached_z_multiclass_100k.md); None off that workload
        traffic = TRAFFIC_CZ_200K.get(ph[3:]) if not args.n and act == 1.0 else None
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "traffic": traffic,
                "kernel": ph[3:], "peak_source": src + " copy bandwidth", "tensor_tflops": achieved,
                "tensor_frac": achieved / bf16_sus}
    else:
        # FP32 SIMT: the measured FFMA throughput of this GPU (independent chains, one launch)
        alu_peak, _ = rff.rff_measure_fma_peaks(stream.cuda_stream)
        roof = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak, "traffic": None, "kernel": ph[3:],
                "peak_source": "measured FFMA chains (rff_measure_fma_peaks)",
                "peak_derived": 152 * 128 * 2 * 2.07e9 / 1e12}

    value = job_throughput(args.steps, world, ms)
    line = {
        "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.prec == "fp32" else "f16x3", "data": "synthetic",
        "config": {"workload": w["name"], "n": w["n"], "d": w["d"], "m": w["m"], "D": w["D"],
                   "grid": "%dx%d" % (w["R"], w["C"]), "sigma": w["sigma"], "loss": w["loss"], "reg": w["reg"],
                   "lambda": w["lam"], "rho": w["rho"], "prec": args.prec, "parallelism": "replicas",
                   "block_fraction": w["block_fraction"], "active_fraction": act, "feature_map": w["feature_map"],
                   "l2": "inputs larger than L2 (X split 358 MB, V 512 MB, factors 2.1 GB)"},
        "e2e": e2e,
        "gpu_launches": int(prof["launches"]),
        "phases_ms_per_iter": {k[3:]: prof[k] / max(prof["iters"], 1) for k in prof if k.startswith("ms_")},
        "useful_tflops": useful / (ms / args.steps * 1e-3) / 1e12,
        "roofline": roof,
        "clocks": clk.summary(),
        "precisions": compare,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    return line


def workload(args):
    """The benchmark workload with the command line's row count, loss and block fraction."""
    w = dict(WORKLOAD)
    if args.n:
        w["n"] = args.n
        w["name"] = w["name"].replace("200k", "%dk" % (args.n // 1000))
    w["loss"] = args.loss
    w["block_fraction"] = args.block_fraction
    w["feature_map"] = args.feature_map
    if args.feature_map == "laplace":
        # histogram inputs (d bins summing to 1) and a bandwidth at the scale of sum_r sqrt(2 x_r)
        w["name"] = w["name"].replace("multiclass", "histograms") + "-laplace"
        w["sigma"] = 8.0
    elif args.feature_map == "fastfood":
        w["name"] += "-fastfood"
    elif args.feature_map == "tensorsketch":
        # the polynomial kernel (<x, y> / sigma^2 + 1)^2
        w["degree"], w["coef0"] = 2, 1.0
        w["name"] += "-tensorsketch-q2"
    if args.loss != "squared":
        w["name"] += "-" + args.loss
    if args.block_fraction < 1.0:
        w["name"] += "-p%g" % args.block_fraction
    return w


def oracle_iter_seconds(w, n_sample, iters):
    """Seconds per iteration of the FP64 oracle on an n_sample-row slice of the workload
    (same d, D, m, grid, loss and block fraction; set-up excluded)."""
    from oracle import admm
    X, Y = make_data(w, n=n_sample)
    p = admm.Problem(X, Y, w["loss"], w["reg"], w["lam"], w["sigma"], w["rho"], w["D"], w["R"], w["C"],
                     w["philox_seed"], feature_map=w["feature_map"], degree=w.get("degree", 2),
                     coef0=w.get("coef0", 1.0))
    admm.admm(p, 1)                       # builds Z and the cached factors (untimed)
    t0 = time.perf_counter()
    admm.admm(p, iters, block_fraction=w["block_fraction"])
    return (time.perf_counter() - t0) / iters


def cpu_baseline(args, n_sample=8000, iters=3):
    w = workload(args)
    sec = oracle_iter_seconds(w, n_sample, iters)
    scale = w["n"] / n_sample
    return {"value": 1.0 / (sec * scale), "unit": "iter/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "%d of %d rows (same d, D, m, 4x4 grid), %d iterations timed, set-up excluded, "
                      "per-iteration time extrapolated linearly in n (x%.0f)" % (n_sample, w["n"], iters, scale)}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    cb = cpu_baseline(args, n_sample=4000, iters=max(1, min(args.steps, 3)))
    return {"metric": METRIC, "value": cb["value"], "unit": "iter/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": workload(args)["name"], "prec": "f64 oracle (explicit Z)"},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ----------------------------------------------------------------- sweep and serving workloads
SWEEP = dict(name="sweep-8sigma-x-8lambda-logistic-d128", sigmas=[1, 2, 4, 8, 16, 32, 64, 128],
             lambdas=[1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-7, 1e-8, 1e-9], Ds=[1024, 2048, 4096, 8192], d=128,
             n_lo=10_000, n_hi=400_000, seed=7)


def run_ridge(args):
    """The small ridge solve (n = 2000, d = 16, D = 512, one 1 x 1 block, squared + l2,
    lambda = 1e-4, 200 iterations): launch- and latency-bound, so the measure is the time of
    one iteration replayed as a CUDA graph, and of the whole 200-iteration solve."""
    import numpy as np
    import torch

    import paper_1409_0940_gb300 as rff
    import synth
    X, y = synth.ridge(n=2000, d=16, seed=0)
    stream = torch.cuda.Stream()
    s = rff.Solver(stream=stream.cuda_stream, prec=args.prec, loss="squared", reg="l2", lam=1e-4, sigma=4.0,
                   rho=1.0, D=512, R=1, C=1, seed=1, m=1)
    s.set_data(X, y)
    s.solve(max(args.warmup, 3), stats=False)        # set-up, eager first iteration, graph capture
    torch.cuda.synchronize()
    iters = 200
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(torch.cuda.current_device()) as clk:
        e0.record(stream)
        s.solve(iters, stats=False)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = s.profile()
    s.close()
    return {"metric": "ridge iteration latency", "value": 1e3 * ms / iters, "unit": "us/iter", "n_gpus": 1,
            "steps": iters, "warmup": max(args.warmup, 3), "ms_per_step": ms / iters, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.prec == "fp32" else "f16x3",
            "data": "synthetic",
            "config": {"workload": "ridge-2000-d16-D512-1x1", "iterations": iters, "prec": args.prec,
                       "timing": "CUDA events around 200 graph-replayed iterations"},
            "gpu_launches_per_iter": int(prof["launches"]) / (iters + max(args.warmup, 3)),
            "solve_ms_200_iters": ms, "clocks": clk.summary()}


def run_columns(args):
    """Column partitions (the paper's Sec. 5 experiment on C, at this workload's shape): the
    multiclass workload (n from --n, default 200k) solved with C = 4, 8, 16, 32, 64 column
    blocks on the command line's precision; per C the cached factors' bytes, the set-up time,
    the device time per iteration, and the objective after 30 iterations relative to C = 4's."""
    import torch

    import paper_1409_0940_gb300 as rff
    w = workload(args)
    X, Y = make_data(w)
    stream = torch.cuda.Stream()
    rows, iters = [], 30
    for C in (4, 8, 16, 32, 64):
        wc = dict(w, C=C)
        s = new_solver(rff, wc, args.prec, stream)
        s.set_data(X, Y)
        t0 = time.perf_counter()
        s.solve(1, stats=False)                    # set-up and the first iteration
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        s.solve(2, stats=False)                    # graph capture
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.solve(iters - 3, stats=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / (iters - 3)
        obj = s.solve(0)["objective"]
        sj = -(-wc["D"] // C)
        rows.append({"C": C, "features_per_block": sj, "factor_bytes": 2 * 3 * wc["R"] * C * sj * sj,
                     "setup_s": setup_s, "ms_per_iter": ms, "objective_30": obj})
        s.close()
    for r in rows:
        r["objective_vs_C4"] = r["objective_30"] / rows[0]["objective_30"]
    return {"metric": "ADMM iter/s by column blocks", "value": 1e3 / rows[0]["ms_per_iter"], "unit": "iter/s",
            "n_gpus": 1, "steps": iters, "warmup": 3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.prec == "fp32" else "f16x3", "data": "synthetic",
            "config": {"workload": w["name"] + "-columns", "prec": args.prec,
                       "factor_bytes": "R C s_j^2 x 3 BF16 terms (the cached Q_ij)"},
            "columns": rows}


def run_rows(args):
    """Scaling the rows at fixed D (the single-GPU analogue of the paper's weak scaling, Sec. 5):
    the multiclass workload with n = 50k, 100k, 200k, 400k, 800k rows on the 4 x 4 grid; per n
    the set-up time, the device time per iteration and the rows processed per second."""
    import torch

    import paper_1409_0940_gb300 as rff
    w = workload(args)
    stream = torch.cuda.Stream()
    rows, iters = [], 20
    for n in (50_000, 100_000, 200_000, 400_000, 800_000):
        wn = dict(w, n=n)
        X, Y = make_data(wn)
        s = new_solver(rff, wn, args.prec, stream)
        s.set_data(X, Y)
        t0 = time.perf_counter()
        s.solve(1, stats=False)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        s.solve(2, stats=False)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.solve(iters, stats=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / iters
        rows.append({"n": n, "setup_s": setup_s, "ms_per_iter": ms, "iter_per_s": 1e3 / ms,
                     "rows_per_s": n * 1e3 / ms})
        s.close()
        del X, Y
    return {"metric": "ADMM rows/s by n", "value": rows[2]["rows_per_s"], "unit": "rows/s", "n_gpus": 1,
            "steps": iters, "warmup": 3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.prec == "fp32" else "f16x3", "data": "synthetic",
            "config": {"workload": w["name"].replace("200k", "n") + "-rows", "prec": args.prec,
                       "value": "rows per second at n = 200k"},
            "rows": rows}


def run_sweep(args):
    """(sigma, lambda) sweep: 64 binary-logistic + l2 solves; per sigma one data set (n log-uniform in
    [10k, 400k], d = 128), one D (cycled over 1k..8k), one handle whose 8 columns are the 8 lambdas
    (one factor per sigma); the 8 handles run side by side (rff_sweep_run, CUDA-graph iterations)."""
    import numpy as np
    import torch

    import paper_1409_0940_gb300 as rff
    import synth
    w = SWEEP
    rng = np.random.default_rng(w["seed"])
    ns = np.exp(rng.uniform(np.log(w["n_lo"]), np.log(w["n_hi"]), len(w["sigmas"]))).astype(int)
    solvers, groups = [], []
    for k, sigma in enumerate(w["sigmas"]):
        n, D = int(ns[k]), w["Ds"][k % len(w["Ds"])]
        X, y = synth.binary(n=n, d=w["d"], seed=100 + k)
        Y = np.ascontiguousarray(np.repeat(y, len(w["lambdas"]), axis=1))
        R, C = -(-n // 50_000), D // 1024
        s = rff.Solver(prec=args.prec, loss="logistic", reg="l2", lam=w["lambdas"][0], sigma=float(sigma), rho=1.0,
                       D=D, R=R, C=C, seed=k, m=len(w["lambdas"]))
        s.set_lambdas(w["lambdas"])
        s.set_data(X, Y)
        solvers.append(s)
        groups.append({"sigma": sigma, "n": n, "D": D, "grid": "%dx%d" % (R, C)})
    rff.rff_sweep_run([s.h for s in solvers], args.warmup)     # set-up (factors) + warm-up
    torch.cuda.synchronize()
    with Clocks(torch.cuda.current_device()) as clk:
        t0 = time.perf_counter()
        rff.rff_sweep_run([s.h for s in solvers], args.steps)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
    tuned = [s.profile() for s in solvers]
    for s, g, pr in zip(solvers, groups, tuned):
        g["tc_kchunk"] = pr["tc_kchunk"]
        s.close()
    nsolve = len(w["sigmas"]) * len(w["lambdas"])
    # executed tensor work of the two regeneration passes of every group per iteration:
    # 3 x 2 n d_pad D (X.G, FP16 x3) + 3 x 2 n D m_pad (chained product), slot-padded sizes
    mpad = -(-len(w["lambdas"]) // 16) * 16
    dpad = -(-w["d"] // 64) * 64
    flops = 0.0
    for g in groups:
        R = int(g["grid"].split("x")[0])
        nslots = sum(-(-(g["n"] // R + (1 if i < g["n"] % R else 0)) // 128) * 128 for i in range(R))
        flops += 2 * (3 * 2 * nslots * dpad * g["D"] + 3 * 2 * nslots * g["D"] * mpad)
    tc_tflops = flops * args.steps / sec / 1e12
    _, _, bf16_sus, src = peaks()
    return {"metric": "sweep solve-iterations/s", "value": nsolve * args.steps / sec, "unit": "solve-iter/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.prec == "fp32" else "f16x3", "data": "synthetic",
            "config": {"workload": w["name"], "solves": nsolve, "groups": groups, "prec": args.prec,
                       "timing": "host wall clock around rff_sweep_run (all streams drained)"},
            "roofline": {"bound": "tensor", "achieved": tc_tflops, "peak": bf16_sus, "unit": "TFLOP/s",
                         "frac": tc_tflops / bf16_sus, "traffic": None, "kernel": "k_regen_tc (all groups)",
                         "peak_source": src + " sustained bf16",
                         "note": "executed passes' tensor work over the whole sweep iteration (the other kernels "
                                 "and the groups' overlap included in the time)"},
            "clocks": clk.summary()}


def run_score(args):
    """Scoring latency of a resident model that keeps its feature parameters against one that
    gave them back (rff_admm_release_features: each call draws G again from Philox): the
    benchmark's d, D, m and grid, a model trained 3 iterations on 20,000 rows, batches of
    1024 queries from host memory, 30 timed calls each after 3 warm-up calls."""
    import numpy as np
    import torch

    import paper_1409_0940_gb300 as rff
    w = dict(WORKLOAD)
    w["n"] = 20_000
    X, Y = make_data(w)
    Xq = make_data(w, n=1024)[0]
    stream = torch.cuda.Stream()
    out = {}
    for mode in ("resident", "released"):
        s = new_solver(rff, w, args.prec, stream)
        s.set_data(X, Y)
        s.solve(3, stats=False)
        freed = s.release_features() if mode == "released" else 0
        for _ in range(3):
            s.predict(Xq)
        ts = []
        for _ in range(30):
            t0 = time.perf_counter()
            s.predict(Xq)
            ts.append((time.perf_counter() - t0) * 1e3)
        s.close()
        out[mode] = {"p50_ms": float(np.percentile(ts, 50)), "p99_ms": float(np.percentile(ts, 99)),
                     "bytes_freed": int(freed)}
    return {"metric": "score latency p50", "value": out["released"]["p50_ms"], "unit": "ms", "n_gpus": 1,
            "higher_is_better": False, "vs_baseline": None, "dtype": "f16x3" if args.prec != "fp32" else "f32",
            "data": "synthetic",
            "config": {"workload": "score-1024q-d440-D16384-m147", "prec": args.prec, "model_rows": w["n"]},
            "resident": out["resident"], "released": out["released"]}


def run_serve(args):
    """Serving: Poisson arrivals of solve requests (n log-uniform 5k..200k, d in 32..784,
    D in 1k..8k, loss in {squared, hinge, logistic}, reg in {l2, l1}) and scoring batches of
    1..4096 queries against resident models; p50/p99 latency per request kind."""
    import numpy as np

    import paper_1409_0940_gb300 as rff
    import synth
    rng = np.random.default_rng(11)
    n_solve, n_score, rate_solve, rate_score = 24, 400, 2.0, 40.0
    events = [(t, "solve") for t in np.cumsum(rng.exponential(1 / rate_solve, n_solve))]
    events += [(t, "score") for t in 1.0 + np.cumsum(rng.exponential(1 / rate_score, n_score))]
    events.sort()
    # request contents are drawn before the clock starts
    losses = ["squared", "hinge", "logistic"]
    solves, k = [], 0
    for t, kind in events:
        if kind != "solve":
            continue
        n = int(np.exp(rng.uniform(np.log(5_000), np.log(200_000))))
        d = int(rng.choice([32, 64, 128, 256, 440, 784]))
        D = int(rng.choice([1024, 2048, 4096, 8192]))
        loss, reg = losses[k % 3], ["l2", "l1"][(k // 3) % 2]
        if loss == "squared":
            X, Y = synth.ridge(n=n, d=d, seed=k)
        else:
            X, Y = synth.binary(n=n, d=d, seed=k)
        pr = rff.make_params(loss=loss, reg=reg, lam=1e-4, sigma=float(np.sqrt(d)), D=D, R=-(-n // 50_000),
                             C=max(1, D // 2048), seed=k, m=1, prec=args.prec)
        solves.append((pr, X, Y, d))
        k += 1
    srv = rff.rff_server_create(0, 8)
    models, kinds, pending, scores = [], {}, set(), []
    solved = set()          # models whose solve has completed (scores against them hit a resident model)
    t_start = time.perf_counter()
    done = []
    ev, si = 0, 0
    while ev < len(events) or pending:
        now = time.perf_counter() - t_start
        while ev < len(events) and events[ev][0] <= now:
            kind = events[ev][1]
            if kind == "solve":
                pr, X, Y, d = solves[si]
                si += 1
                rid = rff.rff_server_submit_solve(srv, pr, X, Y, 30)
                models.append((rid, d))
                kinds[rid] = "solve"
                pending.add(rid)
            elif models:
                mid, d = models[int(rng.integers(len(models)))]
                q = int(np.exp(rng.uniform(0, np.log(4096))))
                Xq = rng.standard_normal((q, d)).astype(np.float32)
                out = np.empty((q, 1), dtype=np.float32)
                scores.append(out)
                rid = rff.rff_server_submit_score(srv, mid, Xq, out)
                kinds[rid] = "score" if mid in solved else "score_waiting"
                pending.add(rid)
            ev += 1
        for c in rff.rff_server_poll(srv, 256, 5):
            pending.discard(c["id"])
            done.append(c)
            if kinds[c["id"]] == "solve" and c["status"] == 0:
                solved.add(c["id"])
    wall = time.perf_counter() - t_start
    rff.rff_server_destroy(srv)
    out = {"metric": "serve p50/p99 ms", "n_gpus": 1, "data": "synthetic", "higher_is_better": False,
           "config": {"workload": "serve-poisson", "solve_requests": n_solve, "score_requests": n_score,
                      "rate_solve_per_s": rate_solve, "rate_score_per_s": rate_score, "max_active": 8,
                      "iterations_per_solve": 30, "prec": args.prec}, "wall_s": wall}
    for kind in ("solve", "score", "score_waiting"):
        lat = np.array([c["latency_ms"] for c in done if kinds[c["id"]] == kind and c["status"] == 0])
        que = np.array([c["queue_ms"] for c in done if kinds[c["id"]] == kind and c["status"] == 0])
        out[kind] = {"count": int(lat.size), "failed": int(sum(1 for c in done if kinds[c["id"]] == kind
                                                              and c["status"] != 0)),
                     "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
                     "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
                     "queue_p50_ms": float(np.percentile(que, 50)) if que.size else None}
    out["value"] = out["score"]["p99_ms"]
    out["unit"] = "ms (p99 of scores against resident models)"
    out["throughput_req_per_s"] = len(done) / wall
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="split_bf16", choices=["split_bf16", "fp32", "cached_z"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--no-compare", action="store_true", help="skip the other precisions (profiling runs)")
    ap.add_argument("--n", type=int, default=0, help="rows of a reduced workload (profiling runs)")
    ap.add_argument("--workload", default="multiclass",
                    choices=["multiclass", "ridge", "sweep", "serve", "score", "columns", "rows"])
    ap.add_argument("--loss", default="squared", choices=["squared", "hinge", "multinomial", "crammer_singer", "l1"],
                    help="loss of the multiclass workload")
    ap.add_argument("--feature-map", default="fourier", choices=["fourier", "laplace", "fastfood", "tensorsketch"],
                    help="laplace: random Laplace features on histogram inputs (fp32 or cached_z precision); "
                         "fastfood: the structured Fastfood projection; tensorsketch: the polynomial "
                         "kernel's sketches (cached_z precision)")
    ap.add_argument("--block-fraction", type=float, default=1.0,
                    help="stochastic variant: probability that a block takes part in an iteration")
    args = ap.parse_args()
    if args.feature_map == "tensorsketch" and args.prec != "cached_z":
        ap.error("--feature-map tensorsketch runs on --prec cached_z")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.workload != "multiclass":
        line = {"sweep": run_sweep, "serve": run_serve, "ridge": run_ridge, "score": run_score,
                "columns": run_columns, "rows": run_rows}[args.workload](args)
        print(json.dumps(line), flush=True)
        return
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    line = run_ours(args, rank, world)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
