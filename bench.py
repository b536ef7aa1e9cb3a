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

The same JSON line carries, at one GPU, two more workloads as sub-objects:
  "large"  the MNIST-8M-shaped implicit solve: n = 8.1M, d = 784 (~20 % non-zero,
           stored dense), m = 10, sigma = 9, D = 65,536 in 32 x 16 blocks, one-vs-rest
           hinge + l2, lambda = 1e-6, split precision; Z (2 TB in FP32) is never stored;
  "serve"  the serving loop: Poisson arrivals of solve requests (n 5k-500k, d 32-784,
           D 1k-32k, three losses, two regularisers) and scoring batches of 1-4096
           queries, the solve rate at 70 % of the measured isolated capacity.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec split_bf16|fp32|cached_z]
                  [--loss squared|hinge|multinomial|crammer_singer|l1] [--block-fraction P]
                  [--workload multiclass|large|serve|ridge|sweep|score] [--no-large] [--no-serve]
  python bench.py --impl reference ...   # the FP64 oracle on the host cores

--loss swaps the loss of the same workload; --block-fraction P < 1 runs the stochastic
variant (each block takes part in an iteration's graph projection with probability P).

One JSON line on rank 0.  With N > 1 (torchrun), each rank solves its own
replica of the workload (the method keeps every block on one GPU) and the value
is the total iterations per second of all ranks ("replicas only", weak scaling);
the "large" and "serve" sub-objects run at N = 1 only.
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
                C=4, loss="squared", reg="l2", lam=1e-5, rho=1.0, data_seed=1, philox_seed=2, data="multiclass")
# the MNIST-8M-shaped implicit solve (its Z would be 8.1M x 65,536 floats, 2 TB in FP32)
LARGE = dict(name="mnist8m-shaped-8.1M-d784-D65536-m10-32x16-hinge", n=8_100_000, d=784, m=10, sigma=9.0,
             D=65536, R=32, C=16, loss="hinge", reg="l2", lam=1e-6, rho=1.0, data_seed=3, philox_seed=4,
             data="sparse01", feature_map="fourier", block_fraction=1.0)
METRIC = "ADMM iter/s"
GOLDEN = os.path.join(ROOT, "tests", "golden")
# DRAM bytes per launch of the fused passes, from an ncu capture of the current kernel at
# n = 100k scaled to 200k rows (X, V, O' grow with n); None once the kernel has changed
TRAFFIC_200K = {"pass1": 1.105e9, "pass2": 1.205e9}
TRAFFIC_CZ_200K = {"pass1": None, "pass2": None}   # the cached-Z streamed passes (not captured since they changed)


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
    if w.get("data") == "sparse01":
        return synth.sparse01(n=n, d=w["d"], m=w["m"], seed=w["data_seed"])
    return synth.multiclass(n=n, d=w["d"], m=w["m"], seed=w["data_seed"])


def solver_kw(w, prec):
    return dict(loss=w["loss"], reg=w["reg"], lam=w["lam"], sigma=w["sigma"], rho=w["rho"], D=w["D"], R=w["R"],
                C=w["C"], seed=w["philox_seed"], m=w["m"], prec=prec, feature_map=w.get("feature_map", "fourier"),
                degree=w.get("degree", 2), coef0=w.get("coef0", 1.0))


def pads(w):
    return -(-w["m"] // 16) * 16, -(-w["d"] // 64) * 64   # m_pad, d_pad (the slot layout's padding)


def algorithmic_flops_per_pass(w):
    """Algorithmic tensor work of one regeneration pass, as the roofline counts it: the
    three split products of X.G at the data's own d (3 x 2 n d D) and one chained product
    at m_pad (2 n D m_pad)."""
    mpad, _ = pads(w)
    return 3 * 2 * w["n"] * w["d"] * w["D"] + 2 * w["n"] * w["D"] * mpad


def flops_per_iter(w, prec):
    """Useful FP32-equivalent flops of one iteration (two regenerations of X.G, 2 n d D each,
    two chained products, 2 n D m each, and the s_j x s_j x m product with the cached inverse
    per block), and the flops one pass executes on its precision's units: on the split path
    3 products for X.G at d_pad (the phase folded into a padding column of ones where one is
    free) and 3 for the chained
    product at m_pad."""
    n, d, D, m, R, C = w["n"], w["d"], w["D"], w["m"], w["R"], w["C"]
    mpad, dpad = pads(w)
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
    n, D, R, C = w["n"], w["D"], w["R"], w["C"]
    mpad, _ = pads(w)
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


def measure(rff, w, X, Y, prec, steps, warmup, stream, objective=False):
    """warmup untimed iterations (the first call also builds the factors), then steps
    iterations timed with CUDA events on the solver's stream; returns the device ms,
    the phase profile, the consensus weights, the clock record and (objective=True) the
    objective at the final consensus weights."""
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
    obj = s.solve(0)["objective"] if objective else None
    s.close()
    return ms, prof, W, clk, obj


def oracle_errors(W, ref):
    """Relative Frobenius error of W on the stored sample of the FP64 oracle's Wbar."""
    import numpy as np
    Wf = W.astype(np.float64).ravel()
    return float(np.linalg.norm(Wf[ref["idx"]] - ref["w"]) / np.linalg.norm(ref["w"]))


def compare_precisions(rff, w, X, Y, main_prec, stream):
    """The three precisions on the same workload, each for the 23 iterations of the stored
    FP64 oracle iterate (tests/golden/multiclass_200k_wbar23_sample.npz, written by a script
    that calls only the oracle): speed over the last 20, and the relative error of the
    consensus weights and of the objective against the oracle's."""
    import numpy as np
    path = os.path.join(GOLDEN, "multiclass_200k_wbar23_sample.npz")
    default = all(w[k] == WORKLOAD[k] for k in ("n", "d", "m", "D", "R", "C", "loss", "reg", "lam", "sigma"))
    ref = np.load(path) if default and w["block_fraction"] == 1.0 and w["feature_map"] == "fourier" else None
    out = {}
    for prec in ("split_bf16", "cached_z", "fp32"):
        if prec == "split_bf16" and w["feature_map"] == "laplace":
            continue                      # the implicit split precision takes the Fourier map only
        if prec != "cached_z" and w["feature_map"] == "tensorsketch":
            continue                      # sketches are formed once: cached-Z precision only
        k = 20 if prec != "fp32" else 5
        ms_p, _, W_p, _, obj = measure(rff, w, X, Y, prec, k, 23 - k, stream, objective=True)
        out[prec] = {"iter_per_s": k / (ms_p * 1e-3), "iterations": 23, "objective": obj}
        if ref is not None:
            out[prec]["rel_err_vs_fp64_oracle"] = oracle_errors(W_p, ref)
            if "objective" in ref.files:
                oo = float(ref["objective"])
                out[prec]["objective_rel_err_vs_fp64_oracle"] = abs(obj - oo) / abs(oo)
    if ref is not None:
        out["oracle"] = "FP64 oracle iterate after 23 iterations, sample of %d Wbar entries" % ref["idx"].size
    return out


def run_ours(args, rank, world):
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
    ms, prof, W_main, clk, _ = measure(rff, w, X, Y, args.prec, args.steps, args.warmup, stream)
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
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        s2.solve(0, stats=False)          # the set-up alone: features, Gram, factors, autotuning
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        s2.solve(args.steps, stats=False)
        s2.weights(Wh)
        e2e_s = time.perf_counter() - t0
        s2.close()
        e2e = {"value": args.steps / e2e_s, "unit": "iter/s", "h2d_bytes_per_step": (X.nbytes + Y.nbytes) // args.steps,
               "d2h_bytes_per_step": Wh.numel() * 4 // args.steps, "set_data_s": t1 - t0, "setup_s": t2 - t1,
               "note": "set_data + set-up + K iterations + get_weights, pinned host buffers"}

    compare = None
    if not args.no_compare and rank == 0:
        compare = compare_precisions(rff, w, X, Y, args.prec, stream)

    useful, exec_pass = flops_per_iter(w, args.prec)
    # the stochastic variant's passes do the work of its active blocks alone
    act = active_fraction(rff, w, args.warmup, args.warmup + args.steps)
    exec_pass *= act
    hbm, bf16, bf16_sus, src = peaks()
    # dominant kernel: the larger of the two fused passes
    ph = "ms_pass2" if prof["ms_pass2"] >= prof["ms_pass1"] else "ms_pass1"
    per_launch_ms = prof[ph] / max(prof["iters"], 1)
    executed = exec_pass / (per_launch_ms * 1e-3) / 1e12
    if args.prec == "split_bf16":
        achieved = algorithmic_flops_per_pass(w) * act / (per_launch_ms * 1e-3) / 1e12
        traffic = TRAFFIC_200K.get(ph[3:]) if not args.n and act == 1.0 else None
        roof = {"bound": "tensor", "achieved": achieved, "peak": bf16_sus, "unit": "TFLOP/s",
                "frac": achieved / bf16_sus, "traffic": traffic, "kernel": "k_regen_tc " + ph[3:],
                "peak_source": src + " sustained bf16",
                "count": "3 x 2 n d D (X.G, three split products at d) + 2 n D m_pad (one chained product) "
                         "per launch",
                "executed_tflops": executed, "executed_frac": executed / bf16_sus,
                "executed_count": "3 x 2 n d_pad D + 3 x 2 n D m_pad (every product the kernel issues)"}
    elif args.prec == "cached_z":
        # the streamed pass reads Z once: HBM-bound (the tensor work, 3 x 2 n D m_pad, would take
        # slightly less time at the sustained BF16 peak)
        gbs = bytes_per_cached_pass(w) * act / (per_launch_ms * 1e-3) / 1e9
        traffic = TRAFFIC_CZ_200K.get(ph[3:]) if not args.n and act == 1.0 else None
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "traffic": traffic,
                "kernel": "k_split_gemm " + ph[3:], "peak_source": src + " copy bandwidth",
                "tensor_tflops": executed, "tensor_frac": executed / bf16_sus}
    else:
        # FP32 SIMT: the measured FFMA throughput of this GPU (independent chains, one launch)
        alu_peak, _ = rff.rff_measure_fma_peaks(stream.cuda_stream)
        roof = {"bound": "alu", "achieved": executed, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": executed / alu_peak, "traffic": None, "kernel": "k_pass_simt " + ph[3:],
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
    if world == 1 and not args.no_large:
        line["large"] = run_large(args)
    if world == 1 and not args.no_serve:
        line["serve"] = run_serve(args)
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


# ----------------------------------------------------------------- the oracle on the host cores
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


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n and n[0]:
            return int(n[0])
    except Exception:
        pass
    return os.cpu_count()


def oracle_rate(w, iters=2):
    """The FP64 oracle's iterations per second on the whole workload, from two slices that
    keep its projection form: every row block at least as tall as a column block is wide
    (n_i >= s_j, the Gram form I + Z_ij^T Z_ij, as at the full size).  The time per
    iteration is fitted as t(n) = a + b n through the two slices (a: the solves with the
    cached factors, whose cost does not depend on n; b n: the passes over Z and the row
    updates) and evaluated at the workload's n.  The one helper behind cpu_baseline and
    the reference arm, so both report the same rate."""
    smax = -(-w["D"] // w["C"])
    n1 = max(w["R"] * smax, 4096)
    n2 = n1 + n1 // 2
    if n2 >= w["n"]:
        n1, n2 = w["n"], None
    t1 = oracle_iter_seconds(w, n1, iters)
    if n2 is None:
        t, fit = t1, "the whole workload (%d rows)" % n1
    else:
        t2 = oracle_iter_seconds(w, n2, iters)
        b = (t2 - t1) / (n2 - n1)
        a = t1 - b * n1
        t = a + b * w["n"]
        fit = ("slices of %d and %d of %d rows (same d, D, m, %dx%d grid, every row block at least as tall as "
               "a column block is wide: the Gram form of the full size), %d iterations each, set-up excluded; "
               "t(n) = a + b n fitted through them: a = %.3g s, b = %.3g s/row, t(%d) = %.3g s"
               % (n1, n2, w["n"], w["R"], w["C"], iters, a, b, w["n"], t))
    return {"value": 1.0 / t, "unit": "iter/s", "cores": blas_threads(), "kind": "oracle", "sample": fit}


def cpu_baseline(args):
    return oracle_rate(workload(args))


def run_reference(args, rank, world):
    if rank != 0:
        return None
    w = workload(args)
    cb = oracle_rate(w)
    return {"metric": METRIC, "value": cb["value"], "unit": "iter/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": w["name"], "prec": "f64 oracle (explicit Z)"},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_large(args, steps=3):
    """The MNIST-8M-shaped implicit solve at full size on one GPU (LARGE): data drawn into
    pinned host memory, then end to end through the public API -- set_data (host to device),
    set-up (Philox, Gram matrices on the tensor cores, FP64-class factorisation of the 512
    blocks' 4096 x 4096 Gram matrices), the first iteration, `steps` iterations timed with
    CUDA events on the solver's stream, the weights back to host memory.  Beside it, the
    seeded 20,000-row sample of the same workload at the same 32 x 16 grid against the FP64
    oracle's iterate after 50 iterations (tests/golden/large_20k_32x16_wbar50.npz)."""
    import numpy as np
    import torch

    import paper_1409_0940_gb300 as rff
    import synth
    w = dict(LARGE)
    n, d, m = w["n"], w["d"], w["m"]
    t0 = time.perf_counter()
    Xp = torch.empty((n, d), dtype=torch.float32, pin_memory=True)
    _, Y = synth.sparse01(n=n, d=d, m=m, seed=w["data_seed"], out=Xp.numpy())
    Yp = torch.from_numpy(Y).pin_memory()
    Wh = torch.empty((w["D"], m), dtype=torch.float32).pin_memory()
    data_s = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = new_solver(rff, w, "split_bf16", stream)
    s.set_data(Xp, Yp)
    torch.cuda.synchronize()
    t_data = time.perf_counter()
    s.solve(1, stats=False)              # set-up and the first iteration
    torch.cuda.synchronize()
    t_first = time.perf_counter()
    s.profiling(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(torch.cuda.current_device()) as clk:
        e0.record(stream)
        s.solve(steps, stats=False)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = s.profile()
    s.weights(Wh)
    e2e_s = time.perf_counter() - t0
    s.close()
    del Xp, Yp
    _, _, bf16_sus, src = peaks()
    ph = "ms_pass2" if prof["ms_pass2"] >= prof["ms_pass1"] else "ms_pass1"
    per_launch_ms = prof[ph] / max(prof["iters"], 1)
    achieved = algorithmic_flops_per_pass(w) / (per_launch_ms * 1e-3) / 1e12
    _, exec_pass = flops_per_iter(w, "split_bf16")
    executed = exec_pass / (per_launch_ms * 1e-3) / 1e12
    out = {"metric": METRIC, "value": steps / (ms * 1e-3), "unit": "iter/s", "steps": steps, "warmup": 1,
           "ms_per_step": ms / steps, "dtype": "f16x3",
           "config": {"workload": w["name"], "n": n, "d": d, "m": m, "D": w["D"], "grid": "32x16",
                      "sigma": w["sigma"], "loss": "hinge (one-vs-rest)", "reg": "l2", "lambda": w["lam"],
                      "rho": w["rho"], "prec": "split_bf16", "data": "synth.sparse01 (MNIST-8M stand-in, "
                      "%.1f %% non-zero, stored dense)" % 20.0,
                      "l2": "inputs larger than L2 (X split 27 GB)"},
           "set_data_s": t_data - t0, "setup_and_first_iteration_s": t_first - t_data, "data_gen_s": data_s,
           "e2e": {"value": (1 + steps) / e2e_s, "unit": "iter/s",
                   "h2d_bytes_per_step": (n * d + n * m) * 4 // (1 + steps),
                   "d2h_bytes_per_step": w["D"] * m * 4 // (1 + steps),
                   "note": "set_data from pinned host memory + set-up + %d iterations + get_weights" % (1 + steps)},
           "gpu_launches": int(prof["launches"]),
           "phases_ms_per_iter": {k[3:]: prof[k] / max(prof["iters"], 1) for k in prof if k.startswith("ms_")},
           "roofline": {"bound": "tensor", "achieved": achieved, "peak": bf16_sus, "unit": "TFLOP/s",
                        "frac": achieved / bf16_sus, "traffic": None, "kernel": "k_regen_tc " + ph[3:],
                        "peak_source": src + " sustained bf16",
                        "count": "3 x 2 n d D + 2 n D m_pad per launch",
                        "executed_tflops": executed, "executed_frac": executed / bf16_sus},
           "clocks": clk.summary(),
           "iterations_of_the_workload": 50,
           "seconds_for_50_iterations": (t_first - t0) + 49 * ms / steps / 1e3}
    out["sample_vs_fp64_oracle"] = large_sample_errors(rff, stream)
    return out


def large_sample_errors(rff, stream):
    """The seeded 20,000-row sample of the large workload at its 32 x 16 grid (625-row blocks:
    the outer form I + Z_ij Z_ij^T) against the FP64 oracle after 50 iterations."""
    import numpy as np
    path = os.path.join(GOLDEN, "large_20k_32x16_wbar50.npz")
    if not os.path.exists(path):
        return None
    ref = np.load(path)
    w = dict(LARGE, n=int(ref["n"]))
    X, Y = make_data(w)
    s = new_solver(rff, w, "split_bf16", stream)
    s.set_data(X, Y)
    st = s.solve(50, stats=True)
    W = s.weights()
    s.close()
    return {"rows": w["n"], "grid": "32x16", "iterations": 50, "rel_err_wbar": oracle_errors(W, ref),
            "objective_rel_err": abs(st["objective"] - float(ref["objective"])) / abs(float(ref["objective"])),
            "tolerance": 1e-4}


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


SERVE = dict(n_solve=24, n_score=400, rate_score=40.0, iters=30, load=0.7, max_active=8, seed=11,
             n_lo=5_000, n_hi=500_000, ds=[32, 64, 128, 256, 440, 784], Ds=[1024, 2048, 4096, 8192, 16384, 32768])


def serve_requests(cfg, prec):
    """The solve requests of the serving workload, drawn before any clock starts: n
    log-uniform in [5k, 500k], d and D from the configured ranges, losses and regularisers
    cycled, FP32 data from seeded Gaussian mixtures."""
    import numpy as np

    import paper_1409_0940_gb300 as rff
    import synth
    rng = np.random.default_rng(cfg["seed"])
    losses = ["squared", "hinge", "logistic"]
    reqs = []
    for k in range(cfg["n_solve"]):
        n = int(np.exp(rng.uniform(np.log(cfg["n_lo"]), np.log(cfg["n_hi"]))))
        d = int(rng.choice(cfg["ds"]))
        D = int(rng.choice(cfg["Ds"]))
        loss, reg = losses[k % 3], ["l2", "l1"][(k // 3) % 2]
        X, Y = synth.ridge(n=n, d=d, seed=k) if loss == "squared" else synth.binary(n=n, d=d, seed=k)
        R, C = -(-n // 50_000), max(1, D // 2048)
        pr = rff.make_params(loss=loss, reg=reg, lam=1e-4, sigma=float(np.sqrt(d)), D=D, R=R, C=C, seed=k, m=1,
                             prec=prec)
        dpad = -(-d // 64) * 64
        # tensor work of the request: the regeneration passes of every iteration and the
        # set-up's Z^T and Gram matrices (the fit below turns it into seconds)
        work = 2 * 3 * 2 * n * dpad * D * (cfg["iters"] + 1) + 3 * 2 * n * D * (D // C)
        reqs.append({"params": pr, "X": X, "Y": Y, "d": d, "n": n, "D": D, "loss": loss, "reg": reg,
                     "work": float(work)})
    return reqs


def run_one_alone(rff, srv, req, iters):
    rid = rff.rff_server_submit_solve(srv, req["params"], req["X"], req["Y"], iters)
    while True:
        for c in rff.rff_server_poll(srv, 16, 50):
            if c["id"] == rid:
                rff.rff_server_release(srv, rid)
                return c["run_ms"]


def run_serve(args):
    """Serving: Poisson arrivals of solve requests and scoring batches of 1..4096 queries
    against resident models, side by side on the device.  The solve rate is set to 70 % of
    the isolated capacity measured first: three requests (the smallest, median and largest
    by work) run alone, a line a + b work through their run times predicts every request's
    isolated service time, and capacity is one over their mean.  Reported: p50/p99 latency
    per request kind (scores against resident models, scores that waited for their model's
    solve, solves) and the throughput."""
    import numpy as np

    import paper_1409_0940_gb300 as rff
    cfg = SERVE
    reqs = serve_requests(cfg, args.prec)
    srv = rff.rff_server_create(0, cfg["max_active"])
    order = np.argsort([r["work"] for r in reqs])
    cal = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    run_ms = [run_one_alone(rff, srv, reqs[i], cfg["iters"]) for i in cal]
    b, a = np.polyfit([reqs[i]["work"] for i in cal], run_ms, 1)
    service_ms = np.maximum(a + b * np.array([r["work"] for r in reqs]), min(run_ms))
    capacity = 1e3 / float(np.mean(service_ms))
    rate_solve = cfg["load"] * capacity
    rng = np.random.default_rng(cfg["seed"] + 1)
    events = [(t, "solve") for t in np.cumsum(rng.exponential(1 / rate_solve, cfg["n_solve"]))]
    t_first = events[0][0]
    events += [(t_first + t, "score") for t in np.cumsum(rng.exponential(1 / cfg["rate_score"], cfg["n_score"]))]
    events.sort()
    # score request contents are drawn before the clock starts too
    score_q = [int(np.exp(rng.uniform(0, np.log(4096)))) for _ in range(cfg["n_score"])]
    score_model = [int(rng.integers(1 << 30)) for _ in range(cfg["n_score"])]
    models, kinds, pending = [], {}, set()
    solved = set()
    done = []
    ev = si = sc = 0
    t_start = time.perf_counter()
    while ev < len(events) or pending:
        now = time.perf_counter() - t_start
        while ev < len(events) and events[ev][0] <= now:
            if events[ev][1] == "solve":
                r = reqs[si]
                si += 1
                rid = rff.rff_server_submit_solve(srv, r["params"], r["X"], r["Y"], cfg["iters"])
                models.append((rid, r["d"]))
                kinds[rid] = "solve"
                pending.add(rid)
            else:
                mid, d = models[score_model[sc] % len(models)]
                q = score_q[sc]
                sc += 1
                Xq = rng.standard_normal((q, d)).astype(np.float32)
                out = np.empty((q, 1), dtype=np.float32)
                rid = rff.rff_server_submit_score(srv, mid, Xq, out)
                kinds[rid] = ("score", out) if mid in solved else ("score_waiting", out)
                pending.add(rid)
            ev += 1
        for c in rff.rff_server_poll(srv, 256, 2):
            pending.discard(c["id"])
            done.append(c)
            if kinds[c["id"]] == "solve" and c["status"] == 0:
                solved.add(c["id"])
    wall = time.perf_counter() - t_start
    rff.rff_server_destroy(srv)
    kind_of = {rid: (k if isinstance(k, str) else k[0]) for rid, k in kinds.items()}
    out = {"metric": "serve p50/p99 ms", "unit": "ms", "higher_is_better": False, "data": "synthetic",
           "config": {"workload": "serve-poisson", "solve_requests": cfg["n_solve"], "score_requests": cfg["n_score"],
                      "n": "log-uniform %d..%d" % (cfg["n_lo"], cfg["n_hi"]), "d": cfg["ds"], "D": cfg["Ds"],
                      "losses": ["squared", "hinge", "logistic"], "regs": ["l2", "l1"],
                      "score_queries": "log-uniform 1..4096", "iterations_per_solve": cfg["iters"],
                      "max_active": cfg["max_active"], "prec": args.prec,
                      "solve_rate_per_s": rate_solve, "score_rate_per_s": cfg["rate_score"],
                      "load": "solve arrivals at %.0f %% of the isolated capacity %.2f solves/s (fit through "
                              "%d requests run alone: %s ms)" % (100 * cfg["load"], capacity, len(cal),
                                                                 ", ".join("%.0f" % x for x in run_ms))},
           "wall_s": wall}
    for kind in ("solve", "score", "score_waiting"):
        ok = [c for c in done if kind_of[c["id"]] == kind and c["status"] == 0]
        lat = np.array([c["latency_ms"] for c in ok])
        que = np.array([c["queue_ms"] for c in ok])
        out[kind] = {"count": len(ok), "failed": sum(1 for c in done if kind_of[c["id"]] == kind and c["status"] != 0),
                     "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
                     "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
                     "queue_p50_ms": float(np.percentile(que, 50)) if que.size else None}
    out["value"] = out["score"]["p99_ms"]
    out["value_is"] = "p99 of scores against resident models"
    out["throughput_req_per_s"] = len(done) / wall
    out["throughput_solves_per_s"] = out["solve"]["count"] / wall
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
    ap.add_argument("--no-large", action="store_true", help="skip the large implicit solve")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving loop")
    ap.add_argument("--n", type=int, default=0, help="rows of a reduced workload (profiling runs)")
    ap.add_argument("--workload", default="multiclass", choices=["multiclass", "large", "serve", "ridge", "sweep", "score"])
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
        if args.workload == "large":
            line = run_large(args, steps=max(1, min(args.steps, 10)))
        else:
            line = {"sweep": run_sweep, "serve": run_serve, "ridge": run_ridge, "score": run_score}[args.workload](args)
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
