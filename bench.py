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

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec split_bf16|fp32]
  python bench.py --impl reference ...   # the FP64 oracle on the host cores

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
    return synth.multiclass(n=n, d=w["d"], m=w["m"], seed=w["data_seed"])


def solver_kw(w, prec):
    return dict(loss=w["loss"], reg=w["reg"], lam=w["lam"], sigma=w["sigma"], rho=w["rho"], D=w["D"], R=w["R"],
                C=w["C"], seed=w["philox_seed"], m=w["m"], prec=prec)


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
    return useful, (pass_tc if prec == "split_bf16" else pass_simt)


def run_ours(args, rank, world):
    import numpy as np
    import torch

    import paper_1409_0940_gb300 as rff

    w = dict(WORKLOAD)
    if args.n:
        w["n"] = args.n
        w["name"] = w["name"].replace("200k", "%dk" % (args.n // 1000))
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    X, Y = make_data(w)
    stream = torch.cuda.Stream()
    s = rff.Solver(stream=stream.cuda_stream, **solver_kw(w, args.prec))
    s.set_data(X, Y)
    s.solve(args.warmup, stats=False)          # set-up + warm-up iterations
    s.profiling(True)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(torch.cuda.current_device()) as clk:
        e0.record(stream)
        s.solve(args.steps, stats=False)
        e1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    prof = s.profile()
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())

    s.close()
    # end to end through the public API with host buffers: set_data (H2D of X, Y),
    # set-up, K iterations, weights back to the host (D2H)
    e2e = None
    if not args.no_e2e:
        t0 = time.perf_counter()
        s2 = rff.Solver(stream=stream.cuda_stream, **solver_kw(w, args.prec))
        s2.set_data(X, Y)
        s2.solve(args.steps, stats=False)
        Wh = s2.weights()
        e2e_s = time.perf_counter() - t0
        s2.close()
        e2e = {"value": args.steps / e2e_s, "unit": "iter/s", "h2d_bytes_per_step": (X.nbytes + Y.nbytes) // args.steps,
               "d2h_bytes_per_step": Wh.nbytes // args.steps,
               "note": "set_data + set-up + K iterations + get_weights, host buffers"}

    useful, exec_pass = flops_per_iter(w, args.prec)
    hbm, bf16, bf16_sus, src = peaks()
    # dominant kernel: the larger of the two fused passes
    ph = "ms_pass2" if prof["ms_pass2"] >= prof["ms_pass1"] else "ms_pass1"
    per_launch_ms = prof[ph] / max(prof["iters"], 1)
    achieved = exec_pass / (per_launch_ms * 1e-3) / 1e12
    if args.prec == "split_bf16":
        roof = {"bound": "tensor", "achieved": achieved, "peak": bf16_sus, "unit": "TFLOP/s",
                "frac": achieved / bf16_sus, "traffic": None, "kernel": ph[3:], "peak_source": src + " sustained bf16"}
    else:
        # FP32 SIMT: 152 SMs x 128 FMA/clk x 2 flop x 2.07 GHz (max boost)
        alu_peak = 152 * 128 * 2 * 2.07e9 / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak, "traffic": None, "kernel": ph[3:],
                "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x 2.07 GHz"}

    iters_total = args.steps * world
    value = iters_total / (ms * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3" if args.prec == "split_bf16" else "f32", "data": "synthetic",
        "config": {"workload": w["name"], "n": w["n"], "d": w["d"], "m": w["m"], "D": w["D"],
                   "grid": "%dx%d" % (w["R"], w["C"]), "sigma": w["sigma"], "loss": w["loss"], "reg": w["reg"],
                   "lambda": w["lam"], "rho": w["rho"], "prec": args.prec, "parallelism": "replicas",
                   "l2": "inputs larger than L2 (X split 358 MB, V 512 MB, factors 2.1 GB)"},
        "e2e": e2e,
        "gpu_launches": int(prof["launches"]),
        "phases_ms_per_iter": {k[3:]: prof[k] / max(prof["iters"], 1) for k in prof if k.startswith("ms_")},
        "useful_tflops": useful / (ms / args.steps * 1e-3) / 1e12,
        "roofline": roof,
        "clocks": clk.summary(),
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    return line


def oracle_iter_seconds(n_sample, iters):
    """Seconds per iteration of the FP64 oracle on an n_sample-row slice of the workload
    (same d, D, m, grid; set-up excluded)."""
    from oracle import admm
    w = WORKLOAD
    X, Y = make_data(w, n=n_sample)
    p = admm.Problem(X, Y, w["loss"], w["reg"], w["lam"], w["sigma"], w["rho"], w["D"], w["R"], w["C"],
                     w["philox_seed"])
    admm.admm(p, 1)                       # builds Z and the cached factors (untimed)
    t0 = time.perf_counter()
    admm.admm(p, iters)
    return (time.perf_counter() - t0) / iters


def cpu_baseline(args, n_sample=8000, iters=3):
    w = WORKLOAD
    sec = oracle_iter_seconds(n_sample, iters)
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
            "config": {"workload": WORKLOAD["name"], "prec": "f64 oracle (explicit Z)"},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="split_bf16", choices=["split_bf16", "fp32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--n", type=int, default=0, help="rows of a reduced workload (profiling runs)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
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
