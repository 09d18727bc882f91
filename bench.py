#!/usr/bin/env python
"""Benchmark of the SG-KKT solve on the 128x128 Q1 workload (M=6, p=3, P=84,
beta in {1e-2, 1e-4, 1e-6}): solves/s at a 1e-8 float64 relative residual.

One step = the three solves of the workload (a batch), in the library's
mixed precision (float32 operator/preconditioner/inner MINRES inside float64
iterative refinement; --precision fp64 for the plain float64 path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Multi-GPU: replicas only (each rank solves its
own batch, no collective on the data path), value = all solves / max time.
`--impl reference` times the float64 CPU oracle on bounded samples of the same
workload on the host cores.
"""
from __future__ import annotations

import os

# independent streams (three per solve: the solve and its two parallel branches) map onto this many
# hardware work queues; the runtime default of 8 serialises concurrent solves against each other
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
import argparse
import datetime
import json
import math
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SG-KKT solves/s at 1e-8 rel. residual, p50/p99 latency; SG matvec HBM GB/s"
UNIT = "solves/s"
WORKLOAD = "steady_128x128_M6_p3_P84_beta{1e-2,1e-4,1e-6}"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip fp64/e2e/profile/matvec legs")
    ap.add_argument("--sequential", action="store_true", help="solve the batch one problem at a time")
    ap.add_argument("--no-autotune", action="store_true", help="keep the built-in SG kernel choice")
    ap.add_argument("--mean-solve", choices=["exact", "vcycle"], default="exact",
                    help="mean solves of the mixed-precision preconditioner: exact (fast diagonalisation on "
                         "the tensor cores) or one V-cycle; float64 solves always use the V-cycle")
    ap.add_argument("--mass-solve", choices=["exact", "chebyshev"], default="exact",
                    help="mass blocks of the preconditioner (Sec. 5): exact (the Cholesky option; in float32 "
                         "on these grids by fast diagonalisation on the tensor cores) or Chebyshev-5")
    ap.add_argument("--serve", action="store_true",
                    help="serving stream: the first --requests seeded requests through the server")
    ap.add_argument("--requests", type=int, default=2000, help="serving stream length with --serve")
    ap.add_argument("--serve-requests", type=int, default=100,
                    help="serving leg of the default run: the first N requests of the stream (0: skip)")
    ap.add_argument("--kernel-case", choices=["vcycle128", "mean128", "sg128", "sg512", "sgr128", "sgr64t", "hgs128",
                                              "solve128"],
                    default=None,
                    help="run one kernel class a few times on a small case (for ncu captures) and exit")
    return ap.parse_args()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6800.0), "measured", d
    return 6800.0, "fallback", {}


# float64 ALU peak from unit counts and clocks: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2070 MHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
SG_KERNEL_NAMES = {0: "one-phase", 1: "quad-32", 2: "quad-16", 3: "two-phase", 4: "quad-32x4", 5: "quad-16x4",
                   6: "direct", -1: "none"}
# DRAM bytes of vcycle_t_kernel<float, 127, 2> (the current kernel) on 56 columns of the 128x128
# workload, from one ncu capture: 3,681,280 B read + 0 B written
VCYCLE_DRAM_BYTES_PER_COLUMN = 3681280 / 56
# DRAM bytes of spectral_mean_kernel<128> (the exact mean solve) on 56 columns of the 128x128
# workload, from one ncu capture: 3,748,608 B read + 0 B written
MEAN_EXACT_DRAM_BYTES_PER_COLUMN = 3740672 / 56
# DRAM bytes per float32 SG launch (all shapes) of the 128x128 mixed solve with the benchmark's
# kernel choices, from one ncu capture of the solve kernel case: 4,292,532 B read + written (the
# X panels, coefficient planes and outputs of the launch; about 2/3 of the algorithmic bytes)
SG_DRAM_BYTES_PER_LAUNCH_128 = 4292532
# tensor work of one tile (one 128 x 128 column) of the exact mean solve: 3 bf16 products for each of
# the four 128 x 128 x 128 products with the sine transform, 2 flop per MAC
MEAN_EXACT_FLOP_PER_TILE = 3 * 2 * 2 * 128 * 128 * (128 + 128)
# float32 non-tensor peak: 152 SMs x 128 FMA/clk x 2 flop x 2070 MHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


class ClockSampler:
    """nvidia-smi clock/throttle sampling, started before the warm-up so that it is running when the
    timed region starts; stop() keeps the samples whose timestamps fall inside [t0, t1]."""

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, t0=None, t1=None):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        lines = open(self.path).read().splitlines()
        os.unlink(self.path)
        return parse_clock_samples(lines, t0, t1)


THROTTLE_NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


def parse_clock_samples(lines, t0=None, t1=None):
    """Summary of nvidia-smi CSV rows (timestamp, index, clocks.sm, clocks.max.sm, power.draw,
    event-reason mask, the four reasons): the median SM clock, the maximum, and the throttle
    reasons active in the samples taken inside [t0, t1] (all samples without a window; the
    sample nearest t0 when none falls inside)."""
    rows = []
    for line in lines:
        f = [x.strip() for x in line.split(",")]
        if len(f) < 10:
            continue
        try:
            ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f")
            rows.append((ts, float(f[2]), float(f[3]), f[6:10]))
        except ValueError:
            continue
    inside = [r for r in rows if t0 is None or (t0 <= r[0] <= t1)]
    window = "timed region"
    if not inside:                             # region shorter than the sampling interval
        inside = [min(rows, key=lambda r: abs((r[0] - t0).total_seconds()))] if rows and t0 else rows
        window = "nearest sample"
    reasons = {nm for r in inside for nm, v in zip(THROTTLE_NAMES, r[3]) if v.lower().startswith("active")}
    sm = [r[1] for r in inside]
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(r[2] for r in inside) if inside else None,
            "reasons": sorted(reasons), "samples": len(sm), "window": window}


def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------- oracle arm --
def host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def blas_threads():
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(k):
            return int(os.environ[k])
    return host_cores()


def oracle_full_solve(beta, mode="vcycle", args=None):
    """One complete float64 oracle solve of the 128x128 workload (set-up, right-hand side,
    preconditioner construction and preconditioned MINRES to the 1e-8 rule) with the mean solves
    of `mode` (one V-cycle, or exact: the oracle's sparse LU) and the GPU arm's mass blocks;
    returns (seconds, iterations, true relative residual)."""
    import sg_inputs as si
    from oracle.solve import solve
    t0 = time.perf_counter()
    res = solve(oracle_problem(beta, args) if args is not None else si.steady_128(beta), mode=mode)
    return time.perf_counter() - t0, res.iterations, res.rel_true


def oracle_iterations():
    """Iteration counts of the oracle's complete solves stored with the test data (used only to
    size the reference arm's steps before its own solves complete)."""
    path = os.path.join(ROOT, "tests", "golden", "full_size_oracle.json")
    out = {}
    if os.path.exists(path):
        g = json.load(open(path))
        for b in (1e-2, 1e-4, 1e-6):
            key = "steady_128_beta%g" % b
            if key in g:
                out[b] = g[key]["iterations"]
    return out


def oracle_mode(args):
    """The oracle's mean-solve mode matching the GPU arm: exact (sparse LU) when the mixed path
    uses the exact mean solves, else one V-cycle."""
    return "exact" if args.precision == "mixed" and args.mean_solve == "exact" else "vcycle"


def oracle_problem(beta, args):
    """The 128x128 workload at beta with the GPU arm's mass-block option."""
    import dataclasses
    import sg_inputs as si
    return dataclasses.replace(si.steady_128(beta), mass_solve=args.mass_solve)


def cpu_baseline_full(beta=1e-2, mode="vcycle", args=None):
    sec, its, rel = oracle_full_solve(beta, mode, args)
    mass = args.mass_solve if args is not None else "chebyshev"
    return {"value": 1.0 / sec, "unit": UNIT, "cores": host_cores(), "blas_threads": blas_threads(),
            "kind": "oracle",
            "sample": f"one complete oracle solve of the 128x128 workload at beta={beta:g} ({its} MINRES "
                      f"iterations, true residual {rel:.2e}, mean solves: {mode}, mass blocks: {mass}) in "
                      f"{sec:.1f} s, set-up included"}


class OracleStream:
    """Complete oracle solves of the workload run back to back (beta cycling through the three
    values) in a worker thread; the oracle itself is unchanged.  Each KKT product the oracle's
    MINRES asks for waits for a permit, so the caller advances the running solve by a chosen
    number of Krylov iterations at a time and times exactly that work (the set-up of a new
    solve falls into the step that first needs it)."""

    def __init__(self, betas, mode="vcycle", args=None):
        import threading
        self.betas = betas
        self.mode = mode
        self.args = args
        self.sem = threading.Semaphore(0)
        self.cv = threading.Condition()
        self.products = 0
        self.cur = 0
        self.completed = []                    # (beta, iterations, products, seconds)
        self.stop = False
        self.error = None
        self.thread = threading.Thread(target=self._run, daemon=True)
        self.thread.start()

    def _run(self):
        import sg_inputs as si
        from oracle.krylov import minres
        from oracle.operators import SGData
        from oracle.precond import BlockPreconditioner
        i = 0
        try:
            while not self.stop:
                beta = self.betas[i % len(self.betas)]
                i += 1
                t0 = time.perf_counter()
                pr = oracle_problem(beta, self.args) if self.args is not None else si.steady_128(beta)
                d = SGData(pr)
                Pc = BlockPreconditioner(d, mode=self.mode)
                b = d.rhs()

                def apply_A(v, d=d):
                    self.sem.acquire()
                    if self.stop:
                        raise SystemExit
                    y = d.kkt_apply(v)
                    with self.cv:
                        self.products += 1
                        self.cur += 1
                        self.cv.notify_all()
                    return y

                res = minres(apply_A, Pc.apply, b, tol=pr.tol, max_iter=pr.max_iter)
                with self.cv:
                    self.completed.append((beta, res.iterations, self.cur, time.perf_counter() - t0))
                    self.cur = 0
        except SystemExit:
            pass
        except Exception as e:                  # reported by advance()
            with self.cv:
                self.error = repr(e)
                self.cv.notify_all()

    def advance(self, k):
        with self.cv:
            goal = self.products + k
        for _ in range(k):
            self.sem.release()
        with self.cv:
            self.cv.wait_for(lambda: self.products >= goal or self.error is not None)
            if self.error:
                raise RuntimeError(self.error)

    def close(self):
        self.stop = True
        for _ in range(4):
            self.sem.release()


def run_reference(args):
    world, rank, _ = dist_info()
    if rank != 0:
        return
    its = oracle_iterations()
    mean_its = sum(its.values()) / len(its) if its else 41.0
    # each timed step advances the running oracle solve by `chunk` KKT products (one per MINRES
    # iteration, one per true-residual check); the timed steps cover at least one whole solve
    chunk = max(1, math.ceil((mean_its + 2) / max(args.steps, 1)))
    stream = OracleStream((1e-2, 1e-4, 1e-6), oracle_mode(args), args)
    for _ in range(args.warmup):
        stream.advance(1)
    p0 = stream.products
    step_s = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        stream.advance(chunk)
        step_s.append(time.perf_counter() - t0)
    products = stream.products - p0
    done = list(stream.completed)
    stream.close()
    per_solve = (sum(c[2] for c in done) / len(done)) if done else mean_its + 1
    total_s = sum(step_s)
    solves = products / per_solve
    value = solves / total_s
    sample = (f"{args.steps} steps of {chunk} KKT products each ({products} in all, {solves:.2f} solves at "
              f"{per_solve:.1f} products per complete solve) of complete oracle solves run back to back "
              f"(beta 1e-2, 1e-4, 1e-6 in turn, set-up included); solves completed so far: "
              + ", ".join(f"beta={b:g} {it} iterations {sec:.1f} s" for b, it, _, sec in done))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "solves_per_step": solves / args.steps,
                   "step": f"{chunk} KKT products of the running oracle solve",
                   "mean_solves": oracle_mode(args), "mass_blocks": args.mass_solve},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": host_cores(), "blas_threads": blas_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm --
def run_ours(args):
    import torch
    import sg_inputs as si
    world, rank, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2512_23804_gb300 import SGProblem, abi, build, solve_batch
    build.build()
    lib = abi.load()
    hbm_peak, peak_kind, _ = load_peaks()

    betas = si.STEADY_128_BETAS
    problems = [si.steady_128(b) for b in betas]
    mean_solve = args.mean_solve if args.precision == "mixed" else "vcycle"
    mass_solve = args.mass_solve
    sps = [SGProblem.from_problem(pr, precision=args.precision, mean_solve=mean_solve, mass_solve=mass_solve).upload()
           for pr in problems]
    for sp in sps:
        sp.workspace()
    # SG kernel per launch shape (process-wide; the three problems share their shapes); untimed
    sg_kernels = None if args.no_autotune else sps[0].autotune()
    xs = [torch.empty(sp.kkt_size, dtype=torch.float64, device="cuda") for sp in sps]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    streams = [torch.cuda.Stream() for _ in sps]

    def step_sequential():
        infos = []
        for sp, x in zip(sps, xs):
            _, info = sp.solve(out=x)
            infos.append(info)
        return infos

    def step():
        if args.sequential:
            return step_sequential()
        _, infos = solve_batch(sps, outs=xs, streams=streams)
        return infos

    sampler = ClockSampler(local)
    sampler.start()                            # running before the timed region starts
    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_region0 = datetime.datetime.now()
    l0 = lib.sgoc_kernel_launches()
    step_ms, solve_ms, iters, outer, resid = [], [], [], [], []
    for _ in range(args.steps):
        flush.fill_(1.0)                       # L2 flush (256 MiB write), outside the events
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        infos = step()
        s1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(s0.elapsed_time(s1))
        for info in infos:
            solve_ms.append(info["ms_total"])
            iters.append(info["iterations"])
            outer.append(info["outer_iterations"])
            resid.append(info["rel_true_residual"])
    torch.cuda.synchronize()
    launches = lib.sgoc_kernel_launches() - l0
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop(t_region0, datetime.datetime.now())
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    solves = 3 * args.steps * world
    value = solves / (total_ms / 1e3)
    assert max(resid) <= 1e-8, resid

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32/f64" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "solves_per_step": 3, "n": sps[0].n, "P": sps[0].P,
                   "kkt_unknowns": sps[0].kkt_size,
                   "precision": ("float32 operator/preconditioner/inner MINRES, float64 refinement"
                                 if args.precision == "mixed" else "float64"),
                   "l2": "flushed between steps (256 MiB write)", "parallelism": f"replicas x{world}",
                   "batching": "sequential" if args.sequential else "3 concurrent solves (sgoc_solve_batch, 3 streams)",
                   "mean_solves": ("exact: fast diagonalisation, tcgen05 tensor cores" if mean_solve == "exact"
                                   else "one V(2,2) multigrid cycle"),
                   "mass_blocks": ("exact (Sec. 5 Cholesky option)" + (": fast diagonalisation, tcgen05 tensor cores"
                                   if args.precision == "mixed" else ": Cholesky factors of M1")
                                   if mass_solve == "exact" else "Chebyshev-5"),
                   "sg_kernels": "built-in choice" if sg_kernels is None else
                   dict(zip(["kkt", "operator"] + [f"hgs_level{d}" for d in range((len(sg_kernels) - 2) // 2)] +
                            [f"hgs_level{d}_first" for d in range((len(sg_kernels) - 2) // 2)],
                            [SG_KERNEL_NAMES[v] for v in sg_kernels]))},
        "latency_ms": {"p50": float(sorted(solve_ms)[len(solve_ms) // 2]),
                       "p99": float(sorted(solve_ms)[min(len(solve_ms) - 1, math.ceil(0.99 * len(solve_ms)) - 1)])},
        "iterations": {"per_solve": iters[:3], "outer": outer[:3], "max_rel_residual": max(resid)},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }

    if not args.no_extras and rank == 0:
        # the same three solves one after the other (no overlap), same precision
        flush.fill_(1.0)
        q0 = torch.cuda.Event(enable_timing=True)
        q1 = torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        step_sequential()
        q1.record(stream)
        torch.cuda.synchronize()
        line["sequential_solves_per_s"] = 3 / (q0.elapsed_time(q1) / 1e3)
        # the merged schedule (sgoc_solve_batch_merged: the three solves in lockstep, each hGS
        # level visit one SG and one V-cycle launch for all three), same solves
        solve_batch(sps, outs=xs, streams=streams, merged=True)          # capture the group graphs
        mt = []
        for _ in range(2):
            flush.fill_(1.0)
            q0.record(stream)
            solve_batch(sps, outs=xs, streams=streams, merged=True)
            q1.record(stream)
            torch.cuda.synchronize()
            mt.append(q0.elapsed_time(q1))
        line["merged_batch_solves_per_s"] = 3 / (min(mt) / 1e3)
        # plain float64 path (same solves), for the mixed-vs-fp64 comparison: the error of every
        # mixed solution of the step against the float64 GPU solution of the same problem
        if args.precision == "mixed":
            xmix = [x.clone() for x in xs]
            sp64 = [SGProblem.from_problem(pr, precision="fp64", mass_solve=mass_solve).upload() for pr in problems]
            t64, it64, err = [], [], []
            for sp, x, xm in zip(sp64, xs, xmix):
                sp.solve(out=x)                    # warm
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                _, info = sp.solve(out=x)
                e1.record(stream)
                torch.cuda.synchronize()
                t64.append(e0.elapsed_time(e1))
                it64.append(info["iterations"])
                err.append(float(torch.linalg.norm(xm - x) / torch.linalg.norm(x)))
                sp.release_workspace()
            line["fp64_path"] = {"solves_per_s": 3 / (sum(t64) / 1e3), "ms_per_solve": t64, "iterations": it64}
            line["iterations"]["mixed_vs_fp64_rel_error"] = err
            del sp64, xmix

        # end to end through the public API: host arrays in, host solutions out, the solves run
        # as in the timed step (concurrently, or one after another with --sequential)
        pin = [torch.empty(sp.kkt_size, dtype=torch.float64, pin_memory=True) for sp in sps]
        h2d = d2h = 0
        e2e_ms = []
        for rep in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sps_e = [SGProblem.from_problem(pr, precision=args.precision, mean_solve=mean_solve,
                                            mass_solve=mass_solve).upload() for pr in problems]
            if args.sequential:
                xs_e = [sp.solve()[0] for sp in sps_e]
            else:
                xs_e, _ = solve_batch(sps_e)
            for x, hx in zip(xs_e, pin):
                hx.copy_(x, non_blocking=True)
            torch.cuda.synchronize()
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
            if rep == 0:
                h2d = sum(sp.persistent_bytes for sp in sps_e)
                d2h = sum(sp.kkt_size * 8 for sp in sps_e)
            del sps_e, xs_e
        line["e2e"] = {"value": 3 / (min(e2e_ms) / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h,
                       "includes": "problem set-up from host arrays, upload, workspaces, the three solves "
                                   + ("one after another" if args.sequential else "concurrently (sgoc_solve_batch)")
                                   + ", D2H of each x"}

        # instrumented pass: per-kernel-class device time with CUDA events on the launching stream
        abi.profile_enable(True)
        flush.fill_(1.0)
        step_sequential()
        torch.cuda.synchronize()
        rep = abi.profile_report()
        abi.profile_enable(False)
        tot = sum(v["ms"] for v in rep.values())
        kinds = {k: dict(v, share=v["ms"] / tot) for k, v in rep.items()}
        dom = max(kinds, key=lambda k: kinds[k]["ms"])
        dv = kinds[dom]
        esize_fp64 = args.precision == "fp64"
        if dom == "mean_exact":
            peaks = load_peaks()[2]
            tpk = peaks.get("bf16_tflops_sustained", 1700.0)
            ach = dv["flops"] / (dv["ms"] / 1e3) / 1e12
            roof = {"bound": "tensor", "achieved": ach, "peak": tpk, "unit": "TFLOP/s", "frac": ach / tpk,
                    "traffic": None, "kernel": dom,
                    "peak_source": ("measured (MEASURED_PEAKS.json bf16_tflops_sustained: cuBLAS bf16, the "
                                    "kernel is timed inside a long step)" if "bf16_tflops_sustained" in peaks
                                    else "fallback 1.7 PFLOP/s sustained"),
                    "flops_note": "bf16 tensor flops executed: three bf16 products per float32-accurate product"}
        elif esize_fp64 and dom in ("sg_operator", "mg_vcycle_fused", "mg_smooth"):
            ach = dv["flops"] / (dv["ms"] / 1e3) / 1e12
            roof = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": ach / FP64_PEAK_TFLOPS, "traffic": None, "kernel": dom,
                    "peak_source": "152 SMs x 2 FP64 FMA/clk x 2 x 2070 MHz"}
        else:
            ach = dv["bytes"] / (dv["ms"] / 1e3) / 1e9
            roof = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                    "traffic": None, "kernel": dom, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"}
        roof["launches"] = dv["launches"]
        roof["avg_launch_us"] = 1e3 * dv["ms"] / dv["launches"]
        pr_main = problems[0]
        if dom == "mg_vcycle_fused" and not esize_fp64 and pr_main.nx == 128 and VCYCLE_DRAM_BYTES_PER_COLUMN:
            # DRAM bytes per column from an ncu capture of this kernel on 56 columns of the
            # 128x128 workload, times the average columns per launch here (each hGS launch reads
            # b and reads + writes the output: 3 x 4 B per node)
            cols = dv["bytes"] / dv["launches"] / (3 * 4 * pr_main.n)
            roof["traffic"] = VCYCLE_DRAM_BYTES_PER_COLUMN * cols
            roof["traffic_note"] = f"ncu DRAM bytes per column x {cols:.1f} columns per launch"
        if dom == "sg_operator" and not esize_fp64 and pr_main.nx == 128 and SG_DRAM_BYTES_PER_LAUNCH_128:
            roof["traffic"] = SG_DRAM_BYTES_PER_LAUNCH_128
            roof["traffic_note"] = "ncu DRAM bytes per float32 SG launch of this solve (kernel case solve128)"
        if dom == "mean_exact" and pr_main.nx == 128 and MEAN_EXACT_DRAM_BYTES_PER_COLUMN:
            cols = dv["flops"] / dv["launches"] / MEAN_EXACT_FLOP_PER_TILE       # one column per tile
            roof["traffic"] = MEAN_EXACT_DRAM_BYTES_PER_COLUMN * cols
            roof["traffic_note"] = f"ncu DRAM bytes per column x {cols:.1f} columns per launch"
        line["roofline"] = roof
        line["kernel_breakdown_note"] = ("summed device time per kernel class of an eager sequential pass of "
                                         "the three solves (CUDA events around every launch; overlapping "
                                         "branches counted separately), not a share of the timed step")
        line["kernel_breakdown"] = {k: {"share": round(v["share"], 4), "launches": v["launches"],
                                        "ms": round(v["ms"], 3),
                                        "GB/s": round(v["bytes"] / max(v["ms"], 1e-9) / 1e6, 1)}
                                    for k, v in sorted(kinds.items(), key=lambda kv: -kv[1]["ms"])}

        # SG matvec bandwidth: 128x128 workload (L2-resident operands) and a 512x512, M=8, p=3
        # operand set (P=165) larger than L2; float32 and float64; L2 flushed between launches
        mv = {}
        for tag, pr in (("128x128_P84", problems[1]), ("512x512_P165", si.steady_512())):
            sp = SGProblem.from_problem(pr).upload()
            for dt, name in ((torch.float32, "f32"), (torch.float64, "f64")):
                X = torch.randn(sp.n * sp.P, dtype=dt, device="cuda")
                Y = torch.empty_like(X)
                w = X.element_size()
                byts = w * (2 * sp.n * sp.P) + w * (pr.M + 1) * pr.nx * pr.nx
                per = {}
                for v in range(7):
                    try:
                        sp.apply_operator_variant(X, v, out=Y)
                    except abi.SgocError:
                        continue
                    ts = []
                    for _ in range(5):
                        flush.fill_(1.0)
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        sp.apply_operator_variant(X, v, out=Y)
                        e1.record(stream)
                        torch.cuda.synchronize()
                        ts.append(e0.elapsed_time(e1))
                    per[SG_KERNEL_NAMES[v]] = statistics.median(ts) / 1e3
                best = min(per, key=per.get)
                t = per[best]
                mv[f"{tag}_{name}"] = {"GB/s": byts / t / 1e9, "frac_hbm": byts / t / 1e9 / hbm_peak,
                                       "us": t * 1e6, "kernel": best,
                                       "us_per_kernel": {k: round(v * 1e6, 1) for k, v in per.items()}}
            del sp
        line["sg_matvec"] = mv

    if not args.no_extras and rank == 0:
        # the other workload shapes: one timed solve each (after a warm-up solve), mixed and float64
        ow = {}
        def paper_setting():
            # the paper's own setting (Hermite chaos, lognormal field with sigma = 0.4, [-1,1]^2,
            # gamma = 1, discontinuous target, n_A = C(9, 6) = 84 coefficient terms, r = m + 1),
            # solved with the paper's Krylov method, unrestarted FGMRES
            pr = si.paper_problem(32, 3, 3, beta=1e-4, sigma=0.4)
            pr.krylov, pr.restart = "fgmres", 256
            return pr

        for name, mk in (("steady_16x16_M2_p2", si.steady_16), ("time_64x64_M4_p3_nt32", si.time_64),
                         ("steady_512x512_M8_p3", si.steady_512),
                         ("paper_hermite_32x32_M3_p3_sigma0.4_fgmres", paper_setting)):
            pr = mk()
            rec = {"kkt_unknowns": pr.kkt_size}
            xkeep = {}
            # library defaults (V-cycle mean solves, Chebyshev-5 mass blocks), and on the grids of the
            # tensor-core transform also the benchmark's setting (exact mean and mass solves)
            variants = ["mixed", "fp64"] + (["mixed_exact"] if pr.nx in (64, 128) else [])
            for prec in variants:
                ex = prec == "mixed_exact"
                sp = SGProblem.from_problem(pr, precision="mixed" if ex else prec,
                                            mean_solve="exact" if ex else "vcycle",
                                            mass_solve="exact" if ex else "chebyshev").upload()
                if not args.no_autotune:
                    sp.autotune()
                x, _ = sp.solve()
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                x, info = sp.solve(out=x)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                rec[prec] = {"ms": ms, "solves_per_s": 1e3 / ms, "iterations": info["iterations"],
                             "outer": info["outer_iterations"], "rel_residual": info["rel_true_residual"]}
                xkeep[prec] = x
                del sp
                torch.cuda.empty_cache()
            rec["mixed_vs_fp64_rel_error"] = float(torch.linalg.norm(xkeep["mixed"] - xkeep["fp64"]) /
                                                   torch.linalg.norm(xkeep["fp64"]))
            del xkeep
            torch.cuda.empty_cache()
            ow[name] = rec
        line["other_workloads"] = ow

    if not args.no_extras and rank == 0 and args.serve_requests > 0:
        line["serving"] = serve_leg(args.serve_requests)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_full(1e-2, oracle_mode(args), args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_kernel_case(args):
    """A few launches of one kernel class on a small case, for hardware-counter captures."""
    import torch
    import sg_inputs as si
    from paper_2512_23804_gb300 import SGProblem, build
    build.build()
    case = args.kernel_case
    pr = si.steady_512() if case == "sg512" else (si.time_64() if case == "sgr64t" else si.steady_128(1e-4))
    sp = SGProblem.from_problem(pr, precision="mixed", mean_solve="exact" if case == "mean128" else "vcycle").upload()
    if case == "solve128":
        # a few MINRES iterations of the 128x128 workload (loose tolerance), launched eagerly
        # (per-kernel timing on) so that a profiler sees ordinary launches, not graph nodes, with
        # the SG kernels the benchmark's tuning chooses on this workload in plain runs (quad on
        # 32-node tiles for the KKT product, the operator and the visits of levels 2 and 3, the
        # direct kernel for the others), pinned rather than tuned: tuning by timing inside a
        # profiled process would time the variants under the profiler.  The profiler range
        # (cudaProfilerStart / Stop, for `ncu --profile-from-start off`) holds the solves only.
        from paper_2512_23804_gb300 import abi
        sq = SGProblem.from_problem(pr, precision="mixed", tol=1e-2, mean_solve=args.mean_solve,
                                    mass_solve=args.mass_solve).upload()
        for shape, var in enumerate([1, 1, 6, 6, 1, 1, 6, 6, 6, 1]):
            sq.set_kernel(shape, var)
        torch.cuda.synchronize()
        abi.profile_enable(True)
        torch.cuda.profiler.start()
        for _ in range(2):
            sq.solve()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        abi.profile_enable(False)
    elif case in ("sg128", "sg512"):
        X = torch.randn(sp.n * sp.P, dtype=torch.float32, device="cuda")
        Y = torch.empty_like(X)
        for _ in range(3):
            sp.apply_operator(X, out=Y)
    elif case in ("sgr128", "sgr64t"):                 # the register SG kernel (variant 7)
        X = torch.randn(sp.n * sp.P * sp.slabs, dtype=torch.float32, device="cuda")
        Y = torch.empty_like(X)
        for _ in range(3):
            sp.apply_operator_variant(X, 7, nslabs=sp.slabs, out=Y)
    elif case in ("vcycle128", "mean128"):
        ncols = 56                                  # the largest chaos level of M=6, p=3
        R = torch.randn(ncols * sp.n, dtype=torch.float32, device="cuda")
        X = torch.empty_like(R)
        for _ in range(3):
            sp.apply_vcycle(R, ncols, out=X)
    else:
        R = torch.randn(sp.n * sp.P, dtype=torch.float32, device="cuda")
        for _ in range(2):
            sp.apply_hgs(R)
    torch.cuda.synchronize()
    print(json.dumps({"kernel_case": case, "ok": True}))


def serve_leg(n_requests, pool_cap_bytes=120e9, max_active=16, keep_every=1, queue_depth=32,
              out_cap=24e9, keep_cap=16e9):
    """Serving stream: the first `n_requests` seeded requests (grids 32..256, M 2..8, p 1..4,
    30 % time-dependent), admitted by the server's own memory-footprint check (a request that
    cannot fit the pool even when empty is rejected by sgoc_server_submit and counted), solved to a
    1e-8 float64 residual in mixed precision (on 64 x 64 and 128 x 128 grids with exact mean solves
    and mass blocks on the tensor cores, float64 with exact mass blocks; library defaults
    elsewhere).  Run once with every request arriving at t = 0
    (capacity mu), then as a Poisson stream at 0.8 mu; compared with sequential plain float64
    solves of the same requests on the same GPU, and each mixed result (every keep_every-th request
    while the kept solutions take at most keep_cap bytes of device memory) with its float64 one."""
    import numpy as np
    import torch
    import sg_inputs as si
    from paper_2512_23804_gb300 import SGProblem, SGServer, abi
    reqs = [si.serving_request(i) for i in range(n_requests)]
    pool_bytes = int(min(torch.cuda.mem_get_info()[0] * 0.6, pool_cap_bytes))

    def options(pr, precision):
        # the benchmark's preconditioner setting where the tensor-core transform applies (64 x 64
        # and 128 x 128 grids: exact mean solves in mixed precision, exact mass blocks), else
        # the library defaults
        if pr.nx not in (64, 128):
            return {}
        return dict(mass_solve="exact", mean_solve="exact" if precision == "mixed" else "vcycle")

    def run_stream(arrivals, keep):
        # Arrived requests wait in a client-side queue and are submitted while fewer than
        # queue_depth are outstanding and their float64 output buffers (the caller's memory,
        # outside the pool) stay under out_cap; latency runs from arrival to retirement.
        sv = SGServer(pool_bytes=pool_bytes, max_active=max_active)
        sps = [SGProblem.from_problem(pr, precision="mixed", **options(pr, "mixed")) for pr in reqs]
        done, lat, rejected, xs, failed = {}, {}, [], {}, []
        queue, out_live, kept_bytes = [], {}, 0
        t0 = time.perf_counter()
        nxt = 0
        while len(done) + len(rejected) < len(reqs):
            now = time.perf_counter() - t0
            while nxt < len(reqs) and arrivals[nxt] <= now:
                queue.append(nxt)
                nxt += 1
            while queue and sv.pending < queue_depth and \
                    sum(out_live.values()) + 8 * sps[queue[0]].kkt_size <= out_cap:
                i = queue.pop(0)
                try:
                    sv.submit(sps[i], i)
                    out_live[i] = 8 * sps[i].kkt_size
                except abi.SgocError as e:
                    if e.status != abi.SGOC_ERR_WORKSPACE_TOO_SMALL:
                        raise
                    rejected.append(i)
            if queue and sv.pending == 0 and not out_live:
                i = queue.pop(0)          # larger than out_cap alone: submit it by itself
                try:
                    sv.submit(sps[i], i)
                    out_live[i] = 8 * sps[i].kkt_size
                except abi.SgocError as e:
                    if e.status != abi.SGOC_ERR_WORKSPACE_TOO_SMALL:
                        raise
                    rejected.append(i)
            if sv.pending == 0:
                if nxt < len(reqs) and not queue:
                    time.sleep(max(0.0, min(arrivals[nxt] - now, 0.01)))
                continue
            sv.step()
            for rid, x, info in sv.poll():
                t_done = time.perf_counter() - t0
                done[rid] = info
                out_live.pop(rid, None)
                sps[rid] = None
                if info["status_name"] != "SGOC_OK" or not info["rel_true_residual"] <= 1e-8:
                    failed.append({"id": rid, "status": info["status_name"],
                                   "rel_residual": info["rel_true_residual"],
                                   "error": abi.load().sgoc_last_error().decode()[:200]})
                    continue
                lat[rid] = (t_done - arrivals[rid]) * 1e3
                nb = x.numel() * 8
                if keep and rid % keep_every == 0 and kept_bytes + nb <= keep_cap:
                    xs[rid] = x
                    kept_bytes += nb
        wall = time.perf_counter() - t0
        stats = sv.stats()
        del sv, sps
        l = sorted(lat.values())
        rec = {"solves_per_s": len(lat) / wall, "wall_s": wall, "completed": len(lat),
               "failed": failed, "rejected": len(rejected), "rejected_ids": rejected,
               "p50_ms": l[len(l) // 2], "p99_ms": l[min(len(l) - 1, int(math.ceil(0.99 * len(l))) - 1)],
               "pool_high_water_GB": stats["pool_high_water"] / 1e9, "admitted": stats["admitted"]}
        return rec, xs, rejected

    sat, xmix, rejected = run_stream([0.0] * len(reqs), keep=True)      # capacity mu
    mu = sat["solves_per_s"]
    rng = np.random.default_rng([5, 2**31])            # the arrival stream of master seed 5
    gaps = rng.exponential(1.0 / (0.8 * mu), size=len(reqs))
    arrivals = list(np.cumsum(gaps) - gaps[0])
    open_loop, _, _ = run_stream(arrivals, keep=False)
    torch.cuda.empty_cache()
    # sequential plain float64 solves of the same (admitted) requests
    torch.cuda.synchronize()
    seq_lat, errs, seq_failed = [], [], []
    t0 = time.perf_counter()
    served = set(i for i in range(len(reqs)) if i not in rejected)
    for i, pr in enumerate(reqs):
        if i not in served:
            continue
        sp = SGProblem.from_problem(pr, precision="fp64", **options(pr, "fp64"))
        t1 = time.perf_counter()
        try:
            x, info = sp.solve()
        except abi.SgocError as e:
            seq_failed.append({"id": i, "error": str(e)[:200]})
            continue
        seq_lat.append((time.perf_counter() - t1) * 1e3)
        if i in xmix:
            errs.append(float(torch.linalg.norm(xmix[i] - x) / torch.linalg.norm(x)))
        del sp, x
    seq_wall = time.perf_counter() - t0
    del xmix
    torch.cuda.empty_cache()
    sl = sorted(seq_lat)
    seq = {"solves_per_s": len(sl) / seq_wall, "failed": seq_failed, "p50_ms": sl[len(sl) // 2],
           "p99_ms": sl[min(len(sl) - 1, int(math.ceil(0.99 * len(sl))) - 1)]}
    return {"requests": len(reqs), "pool_GB": pool_bytes / 1e9, "max_active": max_active,
            "solves_per_s": sat["solves_per_s"], "p50_ms": sat["p50_ms"], "p99_ms": sat["p99_ms"],
            "rejected": sat["rejected"], "saturated": sat, "poisson_at_0.8mu": open_loop,
            "sequential_fp64": seq, "vs_sequential_fp64": sat["solves_per_s"] / seq["solves_per_s"],
            "mixed_vs_fp64_rel_error": {"max": max(errs), "median": statistics.median(errs), "compared": len(errs)}}


def run_serve(args):
    import torch
    from paper_2512_23804_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    rec = serve_leg(args.requests, keep_every=1 if args.requests <= 200 else 10)
    print(json.dumps(dict(mode="serve", **rec)), flush=True)


def main():
    args = parse()
    if args.kernel_case:
        run_kernel_case(args)
        return
    if args.serve:
        run_serve(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
