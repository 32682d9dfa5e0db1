#!/usr/bin/env python
"""Benchmark: KP-SVD preconditioned flexible PCG deblurring of a 1024 x 1024
image (rank-4 Kronecker-sum blur, reflexive BC) on GB300.

One step = the whole path for one synthetic problem: kp_setup (PSF ->
Kronecker sum -> KP-SVD), then for each of the two noise levels (0.5 %, 5 %)
choose_lambda (GCV over the KP spectrum) and tik_pcg (FPCG to the relative
residual that reaches <= 1e-4 relative error against the FP64 oracle).
value = solves per second over all ranks (2 solves per step per rank).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
a bounded sample of the same step and prints its JSON line.
"""
from __future__ import annotations

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

METRIC = "time-to-solution at ≤1e-4 rel. err vs FP64 oracle (1024² deblur); solves/s"
WORKLOAD = "deblur1024_mixed"
TOL = 1e-7          # relative residual that gives <= 1e-4 error vs the oracle's x_lambda
MAXIT = 500
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=25)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--op", default="bf16", choices=["bf16", "bf16x3", "f32"])
    ap.add_argument("--pc", default="f16", choices=["f16", "bf16", "f32", "e4m3"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-form", action="store_true", help="also time the all-FP64 GPU form per iteration")
    ap.add_argument("--no-fp64-form", action="store_true", help="skip the whole-step all-FP64 GPU form")
    ap.add_argument("--n", type=int, default=None, help="override the image size (smaller test runs)")
    ap.add_argument("--host-loop", action="store_true",
                    help="run the (F)PCG iterations as host-launched graph blocks instead of the device-side "
                         "loop (the same kernels; profilers list the kernels of these blocks, not those inside "
                         "the device loop's conditional nodes)")
    ap.add_argument("--quick", action="store_true",
                    help="timed steps only (no phase breakdown, e2e, kernel timing or CPU baseline): for launch lists")
    ap.add_argument("--workload", default="deblur1024_mixed",
                    choices=["deblur1024_mixed", "batched64", "learned_lambda"],
                    help="batched64: 64 independent problems of uneven sizes through kp_solve_batch; "
                         "learned_lambda: train the lambda regressor on generated 256^2 problems and compare it "
                         "with GCV on new ones (each its own JSON line; the default workload is the headline "
                         "metric)")
    ap.add_argument("--train", type=int, default=20000, help="learned_lambda: training problems")
    ap.add_argument("--eval", type=int, default=512, help="learned_lambda: evaluation problems")
    ap.add_argument("--workers", type=int, default=0,
                    help="batched64: 0 = grouped form (one launch per iteration step over all problems, one host "
                         "thread); > 0 = that many host threads, one context each")
    ap.add_argument("--batch-tiles", default="uniform", choices=["uniform", "timed", "per-shape"],
                    help="batched64 (grouped): one tile shape for all problems (each step one launch), shapes "
                         "chosen by timing (autotuner), or the size rule of single solves")
    ap.add_argument("--opt", action="append", default=[], metavar="NAME=VALUE",
                    help="context option (kp_set_option) set before kp_setup, e.g. tc_kcat=1; repeatable "
                         "(1024^2 workload and --kernel-only)")
    ap.add_argument("--kernel-only", choices=["kapply", "minv"], default=None,
                    help="set up once, then run only the operator application (or preconditioner solve) "
                         "--steps times: for kernel profiles")
    return ap.parse_args()


# ------------------------------------------------------------------ distributed
def dist_init(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if ws > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local, dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, v: float) -> float:
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, v: float) -> float:
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t)
    return float(t.item())


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ problem
def synth_problem(name):
    from paper_2311_15393_gb300 import synth
    return synth.make_problem(name)


def make_inputs(n, seed_offset):
    from paper_2311_15393_gb300 import synth
    P = synth.make_problem(WORKLOAD, n=n, seed=synth.SEED_BASE + synth.WORKLOAD_INDEX[WORKLOAD] + seed_offset)
    return P


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# the sources of the K application's kernels (tensor-core GEMM, term sums,
# bf16 split) and the headers they include
KAPPLY_SOURCES = ("kp_gemm_tc.cu", "kp_group.cuh", "kp_internal.h", "kp_ops.cu", "kp_ops.h", "kp_vec.cu",
                  "kp_vec.cuh")


def sources_digest():
    """sha256 over the K application's CUDA sources (names and contents)."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2311_15393_gb300", "csrc")
    for name in KAPPLY_SOURCES:
        h.update(name.encode())
        with open(os.path.join(d, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def kapply_traffic(n, r):
    """DRAM bytes of one K application from the committed ncu capture
    (profiles/kapply_deblur1024_traffic.json), or None when the kernels have
    changed since it was taken or the workload differs."""
    try:
        with open(os.path.join(ROOT, "profiles", "kapply_deblur1024_traffic.json")) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    if t.get("sources_sha256") != sources_digest() or t.get("n") != n or t.get("rank") != r:
        return None
    return t.get("dram_bytes_per_k_application")


def part_rooflines(n_r, n_c, r, parts_ms, parts_launches, lambda_ms, pk_, how, dev, args):
    """Roofline entry per kernel family of the step, from the per-part CUDA
    event timings (algorithmic work per launch / time per launch)."""
    import torch
    N = n_r * n_c
    peak_tf = pk_.get("bf16_tflops")
    hbm = pk_.get("hbm_gbs")
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = pk_.get("sm_max_mhz", 2070.0)
    fp32_tf = sms * 128 * 2 * mhz * 1e6 / 1e12   # FP32 FMA lanes x 2 flops x max clock
    gemm = lambda pairs: 4.0 * pairs * n_r * n_c * (n_r + n_c)  # noqa: E731
    pc_pairs = 2 if args.pc == "bf16" else 1
    # vector phase bytes (FP32 vectors): x / r update reads x, r, p, q, writes
    # x, r, r_old (+ the 16-bit preconditioner input when folded); dots read
    # z, r, r_old; p update reads p, z and writes p and the bf16 slice of p
    folded = args.op in ("bf16", "bf16x3") and args.pc in ("f16", "bf16")
    vec_bytes = 4 * N * (4 + 3) + (2 * N if folded else 0) + 4 * N * 3 + 4 * N * 3 + 2 * N
    lam_flops = 2.0 * N * (n_r + n_c) + 400 * N * 6 + 30 * N * 12
    out = {
        "k_application": {"bound": "tensor", "work": gemm(r), "unit": "TFLOP/s", "peak": peak_tf},
        "preconditioner": {"bound": "tensor", "work": gemm(pc_pairs), "unit": "TFLOP/s", "peak": peak_tf},
        "vector_phase": {"bound": "hbm", "work": vec_bytes, "unit": "GB/s", "peak": hbm},
        "residual_replacement": {"bound": "tensor", "work": gemm(6 * r), "unit": "TFLOP/s", "peak": peak_tf},
        "lambda_gcv": {"bound": "alu", "work": lam_flops, "unit": "TFLOP/s", "peak": fp32_tf},
    }
    ms = {"k_application": parts_ms[0], "preconditioner": parts_ms[1], "vector_phase": parts_ms[2],
          "residual_replacement": parts_ms[3], "lambda_gcv": lambda_ms}
    kern = {"k_application": parts_launches[0], "preconditioner": parts_launches[1],
            "vector_phase": parts_launches[2], "residual_replacement": parts_launches[3]}
    for k, e in out.items():
        scale = 1e12 if e["unit"] == "TFLOP/s" else 1e9
        e["ms_per_launch"] = ms[k]
        e["achieved"] = e["work"] / (ms[k] * 1e-3) / scale
        e["frac"] = e["achieved"] / e["peak"]
        if k in kern:
            e["kernels_per_launch"] = kern[k]
    out["vector_phase"]["note"] = ("FP32 vectors of 4 MiB each stay in the 129 MB L2 during the iteration, so the "
                                   "HBM fraction can exceed 1")
    out["lambda_gcv"]["note"] = ("work = spectral coefficients U_c^T B U_r (FP32) + 400-point grid (~6 flops per "
                                 "term) + ~30 FP64 refinement evaluations (~12 flops per term); peak = FP32 FMA "
                                 f"rate {fp32_tf:.1f} TFLOP/s ({sms} SMs x 128 lanes x 2 x {mhz:.0f} MHz)")
    out["peak_source"] = how
    return out


# ------------------------------------------------------------------ CPU oracle sample
def oracle_sample(P, iters_per_solve, k=3):
    """Bounded sample of the step on the host cores with the FP64 oracle:
    setup, GCV lambda for one noise level, k FPCG iterations; extrapolated to
    one step (setup + 2 x (lambda + iters_per_solve iterations))."""
    import numpy as np
    from oracle import forward, kpsvd as okp, kron, lam as olam, pcg as opcg
    t0 = time.perf_counter()
    op = kron.kron_operator(P.psf, P.center, P.bc, P.op_rank)
    kp = okp.kp_svd(op, "projected")
    t1 = time.perf_counter()
    B, _ = forward.observe(op, P.x_true, P.noise_dirs[0], P.noise_levels[0])
    t2 = time.perf_counter()
    lam = olam.choose_lambda(kp, B, "gcv")
    t3 = time.perf_counter()
    opcg.tik_pcg(op, kp, B, lam, 0.0, k, True)
    t4 = time.perf_counter()
    t_setup, t_lam, t_it = t1 - t0, t3 - t2, (t4 - t3) / (k + 1)  # + A^T b and z0 ~ one iteration
    step = t_setup + 2 * (t_lam + iters_per_solve * t_it)
    return {"step_s": step, "sample_s": t4 - t0, "t_setup": t_setup, "t_lambda": t_lam, "t_iter": t_it}


def oracle_sample_1thread(n, iters_per_solve, k):
    """oracle_sample with the BLAS pinned to one thread: run in a child
    process, since the thread count of numpy's BLAS is fixed when it loads."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = (f"import sys, json; sys.path.insert(0, {ROOT!r}); import bench; "
            f"print(json.dumps(bench.oracle_sample(bench.make_inputs({n!r}, 0), {iters_per_solve}, {k})))")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        return None
    return json.loads(r.stdout.strip().splitlines()[-1])


def blas_threads():
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(k):
            return int(os.environ[k])
    return os.cpu_count()


# ------------------------------------------------------------------ reference arm
def oracle_iterations(P):
    """FP64 oracle FPCG iteration counts to TOL at both noise levels, each at
    the oracle's GCV lambda (measured once, outside the timed samples)."""
    from oracle import forward, kpsvd as okp, kron, lam as olam, pcg as opcg
    op = kron.kron_operator(P.psf, P.center, P.bc, P.op_rank)
    kp = okp.kp_svd(op, "projected")
    its = []
    for g, nl in zip(P.noise_dirs, P.noise_levels):
        B, _ = forward.observe(op, P.x_true, g, nl)
        lam = olam.choose_lambda(kp, B, "gcv")
        _, info = opcg.tik_pcg(op, kp, B, lam, TOL, MAXIT, True)
        its.append(int(info.iters))
    return its


def run_reference(args, ws, rank, dist):
    """The FP64 oracle as it stands on the host cores.  Each timed step is a
    bounded sample of the workload's step (setup, GCV lambda at one noise
    level, 3 FPCG iterations); ms_per_step is that sample's measured time.
    The solves/s value extrapolates the sample to the whole step with the
    oracle's own iteration counts (measured once before the timed samples);
    the extrapolation is reported in its own field."""
    if rank != 0:
        return 0
    n = args.n
    P = make_inputs(n, 0)
    t0 = time.perf_counter()
    iters = oracle_iterations(P)
    t_iters = time.perf_counter() - t0
    k = 3
    for _ in range(args.warmup):
        oracle_sample(P, max(iters), k)
    samples = [oracle_sample(P, max(iters), k) for _ in range(args.steps)]
    sample_s = statistics.mean(t["sample_s"] for t in samples)
    t_setup = statistics.mean(t["t_setup"] for t in samples)
    t_lam = statistics.mean(t["t_lambda"] for t in samples)
    t_it = statistics.mean(t["t_iter"] for t in samples)
    step_est = t_setup + sum(t_lam + (it + 1) * t_it for it in iters)   # + A^T b and z0 ~ one iteration
    value = 2.0 / step_est
    cores = blas_threads()
    sample = (f"per step: FP64 oracle setup (Kronecker sum + KP-SVD), GCV lambda at one noise level, {k} FPCG "
              f"iterations ({sample_s:.2f} s measured); solves/s extrapolated to setup + 2 x (lambda + the "
              f"oracle's own FPCG iteration counts {iters}, measured once in {t_iters:.1f} s)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sample_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": P.n_r, "op_rank": P.op_rank, "bc": P.bc,
                       "noise_levels": P.noise_levels, "solves_per_step": 2, "tol": TOL},
            "extrapolation": {"measured_ms_per_sample": sample_s * 1e3, "est_ms_per_full_step": step_est * 1e3,
                              "oracle_iterations": iters, "ms_setup": t_setup * 1e3, "ms_lambda": t_lam * 1e3,
                              "ms_per_iteration": t_it * 1e3},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm
def run_ours(args, ws, rank, local, dist):
    import numpy as np
    import torch
    from paper_2311_15393_gb300 import build as _build
    _build.build()
    from paper_2311_15393_gb300 import kpsvd

    dev = local
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    P = make_inputs(args.n, 1000 * rank)
    n_r, n_c = P.n_r, P.n_c
    N = n_r * n_c
    f32 = torch.float32
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=f32, device=dev)
    with torch.cuda.stream(stream):
        psf = kpsvd.to_device(P.psf, torch.float64, f"cuda:{dev}")
        xt = kpsvd.to_device(P.x_true, f32, f"cuda:{dev}")
        gs = [kpsvd.to_device(g, f32, f"cuda:{dev}") for g in P.noise_dirs]
        bs = [torch.empty(N, dtype=f32, device=dev) for _ in gs]
        xs = [torch.zeros(N, dtype=f32, device=dev) for _ in gs]
        ctx = kpsvd.KpContext(dev, stream=stream.cuda_stream)
        if args.host_loop:
            ctx.kp_set_option("device_loop", 0)
        for o in args.opt:
            name, _, value = o.partition("=")
            ctx.kp_set_option(name, float(value))
        # observed data with this context's own operator (untimed input preparation)
        ctx.kp_setup(psf, n_r, n_c, P.center, P.bc, P.op_rank, args.op, args.pc, "f32", "projected")
        for g, b, nl in zip(gs, bs, P.noise_levels):
            ctx.kp_forward(xt, g, nl, b)
    torch.cuda.synchronize()

    if args.kernel_only:
        with torch.cuda.stream(stream):
            pk = torch.randn(N, dtype=f32, device=dev)
            qk = torch.empty_like(pk)
            fn = ctx.kp_apply_K if args.kernel_only == "kapply" else ctx.kp_apply_Minv
            for _ in range(args.warmup):
                fn(pk, qk, 0.02)
            k0 = torch.cuda.Event(enable_timing=True)
            k1 = torch.cuda.Event(enable_timing=True)
            k0.record(stream)
            for _ in range(args.steps):
                fn(pk, qk, 0.02)
            k1.record(stream)
            torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"kernel_only": args.kernel_only, "n": n_r, "ms_per_call": k0.elapsed_time(k1) / args.steps,
                              "launches": ctx.kp_launch_count()}), flush=True)
        ctx.close()
        return 0

    phase = {"setup": [], "lambda": [], "solve": []}
    infos = []

    def step(record=False):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        flush.fill_(1.0)
        ev[0].record(stream)
        ctx.kp_setup(psf, n_r, n_c, P.center, P.bc, P.op_rank, args.op, args.pc, "f32", "projected")
        ev[1].record(stream)
        out = []
        for k, b in enumerate(bs):
            lam = ctx.choose_lambda(b, "gcv")
            ev[2 + 2 * k].record(stream)
            info = ctx.tik_pcg(b, lam, TOL, MAXIT, True, xs[k])
            ev[3 + 2 * k].record(stream)
            out.append((lam, info))
        if record:
            torch.cuda.synchronize()
            phase["setup"].append(ev[0].elapsed_time(ev[1]))
            phase["lambda"].append(ev[1].elapsed_time(ev[2]) + ev[3].elapsed_time(ev[4]))
            phase["solve"].append(ev[2].elapsed_time(ev[3]) + ev[4].elapsed_time(ev[5]))
            infos.append(out)
        return out

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        ctx.kp_launch_count(reset=True)
        clocks = ClockSampler(dev)
        clocks.start()
        barrier(dist)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step(record=False)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(dist)
        clk = clocks.stop()
        launches = ctx.kp_launch_count(reset=True)
        ms = e0.elapsed_time(e1) / args.steps
        ms_max = max_over_ranks(dist, ms)
        solves = 2 * args.steps
        value = sum_over_ranks(dist, solves) / (ms_max * args.steps / 1e3)

        if args.quick:
            if rank == 0:
                print(json.dumps({"quick": True, "value": value, "ms_per_step": ms_max, "gpu_launches": launches}),
                      flush=True)
            ctx.close()
            return 0
        # per-phase breakdown (separate, recorded steps)
        for _ in range(2):
            step(record=True)

        # end to end through the public API with host buffers
        pin_psf = torch.from_numpy(np.ascontiguousarray(P.psf.reshape(-1, order="F"))).pin_memory()
        pin_b = [b.to("cpu").pin_memory() for b in bs]
        pin_x = [torch.empty(N, dtype=f32).pin_memory() for _ in bs]
        torch.cuda.synchronize()
        barrier(dist)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1.0)
            psf.copy_(pin_psf, non_blocking=True)
            for b, hb in zip(bs, pin_b):
                b.copy_(hb, non_blocking=True)
            ctx.kp_setup(psf, n_r, n_c, P.center, P.bc, P.op_rank, args.op, args.pc, "f32", "projected")
            for k, b in enumerate(bs):
                lam = ctx.choose_lambda(b, "gcv")
                ctx.tik_pcg(b, lam, TOL, MAXIT, True, xs[k])
                pin_x[k].copy_(xs[k], non_blocking=True)
            stream.synchronize()
        t1 = time.perf_counter()
        barrier(dist)
        e2e_s = max_over_ranks(dist, (t1 - t0) / args.steps)
        e2e_value = sum_over_ranks(dist, 2.0) / e2e_s
        h2d = P.psf.size * 8 + sum(b.numel() * 4 for b in bs)
        d2h = sum(x.numel() * 4 for x in xs)

        # dominant-kernel timing: the operator application K p (four
        # tensor-core GEMMs) launched repeatedly on the same stream
        pk = torch.randn(N, dtype=f32, device=dev)
        qk = torch.empty_like(pk)
        for _ in range(3):
            ctx.kp_apply_K(pk, qk, 0.02)
        reps = 20
        flush.fill_(1.0)
        k0 = torch.cuda.Event(enable_timing=True)
        k1 = torch.cuda.Event(enable_timing=True)
        k0.record(stream)
        for _ in range(reps):
            ctx.kp_apply_K(pk, qk, 0.02)
        k1.record(stream)
        torch.cuda.synchronize()
        kapply_ms = k0.elapsed_time(k1) / reps

        # the iteration's parts, each timed alone on the stream (CUDA events in
        # the library): K application, preconditioner, vector phase, replacement
        lam_last = infos[-1][0][0]
        parts_ms, parts_launches = ctx.kp_time_parts(lam_last, 20)

        # lambda selection alone (GCV, the first noise level)
        l0 = torch.cuda.Event(enable_timing=True)
        l1 = torch.cuda.Event(enable_timing=True)
        ctx.choose_lambda(bs[0], "gcv")
        l0.record(stream)
        for _ in range(5):
            ctx.choose_lambda(bs[0], "gcv")
        l1.record(stream)
        torch.cuda.synchronize()
        lambda_ms = l0.elapsed_time(l1) / 5

        # the setup as the step runs it (FP32 products and rotations for FP32
        # vectors) and with the factor SVDs' work in FP64 (option setup_fp64)
        setup_ms = {}
        for name, opt in (("fp32_products", 0.0), ("fp64", 1.0)):
            ctx.kp_set_option("setup_fp64", opt)
            ctx.kp_setup(psf, n_r, n_c, P.center, P.bc, P.op_rank, args.op, args.pc, "f32", "projected")
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            for _ in range(3):
                ctx.kp_setup(psf, n_r, n_c, P.center, P.bc, P.op_rank, args.op, args.pc, "f32", "projected")
            s1.record(stream)
            torch.cuda.synchronize()
            setup_ms[name] = s0.elapsed_time(s1) / 3
        ctx.kp_set_option("setup_fp64", 0.0)
        ctx.kp_setup(psf, n_r, n_c, P.center, P.bc, P.op_rank, args.op, args.pc, "f32", "projected")

        fp64_form = None
        if not args.no_fp64_form:
            # the plain all-FP64 form on the same GPU (FP64 setup, lambda, SIMT
            # operator and preconditioner, FP64 vectors), one whole step timed
            ctx64 = kpsvd.KpContext(dev, stream=stream.cuda_stream)
            b64 = [b.double() for b in bs]
            x64 = [torch.zeros(N, dtype=torch.float64, device=dev) for _ in bs]
            ctx64.kp_setup(psf, n_r, n_c, P.center, P.bc, P.op_rank, "f64", "f64", "f64", "projected")
            torch.cuda.synchronize()
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            ctx64.kp_setup(psf, n_r, n_c, P.center, P.bc, P.op_rank, "f64", "f64", "f64", "projected")
            res64 = []
            for b64k, x64k in zip(b64, x64):
                lam64 = ctx64.choose_lambda(b64k, "gcv")
                inf64 = ctx64.tik_pcg(b64k, lam64, TOL, MAXIT, True, x64k, check=False)
                res64.append({"lambda": lam64, "iters": inf64.iters, "status": inf64.status})
            f1.record(stream)
            torch.cuda.synchronize()
            ms64 = f0.elapsed_time(f1)
            rel64 = [float(torch.linalg.norm(x.double() - x64k) / torch.linalg.norm(x64k))
                     for x, x64k in zip(xs, x64)]
            fp64_form = {"ms_per_step": ms64, "solves_per_s": 2e3 / ms64, "speedup_of_mixed": ms64 / ms_max,
                         "solves": res64, "mixed_vs_fp64_rel_diff": rel64,
                         "note": "all-FP64 GPU form through the same API (FP64 setup, GCV lambda, SIMT operator and "
                                 "preconditioner, FP64 vectors), one whole step measured with CUDA events"}
            ctx64.close()

        # latency of the small full-rank FP64 problem (64 x 64, 64 Kronecker
        # terms, zero BC, lambda 0.01): device time per FPCG iteration
        lat = None
        if not args.no_fp64_form:
            P64 = synth_problem("deblur64_fp64")
            c64 = kpsvd.KpContext(dev, stream=stream.cuda_stream)
            c64.kp_setup(kpsvd.to_device(P64.psf, torch.float64, f"cuda:{dev}"), P64.n_r, P64.n_c, P64.center,
                         P64.bc, P64.op_rank, "f64", "f64", "f64", "projected")
            xt64 = kpsvd.to_device(P64.x_true, torch.float64, f"cuda:{dev}")
            bb = torch.empty_like(xt64)
            c64.kp_forward(xt64, kpsvd.to_device(P64.noise_dirs[0], torch.float64, f"cuda:{dev}"),
                           P64.noise_levels[0], bb)
            its, ms_sol = 0, 0.0
            for rep in range(4):
                xx = torch.zeros_like(bb)
                inf = c64.tik_pcg(bb, P64.lam, 0.0, 50, True, xx, check=False)
                if rep > 0:   # the first solve builds and captures the iteration graph
                    its += inf.iters
                    ms_sol += inf.ms_solve
            lat = {"workload": "deblur64_fp64", "n": P64.n_r, "op_rank": P64.op_rank, "prec": "f64",
                   "us_per_iteration": 1e3 * ms_sol / max(its, 1), "iterations_timed": its,
                   "note": "FPCG at lambda 0.01 for 50 iterations, device time (CUDA events) per iteration, "
                           "including the solve's start and end"}
            c64.close()

        if args.fp64_form:
            ctx64 = kpsvd.KpContext(dev, stream=stream.cuda_stream)
            psf64 = psf
            ctx64.kp_setup(psf64, n_r, n_c, P.center, P.bc, P.op_rank, "f64", "f64", "f64", "projected")
            b64 = bs[0].double()
            x64 = torch.zeros(N, dtype=torch.float64, device=dev)
            lam = infos[-1][0][0]
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            ctx64.tik_pcg(b64, lam, 0.0, 2, True, x64, check=False)
            f0.record(stream)
            it64 = 5
            ctx64.tik_pcg(b64, lam, 0.0, it64, True, x64, check=False)
            f1.record(stream)
            torch.cuda.synchronize()
            ms_iter = f0.elapsed_time(f1) / (it64 + 1)
            (fp64_form or {})["ms_per_iter"] = ms_iter
            ctx64.close()

    # roofline of the dominant kernel family, the operator's tcgen05 GEMMs, per
    # K application (A and A^T: per term one n_r x n_r by n_r x n_c product and
    # one n_r x n_c by n_c x n_c product each, 4 r n_r n_c (n_r + n_c) flops in
    # all, with the two term sums and the bf16 split of p that belong to one
    # application)
    r = P.op_rank
    flops_kapply = 4.0 * r * n_r * n_c * (n_r + n_c)
    pk_, how = peaks()
    peak_tf = pk_.get("bf16_tflops")   # burst figure: the parts are timed alone
    kapply_iter_ms = parts_ms[0]
    achieved = flops_kapply / (kapply_iter_ms * 1e-3) / 1e12
    traffic = kapply_traffic(n_r, r)
    last = infos[-1]
    rooflines = part_rooflines(n_r, n_c, r, parts_ms, parts_launches, lambda_ms, pk_, how, dev, args)
    result = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n_r, "op_rank": r, "bc": P.bc, "op_prec": args.op,
                   "pc_prec": args.pc, "vec_prec": "f32", "lambda": "gcv", "noise_levels": P.noise_levels,
                   "tol": TOL, "solves_per_step": 2, "parallelism": f"replicas x{ws}",
                   "setup": "FP32 products, rotations and subspace iteration (FP64 norms, sort, Sigma); "
                            "setup_ms.fp64 times the FP64 form",
                   "l2": "256 MiB buffer written before every step",
                   "step": "kp_setup + 2 x (choose_lambda GCV + tik_pcg FPCG)",
                   **({"options": args.opt} if args.opt else {})},
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "roofline": {"kernel": "K application q = (A^T A + lambda^2 I) p as the iteration runs it "
                               f"({parts_launches[0]} kernels: tcgen05 BF16 GEMMs and term sums)",
                     "bound": "tensor", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
                     "frac": achieved / peak_tf, "traffic": traffic,
                     "peak_source": how + " bf16_tflops (burst)",
                     "flops_per_launch": flops_kapply, "ms_per_launch": kapply_iter_ms,
                     "ms_per_kp_apply_K": kapply_ms,
                     "launch": "one K application"},
        "rooflines": rooflines,
        "clocks": clk,
        "phases_ms": {k: (statistics.mean(v) if v else None) for k, v in phase.items()},
        "setup_ms": {**setup_ms, "step_uses": "fp32_products",
                     "value_with_fp64_setup": 2e3 / (ms_max - setup_ms["fp32_products"] + setup_ms["fp64"])},
        "solves": [{"lambda": lam, "iters": inf.iters, "replacements": inf.replacements,
                    "rel_res": inf.rel_res, "status": inf.status} for lam, inf in last],
    }
    if fp64_form:
        result["fp64_form"] = fp64_form
    if lat:
        result["latency_small_fp64"] = lat
    ctx.close()
    if rank == 0 and not args.no_cpu_baseline:
        iters = [inf.iters for _, inf in last]
        k_cpu = 100
        smp = oracle_sample(P, max(iters), k_cpu)
        step_s = smp["t_setup"] + sum(smp["t_lambda"] + (it + 1) * smp["t_iter"] for it in iters)
        result["cpu_baseline"] = {"value": 2.0 / step_s, "unit": "solves/s", "cores": blas_threads(),
                                  "kind": "oracle",
                                  "sample": f"FP64 oracle setup + GCV lambda (one noise level) + {k_cpu} FPCG "
                                            f"iterations ({smp['sample_s']:.1f} s measured), extrapolated to setup "
                                            f"+ 2 x lambda + the step's {iters} iterations"}
        k_one = 5
        one = oracle_sample_1thread(args.n, max(iters), k_one)
        if one is not None:
            step1 = one["t_setup"] + sum(one["t_lambda"] + (it + 1) * one["t_iter"] for it in iters)
            result["cpu_baseline"]["one_thread"] = {
                "value": 2.0 / step1, "unit": "solves/s", "cores": 1,
                "sample": f"the same with the BLAS on one thread: setup + GCV lambda + {k_one} FPCG iterations "
                          f"({one['sample_s']:.1f} s measured), extrapolated the same way"}
    if rank == 0:
        print(json.dumps(result), flush=True)
    return 0


def run_batched(args, ws, rank, local, dist):
    """64 independent problems of uneven sizes (each: own PSF, BC, noise level,
    GCV lambda) per step through kp_solve_batch; solves/s over the batch.
    Inputs are resident on the device (b formed untimed by each problem's own
    operator); e2e re-times the step with the PSFs and b copied from pinned
    host memory and every x copied back inside the timed region."""
    import numpy as np
    import torch
    from paper_2311_15393_gb300 import build as _build
    _build.build()
    from paper_2311_15393_gb300 import kpsvd, synth

    dev = local
    torch.cuda.set_device(dev)
    probs = synth.make_batch(64, seed=synth.SEED_BASE + synth.BATCH_INDEX + 1000 * rank)
    f32 = torch.float32
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=f32, device=dev)
    dp, host = [], []
    with kpsvd.KpContext(dev) as ctx:
        for P in probs:
            psf = kpsvd.to_device(P.psf, torch.float64, f"cuda:{dev}")
            xt = kpsvd.to_device(P.x_true, f32, f"cuda:{dev}")
            g = kpsvd.to_device(P.noise_dirs[0], f32, f"cuda:{dev}")
            b = torch.empty_like(xt)
            ctx.kp_setup(psf, P.n_r, P.n_c, P.center, P.bc, P.op_rank, args.op, args.pc, "f32", "projected")
            ctx.kp_forward(xt, g, P.noise_levels[0], b)
            dp.append(dict(psf=psf, b=b, x=torch.zeros_like(b), n_r=P.n_r, n_c=P.n_c, center=P.center, bc=P.bc,
                           op_rank=P.op_rank))
            host.append((psf.cpu().pin_memory(), b.cpu().pin_memory(), torch.empty_like(b, device="cpu").pin_memory()))
    torch.cuda.synchronize()

    def step():
        for d in dp:
            d["x"].zero_()
        st, ms_, res_ = kpsvd.kp_solve_batch(dp, op_prec=args.op, pc_prec=args.pc, tol=1e-7, maxit=500,
                                             workers=args.workers, device=dev, check=False,
                                             autotune={"uniform": 0, "timed": 1, "per-shape": 2}[args.batch_tiles])
        bad = [i.status for _, i in res_ if i.status not in (kpsvd.KP_OK, kpsvd.KP_ENOCONV)]
        if bad:  # anything but convergence or stagnation at FP32 accuracy is a failure
            raise RuntimeError(f"kp_solve_batch failed: statuses {bad}: {kpsvd._lib.kp_last_error().decode()}")
        return st, ms_, res_

    for _ in range(args.warmup):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        step()
    clocks = ClockSampler(dev)
    clocks.start()
    times, res = [], None
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        barrier(dist)
        t0 = time.perf_counter()
        st, _, res = step()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    clk = clocks.stop()
    barrier(dist)
    ms = max_over_ranks(dist, 1e3 * statistics.median(times))
    # a solve counts when it converged (KP_OK); a problem stopped as stagnated
    # at FP32 accuracy did not reach the metric's bar and is not counted
    n_ok = sum(info.status == kpsvd.KP_OK for _, info in res)
    value = sum_over_ranks(dist, float(n_ok)) / (ms / 1e3)

    # end to end: PSF and b from pinned host memory, x back, inside the timed region
    e2e = []
    for _ in range(max(1, min(args.steps, 3))):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for d, (hp, hb, hx) in zip(dp, host):
            d["psf"].copy_(hp, non_blocking=True)
            d["b"].copy_(hb, non_blocking=True)
        torch.cuda.synchronize()
        step()
        for d, (hp, hb, hx) in zip(dp, host):
            hx.copy_(d["x"], non_blocking=True)
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t0)
    e2e_ms = max_over_ranks(dist, 1e3 * statistics.median(e2e))
    sizes = {}
    for d, (lam, info) in zip(dp, res):
        k = f"{d['n_r']}x{d['n_c']}"
        e = sizes.setdefault(k, {"problems": 0, "iters": []})
        e["problems"] += 1
        e["iters"].append(info.iters)
    for e in sizes.values():
        e["iters"] = [min(e["iters"]), int(np.median(e["iters"])), max(e["iters"])]
    result = {"metric": "solves/s, 64 independent deblurring problems of uneven sizes (setup + GCV lambda + FPCG "
                        "to 1e-7 each; converged problems counted)",
              "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
              "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
              "data": "synthetic",
              "config": {"workload": "batched64", "sizes": [f"{a}x{b}" for a, b in synth.BATCH_SIZES],
                         "op_prec": args.op, "pc_prec": args.pc, "vec_prec": "f32", "lambda": "gcv", "tol": 1e-7,
                         "workers": args.workers,
                         "form": ("grouped: one launch per iteration step over all problems, one CUDA graph with "
                                  "a device-side loop" if args.workers <= 0 else f"{args.workers} host threads"),
                         "tiles": args.batch_tiles, "parallelism": f"replicas x{ws}",
                         "l2": "256 MiB buffer written before every step",
                         "step": "kp_solve_batch over 64 problems"},
              "e2e": {"value": sum_over_ranks(dist, float(n_ok)) / (e2e_ms / 1e3), "unit": "solves/s",
                      "h2d_bytes_per_step": sum(h[0].numel() * 8 + h[1].numel() * 4 for h in host),
                      "d2h_bytes_per_step": sum(h[2].numel() * 4 for h in host)},
              "clocks": clk,
              "converged": sum(info.status == kpsvd.KP_OK for _, info in res),
              "stagnated_above_tol": sum(info.status == kpsvd.KP_ENOCONV for _, info in res),
              "max_rel_res": max(info.rel_res for _, info in res),
              "grouped": (dict(zip(("problems", "passes", "ms", "launches"), kpsvd.kp_batch_grouped(dev)))
                          if args.workers <= 0 else None),
              "per_size": sizes}
    if rank == 0:
        print(json.dumps(result), flush=True)
    return 0


def run_learned(args, ws, rank, local, dist):
    """Learned lambda: features (kp_lambda_features) and discrepancy-principle
    labels (tau = 1.01 times the generator's exact noise norm) of generated
    256 x 256 problems (PSF and noise as in the batched workload), MLP
    training (kp_mlp_*), then on new problems lambda from the MLP vs GCV:
    relative reconstruction error against x_true and FPCG iterations."""
    import numpy as np
    import torch
    from paper_2311_15393_gb300 import build as _build
    _build.build()
    from paper_2311_15393_gb300 import kpsvd, synth

    dev = local
    torch.cuda.set_device(dev)
    f32 = torch.float32
    seed0 = synth.SEED_BASE + 4 + 1000 * rank
    ctx = kpsvd.KpContext(dev)
    feat = torch.empty(256, dtype=f32, device=dev)

    def prepare(P):
        psf = kpsvd.to_device(P.psf, torch.float64, f"cuda:{dev}")
        ctx.kp_setup(psf, P.n_r, P.n_c, P.center, P.bc, P.op_rank, args.op, args.pc, "f32", "projected")
        xt = kpsvd.to_device(P.x_true, f32, f"cuda:{dev}")
        b = torch.empty_like(xt)
        enorm = ctx.kp_forward(xt, kpsvd.to_device(P.noise_dirs[0], f32, f"cuda:{dev}"), P.noise_levels[0], b)
        ctx.kp_lambda_features(b, feat)
        return b, enorm, feat.cpu().numpy().copy()

    t0 = time.perf_counter()
    Xtr, ytr = [], []
    for P in synth.make_batch(args.train, sizes=[(256, 256)], seed=seed0):
        b, enorm, f = prepare(P)
        Xtr.append(f)
        ytr.append(np.log10(ctx.choose_lambda(b, "discrepancy", 1.01 * enorm)))
    t_data = time.perf_counter() - t0
    Xtr, ytr = np.array(Xtr, dtype=np.float64), np.array(ytr)
    mean, std = Xtr.mean(axis=0), np.maximum(Xtr.std(axis=0), 1e-3)
    rng = np.random.default_rng(seed0)
    width, depth, bs = 256, 3, 256
    sizes = [256] + [width] * depth + [1]
    vec = [mean, 1.0 / std]
    for l in range(depth + 1):
        vec += [rng.standard_normal((sizes[l + 1], sizes[l])).ravel() * np.sqrt(2.0 / sizes[l]), np.zeros(sizes[l + 1])]
    vec = np.concatenate(vec).astype(np.float32)
    Xd = torch.tensor(Xtr, dtype=f32, device=dev)
    yd = torch.tensor(ytr, dtype=f32, device=dev)
    epochs = 40
    with kpsvd.Mlp(width, depth, bs, dev) as m:
        m.set_params(vec)
        t1 = time.perf_counter()
        losses = []
        for ep in range(epochs):
            perm = torch.tensor(rng.permutation(len(ytr)), device=dev)
            Xs, ys = Xd[perm], yd[perm]
            el = [m.train_step(Xs[i:i + bs], ys[i:i + bs], 1e-3) for i in range(0, len(ytr) - bs + 1, bs)]
            losses.append(float(np.mean(el)))
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t1
        # evaluation on new problems
        rows = []
        out = torch.empty(1, dtype=f32, device=dev)
        t_inf, t_gcv = 0.0, 0.0
        for P in synth.make_batch(args.eval, sizes=[(256, 256)], seed=seed0 + 500):
            b, enorm, f = prepare(P)
            torch.cuda.synchronize()
            ta = time.perf_counter()
            ctx.kp_lambda_features(b, feat)
            m.forward(feat.view(1, 256), out)
            lam_m = float(10.0 ** out.item())
            tb = time.perf_counter()
            lam_g = ctx.choose_lambda(b, "gcv")
            tc = time.perf_counter()
            t_inf += tb - ta
            t_gcv += tc - tb
            lam_d = ctx.choose_lambda(b, "discrepancy", 1.01 * enorm)
            xt = P.x_true
            r = {"err_disc_log": abs(np.log10(lam_m / lam_d))}
            for name, lam in (("mlp", lam_m), ("gcv", lam_g)):
                x = torch.zeros_like(b)
                info = ctx.tik_pcg(b, lam, 1e-7, 500, True, x, check=False)
                X = kpsvd.from_device(x, P.n_r, P.n_c)
                r[f"err_{name}"] = float(np.linalg.norm(X - xt) / np.linalg.norm(xt))
                r[f"iters_{name}"] = info.iters
            rows.append(r)
    ctx.close()
    med = lambda k: float(np.median([r[k] for r in rows]))  # noqa: E731
    mean_ = lambda k: float(np.mean([r[k] for r in rows]))  # noqa: E731
    result = {"metric": "learned lambda (MLP on KP-spectrum features, trained on discrepancy labels) vs GCV on new "
                        "256^2 problems: median relative reconstruction error",
              "value": med("err_mlp"), "unit": "relative error", "higher_is_better": False, "n_gpus": ws,
              "data": "synthetic", "dtype": "bf16 weights, fp32 accumulation",
              "config": {"workload": "learned_lambda", "train_problems": len(ytr), "eval_problems": len(rows),
                         "size": "256x256", "mlp": f"256 -> {width} x {depth} GELU -> 1", "batch": bs,
                         "epochs": epochs, "optimizer": "Adam lr 1e-3", "label": "discrepancy, tau = 1.01"},
              "gcv": {"median_err": med("err_gcv"), "mean_iters": mean_("iters_gcv")},
              "mlp": {"median_err": med("err_mlp"), "mean_iters": mean_("iters_mlp"),
                      "median_abs_log10_vs_discrepancy": med("err_disc_log")},
              "train": {"first_epoch_loss": losses[0], "last_epoch_loss": losses[-1], "seconds": t_train,
                        "data_seconds": t_data},
              "ms_per_lambda": {"mlp": 1e3 * t_inf / len(rows), "gcv": 1e3 * t_gcv / len(rows)}}
    if rank == 0:
        print(json.dumps(result), flush=True)
    return 0


def main():
    args = parse()
    ws, rank, local, dist = dist_init(args)
    try:
        if args.impl == "reference":
            return run_reference(args, ws, rank, dist)
        if args.workload == "batched64":
            return run_batched(args, ws, rank, local, dist)
        if args.workload == "learned_lambda":
            return run_learned(args, ws, rank, local, dist)
        return run_ours(args, ws, rank, local, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
