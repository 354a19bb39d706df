#!/usr/bin/env python
"""Benchmark: reduced-solve implicit-Euler steps per second on one GB300.

Workload (default): block_twist_960k - block of 101x41x41 nodes (960,000
tets, n = 509,343), x = 0 face fixed, x = L face twisted 2 rad and pushed in
by 0.2 L over 150 frames, implicit Euler dt = 1/60, r = 64, decoder
64-1024-1024-1024-509343 (seeded Xavier weights, output scale 1e-2), every tet
evaluated (no cubature), Stable Neo-Hookean E = 1e5 Pa, nu = 0.45,
rho = 1000.  BF16 form by default: BF16 decoder weights and tensor-core
contractions, FP32 element math, FP64 Cholesky and energy comparison.

A step is one implicit-Euler time step solved by projective Newton (default;
--optimizer lbfgs: L-BFGS with gradient-only passes) to ||g||_inf < 1e-5 (or
its precision-floor / iteration-cap exit): decoder + Jacobian, element kernel
+ contraction, Cholesky, line search, until exit.  The W warm-up steps solve
frames 1..W from rest; the state is then reset to rest and frames 1..K are
timed, so the timed steps are the workload's first K steps (the steps whose
error against the FP64 oracle is reported).  Inputs (constraint targets of
every frame, decoder weights, mesh) are resident in HBM before the timed
region; the L2 is flushed (256 MiB write) between timed steps, outside the
per-step CUDA events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (under torchrun) runs N independent replicas, one per GPU (the solve
does not shard); value = all ranks' steps / max-over-ranks time.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "reduced-solve steps/s on 1 GB300 at stated rel. error vs FP64 oracle; % roofline"
WORKLOAD = "block_twist_960k"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", default="bf16", choices=["fp64", "fp32", "tf32", "bf16"],
                    help="bf16 (default): BF16 weights and tensor-core contractions, FP32 "
                         "element math, FP64 Cholesky and energy comparison")
    ap.add_argument("--optimizer", default="newton", choices=["newton", "lbfgs"],
                    help="newton (default): projective Newton; lbfgs: L-BFGS (Sec. 5), "
                         "gradient-only passes")
    ap.add_argument("--history", type=int, default=10, help="L-BFGS history size")
    ap.add_argument("--r", type=int, default=None,
                    help="override the workload's subspace dimension (r-sweep)")
    ap.add_argument("--cpu-seconds", type=float, default=30.0,
                    help="time budget of the CPU-oracle baseline sample (at least one "
                         "frame is always completed)")
    ap.add_argument("--cpu-workers", type=int, default=None,
                    help="oracle worker processes for the chunked element sums "
                         "(default: every host core on meshes above 20,000 tets)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--train", action="store_true",
                    help="time decoder training steps (lsn_train_step) instead of the solve")
    ap.add_argument("--learned", action="store_true",
                    help="learned-subspace comparison: full-space GPU trajectory of the "
                         "workload as snapshots, decoders trained on the GPU with and "
                         "without the Lipschitz term, reduced solves with each against "
                         "the full-space trajectory (use --steps for the frames)")
    ap.add_argument("--train-steps", type=int, default=3000,
                    help="Adam steps of the first training stage (L_C alone) in --learned")
    ap.add_argument("--finetune-steps", type=int, default=3000,
                    help="Adam steps of the second stage (L_C + lambda L_LS) per weight")
    ap.add_argument("--lambdas", default="0,1e-7,1e-6,1e-5",
                    help="Lipschitz-loss weights of the second stage in --learned "
                         "(0 = vanilla)")
    ap.add_argument("--snapshots", type=int, default=1024,
                    help="quasi-static snapshot loads in --learned (training bar)")
    ap.add_argument("--snapshot-seconds", type=float, default=900.0,
                    help="wall-clock budget of the quasi-static snapshot solves in --learned "
                         "(training continues on the snapshots solved within it)")
    ap.add_argument("--heldout", type=int, default=32,
                    help="held-out loads solved by each decoder in --learned (training bar)")
    ap.add_argument("--train-precision", default="tf32",
                    choices=["fp64", "fp32", "tf32", "bf16"],
                    help="trainer form in --learned")
    ap.add_argument("--train-seed", type=int, default=3,
                    help="seed of the training batches and the evaluation batch in --learned")
    ap.add_argument("--learned-optimizers", default="newton,lbfgs",
                    help="optimisers of the reduced solves in --learned")
    ap.add_argument("--exact-hessian", action="store_true",
                    help="projective Newton with the exact-form reduced Hessian (the decoder's "
                         "curvature added, the r x r sum projected)")
    ap.add_argument("--fullspace", action="store_true",
                    help="time the full-space GPU solve (the comparison) on the workload's "
                         "mesh, constraints and frames, and the reduced solve's error against "
                         "it; use a short run, e.g. --steps 20 --warmup 3")
    ap.add_argument("--fs-precision", default="fp32", choices=["fp64", "fp32"],
                    help="element math of the full-space solve")
    ap.add_argument("--cg-rtol", type=float, default=1e-4,
                    help="relative CG residual of the full-space Newton directions")
    ap.add_argument("--replay", type=int, default=10,
                    help="timed frames replayed with per-kernel CUDA events")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def measured_traffic(cls, workload, precision):
    """DRAM bytes per launch from the ncu capture recorded in
    profiles/traffic.json, or None when there is none or the kernel's source
    has changed since it was taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    ent = json.load(open(path)).get(f"{cls}|{workload}|{precision}")
    if not ent:
        return None
    src = os.path.join(ROOT, ent["source"])
    if not os.path.exists(src):
        return None
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    return ent["bytes"] if sha == ent["sha256_16"] else None


def workload_config(args, p, world):
    """The `config` object of the JSON line (both arms)."""
    c = p.config
    W, K = args.warmup, args.steps
    return {"workload": args.workload,
            "mesh": (f"voxel torus R={c.torus[0]} a={c.torus[1]} h={c.h}, {p.ne} tets, n={p.n}, "
                     f"ground k={c.ground_k:g}" if c.mesh == "torus" else
                     f"{c.dims[0]}x{c.dims[1]}x{c.dims[2]} nodes, {p.ne} tets, n={p.n}"),
            "r": subspace_dim(p), "decoder": "-".join(map(str, p.widths)),
            "affine_modes": 12 if p.affine_center is not None else 0,
            "cubature": len(p.cub_idx), "dt": c.dt, "tol_inf": c.eps,
            "precision": args.precision + " (FP64 Cholesky + line search)",
            "optimizer": (f"L-BFGS (history {args.history})" if args.optimizer == "lbfgs"
                          else "projective Newton" + (
                              ", exact-form reduced Hessian (decoder curvature added, "
                              "r x r projection)" if args.exact_hessian else "")),
            "frames": f"1..{K} (timed from rest, after {W} warm-up steps of frames 1..{W})",
            "l2": "flushed between steps (256 MiB write, outside events)",
            "parallelism": "replicas" if world > 1 else "1 GPU"}


def aggregate_time(total_ms, world, device=None):
    """Timed-region milliseconds of the whole job: the maximum over ranks
    (every rank runs its own replica; the slowest one sets the job time)."""
    if world <= 1:
        return total_ms
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(world, steps, total_ms):
    """Whole-job throughput: the steps of all ranks over the job time."""
    return world * steps / (total_ms / 1000.0)


def oracle_sim(p, args, pool_workers=None):
    """The FP64 CPU oracle's simulator with the optimiser of the run, and the
    oracle's worker pool for the element sums (None on small meshes)."""
    from oracle.reduced import model_from_problem, ReducedSimulator
    c = p.config
    model = model_from_problem(p, chunk=16384)
    pool = None
    workers = pool_workers if pool_workers is not None else (
        (os.cpu_count() or 1) if len(p.cub_idx) > 20000 else 0)
    if workers > 1:
        from oracle.pool import ElementPool
        pool = ElementPool(model, workers)
        model.pool = pool
    sim = ReducedSimulator(model, c.dt, eps=c.eps, max_newton=c.max_newton, max_ls=c.max_ls,
                           c=c.armijo_c, optimizer=args.optimizer, history=args.history,
                           v0=p.v0, exact_hessian=args.exact_hessian)
    return sim, pool, max(workers, 1)


def oracle_run(p, args, frames, budget_s):
    """Run the FP64 CPU oracle over frames 1..`frames` from rest, stopping
    after the first frame that ends past `budget_s` seconds (at least one
    frame).  Returns (frames done, seconds, positions per frame, workers)."""
    c = p.config
    sim, pool, workers = oracle_sim(p, args, args.cpu_workers)
    qs = []
    t0 = time.perf_counter()
    done = 0
    try:
        for k in range(1, frames + 1):
            if not (c.dt > 0):  # quasi-static: every solve from the rest state
                sim.z = np.zeros_like(sim.z)
            sim.step(p.targets(k))
            qs.append(sim.q.copy())
            done = k
            if time.perf_counter() - t0 > budget_s:
                break
        secs = time.perf_counter() - t0
    finally:
        if pool is not None:
            pool.close()
    return done, secs, qs, workers


# --------------------------------------------------------------- reference
def run_reference(args, world, rank):
    """This arm's reference is the FP64 CPU oracle (the paper has no code):
    frames 1..K from rest on the host cores, stopping once 120 s have passed
    (at least one frame); the oracle's set-up (model, worker pool) is not
    timed."""
    if rank != 0:
        return
    p = load_problem(args)
    c = p.config
    budget = 120.0
    sim, pool, workers = oracle_sim(p, args, args.cpu_workers)
    t1 = time.perf_counter()
    steps = 0
    try:
        for k in range(1, args.steps + 1):
            if not (c.dt > 0):  # quasi-static: every solve from the rest state
                sim.z = np.zeros_like(sim.z)
            sim.step(p.targets(k))
            steps += 1
            if time.perf_counter() - t1 > budget:
                break
        el = time.perf_counter() - t1
    finally:
        if pool is not None:
            pool.close()
    value = steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s",
            "n_gpus": world, "steps": steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * el / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, p, world),
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": workers,
                             "kind": "oracle",
                             "sample": f"frames 1..{steps} of {args.workload} from rest (FP64 "
                                       f"NumPy oracle, {workers} worker processes for the "
                                       f"element sums, {el:.1f} s)"},
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------- ours
def load_problem(args):
    """The workload, with the subspace dimension overridden by --r."""
    import dataclasses
    from workloads import build_problem, CONFIGS
    c = CONFIGS[args.workload]
    if args.r is not None:
        c = dataclasses.replace(c, r=args.r)
    return build_problem(c)


def subspace_dim(p):
    """Dimension of z: the network's input width (+ 12 affine modes)."""
    return p.config.r + (12 if p.affine_center is not None else 0)


def algorithmic_bytes(cls, p, precision):
    """Bytes one launch of kernel class `cls` must move at minimum (each datum
    once): weights and inputs read, outputs written."""
    c = p.config
    n, r, H = p.n, subspace_dim(p), p.widths[-2]
    b = 8 if precision == "fp64" else 4
    w = 2 if precision == "bf16" else b          # stored bytes of W_L
    C = r + 4                                    # value, r tangents, 3 trial columns
    cub = p.tets[p.cub_idx] if len(p.cub_idx) else p.tets
    S = cub.shape[0]
    rows = 3 * np.unique(cub).shape[0]           # decoder rows the element kernel reads
    if cls == "decoder_last":
        act = C * H * (4 if precision == "bf16" else b)  # packed columns (BF16 hi + lo)
        per_row = n * (b + 8 + 8) + p.nv * (8 + 4)        # bias, ubar, X0; mass, slot
        out = (n + n * r + 3 * n) * b                      # u, J, trial u
        return n * H * w + act + per_row + out
    if cls == "element":
        return S * (16 + 10 * b) + rows * (r + 4) * b
    if cls == "decoder_hidden":                  # weights once, activations in and out
        widths = p.widths[:-1]
        wb = 8 if precision in ("bf16", "tf32") else b   # tensor-core forms: hi + lo TF32
        return sum(o * i * wb + (i + o) * C * 4 for i, o in zip(widths[:-1], widths[1:]))
    return None


def algorithmic_flops(cls, p):
    """FLOPs of one launch of the compute-bound classes: the per-element
    contraction E (24 r^2 + 288 r) of the reduced Hessian and gradient, and the
    hidden layers' 2 H_out H_in C (C = r + 4 columns) per pass."""
    r = subspace_dim(p)
    S = len(p.cub_idx) if len(p.cub_idx) else p.ne
    if cls == "element":
        return S * (24 * r * r + 288 * r)
    if cls == "decoder_hidden":
        widths = p.widths[:-1]
        return sum(2 * o * i * (r + 4) for i, o in zip(widths[:-1], widths[1:]))
    return None


def peaks_for(precision, sms):
    """Roofline denominators: measured HBM copy bandwidth and BF16 tensor
    throughput (MEASURED_PEAKS.json; the sustained figure, since the kernels
    run inside a long solve), TF32 = BF16 x 1.1 / 2.25 (nominal dense ratio),
    FP32 / FP64 CUDA-core peaks from the unit counts and the maximum SM clock
    (128 FP32 lanes per SM, 2 flops per FMA; FP64: the nominal 1.25 TFLOP/s)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    src = "fallback"
    hbm, bf16, mhz = 6800.0, 1700.0, 2070.0
    if os.path.exists(path):
        m = json.load(open(path))
        hbm, bf16 = m["hbm_gbs"], m.get("bf16_tflops_sustained", m.get("bf16_tflops", bf16))
        mhz = m.get("sm_max_mhz", mhz)
        src = "measured"
    fp32 = sms * 128 * 2 * mhz * 1e6 / 1e12
    return {"hbm": (hbm, "GB/s", src),
            "bf16": (bf16, "TFLOP/s", src + " (bf16_tflops_sustained)"),
            "tf32": (bf16 * 1.1 / 2.25, "TFLOP/s", src + " bf16 sustained x 1.1/2.25 (nominal)"),
            "fp32": (fp32, "TFLOP/s", f"derived: {sms} SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz"),
            "fp64": (1.25, "TFLOP/s", "nominal GB300 FP64 (1.25 TFLOP/s)")}


def run_ours(args, world, rank, local):
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py: no CUDA device (the solver has no CPU path)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2409_03807_gb300.build import build
    if rank == 0:
        build()
    if world > 1:
        torch.distributed.barrier()
    build()
    import paper_2409_03807_gb300 as pkg

    p = load_problem(args)
    c = p.config
    W, K = args.warmup, args.steps
    stream = torch.cuda.Stream(dev)
    ctx = pkg.context_from_problem(p, precision=args.precision, device=local, stream=stream,
                                   optimizer=args.optimizer, history=args.history)
    if args.exact_hessian:
        ctx.set_exact_hessian(True)
    frames = max(W, K)
    targets = torch.tensor(np.stack([p.targets(k) for k in range(1, frames + 1)]),
                           dtype=torch.float64, device=dev)
    z_dev = torch.zeros(subspace_dim(p), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()

    # quasi-static workloads: every step is a solve from the rest state z = 0
    # (the state is restored before the step, outside the timed events)
    quasi_static = not (c.dt > 0)
    rest = ctx.get_state()

    def restart():
        if quasi_static:
            ctx.set_state(*rest)

    def do_step(k, z_out):
        ctx.set_constraints(None, targets[k - 1])
        return ctx.step(dt=c.dt, z_out=z_out)

    # warm-up: frames 1..W from rest (their positions are the error check's)
    warm_q = {}
    for k in range(1, W + 1):
        restart()
        do_step(k, z_dev)
        warm_q[k] = ctx.get_positions()
    # timed: frames 1..K from rest, one CUDA-graph launch per step
    ctx.set_state(*rest)
    ctx.set_profiling([])
    ctx.reset_profile()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    iters = trials = 0
    exits = {}
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for i, k in enumerate(range(1, K + 1)):
        restart()
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
            ev0[i].record(stream)
        rc, st, _ = do_step(k, z_dev)
        with torch.cuda.stream(stream):
            ev1[i].record(stream)
        iters += st["newton_iters"]
        trials += st["ls_trials"]
        exits[rc] = exits.get(rc, 0) + 1
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = sum(a.elapsed_time(b) for a, b in zip(ev0, ev1))
    prof_timed = ctx.get_profile()
    launches = sum(v[0] for v in prof_timed.values())
    q_timed_last = ctx.get_positions()
    total_ms = aggregate_time(total_ms, world, dev)
    ms_per_step = total_ms / K
    value = job_value(world, K, total_ms)

    # kernel durations: frames 1..KR replayed from rest with CUDA events around
    # every kernel class (host-driven loop over the same kernels)
    KR = min(K, args.replay)
    ctx.set_state(*rest)
    ctx.set_profiling(pkg._native.KERNEL_CLASSES)
    ctx.reset_profile()
    torch.cuda.synchronize()
    for i, k in enumerate(range(1, KR + 1)):
        restart()
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
        do_step(k, z_dev)
    torch.cuda.synchronize()
    prof = ctx.get_profile()
    ctx.set_profiling([])
    kernel_profile = {k: {"launches": v[0], "ms": v[2],
                          "avg_us": 1000.0 * v[2] / max(v[1], 1)} for k, v in prof.items()}

    # end to end through the C ABI with host buffers: frames 1..K from rest
    # again, each step timed on the host clock from the host-to-device copy
    # of its constraint targets to the device-to-host copy of z and of the
    # positions (the L2 is flushed before each step, outside the clock)
    ctx.set_state(*rest)
    pin_t = torch.empty((frames, p.cnodes.shape[0], 3), dtype=torch.float64).pin_memory()
    pin_t.copy_(targets.cpu())
    z_host = torch.zeros(subspace_dim(p), dtype=torch.float64).pin_memory()
    q_host = torch.zeros(p.n, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    e2e_s = 0.0
    for i, k in enumerate(range(1, K + 1)):
        restart()
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
        stream.synchronize()
        t0 = time.perf_counter()
        ctx.set_constraints(None, pin_t[k - 1])
        ctx.step(dt=c.dt, z_out=z_host)
        ctx.get_positions(q_host)
        e2e_s += time.perf_counter() - t0
    e2e = {"value": world * K / e2e_s, "unit": "steps/s",
           "h2d_bytes_per_step": int(p.cnodes.shape[0] * 3 * 8),
           "d2h_bytes_per_step": int(subspace_dim(p) * 8 + p.n * 8),
           "timing": "host clock per step, L2 flushed before each step outside the clock"}
    # the solve is deterministic: the third run of frames 1..K ends where the
    # timed run ended, bit for bit
    deterministic = bool(np.array_equal(q_host.numpy(), q_timed_last))

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = peaks_for(args.precision, sms)
    replay_ms = sum(v[2] for v in prof.values())
    tc_form = args.precision in ("bf16", "tf32")

    def roof(cls):
        launches_k, timed_k, ms_k = prof[cls]
        if timed_k == 0 or ms_k <= 0:
            return None
        avg_s = ms_k / timed_k / 1000.0
        ent = {"kernel": cls, "avg_launch_us": avg_s * 1e6, "launches": launches_k,
               "share_of_kernel_time": ms_k / replay_ms if replay_ms > 0 else None,
               "timing": f"CUDA events on the launching stream around each launch, "
                         f"host-driven replay of frames 1..{KR} from rest"}
        if cls == "element" and args.optimizer == "newton":
            fl = algorithmic_flops(cls, p)
            peak, unit, src = peaks[args.precision]
            ach = fl / avg_s / 1e12
            ent.update({"bound": "tensor" if tc_form else "alu", "achieved": ach, "peak": peak,
                        "peak_source": src, "unit": unit, "frac": ach / peak,
                        "algorithmic_flops_per_launch": fl,
                        "flops_rule": "E (24 r^2 + 288 r)",
                        "algorithmic_bytes_per_launch": algorithmic_bytes(cls, p,
                                                                          args.precision)})
        elif cls == "decoder_hidden":
            fl = algorithmic_flops(cls, p)
            # tensor-core forms: tcgen05 TF32 layers (the products as three TF32
            # MMAs; the flops counted are the layer's own); otherwise CUDA cores
            peak, unit, src = peaks["tf32" if tc_form else
                                    ("fp64" if args.precision == "fp64" else "fp32")]
            ach = fl / avg_s / 1e12
            ent.update({"bound": "tensor" if tc_form else "alu", "achieved": ach, "peak": peak,
                        "peak_source": src, "unit": unit, "frac": ach / peak,
                        "algorithmic_flops_per_launch": fl,
                        "algorithmic_bytes_per_launch": algorithmic_bytes(cls, p, args.precision),
                        "note": "all hidden layers of one pass" + (
                            " (tcgen05, two-term TF32 split operands)" if tc_form else
                            " (CUDA-core kernels)")})
        elif cls in ("decoder_last", "element"):
            ab = algorithmic_bytes(cls, p, args.precision)
            peak, unit, src = peaks["hbm"]
            ach = ab / avg_s / 1e9
            ent.update({"bound": "hbm", "achieved": ach, "peak": peak, "peak_source": src,
                        "unit": unit, "frac": ach / peak, "algorithmic_bytes_per_launch": ab})
        else:
            ent.update({"bound": "latency", "achieved": None, "peak": None, "frac": None,
                        "note": "O(r^2) work per launch (partial-row reduction, FP64 "
                                "Cholesky, line-search logic): latency, not a roofline"})
        if ent.get("bound") in ("hbm", "tensor", "alu"):
            ent["traffic"] = measured_traffic(cls, args.workload, args.precision)
        return ent

    roofline_kernels = {cls: roof(cls) for cls in pkg._native.KERNEL_CLASSES}
    roofline_kernels = {k: v for k, v in roofline_kernels.items() if v is not None}
    with_roof = {k: v for k, v in roofline_kernels.items() if v.get("frac") is not None}
    dominant = max(with_roof, key=lambda nm: prof[nm][2])
    roofline = with_roof[dominant]

    cpu = None
    err = None
    if rank == 0 and not args.no_cpu_baseline:
        done, secs, qs, workers = oracle_run(p, args, K, args.cpu_seconds)
        cpu = {"value": done / secs, "unit": "steps/s", "cores": workers, "kind": "oracle",
               "sample": f"frames 1..{done} of {args.workload} from rest, the first of the "
                         f"timed frames (FP64 NumPy oracle, {workers} worker processes for "
                         f"the element sums, {secs:.1f} s)"}
        # GPU positions of every frame the oracle reached: the warm-up run of
        # the same frames from rest (replayed past W when needed, untimed)
        gq = dict(warm_q)
        if done > W:
            ctx.set_state(*rest)
            for k in range(1, done + 1):
                restart()
                do_step(k, z_dev)
                gq[k] = ctx.get_positions()
        errs = {}
        for f in range(1, done + 1):
            uo = qs[f - 1] - p.X0.ravel()
            errs[f] = float(np.linalg.norm(gq[f] - p.X0.ravel() - uo) /
                            max(np.linalg.norm(uo), 1e-300))
        if errs:
            fmax = max(errs, key=errs.get)
            tol = {"fp64": 1e-8, "fp32": 1e-4, "tf32": 1e-3, "bf16": 1e-3}[args.precision]
            err = {"frames": f"1..{done}", "max_rel_displacement_error": errs[fmax],
                   "at_frame": fmax, "per_frame": {str(f): v for f, v in errs.items()},
                   "tolerance": tol, "within_tolerance": errs[fmax] <= tol}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world,
                "steps": K, "warmup": W, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp64": "f64", "fp32": "f32", "tf32": "tf32", "bf16": "bf16"}[args.precision], "data": "synthetic",
                "config": workload_config(args, p, world),
                "newton_iters_per_step": iters / K, "ls_trials_per_step": trials / K,
                "newton_iters_per_s": iters / (total_ms / 1000.0),
                "exits": {str(k): v for k, v in sorted(exits.items())},
                "rel_error_vs_oracle": err,
                "roofline": roofline, "roofline_kernels": roofline_kernels,
                "cpu_baseline": cpu, "e2e": e2e, "deterministic_rerun": deterministic,
                "kernel_profile": kernel_profile,
                "gpu_launches": int(launches), "clocks": clk}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def run_train(args, world, rank, local):
    """Decoder-training throughput: Adam steps of L = L_C + 1e-3 L_LS on a
    batch of 64 seeded smooth displacement fields (twist and bend along the
    bar), 512 cubature tets; the trainer follows --precision (FP64, FP32, or
    FP32 with tensor-core matrix products: TF32 operands in the TF32 form, BF16
    operands with FP32 master weights in the BF16 form)."""
    import torch
    torch.cuda.set_device(local)
    from paper_2409_03807_gb300.build import build
    build()
    import paper_2409_03807_gb300 as pkg
    from workloads import build_problem, draw_cubature
    name = args.workload if args.workload != WORKLOAD else "bar_train_44544"
    p = build_problem(name)
    c = p.config
    rng = np.random.default_rng(2)
    X = p.X0
    L = X[:, 0].max()
    Q = []
    for _ in range(64):
        tw, bd = rng.uniform(0, 0.3), rng.uniform(0, 0.05)
        s = X[:, 0] / L
        d = np.zeros_like(X)
        yc, zc = X[:, 1] - X[:, 1].mean(), X[:, 2] - X[:, 2].mean()
        d[:, 1] = (np.cos(tw * s) - 1) * yc - np.sin(tw * s) * zc
        d[:, 2] = np.sin(tw * s) * yc + (np.cos(tw * s) - 1) * zc - bd * s * s * L
        Q.append((X + d).ravel())
    Q = torch.tensor(np.array(Q), dtype=torch.float64, device="cuda")
    S = c.cubature if c.cubature > 0 else 512
    cub, w = draw_cubature(p.ne, S, c.cubature_seed)
    ctx = pkg.Context()
    ctx.set_mesh(p.X0, p.tets)
    ctx.set_material(c.youngs, c.poisson, c.density, c.gravity)
    ctx.set_decoder(p.Ws, p.bs, c.out_scale, args.precision)
    r, n = c.r, p.n
    ctx.train_init((rng.standard_normal((r, n)) / np.sqrt(n)).astype(np.float32),
                   np.zeros(r, np.float32), cub, w)
    for _ in range(args.warmup):
        ctx.train_step(Q, 1e-3, 1e-4)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        losses = ctx.train_step(Q, 1e-3, 1e-4)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    ctx.close()
    if rank == 0:
        print(json.dumps({"metric": "decoder training steps/s (batch 64, L_C + L_LS, Adam)",
                          "value": args.steps / el, "unit": "steps/s", "n_gpus": 1,
                          "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": 1000.0 * el / args.steps, "higher_is_better": True,
                          "dtype": {"fp64": "f64", "fp32": "f32", "tf32": "tf32",
                                    "bf16": "bf16 (FP32 master)"}[args.precision],
                          "data": "synthetic",
                          "config": {"workload": name, "n": p.n, "decoder": "-".join(
                              map(str, p.widths)), "cubature": S, "batch": 64},
                          "last_losses": list(losses)}), flush=True)


def run_fullspace(args, world, rank, local):
    """The full-space GPU solve (projective Newton, Jacobi-PCG directions,
    every tet) over frames 1..W+K of the workload, timed on frames W+1..W+K
    (host clock around each call; every call ends with a stream
    synchronisation), then the reduced solve (--precision, --optimizer) over
    the same frames: its steps/s and its relative displacement error against
    the full-space positions (the subspace error of the decoder)."""
    import torch
    torch.cuda.set_device(local)
    from paper_2409_03807_gb300.build import build
    build()
    import paper_2409_03807_gb300 as pkg
    p = load_problem(args)
    c = p.config
    if c.ground_k > 0 or not (c.dt > 0):
        raise SystemExit("--fullspace needs a dynamic workload without ground contact")
    W, K = args.warmup, args.steps
    X0 = p.X0.ravel()
    ctx = pkg.Context()
    ctx.set_mesh(p.X0, p.tets)
    ctx.set_material(c.youngs, c.poisson, c.density, c.gravity)
    ctx.set_solver(c.eps, c.max_newton, c.max_ls, c.armijo_c)
    ctx.set_constraints(p.cnodes, p.targets(1))
    ctx.fullspace_setup(args.fs_precision, args.cg_rtol, 4096)
    Qf, t_full, its, cgs, exits = [], 0.0, 0, 0, {}
    for k in range(1, W + K + 1):
        ctx.set_constraints(None, p.targets(k))
        t0 = time.perf_counter()
        rc, st, q = ctx.fullspace_step(c.dt)
        el = time.perf_counter() - t0
        Qf.append(q.copy())
        if k > W:
            t_full += el
            its += st["newton_iters"]
            cgs += st["cg_iters"]
            exits[str(rc)] = exits.get(str(rc), 0) + 1
    ctx.close()
    red = pkg.context_from_problem(p, precision=args.precision, optimizer=args.optimizer,
                                   history=args.history)
    t_red, err = 0.0, 0.0
    for k in range(1, W + K + 1):
        red.set_constraints(None, p.targets(k))
        t0 = time.perf_counter()
        red.step(dt=c.dt)
        el = time.perf_counter() - t0
        if k > W:
            t_red += el
        u, uf = red.get_positions() - X0, Qf[k - 1] - X0
        err = max(err, float(np.linalg.norm(u - uf) / max(np.linalg.norm(uf), 1e-300)))
    red.close()
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        # the FP64 full-space oracle (sparse direct Newton systems) on the host
        # cores, on the same frames from rest within --cpu-seconds, and the
        # GPU full-space positions against it (parity at full size)
        from oracle.fullspace import FullModel, newton_solve
        fm = FullModel(p.X0, p.tets, c.youngs, c.poisson, c.density, c.gravity, p.cnodes)
        q, v = X0.copy(), np.zeros_like(X0)
        gv = np.tile(np.asarray(c.gravity, np.float64), p.nv)
        t0, done, gerr = time.perf_counter(), 0, 0.0
        for k in range(1, W + K + 1):
            fm.set_dynamics(c.dt, q + c.dt * v + c.dt ** 2 * gv)
            q1, _ = newton_solve(fm, q, p.targets(k), c.eps, c.max_newton, c.max_ls, c.armijo_c)
            v, q = (q1 - q) / c.dt, q1
            done = k
            uf, uo = Qf[k - 1] - X0, q - X0
            gerr = max(gerr, float(np.linalg.norm(uf - uo) / max(np.linalg.norm(uo), 1e-300)))
            if time.perf_counter() - t0 > args.cpu_seconds:
                break
        secs = time.perf_counter() - t0
        cpu = {"value": done / secs, "unit": "steps/s", "cores": os.cpu_count(),
               "kind": "oracle (full space, FP64, sparse direct)", "sample": f"frames 1..{done}",
               "max_rel_displacement_error_gpu_vs_oracle": gerr}
    if rank == 0:
        print(json.dumps({
            "metric": "full-space GPU solve steps/s (comparison for the reduced solve)",
            "value": K / t_full, "unit": "steps/s", "n_gpus": 1, "steps": K, "warmup": W,
            "ms_per_step": 1000.0 * t_full / K, "higher_is_better": True,
            "dtype": {"fp64": "f64", "fp32": "f32"}[args.fs_precision], "data": "synthetic",
            "config": {"workload": args.workload, "n": p.n, "tets": p.ne, "dt": c.dt,
                       "tol_inf": c.eps, "cg_rtol": args.cg_rtol,
                       "frames": f"{W + 1}..{W + K}", "timing": "host clock per call"},
            "newton_iters_per_step": its / K, "cg_iters_per_step": cgs / K, "exits": exits,
            "reduced": {"precision": args.precision, "optimizer": args.optimizer,
                        "steps_per_s": K / t_red,
                        "max_rel_displacement_error_vs_fullspace": err,
                        "frames_compared": f"1..{W + K}"},
            "cpu_baseline": cpu}), flush=True)


def unpack_params(th, widths, n):
    """Trainer parameter vector -> (encoder W, encoder b, decoder Ws, decoder bs)."""
    r = widths[0]
    Ew, eb = th[:r * n].reshape(r, n), th[r * n:r * n + r]
    o, Ws, bs = r * n + r, [], []
    for a, b in zip(widths[:-1], widths[1:]):
        Ws.append(th[o:o + a * b].reshape(b, a).astype(np.float32))
        o += a * b
        bs.append(th[o:o + b].astype(np.float32))
        o += b
    return Ew, eb, Ws, bs


def lipschitz_estimate(H, Z):
    """Eq. 7 over the codes Z (B x r) with subspace Hessians H (B x r x r):
    the largest ||H_i - H_j||_F / ||z_i - z_j|| over pairs."""
    B, best = len(Z), 0.0
    for i in range(B):
        dH = np.linalg.norm((H[i] - H).reshape(B, -1), axis=1)
        dz = np.linalg.norm(Z[i] - Z, axis=1)
        m = dz > 0
        if m.any():
            best = max(best, float((dH[m] / dz[m]).max()))
    return best


def run_learned(args, world, rank, local):
    """What the learned subspace gains.  Snapshots come from the full-space
    GPU solve (FP64 element math; it agrees with the FP64 full-space oracle):
    for a dynamic workload its trajectory over frames 1..K; for the quasi-static
    training bar, --snapshots equilibria under seeded random loads (x = 0 face
    fixed, x = L face twisted by U[0, 3] rad about the long axis and bent by
    U[0, 0.5] rad, solved in a serpentine load order, each from the previous
    one) and --heldout further loads (each from the nearest snapshot).
    Decoders of the workload's widths are trained on them on the GPU in the
    two stages of Sec. 4.2: stage 1 minimises the reconstruction loss alone
    (Eq. 3) from the Xavier weights and a PCA encoder; stage 2 continues from
    the stage-1 network once per Lipschitz weight, minimising L_C + lambda
    L_LS (Eq. 9 on the workload's cubature set, codes pulled back through the
    encoder); lambda = 0 is the vanilla decoder, trained for the same number
    of steps.  Each decoder, and the untrained one, then runs the reduced
    solve (--precision) from the code of the rest shape, with each optimiser
    of --learned-optimizers (projective Newton; L-BFGS, the optimiser of the
    paper's main results, Sec. 5): over the same frames (dynamic), or one
    quasi-static solve per held-out load.  Reported per decoder: L_C, L_LS and
    the Eq. 7 estimate on a fixed batch of 64 snapshots, and per optimiser
    steps (or solves) per second, iterations, exits and the relative
    displacement error against the full-space solution."""
    import dataclasses
    import torch
    torch.cuda.set_device(local)
    from paper_2409_03807_gb300.build import build
    build()
    import paper_2409_03807_gb300 as pkg
    from workloads import twist_bend_loads, twist_bend_targets
    p = load_problem(args)
    c = p.config
    if c.ground_k > 0 or p.affine_center is not None:
        raise SystemExit("--learned needs a workload without ground contact or affine modes")
    static = not (c.dt > 0)
    dt = c.dt if not static else 0.0
    X0 = p.X0.ravel()
    if static:
        xs = p.X0[:, 0]
        f0 = np.flatnonzero(xs <= xs.min() + 1e-9).astype(np.int32)
        f1 = np.flatnonzero(xs >= xs.max() - 1e-9).astype(np.int32)
        cn = np.concatenate([f0, f1])

        def targets(ld):
            return twist_bend_targets(p.X0, f0, f1, ld[0], ld[1])
        loads = twist_bend_loads(args.snapshots, 2)
        held = twist_bend_loads(args.heldout, 7)
    else:
        cn = p.cnodes
        targets = p.targets
        loads = list(range(1, args.steps + 1))
        held = loads
    # 1. snapshots from the full-space solve
    fs = pkg.Context()
    fs.set_mesh(p.X0, p.tets)
    fs.set_material(c.youngs, c.poisson, c.density, c.gravity)
    fs.set_solver(c.eps, c.max_newton, c.max_ls, c.armijo_c)
    fs.set_constraints(cn, targets(loads[0]))
    fs.fullspace_setup("fp64", 1e-4 if static else 1e-6, 8192)
    Qf, fex, fits = [], {}, 0
    B0 = 64  # training batch
    t0 = time.perf_counter()
    for i, ld in enumerate(loads):
        if static and i >= 2 * B0 and time.perf_counter() - t0 > args.snapshot_seconds:
            loads = loads[:i]  # the budget ran out: train on the snapshots solved so far
            break
        fs.set_constraints(None, targets(ld))
        rc, st, q = fs.fullspace_step(dt)
        Qf.append(q.copy())
        fex[str(rc)] = fex.get(str(rc), 0) + 1
        fits += st["newton_iters"]
        if static and (i + 1) % 128 == 0:
            print(f"snapshots {i + 1}/{len(loads)}: {time.perf_counter() - t0:.1f} s",
                  file=sys.stderr, flush=True)
    t_fs = time.perf_counter() - t0
    Qf = np.array(Qf)
    if static:
        Qh = []
        for ld in held:
            j = int(np.argmin(np.linalg.norm(loads - ld, axis=1)))
            fs.fullspace_set_state(Qf[j], None)
            fs.set_constraints(None, targets(ld))
            Qh.append(fs.fullspace_step(0.0)[2].copy())
        Qh = np.array(Qh)
    else:
        Qh = Qf
    fs.close()
    # 2. decoders
    K = len(Qf)
    r, n = c.r, p.n
    D = Qf - X0
    _, sv, Vt = np.linalg.svd(D, full_matrices=False)
    Ew0 = (Vt[:r] / np.maximum(sv[:r, None], 1e-12) * np.sqrt(K)).astype(np.float32)
    eb0 = np.zeros(r, np.float32)
    cub, cw = p.cub_idx, p.cub_w
    tprec = args.train_precision
    Qd = torch.tensor(Qf, dtype=torch.float64, device="cuda")
    rs = np.random.default_rng(args.train_seed)
    B = min(64, K)
    evi = np.sort(rs.choice(K, B, replace=False))
    ev = torch.tensor(evi, device="cuda")

    def trainer(theta=None):
        tc = pkg.Context()
        tc.set_mesh(p.X0, p.tets)
        tc.set_material(c.youngs, c.poisson, c.density, c.gravity)
        tc.set_decoder(p.Ws, p.bs, c.out_scale, tprec)
        tc.train_init(Ew0, eb0, cub, cw)
        if theta is not None:
            tc.train_set_params(theta)
        return tc

    def train(tc, lam, steps):
        t1 = time.perf_counter()
        for _ in range(steps):
            idx = torch.tensor(rs.choice(K, B, replace=False), device="cuda")
            tc.train_step(Qd[idx], lam, 1e-3)
        torch.cuda.synchronize()
        return time.perf_counter() - t1

    def measured(tc, t_tr, lam):
        # L_LS is reported unweighted; any positive weight evaluates it
        (lc, lls, _), _ = tc.train_eval(Qd[ev], 1e-30, want_grad=False)
        Ew, eb, Ws, bs = unpack_params(tc.train_get_params(), p.widths, n)
        Z = (Qf[evi] - X0) @ Ew.T + eb
        lip = lipschitz_estimate(tc.train_hessians(Z), Z)
        return Ws, bs, eb, {"lambda": lam, "L_C": lc, "L_LS": lls, "lipschitz_eq7": lip,
                            "train_s": t_tr}

    decoders = {}
    tc = trainer()
    decoders["untrained"] = measured(tc, 0.0, None)
    t_s1 = train(tc, 0.0, args.train_steps)
    theta1 = tc.train_get_params()
    decoders["stage 1"] = measured(tc, t_s1, 0.0)
    tc.close()
    for lam in [float(x) for x in args.lambdas.split(",")]:
        tc = trainer(theta1)
        t_tr = train(tc, lam, args.finetune_steps)
        decoders[f"lambda={lam:g}"] = measured(tc, t_s1 + t_tr, lam)
        tc.close()
    # 3. reduced solves from the rest code, with each optimiser
    out = {}
    for name, (Ws, bs, eb, info) in decoders.items():
        pd = dataclasses.replace(p, Ws=Ws, bs=bs)
        out[name] = {"training": info}
        for opt in args.learned_optimizers.split(","):
            ctx = pkg.context_from_problem(pd, precision=args.precision, optimizer=opt,
                                           history=args.history)
            ctx.set_constraints(cn, targets(held[0]))
            its, ex, errs, t_red = 0, {}, [], 0.0
            if not static:
                ctx.set_state(np.asarray(eb, np.float64), X0, None)
            for k, ld in enumerate(held):
                if static:  # every held-out load from the rest code
                    ctx.set_state(np.asarray(eb, np.float64), X0, None)
                ctx.set_constraints(None, targets(ld))
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rc, st, _ = ctx.step(dt=dt)
                t_red += time.perf_counter() - t0
                its += st["newton_iters"]
                ex[str(rc)] = ex.get(str(rc), 0) + 1
                u, uf = ctx.get_positions() - X0, Qh[k] - X0
                errs.append(float(np.linalg.norm(u - uf) / max(np.linalg.norm(uf), 1e-300)))
            ctx.close()
            out[name][opt] = {"solves_per_s": len(held) / t_red,
                              "iters_per_solve": its / len(held), "exits": ex,
                              "max_rel_error_vs_fullspace": max(errs),
                              "mean_rel_error_vs_fullspace": float(np.mean(errs))}
    if rank == 0:
        snap = (f"{K} quasi-static full-space GPU solves (FP64 element math) under seeded "
                f"twist U[0, 3] rad and bend U[0, 0.5] rad of the x = L face; {len(held)} "
                "held-out loads" if static else
                f"full-space GPU solve, FP64 element math, frames 1..{K}")
        print(json.dumps({
            "metric": "learned subspace vs untrained and vs the full-space GPU solve",
            "config": {"workload": args.workload, "n": n, "tets": p.ne, "r": r,
                       "decoder": "-".join(map(str, p.widths)), "precision": args.precision,
                       "optimizers": args.learned_optimizers, "stage1_steps": args.train_steps,
                       "stage2_steps": args.finetune_steps, "batch": B, "lr": 1e-3,
                       "trainer": tprec, "train_seed": args.train_seed, "snapshots": snap,
                       "cubature": len(cub),
                       "solves": "quasi-static, one per held-out load" if static
                       else f"implicit Euler, frames 1..{K}",
                       "start": "code of the rest shape (the trained encoder's bias)"},
            "fullspace": {"solves_per_s": K / t_fs, "newton_iters_per_solve": fits / K,
                          "exits": fex},
            "decoders": out}), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.train:
        run_train(args, world, rank, local)
        return
    if args.learned:
        run_learned(args, world, rank, local)
        return
    if args.fullspace:
        run_fullspace(args, world, rank, local)
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
