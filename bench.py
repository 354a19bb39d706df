#!/usr/bin/env python
"""Benchmark: reduced-solve implicit-Euler steps per second on one GB300.

Workload (default): bar_twist_dyn_14976 - bar of 40x9x9 nodes (14,976 tets,
n = 9,720), x = 0 face rotated 2 rad about the long axis over 60 frames,
implicit Euler dt = 1/60, r = 16, decoder 16-256-256-256-9720 (seeded Xavier
weights, output scale 1e-2), 256 cubature tets drawn uniformly by seed with
weights 14976/256, Stable Neo-Hookean E = 1e5 Pa, nu = 0.45, rho = 1000.

A step is one implicit-Euler time step solved by projective Newton (default;
--optimizer lbfgs: L-BFGS with gradient-only passes) to
||g||_inf < 1e-5 (or its precision-floor / iteration-cap exit): decoder +
Jacobian, element kernel + contraction, Cholesky, line search, until exit.
Inputs (constraint targets of every frame, decoder weights, mesh) are
resident in HBM before the timed region; the L2 is flushed (256 MiB write)
between timed steps, outside the per-step CUDA events.

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
WORKLOAD = "bar_twist_dyn_14976"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
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
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="time budget of the CPU-oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--train", action="store_true",
                    help="time decoder training steps (lsn_train_step) instead of the solve")
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
                          else "projective Newton"),
            "frames": f"{W + 1}..{W + K}",
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


def oracle_sim(p, args):
    """The FP64 CPU oracle's simulator with the optimiser of the run."""
    from oracle.reduced import model_from_problem, ReducedSimulator
    c = p.config
    return ReducedSimulator(model_from_problem(p), c.dt, eps=c.eps, max_newton=c.max_newton,
                            max_ls=c.max_ls, c=c.armijo_c, optimizer=args.optimizer,
                            history=args.history, v0=p.v0)


def oracle_run(p, args, frames, budget_s):
    """Run the FP64 CPU oracle for up to `frames` frames or `budget_s` seconds.
    Returns (frames done, seconds, positions per frame)."""
    c = p.config
    sim = oracle_sim(p, args)
    qs = []
    t0 = time.perf_counter()
    done = 0
    for k in range(1, frames + 1):
        if not (c.dt > 0):  # quasi-static: every solve from the rest state
            sim = oracle_sim(p, args)
        sim.step(p.targets(k))
        qs.append(sim.q.copy())
        done = k
        if time.perf_counter() - t0 > budget_s:
            break
    return done, time.perf_counter() - t0, qs


# --------------------------------------------------------------- reference
def run_reference(args, world, rank):
    if rank != 0:
        return
    from workloads import build_problem
    p = load_problem(args)
    c = p.config
    budget = 150.0
    # timed: frames after the warm-up, continuing the same trajectory
    sim = oracle_sim(p, args)
    for k in range(1, args.warmup + 1):
        sim.step(p.targets(k))
    t1 = time.perf_counter()
    steps = 0
    for k in range(args.warmup + 1, args.warmup + args.steps + 1):
        if not (c.dt > 0):  # quasi-static: every solve from the rest state
            sim = oracle_sim(p, args)
        sim.step(p.targets(k))
        steps += 1
        if time.perf_counter() - t1 > budget:
            break
    el = time.perf_counter() - t1
    value = steps / el
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s",
            "n_gpus": world, "steps": steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * el / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, p, world),
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"frames {args.warmup + 1}..{args.warmup + steps} of "
                                       f"{args.workload} (FP64 NumPy oracle, implicit Euler)"},
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
    return None


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
    from workloads import build_problem

    p = load_problem(args)
    c = p.config
    W, K = args.warmup, args.steps
    stream = torch.cuda.Stream(dev)
    ctx = pkg.context_from_problem(p, precision=args.precision, device=local, stream=stream,
                                   optimizer=args.optimizer, history=args.history)
    frames = W + K
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

    # warm-up frames 1..W
    warm_q = {}
    for k in range(1, W + 1):
        restart()
        do_step(k, z_dev)
        warm_q[k] = ctx.get_positions()
    snap = ctx.get_state()
    # timed frames W+1..W+K: one CUDA-graph launch per step
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
    for i, k in enumerate(range(W + 1, W + K + 1)):
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
    total_ms = aggregate_time(total_ms, world, dev)
    ms_per_step = total_ms / K
    value = job_value(world, K, total_ms)

    # kernel durations: the first frames of the timed region replayed from the
    # same state with CUDA events around every kernel class (host-driven loop)
    KR = min(K, args.replay)
    ctx.set_state(*snap)
    ctx.set_profiling(pkg._native.KERNEL_CLASSES)
    ctx.reset_profile()
    torch.cuda.synchronize()
    for i, k in enumerate(range(W + 1, W + KR + 1)):
        restart()
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
        do_step(k, z_dev)
    torch.cuda.synchronize()
    prof = ctx.get_profile()
    ctx.set_profiling([])
    kernel_profile = {k: {"launches": v[0], "ms": v[2],
                          "avg_us": 1000.0 * v[2] / max(v[1], 1)} for k, v in prof.items()}
    dominant = max(("decoder_last", "element"), key=lambda nm: prof[nm][2])

    # end to end through the C ABI with host buffers: the same frames again
    ctx.set_state(*snap)
    pin_t = torch.empty((frames, p.cnodes.shape[0], 3), dtype=torch.float64).pin_memory()
    pin_t.copy_(targets.cpu())
    z_host = torch.zeros(subspace_dim(p), dtype=torch.float64).pin_memory()
    q_host = torch.zeros(p.n, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(W + 1, W + K + 1):
        restart()
        ctx.set_constraints(None, pin_t[k - 1])
        ctx.step(dt=c.dt, z_out=z_host)
        ctx.get_positions(q_host)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": world * K / e2e_s, "unit": "steps/s",
           "h2d_bytes_per_step": int(p.cnodes.shape[0] * 3 * 8),
           "d2h_bytes_per_step": int(subspace_dim(p) * 8 + p.n * 8)}

    replay_ms = sum(v[2] for v in prof.values())
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak, peak_src = 6800.0, "fallback"
    if os.path.exists(peaks_path):
        peak = json.load(open(peaks_path))["hbm_gbs"]
        peak_src = "measured"

    def roof(cls):
        launches_k, timed_k, ms_k = prof[cls]
        avg_ms = ms_k / max(timed_k, 1)
        ab = algorithmic_bytes(cls, p, args.precision)
        achieved = ab / (avg_ms / 1000.0) / 1e9 if ab and avg_ms > 0 else None
        return {"kernel": cls, "bound": "hbm", "achieved": achieved, "peak": peak,
                "peak_source": peak_src, "unit": "GB/s",
                "frac": achieved / peak if achieved else None,
                "traffic": measured_traffic(cls, args.workload, args.precision),
                "avg_launch_us": avg_ms * 1000.0, "launches": launches_k,
                "algorithmic_bytes_per_launch": ab,
                "share_of_kernel_time": ms_k / replay_ms if replay_ms > 0 else None,
                "timing": f"CUDA events around each launch, host-driven replay of frames "
                          f"{W + 1}..{W + KR} from the same state"}

    roofline = roof(dominant)
    roofline_kernels = {cls: roof(cls) for cls in ("decoder_last", "element")}

    cpu = None
    err = None
    if rank == 0 and not args.no_cpu_baseline:
        done, secs, qs = oracle_run(p, args, max(W, 200), args.cpu_seconds)
        cpu = {"value": done / secs, "unit": "steps/s", "cores": os.cpu_count(),
               "kind": "oracle",
               "sample": f"frames 1..{done} of {args.workload} from rest "
                         f"(FP64 NumPy oracle, {secs:.1f} s)"}
        # GPU positions of every frame the oracle reached: the warm-up frames,
        # then a replay of the timed frames from the snapshot (untimed)
        gq = dict(warm_q)
        last = min(done, W + K)
        if last > W:
            ctx.set_state(*snap)
            for k in range(W + 1, last + 1):
                restart()
                do_step(k, z_dev)
                gq[k] = ctx.get_positions()
        errs = {}
        for f in range(1, last + 1):
            uo = qs[f - 1] - p.X0.ravel()
            errs[f] = float(np.linalg.norm(gq[f] - p.X0.ravel() - uo) /
                            max(np.linalg.norm(uo), 1e-300))
        if errs:
            fmax = max(errs, key=errs.get)
            err = {"frames": f"1..{last}", "max_rel_displacement_error": errs[fmax],
                   "at_frame": fmax, "last_frame_error": errs[last]}

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
                "cpu_baseline": cpu, "e2e": e2e,
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
    FP32 with TF32 tensor-core matrix products for the tensor-core forms)."""
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
    # tensor-core forms train with TF32 tensor-core matrix products
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
                          "dtype": {"fp64": "f64", "fp32": "f32"}.get(args.precision,
                                                                      "tf32"),
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


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.train:
        run_train(args, world, rank, local)
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
