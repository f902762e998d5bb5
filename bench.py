#!/usr/bin/env python
"""Benchmark of the domain decomposition primal-dual TV solver on one GB300.

Workload: ROF denoising of a 4096 x 4096 float32 image (seeded piecewise-constant
scene of 400 rectangles/disks + Gaussian noise sigma = 0.1), alpha = 8, 32 x 32
subdomains of 128 x 128, 10 inner iterations per outer iteration, the paper's
steps (tau = 50, sigma tau = 1/2, tau0 = 10, sigma0 tau0 = 1/8, gamma = 1/(8 tau)).

One step = one outer iteration of Algorithm 1 (interface multiplier update, proximal
centre, all local solves, assembly), plus every 5th step the energy reduction of the
outer stopping rule.  Metric: Mpixel-iter/s = H * W * inner iterations / s / 1e6.
The state (u, torn p, f: ~470 MB) is larger than L2, so no flush is needed.

Also reported: time to relative energy error 1e-4 against a certified J* (fused vs
plain vs full-dimension GPU paths), the end-to-end number through dd_tv_solve with
host buffers, the fused kernel's roofline, and the FP64 oracle on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H = W = 4096
NR = NC = 32
INNER = 10
ALPHA = 8.0
N_SHAPES = 400
NOISE = 0.1
SEED = 0
ENERGY_EVERY = 5
METRIC = "Mpixel*iter/s at 4096^2 ROF"
UNIT = "Mpixel*iter/s"
ADAPT_CAP = 20  # inner iterations allowed per local solve under the adaptive stop
ADAPT_TOL_F32 = 1e-4  # inner tolerance standing in for the paper's 1e-6 in float32
WORKLOAD = "rof4096: ROF L2 denoising 4096x4096 fp32, alpha=8, 32x32 subdomains of 128x128, 10 inner/outer"
SMEM_BYTES_PER_PX_ITER = 28  # minimum neighbour exchange per pixel per inner iteration
JSTAR_FILE = os.path.join(ROOT, "tests", "golden", "jstar_rof4096_seed0.json")
JSTAR_BATCH_FILE = os.path.join(ROOT, "tests", "golden", "jstar_batch64_seed0.json")
PROFILE_FILE = os.path.join(ROOT, "profiles", "fused_local_rof4096.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-tta", action="store_true", help="skip the time-to-accuracy runs")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched multi-image measurement")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuned time-to-accuracy")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the unrolled-adjoint measurement")
    ap.add_argument("--no-tvl1", action="store_true", help="skip the TV-L1 inpainting measurement")
    ap.add_argument("--replicas", action="store_true",
                    help="with --gpus N > 1: N independent replicas instead of one sharded image")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, pg=None, device=None) -> float:
    """The maximum of x over all ranks of the process group (x itself without one)."""
    if pg is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(work_per_rank: float, world: int, seconds: float) -> float:
    """Units of all ranks per second, in millions (every rank does the same work; the
    job takes as long as its slowest rank)."""
    return world * work_per_rank / seconds / 1e6


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.rows = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        self.t0 = time.time()

    def stop(self):
        if not self.proc:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k].lower() == "active"})
        loaded = [s for s in sm if s >= 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(self.rows)}


def make_input():
    import synth
    f, clean = synth.rof_image(H, W, N_SHAPES, NOISE, SEED)
    return f, clean


def load_jstar(f):
    import synth
    if not os.path.exists(JSTAR_FILE):
        return None, "no certified J* file"
    rec = json.load(open(JSTAR_FILE))
    if rec.get("f_sha256") != synth.array_digest(f):
        return None, "generated image differs from the one J* was certified on"
    return rec, None


def load_batch_jstar(ims):
    """Certified per-image J* of the 64-image batch (FP64 oracle, duality gap), or
    (None, why) when the file is missing or the images differ."""
    import synth
    if not os.path.exists(JSTAR_BATCH_FILE):
        return None, "no certified batch J* file"
    recs = json.load(open(JSTAR_BATCH_FILE))["images"]
    if len(recs) != len(ims) or any(r["f_sha256"] != synth.array_digest(m["f"]) for r, m in zip(recs, ims)):
        return None, "generated batch differs from the one J* was certified on"
    return recs, None


def kernel_source_sha():
    """First 16 hex digits of the SHA-256 of the fused kernel's sources (the kernel file
    and the device headers it includes), to tell whether a capture is still current."""
    h = hashlib.sha256()
    for name in ("kernels_fused_mt4.cu", "fused_common.cuh", "pointwise.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1901_00682_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def profile_data():
    """The committed ncu figures of the fused kernel (profiles/fused_local_rof4096.json),
    or None when the kernel source changed since the capture."""
    if not os.path.exists(PROFILE_FILE):
        return None
    try:
        rec = json.load(open(PROFILE_FILE))
    except ValueError:
        return None
    return rec if rec.get("kernel_source_sha256") == kernel_source_sha() else None


def cpu_baseline(f, outer=2):
    """The FP64 oracle (as it stands) on a bounded sample: `outer` outer iterations of
    the same 4096^2 workload on the host cores."""
    import numpy as np

    import oracle
    pr = oracle.Problem(H, W, NR, NC, fidelity="l2", alpha=ALPHA, inner=INNER)
    f64 = f.astype(np.float64)
    st = oracle.dd_init(pr, f64)
    oracle.dd_run(pr, f64, 0, state=st)  # builds/loads the oracle library
    t = time.perf_counter()
    oracle.dd_run(pr, f64, outer, state=st)
    dt = time.perf_counter() - t
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": H * W * INNER * outer / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{outer} outer iterations (x{INNER} inner) of the 4096^2 32x32-subdomain workload, "
                      f"FP64, OpenMP over subdomains, {dt:.1f} s"}


def cpu_baseline_one_core(outer=1):
    """The same oracle sample on one host core (OpenMP pinned to one thread in a child
    process, so the parent's thread pool is untouched)."""
    code = ("import sys, time, json, numpy as np; sys.path.insert(0, %r); import oracle, synth; "
            "f, _ = synth.rof_image(%d, %d, %d, %r, %d); f = f.astype(np.float64); "
            "pr = oracle.Problem(%d, %d, %d, %d, fidelity='l2', alpha=%r, inner=%d); "
            "st = oracle.dd_init(pr, f); oracle.dd_run(pr, f, 0, state=st); t = time.perf_counter(); "
            "oracle.dd_run(pr, f, %d, state=st); print(json.dumps(time.perf_counter() - t))"
            % (ROOT, H, W, N_SHAPES, NOISE, SEED, H, W, NR, NC, ALPHA, INNER, outer))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        return {"error": r.stderr[-300:]}
    dt = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": H * W * INNER * outer / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{outer} outer iteration (x{INNER} inner) of the 4096^2 workload on one core, {dt:.1f} s"}


def measure_tvl1(dev, stream):
    """TV-L1 inpainting + impulse denoising (2048^2, 10 % salt and pepper, Bernoulli(0.2)
    mask, alpha 1.5, 16 x 16 subdomains of 128^2, K = 10), 500 outer iterations: device
    throughput, the fused kernel's roofline, and the energy against the FP64 oracle at
    equal iteration counts (20 outer iterations of both, from the same start)."""
    import numpy as np
    import torch

    import oracle
    import synth
    from paper_1901_00682_gb300 import _lib as L
    S, NT, OUT = 2048, 16, 500
    f, mask, _ = synth.tvl1_inpaint_image(S, S, 100, 0.1, 0.2, 0)
    fd = torch.from_numpy(f).to(dev)
    md = torch.from_numpy(mask).to(dev)
    p = L.make_params(S, S, NT, NT, fidelity="l1", alpha=1.5, inner_iters=INNER)
    s = L.Solver(p, stream)
    s.load(fd, md)
    s.iterate(20)
    J20 = s.current_energy()
    s.load(fd, md)
    s.iterate(OUT)                      # warm-up (graph capture)
    s.load(fd, md)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.iterate(OUT)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    J500 = s.current_energy()
    s.load(fd, md)
    s.profile_read()
    s.set_profiling(True)
    s.iterate(40)
    prof_ms, prof_n = s.profile_read()
    s.set_profiling(False)
    s.close()
    local_ms = prof_ms["local"] / max(prof_n["local"], 1)
    peak = L.measure_smem_bandwidth()
    ach = SMEM_BYTES_PER_PX_ITER * S * S * INNER / (local_ms * 1e-3) / 1e9
    pr = oracle.Problem(S, S, NT, NT, fidelity="l1", alpha=1.5, inner=INNER)
    st = oracle.dd_run(pr, f.astype(np.float64), 20, mask=mask)
    Jo = oracle.energy(pr, st.u, f.astype(np.float64), mask)
    return {"workload": "tvl1_2048: TV-L1 inpainting + impulse denoising 2048x2048 fp32, 10% salt and pepper, "
                        "Bernoulli(0.2) mask, alpha=1.5, 16x16 subdomains of 128x128, 10 inner/outer, 500 outer",
            "ms_500_outer": ms, "value": S * S * INNER * OUT / (ms * 1e-3) / 1e6, "unit": UNIT,
            "energy_500": J500,
            "roofline": {"bound": "smem", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                         "avg_launch_ms": local_ms, "kernel": "k_fused_mt4t<L1, mask>"},
            "energy_vs_oracle_20_outer": {"gpu": J20, "oracle": Jo, "rel_diff": abs(J20 - Jo) / abs(Jo)}}


def measure_adjoint(dev):
    """Forward and backward time of the unrolled solver on the differentiation workload:
    8 ROF images 1024 x 1024 (sigma 0.08, alpha 10), 8 x 8 subdomains, 100 outer x 10
    inner iterations, checkpoints every 10, loss 1/2 ||u - g||^2."""
    import numpy as np
    import torch

    import synth
    from paper_1901_00682_gb300.autograd import UnrolledDDTV
    B, S, N, M = 8, 1024, 100, 10
    pairs = [synth.rof_image(S, S, 400 // 16, 0.08, 500 + b) for b in range(B)]
    f = torch.from_numpy(np.stack([p[0] for p in pairs])).to(dev).requires_grad_(True)
    g = torch.from_numpy(np.stack([p[1] for p in pairs])).to(dev)
    alpha = torch.tensor(10.0, dtype=torch.float64, device=dev, requires_grad=True)
    mod = UnrolledDDTV(S, S, 8, 8, N, checkpoint_every=M, inner_iters=INNER)
    fw, bw = [], []
    for rep in range(3):
        f.grad = None
        alpha.grad = None
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        u = mod(f, alpha)
        loss = 0.5 * ((u - g) ** 2).sum()
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        loss.backward()
        torch.cuda.synchronize(dev)
        t2 = time.perf_counter()
        if rep:  # the first repetition allocates the workspaces and captures graphs
            fw.append((t1 - t0) * 1e3)
            bw.append((t2 - t1) * 1e3)
    mod.close()
    ms_f, ms_b = min(fw), min(bw)
    px_it = B * S * S * INNER * N
    return {"workload": "8 ROF images 1024x1024 (sigma .08, alpha 10), 8x8 subdomains, 100 outer x 10 inner, "
                        "checkpoint every 10, loss 1/2||u_K - g||^2, dL/df and dL/dalpha",
            "ms_forward": ms_f, "ms_backward": ms_b, "backward_over_forward": ms_b / ms_f,
            "backward_Mpixel_iter_per_s": px_it / (ms_b * 1e-3) / 1e6,
            "backward_work": "per outer iteration: the segment's forward recomputation (fused path) and one "
                             "tile-fused kernel that recomputes the K inner iterations with the tape in L2 and "
                             "runs their K reverse iterations",
            "timing": "host wall clock with device synchronisation, best of 2 after one warm-up"}


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, each step one outer iteration
    on a bounded sample (the top-left S x S block, subdomains of 128 x 128, 10 inner
    iterations; S shrinks with the step count)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np

    import oracle
    f, _ = make_input()
    # sample size per step keeps the whole run within about a minute of host time
    S = 512 if args.steps <= 200 else (256 if args.steps <= 2000 else 128)
    sub = np.ascontiguousarray(f[:S, :S]).astype(np.float64)
    pr = oracle.Problem(S, S, S // 128, S // 128, fidelity="l2", alpha=ALPHA, inner=INNER)
    st = oracle.dd_init(pr, sub)
    oracle.dd_run(pr, sub, args.warmup, state=st)
    t = time.perf_counter()
    oracle.dd_run(pr, sub, args.steps, state=st)
    dt = time.perf_counter() - t
    val = S * S * INNER * args.steps / dt / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"each step: 1 outer iteration (x{INNER} inner) on the top-left {S}x{S} block of the workload, "
              f"{S // 128}x{S // 128} subdomains of 128x128, FP64 oracle")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_sharded(args, rank, world, local, dev, stream, pg):
    """Weak scaling of one image over `world` GPUs: 4096 * world rows x 4096 columns
    (the ranks' 4096^2 blocks are independent synthetic scenes, seeds 0..world-1),
    32 * world x 32 subdomains of 128^2, rank r owning tile rows [32 r, 32 r + 32).  One
    step = one outer iteration on every rank, including the exchange of the cut strips
    (NCCL point-to-point); the energy of the stopping rule every 5 steps adds the ranks'
    parts (float64 all-reduce).  Returns the bench JSON fields (rank 0)."""
    import numpy as np
    import torch

    import synth
    from paper_1901_00682_gb300 import _lib as L
    from paper_1901_00682_gb300.shard import ShardedSolver, TorchDistComm
    p = L.make_params(H * world, W, NR * world, NC, fidelity="l2", alpha=ALPHA, inner_iters=INNER, path="fused")
    comm = TorchDistComm(pg)
    ss = ShardedSolver(p, rank, world, comm, stream=stream)
    r0, nrows = ss.rows()
    assert nrows == H
    f, _ = synth.rof_image(H, W, N_SHAPES, NOISE, SEED + rank)
    fd = torch.from_numpy(f).to(dev)
    ss.load(fd)
    pg.barrier()
    for q in range(args.warmup):
        ss.step(1)
        if (q + 1) % ENERGY_EVERY == 0:
            ss.energy()
    torch.cuda.synchronize(dev)
    ss.solver.profile_read()
    ss.solver.set_profiling(True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    pg.barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for q in range(args.steps):
        ss.solver.set_profiling(q % ENERGY_EVERY != 0)   # as in the single-GPU loop
        ss.step(1)
        if (q + 1) % ENERGY_EVERY == 0:
            ss.solver.set_profiling(True)
            ss.energy()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    pg.barrier()
    clocks.stop()
    prof_ms, prof_n = ss.solver.profile_read()
    ss.solver.set_profiling(False)
    t_max = max_over_ranks(e0.elapsed_time(e1), pg, dev)
    work = H * W * INNER * args.steps
    value = whole_job_rate(work, world, t_max * 1e-3)
    local_avg_ms = prof_ms["local"] / max(prof_n["local"], 1)
    smem_peak = L.measure_smem_bandwidth()
    bytes_per_launch = SMEM_BYTES_PER_PX_ITER * H * W * INNER
    achieved = bytes_per_launch / (local_avg_ms * 1e-3) / 1e9
    roofline = {"bound": "smem", "achieved": achieved, "peak": smem_peak, "unit": "GB/s",
                "frac": achieved / smem_peak, "traffic": None,
                "kernel": "fused local solver of the rank's 4096x4096 block (k_fused_mt4t)",
                "peak_source": "measured live: ld.shared probe kernel (dd_tv_measure_smem_bandwidth)",
                "algorithmic_bytes_per_launch": bytes_per_launch, "avg_launch_ms": local_avg_ms}
    row_tv = args.steps // ENERGY_EVERY if rank < world - 1 else 0   # the cut's TV kernel of each energy
    # end to end: the rank's f block from pinned host memory, the steps, u back to the host
    f_pin = torch.from_numpy(f).pin_memory()
    u_pin = torch.empty_like(f_pin).pin_memory()
    ud = torch.empty_like(fd)
    pg.barrier()
    torch.cuda.synchronize(dev)
    t = time.perf_counter()
    fd.copy_(f_pin, non_blocking=True)
    ss.load(fd)
    for q in range(args.steps):
        ss.step(1)
        if (q + 1) % ENERGY_EVERY == 0:
            ss.energy()
    ss.solver.get_u(ud)
    u_pin.copy_(ud, non_blocking=True)
    torch.cuda.synchronize(dev)
    dt_e2e = max_over_ranks(time.perf_counter() - t, pg, dev)
    ss.solver.close()
    e2e = {"value": whole_job_rate(work, world, dt_e2e), "unit": UNIT,
           "h2d_bytes_per_step": 4 * H * W / args.steps, "d2h_bytes_per_step": 4 * H * W / args.steps,
           "call": "per rank: H2D of its f block, dd_tv_load, the sharded outer iterations with the cut exchange, "
                   "D2H of its u block"}
    return {"value": value, "t_max": t_max, "e2e": e2e, "clocks": clocks.summary(), "roofline": roofline,
            "phase_ms": prof_ms, "launches_by_phase": prof_n,
            "config": {"workload": f"rof{H * world}x{W}: ROF L2 denoising {H * world}x{W} fp32 ({world} stacked "
                                   f"4096^2 scenes), alpha=8, {NR * world}x{NC} subdomains of 128x128, 10 inner/outer",
                       "l2": "state larger than L2; no flush",
                       "parallelism": f"row-block shards x{world} (tile rows per rank: {NR}), cut strips exchanged "
                                      "by NCCL point-to-point every outer iteration, energy by float64 all-reduce",
                       "step": "1 outer iteration on every rank incl. the cut exchange, energy every 5 steps"},
            "gpu_launches": 2 * args.steps + args.steps // ENERGY_EVERY + row_tv}


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    if world > 1 and not args.replicas:
        from paper_1901_00682_gb300 import _lib as L
        L.load()
        stream = torch.cuda.Stream(dev)
        torch.cuda.set_stream(stream)
        r = run_sharded(args, rank, world, local, dev, stream, pg)
        if rank == 0:
            print(json.dumps({
                "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": r["t_max"] / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": r["config"],
                "roofline": r["roofline"], "cpu_baseline": None, "e2e": r["e2e"], "clocks": r["clocks"],
                "gpu_launches": r["gpu_launches"], "launches_by_phase": r["launches_by_phase"],
                "phase_ms": r["phase_ms"]}), flush=True)
        pg.destroy_process_group()
        return
    from paper_1901_00682_gb300 import _lib as L

    L.load()
    f, _ = make_input()
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    fd = torch.from_numpy(f).to(dev)

    # ---- throughput: resident inputs, K steps
    p = L.make_params(H, W, NR, NC, fidelity="l2", alpha=ALPHA, inner_iters=INNER, path="fused")
    s = L.Solver(p, stream)
    s.load(fd)
    for q in range(args.warmup):
        s.iterate(1)
        if (q + 1) % ENERGY_EVERY == 0:
            s.current_energy()
    torch.cuda.synchronize(dev)
    s.profile_read()
    s.set_profiling(True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for q in range(args.steps):
        # per-phase CUDA events on every step except the first after a host read-back of
        # the energy (there the stream runs dry and the bracket would include the host's
        # submission of the next launches)
        s.set_profiling(q % ENERGY_EVERY != 0)
        s.iterate(1)
        if (q + 1) % ENERGY_EVERY == 0:
            s.set_profiling(True)
            s.current_energy()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    clocks.stop()
    ms_total = e0.elapsed_time(e1)
    prof_ms, prof_n = s.profile_read()
    s.set_profiling(False)
    t_max = max_over_ranks(ms_total, pg, dev)
    work = H * W * INNER * args.steps
    value = whole_job_rate(work, world, t_max * 1e-3)

    # ---- roofline of the fused local solver (dominant kernel)
    local_avg_ms = prof_ms["local"] / max(prof_n["local"], 1)
    smem_peak = L.measure_smem_bandwidth()
    bytes_per_launch = SMEM_BYTES_PER_PX_ITER * H * W * INNER
    achieved = bytes_per_launch / (local_avg_ms * 1e-3) / 1e9
    prof = profile_data()
    traffic = prof.get("dram_bytes_per_launch") if prof else None
    iface_avg_ms = prof_ms["interface"] / max(prof_n["interface"], 1)
    energy_avg_ms = prof_ms["energy"] / max(prof_n["energy"], 1)
    n_if = 2 * (NR - 1) * W
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    roofline = {
        "bound": "smem", "achieved": achieved, "peak": smem_peak, "unit": "GB/s", "frac": achieved / smem_peak,
        "traffic": traffic,
        "traffic_note": ("DRAM bytes per launch from the committed ncu capture; the bound is shared memory, "
                         "the HBM state stream is hbm_state_stream below (writes still in L2 at kernel exit "
                         "are not counted by ncu)") if traffic else None,
        "kernel": "fused local solver (k_fused_mt4t: persistent clusters of 8 CTAs x 128 threads, 3 CTAs per SM, one 128x128 subdomain per cluster at a time, 4x4 pixel micro-tile per thread, state moved by tensor copies)",
        "peak_source": "measured live: ld.shared probe kernel (dd_tv_measure_smem_bandwidth)",
        "algorithmic_bytes_per_launch": bytes_per_launch, "avg_launch_ms": local_avg_ms,
        "occupancy": ({"achieved_warps_frac": prof.get("warps_active_frac"),
                       "theoretical_warps_frac": prof.get("theoretical_warps_frac"),
                       "ctas_per_sm": prof.get("ctas_per_sm"), "registers_per_thread": prof.get("registers"),
                       "source": "ncu capture committed in profiles/fused_local_rof4096.json"}
                      if prof else None),
        "hbm_state_stream": {"bytes_per_launch": 28 * H * W,
                             "achieved_gbs": 28 * H * W / (local_avg_ms * 1e-3) / 1e9,
                             "peak_gbs": hbm_peak, "peak_source": "MEASURED_PEAKS.json hbm_gbs"},
        "interface_kernel": {"avg_launch_ms": iface_avg_ms, "bytes_per_launch": 24 * n_if,
                             "achieved_gbs": 24 * n_if / (iface_avg_ms * 1e-3) / 1e9 if iface_avg_ms else None,
                             "peak_gbs": hbm_peak},
        "energy_kernel": {"avg_launch_ms": energy_avg_ms, "bytes_per_launch": 8 * H * W,
                          "achieved_gbs": 8 * H * W / (energy_avg_ms * 1e-3) / 1e9 if energy_avg_ms else None,
                          "peak_gbs": hbm_peak},
    }

    # ---- end to end through dd_tv_solve with pinned host buffers
    f_pin = torch.from_numpy(f).pin_memory()
    u_pin = torch.empty_like(f_pin).pin_memory()
    # the same step as the timed loop: every ENERGY_EVERY outer iterations the energy of
    # the stopping rule is evaluated and read back (an unreachable tolerance keeps the
    # solve running for exactly `steps` outer iterations)
    pe = L.make_params(H, W, NR, NC, fidelity="l2", alpha=ALPHA, inner_iters=INNER, path="fused",
                       outer_iters=args.steps, outer_tol=1e-30, energy_ref=1e-30, energy_every=ENERGY_EVERY)
    se = L.Solver(pe, stream)
    se.solve_host(f_pin.numpy(), None, u_pin.numpy())  # warm-up (graph capture)
    if pg:
        pg.barrier()
    t = time.perf_counter()
    _, st_e2e, _ = se.solve_host(f_pin.numpy(), None, u_pin.numpy())
    dt_e2e = max_over_ranks(time.perf_counter() - t, pg, dev)
    e2e = {"value": whole_job_rate(work, world, dt_e2e), "unit": UNIT,
           "h2d_bytes_per_step": 4 * H * W / args.steps,
           "d2h_bytes_per_step": (4 * H * W + 16 * (args.steps // ENERGY_EVERY)) / args.steps,
           "call": "dd_tv_solve(host f, host u), one call of K outer iterations with the energy check "
                   f"every {ENERGY_EVERY}"}
    se.close()

    # ---- time to relative energy error 1e-4 (fused vs plain vs full-dimension)
    tta = None
    if not args.no_tta:
        rec, why = load_jstar(f)
        if rec is None:
            tta = {"skipped": why}
        else:
            tta = {"J_star": rec["J_star"], "J_star_rel_gap": rec["rel_gap"], "tol": 1e-4,
                   "energy_every": ENERGY_EVERY}
            for path, cap in (("fused", 3000), ("plain", 3000), ("fulldim", 2000)):
                pt = L.make_params(H, W, NR, NC, fidelity="l2", alpha=ALPHA, inner_iters=INNER, path=path,
                                   outer_iters=cap, outer_tol=1e-4, energy_ref=rec["J_star"],
                                   energy_every=ENERGY_EVERY)
                sp = L.Solver(pt, stream)
                u_out = torch.empty_like(fd)
                sp.solve_device(fd, None, u_out)  # warm-up run (graph capture, clocks)
                torch.cuda.synchronize(dev)
                t = time.perf_counter()
                _, stt, rc = sp.solve_device(fd, None, u_out)
                torch.cuda.synchronize(dev)
                dt = time.perf_counter() - t
                tta[path] = {"ms": dt * 1e3, "device_ms": stt.ms, "outer_iters": stt.outer_done,
                             "rel_err": stt.rel_err, "reached": bool(stt.converged)}
                if path != "fused":
                    # one kernel per step streams the state through HBM: u-step 20 B/px (u
                    # read and written, f, pbar1, pbar2), p-step 36 B/px (u; p1, p2 and their
                    # proximal centres read; p1, p2, pbar1, pbar2 written)
                    gbs = 56 * H * W * INNER * stt.outer_done / (stt.ms * 1e-3) / 1e9
                    tta[path]["hbm"] = {"bytes_per_px_inner_iter": 56, "achieved_gbs": gbs, "peak_gbs": hbm_peak,
                                        "frac": gbs / hbm_peak,
                                        "note": "over the whole run, energy checks and multiplier updates included"}
                sp.close()
            if tta["fused"]["reached"] and tta["plain"]["reached"]:
                tta["speedup_vs_plain"] = tta["plain"]["ms"] / tta["fused"]["ms"]
            if tta["fused"]["reached"]:
                # m = infinity: the outer count the checked run stopped at, run without any
                # energy evaluation (one graph replay), the tolerance checked after the fact
                n_star = tta["fused"]["outer_iters"]
                pt = L.make_params(H, W, NR, NC, fidelity="l2", alpha=ALPHA, inner_iters=INNER, path="fused")
                sp = L.Solver(pt, stream)
                sp.load(fd)
                sp.iterate(n_star)          # warm-up (graph capture)
                sp.load(fd)
                torch.cuda.synchronize(dev)
                t = time.perf_counter()
                sp.iterate(n_star)
                torch.cuda.synchronize(dev)
                dt = time.perf_counter() - t
                Jn = sp.current_energy()
                sp.close()
                tta["fused_no_checks"] = {"ms": dt * 1e3, "outer_iters": n_star,
                                          "rel_err": (Jn - rec["J_star"]) / rec["J_star"],
                                          "reached": (Jn - rec["J_star"]) / rec["J_star"] <= 1e-4,
                                          "note": "m = infinity: energy evaluated once, after the timed run"}
            # adaptive inner stopping (eq. stop_inner1), at most ADAPT_CAP inner iterations per
            # local solve: the paper's tolerance (below what float32 iterates resolve: every
            # solve runs to the cap), ADAPT_TOL_F32 (the float32 stand-in) and a loose one
            adaptive = {}
            for itol in (1e-6, ADAPT_TOL_F32, 1e-3):
                key = f"inner_tol={itol:g}"
                try:
                    pt = L.make_params(H, W, NR, NC, fidelity="l2", alpha=ALPHA, inner_iters=ADAPT_CAP,
                                       inner_tol=itol, outer_iters=3000, outer_tol=1e-4, energy_ref=rec["J_star"],
                                       energy_every=ENERGY_EVERY)
                    sp = L.Solver(pt, stream)
                    u_out = torch.empty_like(fd)
                    sp.solve_device(fd, None, u_out)  # warm-up run
                    torch.cuda.synchronize(dev)
                    t = time.perf_counter()
                    _, stt, rc = sp.solve_device(fd, None, u_out)
                    torch.cuda.synchronize(dev)
                    dt = time.perf_counter() - t
                    adaptive[key] = {"ms": dt * 1e3, "device_ms": stt.ms, "outer_iters": stt.outer_done,
                                     "inner_cap": ADAPT_CAP, "max_inner_iters": stt.inner_max,
                                     "mean_inner_iters": stt.pixel_iters / (H * W * max(stt.outer_done, 1)),
                                     "rel_err": stt.rel_err, "reached": bool(stt.converged)}
                    sp.close()
                except L.DDTVError as e:
                    adaptive[key] = {"error": str(e)}
            tta["adaptive"] = adaptive
            if not args.no_tune:
                from paper_1901_00682_gb300 import autotune
                r = autotune.tune(fd, dict(fidelity="l2", alpha=ALPHA), tol=1e-4, j_ref=rec["J_star"],
                                  tiles=(64, 128), inners=(5, 10, 20), max_outer=3000, stream=stream)
                b = r.best
                tta["autotuned"] = {"tile": b.tile, "inner_iters": b.inner, "variant": b.variant, "ms": b.ms,
                                    "outer_iters": b.outer, "reached": b.reached, "trials": r.table()}

    batch = None
    if not args.no_batch:
        import synth
        ims = synth.batch_workload(64, 0)
        bt = L.Batch(ims, inner_iters=INNER, stream=stream)
        fs = [torch.from_numpy(m["f"]).to(dev) for m in ims]
        bt.load(fs)
        n_b = 40
        bt.iterate(n_b)   # warm-up: captures the graph of n_b outer iterations (even start parity)
        torch.cuda.synchronize(dev)
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        bt.iterate(n_b)
        b1.record(stream)
        torch.cuda.synchronize(dev)
        ms_b = b0.elapsed_time(b1) / n_b
        batch = {"workload": "64 images, short side s in {256,512,1024,2048} x aspect {1:1 (s x s), 2:1 (s x 2s), "
                             "1:2 (2s x s)}, even ROF (sigma .05, alpha 10), odd segmentation (c1 .2, c2 .8, "
                             f"alpha 20, tau 1), 128x128 subdomains, {INNER} inner", "pixels": bt.pixels(),
                 "ms_per_outer": ms_b,
                 "value": bt.pixels() * INNER / (ms_b * 1e-3) / 1e6, "unit": UNIT,
                 "launch": f"one CUDA graph of {n_b} outer iterations (2 kernels per outer iteration: batched "
                           "multiplier update, persistent clusters over the (image, subdomain) work list)",
                 "kernel": "k_fused_mt4_batch: the 4x4 micro-tile kernel over the work list (cp.async copies, "
                           "per-image descriptors cached in shared memory)"}
        smem_peak_b = L.measure_smem_bandwidth()
        ach_b = SMEM_BYTES_PER_PX_ITER * bt.pixels() * INNER / (ms_b * 1e-3) / 1e9
        batch["roofline"] = {"bound": "smem", "achieved": ach_b, "peak": smem_peak_b, "unit": "GB/s",
                             "frac": ach_b / smem_peak_b,
                             "note": "whole outer iteration (multiplier update + local solves) against the "
                                     "local solver's algorithmic 28 B per pixel and inner iteration"}
        bt.close()
        if not args.no_tune:
            # subdomain side and inner-iteration count of the batch by time until every
            # image reaches relative energy error 1e-4 against its certified J*
            from paper_1901_00682_gb300 import autotune
            recs, why = load_batch_jstar(ims)
            if recs is not None:
                jr = [r["J_star"] for r in recs]
                jr_note = ("certified per image by the FP64 oracle's duality gap (max rel. gap "
                           f"{max(r['rel_gap'] for r in recs):.1e}; tests/golden/make_batch_jstar.py)")
            else:
                jr = autotune.batch_reference_energies(ims, fs, inner=20, outer=2000, stream=stream)
                jr_note = f"lowest energy of a 2000-outer batched run (K = 20) per image ({why})"
            rb = autotune.tune_batch(ims, fs, tol=1e-4, j_ref=jr, inners=(5, 10, 20), tiles=(64, 128),
                                     max_outer=3000, stream=stream)
            bb = rb.best
            batch["autotuned"] = {"tile": bb.tile, "inner_iters": bb.inner, "device_ms_to_tol": bb.ms,
                                  "outer_iters": bb.outer, "reached": bb.reached, "tol": 1e-4, "j_ref": jr_note,
                                  "trials": rb.table()}
            if bb.reached:
                # the tuned fixed-count solve as one CUDA-graph launch
                bt = L.Batch(ims, inner_iters=bb.inner, stream=stream, tile=bb.tile)
                bt.load(fs)
                bt.iterate(bb.outer)            # capture + warm-up
                bt.load(fs)
                torch.cuda.synchronize(dev)
                b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                b0.record(stream)
                bt.iterate(bb.outer)
                b1.record(stream)
                torch.cuda.synchronize(dev)
                worst = max((bt.energy(i) - jr[i]) / abs(jr[i]) for i in range(len(ims)))
                batch["autotuned"]["one_graph_solve"] = {
                    "ms": b0.elapsed_time(b1), "outer_iters": bb.outer, "worst_rel_err": worst,
                    "launch": f"one CUDA graph of {bb.outer} outer iterations (dd_tv_batch_iterate)"}
                bt.close()
        del fs

    adjoint = None
    if not args.no_adjoint:
        adjoint = measure_adjoint(dev)

    tvl1 = None
    if not args.no_tvl1:
        tvl1 = measure_tvl1(dev, stream)

    cpu = cpu1 = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(f)
        cpu1 = cpu_baseline_one_core()

    if rank == 0:
        # kernels of the timed region: per step the multiplier update and the local
        # solves, per energy check the row-energy reduction
        launches = 2 * args.steps + args.steps // ENERGY_EVERY
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "value_outer": {"value": value / INNER, "unit": "Mpixel*outer-iter/s"},
            "config": {"workload": WORKLOAD, "l2": "state (~470 MB) larger than L2; no flush",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "step": "1 outer iteration (interface + fused local solves), energy every 5 steps"},
            "roofline": roofline, "cpu_baseline": cpu, "cpu_baseline_one_core": cpu1, "e2e": e2e,
            "time_to_accuracy": tta, "batch": batch, "tvl1": tvl1, "adjoint": adjoint,
            "clocks": clocks.summary(), "gpu_launches": launches,
            "launches_by_phase": prof_n, "phase_ms": prof_ms,
            "phase_note": "CUDA-event brackets of every phase launch in the timed steps except the first step "
                          "after each energy read-back",
        }
        print(json.dumps(out), flush=True)
    s.close()
    if pg:
        pg.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
