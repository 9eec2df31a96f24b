"""Throughput of the GeoSSTV P-PDS iteration (Algorithm 1) on GB300.

A step is one full pass of Algorithm 1 over one cube: the fused stencil pass
and the finish of its l1 windows, the threshold search (retry window and its
finish, three radix passes, the gather and its finish) when the fused pass's
windows missed, and the light pass.  The timed passes run as the solver runs
them, in CUDA graphs of 16 passes, where the finish of K1's windows skips the
seven search launches in the passes that need none; K1's duration comes from CUDA events
captured around it in those graphs.  The workload is the 512 x 512 x 224 synthetic cube
(sigma 0.1, 5% salt and pepper, stripes on 10% of the columns, dead lines on
2% of the columns of 10% of the bands), float32 iterates.  The state (about
10 GB) is far larger than L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--storage fp32|bf16|fp16]
    python bench.py --impl reference ...   # the FP64 CPU oracle on host cores

Other measurements, one JSON line each (not bench lines): --quality-grid
(5000 passes over a noise grid), --grad N1xN2xN3 (reverse mode), --batch N
(uneven cubes), --omega-sweep N1xN2xN3, --precision-study N1xN2xN3.

Multi-GPU (torchrun, one rank per GPU): every rank solves its own cube
(replicas, weak scaling); ranks only meet for the barrier and the max-time
reduction.  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PPDS voxel-iters/s & HBM GB/s vs peak; mixed vs FP32 at <=0.01 dB MPSNR loss"
UNIT = "voxel-iter/s"
SHAPE = (512, 512, 224)                   # N1, N2, N3
NOISE = dict(sigma=0.1, sp_rate=0.05, stripe_rate=0.1, stripe_amp=0.25,
             dead_col_rate=0.02, dead_band_rate=0.1)
WORKLOAD = ("GeoSSTV P-PDS (Algorithm 1) on a 512x512x224 synthetic cube: 6 polygonal regions x "
            "3-Gaussian spectra, sigma 0.1, salt-and-pepper 5%, stripes 10% of columns, "
            "dead lines 2% of columns in 10% of bands")
# K1 (fused stencil pass) algorithmic words per voxel: reads u, y1 (2), y2 (2),
# q, w1 (6), w2 (6), s, t, y3 = 21; writes u, w1 (6), w2 (6), y1 (2), y2 (2) = 17.
K1_WORDS = 38
# whole iteration as scheduled: K1 38 + K2 (reads s, t, y3, q, u, u+, v; writes s, t, y3, q) 11
ITER_WORDS = 49
FLOOR_WORDS_FP32 = 43                     # every state word read and written once, v read once
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0       # GB300 HBM3e nominal, reported beside the measured peak
CPU_SAMPLE = (128, 128, 224)              # spatial crop of the workload for the oracle timing


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


K1_SOURCE = {"tma": "k_stencil_tma.cu", "coop": "k_stencil.cu"}
K1_KERNEL = {"tma": "k1_tma (fused stencil pass, TMA-fed)", "coop": "k1_stencil (fused stencil pass)"}


def k1_variant():
    return "coop" if os.environ.get("GSSTV_K1") == "coop" else "tma"


def k1_source_sha(variant):
    """sha256 of K1's translation unit: its source and, depth first in include
    order, every header of the package it includes (each counted once)."""
    import hashlib
    import re
    from paper_2510_00562_gb300 import build
    seen, parts = set(), []

    def add(name):
        if name in seen:
            return
        seen.add(name)
        data = open(os.path.join(build.CSRC, name), "rb").read()
        parts.append(data)
        for inc in re.findall(rb'^\s*#\s*include\s+"([^"]+)"', data, re.M):
            if os.path.exists(os.path.join(build.CSRC, inc.decode())):
                add(inc.decode())

    add(K1_SOURCE[variant])
    return hashlib.sha256(b"".join(parts)).hexdigest()


def k1_traffic_record(storage, variant):
    """ncu dram bytes per voxel of one K1 launch, if recorded for the current
    translation unit of that kernel (source and included headers)."""
    path = os.path.join(ROOT, "profiles", "k1_traffic.json")
    try:
        rec = json.load(open(path))
    except Exception:
        return None
    ent = rec.get(variant)
    if not ent:
        return None
    if ent.get("sha256") != k1_source_sha(variant):
        return None
    st = ent.get(storage)
    return float(st["bytes_per_voxel"]) if st else None


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                rows.append((float(f[0]), float(f[1]), f[3:7]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def dist_setup(world):
    if world <= 1:
        return None
    import torch.distributed as dist
    backend = "nccl" if _cuda_ok() else "gloo"
    dist.init_process_group(backend=backend)
    return dist


def _cuda_ok():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def max_over_ranks(x, dist):
    """Barrier plus maximum of a host float over the ranks (timing only)."""
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


def job_throughput(world, nvox, steps, ms_max):
    """Whole-job voxel-iterations per second: every rank ran `steps` passes over
    its own cube of `nvox` voxels, and the job took the slowest rank's time."""
    return world * nvox * steps / (ms_max * 1e-3)


# ---------------------------------------------------------------------------
# oracle (CPU) timing
# ---------------------------------------------------------------------------
def oracle_problem(shape):
    import numpy as np
    from paper_2510_00562_gb300 import synth
    n1, n2, n3 = shape
    pb = synth.make_problem(n1, n2, n3, seed=0, noise=synth.NoiseSpec(**NOISE))
    return pb


def time_oracle(steps, warmup, shape=CPU_SAMPLE):
    """Runs the FP64 oracle as it stands on a spatial crop; returns (value, seconds, steps)."""
    import numpy as np
    from oracle import ppds as o
    pb = oracle_problem(shape)
    v = pb["v"].astype(np.float64)
    p = o.Params(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], omega=0.03)
    st = o.init_state(v)
    for _ in range(warmup):
        st = o.ppds_step(st, v, p)
    t0 = time.perf_counter()
    for _ in range(steps):
        st = o.ppds_step(st, v, p)
    dt = time.perf_counter() - t0
    nvox = shape[0] * shape[1] * shape[2]
    return nvox * steps / dt, dt


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _oracle_replica(shape, steps, warmup, seed, barrier, queue):
    """One process of the all-core oracle timing: the oracle as it stands on
    its own crop; times `steps` passes between two barriers shared with the
    other replicas."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import numpy as np
    from oracle import ppds as o
    from paper_2510_00562_gb300 import synth
    n1, n2, n3 = shape
    pb = synth.make_problem(n1, n2, n3, seed=seed, noise=synth.NoiseSpec(**NOISE))
    v = pb["v"].astype(np.float64)
    p = o.Params(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], omega=0.03)
    st = o.init_state(v)
    for _ in range(warmup):
        st = o.ppds_step(st, v, p)
    barrier.wait(timeout=600)
    t0 = time.perf_counter()
    for _ in range(steps):
        st = o.ppds_step(st, v, p)
    barrier.wait(timeout=600)
    queue.put(time.perf_counter() - t0)


def time_oracle_all_cores(steps, warmup, shape=CPU_SAMPLE, procs=None):
    """The oracle on every host core: `procs` spawned processes (default: the
    cores this process may run on), each running the single-threaded oracle
    on its own crop of the workload generator (different seeds), timed between
    barriers.  Returns (voxel-iterations/s of all of them, seconds, procs).
    Spawned, not forked: the parent may already hold a CUDA context."""
    import multiprocessing as mp
    procs = procs or host_cores()
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(procs)
    queue = ctx.Queue()
    ps = [ctx.Process(target=_oracle_replica, args=(shape, steps, warmup, 100 + k, barrier, queue))
          for k in range(procs)]
    for q in ps:
        q.start()
    import queue as queue_mod
    times = []
    while len(times) < procs:
        try:
            times.append(queue.get(timeout=2.0))
        except queue_mod.Empty:
            dead = [q.exitcode for q in ps if q.exitcode not in (None, 0)]
            if dead:
                for q in ps:
                    if q.is_alive():
                        q.terminate()
                raise RuntimeError(f"an oracle timing process failed (exit codes {dead})")
    for q in ps:
        q.join(timeout=60)
    dt = max(times)
    nvox = shape[0] * shape[1] * shape[2]
    return procs * nvox * steps / dt, dt, procs


ORACLE_BYTES_PER_VOXEL = 800     # peak resident memory of one oracle process (measured: about 690)


def mem_available():
    """Bytes of memory available to new processes (Linux MemAvailable), or None."""
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return None


def reference_crop(steps, warmup, budget_s=120.0, rate=1.5e6, procs=1, avail=None):
    """Spatial crop of the workload sized so that steps + warmup oracle passes
    take about budget_s seconds at ~rate voxel-iterations per second, and so
    that `procs` oracle processes together hold at most 60 % of the available
    memory."""
    per_step = budget_s * rate / max(steps + warmup, 1)
    avail = mem_available() if avail is None else avail
    if avail:
        per_step = min(per_step, 0.6 * avail / (max(procs, 1) * ORACLE_BYTES_PER_VOXEL))
    side = int(math.sqrt(per_step / SHAPE[2]) // 16 * 16)
    side = max(16, min(side, 512))
    return (side, side, SHAPE[2])


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    # one crop per host core, each the size one core runs in the time budget
    cores = host_cores()
    crop = reference_crop(args.steps, args.warmup, procs=cores)
    value, dt, cores = time_oracle_all_cores(args.steps, args.warmup, shape=crop, procs=cores)
    n1, n2, n3 = crop
    sample = (f"FP64 NumPy oracle as it stands, one Algorithm-1 pass per step on a {n1}x{n2}x{n3} "
              f"spatial crop of the workload generator in each of {cores} single-threaded processes "
              f"(one per host core, {host_cores()} cores available; {args.steps} steps, "
              f"{args.warmup} warm-up)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n1": SHAPE[0], "n2": SHAPE[1], "n3": SHAPE[2],
                   "sample": f"{n1}x{n2}x{n3} crop"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                         "host_cores": host_cores()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
GRAPH_PASSES = 16            # passes per CUDA graph (graph_iters), the solver's default


def gpu_launches(steps, search_passes, graph_passes=GRAPH_PASSES):
    """Kernels launched in `steps` timed passes: whole graphs of graph_passes
    passes launch K1, its window finish (which opens the search launches'
    conditional node when needed) and K2, plus the seven search launches in
    the passes whose node opened (search_passes); the remaining passes run
    eagerly, all ten launches each."""
    in_graphs = (steps // graph_passes) * graph_passes if graph_passes > 0 else 0
    return 3 * in_graphs + 7 * search_passes + 10 * (steps - in_graphs)


def run_gpu(args):
    import numpy as np
    import torch

    from paper_2510_00562_gb300 import build, metrics, synth
    from paper_2510_00562_gb300.solver import GeoSSTVSolver, make_params

    rank, world, local = _env_rank()
    dist = dist_setup(world)
    torch.cuda.set_device(local)
    build.build()

    n1, n2, n3 = args.shape
    nvox = n1 * n2 * n3
    pb = synth.make_problem(n1, n2, n3, seed=rank, noise=synth.NoiseSpec(**NOISE))
    esz = 4 if args.storage == "fp32" else 2
    p = make_params(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], omega=0.03,
                    max_iter=args.steps, storage=args.storage, graph_iters=args.graph_passes)
    stream = torch.cuda.current_stream()
    sol = GeoSSTVSolver(n1, n2, n3, p, stream=stream)
    v_dev = torch.from_numpy(pb["v"]).cuda()
    sol.load(v_dev)
    sol.iterate(args.warmup)
    sol.reset_stats()
    sol.set_timing(True)          # CUDA events around every K1 launch, on the solver's stream

    torch.cuda.synchronize()
    barrier(dist)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        sol.iterate(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(dist)
    ms = ev0.elapsed_time(ev1)
    st = sol.stats()
    sol.set_timing(False)
    ms_max = max_over_ranks(ms, dist)
    value = job_throughput(world, nvox, args.steps, ms_max)

    # end to end through the public host API: copies in, solve, copies out;
    # right after the device-timed region, so that both see the GPU in the
    # same state (not after the precision form's thousand passes)
    sol.set_params(make_params(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], omega=0.03,
                               max_iter=args.steps, storage=args.storage, graph_iters=16))
    vh = torch.from_numpy(pb["v"]).pin_memory()
    uh = torch.empty_like(vh).pin_memory()
    sh = torch.empty_like(vh).pin_memory()
    th = torch.empty_like(vh).pin_memory()
    sol.solve_host(vh, uh, sh, th)           # untimed: the solver's graphs built for these parameters
    torch.cuda.synchronize()
    barrier(dist)
    with ClockSampler(local) as clk_e2e:
        t0 = time.perf_counter()
        sol.solve_host(vh, uh, sh, th)
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0, dist)
    e2e_value = world * nvox * args.steps / e2e_s

    pf = None
    if not args.no_precision_form and args.storage == "fp32" and world == 1:
        pf = precision_form(sol, pb, args.shape, args.pf_iters, args.steps)
    sol.close()
    quality = None
    if rank == 0:
        # Sec. IV-A metrics of the end-to-end result (`steps` iterations from the
        # initial point) against the clean cube; MSSIM on every 8th band to keep
        # the host time short
        u_np = uh.numpy()
        quality = {"iterations": args.steps,
                   "mpsnr_db": metrics.mpsnr(u_np, pb["u_bar"]),
                   "mssim_every_8th_band": metrics.mssim(u_np[::8], pb["u_bar"][::8]),
                   "observation_mpsnr_db": metrics.mpsnr(pb["v"], pb["u_bar"])}

    if rank != 0:
        return 0
    peak, peak_kind = measured_peaks()
    k1_ms = st["k1_ms"] / max(st["k1_launches"], 1)
    k1_bytes = K1_WORDS * esz * nvox
    achieved = k1_bytes / (k1_ms * 1e-3) / 1e9
    variant = k1_variant()
    traffic_bpv = k1_traffic_record(args.storage, variant)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.storage == "fp32" else
        f"f32 math, {args.storage} storage", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.shape == SHAPE else
                   f"GeoSSTV P-PDS (Algorithm 1) on a {n1}x{n2}x{n3} synthetic cube (profiling case)",
                   "n1": n1, "n2": n2, "n3": n3, "storage": args.storage,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (no flush): state "
                         f"{ITER_WORDS * esz * nvox / 1e9:.1f} GB moved per step"},
        "roofline": {"bound": "hbm", "kernel": K1_KERNEL[variant],
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": f"{peak_kind} copy bandwidth",
                     "frac_of_nominal": achieved / NOMINAL_HBM_GBS, "nominal_peak": NOMINAL_HBM_GBS,
                     "traffic": traffic_bpv * nvox if traffic_bpv else None,
                     "algorithmic_bytes": k1_bytes, "k1_ms": k1_ms},
        "iteration_bandwidth": {
            "scheduled_gbs": ITER_WORDS * esz * nvox * args.steps / (ms_max * 1e-3) / 1e9,
            "floor_gbs": FLOOR_WORDS_FP32 * 4 * nvox * args.steps / (ms_max * 1e-3) / 1e9 if esz == 4 else None,
        },
        "tau_search": {"window_hits": st["tau_window_hits"], "retry_hits": st["tau_retry_hits"],
                       "exact_runs": st["tau_exact_runs"], "search_passes": st["search_passes"]},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * nvox / args.steps,
                "d2h_bytes_per_step": 3 * 4 * nvox / args.steps,
                "note": "one gsstv_solve_host call of `steps` iterations after an untimed one (the "
                        "solver's graphs built): pinned H2D of v, state reset, iterations, D2H of u, s, t",
                "clocks": clk_e2e.summary()},
        "gpu_launches": gpu_launches(args.steps, st["search_passes"], args.graph_passes),
        "quality": quality,
    }
    if pf:
        line["precision_form"] = pf
    clk_s = clk.summary()
    if clk_s:
        line["clocks"] = clk_s
    if world == 1 and not args.no_cpu_baseline and args.shape == SHAPE:
        c1, c2, c3 = CPU_SAMPLE
        cv1, cdt1 = time_oracle(args.cpu_steps, 1)
        cv, cdt, cores = time_oracle_all_cores(args.cpu_steps, 1)
        line["cpu_baseline"] = {
            "value": cv, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 NumPy oracle as it stands, {args.cpu_steps} Algorithm-1 passes on a "
                      f"{c1}x{c2}x{c3} spatial crop of the workload in each of {cores} single-threaded "
                      f"processes, one per host core ({cdt:.1f} s)",
            "host_cores": host_cores(),
            "value_1core": cv1,
            "sample_1core": f"the same crop in this process alone ({cdt1:.1f} s)"}
    print(json.dumps(line), flush=True)
    return 0


def precision_form(sol32, pb, shape, N, steps_after):
    """Mixed storage vs FP32 on the same cube and iteration budget N: FP32 for N
    passes, against BF16 iterates (FP32 arithmetic) for 0.8 N passes followed
    by an FP32 phase of 0.2 N passes warm-started from the 16-bit state.
    Returns the 16-bit phase throughput and the MPSNR of both results against
    the clean cube."""
    import torch
    from paper_2510_00562_gb300 import metrics
    from paper_2510_00562_gb300.solver import GeoSSTVSolver, make_params
    n1, n2, n3 = shape
    nvox = n1 * n2 * n3
    n16 = (N * 4) // 5
    kw = dict(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], omega=0.03, graph_iters=16)
    v = torch.from_numpy(pb["v"]).cuda()
    stream = torch.cuda.current_stream()
    sol32.set_params(make_params(max_iter=N, **kw))
    u32 = sol32.solve(v)[0]
    m32 = metrics.mpsnr(u32.cpu().numpy(), pb["u_bar"])
    del u32
    out = {"iterations": N, "fp32_mpsnr_db": m32}
    for storage in ("bf16", "fp16"):
        with GeoSSTVSolver(n1, n2, n3, make_params(max_iter=n16, storage=storage, **kw), stream=stream) as lo:
            lo.load(v)
            lo.iterate(8)                        # graphs built, caches warm
            lo.reset()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            lo.iterate(n16)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            st = lo.get_state()
        m16 = metrics.mpsnr(st["u"].cpu().numpy(), pb["u_bar"])
        sol32.set_params(make_params(max_iter=N - n16, **kw))
        sol32.load(v, reset=False)
        sol32.set_state(st)
        del st
        sol32.iterate(N - n16)
        uf = sol32.get_state()["u"]
        mf = metrics.mpsnr(uf.cpu().numpy(), pb["u_bar"])
        del uf
        out[storage] = {"passes_16bit": n16, "passes_fp32": N - n16,
                        "value_16bit_phase": nvox * n16 / (ms * 1e-3), "unit": UNIT,
                        "mpsnr_after_16bit_db": m16, "mpsnr_db": mf, "delta_vs_fp32_db": mf - m32}
    sol32.set_params(make_params(max_iter=steps_after, **kw))
    return out


BATCH_SIDES = (32, 48, 96, 128, 256, 512)
BATCH_BANDS = (31, 64, 128, 224)


def batch_workload(ncubes, seed=0):
    """Uneven cubes: N1, N2 drawn independently from BATCH_SIDES, N3 from
    BATCH_BANDS; Gaussian sigma ~ U[0.02, 0.15], salt-and-pepper and stripe
    rates ~ U[0, 0.15]."""
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(ncubes):
        n1, n2 = (int(x) for x in rng.choice(BATCH_SIDES, 2))
        n3 = int(rng.choice(BATCH_BANDS))
        out.append((n1, n2, n3, float(rng.uniform(0.02, 0.15)), float(rng.uniform(0.0, 0.15)),
                    float(rng.uniform(0.0, 0.15))))
    return out


def run_batch(args):
    """Many uneven cubes, each with its own Eq. 28 stopping rule (< 1e-5, at
    most 3000 passes): the batch solver against looping the plain solver over
    the same cubes.  One JSON line."""
    # more hardware work queues than the default 8, so that the streams of the
    # one-stream-per-cube batch do not share queues (read when the CUDA context
    # is created)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    import numpy as np
    import torch
    from paper_2510_00562_gb300 import synth
    from paper_2510_00562_gb300.solver import GeoSSTVBatch, GeoSSTVSolver, make_params
    cubes = batch_workload(args.batch)
    pbs, params, vs = [], [], []
    for k, (n1, n2, n3, sg, ps, pt) in enumerate(cubes):
        pb = synth.make_problem(n1, n2, n3, seed=1000 + k,
                                noise=synth.NoiseSpec(sigma=sg, sp_rate=ps, stripe_rate=pt, stripe_amp=0.25))
        params.append(make_params(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], omega=0.03,
                                  tol=1e-5, check_every=50, max_iter=3000, graph_iters=16))
        vs.append(torch.from_numpy(pb["v"]).cuda())
        pbs.append(pb)
    shapes = [c[:3] for c in cubes]
    vox = np.array([n1 * n2 * n3 for n1, n2, n3 in shapes], dtype=np.float64)

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, time.perf_counter() - t0

    # the batch with one stream per cube (the path 16-bit cubes take)
    os.environ["GSSTV_BATCH"] = "streams"
    with GeoSSTVBatch(shapes, params) as bs:
        del os.environ["GSSTV_BATCH"]
        bs.solve(vs)
        (us_s, _, _, done_s), t_streams = timed(lambda: bs.solve(vs))
    with GeoSSTVBatch(shapes, params) as bt:
        bt.solve(vs)                                     # graphs built
        (us, _, _, done_b), t_batch = timed(lambda: bt.solve(vs))
        d_streams = max(float((a - b).abs().max().item()) for a, b in zip(us_s, us))
        del us_s
        # the same batch with every cube's band runs chosen by measurement
        chunks, t_tune = timed(lambda: bt.autotune(vs, passes=20))
        bt.solve(vs)                                     # graphs built again
        (us_t, _, _, done_t), t_tuned = timed(lambda: bt.solve(vs))
        d_tuned = max(float((a - b).abs().max().item()) for a, b in zip(us_t, us))
        del us_t
    sols = [GeoSSTVSolver(n1, n2, n3, p) for (n1, n2, n3), p in zip(shapes, params)]

    def loop():
        res = [s.solve(v) for s, v in zip(sols, vs)]
        return [r[0] for r in res], [r[3] for r in res]

    loop()                                               # graphs built
    (u_loop, done_l), t_loop = timed(loop)
    dmax = max(float((a - b).abs().max().item()) for a, b in zip(us, u_loop))
    for s_ in sols:
        s_.close()
    vi_b = float((vox * np.array(done_b)).sum())
    vi_l = float((vox * np.array(done_l)).sum())
    line = {"batch": {
        "cubes": len(cubes), "data": "synthetic",
        "workload": "N1, N2 from {32,48,96,128,256,512}, N3 from {31,64,128,224}, sigma ~ U[0.02,0.15], "
                    "salt-and-pepper and stripe rates ~ U[0,0.15]; Eq. 28 < 1e-5 checked every 50 passes, "
                    "at most 3000 passes",
        "voxels": float(vox.sum()), "passes": {"min": int(min(done_b)), "median": float(np.median(done_b)),
                                               "max": int(max(done_b))},
        "batch_s": t_batch, "batch_value": vi_b / t_batch,
        "launch": "every stage one launch over all cubes (a table of the cubes' first CTAs), device-side "
                  "stopping rules, 16 passes per CUDA graph",
        "streams_s": t_streams, "streams_same_passes": list(done_s) == list(done_b),
        "max_abs_u_diff_streams": d_streams,
        "loop_s": t_loop, "loop_value": vi_l / t_loop, "unit": UNIT,
        "speedup": t_loop / t_batch, "same_passes": list(done_b) == list(done_l),
        "max_abs_u_diff": dmax,
        "autotuned": {"tune_s": t_tune, "batch_s": t_tuned,
                      "batch_value": float((vox * np.array(done_t)).sum()) / t_tuned,
                      "speedup_vs_loop": t_loop / t_tuned, "bands_per_cta": chunks,
                      "max_abs_u_diff_vs_model_runs": d_tuned}}}
    print(json.dumps(line), flush=True)
    return 0


OMEGAS = (0.001, 0.003, 0.01, 0.03, 0.05, 0.1, 0.3, 1.0)


def run_omega_sweep(args):
    """MPSNR and MSSIM against the balance parameter omega for the five noise
    cases of Sec. IV-A, radii from Eqs. 25-27, stopping rule Eq. 28 (< 1e-5, at
    most 3000 passes); every (case, omega) problem runs in one batch.  One
    JSON line."""
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    import torch
    from paper_2510_00562_gb300 import metrics, radii, synth
    from paper_2510_00562_gb300.solver import GeoSSTVBatch, make_params
    n1, n2, n3 = (int(x) for x in args.omega_sweep.split("x"))
    problems, shapes, params, vs = [], [], [], []
    for case in (1, 2, 3, 4, 5):
        nz = synth.paper_case(case)
        pb = synth.make_problem(n1, n2, n3, seed=100 + case, noise=nz)
        r = radii.paper_radii(pb["v"], nz.sigma, nz.sp_rate, nz.stripe_rate, nz.dead_col_rate,
                              (1 + nz.dead_width_max) / 2.0)
        v = torch.from_numpy(pb["v"]).cuda()
        for om in OMEGAS:
            problems.append((case, om, pb, r))
            shapes.append((n1, n2, n3))
            params.append(make_params(eps=r["eps"], alpha=r["alpha"], beta=r["beta"], omega=om, tol=1e-5,
                                      check_every=10, max_iter=3000, graph_iters=16))
            vs.append(v)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with GeoSSTVBatch(shapes, params) as bt:
        us, _, _, done = bt.solve(vs)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    table = {}
    for (case, om, pb, r), u, n in zip(problems, us, done):
        un = u.cpu().numpy()
        table.setdefault(f"case{case}", {})[str(om)] = {
            "mpsnr_db": metrics.mpsnr(un, pb["u_bar"]),
            "mssim_every_4th_band": metrics.mssim(un[::4], pb["u_bar"][::4]), "passes": int(n)}
    best = {c: max(row, key=lambda k: row[k]["mpsnr_db"]) for c, row in table.items()}
    print(json.dumps({"omega_sweep": {"cube": f"{n1}x{n2}x{n3}", "data": "synthetic", "omegas": list(OMEGAS),
                                      "radii": "Eqs. 25-27", "solve_s": wall, "best_omega_by_mpsnr": best,
                                      "results": table}}), flush=True)
    return 0


def run_slabs(args):
    """The bench cube stored as S band slabs on this one GPU (gsstv_slabs_*):
    every kernel once per slab, the slabs' sums finished together, halo
    planes copied after each pass; against the single handle on the same
    passes.  One JSON line (the cost of the split on one device: extra
    launches, halo copies, and each slab's halo bands)."""
    import numpy as np
    import torch
    from paper_2510_00562_gb300 import build, synth
    from paper_2510_00562_gb300.solver import GeoSSTVSlabs, GeoSSTVSolver, make_params
    build.build()
    n1, n2, n3 = args.shape
    nvox = n1 * n2 * n3
    pb = synth.make_problem(n1, n2, n3, seed=0, noise=synth.NoiseSpec(**NOISE))
    p = make_params(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], omega=0.03, max_iter=args.steps,
                    graph_iters=16)
    v = torch.from_numpy(pb["v"]).cuda()
    out = {"slabs": {"workload": WORKLOAD if args.shape == SHAPE else f"{n1}x{n2}x{n3} cube", "steps": args.steps,
                     "warmup": args.warmup, "unit": UNIT}}

    def timed(obj):
        obj.load(v)
        obj.iterate(args.warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        obj.iterate(args.steps)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    with GeoSSTVSolver(n1, n2, n3, p) as sol:
        ms = timed(sol)
        u_ref = sol.get_state()["u"]
    out["slabs"]["single"] = {"ms_per_step": ms / args.steps, "value": nvox * args.steps / (ms * 1e-3)}
    for S in args.slabs:
        with GeoSSTVSlabs(n1, n2, n3, S, p) as sl:
            ms = timed(sl)
            du = float((sl.get_state()["u"] - u_ref).abs().max().item())
        out["slabs"][str(S)] = {"ms_per_step": ms / args.steps, "value": nvox * args.steps / (ms * 1e-3),
                                "max_abs_u_diff_vs_single": du}
    print(json.dumps(out), flush=True)
    return 0


def run_precision_study(args):
    """The precision form on a cube of its own (default 1024x1024x200, 5000
    iterations: 4000 16-bit + 1000 FP32 against 5000 FP32), one JSON line."""
    import torch
    from paper_2510_00562_gb300 import synth
    from paper_2510_00562_gb300.solver import GeoSSTVSolver, make_params
    n1, n2, n3 = (int(x) for x in args.precision_study.split("x"))
    pb = synth.make_problem(n1, n2, n3, seed=0, noise=synth.NoiseSpec(**NOISE))
    stream = torch.cuda.current_stream()
    with GeoSSTVSolver(n1, n2, n3, make_params(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"],
                                               omega=0.03, graph_iters=16), stream=stream) as sol32:
        t0 = time.perf_counter()
        out = precision_form(sol32, pb, (n1, n2, n3), args.pf_iters, args.pf_iters)
        wall = time.perf_counter() - t0
    print(json.dumps({"precision_study": {"cube": f"{n1}x{n2}x{n3}", "data": "synthetic",
                                          "noise": NOISE, "wall_s": wall, **out}}), flush=True)
    return 0


QUALITY_SHAPES = ((256, 256, 128), (512, 512, 224))
QUALITY_SIGMAS = (0.05, 0.1)
QUALITY_SP = (0.05, 0.1)


def run_quality_grid(args):
    """The plain FP32 method at paper-like scale: 5000 fixed passes (tol off)
    on 256x256x128 and 512x512x224 cubes of the bench generator, for
    sigma in {0.05, 0.1} x salt-and-pepper rate in {0.05, 0.1}, stripes on 10 %
    of columns, dead lines on 2 % of columns in 10 % of bands.  Throughput
    (CUDA events around gsstv_solve: state reset, the passes, the copy-out),
    the scheduled iteration bandwidth, MPSNR and MSSIM (every 4th band)
    against the clean cube.  One JSON line."""
    import torch
    from paper_2510_00562_gb300 import metrics, synth
    from paper_2510_00562_gb300.solver import GeoSSTVSolver, make_params
    iters = args.quality_iters
    stream = torch.cuda.current_stream()
    peak, src = measured_peaks()
    rows = []
    for n1, n2, n3 in QUALITY_SHAPES:
        nvox = n1 * n2 * n3
        with GeoSSTVSolver(n1, n2, n3, make_params(max_iter=iters, graph_iters=16), stream=stream) as sol:
            for sg in QUALITY_SIGMAS:
                for sp in QUALITY_SP:
                    nz = synth.NoiseSpec(sigma=sg, sp_rate=sp, stripe_rate=0.1, stripe_amp=0.25,
                                         dead_col_rate=0.02, dead_band_rate=0.1)
                    pb = synth.make_problem(n1, n2, n3, seed=7, noise=nz)
                    sol.set_params(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], omega=0.03)
                    v = torch.from_numpy(pb["v"]).cuda()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    with ClockSampler(torch.cuda.current_device()) as clk:
                        e0.record(stream)
                        u, _, _, done = sol.solve(v)
                        e1.record(stream)
                        torch.cuda.synchronize()
                    ms = e0.elapsed_time(e1)
                    un = u.cpu().numpy()
                    rows.append({
                        "cube": f"{n1}x{n2}x{n3}", "sigma": sg, "sp_rate": sp, "passes": done,
                        "seconds": ms / 1e3, "value": nvox * done / (ms * 1e-3), "unit": UNIT,
                        "iteration_gbs": ITER_WORDS * 4 * nvox * done / (ms * 1e-3) / 1e9,
                        "mpsnr_db": metrics.mpsnr(un, pb["u_bar"]),
                        "mssim_every_4th_band": metrics.mssim(un[::4], pb["u_bar"][::4]),
                        "observation_mpsnr_db": metrics.mpsnr(pb["v"], pb["u_bar"]),
                        "clocks": clk.summary()})
                    del v, u
    print(json.dumps({"quality_grid": {"data": "synthetic", "storage": "fp32", "omega": 0.03,
                                       "radii": "make_problem (rho 0.95, 0.9, 0.9)", "peak_gbs": peak,
                                       "peak_source": src, "runs": rows}}), flush=True)
    return 0


# words per voxel of one transposed pass in place (k_adjoint.cu), every array
# element read or written once per kernel: SUMS reads 10; CUBE reads 18
# (states k and k+1 where q and the box need them, the adjoints of u, s, t,
# y1..y4, v, v_bar) and writes 8; AUX reads 32 (w1, w2 and their adjoints,
# y1, y2 and theirs) and writes 24; FIN1 reads 9 and writes 4; FIN2 reads
# 17 and writes 4.
ADJ_WORDS = 126


def run_grad(args):
    """Reverse mode at one size: K passes forward (gsstv_solve) against the
    gradient of the MSE loss of u_K with respect to v and (eps, alpha, beta,
    omega) (gsstv_unrolled_vjp), central finite differences of the loss
    (step 1e-3 relative) beside the parameter gradients and one directional
    derivative in v, and the transposed pass alone against the HBM roofline.
    One JSON line."""
    import numpy as np
    import torch
    from paper_2510_00562_gb300 import synth
    from paper_2510_00562_gb300.solver import GRAD_PARAMS, GeoSSTVSolver, make_params
    n1, n2, n3 = (int(x) for x in args.grad.split("x"))
    K, C = args.grad_iters, args.grad_ckpt
    N = n1 * n2 * n3
    pb = synth.make_problem(n1, n2, n3, seed=0, noise=synth.NoiseSpec(**NOISE))
    v = torch.from_numpy(pb["v"]).cuda()
    ub = torch.from_numpy(pb["u_bar"].astype("float32")).cuda()
    stream = torch.cuda.current_stream()
    peak, src = measured_peaks()
    prm = dict(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], omega=0.03)

    def ev_time(fn, r):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(r):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / r

    with GeoSSTVSolver(n1, n2, n3, make_params(max_iter=K, graph_iters=16, **prm), stream=stream) as sol:
        def loss_of(vv, **over):
            sol.set_params(**{**prm, **over})
            u_, _, _, _ = sol.solve(vv)
            return float(((u_.double() - ub.double()) ** 2).mean()), u_

        loss, u = loss_of(v)
        seed = (2.0 / N) * (u - ub)
        fwd_ms = ev_time(lambda: sol.solve(v), 3)

        def bwd():
            sol.load(v)
            return sol.unrolled_vjp(K, seed, ckpt_every=C)

        vbar, pbar = bwd()
        bwd_ms = ev_time(bwd, 3)
        free0, _ = torch.cuda.mem_get_info()
        P = (N + 63) // 64 * 64
        scratch = ((K + C - 1) // C + C + 1) * 21 * P * 4 + 15 * P * 4 + 160
        # every state kept (checkpoint every pass): nothing run twice
        keep_bytes = (K + 2) * 21 * P * 4 + 15 * P * 4 + 160
        keep = None
        if keep_bytes < 0.8 * free0:
            def bwd_keep():
                sol.load(v)
                return sol.unrolled_vjp(K, seed, ckpt_every=1)
            vk, pk = bwd_keep()
            keep = {"backward_ms": ev_time(bwd_keep, 3), "scratch_bytes": keep_bytes,
                    "max_rel_diff_params": max(abs(pk[k] - pbar[k]) / abs(pbar[k]) for k in GRAD_PARAMS),
                    "rel_diff_vbar": float((vk - vbar).norm() / vbar.norm())}
            keep["backward_over_forward"] = keep["backward_ms"] / fwd_ms
        # central differences, steps 1e-3 and 1e-4 of each parameter
        fd = {}
        for k in GRAD_PARAMS:
            fd[k] = {"adjoint": pbar[k]}
            for rs in (1e-3, 1e-4):
                h = rs * prm[k]
                lp, _ = loss_of(v, **{k: prm[k] + h})
                lm, _ = loss_of(v, **{k: prm[k] - h})
                fd[k][f"fd_{rs:g}"] = (lp - lm) / (2 * h)
        # one direction in v, zero on the salt-and-pepper and dead voxels (0 or
        # 1 exactly: the box's kinks, where only one-sided derivatives exist)
        g = torch.from_numpy(np.random.default_rng(1).standard_normal(pb["v"].shape).astype("float32")).cuda()
        g = torch.where((v == 0) | (v == 1), torch.zeros_like(g), g)
        fd["v_direction"] = {"adjoint": float((vbar.double() * g.double()).sum())}
        for rs in (1e-3, 1e-4):
            hv = rs * float(v.abs().mean())
            lp, _ = loss_of((v + hv * g).contiguous())
            lm, _ = loss_of((v - hv * g).contiguous())
            fd["v_direction"][f"fd_{rs:g}"] = (lp - lm) / (2 * hv)
        for ent in fd.values():
            for rs in ("0.001", "0.0001"):
                f_ = ent[f"fd_{rs}"]
                ent[f"rel_diff_{rs}"] = abs(f_ - ent["adjoint"]) / max(abs(f_), 1e-300)
        sol.set_params(**prm)
        # the transposed pass alone, in place, no parameter read-back
        sol.load(v)
        sol.iterate(5)
        x = sol.get_state()
        sol.iterate(1)
        x1 = sol.get_state()
        bar = {k: 1e-3 * torch.randn_like(t) for k, t in x.items()}
        vb = torch.zeros_like(v)
        for _ in range(3):
            sol.vjp_step(x, x1, bar, vbar=vb, in_place=True, want_params=False)
        step_ms = ev_time(lambda: sol.vjp_step(x, x1, bar, vbar=vb, in_place=True, want_params=False), 20)
        handle_bytes = sol.device_bytes()
    ach = ADJ_WORDS * 4 * N / (step_ms * 1e-3) / 1e9
    line = {"grad": {
        "cube": f"{n1}x{n2}x{n3}", "passes": K, "data": "synthetic", "noise": NOISE,
        "loss": "mean((u_K - u_bar)^2)", "loss_value": loss,
        "forward_ms": fwd_ms, "backward_ms": bwd_ms, "backward_over_forward": bwd_ms / fwd_ms,
        "checkpoint_every": C, "scratch_bytes": scratch, "handle_bytes": handle_bytes,
        "every_state_kept": keep,
        "free_bytes_after_backward": free0,
        "gradients_vs_central_differences": fd,
        "adjoint_pass": {"ms": step_ms, "kernels": 5, "algorithmic_bytes_per_voxel": ADJ_WORDS * 4,
                         "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                                      "frac": ach / peak, "peak_source": src}},
        "unit": "ms"}}
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--storage", default="fp32", choices=["fp32", "bf16", "fp16"])
    ap.add_argument("--cpu-steps", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-precision-form", action="store_true")
    ap.add_argument("--pf-iters", type=int, default=500,
                    help="iteration budget of the mixed-vs-FP32 comparison")
    ap.add_argument("--precision-study", default=None, metavar="N1xN2xN3",
                    help="run only the mixed-vs-FP32 comparison on a cube of this size "
                         "(with --pf-iters 5000 for the 4000 + 1000 split) and print one JSON line")
    ap.add_argument("--omega-sweep", default=None, metavar="N1xN2xN3",
                    help="run only the omega sweep of the five noise cases on a cube of this size")
    ap.add_argument("--batch", type=int, default=0, metavar="NCUBES",
                    help="run only the batch measurement on NCUBES uneven cubes and print one JSON line")
    ap.add_argument("--quality-grid", action="store_true",
                    help="run only the 5000-pass quality grid on 256x256x128 and 512x512x224")
    ap.add_argument("--quality-iters", type=int, default=5000)
    ap.add_argument("--grad", default=None, metavar="N1xN2xN3",
                    help="run only the reverse-mode measurement on a cube of this size")
    ap.add_argument("--grad-iters", type=int, default=200)
    ap.add_argument("--grad-ckpt", type=int, default=20, help="passes between checkpoints")
    ap.add_argument("--slabs", type=int, nargs="*", default=None, metavar="S",
                    help="run only the band-slab measurement with these slab counts")
    ap.add_argument("--graph-passes", type=int, default=GRAPH_PASSES,
                    help="passes per CUDA graph (0: every launch from the host, e.g. for a per-kernel launch list)")
    ap.add_argument("--shape", default="512x512x224",
                    help="N1xN2xN3; anything but the default is a profiling case, not a bench line")
    args = ap.parse_args(argv)
    args.shape = tuple(int(x) for x in args.shape.lower().split("x"))
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.slabs:
        return run_slabs(args)
    if args.precision_study:
        return run_precision_study(args)
    if args.batch:
        return run_batch(args)
    if args.omega_sweep:
        return run_omega_sweep(args)
    if args.grad:
        return run_grad(args)
    if args.quality_grid:
        return run_quality_grid(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
