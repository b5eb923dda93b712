"""Benchmark: demag-convolution + exchange + LLG/RK4 throughput on one GB300 (or N replicas).

Workload (default): thin film 1024 x 1024 x 1 cells of 2 x 2 x 3 nm, Ms = 8.6e5 A/m,
A_ex = 1.3e-11 J/m, alpha = 0.02, dt = 1e-13 s, seeded vortex + noise initial state,
1000 RK4 steps per benchmark step (4 demag evaluations per RK4 step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

value  = cells x demag evaluations / s over the K timed steps (Gcell-demag/s), inputs resident
         in HBM; L2 is flushed (512 MB write) before each timed step.
e2e    = the same metric through the public API with host buffers: pinned-host m -> device,
         gbd_llg_step, device -> pinned-host m, inside the timed region.
Multi-GPU: the meshes are independent, so N ranks run N replicas (no collective on the data
path); value is the sum over ranks divided by the slowest rank's time ("scaling": "weak").
--impl reference times the FP64 CPU oracle on the host cores on a bounded sample of the same
workload (one RK4 step = 4 demag evaluations of the full film), rank 0 only.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gcell-demag/s & LLG steps/s; served p50/p99 vs plain path at rel err ≤1e-5"
UNIT = "Gcell-demag/s"
L2_FLUSH_BYTES = 512 << 20


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

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
        if self.t:
            self.t.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def film_bytes_per_launch(n, Hx, Ky):
    """Algorithmic DRAM bytes of one launch of each film pass (FP32 data, complex64 spectra).

    row_rk (x C2R + exchange + LLG + RK4 stage + next x R2C), averaged over the four stages:
      spectrum read 8*3*Hx*ny + spectrum write 8*3*Hx*ny (the last stage of a call skips it)
      + m_stage 12 B/cell + m0/acc reads (stages 2-4: 24 B/cell) + acc/next writes
      (stages 1-3: 24 B/cell, stage 4: 12 B/cell): 12 + 18 + 21 = 51 B/cell on average.
    film_conv (y FFT -> kernel product -> y IFFT): spectrum read + write 2*8*3*Hx*ny
      + kernel 16*Hx*Ky.
    row_fwd (x R2C of m): 12 B/cell + spectrum write 8*3*Hx*ny.
    """
    nx, ny, nz = n
    N = nx * ny * nz
    spec = 8 * 3 * Hx * ny * nz
    return {
        "row_rk": 2 * spec + 51 * N,
        "film_conv": 2 * spec + 16 * Hx * Ky,
        "row_fwd": spec + 12 * N,
    }


def bytes_per_pass_3d(n, dims):
    """Algorithmic DRAM bytes of each pass of one 3D demag evaluation (FP32 fields, complex64
    spectra): x R2C reads M 12 B/cell, writes S [3][nz][Hx][ny]; y_fwd reads S, writes T
    [3][nz][Hx][Py]; z_conv reads and writes T and reads the kernel [Hx][Py/2+1][Pz/2+1][6];
    y_inv reads T, writes S; x C2R reads S and writes H 12 B/cell."""
    nx, ny, nz = n
    Px, Py, Pz, Hx, Ky, Kz = dims
    N = nx * ny * nz
    S = 24 * Hx * ny * nz
    Tb = 24 * Hx * Py * nz
    K = 24 * Hx * Ky * Kz
    return {"row_fwd": 12 * N + S, "y_fwd": S + Tb, "z_conv": 2 * Tb + K, "y_inv": Tb + S, "row_inv": S + 12 * N}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the kernel sources with // comments and blank lines left out, so that a comment
    edit does not separate the sources from counters taken on them."""
    h = hashlib.sha256()
    for f in ("gbd_fft.cuh", "gbd_tc.cuh", "gbd_kernels.cuh", "gbd_launch.cuh", "gbd_row.cuh", "gbd_row.cu", "gbd_row_io.cu", "gbd_row_rk.cu",
              "gbd_rowpipe.cuh", "gbd_conv.cuh", "gbd_conv.cu", "gbd_ypass.cuh", "gbd_ypass.cu", "gbd_mixed_row.cu",
              "gbd_mixed_conv.cu"):
        with open(os.path.join(ROOT, "paper_2308_08447_gb300", "csrc", f), encoding="utf-8") as fh:
            for line in fh:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if taken on the current kernels."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    v = d.get("bytes_per_launch", {}).get(kernel)
    return float(v) if v is not None else None


def run_ours(args):
    import numpy as np
    import torch

    from paper_2308_08447_gb300 import gbdemag
    from paper_2308_08447_gb300 import replicas
    from paper_2308_08447_gb300 import workloads as W

    rank, world, local = _dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    gbdemag.load()

    spec = W.thin_film()
    nsteps = args.llg_steps
    m0 = W.vortex_noise(spec.n, spec.cell, spec.seed)
    mesh = gbdemag.Mesh(spec.n, spec.cell, spec.Ms, A_ex=spec.A_ex, alpha=spec.alpha)
    mesh.autotune()   # tile variant per pass (set-up, before the timed region)
    m = torch.from_numpy(m0).cuda()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    cells = spec.cells
    evals_per_step = 4 * nsteps

    barrier = replicas.barrier

    # warm-up
    for _ in range(args.warmup):
        mesh.llg_step(m, nsteps, spec.dt)
    torch.cuda.synchronize()

    # timed region: K steps, L2 flushed before each, device time by CUDA events on the stream
    sampler = ClockSampler(local)
    sampler.start()
    times = []
    barrier()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mesh.llg_step(m, nsteps, spec.dt)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    # whole job: the cells x evaluations of every replica over the slowest replica's time
    thr, t_total, _ = replicas.job_throughput(cells * evals_per_step * args.steps, sum(times) / 1e3, "cuda")
    value = thr / 1e9
    ms_per_step = t_total * 1e3 / args.steps

    # end to end through the public API with host buffers
    host_in = torch.from_numpy(m0).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    md = torch.empty_like(m)
    e2e_times = []
    for i in range(args.steps + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        md.copy_(host_in, non_blocking=True)
        mesh.llg_step(md, nsteps, spec.dt)
        host_out.copy_(md, non_blocking=True)
        torch.cuda.synchronize()
        if i > 0:
            e2e_times.append(time.perf_counter() - t0)
    e2e_thr, _, _ = replicas.job_throughput(cells * evals_per_step * len(e2e_times), sum(e2e_times), "cuda")
    e2e_value = e2e_thr / 1e9
    assert np.isfinite(host_out.numpy()).all()

    # per-pass device time (CUDA events around every launch), one instrumented step
    gbdemag.gbd_mesh_set_timing(mesh.handle, True)
    flush.zero_()
    mesh.llg_step(m, nsteps, spec.dt)
    torch.cuda.synchronize()
    passes = gbdemag.gbd_mesh_read_timing(mesh.handle)
    gbdemag.gbd_mesh_set_timing(mesh.handle, False)
    dims = gbdemag.gbd_plan_dims(mesh.desc)
    bpl = film_bytes_per_launch(spec.n, dims[3], dims[4])
    top = max(passes, key=lambda k: passes[k][0])
    # Events around every launch stretch each pass a little, so the average launch time of the
    # top pass is taken from the uninstrumented timed region instead: its time per benchmark
    # step times the pass's share of the instrumented step, over its launches per step.
    share = {k: v[0] / sum(x[0] for x in passes.values()) for k, v in passes.items()}
    avg_ms = ms_per_step * share[top] / passes[top][1]
    peak, peak_kind = measured_peaks()
    achieved = bpl[top] / (avg_ms * 1e-3) / 1e9
    launches_per_step = sum(c for _, c in passes.values())
    roofline = {"bound": "hbm", "kernel": top, "achieved": round(achieved, 1), "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": ncu_traffic(top), "algorithmic_bytes_per_launch": bpl[top],
                "avg_launch_us": round(avg_ms * 1e3, 2),
                "avg_launch_us_how": "uninstrumented step time x the pass's share of an event-instrumented step",
                "passes_us_instrumented": {k: round(v[0] / v[1] * 1e3, 2) for k, v in passes.items()},
                "tuning": list(gbdemag.gbd_mesh_get_tuning(mesh.handle)),
                "share": {k: round(v, 3) for k, v in share.items()}}

    # the same run with the demag extrapolated at RK4 sub-steps (Sec. III; one demag evaluation
    # per step after four start-up steps), timed alike, and its end state against the exact run's
    extrap = None
    if not args.no_extrap:
        mx = torch.from_numpy(m0).cuda()
        mesh.llg_step(mx, nsteps, spec.dt, extrap=True)
        xt = []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mesh.llg_step(mx, nsteps, spec.dt, extrap=True)
            e1.record(stream)
            torch.cuda.synchronize()
            xt.append(e0.elapsed_time(e1) / 1e3)
        xt_max = replicas.max_over_ranks(sum(xt), "cuda")
        a_, b_ = torch.from_numpy(m0).cuda(), torch.from_numpy(m0).cuda()
        mesh.llg_step(a_, nsteps, spec.dt)
        mesh.llg_step(b_, nsteps, spec.dt, extrap=True)
        evals = 4 * min(nsteps, 4) + max(nsteps - 4, 0)
        extrap = {"llg_steps_per_s": round(world * nsteps * args.steps / xt_max, 1),
                  "speedup_vs_exact_steps": round(t_total / xt_max, 3),
                  "demag_evals_per_llg_step": round(evals / nsteps, 4),
                  "gcell_demag_per_s": round(world * cells * evals * args.steps / xt_max / 1e9, 3),
                  "max_abs_dm_vs_exact_after_%d_steps" % nsteps: float((a_ - b_).abs().max())}

    # bounded device-side waits that gave up during the runs above (after the timed regions)
    dev_status = "ok" if mesh.device_status() == gbdemag.GBD_OK else "a staged-copy wait gave up"
    result = None
    if rank == 0:
        result = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "llg_steps_per_s": round(world * nsteps * args.steps / t_total, 1),
            "config": {"workload": "thin film 1024x1024x1, 2x2x3 nm cells, demag + exchange + LLG RK4, "
                                   "%d RK4 steps per benchmark step" % nsteps,
                       "cells_per_gpu": cells, "demag_evals_per_step": evals_per_step, "dt_s": spec.dt,
                       "parallelism": "replicas x%d" % world, "l2": "flushed (512 MB write) before each step"},
            "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": host_in.numel() * 4,
                    "d2h_bytes_per_step": host_out.numel() * 4},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
            "roofline": roofline,
        }
        result["device_status"] = dev_status
        if extrap is not None:
            result["extrapolated_demag"] = extrap
        if world == 1 and not args.no_cpu_baseline:
            result["cpu_baseline"] = cpu_baseline(spec, m0, repeats=4)
            result["cpu_baseline_all_cores"] = cpu_baseline_all_cores(spec)
    mesh.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return result


def oracle_tensor(spec):
    """The oracle's tensor at every offset of the mesh (set-up of the CPU baseline, untimed)."""
    from oracle import tensor as T
    return T.tensor_all_offsets(spec.n, spec.cell)


def cpu_baseline(spec, m0, repeats=1, Nf=None):
    """The FP64 oracle, as it stands, on the host cores: `repeats` RK4 steps of the full film
    (4 FFT-convolution demag evaluations each). Tensor set-up is outside the timed region."""
    import numpy as np

    from oracle import llg as L

    if Nf is None:
        Nf = oracle_tensor(spec)
    m = m0.astype(np.float64)
    f = lambda v: L.rhs(v, Nf, spec.cell, spec.Ms, spec.A_ex, spec.alpha)
    t0 = time.perf_counter()
    for _ in range(repeats):
        m = L.rk4_step(m, spec.dt, f)
    t = time.perf_counter() - t0
    value = spec.cells * 4 * repeats / t / 1e9
    return {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d RK4 step(s) of the 1024x1024x1 film = %d demag evaluations (numpy FP64, "
                      "single-threaded FFT); %.1f s" % (repeats, 4 * repeats, t)}


def _oracle_replica(q, barrier, repeats):
    """One replica of the CPU baseline in its own process: set-up, wait for all replicas, then
    `repeats` RK4 steps of the full film; puts the timed seconds on q."""
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    import numpy as np

    from oracle import llg as L
    from paper_2308_08447_gb300 import workloads as W
    spec = W.thin_film()
    m = W.vortex_noise(spec.n, spec.cell, spec.seed).astype(np.float64)
    Nf = oracle_tensor(spec)
    f = lambda v: L.rhs(v, Nf, spec.cell, spec.Ms, spec.A_ex, spec.alpha)
    barrier.wait()
    t0 = time.perf_counter()
    for _ in range(repeats):
        m = L.rk4_step(m, spec.dt, f)
    q.put(time.perf_counter() - t0)


def cpu_baseline_all_cores(spec, repeats=1):
    """The same oracle on every host core at once: one independent replica per core (spawned
    processes, one thread each), started together after their untimed set-up; the value is
    the work of all replicas over the slowest replica's time."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    ctx = mp.get_context("spawn")
    q, barrier = ctx.Queue(), ctx.Barrier(cores)
    procs = [ctx.Process(target=_oracle_replica, args=(q, barrier, repeats)) for _ in range(cores)]
    for p in procs:
        p.start()
    times = [q.get(timeout=900) for _ in procs]
    for p in procs:
        p.join()
    value = cores * spec.cells * 4 * repeats / max(times) / 1e9
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d concurrent replicas x %d RK4 step(s) of the 1024x1024x1 film (numpy FP64, one thread "
                      "each); slowest replica %.1f s" % (cores, repeats, max(times))}


def run_batch(args):
    """64 uneven meshes (nx, ny in {64..512} step 32, nz in {1, 2, 4, 8, 16}, cubic 2-5 nm cells,
    Ms in [4e5, 1.4e6] A/m, random unit m, 100 RK4 steps each): the plain path (each mesh alone,
    one gbd_llg_step call after another) against one batched CUDA-graph launch (gbd_batch_run)."""
    import numpy as np
    import torch

    from paper_2308_08447_gb300 import gbdemag
    from paper_2308_08447_gb300 import workloads as W

    torch.cuda.set_device(0)
    gbdemag.load()
    specs = W.batch_meshes(count=args.batch_count, seed=4, steps=args.llg_steps if args.llg_steps != 1000 else 100)
    t0 = time.perf_counter()
    meshes = [gbdemag.Mesh(s.n, s.cell, s.Ms, A_ex=s.A_ex, alpha=s.alpha, pow2_pad=args.pow2_pad) for s in specs]
    tunings = [m.autotune() for m in meshes]
    setup_s = time.perf_counter() - t0
    init = [torch.from_numpy(W.random_unit(s.n, s.seed)).cuda() for s in specs]
    steps = [s.steps for s in specs]
    dts = [s.dt for s in specs]
    evals = sum(s.cells * 4 * s.steps for s in specs)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        return ts

    plain_m = [m.clone() for m in init]

    def plain():
        for mesh, m, n, dt in zip(meshes, plain_m, steps, dts):
            mesh.llg_step(m, n, dt)

    batch = gbdemag.Batch(meshes)
    batch_m = [m.clone() for m in init]

    def batched():
        batch.run(batch_m, steps, dts)

    # one run of each from the same initial state: results must be bit-identical
    plain()
    batched()
    torch.cuda.synchronize()
    identical = all(torch.equal(a, b) for a, b in zip(plain_m, batch_m))
    for _ in range(max(0, args.warmup - 1)):
        plain()
        batched()
    sampler = ClockSampler(0)
    sampler.start()
    t_plain = timed(plain, args.steps)
    t_batch = timed(batched, args.steps)
    clocks = sampler.stop()
    v_plain = evals * len(t_plain) / sum(t_plain) / 1e9
    v_batch = evals * len(t_batch) / sum(t_batch) / 1e9
    # padded grid points of the meshes' plans against powers of two on every axis
    vol = lambda d: d[0] * d[1] * d[2]
    pad_vol = sum(vol(gbdemag.gbd_mesh_plan_dims(m.handle)) for m in meshes)
    pad_vol2 = sum(vol(gbdemag.gbd_plan_dims(gbdemag.make_desc(s.n, s.cell, s.Ms, pow2_pad=True))) for s in specs)
    batch.close()
    for m in meshes:
        m.close()
    return {"metric": METRIC, "value": round(v_batch, 3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * sum(t_batch) / len(t_batch), 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "batched: %d uneven meshes, %d RK4 steps each, one CUDA-graph launch per run"
                                   % (len(specs), steps[0]),
                       "cells": sum(s.cells for s in specs), "demag_evals_per_step": evals,
                       "l2": "flushed (512 MB write) before each step", "setup_s": round(setup_s, 1)},
            "plain_path": {"value": round(v_plain, 3), "unit": UNIT,
                           "ms_per_step": round(1e3 * sum(t_plain) / len(t_plain), 3)},
            "speedup_vs_plain": round(v_batch / v_plain, 3), "results_bit_identical": bool(identical),
            "padded_volume_vs_pow2": round(pad_vol / pad_vol2, 4),
            "tunings": {"%dx%dx%d" % s.n: list(t) for s, t in zip(specs, tunings)},
            "gpu_launches": sum(1 + 8 * n for n in steps) * args.steps, "clocks": clocks}


def run_serve(args):
    """Poisson arrivals (200 requests/s) of relaxation jobs (alpha = 0.5, 200-2000 steps, mesh
    sides log-uniform 64..1024, nz 1..16), admitted by a 150 GB budget, continuously batched;
    latency percentiles and throughput against the plain path (each job alone, in arrival order,
    on the same trace). At 200 requests/s the offered load is many times what one GPU serves
    (saturation: latency is queueing). With --rho r the same jobs are then served again at the
    arrival rate r / s, s the plain path's mean service time measured in the saturated run (the
    Poisson trace rescaled in time), labelled as the load factor r."""
    import numpy as np
    import torch

    from paper_2308_08447_gb300 import serve

    torch.cuda.set_device(0)
    os.environ.setdefault("GBD_KERNEL_CACHE_BYTES", str(64 << 30))
    ex = serve.GpuExecutor(extrap=args.extrap)
    jobs = serve.make_jobs(args.requests, args.rate, seed=5)
    t0 = time.perf_counter()
    ex.prewarm(jobs)
    setup_s = time.perf_counter() - t0
    sampler = ClockSampler(0)
    sampler.start()

    def one_trace(scale):
        trace = [serve.Job(j.id, j.spec, j.arrival * scale) for j in jobs]
        srv = serve.Server(ex, 150e9, chunk=args.chunk, max_active=args.max_active or None)
        served = srv.run(trace)
        ex.close()
        plain = serve.run_plain(ex, [serve.Job(j.id, j.spec, j.arrival * scale) for j in jobs])
        by_id = {j.id: j for j in plain}
        identical = all(np.array_equal(j.result, by_id[j.id].result) for j in served)
        for j in served + plain:
            j.result = None
        s_served, s_plain = serve.summarize(served, args.extrap), serve.summarize(plain, args.extrap)
        busy = sum(j.finished - j.admitted for j in plain)   # the plain path runs one job at a time
        return s_served, s_plain, identical, srv, busy

    s_served, s_plain, identical, srv, busy = one_trace(1.0)
    out = {"metric": METRIC, "value": round(s_served["gcell_demag_per_s"], 3), "unit": UNIT, "n_gpus": 1,
           "steps": 1, "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": "served: %d Poisson-arrival jobs at %.0f/s, continuous batching, %d-step chunks, "
                                  "150 GB budget" % (len(jobs), args.rate, args.chunk),
                      "max_active_cap": args.max_active or None, "setup_s": round(setup_s, 1),
                      "demag_extrapolation": bool(args.extrap)},
           "served": s_served, "plain_path": s_plain, "results_bit_identical": bool(identical),
           "plain_mean_service_s": round(busy / len(jobs), 4),
           "max_active": max(a for _, a, _ in srv.trace), "iterations": len(srv.trace)}
    if args.rho:
        rate = args.rho * len(jobs) / busy
        s2, p2, ident2, srv2, _ = one_trace(args.rate / rate)
        out["load_%g" % args.rho] = {"rate_per_s": round(rate, 3),
                                     "how": "rate = %g / (plain mean service time of the saturated run)" % args.rho,
                                     "served": s2, "plain_path": p2, "results_bit_identical": bool(ident2),
                                     "max_active": max(a for _, a, _ in srv2.trace), "iterations": len(srv2.trace)}
    out["clocks"] = sampler.stop()
    return out


def run_3d(args):
    """512 x 512 x 64 cells of 4 nm, Ms = 8e5 A/m, random unit m: one demag evaluation and 100 RK4
    steps with FP32 stages and with split-BF16 and split-FP16 tensor-core stages. The demag error of each is
    taken against the FP64 oracle's FFT convolution of the full mesh (--oracle-3d); the 100-step
    error against the oracle's RK4 run is taken on a 64 x 64 x 8 mesh of the same material."""
    import numpy as np
    import torch

    from paper_2308_08447_gb300 import gbdemag
    from paper_2308_08447_gb300 import workloads as W

    torch.cuda.set_device(0)
    gbdemag.load()
    spec = W.large_3d()
    if args.n3d:
        spec.n = tuple(args.n3d)   # a smaller mesh of the same material (profiling)
    nsteps = 100
    m0 = W.random_unit(spec.n, spec.seed)
    res = {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "data": "synthetic", "steps": args.steps, "warmup": args.warmup,
           "config": {"workload": "3D 512x512x64, 4 nm cubes: 1 demag + %d RK4 steps, FP32 vs split-BF16 / split-FP16" % nsteps,
                      "l2": "inputs larger than L2 (M 201 MB, spectra 1.2 GB)"}}
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(0)
    sampler.start()
    H = {}
    precs = (("fp32", gbdemag.GBD_FP32), ("split_bf16", gbdemag.GBD_SPLIT_BF16), ("split_fp16", gbdemag.GBD_SPLIT_FP16))
    precs = tuple(p for p in precs if p[0] in args.precisions.split(","))
    for name, prec in precs:
        mesh = gbdemag.Mesh(spec.n, spec.cell, spec.Ms, A_ex=spec.A_ex, alpha=spec.alpha, precision=prec)
        mesh.autotune()
        M = torch.from_numpy(spec.Ms * m0).cuda()
        Hd = torch.empty_like(M)
        for _ in range(args.warmup):
            mesh.demag(M, Hd)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            mesh.demag(M, Hd)
        e1.record(stream)
        torch.cuda.synchronize()
        t_demag = e0.elapsed_time(e1) / 1e3 / args.steps
        # per-pass device time of one evaluation (events around every launch) against the
        # algorithmic bytes of each pass
        gbdemag.gbd_mesh_set_timing(mesh.handle, True)
        mesh.demag(M, Hd)
        torch.cuda.synchronize()
        passes = gbdemag.gbd_mesh_read_timing(mesh.handle)
        gbdemag.gbd_mesh_set_timing(mesh.handle, False)
        dims = gbdemag.gbd_plan_dims(mesh.desc)
        bpp = bytes_per_pass_3d(spec.n, dims)
        peak, _ = measured_peaks()
        pass_info = {k: {"us": round(v[0] / v[1] * 1e3, 1), "algorithmic_MB": round(bpp[k] / 1e6, 1),
                         "GBps": round(bpp[k] / (v[0] / v[1] * 1e-3) / 1e9, 1),
                         "frac_of_hbm": round(bpp[k] / (v[0] / v[1] * 1e-3) / 1e9 / peak, 3)}
                     for k, v in passes.items() if k in bpp}
        H[name] = Hd.cpu().numpy()
        m = torch.from_numpy(m0).cuda()
        mesh.llg_step(m, 2, spec.dt)
        m = torch.from_numpy(m0).cuda()
        e0.record(stream)
        mesh.llg_step(m, nsteps, spec.dt)
        e1.record(stream)
        torch.cuda.synchronize()
        t_llg = e0.elapsed_time(e1) / 1e3
        res[name] = {"demag_ms": round(t_demag * 1e3, 3), "demag_gcell_per_s": round(spec.cells / t_demag / 1e9, 3),
                     "llg_100_steps_s": round(t_llg, 4),
                     "llg_gcell_demag_per_s": round(spec.cells * 4 * nsteps / t_llg / 1e9, 3),
                     "tuning": list(gbdemag.gbd_mesh_get_tuning(mesh.handle)), "passes": pass_info}
        res[name + "_m_after_100"] = m.cpu().numpy()
        mesh.close()
    res["clocks"] = sampler.stop()
    m32 = res.pop("fp32_m_after_100", None)
    for name, _ in precs:
        if name != "fp32" and m32 is not None:
            res[name]["m_after_100_max_abs_vs_fp32"] = float(np.abs(res.pop(name + "_m_after_100") - m32).max())
    res["value"] = res[precs[0][0]]["llg_gcell_demag_per_s"]
    res["dtype"] = "f32"
    if args.oracle_3d:
        from oracle import conv as C
        from oracle import tensor as T
        t0 = time.perf_counter()
        Href = C.fft_conv((spec.Ms * m0).astype(np.float64), T.tensor_all_offsets(spec.n, spec.cell))
        nrm = np.sqrt((Href ** 2).sum(0)).max()
        for name, _ in precs:
            res[name]["demag_e_inf_vs_fp64_oracle"] = float(np.sqrt(((H[name] - Href) ** 2).sum(0)).max() / nrm)
        res["oracle_s"] = round(time.perf_counter() - t0, 1)
    # RK4 steps against the FP64 oracle on a 64 x 64 x 8 mesh of the same material
    from oracle import llg as L
    from oracle import tensor as T
    small = (64, 64, 8)
    csteps = args.check_steps
    ms0 = W.random_unit(small, spec.seed)
    Nf = T.tensor_all_offsets(small, spec.cell)
    want = L.llg_run(ms0.astype(np.float64), csteps, spec.dt, Nf, spec.cell, spec.Ms, spec.A_ex, spec.alpha)
    for name, prec in precs:
        mesh = gbdemag.Mesh(small, spec.cell, spec.Ms, A_ex=spec.A_ex, alpha=spec.alpha, precision=prec)
        m = torch.from_numpy(ms0).cuda()
        mesh.llg_step(m, csteps, spec.dt)
        got = m.cpu().numpy().astype(np.float64)
        res[name]["llg_%d_steps_64x64x8_max_abs_vs_fp64_oracle" % csteps] = float(np.abs(got - want).max())
        mesh.close()
    return res


def run_cufft(args):
    """Film 1024 x 1024 x 1: one demag evaluation by this library (gbd_demag) beside the same
    zero-padded convolution written with torch.fft (cuFFT R2C / C2R and torch elementwise ops
    for the kernel product), both timed back to back with CUDA events on one stream. cuFFT is a
    comparison only; it is never on the library's path."""
    import numpy as np
    import torch

    from paper_2308_08447_gb300 import gbdemag
    from paper_2308_08447_gb300 import workloads as W

    torch.cuda.set_device(0)
    gbdemag.load()
    spec = W.thin_film()
    nx, ny, nz = spec.n
    mesh = gbdemag.Mesh(spec.n, spec.cell, spec.Ms, A_ex=spec.A_ex, alpha=spec.alpha)
    mesh.autotune()
    M = torch.from_numpy(spec.Ms * W.vortex_noise(spec.n, spec.cell, spec.seed)).cuda()
    H = torch.empty_like(M)
    stream = torch.cuda.current_stream()
    reps = 200

    def timed(fn):
        for _ in range(max(args.warmup, 3)):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e3 / reps

    t_ours = timed(lambda: mesh.demag(M, H))
    H_ours = H.clone()
    # full (Py, Hx) kernel from the library's FP64 packed spectrum; rows ky > Py/2 mirror, with
    # the sign flip of N_xy (odd in y). The stored spectrum carries -1/(Px Py); torch's inverse
    # divides by Px Py itself, so the product uses Px Py times the stored values.
    Px, Py, Pz, Hx, Ky, Kz = gbdemag.gbd_plan_dims(mesh.desc)
    ks = gbdemag.gbd_kernel_spectrum_host(mesh.desc)[:4, 0] * (Px * Py)     # (4, Ky, Hx)
    rows = np.concatenate([np.arange(Ky), Py - np.arange(Ky, Py)])
    sign = np.where(np.arange(Py) < Ky, 1.0, -1.0)[:, None]
    kf = ks[:, rows, :]
    kf[3] *= sign
    Kt = torch.from_numpy(kf.astype(np.float32)).cuda()
    Mp = M[:, 0]

    def cufft_demag():
        X = torch.fft.rfft2(Mp, s=(Py, Px))
        Y = torch.stack([Kt[0] * X[0] + Kt[3] * X[1], Kt[3] * X[0] + Kt[1] * X[1], Kt[2] * X[2]])
        return torch.fft.irfft2(Y, s=(Py, Px))[:, :ny, :nx]

    t_cufft = timed(cufft_demag)
    H_cufft = cufft_demag().unsqueeze(1)
    d = (H_cufft - H_ours).double()
    e = float(d.pow(2).sum(0).sqrt().max() / H_ours.double().pow(2).sum(0).sqrt().max())
    mesh.close()
    return {"metric": METRIC, "value": round(spec.cells / t_ours / 1e3, 3), "unit": UNIT, "n_gpus": 1,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "steps": reps, "warmup": max(args.warmup, 3),
            "config": {"workload": "thin film 1024x1024x1 demag evaluation: this library vs torch.fft (cuFFT)",
                       "l2": "not flushed (back-to-back evaluations, as inside a time loop)"},
            "ours_demag_us": round(t_ours, 2), "cufft_demag_us": round(t_cufft, 2),
            "cufft_gcell_demag_per_s": round(spec.cells / t_cufft / 1e3, 3),
            "speedup_vs_cufft": round(t_cufft / t_ours, 3), "e_inf_ours_vs_cufft": e}


def run_switching(args):
    """The switching problem of Fig. 2 (Sec. II), 480 x 240 x 2 cells of 5 nm: S state by the
    stated relax protocol, then 1 ns under H = (-20, 1, 0) kA/m with <m> recorded every 10 ps,
    at several time steps, exact and with the demag extrapolated at RK4 sub-steps. The error of
    each run is the paper's mean relative error eps = sum_i |M(t_i) - M_ref(t_i)| / (n Ms)
    against the 25 fs exact run (all FP32 on this GPU); throughput is taken on the 100 fs run."""
    import numpy as np
    import torch

    from paper_2308_08447_gb300 import gbdemag
    from paper_2308_08447_gb300 import workloads as W

    from oracle import llg as L   # the paper's error measure eps (pinned oracle function)

    torch.cuda.set_device(0)
    gbdemag.load()
    spec = W.switching()
    meta = spec.meta
    mesh = gbdemag.Mesh(spec.n, spec.cell, spec.Ms, A_ex=spec.A_ex, alpha=meta["relax_alpha"])
    mesh.autotune()
    stream = torch.cuda.current_stream()
    m = torch.from_numpy(W.uniform(spec.n, meta["m_init"])).cuda()
    t0 = time.perf_counter()
    dt_relax = 1e-13
    for h in meta["relax_fields"]:
        mesh.set_params(Hext=tuple(h * c for c in meta["relax_dir"]), alpha=meta["relax_alpha"])
        mesh.llg_step(m, int(round(meta["relax_hold"] / dt_relax)), dt_relax)
    torch.cuda.synchronize()
    relax_s = time.perf_counter() - t0
    mS = m.clone()
    mesh.set_params(Hext=spec.Hext, alpha=spec.alpha)
    interval, t_end = 10e-12, meta["t_switch"]
    n_rec = int(round(t_end / interval))

    def run(dt, extrap):
        mm = mS.clone()
        per = int(round(interval / dt))
        rec = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(n_rec):
            mesh.llg_step(mm, per, dt, extrap=extrap, cont=extrap and i > 0)
            rec.append(mm.mean(dim=(1, 2, 3)))
        e1.record(stream)
        torch.cuda.synchronize()
        return torch.stack(rec).double().cpu().numpy(), e0.elapsed_time(e1) / 1e3, per * n_rec

    def run_rkf(tol, extrap=False, host_loop=False):
        # host_loop: per-launch timing on, which makes gbd_llg_run_rkf56 take its host-driven loop
        # (a stream wait per attempt) instead of the device-controlled graph loop
        mm = mS.clone()
        rec, dt, acc, rej = [], 100e-15, 0, 0
        if host_loop:
            gbdemag.gbd_mesh_set_timing(mesh.handle, True)
        t0 = time.perf_counter()
        for i in range(n_rec):
            dt, a_, r_ = mesh.run_rkf56(mm, interval, dt, tol, extrap=extrap, cont=extrap and i > 0)
            acc, rej = acc + a_, rej + r_
            rec.append(mm.mean(dim=(1, 2, 3)))
            if host_loop:
                gbdemag.gbd_mesh_read_timing(mesh.handle)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        if host_loop:
            gbdemag.gbd_mesh_set_timing(mesh.handle, False)
        return torch.stack(rec).double().cpu().numpy(), secs, acc, rej

    ref, _, _ = run(25e-15, False)
    scaling = {}
    timing = {}
    for dt in (400e-15, 200e-15, 100e-15, 50e-15):
        row = {}
        for extrap in (False, True):
            traj, secs, steps = run(dt, extrap)
            row["extrap" if extrap else "exact"] = float(L.trajectory_error(traj, ref, 1.0))
            timing[(dt, extrap)] = (secs, steps)
        scaling["%g fs" % (dt * 1e15)] = row
    adaptive = {}
    for tol in (1e-4, 1e-5):
        for extrap in (False, True):
            traj, secs_a, acc, rej = run_rkf(tol, extrap)
            row = {"eps": float(L.trajectory_error(traj, ref, 1.0)), "accepted": acc, "rejected": rej,
                   "mean_step_fs": round(t_end / acc * 1e15, 1), "s": round(secs_a, 3)}
            if not extrap:
                _, secs_h, acc_h, rej_h = run_rkf(tol, False, host_loop=True)
                row["s_host_driven_loop"] = round(secs_h, 3)
                row["host_loop_steps"] = [acc_h, rej_h]
            adaptive["tol %g%s" % (tol, ", quintic demag extrapolation" if extrap else "")] = row
    secs, steps = timing[(100e-15, False)]
    xsecs, xsteps = timing[(100e-15, True)]
    mesh.close()
    fp64_study = switching_fp64_study()
    samples = {"%g ns" % (t * 1e9): [round(float(v), 5) for v in ref[int(round(t / interval)) - 1]]
               for t in (0.1e-9, 0.25e-9, 0.5e-9, 0.75e-9, 1e-9)}
    return {"metric": METRIC, "value": round(spec.cells * 4 * steps / secs / 1e9, 3), "unit": UNIT,
            "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "switching problem of the time-step study: 480x240x2 cells of 5 nm, Ms 800 kA/m, "
                                   "S state relaxed, then 1 ns at H = (-20, 1, 0) kA/m", "cells": spec.cells,
                       "l2": "not flushed (1 ns of dynamics per run)"},
            "llg_steps_per_s": round(steps / secs, 1), "llg_steps_per_s_extrap": round(xsteps / xsecs, 1),
            "relax_s": round(relax_s, 2),
            "eps_vs_25fs_exact": scaling, "adaptive_rkf56": adaptive, "mean_m_25fs_exact": samples,
            "eps_vs_fp64_oracle_96x48x2": fp64_study}


def switching_fp64_study(dts=(400e-15, 200e-15, 100e-15, 50e-15, 25e-15)):
    """The time-step study of Fig. 2 (Sec. II) against a double-precision reference: the switching
    problem on the film reduced to 96 x 48 x 2 cells (same 5 nm cells and protocol), from the S
    state the FP64 oracle relaxed, 1 ns under the switching field, <m> every 10 ps. The FP32 GPU
    runs at each dt (exact and with the demag extrapolated at RK4 sub-steps) are compared with
    the oracle's FP64 RK4 trajectory at 50 fs (both stored under tests/golden by
    make_switching_reference.py) by the paper's mean error eps (oracle.llg.trajectory_error)."""
    import numpy as np
    import torch

    from oracle import llg as L
    from paper_2308_08447_gb300 import gbdemag
    from paper_2308_08447_gb300 import workloads as W

    gold = os.path.join(ROOT, "tests", "golden")
    m_s = np.load(os.path.join(gold, "switching_96x48x2_S_state.npy"))
    ref = np.loadtxt(os.path.join(gold, "switching_96x48x2_fp64_traj.txt"))
    spec = W.switching(scale=5)
    mesh = gbdemag.Mesh(spec.n, spec.cell, spec.Ms, A_ex=spec.A_ex, alpha=spec.alpha, Hext=spec.Hext)
    interval, n_rec = 10e-12, len(ref)
    out = {"reference": "FP64 oracle RK4 at 50 fs (its own eps against the 100 fs FP64 run: 1.1e-10)",
           "mesh": "96x48x2 cells of 5 nm", "samples": n_rec}
    for dt in dts:
        row = {}
        for extrap in (False, True):
            m = torch.from_numpy(m_s).cuda()
            per = int(round(interval / dt))
            rec = []
            for i in range(n_rec):
                mesh.llg_step(m, per, dt, extrap=extrap, cont=extrap and i > 0)
                rec.append(m.double().mean(dim=(1, 2, 3)))
            traj = torch.stack(rec).cpu().numpy()
            row["extrap" if extrap else "exact"] = float(L.trajectory_error(traj, ref, 1.0))
        out["%g fs" % (dt * 1e15)] = row
    mesh.close()
    return out


def run_extras(args):
    """The rest of the metric beside the film headline, each with its own clock record: the 3D
    mesh (FP32 and both split precisions, error against the FP64 oracle, per-pass rooflines),
    the 64-mesh batch against the plain path, and a short served trace against the plain path."""
    import copy
    out = {}
    a = copy.copy(args)
    a.steps, a.warmup, a.oracle_3d, a.check_steps = 5, 2, True, 20
    r = run_3d(a)
    out["3d"] = {k: r[k] for k in ("config", "fp32", "split_bf16", "split_fp16", "oracle_s", "clocks") if k in r}
    a = copy.copy(args)
    a.steps, a.warmup, a.llg_steps = 2, 2, 100
    r = run_batch(a)
    out["batch"] = {k: r[k] for k in ("value", "unit", "ms_per_step", "config", "plain_path", "speedup_vs_plain",
                                      "results_bit_identical", "padded_volume_vs_pow2", "clocks") if k in r}
    a = copy.copy(args)
    r = run_serve(a)
    out["served"] = {k: r[k] for k in ("value", "unit", "config", "served", "plain_path", "results_bit_identical",
                                       "max_active", "iterations", "clocks") if k in r}
    return out


def run_reference(args):
    rank, world, local = _dist_env()
    if rank != 0:
        return None
    from paper_2308_08447_gb300 import workloads as W
    spec = W.thin_film()
    m0 = W.vortex_noise(spec.n, spec.cell, spec.seed)
    Nf = oracle_tensor(spec)   # set-up, untimed; the oracle has no warm-up state
    vals = []
    cb = None
    for _ in range(args.steps):
        cb = cpu_baseline(spec, m0, Nf=Nf)
        vals.append(cb["value"])
    value = statistics.mean(vals)
    cb["value"] = value
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "thin film 1024x1024x1, 2x2x3 nm cells, demag + exchange + LLG RK4; "
                                   "each step one RK4 step (4 demag evaluations) of the FP64 CPU oracle"},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--llg-steps", type=int, default=1000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extrap", action="store_true", help="skip the demag-extrapolation run of the film")
    ap.add_argument("--workload", default="film", choices=["film", "batch", "serve", "3d", "cufft", "switching"])
    ap.add_argument("--oracle-3d", action="store_true", help="3d: FP64 oracle of the full mesh (minutes, ~30 GB)")
    ap.add_argument("--check-steps", type=int, default=100, help="3d: RK4 steps of the 64x64x8 check against the oracle")
    ap.add_argument("--n3d", type=int, nargs=3, default=None, help="3d: mesh size (default 512 512 64)")
    ap.add_argument("--precisions", default="fp32,split_bf16,split_fp16", help="3d: which precisions to run")
    ap.add_argument("--quick", action="store_true", help="film line only (no 3D / batch / served keys)")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--pow2-pad", action="store_true", help="batch: power-of-two padded lengths only")
    ap.add_argument("--requests", type=int, default=48)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--chunk", type=int, default=50)
    ap.add_argument("--max-active", type=int, default=8, help="served jobs per iteration (0: no cap)")
    ap.add_argument("--rho", type=float, default=0.0,
                    help="serve: also run the trace at this load factor of the plain path's service rate")
    ap.add_argument("--extrap", action="store_true",
                    help="serve: demag extrapolated at RK4 sub-steps on the served and the plain path")
    args = ap.parse_args()
    if args.impl == "reference":
        res = run_reference(args)
    elif args.workload == "batch":
        res = run_batch(args)
    elif args.workload == "serve":
        res = run_serve(args)
    elif args.workload == "3d":
        res = run_3d(args)
    elif args.workload == "cufft":
        res = run_cufft(args)
    elif args.workload == "switching":
        res = run_switching(args)
    else:
        res = run_ours(args)
        if res is not None and res["n_gpus"] == 1 and not args.quick:
            res.update(run_extras(args))
    if res is not None:
        print(json.dumps(res))


if __name__ == "__main__":
    main()
