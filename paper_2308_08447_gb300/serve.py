"""Continuous-batching server for LLG relaxation / field jobs on one GPU.

Requests arrive over time (a trace of arrival times). The scheduler keeps every admitted job's
state (mesh buffers, kernel spectrum, magnetization) resident on the device and advances all
active jobs together: each iteration runs up to `chunk` RK4 steps of every active job in one
batched CUDA-graph launch (gbd_batch_run), then retires finished jobs and frees their memory.
Jobs that arrive while others are running wait until the next iteration boundary and are
admitted, in arrival order, as soon as the device-memory budget allows (a waiting job that
fits may pass one that does not). Per-job latency is finish time minus arrival time.

The "plain path" runs the same trace one job at a time in arrival order with gbd_llg_step.

The executor interface separates the scheduling logic (tested on the CPU with a fake
executor) from the GPU work (GpuExecutor, every step in the library's kernels).
"""
import argparse
import json
import os
import sys
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Job:
    id: int
    spec: object                 # workloads.MeshSpec (n, cell, Ms, A_ex, alpha, dt, steps, seed, meta)
    arrival: float               # seconds after trace start
    remaining: int = 0
    admitted: float = None
    finished: float = None
    handle: object = None        # executor-owned state
    result: object = None

    @property
    def latency(self):
        return None if self.finished is None else self.finished - self.arrival


class Server:
    """Admission by memory budget, per-iteration batching of all active jobs, retirement."""

    def __init__(self, executor, budget_bytes, chunk=50, max_active=None, clock=time.perf_counter,
                 sleep=time.sleep):
        self.ex = executor
        self.budget = int(budget_bytes)
        self.chunk = int(chunk)
        # at most this many jobs share an iteration (None: as many as the budget admits);
        # a cap keeps early jobs from being slowed by every later arrival
        self.max_active = max_active
        self.clock = clock
        self.sleep = sleep
        self.used = 0
        self.trace = []              # (t, active, used bytes) per iteration

    def run(self, jobs):
        jobs = sorted(jobs, key=lambda j: (j.arrival, j.id))
        for j in jobs:
            if self.ex.bytes_for(j) > self.budget:
                raise ValueError("job %d needs more than the whole budget" % j.id)
            j.remaining = j.spec.steps
        pending = list(jobs)          # not yet arrived
        waiting = []                  # arrived, not admitted
        active = []
        done = []
        t0 = self.clock()
        while pending or waiting or active:
            now = self.clock() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.pop(0))
            # admit in arrival order whatever fits
            still = []
            for j in waiting:
                b = self.ex.bytes_for(j)
                full = self.max_active is not None and len(active) >= self.max_active
                if not full and self.used + b <= self.budget:
                    self.ex.admit(j)
                    self.used += b
                    j.admitted = self.clock() - t0
                    active.append(j)
                else:
                    still.append(j)
            waiting = still
            if not active:
                if pending:
                    self.sleep(max(0.0, pending[0].arrival - (self.clock() - t0)))
                continue
            steps = [min(j.remaining, self.chunk) for j in active]
            self.ex.run_iteration(active, steps)
            self.trace.append((self.clock() - t0, len(active), self.used))
            for j, s in zip(active, steps):
                j.remaining -= s
            finished = [j for j in active if j.remaining == 0]
            active = [j for j in active if j.remaining > 0]
            if finished:
                self.ex.sync()
                tf = self.clock() - t0
                for j in finished:
                    self.ex.retire(j)
                    self.used -= self.ex.bytes_for(j)
                    j.finished = tf
                    done.append(j)
        return done


def run_plain(executor, jobs, clock=time.perf_counter, sleep=time.sleep):
    """Each job alone, in arrival order, all its steps in one gbd_llg_step call."""
    jobs = sorted(jobs, key=lambda j: (j.arrival, j.id))
    t0 = clock()
    for j in jobs:
        now = clock() - t0
        if j.arrival > now:
            sleep(j.arrival - now)
        executor.admit(j)
        j.admitted = clock() - t0
        executor.run_alone(j)
        executor.sync()
        j.finished = clock() - t0
        executor.retire(j)
    return jobs


def demag_evals(steps, extrap):
    """Demag evaluations of a run of `steps` RK4 steps: 4 per step, or with the demag
    extrapolated at sub-steps 4 per step for the first four steps and 1 per step after."""
    return 4 * steps if not extrap else 4 * min(steps, 4) + max(steps - 4, 0)


def summarize(jobs, extrap=False):
    lat = np.array([j.latency for j in jobs])
    cells = sum(j.spec.cells * demag_evals(j.spec.steps, extrap) for j in jobs)
    cell_steps = sum(j.spec.cells * j.spec.steps for j in jobs)
    makespan = max(j.finished for j in jobs) - min(j.arrival for j in jobs)
    return {"jobs": len(jobs), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "makespan_s": float(makespan),
            "gcell_demag_per_s": cells / makespan / 1e9, "gcell_steps_per_s": cell_steps / makespan / 1e9}


class GpuExecutor:
    """Jobs as library meshes on the current CUDA device; one gbd_batch per iteration."""

    def __init__(self, autotune=True, extrap=False):
        import torch
        from . import gbdemag
        self.torch = torch
        self.g = gbdemag
        self.g.load()
        self.autotune = autotune
        # demag extrapolated at RK4 sub-steps (GBD_STEP_EXTRAP), continued across a job's chunks
        self.extrap = extrap
        self._started = set()
        self._bytes = {}

    def bytes_for(self, job):
        key = (tuple(job.spec.n), tuple(job.spec.cell))
        if key not in self._bytes:
            desc = self.g.make_desc(job.spec.n, job.spec.cell, job.spec.Ms)
            # mesh buffers + the state tensor the server keeps for the job
            self._bytes[key] = self.g.gbd_mesh_bytes(desc) + 12 * job.spec.cells
        return self._bytes[key]

    def prewarm(self, jobs):
        """Kernel spectra of every geometry in the trace into the library's host cache
        (the per-geometry set-up, like loading a model, before the served clock starts)."""
        seen = set()
        for j in jobs:
            key = (tuple(j.spec.n), tuple(j.spec.cell))
            if key in seen:
                continue
            seen.add(key)
            mesh = self.g.Mesh(j.spec.n, j.spec.cell, j.spec.Ms)
            if self.autotune:
                mesh.autotune()
            mesh.close()

    def admit(self, job):
        from . import workloads as W
        s = job.spec
        mesh = self.g.Mesh(s.n, s.cell, s.Ms, A_ex=s.A_ex, alpha=s.alpha, Hext=s.Hext)
        if self.autotune:
            mesh.autotune()
        m = self.torch.from_numpy(W.random_unit(s.n, s.seed)).cuda()
        job.handle = (mesh, m)

    def run_iteration(self, jobs, steps):
        # one batch per distinct active set; while the set and the step counts repeat, the
        # library relaunches the cached graph
        key = tuple(j.id for j in jobs)
        if getattr(self, "_batch_key", None) != key:
            if getattr(self, "_batch", None) is not None:
                self._batch.close()          # synchronizes: the previous graph has finished
            self._batch = self.g.Batch([j.handle[0] for j in jobs])
            self._batch_key = key
        flags = None
        if self.extrap:
            flags = [self.g.GBD_STEP_EXTRAP | (self.g.GBD_STEP_CONTINUE if j.id in self._started else 0)
                     for j in jobs]
            self._started.update(j.id for j in jobs)
        self._batch.run([j.handle[1] for j in jobs], steps, [j.spec.dt for j in jobs], flags=flags)

    def run_alone(self, job):
        mesh, m = job.handle
        mesh.llg_step(m, job.spec.steps, job.spec.dt, extrap=self.extrap)

    def sync(self):
        self.torch.cuda.synchronize()

    def close(self):
        if getattr(self, "_batch", None) is not None:
            self._batch.close()
            self._batch = None
            self._batch_key = None

    def retire(self, job):
        mesh, m = job.handle
        job.result = m.cpu().numpy()
        mesh.close()
        job.handle = None


def make_jobs(count, rate, seed, max_side=1024, max_nz=16):
    from . import workloads as W
    reqs = W.served_requests(count=count, rate=rate, seed=seed, max_side=max_side, max_nz=max_nz)
    return [Job(id=i, spec=r, arrival=r.meta["arrival"]) for i, r in enumerate(reqs)]


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--requests", type=int, default=48)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--chunk", type=int, default=50)
    ap.add_argument("--max-active", type=int, default=8)
    ap.add_argument("--max-side", type=int, default=1024)
    args = ap.parse_args(argv)
    os.environ.setdefault("GBD_KERNEL_CACHE_BYTES", str(64 << 30))
    ex = GpuExecutor()
    jobs = make_jobs(args.requests, args.rate, args.seed, args.max_side)
    ex.prewarm(jobs)
    served = Server(ex, args.budget_gb * 1e9, chunk=args.chunk, max_active=args.max_active or None).run(
        [Job(j.id, j.spec, j.arrival) for j in jobs])
    ex.close()
    plain = run_plain(ex, [Job(j.id, j.spec, j.arrival) for j in jobs])
    same = all(np.array_equal(a.result, b.result) for a, b in
               zip(sorted(served, key=lambda j: j.id), sorted(plain, key=lambda j: j.id)))
    out = {"served": summarize(served), "plain": summarize(plain), "results_identical": bool(same),
           "requests": args.requests, "rate_per_s": args.rate, "chunk_steps": args.chunk,
           "budget_gb": args.budget_gb}
    print(json.dumps(out))
    return out


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    main()
