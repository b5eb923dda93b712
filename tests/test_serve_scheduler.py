"""The continuous-batching scheduler on the CPU, with a fake executor and a simulated clock.

Checks the host logic of the served pattern: admission by memory budget in arrival order,
jobs admitted while others are in flight, retirement freeing memory, per-iteration step
chunks, latencies, and the one-at-a-time plain path.
"""
import pytest

from paper_2308_08447_gb300.serve import Job, Server, run_plain, summarize
from paper_2308_08447_gb300.workloads import MeshSpec


class SimClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(0.0, dt)


class FakeExecutor:
    """bytes = 100 per cell; an iteration costs 1e-9 s per cell-step of every active job."""

    def __init__(self, clock):
        self.clock = clock
        self.admitted = []
        self.retired = []
        self.iterations = []

    def bytes_for(self, job):
        return 100 * job.spec.cells

    def admit(self, job):
        self.admitted.append(job.id)
        job.handle = 0

    def run_iteration(self, jobs, steps):
        self.iterations.append([(j.id, s) for j, s in zip(jobs, steps)])
        self.clock.t += sum(j.spec.cells * s for j, s in zip(jobs, steps)) * 1e-9
        for j, s in zip(jobs, steps):
            j.handle += s

    def run_alone(self, job):
        self.clock.t += job.spec.cells * job.spec.steps * 1e-9
        job.handle += job.spec.steps

    def sync(self):
        pass

    def retire(self, job):
        self.retired.append(job.id)
        job.result = job.handle


def _job(i, cells_side, steps, arrival):
    spec = MeshSpec(n=(cells_side, cells_side, 1), cell=(2e-9, 2e-9, 2e-9), steps=steps)
    return Job(id=i, spec=spec, arrival=arrival)


def test_all_jobs_complete_with_exact_steps():
    clk = SimClock()
    ex = FakeExecutor(clk)
    jobs = [_job(i, 100 + 10 * i, 120 + 37 * i, 0.001 * i) for i in range(8)]
    srv = Server(ex, budget_bytes=10 ** 9, chunk=50, clock=clk, sleep=clk.sleep)
    done = srv.run(jobs)
    assert sorted(j.id for j in done) == list(range(8))
    for j in done:
        assert j.result == j.spec.steps          # every step run exactly once
        assert j.finished >= j.arrival and j.latency > 0
    # every iteration advances each active job by at most the chunk
    assert all(s <= 50 for it in ex.iterations for _, s in it)


def test_budget_respected_and_late_jobs_join_in_flight():
    clk = SimClock()
    ex = FakeExecutor(clk)
    # two big jobs fill the budget; a third arrives later and must wait for memory;
    # a small fourth arrives while the first two run and fits at once
    jobs = [_job(0, 300, 400, 0.0), _job(1, 300, 100, 0.0), _job(2, 300, 50, 0.0001), _job(3, 50, 60, 0.00001)]
    budget = 2 * 100 * 300 * 300 + 100 * 50 * 50
    srv = Server(ex, budget_bytes=budget, chunk=20, clock=clk, sleep=clk.sleep)
    done = {j.id: j for j in srv.run(jobs)}
    assert all(used <= budget for _, _, used in srv.trace)
    # job 3 was admitted while job 0 was still running (continuous batching)
    assert done[3].admitted < done[0].finished
    assert done[3].admitted > 0.0
    # job 2 did not fit until job 1 retired
    assert done[2].admitted >= done[1].finished
    s = summarize(list(done.values()))
    assert s["p99_s"] >= s["p50_s"] > 0


def test_max_active_caps_concurrency_and_keeps_arrival_order():
    clk = SimClock()
    ex = FakeExecutor(clk)
    jobs = [_job(i, 100, 100 + 10 * i, 0.0) for i in range(6)]
    srv = Server(ex, budget_bytes=10 ** 12, chunk=25, max_active=2, clock=clk, sleep=clk.sleep)
    done = {j.id: j for j in srv.run(jobs)}
    assert max(a for _, a, _ in srv.trace) == 2
    assert ex.admitted == list(range(6))
    # the first two finish before the last two are even admitted
    assert done[1].finished <= done[4].admitted + 1e-12


def test_job_larger_than_budget_is_refused():
    clk = SimClock()
    srv = Server(FakeExecutor(clk), budget_bytes=1000, clock=clk, sleep=clk.sleep)
    with pytest.raises(ValueError):
        srv.run([_job(0, 100, 10, 0.0)])


def test_plain_path_runs_one_job_at_a_time():
    clk = SimClock()
    ex = FakeExecutor(clk)
    jobs = [_job(i, 200, 100, 0.0) for i in range(4)]
    done = run_plain(ex, jobs)
    fin = sorted(j.finished for j in done)
    assert all(b > a for a, b in zip(fin, fin[1:]))
    assert [j.result for j in done] == [100] * 4
