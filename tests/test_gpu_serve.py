"""The served pattern on the GPU: jobs admitted over time and batched per iteration give, for
every job, exactly the result of running that job alone on the plain path."""
import numpy as np
import pytest

from gpu_util import lib
from paper_2308_08447_gb300 import serve
from paper_2308_08447_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_served_results_equal_plain_results():
    lib()
    specs = [((64, 64, 1), 45, 0.0), ((96, 64, 2), 70, 0.0), ((32, 128, 4), 33, 0.02),
             ((128, 96, 1), 58, 0.04), ((64, 32, 8), 21, 0.05), ((160, 64, 1), 40, 0.3)]
    jobs = []
    for i, (n, steps, arrival) in enumerate(specs):
        cell = (3e-9, 3e-9, 3e-9)
        spec = W.MeshSpec(n=n, cell=cell, Ms=8e5, A_ex=1.3e-11, alpha=0.5,
                          dt=W.stable_dt(cell, 8e5, 1.3e-11), steps=steps, seed=900 + i)
        jobs.append(serve.Job(id=i, spec=spec, arrival=arrival))
    ex = serve.GpuExecutor(autotune=True)
    ex.prewarm(jobs)
    budget = sum(ex.bytes_for(j) for j in jobs[:3])       # not everything fits at once
    srv = serve.Server(ex, budget, chunk=16)
    served = srv.run([serve.Job(j.id, j.spec, j.arrival) for j in jobs])
    ex.close()
    assert all(used <= budget for _, _, used in srv.trace)
    plain = serve.run_plain(ex, [serve.Job(j.id, j.spec, j.arrival) for j in jobs])
    by_id = {j.id: j for j in plain}
    for j in served:
        assert np.array_equal(j.result, by_id[j.id].result), j.id
        assert np.isfinite(j.result).all()
    s = serve.summarize(served)
    assert s["jobs"] == len(jobs) and s["p99_s"] >= s["p50_s"] > 0


def test_served_extrapolated_results_equal_plain_results():
    # with the demag extrapolated at RK4 sub-steps, each job's history continues across its
    # chunks (GBD_STEP_CONTINUE) and the result equals the job alone in one call
    lib()
    specs = [((64, 64, 1), 47, 0.0), ((96, 64, 2), 30, 0.0), ((32, 128, 4), 26, 0.02), ((128, 96, 1), 12, 0.03)]
    jobs = []
    for i, (n, steps, arrival) in enumerate(specs):
        cell = (3e-9, 3e-9, 3e-9)
        spec = W.MeshSpec(n=n, cell=cell, Ms=8e5, A_ex=1.3e-11, alpha=0.5,
                          dt=W.stable_dt(cell, 8e5, 1.3e-11), steps=steps, seed=950 + i)
        jobs.append(serve.Job(id=i, spec=spec, arrival=arrival))
    ex = serve.GpuExecutor(autotune=False, extrap=True)
    srv = serve.Server(ex, 1 << 40, chunk=10)
    served = srv.run([serve.Job(j.id, j.spec, j.arrival) for j in jobs])
    ex.close()
    plain = serve.run_plain(ex, [serve.Job(j.id, j.spec, j.arrival) for j in jobs])
    by_id = {j.id: j for j in plain}
    for j in served:
        assert np.array_equal(j.result, by_id[j.id].result), j.id
    s = serve.summarize(served, extrap=True)
    assert s["gcell_steps_per_s"] > 0 and s["gcell_demag_per_s"] < 4 * s["gcell_steps_per_s"]
