"""Mesh creation and destruction do not stall other work on the device (GPU).

Mesh buffers come from the device's stream-ordered memory pool; gbd_mesh_destroy orders the frees
after the mesh's own recorded work and returns at once, so a server retiring one job leaves the
others running. Checked: a mesh created, used and destroyed on one stream while a long run of
another mesh is in flight on a second stream returns before that run ends, and the run's result is
the same as alone; a mesh destroyed with its own work still queued finishes that work without
error and gives its memory back.
"""
import numpy as np
import pytest

from gpu_util import lib, to_dev, to_host
from paper_2308_08447_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    return lib()


def test_destroy_leaves_other_streams_running(g):
    import torch
    spec = W.thin_film()
    big = g.Mesh(spec.n, spec.cell, spec.Ms, A_ex=spec.A_ex, alpha=spec.alpha)
    m0 = W.vortex_noise(spec.n, spec.cell, spec.seed)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    m = to_dev(m0)
    torch.cuda.synchronize()
    with torch.cuda.stream(s1):
        big.llg_step(m, 300, spec.dt, stream=s1)       # tens of milliseconds of work
        done = torch.cuda.Event()
        done.record(s1)
    with torch.cuda.stream(s2):
        n = (64, 64, 1)
        small = g.Mesh(n, (2e-9, 2e-9, 3e-9), 8e5, stream=s2)
        M = to_dev(8e5 * W.random_unit(n, 81))
        H = torch.empty_like(M)
        small.demag(M, H, stream=s2)
        small.close()                                   # must not wait for s1
    still_running = not done.query()
    torch.cuda.synchronize()
    assert still_running
    ref = to_dev(m0)
    big.llg_step(ref, 300, spec.dt)
    assert np.array_equal(to_host(m), to_host(ref))
    big.close()


def test_destroy_with_own_work_queued(g):
    import torch
    n, cell = (256, 256, 4), (3e-9, 3e-9, 3e-9)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    s = torch.cuda.Stream()
    mesh = g.Mesh(n, cell, 8e5, A_ex=1.3e-11, alpha=0.1, stream=s)
    m = to_dev(W.random_unit(n, 82))
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        mesh.llg_step(m, 40, 1e-13, stream=s)
        mesh.close()                                    # frees after the 40 steps, host does not wait
    torch.cuda.synchronize()
    assert np.isfinite(to_host(m)).all()
    assert np.allclose(np.sqrt((to_host(m) ** 2).sum(0)), 1.0, atol=1e-5)
    # the pool returns the memory at a synchronization
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= (64 << 20)
