"""Stream order with programmatic dependent launch (GPU).

The x-row, film-convolution and extrapolated-stage kernels are launched so that a launch may start
while the kernel before it runs; each waits for its predecessor before touching memory it may
write, and the RK-stage row kernel requests its stage input (written by the x-row launch before the
preceding convolution) ahead of that wait. Checked: work that another kernel does on the same
stream between library calls -- here a torch kernel that reverses m between two runs of RK4 steps,
exact and extrapolated -- is seen by the next call exactly as when the host waits for every
launch, and the tile variants (the staged RK stage of variant 1, the unstaged one of variant 0)
agree bit for bit along the way.
"""
import numpy as np
import pytest

from gpu_util import lib, to_dev, to_host
from paper_2308_08447_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    return lib()


@pytest.mark.parametrize("extrap", [False, True])
def test_writes_between_calls_are_seen(g, extrap):
    import torch
    n, cell = (256, 128, 1), (2e-9, 2e-9, 3e-9)
    m0 = W.vortex_noise(n, cell, 5)
    out = {}
    for var in (0, 1):
        for sync in (False, True):
            mesh = g.Mesh(n, cell, 8.6e5, A_ex=1.3e-11, alpha=0.02)
            g.gbd_mesh_set_tuning(mesh.handle, (var, 0, 0, 0))
            m = to_dev(m0)
            for _ in range(3):
                mesh.llg_step(m, 6, 1e-13, extrap=extrap)
                if sync:
                    torch.cuda.synchronize()
                m.mul_(-1.0)                     # a torch kernel on the same stream rewrites m
                if sync:
                    torch.cuda.synchronize()
            torch.cuda.synchronize()
            out[(var, sync)] = to_host(m)
            mesh.close()
    ref = out[(0, True)]
    assert np.all(np.isfinite(ref))
    for key, v in out.items():
        assert np.array_equal(v, ref), key
