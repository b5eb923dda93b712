"""The bounded device-side wait of the RK-stage x-row kernel (GPU).

The RK stages of meshes with nx a multiple of 64 wait for bulk copies of their stage input
through an mbarrier, for at most 100 ms per block. The test hook GBD_TEST_WAIT_TIMEOUT=1 (read when
a mesh is created) makes the copies announce 16 bytes more than they deliver, so every such wait
runs out: the launches still finish, gbd_mesh_device_status reports GBD_ETIMEOUT once and clears
it, and the context stays usable -- a mesh created without the hook then runs the same steps with
status GBD_OK, and, since the copies did deliver their rows, the same result.
"""
import os

import numpy as np
import pytest

from gpu_util import lib, to_dev, to_host
from paper_2308_08447_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    return lib()


def test_wait_that_runs_out_is_reported(g):
    n, cell = (64, 64, 1), (2e-9, 2e-9, 3e-9)   # one 64-row block per RK stage launch
    m0 = W.vortex_noise(n, cell, 3)
    out = {}
    for hook in (True, False):
        os.environ["GBD_TEST_WAIT_TIMEOUT"] = "1" if hook else "0"
        try:
            mesh = g.Mesh(n, cell, 8.6e5, A_ex=1.3e-11, alpha=0.02)
        finally:
            os.environ.pop("GBD_TEST_WAIT_TIMEOUT", None)
        g.gbd_mesh_set_tuning(mesh.handle, (1, 0, 0, 0))
        m = to_dev(m0)
        mesh.llg_step(m, 1, 1e-13)
        out[hook] = (mesh.device_status(), mesh.device_status(), to_host(m))
        mesh.close()
    assert out[True][0] == g.GBD_ETIMEOUT and out[True][1] == g.GBD_OK
    assert out[False][0] == g.GBD_OK and out[False][1] == g.GBD_OK
    assert np.array_equal(out[True][2], out[False][2])
