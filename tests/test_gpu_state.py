"""Checkpoint / resume of the integrator state kept in the mesh (gbd_mesh_get_state /
gbd_mesh_set_state): an extrapolated RK4 run or an extrapolated RKF5(6) step sequence split by a
save into a fresh mesh equals the unsplit run bit for bit; malformed images are refused. Also the
per-launch tracing switch (CUDA events, NVTX ranges) leaves results unchanged."""
import numpy as np
import pytest

from gpu_util import lib, to_dev, to_host
from paper_2308_08447_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    return lib()


def test_rk4_extrapolated_run_resumes_bit_identically(g):
    n, cell = (64, 48, 2), (3e-9, 3e-9, 3e-9)
    m0 = W.random_unit(n, 41)
    args = dict(A_ex=1.3e-11, alpha=0.05)
    whole = g.Mesh(n, cell, 8e5, **args)
    a = to_dev(m0)
    whole.llg_step(a, 24, 1e-13, extrap=True)
    first = g.Mesh(n, cell, 8e5, **args)
    b = to_dev(m0)
    first.llg_step(b, 11, 1e-13, extrap=True)
    state = first.get_state()
    first.close()
    resumed = g.Mesh(n, cell, 8e5, **args)
    resumed.set_state(state)
    resumed.llg_step(b, 13, 1e-13, extrap=True, cont=True)
    assert np.array_equal(to_host(a), to_host(b))
    whole.close()
    resumed.close()


def test_rkf_extrapolated_steps_resume_bit_identically(g):
    n, cell = (48, 40, 1), (2e-9, 2e-9, 3e-9)
    m0 = W.random_unit(n, 42)
    args = dict(A_ex=1.3e-11, alpha=0.1)
    whole = g.Mesh(n, cell, 8.6e5, **args)
    a = to_dev(m0)
    for i in range(12):
        whole.rkf56_step(a, 5e-14, extrap=True, cont=i > 0)
    first = g.Mesh(n, cell, 8.6e5, **args)
    b = to_dev(m0)
    for i in range(7):
        first.rkf56_step(b, 5e-14, extrap=True, cont=i > 0)
    state = first.get_state()
    first.close()
    resumed = g.Mesh(n, cell, 8.6e5, **args)
    resumed.set_state(state)
    for i in range(5):
        resumed.rkf56_step(b, 5e-14, extrap=True, cont=True)
    assert np.array_equal(to_host(a), to_host(b))
    whole.close()
    resumed.close()


def test_malformed_state_refused(g):
    mesh = g.Mesh((32, 32, 1), (2e-9, 2e-9, 3e-9), 8e5, A_ex=1.3e-11, alpha=0.1)
    m = to_dev(W.random_unit((32, 32, 1), 43))
    mesh.llg_step(m, 6, 1e-13, extrap=True)
    state = mesh.get_state()
    other = g.Mesh((16, 32, 1), (2e-9, 2e-9, 3e-9), 8e5)
    for bad in (state[:-4], b"x" * len(state)):
        with pytest.raises(g.GbdError) as ei:
            mesh.set_state(bad)
        assert ei.value.status == g.GBD_EINVAL
    with pytest.raises(g.GbdError) as ei:          # another cell count
        other.set_state(state)
    assert ei.value.status == g.GBD_EINVAL
    # the same cell count in another shape (transposed, or split over z) has another slot layout
    for shape in ((16, 64, 1), (32, 16, 2)):
        same_n = g.Mesh(shape, (2e-9, 2e-9, 3e-9), 8e5, A_ex=1.3e-11, alpha=0.1)
        with pytest.raises(g.GbdError) as ei:
            same_n.set_state(state)
        assert ei.value.status == g.GBD_EINVAL
        same_n.close()
    mesh.set_state(state)                            # the intact image still loads
    other.close()
    mesh.close()


def test_nvtx_tracing_leaves_results_and_event_timing_alone(g):
    # GBD_TIMING_NVTX wraps each launch in an NVTX range; alone it records no events, and the
    # field is the same as untraced
    import torch
    n, cell = (64, 32, 4), (3e-9, 3e-9, 3e-9)
    M = to_dev(8e5 * W.random_unit(n, 44))
    mesh = g.Mesh(n, cell, 8e5)
    H0, H1 = torch.empty_like(M), torch.empty_like(M)
    mesh.demag(M, H0)
    g.gbd_mesh_set_timing(mesh.handle, g.GBD_TIMING_NVTX)
    mesh.demag(M, H1)
    assert sum(c for _, c in g.gbd_mesh_read_timing(mesh.handle).values()) == 0
    g.gbd_mesh_set_timing(mesh.handle, g.GBD_TIMING_NVTX | g.GBD_TIMING_EVENTS)
    mesh.demag(M, H1)
    assert sum(c for _, c in g.gbd_mesh_read_timing(mesh.handle).values()) == 5
    g.gbd_mesh_set_timing(mesh.handle, 0)
    assert np.array_equal(to_host(H0), to_host(H1))
    mesh.close()
