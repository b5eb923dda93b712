"""Periodic boundary conditions on the GPU (GBD_FLAG_PBC_*) against the oracle's reading
(oracle/pbc.py): the demag field, H_eff with the wrapping exchange, RK4 steps, and the circular
shift covariance along periodic axes. Meshes cover periodic x (no zero half in the x
transform), periodic y on the film path, periodic z on the 3D path, and all three, and RK steps
on a mesh whose RK stages take the staged epilogue rows (periodic y).
"""
import numpy as np
import pytest

from gpu_util import TOL_FP32, e_inf, lib, to_dev, to_host
from oracle import pbc as B
from paper_2308_08447_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [((64, 32, 1), (2e-9, 2e-9, 3e-9), (True, True, False), 2),
         ((64, 24, 1), (2e-9, 2e-9, 3e-9), (True, False, False), 1),
         ((40, 32, 1), (2e-9, 2e-9, 3e-9), (False, True, False), 1),
         ((12, 10, 4), (3e-9, 3e-9, 3e-9), (False, False, True), 1),
         ((32, 16, 4), (3e-9, 3e-9, 3e-9), (True, True, True), 1),
         ((64, 16, 2), (4e-9, 4e-9, 4e-9), (True, True, False), 1)]

_KERNELS = {}


def _kernel(n, cell, pbc, images):
    # the oracle's image sums are the slow part; each case needs them once
    key = (n, cell, pbc, images)
    if key not in _KERNELS:
        _KERNELS[key] = B.periodic_kernel(n, cell, pbc, images)
    return _KERNELS[key]


@pytest.fixture(scope="module")
def g():
    return lib()


@pytest.mark.parametrize("n,cell,pbc,images", CASES)
def test_periodic_demag_and_heff(g, n, cell, pbc, images):
    import torch
    Ms, A = 8e5, 1.3e-11
    m = W.random_unit(n, 61)
    Kg = _kernel(n, cell, pbc, images)
    mesh = g.Mesh(n, cell, Ms, A_ex=A, pbc=pbc, pbc_images=images)
    M = to_dev(Ms * m)
    H = torch.empty_like(M)
    mesh.demag(M, H)
    Heff = torch.empty_like(M)
    mesh.effective_field(to_dev(m), Heff)
    h, heff = to_host(H), to_host(Heff)
    mesh.close()
    m64 = m.astype(np.float64)
    assert e_inf(h, B.conv_periodic(Ms * m64, Kg, pbc)) <= TOL_FP32
    assert e_inf(heff, B.effective_field(m64, Kg, cell, Ms, A, pbc)) <= TOL_FP32


# nx a multiple of 64, x not periodic and ny a multiple of the x-row block's rows: the RK stages
# read the stage input's rows from shared memory, the rows above and below a block copied in with
# them -- here wrapped around the periodic y
STAGED = [((64, 64, 1), (2e-9, 2e-9, 3e-9), (False, True, False), 1)]


@pytest.mark.parametrize("n,cell,pbc,images", CASES[:5] + STAGED)
def test_periodic_steps_track_oracle(g, n, cell, pbc, images):
    Ms, A, alpha, dt = 8e5, 1.3e-11, 0.1, 1e-13
    m = W.random_unit(n, 62)
    mesh = g.Mesh(n, cell, Ms, A_ex=A, alpha=alpha, Hext=(0.0, 0.0, 3e4), pbc=pbc, pbc_images=images)
    md = to_dev(m)
    mesh.llg_step(md, 5, dt)
    got = to_host(md)
    mesh.close()
    Kg = _kernel(n, cell, pbc, images)
    want = B.llg_run(m.astype(np.float64), 5, dt, Kg, cell, Ms, A, alpha, pbc, Hext=(0.0, 0.0, 3e4))
    assert np.abs(got - want).max() < 2e-5


def test_circular_shift_covariance_on_gpu(g):
    import torch
    n, cell, pbc = (64, 32, 2), (3e-9, 3e-9, 3e-9), (True, True, False)
    m = W.random_unit(n, 63)
    mesh = g.Mesh(n, cell, 8e5, A_ex=1.3e-11, pbc=pbc, pbc_images=2)
    H0, H1 = torch.empty((3, 2, 32, 64), device="cuda"), torch.empty((3, 2, 32, 64), device="cuda")
    mesh.effective_field(to_dev(m), H0)
    mesh.effective_field(to_dev(np.roll(np.roll(m, 5, axis=3), 3, axis=2)), H1)
    h0, h1 = to_host(H0), to_host(H1)
    mesh.close()
    assert e_inf(h1, np.roll(np.roll(h0, 5, axis=3), 3, axis=2)) <= 1e-6
