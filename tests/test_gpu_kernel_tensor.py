"""gbd_set_kernel_tensor on the GPU: the caller's FP64 tensor drives the same convolution (Eq. 1).

With the oracle's tensor the field matches the oracle's FFT convolution and the built-in
kernel's field; with a tensor that is only a self term the field is local, H_i = -N(0) M_i;
a tensor without the demag parities is refused and leaves the previous kernel in place; on a
periodic mesh one period of an image-summed tensor gives the circular convolution.
"""
import numpy as np
import pytest

from gpu_util import TOL_FP32, e_inf, lib, to_dev, to_host
from oracle import conv as C
from oracle import tensor as T
from paper_2308_08447_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    return lib()


@pytest.mark.parametrize("n,cell", [((24, 20, 6), (3e-9, 2e-9, 4e-9)), ((64, 40, 1), (2e-9, 2e-9, 3e-9))])
def test_oracle_tensor_through_caller_path(g, n, cell):
    import torch
    Ms = 8e5
    M = (Ms * W.random_unit(n, 11)).astype(np.float32)
    Nf = T.tensor_all_offsets(n, cell)
    Href = C.fft_conv(M.astype(np.float64), Nf)
    mesh = g.Mesh(n, cell, Ms)
    Md, H0, H1 = to_dev(M), torch.empty(M.shape, device="cuda"), torch.empty(M.shape, device="cuda")
    mesh.demag(Md, H0)
    mesh.set_kernel_tensor(Nf)
    mesh.demag(Md, H1)
    h0, h1 = to_host(H0), to_host(H1)
    mesh.close()
    assert e_inf(h1, Href) <= TOL_FP32
    assert e_inf(h1, h0) <= 1e-6


def test_self_term_only_tensor_gives_local_field(g):
    import torch
    n, cell = (33, 17, 5), (2e-9, 2e-9, 2e-9)
    diag = (0.21, 0.33, 0.46)
    N6 = np.zeros((6, 2 * n[2] - 1, 2 * n[1] - 1, 2 * n[0] - 1))
    for c in range(3):
        N6[c, n[2] - 1, n[1] - 1, n[0] - 1] = diag[c]
    M = (8e5 * W.random_unit(n, 12)).astype(np.float32)
    mesh = g.Mesh(n, cell, 8e5, set_kernel=False)
    mesh.set_kernel_tensor(N6)
    H = torch.empty(M.shape, device="cuda")
    mesh.demag(to_dev(M), H)
    h = to_host(H)
    mesh.close()
    want = -np.asarray(diag)[:, None, None, None] * M.astype(np.float64)
    assert e_inf(h, want) <= 1e-6


def test_asymmetric_tensor_refused_kernel_kept(g):
    import torch
    n, cell = (16, 12, 3), (2e-9, 2e-9, 2e-9)
    M = to_dev((8e5 * W.random_unit(n, 13)).astype(np.float32))
    mesh = g.Mesh(n, cell, 8e5)
    H0, H1 = torch.empty(M.shape, device="cuda"), torch.empty(M.shape, device="cuda")
    mesh.demag(M, H0)
    bad = T.tensor_all_offsets(n, cell)
    bad[3, 2, 11, 15 + 3] += 1e-3      # xy at (X, Y, Z) = (3, 0, 0) must be 0 (odd in Y)
    with pytest.raises(g.GbdError) as ei:
        mesh.set_kernel_tensor(bad)
    assert ei.value.status == g.GBD_EINVAL
    mesh.demag(M, H1)
    assert torch.equal(H0, H1)
    mesh.close()


@pytest.mark.parametrize("n,cell,pbc", [((32, 16, 1), (2e-9, 2e-9, 3e-9), (True, True, False)),
                                        ((16, 12, 4), (3e-9, 3e-9, 3e-9), (False, False, True))])
def test_periodic_caller_tensor(g, n, cell, pbc):
    # one period of the oracle's image-summed tensor, set by the caller on a periodic mesh, gives
    # the oracle's circular convolution (the reading of the periodic kernel in oracle/pbc.py)
    import torch
    from oracle import pbc as B
    Ms = 8e5
    Kg = B.periodic_kernel(n, cell, pbc, 1)
    M = (Ms * W.random_unit(n, 13)).astype(np.float32)
    mesh = g.Mesh(n, cell, Ms, pbc=pbc, pbc_images=1, set_kernel=False)
    mesh.set_kernel_tensor(Kg)
    H = torch.empty(M.shape, device="cuda")
    mesh.demag(to_dev(M), H)
    h = to_host(H)
    mesh.close()
    assert e_inf(h, B.conv_periodic(M.astype(np.float64), Kg, pbc)) <= TOL_FP32
