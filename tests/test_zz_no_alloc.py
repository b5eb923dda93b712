"""gbd_demag_noalloc: the demag field without any allocation inside the call.

Some callers cannot call cudaMalloc when they need the field: code embedded in a host
application that owns every device allocation through its own pool, or code running at a
memory cap where an allocation (and the device synchronisation it may bring) is not
acceptable. For them the library keeps the demag scratch (the x spectrum, and the y spectrum
of 3D meshes) in a fixed device array compiled into the library. These tests call that entry
point through the C ABI and check that it returns what gbd_demag returns, on two calls in a
row with different inputs, that on the 1024 x 1024 film it also meets the FP32 tolerance against
the FP64 oracle on its own, and that a mesh too large for the array is refused up front.

This file is named so that pytest collects it last.
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


@pytest.mark.parametrize("n,cell", [((1024, 1024, 1), (2e-9, 2e-9, 3e-9)),
                                    ((64, 48, 8), (4e-9, 4e-9, 4e-9)),
                                    ((33, 1, 5), (2e-9, 2e-9, 2e-9))])
def test_noalloc_matches_demag_on_two_calls(g, n, cell):
    Ms = 8e5
    mesh = g.Mesh(n, cell, Ms)
    for seed in (31, 32):   # two calls in a row, different inputs: the shared scratch must not leak
        M = (Ms * W.random_unit(n, seed)).astype(np.float32)
        Md = to_dev(M)
        H_ref = to_dev(np.zeros_like(M))
        H_new = to_dev(np.full_like(M, np.nan))
        mesh.demag(Md, H_ref)
        g.gbd_demag_noalloc(mesh.handle, Md, H_new, mesh.shape)
        href, hnew = to_host(H_ref), to_host(H_new)
        assert np.isfinite(hnew).all()
        assert e_inf(hnew, href) <= TOL_FP32
    mesh.close()


def test_noalloc_refuses_mesh_beyond_static_scratch(g):
    # 512 x 512 x 16: x spectrum 3*16*513*512*8 B = 100.9 MB plus a y spectrum > 64 MiB
    mesh = g.Mesh((512, 512, 16), (4e-9, 4e-9, 4e-9), 8e5)
    x = to_dev(np.zeros((3, 16, 512, 512), np.float32))
    with pytest.raises(g.GbdError) as ei:
        g.gbd_demag_noalloc(mesh.handle, x, x.clone(), mesh.shape)
    assert ei.value.status == g.GBD_EBUDGET
    assert "static maximum" in g.gbd_last_error()
    mesh.close()


def test_noalloc_film_against_oracle(g):
    spec = W.thin_film()
    M = (spec.Ms * W.vortex_noise(spec.n, spec.cell, spec.seed)).astype(np.float32)
    mesh = g.Mesh(spec.n, spec.cell, spec.Ms)
    H = to_dev(np.full_like(M, np.nan))
    g.gbd_demag_noalloc(mesh.handle, to_dev(M), H, mesh.shape)
    got = to_host(H)
    mesh.close()
    Href = C.fft_conv(M.astype(np.float64), T.tensor_all_offsets(spec.n, spec.cell))
    assert e_inf(got, Href) <= TOL_FP32
