"""The split 16-bit tensor-core variants of the FFT stages (GBD_SPLIT_BF16, GBD_SPLIT_FP16)
against the FP64 oracle.

Stated bounds on the demag field: e_inf <= 1e-4 for split BF16 (each radix-16 DFT carries about
2^-16 relative error from the two-term BF16 operands; measured 3e-6 to 1e-5 on meshes up to
256^2, FP32 gives ~3e-7) and e_inf <= 1e-5 for split FP16 (two-term FP16 operands after a
power-of-two scaling per butterfly: about 2^-22). A mesh whose transforms have no radix-16 stage
runs the FP32 arithmetic unchanged, so its result is bit-identical to the FP32 mesh; a mesh that
has them differs from FP32 (the tensor-core stages ran).
"""
import numpy as np
import pytest

from gpu_util import TOL_FP32, e_inf, lib, to_dev, to_host
from oracle import conv as C
from oracle import llg as L
from oracle import tensor as T
from paper_2308_08447_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_SPLIT = {1: 1e-4, 2: 1e-5}     # by precision: split BF16, split FP16


@pytest.fixture(scope="module")
def g():
    return lib()


def _demag(g, n, cell, M, prec):
    mesh = g.Mesh(n, cell, 8e5, precision=prec)
    H = to_dev(np.zeros_like(M))
    mesh.demag(to_dev(M), H)
    out = to_host(H)
    mesh.close()
    return out


@pytest.mark.parametrize("n,cell", [((64, 48, 1), (2e-9, 2e-9, 3e-9)), ((128, 128, 1), (2e-9, 2e-9, 3e-9)),
                                    ((257, 3, 2), (2e-9, 2e-9, 2e-9)), ((64, 64, 32), (4e-9, 4e-9, 4e-9)),
                                    ((100, 37, 1), (2e-9, 2e-9, 3e-9)), ((256, 256, 1), (2e-9, 2e-9, 3e-9))])
def test_split_demag_within_bound(g, n, cell):
    M = (8e5 * W.random_unit(n, 21)).astype(np.float32)
    Href = C.fft_conv(M.astype(np.float64), T.tensor_all_offsets(n, cell))
    e32 = e_inf(_demag(g, n, cell, M, g.GBD_FP32), Href)
    assert e32 <= TOL_FP32
    for prec in (g.GBD_SPLIT_BF16, g.GBD_SPLIT_FP16):
        e16 = e_inf(_demag(g, n, cell, M, prec), Href)
        assert e16 <= TOL_SPLIT[prec], (prec, e16)
        assert e16 != e32     # the tensor-core stages ran (these sizes have radix-16 passes)


@pytest.mark.parametrize("scale", [1e-20, 1.0, 1e20])
def test_split_fp16_scaling_covers_the_float_range(g, scale):
    # FP16 alone holds 6e-8 .. 65504; the per-butterfly power-of-two scaling keeps the relative
    # error at any magnitude FP32 represents (unscaled, these inputs would flush or overflow)
    n, cell = (64, 64, 1), (2e-9, 2e-9, 3e-9)
    M = (scale * 8e5 * W.random_unit(n, 24)).astype(np.float32)
    Href = C.fft_conv(M.astype(np.float64), T.tensor_all_offsets(n, cell))
    H = _demag(g, n, cell, M, g.GBD_SPLIT_FP16)
    assert np.isfinite(H).all()
    assert e_inf(H, Href) <= TOL_SPLIT[g.GBD_SPLIT_FP16]


def test_split_without_radix16_stage_equals_fp32(g):
    n, cell = (32, 32, 8), (4e-9, 4e-9, 4e-9)     # lengths 64/64/16: radices 8, 8 and 2, 8
    M = (8e5 * W.random_unit(n, 22)).astype(np.float32)
    H32 = _demag(g, n, cell, M, g.GBD_FP32)
    assert np.array_equal(H32, _demag(g, n, cell, M, g.GBD_SPLIT_BF16))
    assert np.array_equal(H32, _demag(g, n, cell, M, g.GBD_SPLIT_FP16))


@pytest.mark.parametrize("prec", [1, 2])
def test_split_llg_steps_track_oracle(g, prec):
    n, cell, Ms, A, alpha, dt = (48, 64, 2), (3e-9, 3e-9, 3e-9), 8e5, 1.3e-11, 0.02, 1e-13
    m = W.random_unit(n, 23)
    mesh = g.Mesh(n, cell, Ms, A_ex=A, alpha=alpha, precision=prec)
    md = to_dev(m)
    mesh.llg_step(md, 5, dt)
    got = to_host(md)
    want = L.llg_run(m.astype(np.float64), 5, dt, T.tensor_all_offsets(n, cell), cell, Ms, A, alpha)
    d = want - m.astype(np.float64)
    assert e_inf(got - m, d) <= TOL_SPLIT[prec]
    mesh.close()
