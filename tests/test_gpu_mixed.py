"""Padded lengths 3 * 2^k and 5 * 2^k (GPU).

Sec. II pads each axis to 2n; any padded length P >= 2n - 1 gives the same cropped convolution
(the oracle's padded-length independence pin). FP32 meshes take the shortest length among the
powers of two and 3 * 2^k, 5 * 2^k along x and y, which runs the radix-3 / radix-5 first passes.
Checked here: the demag field of such meshes element by element against the FP64 oracle (which
pads to 2n), against the same mesh forced to powers of two (GBD_FLAG_POW2_PAD), one RK4 step
against the oracle, every row tile variant bit-identical, and a batch equal to each mesh alone.
"""
import numpy as np
import pytest

from gpu_util import TOL_FP32, e_inf, lib, to_dev, to_host
from oracle import conv as C
from oracle import llg as L
from oracle import tensor as T
from paper_2308_08447_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# (mesh, cell, expected (Px, Py)): x lengths 2 * {96, 160, 384, 320, 1536, 2560}, y lengths
# {96, 160, 320, 1536}, films and 3D meshes
CASES = [((80, 48, 2), (2e-9, 2e-9, 3e-9), (192, 96)),
         ((150, 72, 1), (3e-9, 3e-9, 3e-9), (320, 160)),
         ((352, 480, 1), (2e-9, 2e-9, 3e-9), (768, 1024)),
         ((300, 150, 4), (4e-9, 4e-9, 4e-9), (640, 320)),
         ((1000, 700, 1), (2e-9, 2e-9, 3e-9), (2048, 1536)),
         ((1500, 64, 1), (2e-9, 2e-9, 3e-9), (3072, 128)),
         ((2500, 8, 1), (2e-9, 2e-9, 3e-9), (5120, 16))]


@pytest.fixture(scope="module")
def g():
    return lib()


@pytest.mark.parametrize("n,cell,P", CASES)
def test_mixed_length_demag_against_oracle(g, n, cell, P):
    Ms = 8e5
    mesh = g.Mesh(n, cell, Ms)
    assert tuple(g.gbd_plan_dims(mesh.desc)[:2]) == P
    M = (Ms * W.random_unit(n, 61)).astype(np.float32)
    H = to_dev(np.zeros_like(M))
    mesh.demag(to_dev(M), H)
    got = to_host(H)
    # the same mesh on power-of-two lengths gives the same cropped field
    ref = g.Mesh(n, cell, Ms, pow2_pad=True)
    H2 = to_dev(np.zeros_like(M))
    ref.demag(to_dev(M), H2)
    got2 = to_host(H2)
    mesh.close()
    ref.close()
    Href = C.fft_conv(M.astype(np.float64), T.tensor_all_offsets(n, cell))
    assert e_inf(got, Href) <= TOL_FP32
    assert e_inf(got2, Href) <= TOL_FP32
    assert e_inf(got, got2) <= TOL_FP32


@pytest.mark.parametrize("n,cell", [((150, 72, 1), (3e-9, 3e-9, 3e-9)), ((96, 96, 2), (3e-9, 3e-9, 3e-9))])
def test_mixed_length_rk4_step_and_tile_variants(g, n, cell):
    Ms, A, alpha, dt = 8e5, 1.3e-11, 0.05, 5e-14
    mesh = g.Mesh(n, cell, Ms, A_ex=A, alpha=alpha)
    m0 = W.random_unit(n, 62)
    outs = []
    for v in ((1, 0, 0, 0), (2, 0, 0, 0), (3, 0, 0, 0)):     # row_kernel and the pipelined kernel
        g.gbd_mesh_set_tuning(mesh.handle, v)
        md = to_dev(m0)
        mesh.llg_step(md, 2, dt)
        outs.append(to_host(md))
    mesh.close()
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    Nf = T.tensor_all_offsets(n, cell)
    want = L.llg_run(m0.astype(np.float64), 2, dt, Nf, cell, Ms, A, alpha)
    assert np.abs(outs[0] - want).max() < 2e-6


def test_mixed_length_batch_equals_each_alone(g):
    specs = [((150, 72, 1), (3e-9, 3e-9, 3e-9), 8e5), ((80, 48, 2), (2e-9, 2e-9, 3e-9), 1.1e6),
             ((352, 96, 1), (2e-9, 2e-9, 2e-9), 6e5), ((64, 64, 4), (3e-9, 3e-9, 3e-9), 9e5)]
    meshes = [g.Mesh(n, c, Ms, A_ex=1.3e-11, alpha=0.05) for n, c, Ms in specs]
    states = [W.random_unit(n, 70 + i) for i, (n, _, _) in enumerate(specs)]
    dts = [W.stable_dt(c, Ms, 1.3e-11) for _, c, Ms in specs]
    steps = [3, 2, 4, 1]
    batch = g.Batch(meshes)
    dev = [to_dev(s) for s in states]
    batch.run(dev, steps, dts)
    got = [to_host(d) for d in dev]
    for mesh, s, n_, dt, bg in zip(meshes, states, steps, dts, got):
        md = to_dev(s)
        mesh.llg_step(md, n_, dt)
        assert np.array_equal(to_host(md), bg)
    batch.close()
    for m in meshes:
        m.close()


def test_autotune_chooses_padded_length(g):
    # the autotuner times the mesh against its power-of-two twin and may move it there; either
    # way the plan it reports is one of the two and the field still matches the oracle
    n, cell, Ms = (352, 96, 2), (3e-9, 3e-9, 3e-9), 8e5
    mesh = g.Mesh(n, cell, Ms, A_ex=1.3e-11, alpha=0.05)
    before = g.gbd_mesh_plan_dims(mesh.handle)
    assert before[:2] == (768, 192)
    mesh.autotune()
    after = g.gbd_mesh_plan_dims(mesh.handle)
    assert after[:2] in ((768, 192), (1024, 256)) and after[2] == 4
    M = (Ms * W.random_unit(n, 63)).astype(np.float32)
    H = to_dev(np.zeros_like(M))
    mesh.demag(to_dev(M), H)
    got = to_host(H)
    m0 = W.random_unit(n, 64)
    md = to_dev(m0)
    mesh.llg_step(md, 2, 5e-14)
    mesh.close()
    assert e_inf(got, C.fft_conv(M.astype(np.float64), T.tensor_all_offsets(n, cell))) <= TOL_FP32
    want = L.llg_run(m0.astype(np.float64), 2, 5e-14, T.tensor_all_offsets(n, cell), cell, Ms, 1.3e-11, 0.05)
    assert np.abs(to_host(md) - want).max() < 2e-6
