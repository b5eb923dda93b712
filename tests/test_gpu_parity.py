"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Eq. 1 (Sec. II) as gbd_demag; H_eff and dm/dt (Eqs. 4, 5, Sec. III) as
gbd_effective_field / gbd_llg_rhs; the RK4 step as gbd_llg_step. Inputs are seeded,
FP32-rounded, and the oracle consumes the same rounded values in FP64. Shapes cover
several tiles, ragged tails, sizes of 1 along each axis, odd and prime sizes.
"""
import numpy as np
import pytest

from gpu_util import TOL_FP32, e_inf, lib, to_dev, to_host
from oracle import conv as C
from oracle import llg as L
from oracle import tensor as T
from paper_2308_08447_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SHAPES = [
    ((1, 1, 1), (3e-9, 3e-9, 3e-9)),
    ((3, 5, 1), (2e-9, 2e-9, 3e-9)),
    ((7, 4, 3), (2e-9, 3e-9, 4e-9)),
    ((16, 1, 1), (1e-9, 1e-9, 1e-9)),
    ((1, 16, 1), (1e-9, 1e-9, 1e-9)),
    ((1, 1, 9), (1e-9, 1e-9, 1e-9)),
    ((1, 6, 3), (1e-9, 2e-9, 1e-9)),
    ((9, 1, 4), (2e-9, 1e-9, 3e-9)),
    ((33, 17, 5), (4e-9, 4e-9, 4e-9)),
    ((64, 48, 1), (2e-9, 2e-9, 3e-9)),
    ((100, 37, 1), (2e-9, 2e-9, 3e-9)),
    ((13, 29, 7), (3e-9, 2e-9, 2e-9)),
    ((128, 128, 1), (2e-9, 2e-9, 3e-9)),
    ((40, 30, 20), (4e-9, 4e-9, 4e-9)),
    ((257, 3, 2), (2e-9, 2e-9, 2e-9)),
]


@pytest.fixture(scope="module")
def g():
    return lib()


def _M(n, seed, Ms):
    return (Ms * W.random_unit(n, seed)).astype(np.float32)


@pytest.mark.parametrize("n,cell", SHAPES)
def test_demag_parity(g, n, cell):
    Ms = 8e5
    M = _M(n, 21, Ms)
    mesh = g.Mesh(n, cell, Ms)
    Md = to_dev(M)
    Hd = to_dev(np.zeros_like(M))
    mesh.demag(Md, Hd)
    H = to_host(Hd)
    Href = C.fft_conv(M.astype(np.float64), T.tensor_all_offsets(n, cell))
    assert e_inf(H, Href) <= TOL_FP32
    # a second call on the same mesh gives the same result bit for bit
    Hd2 = to_dev(np.zeros_like(M))
    mesh.demag(Md, Hd2)
    assert np.array_equal(to_host(Hd2), H)
    mesh.close()


def test_parity_cube_32x32x8_against_direct_sum(g):
    spec = W.parity_cube()
    M = _M(spec.n, spec.seed, spec.Ms)
    mesh = g.Mesh(spec.n, spec.cell, spec.Ms)
    Md, Hd = to_dev(M), to_dev(np.zeros_like(M))
    mesh.demag(Md, Hd)
    H = to_host(Hd)
    Href = C.direct_sum(M.astype(np.float64), T.tensor_all_offsets(spec.n, spec.cell))
    assert e_inf(H, Href) <= TOL_FP32
    mesh.close()


@pytest.mark.parametrize("n,cell", [((64, 48, 1), (2e-9, 2e-9, 3e-9)), ((13, 29, 7), (3e-9, 2e-9, 2e-9)),
                                    ((1, 1, 1), (3e-9, 3e-9, 3e-9)), ((33, 17, 5), (4e-9, 4e-9, 4e-9))])
def test_effective_field_and_rhs(g, n, cell):
    Ms, A, alpha, Hext = 8.6e5, 1.3e-11, 0.02, (1.5e4, -2e4, 3e4)
    m = W.random_unit(n, 5)
    mesh = g.Mesh(n, cell, Ms, A_ex=A, alpha=alpha, Hext=Hext)
    md = to_dev(m)
    out = to_dev(np.zeros_like(m))
    mesh.effective_field(md, out)
    Heff = to_host(out)
    m64 = m.astype(np.float64)
    Nf = T.tensor_all_offsets(n, cell)
    Href = L.effective_field(m64, Nf, cell, Ms, A, Hext)
    assert e_inf(Heff, Href) <= TOL_FP32
    mesh.llg_rhs(md, out)
    f = to_host(out)
    fref = L.llg_rhs(m64, Href, alpha)
    assert e_inf(f, fref) <= TOL_FP32
    mesh.close()


# (64, 64, 1) and (128, 64, 2): nx a multiple of 64 and ny a multiple of the x-row block's rows,
# so the RK stages read the stage input's rows from shared memory (the 3D mesh its z neighbours
# from global memory); the others take the global-memory epilogue
@pytest.mark.parametrize("n,cell", [((64, 48, 1), (2e-9, 2e-9, 3e-9)), ((13, 29, 7), (3e-9, 2e-9, 2e-9)),
                                    ((100, 37, 1), (2e-9, 2e-9, 3e-9)), ((64, 64, 1), (2e-9, 2e-9, 3e-9)),
                                    ((128, 64, 2), (3e-9, 3e-9, 3e-9))])
def test_one_rk4_step(g, n, cell):
    Ms, A, alpha, dt = 8.6e5, 1.3e-11, 0.02, 1e-13
    m = W.random_unit(n, 9)
    mesh = g.Mesh(n, cell, Ms, A_ex=A, alpha=alpha)
    md = to_dev(m)
    mesh.llg_step(md, 1, dt)
    got = to_host(md)
    m64 = m.astype(np.float64)
    Nf = T.tensor_all_offsets(n, cell)
    want = L.rk4_step(m64, dt, lambda v: L.rhs(v, Nf, cell, Ms, A, alpha))
    # the step's change dm is O(0.05); FP32 storage of |m| = 1 adds ~6e-8 absolute
    dm_ref = want - m64
    assert e_inf(got - m64, dm_ref) <= TOL_FP32 + 2e-7 / np.sqrt((dm_ref ** 2).sum(0)).max()
    assert np.abs(np.sqrt((got ** 2).sum(0)) - 1).max() < 1e-6
    mesh.close()


def test_twenty_steps_track_oracle(g):
    n, cell = (32, 24, 2), (3e-9, 3e-9, 3e-9)
    Ms, A, alpha, dt = 8e5, 1.3e-11, 0.1, 1e-13
    m = W.random_unit(n, 12)
    mesh = g.Mesh(n, cell, Ms, A_ex=A, alpha=alpha, Hext=(0.0, 0.0, 5e4))
    md = to_dev(m)
    mesh.llg_step(md, 20, dt)
    got = to_host(md)
    Nf = T.tensor_all_offsets(n, cell)
    want = L.llg_run(m.astype(np.float64), 20, dt, Nf, cell, Ms, A, alpha, Hext=(0.0, 0.0, 5e4))
    assert np.abs(got - want).max() < 2e-5
    mesh.close()


def test_calls_split_across_launches_match_one_call(g):
    n, cell = (48, 40, 1), (2e-9, 2e-9, 3e-9)
    m = W.random_unit(n, 13)
    mesh = g.Mesh(n, cell, 8.6e5, A_ex=1.3e-11, alpha=0.02)
    a, b = to_dev(m), to_dev(m)
    mesh.llg_step(a, 6, 1e-13)
    for _ in range(3):
        mesh.llg_step(b, 2, 1e-13)
    assert np.array_equal(to_host(a), to_host(b))
    mesh.close()


def test_errors_reported(g):
    import torch
    mesh = g.Mesh((8, 8, 1), (2e-9, 2e-9, 3e-9), 8e5, set_kernel=False)
    x = torch.zeros((3, 1, 8, 8), device="cuda")
    with pytest.raises(g.GbdError) as ei:
        mesh.demag(x, x.clone())
    assert ei.value.status == g.GBD_ESTATE
    g.gbd_set_kernel(mesh.handle)
    with pytest.raises(g.GbdError) as ei:
        g._check(g.load().gbd_llg_step(mesh.handle, None, 1, 1e-13, None))
    assert ei.value.status == g.GBD_EINVAL
    with pytest.raises(g.GbdError) as ei:
        mesh.llg_step(x, 1, -1.0)
    assert ei.value.status == g.GBD_EINVAL
    mesh.close()


def test_fields_only_4_byte_aligned(g):
    # the ABI asks for 4-byte aligned fields; one that starts 4 bytes into its allocation
    # takes the row kernel's scalar path and must give the aligned result up to the order
    # of the Laplacian's sums (and the oracle's field within the FP32 bar)
    import torch
    n, cell, Ms, A, alpha, dt = (256, 64, 1), (2e-9, 2e-9, 3e-9), 8e5, 1.3e-11, 0.02, 2e-14
    m0 = W.random_unit(n, 31).astype(np.float32)
    res = []
    for off in (0, 1):
        mesh = g.Mesh(n, cell, Ms, A_ex=A, alpha=alpha)
        bufs = [torch.zeros(m0.size + off, device="cuda") for _ in range(3)]
        m, M, H = (b[off:].view(m0.shape) for b in bufs)
        m.copy_(torch.from_numpy(m0))
        M.copy_(torch.from_numpy(Ms * m0))
        Heff = torch.empty(m0.shape, device="cuda")
        mesh.demag(M, H)
        mesh.effective_field(m, Heff)
        mesh.llg_step(m, 3, dt)
        res.append((to_host(H), to_host(Heff), to_host(m)))
        mesh.close()
    for a, b in zip(*res):
        assert e_inf(a, b) <= 1e-6
    Href = C.fft_conv((Ms * m0).astype(np.float64), T.tensor_all_offsets(n, cell))
    assert e_inf(res[1][0], Href) <= TOL_FP32
