"""Parity at the full benchmark sizes, in the launch configuration the benchmark times.

* Thin film 1024 x 1024 x 1, 2 x 2 x 3 nm cells (vortex + noise state): gbd_demag element
  by element against the oracle's FP64 FFT convolution, and one gbd_llg_step (the call the
  benchmark times) against the oracle's RK4 step.
* 3D mesh 512 x 512 x 64, 4 nm cubes: the seeded random-unit-vector M of the benchmark,
  element by element against the oracle's FP64 FFT convolution of the full mesh, for FP32
  stages (e_inf <= 1e-5) and for split-BF16 (<= 1e-4) and split-FP16 (<= 1e-5) tensor-core
  stages, each mesh autotuned as the benchmark does; and properties that hold at any size --
  a uniformly magnetized mesh has mean field -D M with D from Aharoni's prism formula; a
  single magnetized cell j gives H_i = -Ms N(i - j) e_b, checked on sampled cells i against
  the oracle's tensor evaluated one offset at a time.
"""
import numpy as np
import pytest

from gpu_util import TOL_FP32, e_inf, lib, to_dev, to_host
from oracle import conv as C
from oracle import llg as L
from oracle import tensor as T
from paper_2308_08447_gb300 import workloads as W
from pins import aharoni_factors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    return lib()


@pytest.fixture(scope="module")
def film():
    spec = W.thin_film()
    m = W.vortex_noise(spec.n, spec.cell, spec.seed)
    Nf = T.tensor_all_offsets(spec.n, spec.cell)
    return spec, m, Nf


def test_film_demag_full_size(g, film):
    spec, m, Nf = film
    M = (spec.Ms * m).astype(np.float32)
    mesh = g.Mesh(spec.n, spec.cell, spec.Ms)
    Hd = to_dev(np.zeros_like(M))
    mesh.demag(to_dev(M), Hd)
    H = to_host(Hd)
    Href = C.fft_conv(M.astype(np.float64), Nf)
    assert e_inf(H, Href) <= TOL_FP32
    mesh.close()


def test_film_llg_step_full_size(g, film):
    spec, m, Nf = film
    mesh = g.Mesh(spec.n, spec.cell, spec.Ms, A_ex=spec.A_ex, alpha=spec.alpha)
    md = to_dev(m)
    mesh.llg_step(md, 1, spec.dt)
    got = to_host(md)
    m64 = m.astype(np.float64)
    want = L.rk4_step(m64, spec.dt, lambda v: L.rhs(v, Nf, spec.cell, spec.Ms, spec.A_ex, spec.alpha))
    dm_ref = want - m64
    assert e_inf(got - m64, dm_ref) <= TOL_FP32 + 2e-7 / np.sqrt((dm_ref ** 2).sum(0)).max()
    mesh.close()


@pytest.fixture(scope="module")
def cube3d(g):
    spec = W.large_3d()
    mesh = g.Mesh(spec.n, spec.cell, spec.Ms)
    yield spec, mesh
    mesh.close()


def test_3d_uniform_mean_matches_aharoni(g, cube3d):
    import torch
    spec, mesh = cube3d
    nx, ny, nz = spec.n
    D = aharoni_factors(nx * spec.cell[0], ny * spec.cell[1], nz * spec.cell[2])
    M = torch.zeros((3, nz, ny, nx), device="cuda")
    H = torch.empty_like(M)
    for a in range(3):
        M.zero_()
        M[a] = spec.Ms
        mesh.demag(M, H)
        mean = H.double().mean(dim=(1, 2, 3)).cpu().numpy() / spec.Ms
        want = np.zeros(3)
        want[a] = -D[a]
        assert np.abs(mean - want).max() < 1e-5, (a, mean, want)


@pytest.mark.parametrize("j", [(0, 0, 0), (255, 300, 31), (511, 511, 63)])
def test_3d_single_cell_response_sampled(g, cube3d, j):
    import torch
    spec, mesh = cube3d
    nx, ny, nz = spec.n
    rng = np.random.default_rng(7)
    b = int(rng.integers(0, 3))
    M = torch.zeros((3, nz, ny, nx), device="cuda")
    M[b, j[2], j[1], j[0]] = spec.Ms
    H = torch.empty_like(M)
    mesh.demag(M, H)
    # sampled cells: the source, its neighbours, random cells
    pts = [j] + [(min(nx - 1, max(0, j[0] + dx)), min(ny - 1, max(0, j[1] + dy)), min(nz - 1, max(0, j[2] + dz)))
                 for dx in (-2, -1, 0, 1, 2) for dy in (-1, 0, 1) for dz in (-1, 0, 1)]
    pts += [(int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz))) for _ in range(3000)]
    xi = np.array([p[0] for p in pts]); yi = np.array([p[1] for p in pts]); zi = np.array([p[2] for p in pts])
    Hs = H[:, torch.as_tensor(zi), torch.as_tensor(yi), torch.as_tensor(xi)].double().cpu().numpy()
    Nt = T.demag_tensor(xi - j[0], yi - j[1], zi - j[2], *spec.cell)   # (6, S)
    ab = [[0, 3, 4], [3, 1, 5], [4, 5, 2]]
    want = np.stack([-spec.Ms * Nt[ab[a][b]] for a in range(3)])
    assert e_inf(Hs, want) <= TOL_FP32


@pytest.fixture(scope="module")
def random3d():
    """The 512 x 512 x 64 random-M input and its FP64 oracle field (about a minute and ~30 GB
    of host memory, once per module)."""
    spec = W.large_3d()
    M = (spec.Ms * W.random_unit(spec.n, spec.seed)).astype(np.float32)
    Href = C.fft_conv(M.astype(np.float64), T.tensor_all_offsets(spec.n, spec.cell))
    return spec, M, Href


@pytest.mark.parametrize("prec,tol", [("GBD_FP32", TOL_FP32), ("GBD_SPLIT_BF16", 1e-4), ("GBD_SPLIT_FP16", 1e-5)])
def test_3d_random_full_size(g, random3d, prec, tol):
    spec, M, Href = random3d
    mesh = g.Mesh(spec.n, spec.cell, spec.Ms, precision=getattr(g, prec))
    mesh.autotune()
    Hd = to_dev(np.zeros_like(M))
    mesh.demag(to_dev(M), Hd)
    err = e_inf(to_host(Hd), Href)
    mesh.close()
    assert err <= tol, (prec, err)
