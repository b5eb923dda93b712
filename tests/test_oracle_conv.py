"""Pins of the oracle's Eq. 1 evaluation (direct sum and zero-padded FFT convolution, Sec. II / Appendix A).

* Direct O(N^2) sum and FFT convolution agree on tiny meshes (FP64).
* The cropped FFT result does not depend on the padded length P >= 2n - 1.
* A single magnetized cell j gives H_i = -Ms N(i - j) e_b (index and sign
  conventions), with N taken component by component from the closed form.
* Far from a single magnetized cell the field is the point-dipole field
  V Ms (3 (m.r) r / r^2 - m) / (4 pi r^3) (sign of Eq. 1).
* A uniformly magnetized mesh has mean field -D M, D the whole prism's
  demagnetizing factors from Aharoni's formula; for a cube -M/3 exactly.
* Deep inside a wide thin film magnetized out of plane H_z -> -Ms, approaching
  the centre-point closed form for the whole plate.
* The magnetostatic energy -(mu0/2) sum M.H V is >= 0 for any M.
"""
import math

import numpy as np
import pytest

from oracle import conv as C
from oracle import tensor as T
from pins import aharoni_factors, prism_centre_Nzz


def _rand_M(n, seed, Ms=8e5):
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((3, n[2], n[1], n[0]))
    return Ms * g / np.linalg.norm(g, axis=0, keepdims=True)


TINY = [((1, 1, 1), (4e-9, 4e-9, 4e-9)), ((3, 5, 1), (2e-9, 2e-9, 3e-9)),
        ((7, 4, 3), (2e-9, 3e-9, 4e-9)), ((4, 4, 4), (4e-9, 4e-9, 4e-9)),
        ((2, 1, 5), (3e-9, 1e-9, 2e-9)), ((1, 6, 2), (1e-9, 1e-9, 1e-9))]


@pytest.mark.parametrize("n,cell", TINY)
def test_direct_sum_equals_fft_convolution(n, cell):
    M = _rand_M(n, 7)
    Nf = T.tensor_all_offsets(n, cell)
    Hd = C.direct_sum(M, Nf)
    Hf = C.fft_conv(M, Nf)
    assert np.abs(Hd - Hf).max() <= 1e-12 * np.abs(Hd).max()


def test_padded_length_independence():
    n, cell = (7, 4, 3), (2e-9, 3e-9, 4e-9)
    M = _rand_M(n, 8)
    Nf = T.tensor_all_offsets(n, cell)
    H0 = C.fft_conv(M, Nf)
    for P in [(13, 7, 5), (16, 8, 8), (17, 11, 6)]:
        H1 = C.fft_conv(M, Nf, P=P)
        assert np.abs(H1 - H0).max() <= 1e-12 * np.abs(H0).max()


_NAMES = {(0, 0): "xx", (1, 1): "yy", (2, 2): "zz", (0, 1): "xy", (1, 0): "xy",
          (0, 2): "xz", (2, 0): "xz", (1, 2): "yz", (2, 1): "yz"}


@pytest.mark.parametrize("j", [(0, 0, 0), (4, 2, 1), (6, 3, 2)])
@pytest.mark.parametrize("b", [0, 1, 2])
def test_single_cell_response(j, b):
    n, cell = (7, 4, 3), (2e-9, 3e-9, 4e-9)
    Ms = 8e5
    M = np.zeros((3, n[2], n[1], n[0]))
    M[b, j[2], j[1], j[0]] = Ms
    H = C.fft_conv(M, T.tensor_all_offsets(n, cell))
    zz, yy, xx = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    ex = T.newell_exact((xx - j[0]) * cell[0], (yy - j[1]) * cell[1], (zz - j[2]) * cell[2], *cell)
    for a in range(3):
        want = -Ms * ex[T.COMPONENTS.index(_NAMES[(a, b)])]
        assert np.abs(H[a] - want).max() <= 1e-9 * Ms


def test_far_cell_gives_point_dipole_field():
    n, cell, Ms = (41, 3, 3), (2e-9, 2e-9, 2e-9), 1e6
    V = cell[0] * cell[1] * cell[2]
    mdir = np.array([0.6, 0.0, 0.8])
    M = np.zeros((3, 3, 3, 41))
    M[:, 1, 1, 0] = Ms * mdir
    H = C.fft_conv(M, T.tensor_all_offsets(n, cell))
    for xi, yi, zi in [(40, 1, 1), (30, 0, 2), (20, 2, 0)]:
        r = np.array([xi * cell[0], (yi - 1) * cell[1], (zi - 1) * cell[2]])
        rn = np.linalg.norm(r)
        rh = r / rn
        dip = V * Ms * (3 * np.dot(mdir, rh) * rh - mdir) / (4 * math.pi * rn ** 3)
        got = H[:, zi, yi, xi]
        assert np.linalg.norm(got - dip) <= 3 * (cell[0] / rn) ** 2 * np.linalg.norm(dip)


def test_uniform_cube_mean_is_minus_third():
    n, cell, Ms = (6, 6, 6), (4e-9, 4e-9, 4e-9), 8e5
    m = np.array([0.3, -0.5, 0.8])
    m /= np.linalg.norm(m)
    M = Ms * m[:, None, None, None] * np.ones((3, 6, 6, 6))
    H = C.fft_conv(M, T.tensor_all_offsets(n, cell))
    np.testing.assert_allclose(H.mean(axis=(1, 2, 3)), -Ms * m / 3, rtol=0, atol=1e-10 * Ms)


@pytest.mark.parametrize("n,cell", [((5, 3, 2), (2e-9, 3e-9, 1e-9)), ((8, 8, 1), (2e-9, 2e-9, 3e-9)),
                                    ((3, 7, 4), (1e-9, 1e-9, 2e-9))])
def test_uniform_prism_mean_matches_aharoni(n, cell):
    Ms = 1e6
    D = aharoni_factors(n[0] * cell[0], n[1] * cell[1], n[2] * cell[2])
    Nf = T.tensor_all_offsets(n, cell)
    for a in range(3):
        M = np.zeros((3, n[2], n[1], n[0]))
        M[a] = Ms
        Hm = C.fft_conv(M, Nf).mean(axis=(1, 2, 3))
        want = np.zeros(3)
        want[a] = -Ms * D[a]
        np.testing.assert_allclose(Hm, want, rtol=0, atol=1e-11 * Ms)


def test_thin_film_centre_field_tends_to_minus_Ms():
    cell, Ms = (2e-9, 2e-9, 3e-9), 8.6e5
    devs = []
    for side in (16, 64, 256):
        n = (side, side, 1)
        M = np.zeros((3, 1, side, side))
        M[2] = Ms
        H = C.fft_conv(M, T.tensor_all_offsets(n, cell))
        c = side // 2
        hz = H[2, 0, c - 1:c + 1, c - 1:c + 1].mean() / Ms
        point = prism_centre_Nzz(side * cell[0], side * cell[1], cell[2])
        assert abs(hz + point) < 3e-4 * (16 / side) ** 2
        devs.append(abs(hz + 1.0))
    assert devs[0] > devs[1] > devs[2]
    assert devs[2] < 6e-3


def test_energy_nonnegative():
    n, cell = (6, 5, 3), (2e-9, 3e-9, 4e-9)
    Nf = T.tensor_all_offsets(n, cell)
    for s in range(5):
        M = _rand_M(n, 100 + s)
        H = C.fft_conv(M, Nf)
        assert -(M * H).sum() >= 0.0
