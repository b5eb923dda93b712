"""Pins of the oracle's periodic boundary conditions (reading in oracle/pbc.py; Sec. II).

From outside the module: a circular shift of M along a periodic axis shifts H exactly (circular
convolution); without periodic axes the result is the zero-padded convolution of oracle.conv; a
one-cell film periodic in x and y tends to the infinite plate, N = diag(0, 0, 1), as images are
added; the periodic Laplacian has the discrete Fourier modes as eigenvectors with eigenvalues
-(2 - 2 cos(2 pi p / n)) / d^2; odd kernel components vanish at the half-period slot.
"""
import numpy as np

from oracle import conv as C
from oracle import pbc as B
from oracle import tensor as T


def test_circular_shift_covariance():
    n, cell, per = (8, 6, 2), (2e-9, 3e-9, 2e-9), (True, True, False)
    K = B.periodic_kernel(n, cell, per, 2)
    rng = np.random.default_rng(1)
    M = rng.standard_normal((3, n[2], n[1], n[0]))
    H = B.conv_periodic(M, K, per)
    for axis, sh in ((3, 3), (2, 2)):
        Hs = B.conv_periodic(np.roll(M, sh, axis=axis), K, per)
        assert np.abs(Hs - np.roll(H, sh, axis=axis)).max() <= 1e-12 * np.abs(H).max()
    # not covariant along the non-periodic z axis
    Hz = B.conv_periodic(np.roll(M, 1, axis=1), K, per)
    assert np.abs(Hz - np.roll(H, 1, axis=1)).max() > 1e-3 * np.abs(H).max()


def test_no_periodic_axis_is_the_padded_convolution():
    n, cell = (5, 4, 3), (2e-9, 3e-9, 4e-9)
    K = B.periodic_kernel(n, cell, (False, False, False), 3)
    Nf = T.tensor_all_offsets(n, cell)
    # (the oracle's full tensor mirrors the octant; here negative offsets are evaluated directly)
    assert np.abs(K - Nf).max() <= 1e-13 * np.abs(Nf).max()
    rng = np.random.default_rng(2)
    M = rng.standard_normal((3, n[2], n[1], n[0]))
    assert np.abs(B.conv_periodic(M, K, (False,) * 3) - C.fft_conv(M, Nf)).max() <= 1e-12 * np.abs(M).max()


def test_periodic_film_tends_to_infinite_plate():
    n, cell, per = (8, 8, 1), (4e-9, 4e-9, 2e-9), (True, True, False)
    errs_z, errs_x = [], []
    for Kimg in (2, 4, 8):
        K = B.periodic_kernel(n, cell, per, Kimg)
        Mz = np.zeros((3, 1, 8, 8))
        Mz[2] = 1.0
        Mx = np.zeros((3, 1, 8, 8))
        Mx[0] = 1.0
        errs_z.append(np.abs(B.conv_periodic(Mz, K, per)[2] + 1.0).max())
        errs_x.append(np.abs(B.conv_periodic(Mx, K, per)[0]).max())
    assert errs_z[0] > errs_z[1] > errs_z[2] and errs_z[2] < 5e-3
    assert errs_x[0] > errs_x[1] > errs_x[2] and errs_x[2] < 5e-3


def test_periodic_laplacian_fourier_modes():
    n, cell = (16, 12, 8), (2e-9, 3e-9, 5e-9)
    z, y, x = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    for p, (axis, coord, d, nn) in ((3, (0, x, cell[0], n[0])), (2, (1, y, cell[1], n[1])), (1, (2, z, cell[2], n[2]))):
        mode = np.cos(2 * np.pi * p * coord / nn + 0.3)
        m = np.stack([mode, 0.5 * mode, -mode])
        lam = -(2.0 - 2.0 * np.cos(2 * np.pi * p / nn)) / (d * d)
        lap = B.laplacian(m, cell, (True, True, True))
        assert np.abs(lap - lam * m).max() <= 1e-9 * abs(lam)


def test_odd_components_vanish_at_half_period():
    n, cell, per = (8, 6, 4), (2e-9, 2e-9, 3e-9), (True, True, True)
    K = B.periodic_kernel(n, cell, per, 1)
    tol = 1e-13 * np.abs(K).max()      # the +n/2 and -n/2 image sets cancel up to rounding
    assert np.abs(K[3][:, :, 4]).max() <= tol and np.abs(K[3][:, 3, :]).max() <= tol   # xy: X, Y = n/2
    assert np.abs(K[4][2, :, :]).max() <= tol and np.abs(K[5][2, :, :]).max() <= tol   # xz, yz: Z = n/2
    assert np.abs(K[3][:, :, 3]).max() > 1e-4 * np.abs(K).max()                        # not elsewhere
