"""The C-ABI library on the host (no GPU): symbols, argument checks, planning, and the
library's own FP64 tensor / kernel spectrum against the independent oracle.

The tensor (Eq. 1's N) and its packed spectrum are host code in the library, written
separately from ``oracle/``; here the two implementations are compared, and the spectrum
is compared with the oracle's FFT of the tensor placed on the padded grid (Sec. II).
"""
import ctypes
import math

import numpy as np
import pytest

from oracle import conv as C
from oracle import tensor as T


@pytest.fixture(scope="module")
def g():
    from paper_2308_08447_gb300 import build, gbdemag
    build.build()
    gbdemag.load()
    return gbdemag


def test_library_exports_every_header_symbol(g):
    lib = g.load()
    names = g.header_symbols()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


@pytest.mark.parametrize("n,dims", [((1024, 1024, 1), (2048, 2048, 1, 1025, 1025, 1)),
                                    ((32, 32, 8), (64, 64, 16, 33, 33, 9)),
                                    ((512, 512, 64), (1024, 1024, 128, 513, 513, 65)),
                                    ((1, 1, 1), (2, 1, 1, 2, 1, 1)),
                                    ((33, 17, 5), (128, 64, 16, 65, 33, 9)),
                                    # lengths 3 * 2^k, 5 * 2^k where shorter than the power of two
                                    ((352, 480, 1), (768, 1024, 1, 385, 513, 1)),
                                    ((96, 96, 1), (192, 192, 1, 97, 97, 1)),
                                    ((160, 64, 4), (320, 128, 8, 161, 65, 5)),
                                    ((640, 320, 2), (1280, 640, 4, 641, 321, 3)),
                                    ((300, 150, 1), (640, 320, 1, 321, 161, 1))])
def test_plan_dims(g, n, dims):
    assert g.gbd_plan_dims(g.make_desc(n, (1e-9, 1e-9, 1e-9), 8e5)) == dims


@pytest.mark.parametrize("n", [(352, 480, 1), (160, 64, 4), (300, 150, 1)])
def test_plan_dims_powers_of_two_when_asked(g, n):
    # GBD_FLAG_POW2_PAD, and the split precisions, keep every padded length a power of two
    for d in (g.make_desc(n, (1e-9,) * 3, 8e5, pow2_pad=True),
              g.make_desc(n, (1e-9,) * 3, 8e5, precision=g.GBD_SPLIT_BF16)):
        Px, Py, Pz = g.gbd_plan_dims(d)[:3]
        for P, m in ((Px, n[0]), (Py, n[1]), (Pz, n[2])):
            assert P & (P - 1) == 0 and P >= 2 * m - 1


def test_argument_errors(g):
    cases = [(((0, 4, 4), (1e-9,) * 3, 8e5), g.GBD_EINVAL),
             (((4, 4, 4), (1e-9, 0.0, 1e-9), 8e5), g.GBD_EINVAL),
             (((4, 4, 4), (1e-9,) * 3, -1.0), g.GBD_EINVAL),
             (((4, 4, 4), (1e-9, float("nan"), 1e-9), 8e5), g.GBD_EINVAL),
             (((5000, 4, 4), (1e-9,) * 3, 8e5), g.GBD_EUNSUPPORTED),
             (((4, 3000, 4), (1e-9,) * 3, 8e5), g.GBD_EUNSUPPORTED)]
    for (n, cell, Ms), want in cases:
        with pytest.raises(g.GbdError) as ei:
            g.gbd_mesh_bytes(g.make_desc(n, cell, Ms))
        assert ei.value.status == want
        assert g.gbd_last_error()
    with pytest.raises(g.GbdError) as ei:
        g.gbd_mesh_bytes(g.make_desc((4, 4, 4), (1e-9,) * 3, 8e5, alpha=-0.1))
    assert ei.value.status == g.GBD_EINVAL


def test_mesh_bytes_counts_buffers(g):
    n = (1024, 1024, 1)
    b = g.gbd_mesh_bytes(g.make_desc(n, (2e-9, 2e-9, 3e-9), 8.6e5))
    N = n[0] * n[1]
    S = 3 * 1025 * 1024 * 8
    K = 1025 * 1025 * 16
    state = 9 * N * 4
    # power-of-two levels up to 8192; split DFT-16 fragments; levels 3 * 2^j (up to 6144) and
    # 5 * 2^j (up to 5120)
    twiddles = 2 * 8192 * 8 + 4 * 32 * 32 * 4 + 2 * 6144 * 8 + 2 * 5120 * 8 + 16   # + device status word
    assert b == S + K + state + twiddles


def _scale(X, Y, Z, cell):
    r = math.sqrt((X * cell[0]) ** 2 + (Y * cell[1]) ** 2 + (Z * cell[2]) ** 2)
    return cell[0] * cell[1] * cell[2] / (4 * math.pi * max(r, max(cell)) ** 3)


@pytest.mark.parametrize("cell", [(4e-9, 4e-9, 4e-9), (2e-9, 2e-9, 3e-9), (1e-9, 2e-9, 1.5e-9)])
def test_library_tensor_matches_oracle(g, cell):
    desc = g.make_desc((8, 8, 8), cell, 8e5)
    rng = np.random.default_rng(5)
    offs = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1), (-3, 2, -1)]
    offs += [tuple(int(v) for v in rng.integers(-12, 13, 3)) for _ in range(40)]
    offs += [tuple(int(v) for v in rng.integers(-300, 301, 3)) for _ in range(40)]
    for X, Y, Z in offs:
        lib = np.array(g.gbd_tensor_at(desc, X, Y, Z))
        ora = T.demag_tensor(np.array([X]), np.array([Y]), np.array([Z]), *cell)[:, 0]
        # both sit within ~1e-9 of the exact value near the 8-cell switch (FP64 cancellation)
        assert np.abs(lib - ora).max() <= 1e-8 * _scale(X, Y, Z, cell), (X, Y, Z, lib, ora)


def test_library_tensor_matches_exact_golden(g):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "newell_exact.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for v in rows:
        cell = tuple(float(x) * 1e-9 for x in v[:3])
        X, Y, Z = (int(x) for x in v[3:6])
        exact = np.array([float(x) for x in v[6:]])
        lib = np.array(g.gbd_tensor_at(g.make_desc((1, 1, 1), cell, 1.0), X, Y, Z))
        tol = 2e-8 if max(cell) <= 1.5 * min(cell) else 1e-7
        assert np.abs(lib - exact).max() <= tol * _scale(X, Y, Z, cell), (cell, X, Y, Z)


@pytest.mark.parametrize("n,cell", [((8, 6, 1), (2e-9, 2e-9, 3e-9)), ((5, 4, 3), (2e-9, 3e-9, 4e-9)),
                                    ((1, 1, 1), (3e-9, 3e-9, 3e-9)), ((1, 7, 4), (1e-9, 1e-9, 2e-9)),
                                    ((16, 1, 1), (1e-9, 1e-9, 1e-9)), ((32, 32, 8), (4e-9, 4e-9, 4e-9)),
                                    ((80, 48, 2), (2e-9, 2e-9, 3e-9)),    # Px = 192, Py = 96
                                    ((150, 72, 1), (3e-9, 3e-9, 3e-9))])  # Px = 320, Py = 160
def test_library_spectrum_matches_oracle_fft(g, n, cell):
    desc = g.make_desc(n, cell, 8e5)
    Px, Py, Pz, Hx, Ky, Kz = g.gbd_plan_dims(desc)
    spec = g.gbd_kernel_spectrum_host(desc)
    Nf = T.tensor_all_offsets(n, cell)
    Kt = C.place_kernel(Nf, n, (Px, Py, Pz))
    Kh = np.fft.fft(np.fft.fft(np.fft.rfft(Kt, axis=3), axis=2), axis=1)  # (6, Pz, Py, Hx)
    assert np.abs(Kh.imag).max() <= 1e-12 * np.abs(Kh).max()
    want = -Kh.real[:, :Kz, :Ky, :] / (Px * Py * Pz)
    if n[2] == 1:
        want[4:] = 0.0
    assert np.abs(spec - want).max() <= 1e-11 * np.abs(want).max()


# ---- caller tensors (gbd_set_kernel_tensor / gbd_kernel_spectrum_from_tensor_host) ----------

@pytest.mark.parametrize("n,cell", [((8, 6, 1), (2e-9, 2e-9, 3e-9)), ((5, 4, 3), (2e-9, 3e-9, 4e-9)),
                                    ((1, 1, 1), (3e-9, 3e-9, 3e-9)), ((1, 7, 4), (1e-9, 1e-9, 2e-9))])
def test_spectrum_of_caller_tensor_matches_numpy_fft(g, n, cell):
    # the oracle's tensor through the caller path equals numpy's FFT of the placed tensor
    desc = g.make_desc(n, cell, 8e5)
    Px, Py, Pz, Hx, Ky, Kz = g.gbd_plan_dims(desc)
    Nf = T.tensor_all_offsets(n, cell)
    spec = g.gbd_kernel_spectrum_from_tensor_host(desc, Nf)
    Kt = C.place_kernel(Nf, n, (Px, Py, Pz))
    Kh = np.fft.fft(np.fft.fft(np.fft.rfft(Kt, axis=3), axis=2), axis=1)
    want = -Kh.real[:, :Kz, :Ky, :] / (Px * Py * Pz)
    if n[2] == 1:
        want[4:] = 0.0
    assert np.abs(spec - want).max() <= 1e-12 * np.abs(want).max()
    # and agrees with the built-in tensor's spectrum to the tensors' agreement (<= 1e-8 scale)
    assert np.abs(spec - g.gbd_kernel_spectrum_host(desc)).max() <= 1e-8 * np.abs(want).max()


def _sparse_tensor(n, a, b, c, v, u):
    """Self term diag(a, b, c); N_xy = v sign(X) sign(Y) at (+-1, +-1, 0); N_xz = u sign(X) sign(Z)
    at (+-1, 0, +-1); everything else 0."""
    nx, ny, nz = n
    N6 = np.zeros((6, 2 * nz - 1, 2 * ny - 1, 2 * nx - 1))
    o = (nz - 1, ny - 1, nx - 1)
    N6[0][o], N6[1][o], N6[2][o] = a, b, c
    for sx in (1, -1):
        for sy in (1, -1):
            N6[3][o[0], o[1] + sy, o[2] + sx] = v * sx * sy
        for sz in (1, -1):
            N6[4][o[0] + sz, o[1], o[2] + sx] = u * sx * sz
    return N6


def test_spectrum_of_sparse_tensor_closed_form(g):
    # DFT of the sparse tensor by hand: a constant for the self term, and
    # sum_(X,Y=+-1) v sgn(X) sgn(Y) e^{-i(aX+bY)} = -4 v sin(a) sin(b); stored: -F / (Px Py Pz)
    n = (4, 3, 2)
    a_, b_, c_, v, u = 0.3, 0.25, 0.45, 0.07, -0.05
    desc = g.make_desc(n, (2e-9, 2e-9, 2e-9), 8e5)
    Px, Py, Pz, Hx, Ky, Kz = g.gbd_plan_dims(desc)
    spec = g.gbd_kernel_spectrum_from_tensor_host(desc, _sparse_tensor(n, a_, b_, c_, v, u))
    P = Px * Py * Pz
    kz, ky, kx = np.meshgrid(np.arange(Kz), np.arange(Ky), np.arange(Hx), indexing="ij")
    sx, sy, sz = np.sin(2 * np.pi * kx / Px), np.sin(2 * np.pi * ky / Py), np.sin(2 * np.pi * kz / Pz)
    want = np.stack([np.full(kx.shape, -a_ / P), np.full(kx.shape, -b_ / P), np.full(kx.shape, -c_ / P),
                     4 * v * sx * sy / P, 4 * u * sx * sz / P, np.zeros(kx.shape)])
    assert np.abs(spec - want).max() <= 1e-15


def test_caller_tensor_checks(g):
    n = (4, 3, 2)
    desc = g.make_desc(n, (2e-9, 2e-9, 2e-9), 8e5)
    N6 = _sparse_tensor(n, 0.3, 0.3, 0.4, 0.1, 0.1)
    bad = N6.copy()
    bad[3, 1, 2, 4] = -bad[3, 1, 2, 4] + 0.01        # breaks the oddness of xy in X
    with pytest.raises(g.GbdError) as ei:
        g.gbd_kernel_spectrum_from_tensor_host(desc, bad)
    assert ei.value.status == g.GBD_EINVAL
    bad = N6.copy()
    bad[0, 0, 0, 0] = np.nan
    with pytest.raises(g.GbdError) as ei:
        g.gbd_kernel_spectrum_from_tensor_host(desc, bad)
    assert ei.value.status == g.GBD_EINVAL
    bad = N6.copy()
    bad[3, 1, 2, 3] = 0.2                             # xy must vanish at X = 0
    bad[3, 1, 0, 3] = -0.2
    bad[3, 1, 4, 3] = 0.2
    with pytest.raises(g.GbdError):
        g.gbd_kernel_spectrum_from_tensor_host(desc, bad)
    with pytest.raises(ValueError):
        g.gbd_kernel_spectrum_from_tensor_host(desc, N6[:, :, :, :-1])


# ---- periodic boundary conditions ----------------------------------------------------------

@pytest.mark.parametrize("n,pbc,images", [((16, 8, 1), (True, True, False), 3), ((16, 12, 4), (True, False, False), 2),
                                          ((8, 8, 4), (False, False, True), 2), ((4, 8, 4), (True, True, True), 1)])
def test_periodic_spectrum_matches_oracle(g, n, pbc, images):
    from oracle import pbc as B
    cell = (2e-9, 3e-9, 2.5e-9)
    desc = g.make_desc(n, cell, 8e5, pbc=pbc, pbc_images=images)
    Px, Py, Pz, Hx, Ky, Kz = g.gbd_plan_dims(desc)
    assert (Px, Py, Pz) == tuple(n[d] if pbc[d] else (1 if n[d] == 1 and d > 0 else max(2, 1 << (2 * n[d] - 2).bit_length()))
                                 for d in range(3))
    spec = g.gbd_kernel_spectrum_host(desc)
    Kg = B.periodic_kernel(n, cell, pbc, images)
    P = (Px, Py, Pz)
    Kp = np.zeros((6, Pz, Py, Px))
    idx = [np.arange(Kg.shape[3 - d]) if pbc[d] else (np.arange(Kg.shape[3 - d]) - (n[d] - 1)) % P[d] for d in range(3)]
    for c in range(6):
        Kp[c][np.ix_(idx[2], idx[1], idx[0])] = Kg[c]
    Kh = np.fft.fftn(Kp, axes=(1, 2, 3))
    assert np.abs(Kh.imag).max() <= 1e-10 * np.abs(Kh).max()
    want = -Kh.real[:, :Kz, :Ky, :Hx] / (Px * Py * Pz)
    if n[2] == 1:
        want[4:] = 0.0
    assert np.abs(spec - want).max() <= 1e-8 * np.abs(want).max()


def test_periodic_desc_checks(g):
    cell = (2e-9, 2e-9, 2e-9)
    with pytest.raises(g.GbdError) as ei:          # a periodic axis needs a power of two
        g.gbd_plan_dims(g.make_desc((12, 8, 1), cell, 8e5, pbc=(True, False, False), pbc_images=2))
    assert ei.value.status == g.GBD_EUNSUPPORTED
    with pytest.raises(g.GbdError) as ei:          # images >= 1 with a periodic axis
        g.gbd_plan_dims(g.make_desc((16, 8, 1), cell, 8e5, pbc=(True, False, False), pbc_images=0))
    assert ei.value.status == g.GBD_EINVAL
    d = g.make_desc((16, 8, 1), cell, 8e5)
    d.flags = 64
    with pytest.raises(g.GbdError) as ei:
        g.gbd_plan_dims(d)
    assert ei.value.status == g.GBD_EINVAL
    for n, pbc in (((16, 2, 1), (True, True, False)), ((8, 8, 2), (False, False, True))):
        with pytest.raises(g.GbdError) as ei:      # no length-2 y or z transforms
            g.gbd_plan_dims(g.make_desc(n, cell, 8e5, pbc=pbc, pbc_images=2))
        assert ei.value.status == g.GBD_EUNSUPPORTED


def _periodic_fft_spectrum(Kg, n, pbc, dims):
    """numpy FFT of a tensor on the convolution grid (one period along periodic axes, offsets
    1-n .. n-1 along the others), placed on the padded lengths, packed and scaled."""
    Px, Py, Pz, Hx, Ky, Kz = dims
    P = (Px, Py, Pz)
    Kp = np.zeros((6, Pz, Py, Px))
    idx = [np.arange(Kg.shape[3 - d]) if pbc[d] else (np.arange(Kg.shape[3 - d]) - (n[d] - 1)) % P[d] for d in range(3)]
    for c in range(6):
        Kp[c][np.ix_(idx[2], idx[1], idx[0])] = Kg[c]
    Kh = np.fft.fftn(Kp, axes=(1, 2, 3))
    want = -Kh.real[:, :Kz, :Ky, :Hx] / (Px * Py * Pz)
    if n[2] == 1:
        want[4:] = 0.0
    return want


@pytest.mark.parametrize("n,pbc,images", [((16, 8, 1), (True, True, False), 2), ((16, 12, 4), (True, False, False), 1),
                                          ((8, 8, 4), (False, False, True), 1), ((4, 8, 4), (True, True, True), 1)])
def test_periodic_caller_tensor_spectrum(g, n, pbc, images):
    # one period of the oracle's image-summed tensor through the caller path equals numpy's FFT of
    # it, and the built-in periodic spectrum to the two image sums' agreement
    from oracle import pbc as B
    cell = (2e-9, 3e-9, 2.5e-9)
    desc = g.make_desc(n, cell, 8e5, pbc=pbc, pbc_images=images)
    dims = g.gbd_plan_dims(desc)
    Kg = B.periodic_kernel(n, cell, pbc, images)
    spec = g.gbd_kernel_spectrum_from_tensor_host(desc, Kg)
    want = _periodic_fft_spectrum(Kg, n, pbc, dims)
    assert np.abs(spec - want).max() <= 1e-12 * np.abs(want).max()
    assert np.abs(spec - g.gbd_kernel_spectrum_host(desc)).max() <= 1e-8 * np.abs(want).max()


def test_periodic_caller_tensor_checks(g):
    from oracle import pbc as B
    n, pbc, cell = (8, 4, 1), (True, False, False), (2e-9, 2e-9, 3e-9)
    desc = g.make_desc(n, cell, 8e5, pbc=pbc, pbc_images=1)
    Kg = B.periodic_kernel(n, cell, pbc, 1)
    assert Kg.shape == (6, 1, 7, 8)
    g.gbd_kernel_spectrum_from_tensor_host(desc, Kg)
    bad = Kg.copy()
    bad[3, 0, 4, 4] += 1e-3 * np.abs(Kg).max()         # xy is odd in X: it vanishes at X = n/2
    bad[3, 0, 2, 4] -= 1e-3 * np.abs(Kg).max()
    with pytest.raises(g.GbdError) as ei:
        g.gbd_kernel_spectrum_from_tensor_host(desc, bad)
    assert ei.value.status == g.GBD_EINVAL
    bad = Kg.copy()
    bad[0, 0, 3, 1] += 1e-3 * np.abs(Kg).max()         # xx at X = 1 without its mirror X = 7
    with pytest.raises(g.GbdError) as ei:
        g.gbd_kernel_spectrum_from_tensor_host(desc, bad)
    assert ei.value.status == g.GBD_EINVAL
    with pytest.raises(ValueError):                    # open-boundary shape on a periodic axis
        g.gbd_kernel_spectrum_from_tensor_host(desc, np.zeros((6, 1, 7, 15)))


def test_precision_values(g):
    cell = (2e-9, 2e-9, 2e-9)
    for prec in (g.GBD_FP32, g.GBD_SPLIT_BF16, g.GBD_SPLIT_FP16):
        assert g.gbd_plan_dims(g.make_desc((64, 32, 4), cell, 8e5, precision=prec))[:3] == (128, 64, 8)
    for prec in (-1, 3):
        with pytest.raises(g.GbdError) as ei:
            g.gbd_plan_dims(g.make_desc((64, 32, 4), cell, 8e5, precision=prec))
        assert ei.value.status == g.GBD_EINVAL
