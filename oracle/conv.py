"""Eq. 1 of Sec. II in FP64: direct sum and zero-padded FFT convolution (oracle; test infrastructure).

Arrays are indexed [component, z, y, x] with component order (x, y, z); M and H
are in A/m. The tensor comes from ``oracle.tensor.tensor_all_offsets`` with
index X + n_x - 1 (and likewise for y, z).
"""
import numpy as np

# (a, b) -> tensor component index in (xx, yy, zz, xy, xz, yz)
_AB = [[0, 3, 4], [3, 1, 5], [4, 5, 2]]


def direct_sum(M, Nfull):
    """H_i = -sum_j N(i - j) M_j over all cells j (Eq. 1), O(N^2), for small meshes."""
    _, nz, ny, nx = M.shape
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    zz, yy, xx = zz.ravel(), yy.ravel(), xx.ravel()
    Mf = M.reshape(3, -1)
    H = np.zeros_like(Mf)
    block = 256
    for i0 in range(0, xx.size, block):
        i = slice(i0, min(i0 + block, xx.size))
        # offsets i - j for a block of targets i and every source j
        oz = zz[i, None] - zz[None, :] + nz - 1
        oy = yy[i, None] - yy[None, :] + ny - 1
        ox = xx[i, None] - xx[None, :] + nx - 1
        for a in range(3):
            acc = np.zeros(oz.shape[0])
            for b in range(3):
                acc += (Nfull[_AB[a][b]][oz, oy, ox] * Mf[b][None, :]).sum(axis=1)
            H[a, i] = -acc
    return H.reshape(M.shape)


def padded_length(n):
    """The paper's padded length N_d = 2 n_d (Sec. II), and 1 where n_d = 1 (no padding needed)."""
    return 1 if n == 1 else 2 * n


def place_kernel(Nfull, n, P):
    """Spatial kernel on the periodic grid P: N(X) at X mod P_d for |X_d| <= n_d - 1, else 0."""
    nx, ny, nz = n
    Px, Py, Pz = P
    K = np.zeros((6, Pz, Py, Px))
    zi = np.arange(-(nz - 1), nz) % Pz
    yi = np.arange(-(ny - 1), ny) % Py
    xi = np.arange(-(nx - 1), nx) % Px
    for c in range(6):
        K[c][np.ix_(zi, yi, xi)] = Nfull[c]
    return K


def fft_conv(M, Nfull, P=None):
    """Eq. 1 as a zero-padded FFT convolution, steps in the order of Appendix A with one GPU.

    In = M zero padded to P; x R2C; y FFT; z FFT; multiply by the transformed
    kernel; z IFFT; y IFFT; x C2R; keep the first n_d points; H = -result.
    Any P_d >= 2 n_d - 1 gives the same cropped result (no circular wrap).
    """
    _, nz, ny, nx = M.shape
    n = (nx, ny, nz)
    if P is None:
        P = tuple(padded_length(v) for v in n)
    Px, Py, Pz = P
    assert Px >= 2 * nx - 1 and Py >= 2 * ny - 1 and Pz >= 2 * nz - 1
    # Convolution kernel: transform of the placed tensor (same axis order as the data).
    Kt = place_kernel(Nfull, n, P)
    Kh = np.fft.fft(np.fft.fft(np.fft.rfft(Kt, axis=3), axis=2), axis=1)
    # Forward pipeline.
    In = np.zeros((3, nz, ny, Px))
    In[..., :nx] = M
    S1 = np.fft.rfft(In, axis=3)                       # (3, nz, ny, Px/2+1)
    S2 = np.zeros((3, Pz, Py, S1.shape[3]), complex)
    S2[:, :nz, :ny, :] = S1
    S2 = np.fft.fft(S2, axis=2)                        # y
    S2 = np.fft.fft(S2, axis=1)                        # z
    # Kernel multiplication: H~_a = sum_b N~_ab M~_b.
    R2 = np.zeros_like(S2)
    for a in range(3):
        for b in range(3):
            R2[a] += Kh[_AB[a][b]] * S2[b]
    R2 = np.fft.ifft(R2, axis=1)                       # z
    R2 = np.fft.ifft(R2, axis=2)                       # y
    S1o = R2[:, :nz, :ny, :]
    Out = np.fft.irfft(S1o, n=Px, axis=3)
    return -Out[..., :nx]
