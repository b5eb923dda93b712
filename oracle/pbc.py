"""Periodic boundary conditions for the demag convolution and the exchange field in FP64 (oracle;
test infrastructure).

Sec. II notes that periodic boundary conditions need a modified convolution kernel (Ref. [25],
which the paper does not reproduce) and no zero padding along the periodic direction. Reading:

* along a periodic axis d the magnetization repeats with period n_d cells, and the convolution
  along d is circular of length n_d (no padding); along the other axes it is zero padded as in
  ``oracle.conv``;
* the kernel along a periodic axis is the demag tensor summed over K images on each side: at
  index b in [0, n_d) with signed offset s = b (b < n_d/2) or b - n_d (b > n_d/2),
  N_per = sum_{i=-K..K} N(s + i n_d); at b = n_d/2 (even n_d) the image sets of +n_d/2 and
  -n_d/2 are averaged, so every component keeps its parity (the odd ones vanish there);
* the exchange Laplacian wraps around a periodic axis.

Arrays are [component, z, y, x]; ``per`` is (px, py, pz) booleans.
"""
import numpy as np

from . import GAMMA
from .llg import llg_rhs, rk4_step
from .tensor import demag_tensor

_AB = [[0, 3, 4], [3, 1, 5], [4, 5, 2]]


def _axis_terms(n, periodic, K):
    """Per grid index b of one axis: the list of (offset, weight) whose tensor values sum there.

    Periodic: grid [0, n), images of the signed offset. Not periodic: grid of the offsets
    -(n-1) .. n-1 at index X + n - 1, one term each."""
    if not periodic:
        return [[(b - (n - 1), 1.0)] for b in range(2 * n - 1)]
    out = []
    for b in range(n):
        if 2 * b == n:
            terms = [(s + i * n, 0.5) for s in (b, -b) for i in range(-K, K + 1)]
        else:
            s = b if 2 * b < n else b - n
            terms = [(s + i * n, 1.0) for i in range(-K, K + 1)]
        out.append(terms)
    return out


def periodic_kernel(n, cell, per, K):
    """The kernel on the convolution grid: (6, Gz, Gy, Gx), G_d = n_d on periodic axes (index
    X mod n_d), 2 n_d - 1 on the others (index X + n_d - 1); image sums as in the reading."""
    dx, dy, dz = cell
    terms = [_axis_terms(n[d], per[d], K) for d in range(3)]
    offs = [sorted({o for t in terms[d] for o, _ in t}) for d in range(3)]
    pos = [{o: i for i, o in enumerate(offs[d])} for d in range(3)]
    # weight matrices: grid index x offset
    W = []
    for d in range(3):
        w = np.zeros((len(terms[d]), len(offs[d])))
        for b, t in enumerate(terms[d]):
            for o, wt in t:
                w[b, pos[d][o]] += wt
        W.append(w)
    Z, Y, X = np.meshgrid(np.array(offs[2], float), np.array(offs[1], float), np.array(offs[0], float),
                          indexing="ij")
    T = demag_tensor(X, Y, Z, dx, dy, dz)                   # (6, |Oz|, |Oy|, |Ox|)
    return np.einsum("zZ,yY,xX,cZYX->czyx", W[2], W[1], W[0], T)


def conv_periodic(M, Kgrid, per):
    """H = -N * M (Eq. 1) with circular convolution along periodic axes and zero padding (P = 2n)
    along the others; full complex FFTs."""
    _, nz, ny, nx = M.shape
    n = (nx, ny, nz)
    P = tuple(n[d] if per[d] else 2 * n[d] for d in range(3))
    Kp = np.zeros((6, P[2], P[1], P[0]))
    idx = []
    for d in range(3):
        G = Kgrid.shape[3 - d]
        idx.append(np.arange(G) if per[d] else (np.arange(G) - (n[d] - 1)) % P[d])
    for c in range(6):
        Kp[c][np.ix_(idx[2], idx[1], idx[0])] = Kgrid[c]
    Kh = np.fft.fftn(Kp, axes=(1, 2, 3))
    Mp = np.zeros((3, P[2], P[1], P[0]))
    Mp[:, :nz, :ny, :nx] = M
    Mh = np.fft.fftn(Mp, axes=(1, 2, 3))
    Hh = np.zeros_like(Mh)
    for a in range(3):
        for b in range(3):
            Hh[a] += Kh[_AB[a][b]] * Mh[b]
    return -np.fft.ifftn(Hh, axes=(1, 2, 3)).real[:, :nz, :ny, :nx]


def laplacian(m, cell, per):
    """sum_d (m_{i+e_d} - 2 m_i + m_{i-e_d}) / d_d^2: periodic wrap on periodic axes, the cell
    itself for a missing neighbour on the others."""
    dx, dy, dz = cell
    out = np.zeros_like(m)
    for axis, d, p in ((3, dx, per[0]), (2, dy, per[1]), (1, dz, per[2])):
        n = m.shape[axis]
        if n == 1:
            continue
        if p:
            up, dn = np.roll(m, -1, axis=axis), np.roll(m, 1, axis=axis)
        else:
            up = np.concatenate([np.take(m, range(1, n), axis=axis), np.take(m, [n - 1], axis=axis)], axis=axis)
            dn = np.concatenate([np.take(m, [0], axis=axis), np.take(m, range(0, n - 1), axis=axis)], axis=axis)
        out += (up - 2.0 * m + dn) / (d * d)
    return out


def effective_field(m, Kgrid, cell, Ms, A, per, Hext=(0.0, 0.0, 0.0)):
    """H_eff = H_d(Ms m) + H_ex(m) + H_ext with the periodic convolution and Laplacian."""
    from . import MU0
    H = conv_periodic(Ms * m, Kgrid, per) + (2.0 * A / (MU0 * Ms)) * laplacian(m, cell, per)
    for c in range(3):
        H[c] += Hext[c]
    return H


def llg_run(m, nsteps, dt, Kgrid, cell, Ms, A, alpha, per, Hext=(0.0, 0.0, 0.0), gamma=GAMMA):
    """nsteps RK4 steps (as oracle.llg.rk4_step) with periodic demag and exchange."""
    f = lambda v: llg_rhs(v, effective_field(v, Kgrid, cell, Ms, A, per, Hext), alpha, gamma)
    for _ in range(nsteps):
        m = rk4_step(m, dt, f)
    return m

