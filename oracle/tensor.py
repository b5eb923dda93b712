"""Cell-averaged demagnetizing tensor N(X, Y, Z) in FP64 (oracle; test infrastructure).

Sec. II, Eq. 1 writes H_d,i = -sum_j N(i-j) M_j with N "computed using the
formulas in Ref. [23]". That reference is the cell-averaged tensor of two
uniformly magnetized rectangular cells (Newell, Williams and Dunlop, J. Geophys.
Res. 98, 9551 (1993)): N(R) = (1/V) * int_cell_i int_cell_j K(r - r') with the
point-dipole kernel K(r) = (I - 3 r r^T / r^2) / (4 pi r^3), so that a dipole
field is H = -K m.

Near field (|R| < 8 d_max): the closed form. Each component is a 27-point
second-difference stencil (weights 2, -1, -1 along each axis) of an
antiderivative f (diagonal) or g (off-diagonal), divided by 4 pi dx dy dz.

Far field (|R| >= 8 d_max): in FP64 the 27-point stencil cancels away the
leading digits (relative error ~1e-9 at 10 cells, growing as R^2). There the
same integral is evaluated by quadrature: with u = r - r' - R, the overlap of
two boxes gives N(R) = int prod_d (1 - |u_d|/d_d) K(R + u) du over
|u_d| <= d_d, split at u_d = 0 and integrated by G-point Gauss-Legendre per
half-axis; G = 4, 3, 2 for |R| < 16, < 64, >= 64 d_max. Against the closed form
evaluated in 60-digit arithmetic, both branches are within 2e-8 of
|V/(4 pi |R|^3)| per element (the golden file under tests/golden pins this).

Components are indexed (xx, yy, zz, xy, xz, yz). Diagonal ones are even in X,
Y and Z; N_xy is odd in X and Y and even in Z, N_xz odd in X and Z, N_yz odd in
Y and Z.
"""
import math

import numpy as np

COMPONENTS = ("xx", "yy", "zz", "xy", "xz", "yz")
R_NEAR = 8.0     # closed-form stencil below this distance, in units of max cell side
R_G4 = 16.0      # 4 Gauss-Legendre nodes per half-axis below this distance
R_G3 = 64.0      # 3 nodes below this, 2 nodes beyond


def _safe_div(a, b):
    """a / b where b != 0, else 0 (the term it feeds has a zero prefactor there)."""
    out = np.zeros(np.broadcast(a, b).shape)
    np.divide(a, b, out=out, where=(b != 0))
    return out


def newell_f(x, y, z):
    """Antiderivative for N_xx (Newell et al. 1993), evaluated on |x|, |y|, |z|.

    f = y/2 (z^2 - x^2) asinh(y / sqrt(x^2 + z^2))
      + z/2 (y^2 - x^2) asinh(z / sqrt(x^2 + y^2))
      - x y z atan(y z / (x R)) + (2 x^2 - y^2 - z^2) R / 6,   R = |(x, y, z)|.
    A term whose prefactor vanishes where its argument is 0/0 is taken as 0.
    """
    x, y, z = np.abs(x), np.abs(y), np.abs(z)
    x2, y2, z2 = x * x, y * y, z * z
    R = np.sqrt(x2 + y2 + z2)
    t = 0.5 * y * (z2 - x2) * np.arcsinh(_safe_div(y, np.sqrt(x2 + z2)))
    t = t + 0.5 * z * (y2 - x2) * np.arcsinh(_safe_div(z, np.sqrt(x2 + y2)))
    t = t - x * y * z * np.arctan(_safe_div(y * z, x * R))
    t = t + (2.0 * x2 - y2 - z2) * R / 6.0
    return t


def newell_g(x, y, z):
    """Antiderivative for N_xy (Newell et al. 1993): g(|x|,|y|,|z|) * sign(x) sign(y).

    g = x y z asinh(z / sqrt(x^2 + y^2)) + y/6 (3 z^2 - y^2) asinh(x / sqrt(y^2 + z^2))
      + x/6 (3 z^2 - x^2) asinh(y / sqrt(x^2 + z^2)) - z^3/6 atan(x y / (z R))
      - z y^2/2 atan(x z / (y R)) - z x^2/2 atan(y z / (x R)) - x y R / 3.
    """
    s = np.sign(x) * np.sign(y)
    x, y, z = np.abs(x), np.abs(y), np.abs(z)
    x2, y2, z2 = x * x, y * y, z * z
    R = np.sqrt(x2 + y2 + z2)
    t = x * y * z * np.arcsinh(_safe_div(z, np.sqrt(x2 + y2)))
    t = t + y / 6.0 * (3.0 * z2 - y2) * np.arcsinh(_safe_div(x, np.sqrt(y2 + z2)))
    t = t + x / 6.0 * (3.0 * z2 - x2) * np.arcsinh(_safe_div(y, np.sqrt(x2 + z2)))
    t = t - z2 * z / 6.0 * np.arctan(_safe_div(x * y, z * R))
    t = t - z * y2 / 2.0 * np.arctan(_safe_div(x * z, y * R))
    t = t - z * x2 / 2.0 * np.arctan(_safe_div(y * z, x * R))
    t = t - x * y * R / 3.0
    return s * t


def _stencil(F, X, Y, Z, dx, dy, dz):
    """(1 / (4 pi dx dy dz)) * sum_{i,j,k in -1,0,1} w_i w_j w_k F(X+i dx, Y+j dy, Z+k dz),
    with w_0 = 2 and w_{+-1} = -1."""
    w = {-1: -1.0, 0: 2.0, 1: -1.0}
    acc = np.zeros(np.broadcast(X, Y, Z).shape)
    for i in (-1, 0, 1):
        for j in (-1, 0, 1):
            for k in (-1, 0, 1):
                acc = acc + w[i] * w[j] * w[k] * F(X + i * dx, Y + j * dy, Z + k * dz)
    return acc / (4.0 * math.pi * dx * dy * dz)


def newell_exact(X, Y, Z, dx, dy, dz):
    """Closed-form tensor at physical offsets (X, Y, Z) in metres; returns (6, ...) array."""
    X, Y, Z = np.broadcast_arrays(np.asarray(X, float), np.asarray(Y, float), np.asarray(Z, float))
    return np.stack([
        _stencil(newell_f, X, Y, Z, dx, dy, dz),            # xx
        _stencil(newell_f, Y, X, Z, dy, dx, dz),            # yy: x <-> y
        _stencil(newell_f, Z, Y, X, dz, dy, dx),            # zz: x <-> z
        _stencil(newell_g, X, Y, Z, dx, dy, dz),            # xy
        _stencil(newell_g, X, Z, Y, dx, dz, dy),            # xz: y <-> z
        _stencil(newell_g, Y, Z, X, dy, dz, dx),            # yz: (x, y, z) -> (y, z, x)
    ])


def _half_axis_rule(G):
    """Nodes s in [-1, 1] and weights for int_{-1}^{1} (1 - |s|) h(s) ds, G nodes per half."""
    xg, wg = np.polynomial.legendre.leggauss(G)
    s = 0.5 * (xg + 1.0)                 # nodes on [0, 1]
    w = 0.5 * wg * (1.0 - s)             # Gauss-Legendre weight times the overlap weight
    return np.concatenate([-s, s]), np.concatenate([w, w])


def dipole_quadrature(X, Y, Z, dx, dy, dz, G):
    """N(R) = V * int prod_d (1 - |s_d|) K(R + d o s) ds, tensor-product rule; returns (6, ...)."""
    X, Y, Z = np.broadcast_arrays(np.asarray(X, float), np.asarray(Y, float), np.asarray(Z, float))
    s, w = _half_axis_rule(G)
    out = np.zeros((6,) + X.shape)
    V = dx * dy * dz
    for sa, wa in zip(s, w):
        for sb, wb in zip(s, w):
            for sc, wc in zip(s, w):
                rx = X + sa * dx
                ry = Y + sb * dy
                rz = Z + sc * dz
                r2 = rx * rx + ry * ry + rz * rz
                r = np.sqrt(r2)
                c = wa * wb * wc * V / (4.0 * math.pi * r2 * r)
                q = 3.0 / r2
                out[0] += c * (1.0 - q * rx * rx)
                out[1] += c * (1.0 - q * ry * ry)
                out[2] += c * (1.0 - q * rz * rz)
                out[3] += c * (-q * rx * ry)
                out[4] += c * (-q * rx * rz)
                out[5] += c * (-q * ry * rz)
    return out


def demag_tensor(X, Y, Z, dx, dy, dz):
    """Cell-averaged tensor at integer cell offsets (X, Y, Z) (arrays); returns (6, ...) FP64.

    Chooses the closed form or the quadrature per offset by the distance rule in
    the module docstring.
    """
    X, Y, Z = np.broadcast_arrays(np.asarray(X, float), np.asarray(Y, float), np.asarray(Z, float))
    px, py, pz = X * dx, Y * dy, Z * dz
    r = np.sqrt(px * px + py * py + pz * pz) / max(dx, dy, dz)
    out = np.zeros((6,) + X.shape)
    bands = [(r < R_NEAR, None), ((r >= R_NEAR) & (r < R_G4), 4),
             ((r >= R_G4) & (r < R_G3), 3), (r >= R_G3, 2)]
    for mask, G in bands:
        if not mask.any():
            continue
        if G is None:
            out[:, mask] = newell_exact(px[mask], py[mask], pz[mask], dx, dy, dz)
        else:
            out[:, mask] = dipole_quadrature(px[mask], py[mask], pz[mask], dx, dy, dz, G)
    return out


# Parity of each component along (x, y, z): +1 even, -1 odd.
PARITY = np.array([[1, 1, 1], [1, 1, 1], [1, 1, 1],
                   [-1, -1, 1], [-1, 1, -1], [1, -1, -1]])


def tensor_all_offsets(n, cell):
    """N at every offset -n_d < X_d < n_d; returns (6, 2nz-1, 2ny-1, 2nx-1), index X + n_x - 1.

    Evaluated on the octant X, Y, Z >= 0 and extended by the component parities
    (a property of the integral, checked against direct evaluation in the tests).
    """
    nx, ny, nz = n
    dx, dy, dz = cell
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    oct_ = demag_tensor(X, Y, Z, dx, dy, dz)           # (6, nz, ny, nx)
    full = np.zeros((6, 2 * nz - 1, 2 * ny - 1, 2 * nx - 1))
    for c in range(6):
        px, py, pz = PARITY[c]
        for sz in (1, -1):
            for sy in (1, -1):
                for sx in (1, -1):
                    sign = (px if sx < 0 else 1) * (py if sy < 0 else 1) * (pz if sz < 0 else 1)
                    zi = nz - 1 + sz * np.arange(nz)
                    yi = ny - 1 + sy * np.arange(ny)
                    xi = nx - 1 + sx * np.arange(nx)
                    full[c][np.ix_(zi, yi, xi)] = sign * oct_[c]
    return full
