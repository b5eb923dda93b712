"""The closed-form cell-averaged tensor in arbitrary precision (oracle; test infrastructure).

Same antiderivatives and 27-point stencil as ``oracle.tensor.newell_exact``
(Newell, Williams and Dunlop 1993, the formulas Sec. II cites for Eq. 1), but
carried out in mpmath with 60 significant digits, so that the stencil's
cancellation costs nothing. It is used only to write the golden file that pins
the FP64 tensor (near-field rounding and far-field quadrature) to the exact
integral.
"""
import mpmath as mp

mp.mp.dps = 60


def _f(x, y, z):
    x, y, z = abs(x), abs(y), abs(z)
    R = mp.sqrt(x * x + y * y + z * z)
    t = mp.mpf(0)
    if y != 0 and (x != 0 or z != 0):
        t += y * (z * z - x * x) * mp.asinh(y / mp.sqrt(x * x + z * z)) / 2
    if z != 0 and (x != 0 or y != 0):
        t += z * (y * y - x * x) * mp.asinh(z / mp.sqrt(x * x + y * y)) / 2
    if x != 0 and y != 0 and z != 0:
        t -= x * y * z * mp.atan(y * z / (x * R))
    t += (2 * x * x - y * y - z * z) * R / 6
    return t


def _g(x, y, z):
    s = mp.sign(x) * mp.sign(y)
    x, y, z = abs(x), abs(y), abs(z)
    R = mp.sqrt(x * x + y * y + z * z)
    t = mp.mpf(0)
    if z != 0 and (x != 0 or y != 0):
        t += x * y * z * mp.asinh(z / mp.sqrt(x * x + y * y))
    if x != 0 and (y != 0 or z != 0):
        t += y * (3 * z * z - y * y) * mp.asinh(x / mp.sqrt(y * y + z * z)) / 6
    if y != 0 and (x != 0 or z != 0):
        t += x * (3 * z * z - x * x) * mp.asinh(y / mp.sqrt(x * x + z * z)) / 6
    if x != 0 and y != 0 and z != 0:
        t -= z ** 3 * mp.atan(x * y / (z * R)) / 6
        t -= z * y * y * mp.atan(x * z / (y * R)) / 2
        t -= z * x * x * mp.atan(y * z / (x * R)) / 2
    t -= x * y * R / 3
    return s * t


def _stencil(F, X, Y, Z, dx, dy, dz):
    w = {-1: -1, 0: 2, 1: -1}
    acc = mp.mpf(0)
    for i in (-1, 0, 1):
        for j in (-1, 0, 1):
            for k in (-1, 0, 1):
                acc += w[i] * w[j] * w[k] * F(X + i * dx, Y + j * dy, Z + k * dz)
    return acc / (4 * mp.pi * dx * dy * dz)


def newell_exact_mp(X, Y, Z, dx, dy, dz):
    """(xx, yy, zz, xy, xz, yz) at physical offset (X, Y, Z); arguments as decimal strings or numbers."""
    X, Y, Z, dx, dy, dz = (mp.mpf(v) for v in (X, Y, Z, dx, dy, dz))
    return (
        _stencil(_f, X, Y, Z, dx, dy, dz),
        _stencil(_f, Y, X, Z, dy, dx, dz),
        _stencil(_f, Z, Y, X, dz, dy, dx),
        _stencil(_g, X, Y, Z, dx, dy, dz),
        _stencil(_g, X, Z, Y, dx, dz, dy),
        _stencil(_g, Y, Z, X, dy, dz, dx),
    )
