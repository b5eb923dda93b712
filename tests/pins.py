"""Closed forms from the literature that pin the oracle (independent of its code)."""
import math


def aharoni_Dz(a, b, c):
    """Aharoni's demagnetizing factor along z of a prism 2a x 2b x 2c (J. Appl. Phys. 83, 3432)."""
    r = math.sqrt(a * a + b * b + c * c)
    ab, bc, ac = math.hypot(a, b), math.hypot(b, c), math.hypot(a, c)
    t = ((b * b - c * c) / (2 * b * c) * math.log((r - a) / (r + a))
         + (a * a - c * c) / (2 * a * c) * math.log((r - b) / (r + b))
         + b / (2 * c) * math.log((ab + a) / (ab - a))
         + a / (2 * c) * math.log((ab + b) / (ab - b))
         + c / (2 * a) * math.log((bc - b) / (bc + b))
         + c / (2 * b) * math.log((ac - a) / (ac + a))
         + 2 * math.atan(a * b / (c * r))
         + (a ** 3 + b ** 3 - 2 * c ** 3) / (3 * a * b * c)
         + (a * a + b * b - 2 * c * c) / (3 * a * b * c) * r
         + c / (a * b) * (ac + bc)
         - (ab ** 3 + bc ** 3 + ac ** 3) / (3 * a * b * c))
    return t / math.pi


def aharoni_factors(Lx, Ly, Lz):
    """(Dx, Dy, Dz) of an Lx x Ly x Lz prism."""
    a, b, c = Lx / 2, Ly / 2, Lz / 2
    return aharoni_Dz(b, c, a), aharoni_Dz(c, a, b), aharoni_Dz(a, b, c)


def prism_centre_Nzz(Lx, Ly, Lz):
    """N_zz at the centre point of a uniformly magnetized Lx x Ly x Lz prism:
    (2/pi) atan(a b / (c sqrt(a^2 + b^2 + c^2))) with half-sides a, b, c (the two charged
    faces z = +-c seen from the centre, each subtending solid angle Omega = 4 atan(...))."""
    a, b, c = Lx / 2, Ly / 2, Lz / 2
    return 2.0 / math.pi * math.atan(a * b / (c * math.sqrt(a * a + b * b + c * c)))
