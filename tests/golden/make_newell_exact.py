"""Writes newell_exact.txt: the cell-averaged demag tensor at chosen cell offsets, in 60-digit arithmetic.

The values come from ``oracle.newell_mp`` (closed-form Newell stencil evaluated
with mpmath), the tensor that Sec. II cites for Eq. 1. They pin the FP64 tensor
of ``oracle.tensor`` -- both its near-field rounding and its far-field
quadrature -- to the exact integral. Run from the repository root:

    python tests/golden/make_newell_exact.py
"""
import os
import sys

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "..", ".."))
from oracle.newell_mp import newell_exact_mp  # noqa: E402

# (cell in nm, integer offsets): cubes, the 2x2x3 nm film cell, a needle-like cell.
CASES = [
    ((4, 4, 4), [(0, 0, 0), (1, 0, 0), (1, 1, 0), (1, 1, 1), (3, -2, 1), (7, 0, 0), (5, 5, 4),
                 (9, -3, 2), (14, 6, -5), (30, -20, 10), (60, 33, -17), (120, -70, 31), (300, 150, 40)]),
    ((2, 2, 3), [(0, 0, 0), (1, 0, 0), (0, 0, 1), (2, -1, 0), (11, 5, 0), (13, 0, 0), (25, -17, 0),
                 (40, 22, 0), (100, -3, 0), (400, 250, 0), (1023, 1023, 0)]),
    ((1, 1, 5), [(0, 0, 0), (1, 0, 0), (0, 0, 1), (4, 3, 1), (30, 10, 2), (90, -40, 3)]),
]


def main():
    out = os.path.join(os.path.dirname(__file__), "newell_exact.txt")
    with open(out, "w") as fh:
        fh.write("# Cell-averaged demag tensor (Newell et al. 1993; cited for Eq. 1, Sec. II), exact to\n")
        fh.write("# ~50 digits: columns dx dy dz [nm]  X Y Z [cells]  Nxx Nyy Nzz Nxy Nxz Nyz.\n")
        fh.write("# Written by tests/golden/make_newell_exact.py (oracle.newell_mp, mpmath dps=60).\n")
        for cell, offs in CASES:
            for (X, Y, Z) in offs:
                vals = newell_exact_mp(X * cell[0], Y * cell[1], Z * cell[2], *cell)
                fh.write("%d %d %d %d %d %d %s\n" % (cell + (X, Y, Z) + (" ".join("%.20e" % float(v) for v in vals),)))
    print("wrote", out)


if __name__ == "__main__":
    main()
