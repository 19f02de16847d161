"""Writes ``gd_exact_small.txt``: exact rational solutions of the 3-D gradient-domain smoothing
(the earlier method's phase 1, Sec. 3 "Alternate Solutions") on tiny stacks.

Run from the repository root:  python tests/golden/make_gd_exact.py

Inputs are fixed integer patterns (8-bit range, no random numbers) with per-slice offsets (the
inter-slice artefact the smoothing removes); alpha values are powers of two or small integers
(exact in FP32 and FP64).  Every expected value comes from ``oracle.exact_small`` (Gaussian
elimination over rationals of the energy's normal equations on the 6-neighbour graph).
"""
from __future__ import annotations

import os
import sys
from fractions import Fraction

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.exact_small import exact_gradient_domain  # noqa: E402

# (name, nz, ny, nx, alpha)
CASES = [
    ("one_slice", 1, 3, 3, Fraction(1, 1024)),
    ("column", 4, 1, 1, Fraction(1, 4)),
    ("cube", 2, 2, 3, Fraction(1, 4)),
    ("tall", 5, 2, 2, Fraction(1, 1024)),
    ("flat", 3, 3, 4, Fraction(1, 16)),
    ("screened", 4, 1, 3, Fraction(3)),
]


def stack(nz, ny, nx):
    """A shared in-plane pattern plus per-slice offsets and a small z-varying detail."""
    return [[[(23 * x + 41 * y + 9 * ((x * y + z) % 3) + 30 * (z % 2) + 11 * z) % 256
              for x in range(nx)] for y in range(ny)] for z in range(nz)]


def main():
    lines = [
        "# Exact minimisers of alpha |f - I|^2 + |grad_xy f - grad_xy I|^2 + |d_z f|^2 on the",
        "# 6-neighbour graph of a stack (Neumann, unit spacing); written by",
        "# tests/golden/make_gd_exact.py (rational Gaussian elimination of the normal equations).",
        "# case <name> <nz> <ny> <nx> <alpha as p/q>, then 'I' (ints) and 'f' (exact fractions",
        "# p/q), both in [z][y][x] order.",
    ]
    for name, nz, ny, nx, alpha in CASES:
        I0 = stack(nz, ny, nx)
        f = exact_gradient_domain(I0, alpha)
        lines.append(f"case {name} {nz} {ny} {nx} {alpha.numerator}/{alpha.denominator}")
        lines.append("I " + " ".join(str(v) for sl in I0 for row in sl for v in row))
        lines.append("f " + " ".join(f"{v.numerator}/{v.denominator}" for sl in f for row in sl for v in row))
    with open(os.path.join(HERE, "gd_exact_small.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
