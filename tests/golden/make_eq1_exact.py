"""Writes ``eq1_exact_small.txt``: exact rational solutions of Eq. (1) on tiny slices.

Run from the repository root:  python tests/golden/make_eq1_exact.py

The inputs are fixed integer patterns (8-bit range, no random numbers), alpha values are
powers of two or small integers (exactly representable in FP32 and FP64, so a GPU solve
sees the same problem), and every expected value comes from ``oracle.exact_small`` (Gaussian
elimination over rationals of the energy's normal equations, Sec. 3 "Screened-Poisson
Blending").
"""
from __future__ import annotations

import os
import sys
from fractions import Fraction

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.exact_small import exact_solve  # noqa: E402

# (name, ny, nx, alpha)
CASES = [
    ("one_pixel", 1, 1, Fraction(1, 1024)),
    ("row", 1, 6, Fraction(1, 16)),
    ("column", 5, 1, Fraction(3)),
    ("square", 3, 3, Fraction(1, 1024)),
    ("ragged", 4, 7, Fraction(1, 16)),
    ("wide", 5, 9, Fraction(1, 1024)),
    ("stiff", 6, 6, Fraction(1, 4096)),
]


def inputs(ny, nx):
    """s: a smooth ramp plus a step; o: a different pattern with edges (both 0..255 ints)."""
    s = [[(37 * x + 23 * y + (60 if x >= nx // 2 else 0)) % 256 for x in range(nx)] for y in range(ny)]
    o = [[(11 * x * x + 53 * y + 17 * ((x + y) % 3)) % 256 for x in range(nx)] for y in range(ny)]
    return s, o


def main():
    lines = [
        "# Exact solutions of Eq. (1), (alpha I - Lap) f = alpha s - Lap o, Neumann 4-neighbour",
        "# Laplacian, unit spacing; written by tests/golden/make_eq1_exact.py (rational Gaussian",
        "# elimination of the energy's normal equations, Sec. 3 \"Screened-Poisson Blending\").",
        "# case <name> <ny> <nx> <alpha as p/q>, then rows 's', 'o' (ints, row-major) and",
        "# 'f' (exact fractions p/q, row-major).",
    ]
    for name, ny, nx, alpha in CASES:
        s, o = inputs(ny, nx)
        f = exact_solve(s, o, alpha)
        lines.append(f"case {name} {ny} {nx} {alpha.numerator}/{alpha.denominator}")
        lines.append("s " + " ".join(str(v) for row in s for v in row))
        lines.append("o " + " ".join(str(v) for row in o for v in row))
        lines.append("f " + " ".join(f"{v.numerator}/{v.denominator}" for row in f for v in row))
    with open(os.path.join(HERE, "eq1_exact_small.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
