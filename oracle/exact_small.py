"""Exact rational solutions of Eq. (1) on tiny slices (test infrastructure only).

TEST INFRASTRUCTURE ONLY.  Used by ``tests/golden/make_eq1_exact.py`` to write the stored
expected values under ``tests/golden/``; the CUDA library never calls it and shares nothing
with it.

What it computes: the minimiser of the discrete screened-Poisson energy of Sec. 3
"Screened-Poisson Blending",

    E(f) = alpha sum_p (f_p - s_p)^2 + sum_{edges pq} ((f_p - f_q) - (o_p - o_q))^2,

over the 4-neighbour edges of an ny x nx slice (Neumann boundaries: no edge leaves the
slice).  Setting dE/df_p = 0 gives, row by row,

    alpha f_p + sum_{q ~ p} (f_p - f_q) = alpha s_p + sum_{q ~ p} (o_p - o_q),

i.e. Eq. (1) with the graph Laplacian, assembled here edge by edge and solved by Gaussian
elimination over ``fractions.Fraction``, so the result carries no rounding at all.  It is
independent of the DCT solve in ``emfuse_oracle`` (no transform, no eigenvalues).

``exact_gradient_domain`` does the same for the 3-D gradient-domain smoothing of the earlier
method (Sec. 3 "Alternate Solutions": target gradients with their z-components zeroed),
minimising alpha sum (f - I0)^2 + sum over x/y edges ((f_p - f_q) - (I0_p - I0_q))^2 +
sum over z edges (f_p - f_q)^2 on the 6-neighbour graph of a tiny stack.
"""
from __future__ import annotations

from fractions import Fraction

__all__ = ["exact_solve", "exact_gradient_domain"]


def _solve_spd(A, b):
    """Gaussian elimination over Fractions (A symmetric positive definite: pivots > 0)."""
    n = len(b)
    for k in range(n):
        piv = A[k][k]
        if piv == 0:
            raise ArithmeticError("zero pivot")
        for i in range(k + 1, n):
            if A[i][k] != 0:
                m = A[i][k] / piv
                row_i, row_k = A[i], A[k]
                for j in range(k, n):
                    if row_k[j] != 0:
                        row_i[j] -= m * row_k[j]
                b[i] -= m * b[k]
    f = [Fraction(0)] * n
    for k in range(n - 1, -1, -1):
        acc = b[k]
        for j in range(k + 1, n):
            acc -= A[k][j] * f[j]
        f[k] = acc / A[k][k]
    return f


def exact_gradient_domain(I0, alpha):
    """Exact smoothed stack for a tiny stack ``I0`` (nz x ny x nx nested lists of ints or
    Fractions) and a positive Fraction ``alpha``; returns nested lists of Fractions."""
    alpha = Fraction(alpha)
    if alpha <= 0:
        raise ValueError("alpha must be > 0")
    nz, ny, nx = len(I0), len(I0[0]), len(I0[0][0])
    n = nz * ny * nx
    idx = lambda z, y, x: (z * ny + y) * nx + x
    A = [[Fraction(0)] * n for _ in range(n)]
    b = [Fraction(0)] * n
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                p = idx(z, y, x)
                A[p][p] += alpha
                b[p] += alpha * Fraction(I0[z][y][x])
                for dz, dy, dx in ((0, 0, 1), (0, 1, 0), (1, 0, 0)):
                    z2, y2, x2 = z + dz, y + dy, x + dx
                    if z2 < nz and y2 < ny and x2 < nx:
                        q = idx(z2, y2, x2)
                        # target difference: the input's along x and y, zero along z
                        g = Fraction(0) if dz else Fraction(I0[z][y][x]) - Fraction(I0[z2][y2][x2])
                        A[p][p] += 1
                        A[q][q] += 1
                        A[p][q] -= 1
                        A[q][p] -= 1
                        b[p] += g
                        b[q] -= g
    f = _solve_spd(A, b)
    return [[[f[idx(z, y, x)] for x in range(nx)] for y in range(ny)] for z in range(nz)]


def exact_solve(s, o, alpha):
    """Exact f for one slice.  ``s``, ``o``: ny x nx nested lists of ints or Fractions;
    ``alpha``: a positive Fraction (or int).  Returns an ny x nx nested list of Fractions."""
    alpha = Fraction(alpha)
    if alpha <= 0:
        raise ValueError("alpha must be > 0")
    ny, nx = len(s), len(s[0])
    n = ny * nx
    A = [[Fraction(0)] * n for _ in range(n)]
    b = [Fraction(0)] * n
    for y in range(ny):
        for x in range(nx):
            p = y * nx + x
            A[p][p] += alpha
            b[p] += alpha * Fraction(s[y][x])
    # each undirected edge pq adds (f_p - f_q) - (o_p - o_q) to row p and its negative to row q
    for y in range(ny):
        for x in range(nx):
            p = y * nx + x
            for (yq, xq) in ((y, x + 1), (y + 1, x)):
                if yq < ny and xq < nx:
                    q = yq * nx + xq
                    g = Fraction(o[y][x]) - Fraction(o[yq][xq])
                    A[p][p] += 1
                    A[q][q] += 1
                    A[p][q] -= 1
                    A[q][p] -= 1
                    b[p] += g
                    b[q] -= g
    f = _solve_spd(A, b)
    return [[f[y * nx + x] for x in range(nx)] for y in range(ny)]
