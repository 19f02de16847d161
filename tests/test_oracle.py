"""Pins of the CPU FP64 oracle against things other than itself.

The paper prints no worked numeric example, so each oracle function is pinned by
brute force on tiny inputs (among them the exact rational solutions of Eq. (1) stored in
tests/golden/eq1_exact_small.txt), by explicit matrices built from first principles, by closed
forms and limits stated in Sec. 3, and by finite differences.  Each pin is chosen so that a
plausible slip (a dropped term, a wrong sign, swapped W/H, a missing renormalisation)
fails at least one test.
"""
import math

import numpy as np
import pytest

from oracle import emfuse_oracle as O

RNG = np.random.default_rng(1234)


# ----------------------------------------------------------------------------- helpers
def neighbours(ny, nx):
    """4-neighbour edges of an ny x nx pixel grid (each undirected edge once)."""
    edges = []
    for y in range(ny):
        for x in range(nx):
            if x + 1 < nx:
                edges.append(((y, x), (y, x + 1)))
            if y + 1 < ny:
                edges.append(((y, x), (y + 1, x)))
    return edges


def energy_minimiser(s, o, alpha):
    """Brute force: the discrete energy of Sec. 3 "Screened-Poisson Blending",
    E(f) = alpha sum_p (f_p - s_p)^2 + sum_edges ((f_p - f_q) - (o_p - o_q))^2,
    minimised as a dense linear least-squares problem (no Euler-Lagrange step, no DCT)."""
    ny, nx = s.shape
    n = ny * nx
    idx = lambda y, x: y * nx + x
    rows, rhs = [], []
    sa = math.sqrt(alpha)
    for y in range(ny):
        for x in range(nx):
            r = np.zeros(n); r[idx(y, x)] = sa
            rows.append(r); rhs.append(sa * s[y, x])
    for (p, q) in neighbours(ny, nx):
        r = np.zeros(n); r[idx(*p)] = 1.0; r[idx(*q)] = -1.0
        rows.append(r); rhs.append(o[p] - o[q])
    f, *_ = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)
    return f.reshape(ny, nx)


def dense_A(ny, nx, alpha):
    """alpha I + graph Laplacian of the 4-neighbour grid, assembled edge by edge."""
    n = ny * nx
    A = alpha * np.eye(n)
    for (p, q) in neighbours(ny, nx):
        i, j = p[0] * nx + p[1], q[0] * nx + q[1]
        A[i, i] += 1; A[j, j] += 1; A[i, j] -= 1; A[j, i] -= 1
    return A


def cosine_matrix(n):
    """Orthonormal DCT-II matrix from its definition C[k, x] = c_k cos(pi k (x + 1/2) / n)."""
    C = np.zeros((n, n))
    for k in range(n):
        ck = math.sqrt(1.0 / n) if k == 0 else math.sqrt(2.0 / n)
        for x in range(n):
            C[k, x] = ck * math.cos(math.pi * k * (x + 0.5) / n)
    return C


# ----------------------------------------------------------------------------- DCT / spectrum
@pytest.mark.parametrize("n", [1, 2, 5, 8])
def test_dct_matches_cosine_matrix(n):
    import scipy.fft as sfft
    x = RNG.normal(size=n)
    assert np.allclose(sfft.dct(x, type=2, norm="ortho"), cosine_matrix(n) @ x, atol=1e-13)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 16])
def test_neumann_eigenpairs(n):
    """cos(pi k (x+1/2)/n) is an eigenvector of the 1-D Neumann graph Laplacian."""
    A = dense_A(1, n, 0.0)
    lam = O.neumann_eigenvalues(n)
    C = cosine_matrix(n)
    for k in range(n):
        v = C[k]
        assert np.allclose(A @ v, lam[k] * v, atol=1e-12)


# ----------------------------------------------------------------------------- Eq. (1)
@pytest.mark.parametrize("shape", [(8, 8), (7, 5), (5, 7), (1, 9), (1, 1), (2, 3), (6, 1)])
@pytest.mark.parametrize("alpha", [1e-3, 0.01, 0.1, 2.0])
def test_solve_equals_energy_minimiser(shape, alpha):
    s = RNG.uniform(0, 255, size=shape)
    o = RNG.uniform(0, 255, size=shape)
    f = O.solve_dct(s, o, alpha)
    ref = energy_minimiser(s, o, alpha)
    assert np.max(np.abs(f - ref)) <= 1e-8 * 255 / min(1.0, alpha) * 10


@pytest.mark.parametrize("shape", [(8, 8), (7, 5), (1, 6)])
def test_operator_is_the_dense_euler_lagrange_system(shape):
    alpha = 0.37
    u = RNG.normal(size=shape)
    A = dense_A(*shape, alpha)
    assert np.allclose(O.apply_A(u, alpha).ravel(), A @ u.ravel(), atol=1e-12)
    s = RNG.normal(size=shape); o = RNG.normal(size=shape)
    b = O.screened_rhs(s, o, alpha)
    assert np.allclose(b.ravel(), alpha * s.ravel() + dense_A(*shape, 0.0) @ o.ravel(), atol=1e-12)
    x = np.linalg.solve(A, b.ravel()).reshape(shape)
    assert np.allclose(O.solve_dct(s, o, alpha), x, atol=1e-10)


def test_operator_symmetric_positive_definite():
    ny, nx, alpha = 6, 5, 0.01
    u = RNG.normal(size=(ny, nx)); v = RNG.normal(size=(ny, nx))
    assert abs(np.sum(O.apply_A(u, alpha) * v) - np.sum(u * O.apply_A(v, alpha))) < 1e-10
    ev = np.linalg.eigvalsh(dense_A(ny, nx, alpha))
    assert ev.min() == pytest.approx(alpha, rel=1e-9)  # the constant mode: A 1 = alpha 1


def test_constant_is_fixed_point():
    c = 93.25
    s = np.full((9, 11), c); o = np.full((9, 11), c)
    assert np.allclose(O.solve_dct(s, o, 1e-3), c, atol=1e-10)
    stack = np.full((5, 6, 7), c)
    assert np.allclose(O.smooth_stack(stack, 1.0, 3.0), c, atol=1e-12)


def test_limits_of_alpha():
    """Sec. 3: large alpha interpolates I1 (f -> s); small alpha keeps the gradients of I0,
    with the DC term from s (f -> o - mean(o) + mean(s))."""
    s = RNG.uniform(0, 255, size=(12, 10)); o = RNG.uniform(0, 255, size=(12, 10))
    assert np.max(np.abs(O.solve_dct(s, o, 1e12) - s)) < 1e-6
    f0 = O.solve_dct(s, o, 1e-10)
    assert np.max(np.abs(f0 - (o - o.mean() + s.mean()))) < 1e-4


def test_mean_preserved_from_s():
    s = RNG.uniform(0, 255, size=(13, 17)); o = RNG.uniform(0, 255, size=(13, 17))
    for alpha in (1e-3, 0.1, 10.0):
        assert O.solve_dct(s, o, alpha).mean() == pytest.approx(s.mean(), abs=1e-9)


@pytest.mark.parametrize("kl", [(0, 1), (3, 2), (4, 0)])
def test_single_cosine_mode_gain(kl):
    """Frequency-space blend (Sec. 3): one mode of s is scaled by alpha/(alpha+lam) and the
    same mode of o by lam/(alpha+lam), with lam the eigenvalue found by brute force."""
    ny, nx, alpha = 9, 7, 0.05
    l, k = kl
    mode = np.outer(cosine_matrix(ny)[l], cosine_matrix(nx)[k])
    lam = (mode.ravel() @ (dense_A(ny, nx, 0.0) @ mode.ravel())) / (mode.ravel() @ mode.ravel())
    f = O.solve_dct(mode, np.zeros_like(mode), alpha)
    assert np.allclose(f, alpha / (alpha + lam) * mode, atol=1e-12)
    f = O.solve_dct(np.zeros_like(mode), mode, alpha)
    assert np.allclose(f, lam / (alpha + lam) * mode, atol=1e-12)


def test_linearity():
    shape = (10, 8); alpha = 0.02
    s1, s2, o1, o2 = (RNG.normal(size=shape) for _ in range(4))
    a, b = 0.3, -1.7
    lhs = O.solve_dct(a * s1 + b * s2, a * o1 + b * o2, alpha)
    rhs = a * O.solve_dct(s1, o1, alpha) + b * O.solve_dct(s2, o2, alpha)
    assert np.allclose(lhs, rhs, atol=1e-10)


def test_residual_of_exact_solution_is_zero_and_detects_error():
    s = RNG.uniform(0, 255, size=(32, 24)); o = RNG.uniform(0, 255, size=(32, 24))
    f = O.solve_dct(s, o, 1e-3)
    assert O.relative_residual(f, s, o, 1e-3) < 1e-12
    assert O.relative_residual(f + 1e-3, s, o, 1e-3) > 1e-9


def test_alpha_must_be_positive():
    with pytest.raises(ValueError):
        O.solve_dct(np.ones((2, 2)), np.ones((2, 2)), 0.0)


# ----------------------------------------------------------------------------- smoothing
def test_truncation_rule():
    """Sec. 3 "Implementation": weight zero beyond three standard deviations."""
    assert len(O.gaussian_taps(1.0)) == 7       # |d| <= 3
    assert len(O.gaussian_taps(3.0)) == 19      # |d| <= 9
    assert len(O.gaussian_taps(0.5)) == 3       # floor(1.5) = 1
    w = O.gaussian_taps(3.0)
    assert w[0] == pytest.approx(math.exp(-4.5))
    assert len(O.gaussian_taps(0.0)) == 1


def brute_force_3d(vol, sxy, sz):
    """Direct renormalised 3-D sum with the paper's anisotropic Gaussian G (constant
    prefactor included) over the truncated support |dx|,|dy| <= 3 sxy, |dz| <= 3 sz."""
    nz, ny, nx = vol.shape
    Rxy, Rz = int(math.floor(3 * sxy)), int(math.floor(3 * sz))
    norm = 1.0 / (sxy * sxy * sz * (2 * math.pi) ** 1.5)
    out = np.zeros_like(vol, dtype=np.float64)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                num = den = 0.0
                for dz in range(-Rz, Rz + 1):
                    for dy in range(-Rxy, Rxy + 1):
                        for dx in range(-Rxy, Rxy + 1):
                            zz, yy, xx = z + dz, y + dy, x + dx
                            if 0 <= zz < nz and 0 <= yy < ny and 0 <= xx < nx:
                                g = norm * math.exp(-(dx * dx + dy * dy) / (2 * sxy * sxy)) \
                                    * math.exp(-(dz * dz) / (2 * sz * sz))
                                num += g * vol[zz, yy, xx]; den += g
                out[z, y, x] = num / den
    return out


@pytest.mark.parametrize("sig", [(1.0, 3.0), (0.7, 1.4), (1.0, 0.0)])
def test_separable_equals_brute_force_3d(sig):
    vol = RNG.uniform(0, 255, size=(5, 6, 7))
    sxy, sz = sig
    if sz == 0.0:
        ref = np.stack([brute_force_3d(vol[j:j + 1], sxy, 1e-9)[0] for j in range(vol.shape[0])])
    else:
        ref = brute_force_3d(vol, sxy, sz)
    assert np.allclose(O.smooth_stack(vol, sxy, sz), ref, atol=1e-9)


def test_z_ramp_preserved_away_from_ends():
    nz = 30
    vol = np.broadcast_to(np.arange(nz, dtype=float)[:, None, None] * 2.5 + 7, (nz, 4, 5)).copy()
    out = O.smooth_stack(vol, 1.0, 3.0)
    assert np.allclose(out[9:nz - 9], vol[9:nz - 9], atol=1e-10)
    # renormalisation at the ends pulls the ramp inwards (not a fixed point there)
    assert out[0, 0, 0] > vol[0, 0, 0] + 1.0


def test_smooth_transpose_dot_product():
    x = RNG.normal(size=(11, 6, 5)); y = RNG.normal(size=(11, 6, 5))
    lhs = np.sum(O.smooth_stack(x, 1.0, 2.0) * y)
    rhs = np.sum(x * O.smooth_transpose(y, 1.0, 2.0))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_dsmooth_dsigma_z_matches_finite_difference():
    vol = RNG.uniform(0, 255, size=(12, 4, 5))
    sz, h, R = 2.2, 1e-5, 6
    fd = (O.smooth_stack(vol, 1.0, sz + h, radius_z=R) - O.smooth_stack(vol, 1.0, sz - h, radius_z=R)) / (2 * h)
    assert np.allclose(O.dsmooth_dsigma_z(vol, 1.0, sz, radius_z=R), fd, atol=1e-5)


# ----------------------------------------------------------------------------- adjoint
def test_backward_slice_matches_dense_jacobians():
    ny, nx, alpha = 5, 4, 0.3
    n = ny * nx
    s = RNG.uniform(0, 255, size=(ny, nx)); o = RNG.uniform(0, 255, size=(ny, nx))
    g = RNG.normal(size=(ny, nx))
    A = dense_A(ny, nx, alpha); Lm = dense_A(ny, nx, 0.0)
    # f = A^{-1}(alpha s + L o): Jacobians by dense inverse, written out directly
    Ainv = np.linalg.inv(A)
    f = (Ainv @ (alpha * s.ravel() + Lm @ o.ravel())).reshape(ny, nx)
    ds, do, da = O.backward_slice(g, s, o, f, alpha)
    assert np.allclose(ds.ravel(), (alpha * Ainv).T @ g.ravel(), atol=1e-10)
    assert np.allclose(do.ravel(), (Ainv @ Lm).T @ g.ravel(), atol=1e-10)
    # d f / d alpha = A^{-1}(s - f) (differentiate A f = alpha s + L o)
    assert da == pytest.approx(g.ravel() @ (Ainv @ (s - f).ravel()), rel=1e-10)


def test_backward_stack_matches_finite_differences():
    """Central differences in FP64: in log(alpha) (alpha - h would be singular at small
    alpha) and in sigma_z with the support radius frozen."""
    nz, ny, nx = 6, 5, 4
    I0 = RNG.uniform(0, 255, size=(nz, ny, nx))
    g = RNG.normal(size=(nz, ny, nx))
    sxy, sz, alpha, R = 1.0, 1.3, 0.05, 3

    def loss(I, a, s_z):
        s = O.smooth_stack(I, sxy, s_z, radius_z=R)
        f = np.stack([O.solve_dct(s[j], I[j], a) for j in range(nz)])
        return float(np.sum(g * f))

    dI0, dalpha, dsig = O.backward_stack(g, I0, sxy, sz, alpha, radius_z=R)
    h = 1e-3
    fd_alpha = (loss(I0, alpha * math.exp(h), sz) - loss(I0, alpha * math.exp(-h), sz)) / (2 * h) / alpha
    assert dalpha == pytest.approx(fd_alpha, rel=1e-5)
    fd_sig = (loss(I0, alpha, sz + h) - loss(I0, alpha, sz - h)) / (2 * h)
    assert dsig == pytest.approx(fd_sig, rel=1e-5)
    for idx in [(0, 0, 0), (3, 2, 1), (5, 4, 3)]:
        e = np.zeros_like(I0); e[idx] = 1.0
        fd = (loss(I0 + h * e, alpha, sz) - loss(I0 - h * e, alpha, sz)) / (2 * h)
        assert dI0[idx] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_correct_stack_shapes_and_continuity():
    """End-to-end on a tiny stack with per-slice gain: the corrected stack has smaller
    inter-slice jumps than the input (the purpose stated in Sec. 1)."""
    from paper_1506_02079_gb300.synthetic import make_stack
    I0 = make_stack(12, 32, 32, seed=7).double().numpy()
    I1, I2 = O.correct_stack(I0, 1.0, 3.0, 1e-3)
    assert I2.shape == I0.shape
    jump = lambda v: float(np.mean((v[1:] - v[:-1]) ** 2))
    assert jump(I2) < 0.5 * jump(I0)


# ----------------------------------------------------------------------------- robust averaging
def test_robust_constant_stack_with_a_corrupt_slice_closed_form():
    """A constant stack (100) with one slice zeroed (missing data): in every z-window that
    contains it, the zero sample has weight fraction p <= 1/sum(w) < 0.2, so |0 - mu| =
    100 (1 - p) exceeds 2 sigma = 200 sqrt(p (1 - p)) while the constant samples stay within
    it; the robust average is exactly 100 everywhere, the zeroed slice included, whereas the
    plain average is pulled down next to it."""
    I0 = np.full((15, 4, 5), 100.0)
    I0[7] = 0.0
    out = O.robust_smooth_stack(I0, 0.0, 3.0)
    np.testing.assert_allclose(out, 100.0, rtol=0, atol=1e-12)
    plain = O.smooth_stack(I0, 0.0, 3.0)
    assert plain[6].max() < 90.0


def test_robust_reduces_to_plain_for_large_kappa():
    I0 = np.random.default_rng(4).uniform(0, 255, size=(9, 7, 6))
    np.testing.assert_allclose(O.robust_smooth_stack(I0, 1.0, 1.5, kappa=1e9), O.smooth_stack(I0, 1.0, 1.5),
                               rtol=0, atol=1e-10)


def test_robust_is_affine_equivariant_and_within_window_range():
    """robust(a v + b) = a robust(v) + b (mean, deviation and decisions scale together), and
    each output lies between the smallest and largest xy-smoothed value of its z-window."""
    I0 = np.random.default_rng(6).uniform(0, 255, size=(10, 6, 5))
    r = O.robust_smooth_stack(I0, 1.0, 2.0)
    np.testing.assert_allclose(O.robust_smooth_stack(-3.0 * I0 + 7.0, 1.0, 2.0), -3.0 * r + 7.0,
                               rtol=0, atol=1e-9)
    xy = O.smooth_axis(O.smooth_axis(I0, 1.0, 2), 1.0, 1)
    R = O.support_radius(2.0)
    for z in range(10):
        win = xy[max(0, z - R):min(10, z + R + 1)]
        assert np.all(r[z] >= win.min(axis=0) - 1e-9) and np.all(r[z] <= win.max(axis=0) + 1e-9)


def test_robust_keep_and_drop_on_hand_computed_windows():
    """With sigma_z = 100 every plane of a short stack is in every window with almost equal
    weights.  Six samples 10, 10, 10, 10, 10, 40: mean 15, variance 125, 2 sigma = 22.4 < 25,
    so the 40 is dropped and the average is 10.  Three samples 10, 10, 40: mean 20, variance
    200, 2 sigma = 28.3 > 20, so nothing is dropped and the average is the plain one."""
    I0 = np.full((6, 1, 1), 10.0)
    I0[5] = 40.0
    np.testing.assert_allclose(O.robust_smooth_stack(I0, 0.0, 100.0), 10.0, rtol=0, atol=1e-9)
    I3 = np.array([10.0, 10.0, 40.0]).reshape(3, 1, 1)
    np.testing.assert_allclose(O.robust_smooth_stack(I3, 0.0, 100.0), O.smooth_stack(I3, 0.0, 100.0),
                               rtol=0, atol=1e-12)


def test_robust_uses_weighted_statistics_and_kappa_in_sigma_units():
    """Window [10, 40, 10] at the middle plane with sigma_z = 1 (weights e^-1/2, 1, e^-1/2):
    the 40 has weight fraction p = 1 / (1 + 2 e^-1/2) = 0.452, and its deviation is
    sqrt((1 - p) / p) = 1.101 weighted standard deviations (with equal weights it would be
    sqrt(2) = 1.414).  So kappa = 1.2 keeps it (the plain average) and kappa = 1.05 drops it
    (the average of the two 10s); an unweighted or variance-scaled threshold fails one of the
    two."""
    I0 = np.array([10.0, 40.0, 10.0]).reshape(3, 1, 1)
    keep = O.robust_smooth_stack(I0, 0.0, 1.0, kappa=1.2)
    assert keep[1, 0, 0] == pytest.approx(O.smooth_stack(I0, 0.0, 1.0)[1, 0, 0], abs=1e-12)
    drop = O.robust_smooth_stack(I0, 0.0, 1.0, kappa=1.05)
    assert drop[1, 0, 0] == pytest.approx(10.0, abs=1e-12)


# sigma_z with taps w(1) = 1/2 and w(2) = 1/16 exactly: exp(-1 / (2 sigma^2)) = 1/2
SIGMA_HALF = math.sqrt(1.0 / (2.0 * math.log(2.0)))   # floor(3 sigma) = 2


def test_robust_margin_on_hand_computed_windows():
    """robust_margin = min over the window of |(v_d - mu)^2 - kappa^2 var| / (kappa^2 var + 1).
    Stack -1, 0, 1 (one pixel per plane), kappa = 2, weights 1, 1/2, 1/16 at |d| = 0, 1, 2.
    Middle plane: taps -1, 0, 1 with weights 1/2, 1, 1/2: mu = 0, var = 1/2, threshold 2,
    squared deviations 1, 0, 1, margin |1 - 2| / 3 = 1/3.  First plane: taps 0, 1, 2 with
    values -1, 0, 1 and weights 1, 1/2, 1/16 (W = 25/16): mu = -0.6, var = 0.5 / W = 0.32,
    threshold 1.28, squared deviations 0.16, 0.36, 2.56, margin 0.92 / 2.28; the last plane
    mirrors it.  A one-plane window (sigma_z with floor(3 sigma_z) = 0) is an exact tie at
    every voxel (0 <= 0): margin 0."""
    assert O.support_radius(SIGMA_HALF) == 2
    I0 = np.array([-1.0, 0.0, 1.0]).reshape(3, 1, 1)
    m = O.robust_margin(I0, 0.0, SIGMA_HALF, kappa=2.0)[:, 0, 0]
    np.testing.assert_allclose(m, [0.92 / 2.28, 1.0 / 3.0, 0.92 / 2.28], rtol=0, atol=1e-12)
    flat = np.random.default_rng(3).uniform(0, 255, size=(4, 3, 5))
    np.testing.assert_allclose(O.robust_margin(flat, 1.0, 0.2), 0.0, rtol=0, atol=0)


def test_robust_margin_zero_at_an_exact_tie_and_outcomes_list_both_decisions():
    """Stack 0, 0, 4 with the same weights: at the middle plane W = 2, mu = 1, var = 3 and the
    squared deviations are 1, 1, 9.  With kappa = sqrt(3) the sample 4 sits exactly on the
    threshold 9: margin 0 (to the rounding of kappa^2), and both decisions are valid: keep it
    (average 1) or drop it (average 0).  robust_outcomes lists exactly these two values there,
    the oracle's own decision among them, and nothing at the clear first plane (samples 0, 0,
    4 with weights 1, 1/2, 1/16: margins far from 0)."""
    I0 = np.array([0.0, 0.0, 4.0]).reshape(3, 1, 1)
    k = math.sqrt(3.0)
    assert O.robust_margin(I0, 0.0, SIGMA_HALF, kappa=k)[1, 0, 0] == pytest.approx(0.0, abs=1e-12)
    ref, alts = O.robust_outcomes(I0, 0.0, SIGMA_HALF, kappa=k, tie=1e-6)
    assert sorted(alts) == [1]
    np.testing.assert_allclose(np.sort(alts[1]), [0.0, 1.0], rtol=0, atol=1e-12)
    assert np.min(np.abs(alts[1] - ref[1, 0, 0])) <= 1e-12
    # away from the tie (kappa = 2: threshold 12 > 9) the sample is kept and nothing is listed
    ref2, alts2 = O.robust_outcomes(I0, 0.0, SIGMA_HALF, kappa=2.0, tie=1e-6)
    assert alts2 == {} and ref2[1, 0, 0] == pytest.approx(1.0, abs=1e-12)


# ----------------------------------------------------------------------------- colour fusion
def test_fuse_color_closed_forms():
    """Colour / monochrome fusion (Sec. 3): (1) a grey colour image (three equal channels)
    gives three copies of the monochrome solve; (2) each channel keeps the mean of its colour
    channel (the DCT mode 0 has gain 1); (3) the difference of two channels is
    alpha A^-1 (s_c - s_d), so it does not depend on the monochrome image at all, and it is
    the low-pass of the colour difference (checked against the dense inverse)."""
    rng = np.random.default_rng(12)
    ny, nx, alpha = 6, 7, 0.2
    s = rng.uniform(0, 255, size=(3, ny, nx))
    o = rng.uniform(0, 255, size=(ny, nx))
    f = O.fuse_color(s, o, alpha)
    grey = O.fuse_color(np.stack([s[0]] * 3), o, alpha)
    for c in range(3):
        np.testing.assert_allclose(grey[c], O.solve_dct(s[0], o, alpha), rtol=0, atol=1e-9)
        assert f[c].mean() == pytest.approx(s[c].mean(), rel=1e-12)
    f2 = O.fuse_color(s, rng.uniform(0, 255, size=(ny, nx)), alpha)
    np.testing.assert_allclose(f[0] - f[1], f2[0] - f2[1], rtol=0, atol=1e-9)
    # dense (alpha I + L) on the ny x nx grid, built edge by edge
    n = ny * nx
    A = alpha * np.eye(n)
    for y in range(ny):
        for x in range(nx):
            p = y * nx + x
            for qy, qx in ((y, x + 1), (y + 1, x)):
                if qy < ny and qx < nx:
                    q = qy * nx + qx
                    A[p, p] += 1; A[q, q] += 1; A[p, q] -= 1; A[q, p] -= 1
    diff = alpha * np.linalg.solve(A, (s[0] - s[2]).ravel()).reshape(ny, nx)
    np.testing.assert_allclose(f[0] - f[2], diff, rtol=0, atol=1e-8)


# ----------------------------------------------------------------------------- stored exact solutions
def load_eq1_exact():
    """Cases of tests/golden/eq1_exact_small.txt: (name, alpha, s, o, f) with f exact Fractions."""
    import os
    from fractions import Fraction
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "eq1_exact_small.txt")
    cases, cur = [], None
    for line in open(path):
        tok = line.split()
        if not tok or tok[0].startswith("#"):
            continue
        if tok[0] == "case":
            cur = {"name": tok[1], "ny": int(tok[2]), "nx": int(tok[3]), "alpha": Fraction(tok[4])}
            cases.append(cur)
        else:
            cur[tok[0]] = [Fraction(v) for v in tok[1:]]
    return cases


EQ1_CASES = load_eq1_exact()


@pytest.mark.parametrize("case", EQ1_CASES, ids=lambda c: c["name"])
def test_stored_exact_solution_satisfies_eq1_exactly(case):
    """The stored f solves Eq. (1) with zero residual in rational arithmetic (rows assembled
    here from the 4-neighbour definition), and keeps the sum of s exactly (summing the rows of
    Eq. (1) cancels every Laplacian term)."""
    ny, nx, a = case["ny"], case["nx"], case["alpha"]
    s, o, f = case["s"], case["o"], case["f"]
    assert len(s) == len(o) == len(f) == ny * nx
    for y in range(ny):
        for x in range(nx):
            p = y * nx + x
            lhs, rhs = a * f[p], a * s[p]
            for yq, xq in ((y - 1, x), (y + 1, x), (y, x - 1), (y, x + 1)):
                if 0 <= yq < ny and 0 <= xq < nx:
                    q = yq * nx + xq
                    lhs += f[p] - f[q]
                    rhs += o[p] - o[q]
            assert lhs == rhs
    assert sum(f) == sum(s)


@pytest.mark.parametrize("case", EQ1_CASES, ids=lambda c: c["name"])
def test_solve_dct_matches_stored_exact_solution(case):
    """The DCT solve reaches the exact rational solution up to FP64 rounding amplified by at most
    kappa(A) = 1 + 8 / alpha (<= 3.3e4 here): within 1e-8 on values of up to 255."""
    ny, nx, a = case["ny"], case["nx"], float(case["alpha"])
    grid = lambda v: np.array([float(t) for t in v]).reshape(ny, nx)
    f = O.solve_dct(grid(case["s"]), grid(case["o"]), a)
    assert np.max(np.abs(f - grid(case["f"]))) <= 1e-8


# ----------------------------------------------------------------------------- 3-D gradient-domain smoothing
def gd_energy_minimiser(I0, alpha):
    """Brute force for the gradient-domain smoothing: the energy alpha sum (f - I0)^2 +
    sum over x/y edges ((f_p - f_q) - (I0_p - I0_q))^2 + sum over z edges (f_p - f_q)^2 as a
    dense least-squares problem (no normal equations, no transform)."""
    nz, ny, nx = I0.shape
    n = I0.size
    idx = lambda z, y, x: (z * ny + y) * nx + x
    rows, rhs = [], []
    sa = math.sqrt(alpha)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                r = np.zeros(n); r[idx(z, y, x)] = sa
                rows.append(r); rhs.append(sa * I0[z, y, x])
                for dz, dy, dx in ((0, 0, 1), (0, 1, 0), (1, 0, 0)):
                    z2, y2, x2 = z + dz, y + dy, x + dx
                    if z2 < nz and y2 < ny and x2 < nx:
                        r = np.zeros(n); r[idx(z, y, x)] = 1.0; r[idx(z2, y2, x2)] = -1.0
                        rows.append(r)
                        rhs.append(0.0 if dz else I0[z, y, x] - I0[z2, y2, x2])
    f, *_ = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)
    return f.reshape(nz, ny, nx)


@pytest.mark.parametrize("shape", [(3, 4, 5), (4, 1, 6), (5, 3, 1), (1, 3, 4), (2, 2, 2)])
@pytest.mark.parametrize("alpha", [1e-3, 0.3, 4.0])
def test_gradient_domain_smooth_equals_energy_minimiser(shape, alpha):
    I0 = RNG.uniform(0, 255, size=shape)
    assert np.allclose(O.gradient_domain_smooth(I0, alpha), gd_energy_minimiser(I0, alpha), atol=1e-7, rtol=0)


def test_gradient_domain_smooth_removes_slice_offsets_by_a_1d_screened_solve():
    """I0 = B(x, y) + c_z: the in-plane part carries no z-gradient and stays; the offsets
    solve the 1-D z problem (alpha I + L_z) g = alpha c, written here as a dense tridiagonal
    matrix (closed form, independent of the DCT)."""
    nz, ny, nx, alpha = 7, 5, 6, 0.05
    B = RNG.uniform(0, 200, size=(ny, nx))
    c = RNG.uniform(-30, 30, size=nz)
    I0 = B[None] + c[:, None, None]
    Lz = np.zeros((nz, nz))
    for z in range(nz - 1):
        Lz[z, z] += 1; Lz[z + 1, z + 1] += 1; Lz[z, z + 1] -= 1; Lz[z + 1, z] -= 1
    g = np.linalg.solve(alpha * np.eye(nz) + Lz, alpha * c)
    assert np.allclose(O.gradient_domain_smooth(I0, alpha), B[None] + g[:, None, None], atol=1e-9, rtol=0)


def test_gradient_domain_smooth_invariants():
    I0 = RNG.uniform(0, 255, size=(6, 9, 8))
    f = O.gradient_domain_smooth(I0, 0.01)
    # summing the normal equations cancels every Laplacian term: the total is kept
    assert abs(f.sum() - I0.sum()) <= 1e-8 * abs(I0.sum())
    # a stack constant in z is a fixed point (no z-gradient to remove); one slice is unchanged
    flat = np.repeat(I0[:1], 6, axis=0)
    assert np.allclose(O.gradient_domain_smooth(flat, 0.01), flat, atol=1e-9, rtol=0)
    assert np.allclose(O.gradient_domain_smooth(I0[:1], 0.01), I0[:1], atol=1e-9, rtol=0)
    # alpha -> infinity: the value constraint wins
    assert np.allclose(O.gradient_domain_smooth(I0, 1e12), I0, atol=1e-6, rtol=0)
    # inter-slice differences shrink
    assert np.abs(np.diff(f, axis=0)).mean() < np.abs(np.diff(I0, axis=0)).mean()


def load_gd_exact():
    """Cases of tests/golden/gd_exact_small.txt: (name, nz, ny, nx, alpha, I, f), f exact."""
    import os
    from fractions import Fraction
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "gd_exact_small.txt")
    cases, cur = [], None
    for line in open(path):
        tok = line.split()
        if not tok or tok[0].startswith("#"):
            continue
        if tok[0] == "case":
            cur = {"name": tok[1], "nz": int(tok[2]), "ny": int(tok[3]), "nx": int(tok[4]),
                   "alpha": Fraction(tok[5])}
            cases.append(cur)
        else:
            cur[tok[0]] = [Fraction(v) for v in tok[1:]]
    return cases


GD_CASES = load_gd_exact()


@pytest.mark.parametrize("case", GD_CASES, ids=lambda c: c["name"])
def test_stored_gradient_domain_solution_is_exact(case):
    """The stored f satisfies the normal equations of the gradient-domain energy with zero
    rational residual (rows assembled here from the 6-neighbour definition: x/y edges carry
    the input's differences, z edges zero), keeps the total exactly, and the oracle's 3-D DCT
    solve reaches it within 1e-9."""
    nz, ny, nx, a = case["nz"], case["ny"], case["nx"], case["alpha"]
    I, f = case["I"], case["f"]
    idx = lambda z, y, x: (z * ny + y) * nx + x
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                p = idx(z, y, x)
                lhs, rhs = a * f[p], a * I[p]
                for dz, dy, dx in ((0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)):
                    z2, y2, x2 = z + dz, y + dy, x + dx
                    if 0 <= z2 < nz and 0 <= y2 < ny and 0 <= x2 < nx:
                        q = idx(z2, y2, x2)
                        lhs += f[p] - f[q]
                        if dz == 0:
                            rhs += I[p] - I[q]
                assert lhs == rhs
    assert sum(f) == sum(I)
    grid = lambda v: np.array([float(t) for t in v]).reshape(nz, ny, nx)
    got = O.gradient_domain_smooth(grid(I), float(a))
    assert np.max(np.abs(got - grid(f))) <= 1e-9
