"""Plain CPU FP64 oracle for the EM-stack colour correction of Kazhdan et al.,
"Gradient-Domain Fusion for Color Correction in Large EM Image Stacks" (arXiv 1506.02079).

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct statement of what
the GPU path computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it; the CUDA library never calls it and shares no code,
table or constant with it.

What it computes (every function cites the passage it follows):

* ``smooth_stack``  -- phase 1, Sec. 3 "Anisotropic Smoothing": I1 = I0 * G_{sxy,sz},
  with the Gaussian truncated at three standard deviations (Sec. 3 "Implementation").
* ``robust_smooth_stack`` -- phase 1 with robust averaging across slices (Sec. 3, the
  outlier example): z-window samples beyond kappa = 2 weighted standard deviations of the
  weighted mean are left out of the average.  ``robust_margin`` is how far a window's
  decisions are from a tie; ``robust_outcomes`` lists every valid average where one is near.
* ``solve_dct``     -- phase 2, Sec. 3 "Screened-Poisson Blending", Eq. (1):
  (alpha - Lap) I2_j = alpha I1_j - Lap I0_j, solved exactly by the frequency-space blend of
  Sec. 3 "Frequency-Space Interpretation" written for the discrete Neumann problem.
* ``correct_stack`` -- both phases.
* ``fuse_color``    -- the colour / monochrome fusion example of Sec. 3: one solve per colour
  channel with the grey image as the gradient constraint.
* ``gradient_domain_smooth`` -- phase 1 as the 3-D gradient-domain problem of the earlier
  method (Sec. 3 "Alternate Solutions": target gradients with the z-components zeroed),
  solved exactly by the 3-D DCT.
* ``backward_*``    -- the adjoint of both phases (gradients w.r.t. s, o, alpha, I0, sigma_z).

Readings of points the paper leaves open:

* taps are the point-sampled Gaussian exp(-d^2/2s^2), normalised to sum 1 (the constant
  prefactor of G cancels);
* "zero beyond three standard deviations" keeps integer offsets |d| <= floor(3 s);
* at stack ends and slice edges the weights are renormalised over in-bounds taps;
* Lap is the 5-point graph Laplacian with Neumann (no-flux) boundaries and unit spacing:
  (L u)_p = sum_{q in N4(p), q inside} (u_p - u_q),  L = -Lap;
* alpha must be > 0 (Eq. (1) is singular at alpha = 0 with Neumann boundaries);
* relative residual = ||b - A f||_2 / ||b||_2 with b = alpha s + L o, A = alpha I + L;
* for d/d sigma_z the support radius R is held at its nominal value.

Parity status: every function here is pinned by ``tests/test_oracle.py`` (brute-force
energy minimisation, explicit cosine matrices, brute-force 3-D sums, finite differences,
closed forms); none is "parity unpinned".
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft as sfft

__all__ = [
    "gaussian_taps", "smooth_axis", "smooth_stack", "robust_smooth_stack", "robust_margin", "robust_outcomes",
    "smooth_transpose", "dsmooth_dsigma_z",
    "laplacian", "screened_rhs", "apply_A", "neumann_eigenvalues", "solve_dct", "fuse_color", "apply_Ainv",
    "gradient_domain_smooth",
    "relative_residual", "correct_stack", "backward_slice", "backward_stack",
]


# --------------------------------------------------------------------------------------
# Phase 1: anisotropic Gaussian smoothing (Sec. 3 "Anisotropic Smoothing" and
# "Implementation": compact support at three standard deviations).
# --------------------------------------------------------------------------------------
def support_radius(sigma: float) -> int:
    """R(sigma) = floor(3 sigma): taps with |d| <= R are kept (Sec. 3 "Implementation")."""
    if sigma < 0:
        raise ValueError("sigma must be >= 0")
    return int(math.floor(3.0 * sigma + 1e-12))


def gaussian_taps(sigma: float, radius: int | None = None) -> np.ndarray:
    """Unnormalised point-sampled 1-D Gaussian exp(-d^2 / (2 sigma^2)), d = -R..R.

    The separable factor of G_{sxy,sz} in Sec. 3 "Anisotropic Smoothing"; the constant
    1/(sxy^2 sz (2 pi)^{3/2}) is dropped because the weights are renormalised.
    sigma = 0 is the identity (a single tap).
    """
    R = support_radius(sigma) if radius is None else int(radius)
    if sigma == 0.0:
        return np.ones(1)
    d = np.arange(-R, R + 1, dtype=np.float64)
    return np.exp(-(d * d) / (2.0 * sigma * sigma))


def smooth_axis(vol: np.ndarray, sigma: float, axis: int, radius: int | None = None) -> np.ndarray:
    """Renormalised truncated Gaussian along one axis (point-sampled taps, |d| <= floor(3 sigma), renormalised over in-bounds taps).

    out(p) = sum_{|d|<=R, p+d e_a inside} w(d) in(p + d e_a)  /  sum_{same d} w(d).
    """
    vol = np.asarray(vol, dtype=np.float64)
    w = gaussian_taps(sigma, radius)
    R = (len(w) - 1) // 2
    n = vol.shape[axis]
    src = np.moveaxis(vol, axis, 0)
    num = np.zeros_like(src)
    den = np.zeros(n)
    for i in range(n):
        for d in range(-R, R + 1):
            j = i + d
            if 0 <= j < n:
                num[i] += w[d + R] * src[j]
                den[i] += w[d + R]
    out = num / den.reshape((n,) + (1,) * (src.ndim - 1))
    return np.moveaxis(out, 0, axis)


def smooth_stack(I0: np.ndarray, sigma_xy: float, sigma_z: float,
                 radius_xy: int | None = None, radius_z: int | None = None) -> np.ndarray:
    """I1 = I0 * G_{sigma_xy, sigma_z} for a stack laid out [z][y][x] (Sec. 3, phase 1).

    Applied as x, then y, then z.  Because the in-bounds tap set at every voxel is a box,
    the separable renormalised passes equal the direct 3-D renormalised sum.
    """
    v = np.asarray(I0, dtype=np.float64)
    v = smooth_axis(v, sigma_xy, 2, radius_xy)
    v = smooth_axis(v, sigma_xy, 1, radius_xy)
    v = smooth_axis(v, sigma_z, 0, radius_z)
    return v


def robust_smooth_stack(I0: np.ndarray, sigma_xy: float, sigma_z: float, kappa: float = 2.0) -> np.ndarray:
    """Phase 1 with robust averaging across slices (Sec. 3, the outlier example of Fig.
    "f:outliers": only colour values within two standard deviations are averaged).

    Reading: x and y are smoothed as in ``smooth_stack``; along z, the window of every voxel
    (the in-stack taps |d| <= floor(3 sigma_z), weights w_d, values v_d) has weighted mean
        mu = sum w_d v_d / sum w_d   and variance   var = sum w_d (v_d - mu)^2 / sum w_d;
    the samples with (v_d - mu)^2 <= kappa^2 var are kept and averaged with their weights
    renormalised.  kappa = inf gives ``smooth_stack``.
    """
    v = np.asarray(I0, dtype=np.float64)
    v = smooth_axis(v, sigma_xy, 2)
    v = smooth_axis(v, sigma_xy, 1)
    w = gaussian_taps(sigma_z)
    R = (len(w) - 1) // 2
    nz = v.shape[0]
    out = np.empty_like(v)
    for z in range(nz):
        ds = [d for d in range(-R, R + 1) if 0 <= z + d < nz]
        ws = np.array([w[d + R] for d in ds])
        vals = np.stack([v[z + d] for d in ds])               # [taps][y][x]
        W = ws.sum()
        mu = np.tensordot(ws, vals, axes=1) / W
        var = np.tensordot(ws, (vals - mu) ** 2, axes=1) / W
        keep = (vals - mu) ** 2 <= (kappa * kappa) * var      # [taps][y][x]
        wk = ws[:, None, None] * keep
        out[z] = (wk * vals).sum(axis=0) / wk.sum(axis=0)
    return out


def robust_margin(I0: np.ndarray, sigma_xy: float, sigma_z: float, kappa: float = 2.0) -> np.ndarray:
    """For every voxel, min over its window of | (v_d - mu)^2 - kappa^2 var | / (kappa^2 var + 1):
    how far the keep / drop decisions of ``robust_smooth_stack`` are from a tie (0 = a tie)."""
    v = np.asarray(I0, dtype=np.float64)
    v = smooth_axis(v, sigma_xy, 2)
    v = smooth_axis(v, sigma_xy, 1)
    w = gaussian_taps(sigma_z)
    R = (len(w) - 1) // 2
    nz = v.shape[0]
    out = np.empty_like(v)
    for z in range(nz):
        ds = [d for d in range(-R, R + 1) if 0 <= z + d < nz]
        ws = np.array([w[d + R] for d in ds])
        vals = np.stack([v[z + d] for d in ds])
        W = ws.sum()
        mu = np.tensordot(ws, vals, axes=1) / W
        var = np.tensordot(ws, (vals - mu) ** 2, axes=1) / W
        thr = (kappa * kappa) * var
        out[z] = (np.abs((vals - mu) ** 2 - thr) / (thr + 1.0)).min(axis=0)
    return out


def robust_outcomes(I0: np.ndarray, sigma_xy: float, sigma_z: float, kappa: float = 2.0,
                    tie: float = 1e-3, max_ties: int = 8):
    """Every valid result of ``robust_smooth_stack`` where a keep / drop decision is near a tie.

    A sample of a window whose margin | (v_d - mu)^2 - kappa^2 var | / (kappa^2 var + 1) is at
    most ``tie`` may be kept or dropped by an evaluation in other precision: both decisions
    are valid readings of the rule (Sec. 3, the outlier example).  Returns (ref, alts): ref is
    ``robust_smooth_stack``; alts maps the flat index of every voxel with such samples to the
    array of weighted averages over all keep / drop choices of its near-tie samples (the other
    samples as decided), ref's value among them.
    """
    v = np.asarray(I0, dtype=np.float64)
    v = smooth_axis(v, sigma_xy, 2)
    v = smooth_axis(v, sigma_xy, 1)
    w = gaussian_taps(sigma_z)
    R = (len(w) - 1) // 2
    nz, ny, nx = v.shape
    ref = robust_smooth_stack(I0, sigma_xy, sigma_z, kappa)
    alts = {}
    for z in range(nz):
        ds = [d for d in range(-R, R + 1) if 0 <= z + d < nz]
        ws = np.array([w[d + R] for d in ds])
        vals = np.stack([v[z + d] for d in ds])
        W = ws.sum()
        mu = np.tensordot(ws, vals, axes=1) / W
        var = np.tensordot(ws, (vals - mu) ** 2, axes=1) / W
        thr = (kappa * kappa) * var
        keep = (vals - mu) ** 2 <= thr
        near = np.abs((vals - mu) ** 2 - thr) / (thr + 1.0) <= tie       # [taps][y][x]
        for y, x in zip(*np.nonzero(near.any(axis=0))):
            ties = np.nonzero(near[:, y, x])[0]
            if len(ties) > max_ties:
                raise ValueError(f"{len(ties)} near-tie samples in one window")
            outs = []
            for bits in range(1 << len(ties)):
                k = keep[:, y, x].copy()
                for b, t in enumerate(ties):
                    k[t] = bool((bits >> b) & 1)
                wk = ws * k
                if wk.sum() > 0:
                    outs.append(float((wk * vals[:, y, x]).sum() / wk.sum()))
            alts[(z * ny + y) * nx + x] = np.array(outs)
    return ref, alts


def _axis_transpose(g: np.ndarray, sigma: float, axis: int, radius: int | None = None) -> np.ndarray:
    """Transpose of ``smooth_axis``: (K^T g)(q) = sum_p w(p - q) g(p) / N(p)."""
    g = np.asarray(g, dtype=np.float64)
    w = gaussian_taps(sigma, radius)
    R = (len(w) - 1) // 2
    n = g.shape[axis]
    src = np.moveaxis(g, axis, 0)
    den = np.zeros(n)
    for i in range(n):
        for d in range(-R, R + 1):
            if 0 <= i + d < n:
                den[i] += w[d + R]
    scaled = src / den.reshape((n,) + (1,) * (src.ndim - 1))
    out = np.zeros_like(src)
    for p in range(n):
        for d in range(-R, R + 1):
            q = p + d
            if 0 <= q < n:
                out[q] += w[d + R] * scaled[p]
    return np.moveaxis(out, 0, axis)


def smooth_transpose(g: np.ndarray, sigma_xy: float, sigma_z: float,
                     radius_xy: int | None = None, radius_z: int | None = None) -> np.ndarray:
    """K^T g for K = Kz Ky Kx of ``smooth_stack`` (needed by the adjoint of phase 1)."""
    v = _axis_transpose(g, sigma_z, 0, radius_z)
    v = _axis_transpose(v, sigma_xy, 1, radius_xy)
    v = _axis_transpose(v, sigma_xy, 2, radius_xy)
    return v


def dsmooth_dsigma_z(I0: np.ndarray, sigma_xy: float, sigma_z: float,
                     radius_xy: int | None = None, radius_z: int | None = None) -> np.ndarray:
    """d(I0 * G)/d sigma_z with the support radius held fixed.

    Along z, K(p, q) = w(p-q) / N(p) with w(d) = exp(-d^2/2s^2), N(p) = sum_in-bounds w;
    dw/ds = w d^2 / s^3, so dK = (w' - w N'/N) / N with N' = sum_in-bounds w'.
    """
    Rz = support_radius(sigma_z) if radius_z is None else int(radius_z)
    v = np.asarray(I0, dtype=np.float64)
    v = smooth_axis(v, sigma_xy, 2, radius_xy)
    v = smooth_axis(v, sigma_xy, 1, radius_xy)
    nz = v.shape[0]
    d = np.arange(-Rz, Rz + 1, dtype=np.float64)
    w = np.exp(-(d * d) / (2.0 * sigma_z * sigma_z))
    dw = w * d * d / sigma_z ** 3
    out = np.zeros_like(v)
    for i in range(nz):
        num = np.zeros_like(v[0]); dnum = np.zeros_like(v[0]); N = 0.0; dN = 0.0
        for k in range(-Rz, Rz + 1):
            j = i + k
            if 0 <= j < nz:
                num += w[k + Rz] * v[j]; dnum += dw[k + Rz] * v[j]
                N += w[k + Rz]; dN += dw[k + Rz]
        out[i] = dnum / N - num * dN / (N * N)
    return out


# --------------------------------------------------------------------------------------
# Phase 2: screened-Poisson blend, Eq. (1), per slice.
# --------------------------------------------------------------------------------------
def laplacian(u: np.ndarray) -> np.ndarray:
    """(L u)_p = sum over in-slice 4-neighbours q of (u_p - u_q); L = -Lap.

    Works on a single slice [y][x] or a stack [z][y][x] (slices are independent).
    """
    u = np.asarray(u, dtype=np.float64)
    out = np.zeros_like(u)
    out[..., :, 1:] += u[..., :, 1:] - u[..., :, :-1]
    out[..., :, :-1] += u[..., :, :-1] - u[..., :, 1:]
    out[..., 1:, :] += u[..., 1:, :] - u[..., :-1, :]
    out[..., :-1, :] += u[..., :-1, :] - u[..., 1:, :]
    return out


def screened_rhs(s: np.ndarray, o: np.ndarray, alpha: float) -> np.ndarray:
    """Right-hand side of Eq. (1): b = alpha I1_j - Lap I0_j = alpha s + L o."""
    return alpha * np.asarray(s, dtype=np.float64) + laplacian(o)


def apply_A(u: np.ndarray, alpha: float) -> np.ndarray:
    """Left-hand operator of Eq. (1): A u = (alpha - Lap) u = alpha u + L u."""
    return alpha * np.asarray(u, dtype=np.float64) + laplacian(u)


def neumann_eigenvalues(n: int) -> np.ndarray:
    """Eigenvalues 4 sin^2(pi k / 2n), k = 0..n-1, of the 1-D Neumann graph Laplacian.

    Their eigenvectors are the DCT-II basis cos(pi k (x + 1/2) / n); this is the discrete
    counterpart of the -4 pi^2 (k^2 + l^2) eigenvalues in Sec. 3 "Frequency-Space
    Interpretation".
    """
    k = np.arange(n, dtype=np.float64)
    return 4.0 * np.sin(np.pi * k / (2.0 * n)) ** 2


def _lambda_grid(ny: int, nx: int) -> np.ndarray:
    return neumann_eigenvalues(ny)[:, None] + neumann_eigenvalues(nx)[None, :]


def solve_dct(s: np.ndarray, o: np.ndarray, alpha: float) -> np.ndarray:
    """Exact solution of Eq. (1) for one slice, via the frequency-space blend.

    f_hat(k,l) = (alpha s_hat + lam o_hat) / (alpha + lam) in the orthonormal 2-D DCT-II
    basis, with lam = 4 sin^2(pi k/2W) + 4 sin^2(pi l/2H): the Neumann-boundary discrete form
    of the blend in Sec. 3 "Frequency-Space Interpretation".
    """
    if not alpha > 0:
        raise ValueError("alpha must be > 0: Eq. (1) is singular at alpha = 0 under Neumann boundaries")
    s = np.asarray(s, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    lam = _lambda_grid(*s.shape)
    s_hat = sfft.dctn(s, type=2, norm="ortho", workers=-1)
    o_hat = sfft.dctn(o, type=2, norm="ortho", workers=-1)
    f_hat = (alpha * s_hat + lam * o_hat) / (alpha + lam)
    return sfft.idctn(f_hat, type=2, norm="ortho", workers=-1)


def fuse_color(s_rgb: np.ndarray, o_grey: np.ndarray, alpha: float) -> np.ndarray:
    """Fusion of a low-frequency colour image with a high-frequency monochrome one (Sec. 3,
    the colour example): the colour channels give the value constraints, the grey image, copied
    into every channel, the gradient constraints; one solve of Eq. (1) per channel.
    s_rgb: [3][ny][nx], o_grey: [ny][nx]."""
    s_rgb = np.asarray(s_rgb, dtype=np.float64)
    return np.stack([solve_dct(s_rgb[c], o_grey, alpha) for c in range(s_rgb.shape[0])])


def gradient_domain_smooth(I0: np.ndarray, alpha: float) -> np.ndarray:
    """Phase 1 as the 3-D gradient-domain problem of the earlier method (Sec. 3 "Alternate
    Solutions": the target gradient field is the input's gradient with its z-components set to
    zero).  With the same screening as Eq. (1), the smoothed stack minimises

        alpha sum_p (f_p - I0_p)^2 + sum_{x, y edges pq} ((f_p - f_q) - (I0_p - I0_q))^2
                                   + sum_{z edges pq} (f_p - f_q)^2

    over the 6-neighbour graph of the stack (Neumann boundaries), i.e.
    (alpha I + L_xy + L_z) f = alpha I0 + L_xy I0.  The 3-D Neumann graph Laplacian is diagonal
    in the orthonormal 3-D DCT-II basis with eigenvalues lam_z + lam_y + lam_x, so
    f_hat = (alpha + lam_xy) / (alpha + lam_xy + lam_z) * I0_hat: a z-frequency is damped
    the more, the lower its in-plane frequency (the anisotropic diffusion of that method).
    I0: [z][y][x]."""
    if not alpha > 0:
        raise ValueError("alpha must be > 0")
    I0 = np.asarray(I0, dtype=np.float64)
    nz, ny, nx = I0.shape
    lam_z = neumann_eigenvalues(nz)[:, None, None]
    lam_xy = _lambda_grid(ny, nx)[None, :, :]
    h = sfft.dctn(I0, type=2, norm="ortho", workers=-1)
    return sfft.idctn(h * (alpha + lam_xy) / (alpha + lam_xy + lam_z), type=2, norm="ortho", workers=-1)


def apply_Ainv(rhs: np.ndarray, alpha: float) -> np.ndarray:
    """A^{-1} rhs for one slice (A = alpha I + L is diagonal in the DCT-II basis)."""
    rhs = np.asarray(rhs, dtype=np.float64)
    lam = _lambda_grid(*rhs.shape)
    r_hat = sfft.dctn(rhs, type=2, norm="ortho", workers=-1)
    return sfft.idctn(r_hat / (alpha + lam), type=2, norm="ortho", workers=-1)


def relative_residual(f: np.ndarray, s: np.ndarray, o: np.ndarray, alpha: float) -> float:
    """||b - A f||_2 / ||b||_2 for one slice: the residual measure of the solver table in
    Sec. 4 (norm of the residual over norm of the initial constraints)."""
    b = screened_rhs(s, o, alpha)
    r = b - apply_A(f, alpha)
    nb = float(np.linalg.norm(b))
    return float(np.linalg.norm(r)) / nb if nb > 0 else float(np.linalg.norm(r))


def correct_stack(I0: np.ndarray, sigma_xy: float, sigma_z: float, alpha: float):
    """Both phases: I1 = smooth(I0), then I2_j = solve(s = I1_j, o = I0_j) for every j.

    Returns (I1, I2) in float64.
    """
    I0 = np.asarray(I0, dtype=np.float64)
    I1 = smooth_stack(I0, sigma_xy, sigma_z)
    I2 = np.empty_like(I0)
    for j in range(I0.shape[0]):
        I2[j] = solve_dct(I1[j], I0[j], alpha)
    return I1, I2


# --------------------------------------------------------------------------------------
# Adjoint.  f = A^{-1}(alpha s + L o) with A = alpha I + L symmetric, so for a loss l with
# g = dl/df:  lam = A^{-1} g,  dl/ds = alpha lam,  dl/do = L lam,  dl/dalpha = <lam, s - f>.
# Through phase 1 (s = K I0, o = I0): dl/dI0 = L lam + K^T(alpha lam) and
# dl/dsigma_z = <alpha lam, (dK/dsigma_z) I0>.
# --------------------------------------------------------------------------------------
def backward_slice(g: np.ndarray, s: np.ndarray, o: np.ndarray, f: np.ndarray, alpha: float):
    """Gradients of one Eq. (1) solve: returns (dl/ds, dl/do, dl/dalpha)."""
    lam = apply_Ainv(g, alpha)
    ds = alpha * lam
    do = laplacian(lam)
    dalpha = float(np.sum(lam * (np.asarray(s, np.float64) - np.asarray(f, np.float64))))
    return ds, do, dalpha


def backward_stack(g: np.ndarray, I0: np.ndarray, sigma_xy: float, sigma_z: float,
                   alpha: float, radius_z: int | None = None):
    """Gradients of ``correct_stack``'s I2 w.r.t. (I0, alpha, sigma_z) for dl/dI2 = g."""
    I0 = np.asarray(I0, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    s = smooth_stack(I0, sigma_xy, sigma_z, radius_z=radius_z)
    ds = np.empty_like(I0); do = np.empty_like(I0); dalpha = 0.0
    for j in range(I0.shape[0]):
        f = solve_dct(s[j], I0[j], alpha)
        a, b, c = backward_slice(g[j], s[j], I0[j], f, alpha)
        ds[j] = a; do[j] = b; dalpha += c
    dI0 = do + smooth_transpose(ds, sigma_xy, sigma_z, radius_z=radius_z)
    dsig = float(np.sum(ds * dsmooth_dsigma_z(I0, sigma_xy, sigma_z, radius_z=radius_z)))
    return dI0, dalpha, dsig
