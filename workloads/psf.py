"""Synthetic pixelized PSFs and their Gaussian-mixture fits.

A pixelized PSF here is an h x w float32 image whose centre is pixel
(h // 2, w // 2) (row, column), normalised to unit sum.  Pixel values are the
continuous profile point-sampled at pixel centres; pixelized PSF models built
from real images are already pixel-convolved (Section 1), so sampling at
centres is the consistent choice for a synthetic stand-in.

The real-space half of the method needs a Gaussian-mixture approximation of
the PSF (Section 2, Step 4, which uses one Gaussian; here a small mixture is
fitted by direct chi-squared minimisation, as Section 1 describes for the
earlier approach).  The fit is input preparation: it is computed once per PSF
and handed to both the CUDA path and the oracle, so both convolve with the
same mixture.  Mixture rows are (weight, mean_x, mean_y, var_xx, var_xy,
var_yy) with the mean relative to the PSF centre pixel.
"""

from dataclasses import dataclass

import numpy as np
from scipy.optimize import least_squares


@dataclass
class PsfInput:
    image: np.ndarray      # (h, w) float32, unit sum, centre at (h // 2, w // 2)
    mog: np.ndarray        # (K, 6) float64: w, mx, my, vxx, vxy, vyy
    mog_exact: np.ndarray = None  # the generating mixture when the PSF is an exact MoG


def _grid(size):
    c = size // 2
    yy, xx = np.mgrid[0:size, 0:size].astype(np.float64)
    return xx - c, yy - c


def _gauss_pix(dx, dy, vxx, vxy, vyy):
    det = vxx * vyy - vxy * vxy
    q = (vyy * dx * dx - 2 * vxy * dx * dy + vxx * dy * dy) / det
    return np.exp(-0.5 * q) / (2 * np.pi * np.sqrt(det))


def gaussian_mixture_psf(weights, sigmas, size=64):
    """Isotropic centred Gaussian mixture sampled at pixel centres, normalised
    to unit sum.  Returns ``(image float32, exact_mog)``."""
    dx, dy = _grid(size)
    img = np.zeros((size, size))
    mog = []
    for w, s in zip(weights, sigmas):
        img += w * _gauss_pix(dx, dy, s * s, 0.0, s * s)
        mog.append([w, 0.0, 0.0, s * s, 0.0, s * s])
    tot = img.sum()
    img /= tot
    mog = np.array(mog)
    mog[:, 0] /= tot
    return img.astype(np.float32), mog


def moffat_image(alpha, beta, size=64):
    dx, dy = _grid(size)
    img = (1.0 + (dx * dx + dy * dy) / (alpha * alpha)) ** (-beta)
    return img / img.sum()


def fit_psf_mog(image, k=3):
    """Chi-squared fit of a k-component Gaussian mixture (free means and full
    covariances) to a pixelized PSF, evaluated at pixel centres.  Returns a
    (k, 6) array sorted by decreasing weight."""
    image = np.asarray(image, dtype=np.float64)
    size = image.shape[0]
    assert image.shape == (size, size)
    dx, dy = _grid(size)
    tot = image.sum()
    s_est = np.sqrt(max((image * (dx * dx + dy * dy)).sum() / (2 * tot), 0.25))
    scales = np.array([0.6, 1.1, 2.2, 4.0, 6.0])[:k]
    w0 = np.array([0.55, 0.35, 0.08, 0.015, 0.005])[:k]
    w0 = w0 / w0.sum() * tot
    p0 = []
    for j in range(k):
        p0 += [np.log(w0[j]), 0.0, 0.0, np.log(s_est * scales[j]), 0.0, np.log(s_est * scales[j])]
    p0 = np.array(p0)

    def unpack(p):
        comps = []
        for j in range(k):
            lw, mx, my, la, b, lc = p[6 * j:6 * j + 6]
            a, c = np.exp(la), np.exp(lc)
            comps.append((np.exp(lw), mx, my, a * a, a * b, b * b + c * c))
        return comps

    def parts(p):
        out = []
        for w, mx, my, vxx, vxy, vyy in unpack(p):
            ex, ey = dx - mx, dy - my
            out.append((w, ex, ey, vxx, vxy, vyy, _gauss_pix(ex, ey, vxx, vxy, vyy)))
        return out

    def resid(p):
        m = -image.copy()
        for w, *_, g in parts(p):
            m += w * g
        return m.ravel()

    def jac(p):
        cols = []
        for j, (w, ex, ey, vxx, vxy, vyy, g) in enumerate(parts(p)):
            a, b, c = np.exp(p[6 * j + 3]), p[6 * j + 4], np.exp(p[6 * j + 5])
            det = vxx * vyy - vxy * vxy
            ixx, ixy, iyy = vyy / det, -vxy / det, vxx / det
            ux, uy = ixx * ex + ixy * ey, ixy * ex + iyy * ey      # P^-1 d
            qxx, qxy, qyy = 0.5 * (ux * ux - ixx), 0.5 * (ux * uy - ixy), 0.5 * (uy * uy - iyy)
            wg = w * g
            cols += [wg, wg * ux, wg * uy,
                     wg * (qxx * 2 * a * a + 2 * qxy * a * b),
                     wg * (2 * qxy * a + qyy * 2 * b),
                     wg * (qyy * 2 * c * c)]
        return np.stack([col.ravel() for col in cols], axis=1)

    res = least_squares(resid, p0, jac=jac, method="lm",
                        xtol=1e-12, ftol=1e-12, gtol=1e-12, max_nfev=4000)
    comps = np.array(unpack(res.x))
    comps = comps[np.argsort(-comps[:, 0])]
    return comps


def single_psf(size=64, k_fit=3):
    """0.8 N(sigma=1.5) + 0.2 N(sigma=3.0) px on a 64 x 64 grid, plus its
    k_fit-component mixture fit."""
    img, exact = gaussian_mixture_psf([0.8, 0.2], [1.5, 3.0], size)
    return PsfInput(image=img, mog=fit_psf_mog(img, k_fit), mog_exact=exact)


def psf_set(n=64, seed=22, size=64, k_fit=3, fit=True):
    """``n`` PSFs: a core 0.8 N(s) + 0.2 N(2 s) with s uniform in 1.2-2.5 px,
    plus Moffat (beta = 3) wings at weight 0.05 whose FWHM equals that of the
    N(2 s) core component (alpha = 4.62 s); each sampled at pixel centres on a
    ``size`` grid and normalised."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        s = rng.uniform(1.2, 2.5)
        core, _ = gaussian_mixture_psf([0.8, 0.2], [s, 2 * s], size)
        wings = moffat_image(4.62 * s, 3.0, size)
        img = 0.95 * core.astype(np.float64) + 0.05 * wings
        img = (img / img.sum()).astype(np.float32)
        out.append(PsfInput(image=img, mog=fit_psf_mog(img, k_fit) if fit else None))
    return out


# ---------------------------------------------------------------------------
# Spatially varying PSFs as eigen-PSF models (Section 2, Step 2): the PSF at
# image position (u, v) is sum_c m_c(X, Y) E_c, X = (u - u0) / su,
# Y = (v - v0) / sv, with the monomials m_c of total degree <= D in the order
# 1, X, Y, X^2, X Y, Y^2 and pixelized components E_c, as PSF-modelling tools
# produce them.  The Gaussian mixture for real-space terms shares its shapes
# across components and varies only its amplitudes the same way.
# ---------------------------------------------------------------------------

@dataclass
class EigenPsfInput:
    components: np.ndarray   # (K, h, w) float32, K = (D + 1)(D + 2) / 2
    degree: int
    norm: tuple              # (u0, v0, su, sv)
    mog_shape: np.ndarray    # (k, 5) float64: mx, my, vxx, vxy, vyy
    mog_amp: np.ndarray      # (K, k) float64: amplitude of each shape in each component


def eigen_monomials(u, v, degree, norm):
    """(K,) or (K, n) monomials 1, X, Y, X^2, X Y, Y^2 (up to ``degree``)."""
    u0, v0, su, sv = norm
    X = (np.asarray(u, dtype=np.float64) - u0) / su
    Y = (np.asarray(v, dtype=np.float64) - v0) / sv
    out = []
    for t in range(degree + 1):
        for j in range(t + 1):
            out.append(X ** (t - j) * Y ** j)
    return np.array(out)


def varying_psf_image(X, Y, size=64):
    """The synthetic field PSF at normalised position (X, Y) in [-1, 1]^2: a
    0.8 / 0.2 two-Gaussian core whose width and ellipticity drift smoothly
    across the image, sampled at pixel centres and normalised."""
    s = 1.6 + 0.3 * X - 0.2 * Y + 0.15 * X * Y
    e1, e2 = 0.06 * X, 0.05 * Y
    dx, dy = _grid(size)
    img = np.zeros((size, size))
    for w, sc in ((0.8, 1.0), (0.2, 2.0)):
        v = (s * sc) ** 2
        img += w * _gauss_pix(dx, dy, v * (1 + e1), v * e2, v * (1 - e1))
    return img / img.sum()


def eigen_psf(degree=2, size=64, image_size=4096.0, grid=7, k_fit=3):
    """Eigen-PSF model of ``varying_psf_image`` over an ``image_size``-pixel
    square image: each pixel's polynomial coefficients fitted by least squares
    to the PSF sampled on a ``grid`` x ``grid`` lattice of positions (as
    PSF-modelling tools do with stars), and a shared-shape Gaussian mixture
    whose amplitudes are fitted per component."""
    h = image_size / 2.0
    norm = (h, h, h, h)
    g = np.linspace(-1.0, 1.0, grid)
    XX, YY = np.meshgrid(g, g)
    pos = np.stack([XX.ravel(), YY.ravel()], axis=1)
    imgs = np.stack([varying_psf_image(X, Y, size).ravel() for X, Y in pos])
    M = eigen_monomials(h + h * pos[:, 0], h + h * pos[:, 1], degree, norm).T   # (n_pos, K)
    coef, *_ = np.linalg.lstsq(M, imgs, rcond=None)
    comps = coef.reshape(-1, size, size)
    # shared shapes: centred isotropic Gaussians spanning the core widths (a
    # free fit gives nearly equal shapes and ill-conditioned amplitudes)
    shapes = np.array([[0.0, 0.0, s * s, 0.0, s * s] for s in (1.3, 1.9, 3.6)[:k_fit]])
    dx, dy = _grid(size)
    G = np.stack([_gauss_pix(dx - mx, dy - my, vxx, vxy, vyy).ravel() for mx, my, vxx, vxy, vyy in shapes], axis=1)
    amp, *_ = np.linalg.lstsq(G, comps.reshape(len(comps), -1).T, rcond=None)
    return EigenPsfInput(components=comps.astype(np.float32), degree=degree, norm=norm,
                         mog_shape=shapes, mog_amp=amp.T.copy())


def eigen_positions(g, seed=24, image_size=4096.0):
    """Image positions (u, v) of ``g`` galaxies, uniform over the image."""
    rng = np.random.default_rng(seed)
    return (rng.uniform(0.0, image_size, g).astype(np.float32),
            rng.uniform(0.0, image_size, g).astype(np.float32))
