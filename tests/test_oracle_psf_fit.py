"""Pins of the PSF-mixture fitting oracle: an image that is exactly a sampled
Gaussian mixture must be recovered (parameters and chi^2 ~ 0), the mixture
image must match the plain Gaussian formula, and the fit of a real PSF must
not be worse than its own starting point or a one-component fit."""

import numpy as np
import pytest

from oracle import psf_fit as F
from workloads import psf_set


def _gauss_image(rows, n=32):
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64)
    img = np.zeros((n, n))
    for w, mx, my, vxx, vxy, vyy in rows:
        cov = np.array([[vxx, vxy], [vxy, vyy]])
        inv = np.linalg.inv(cov)
        d = np.stack([xx - n // 2 - mx, yy - n // 2 - my], axis=-1)
        q = np.einsum("...i,ij,...j->...", d, inv, d)
        img += w * np.exp(-0.5 * q) / (2 * np.pi * np.sqrt(np.linalg.det(cov)))
    return img


def test_mixture_image_is_the_gaussian_formula():
    rows = np.array([[0.7, 0.3, -0.2, 2.0, 0.4, 1.5], [0.3, -0.5, 0.1, 6.0, -1.0, 5.0]])
    assert np.max(np.abs(F.mixture_image(rows, 32, 32) - _gauss_image(rows))) < 1e-15


@pytest.mark.parametrize("truth", [
    [[0.8, 0.0, 0.0, 2.25, 0.0, 2.25], [0.2, 0.0, 0.0, 9.0, 0.0, 9.0]],
    [[0.6, 0.25, -0.15, 2.0, 0.5, 1.6], [0.3, -0.1, 0.2, 6.0, -1.2, 4.5], [0.1, 0.0, 0.0, 20.0, 0.0, 20.0]],
])
def test_exact_mixture_is_recovered(truth):
    truth = np.array(truth)
    img = _gauss_image(truth)
    rows, c2 = F.fit_mog(img, k=len(truth))
    assert c2 < 1e-20
    assert np.max(np.abs(rows - truth[np.argsort(-truth[:, 0])])) < 1e-6


def test_fit_of_a_winged_psf_improves_on_start_and_on_fewer_components():
    psf = psf_set(1, seed=3)[0].image.astype(np.float64)
    rows3, c3 = F.fit_mog(psf, 3)
    rows1, c1 = F.fit_mog(psf, 1)
    start = F.chi2(F.mixture_rows(F.initial_parameters(psf, 3)), psf)
    assert c3 < 1e-2 * start and c3 < c1
    assert abs(rows3[:, 0].sum() - psf.sum()) < 0.05


def test_winged_psf_fit_reaches_the_multistart_optimum():
    """The oracle's fit is local (Levenberg-Marquardt from a fixed start).  On
    a Moffat-winged PSF its chi^2 equals the best of several random starts of
    a different minimiser (BFGS on chi^2 itself) over an objective written
    out here with the plain Gaussian formula, so the fixed start finds the
    global optimum of the objective there, not merely a local one."""
    from scipy.optimize import minimize
    psf = psf_set(1, seed=3)[0].image.astype(np.float64)
    n = psf.shape[0]
    k = 3
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64)

    def c2(p):
        # sum_j w_j N(p - c - m_j; V_j) with V_j = L L^T, L = [[a, 0], [b, c]]:
        # V^-1 = [[vyy, -vxy], [-vxy, vxx]] / det, det = (a c)^2
        model = np.zeros((n, n))
        for j in range(k):
            lw, mx, my, la, b, lc = p[6 * j:6 * j + 6]
            a, c = np.exp(la), np.exp(lc)
            vxx, vxy, vyy = a * a, a * b, b * b + c * c
            det = (a * c) ** 2
            ex, ey = xx - n // 2 - mx, yy - n // 2 - my
            model += np.exp(lw - 0.5 * (vyy * ex * ex - 2 * vxy * ex * ey + vxx * ey * ey) / det) / (2 * np.pi * a * c)
        return float(((model - psf) ** 2).sum())

    rng = np.random.default_rng(0)
    best = np.inf
    for _ in range(5):
        w = rng.dirichlet(np.ones(k)) * psf.sum()
        p = []
        for j in range(k):
            sig = np.exp(rng.uniform(np.log(0.7), np.log(8.0)))
            p += [np.log(w[j]), rng.normal(0, 0.3), rng.normal(0, 0.3), np.log(sig), rng.normal(0, 0.2 * sig),
                  np.log(sig * np.exp(rng.normal(0, 0.2)))]
        best = min(best, minimize(c2, np.array(p), method="BFGS", options=dict(maxiter=1200, gtol=1e-14)).fun)
    _, c_oracle = F.fit_mog(psf, k)
    assert c_oracle <= best * (1 + 1e-4)
