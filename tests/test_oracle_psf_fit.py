"""Pins of the PSF-mixture fitting oracle: an image that is exactly a sampled
Gaussian mixture must be recovered (parameters and chi^2 ~ 0), the mixture
image must match the plain Gaussian formula, and the fit of a real PSF must
not be worse than its own starting point or a one-component fit."""

import numpy as np
import pytest

from oracle import psf_fit as F
from workloads import config2_psfs


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
    psf = config2_psfs(1, seed=3)[0].image.astype(np.float64)
    rows3, c3 = F.fit_mog(psf, 3)
    rows1, c1 = F.fit_mog(psf, 1)
    start = F.chi2(F.mixture_rows(F.initial_parameters(psf, 3)), psf)
    assert c3 < 1e-2 * start and c3 < c1
    assert abs(rows3[:, 0].sum() - psf.sum()) < 0.05
