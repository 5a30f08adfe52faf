"""Pins of the eigen-PSF oracle (Section 2, Step 2, spatially varying PSF)
against closed forms and the constant-PSF method it reduces to."""

from dataclasses import dataclass

import numpy as np

from oracle import eigenpsf as E
from oracle import render as R
from workloads import gaussian_mixture_psf
from workloads.psf import eigen_psf


@dataclass
class _Eig:
    components: np.ndarray
    degree: int
    norm: tuple
    mog_shape: np.ndarray
    mog_amp: np.ndarray


def _gal(**kw):
    g = dict(flux=3.0, x=0.21, y=-0.33, log_re=np.log(4.0), e1=0.2, e2=-0.15, sersic_n=1.0, profile=0, psf=0,
             size=64)
    g.update(kw)
    return g


def test_monomials_closed_form():
    norm = (100.0, 200.0, 50.0, 25.0)
    # X = (150 - 100) / 50 = 1, Y = (150 - 200) / 25 = -2
    m = E.monomials(150.0, 150.0, 2, norm)
    assert np.array_equal(m, np.array([1.0, 1.0, -2.0, 1.0, -2.0, 4.0]))
    assert np.array_equal(E.monomials(7.0, 9.0, 0, norm), np.array([1.0]))
    assert len(E.monomials(0.0, 0.0, 1, norm)) == 3


def _two_psf_model():
    """Degree-1 model whose PSF is A at X = 0 and B at X = 1 (any Y): shapes
    N(1.5), N(3.0); A = 0.7 / 0.3, B = 0.4 / 0.6 of them."""
    a_img, a_mog = gaussian_mixture_psf([0.7, 0.3], [1.5, 3.0], 64)
    b_img, b_mog = gaussian_mixture_psf([0.4, 0.6], [1.5, 3.0], 64)
    a_img, b_img = a_img.astype(np.float64), b_img.astype(np.float64)
    comps = np.stack([a_img, b_img - a_img, np.zeros_like(a_img)])
    shapes = a_mog[:, 1:]
    amp = np.stack([a_mog[:, 0], b_mog[:, 0] - a_mog[:, 0], np.zeros(2)])
    eig = _Eig(comps, 1, (1000.0, 1000.0, 500.0, 500.0), shapes, amp)
    return eig, (a_img, a_mog), (b_img, b_mog)


def test_model_reduces_to_the_constant_psf_at_its_nodes(tables):
    eig, (a_img, a_mog), (b_img, b_mog) = _two_psf_model()
    g = _gal()
    for u, v, (img, mog) in [(1000.0, 1000.0, (a_img, a_mog)), (1000.0, 123.0, (a_img, a_mog)),
                             (1500.0, 1800.0, (b_img, b_mog))]:
        got = E.render_eigen(g, eig, u, v, tables)
        want = R.render(g, img, mog, tables)
        assert np.max(np.abs(got - want)) < 1e-12 * g["flux"]
    # half way: the PSF is the average, so is the image (the method is linear in the PSF)
    got = E.render_eigen(g, eig, 1250.0, 0.0, tables)
    want = 0.5 * (R.render(g, a_img, a_mog, tables) + R.render(g, b_img, b_mog, tables))
    assert np.max(np.abs(got - want)) < 1e-12 * g["flux"]


def test_degree_zero_is_the_constant_psf(tables, psf0):
    eig = _Eig(psf0.image[None].astype(np.float64), 0, (0.0, 0.0, 1.0, 1.0), psf0.mog[:, 1:], psf0.mog[None, :, 0])
    g = _gal(log_re=np.log(15.0), profile=1, sersic_n=4.0)   # real-space terms too
    got = E.render_eigen(g, eig, 123.0, 456.0, tables)
    assert np.max(np.abs(got - R.render(g, psf0.image, psf0.mog, tables))) < 1e-12 * g["flux"]


def test_linear_in_the_components(tables):
    """The image at (u, v) is sum_c m_c (image rendered with component c and
    its mixture amplitudes), the weighted sum the GPU forms in Fourier space."""
    eig = eigen_psf()
    g = _gal(log_re=np.log(12.0), profile=1, sersic_n=4.0, x=-0.4, y=0.45)
    u, v = 3100.0, 700.0
    m = E.monomials(u, v, eig.degree, eig.norm)
    want = np.zeros((64, 64))
    for c in range(len(m)):
        mog = np.column_stack([eig.mog_amp[c], eig.mog_shape])
        want += m[c] * R.render(g, eig.components[c].astype(np.float64), mog, tables)
    got = E.render_eigen(g, eig, u, v, tables)
    assert np.max(np.abs(got - want)) < 1e-11 * g["flux"]
