"""Pins of the Lanczos sub-pixel-shift oracle (Section 2, Step 8 variant)
against closed forms, exact identities of the periodic convolution and the
phase-shift method it approximates."""

import numpy as np
import pytest

from oracle import lanczos as L
from oracle import render as R


def _gal(**kw):
    g = dict(flux=1.0, x=0.0, y=0.0, log_re=np.log(3.0), e1=0.0, e2=0.0, sersic_n=1.0, profile=0, psf=0, size=64)
    g.update(kw)
    return g


def _gauss_img(sig, cx, cy, n=64):
    yy, xx = np.mgrid[0:n, 0:n].astype(float)
    return np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * sig * sig))


def test_kernel_closed_form_values():
    # L(t) = sinc(t) sinc(t/3): L(1/2) = (2/pi) (3/pi) = 6/pi^2,
    # L(3/2) = (-2/(3 pi)) (2/pi) = -4/(3 pi^2), zero at non-zero integers
    # and outside |t| < 3.
    assert L.lanczos3(0.0) == 1.0
    assert abs(L.lanczos3(0.5) - 6.0 / np.pi ** 2) < 1e-15
    assert abs(L.lanczos3(-1.5) + 4.0 / (3.0 * np.pi ** 2)) < 1e-15
    assert np.all(np.abs(L.lanczos3(np.array([1.0, 2.0, -1.0, -2.0]))) < 1e-16)
    assert np.all(L.lanczos3(np.array([3.0, -3.0, 3.2, -7.0])) == 0.0)


def test_zero_shift_is_identity():
    img = np.random.default_rng(0).standard_normal((64, 64))
    w = L.lanczos_weights(0.0)
    assert np.array_equal(w, np.array([0, 0, 0, 1, 0, 0, 0], dtype=float))
    assert np.array_equal(L.lanczos_shift(img, 0.0, 0.0), img)


def test_weights_normalised_and_constant_kept():
    for d in (-0.5, -0.37, 0.01, 0.25, 0.49):
        assert abs(L.lanczos_weights(d).sum() - 1.0) < 1e-15
    img = np.full((32, 32), 2.5)
    assert np.max(np.abs(L.lanczos_shift(img, 0.31, -0.42) - img)) < 1e-14


def test_half_pixel_conventions_agree_with_a_roll():
    """Shifting by +1/2 equals shifting by -1/2 and rolling one pixel: this
    fixes the sign and the tap range (taps -3..3 cover both)."""
    img = np.random.default_rng(1).standard_normal((32, 32))
    a = L.lanczos_shift(img, 0.5, 0.0)
    b = np.roll(L.lanczos_shift(img, -0.5, 0.0), 1, axis=1)
    assert np.max(np.abs(a - b)) < 1e-13
    a = L.lanczos_shift(img, 0.0, 0.5)
    b = np.roll(L.lanczos_shift(img, 0.0, -0.5), 1, axis=0)
    assert np.max(np.abs(a - b)) < 1e-13


def test_separable_and_mirror():
    img = np.random.default_rng(2).standard_normal((32, 32))
    both = L.lanczos_shift(img, 0.3, -0.2)
    seq = L.lanczos_shift(L.lanczos_shift(img, 0.3, 0.0), 0.0, -0.2)
    assert np.max(np.abs(both - seq)) < 1e-13
    # x -> -x (mod N) turns a shift by d into a shift by -d
    flip = lambda a: np.roll(a[:, ::-1], 1, axis=1)
    assert np.max(np.abs(flip(L.lanczos_shift(img, 0.3, 0.0)) - L.lanczos_shift(flip(img), -0.3, 0.0))) < 1e-13


def test_shift_of_well_sampled_gaussian():
    """A sampled Gaussian of sigma 3 px shifted by d is the Gaussian sampled at
    the shifted centre, up to Lanczos-3 interpolation error (measured 3.4e-3
    of the peak at sigma 3 and 2.4e-3 at sigma 6: the normalised Lanczos-3
    response is not flat in the pass band)."""
    for dx, dy in [(0.3, -0.2), (-0.5, 0.45), (0.11, 0.0)]:
        got = L.lanczos_shift(_gauss_img(3.0, 32, 32), dx, dy)
        want = _gauss_img(3.0, 32 + dx, 32 + dy)
        assert np.max(np.abs(got - want)) < 6e-3
        got = L.lanczos_shift(_gauss_img(6.0, 32, 32), dx, dy)
        want = _gauss_img(6.0, 32 + dx, 32 + dy)
        assert np.max(np.abs(got - want)) < 4e-3


def test_split_offset():
    for x, n, d in [(0.3, 0.0, 0.3), (-0.5, 0.0, -0.5), (0.5, 1.0, -0.5), (1.3, 1.0, 0.3), (-2.7, -3.0, 0.3)]:
        gn, gd = L.split_offset(x)
        assert gn == n and abs(gd - d) < 1e-12


def test_point_source_is_shifted_psf(tables, psf0):
    """A galaxy of negligible size rendered with the Lanczos shift is the
    embedded PSF rolled by the integer offset and Lanczos-shifted by the rest
    (the point-source limit the paper gives as the reason for this variant)."""
    g = _gal(log_re=np.log(1e-7), x=1.3, y=-0.4, flux=2.0)
    got = L.render_lanczos(g, psf0.image, psf0.mog, tables)
    want = 2.0 * L.lanczos_shift(np.roll(R.embed_psf(psf0.image, 64), (0, 1), axis=(0, 1)), 0.3, -0.4)
    assert np.max(np.abs(got - want)) < 1e-12


def test_integer_offsets_need_no_interpolation(tables, psf0):
    g = _gal(x=2.0, y=-1.0, e1=0.2, e2=-0.1, log_re=np.log(5.0), profile=1, sersic_n=4.0)
    assert np.array_equal(L.render_lanczos(g, psf0.image, psf0.mog, tables), R.render(g, psf0.image, psf0.mog, tables))


@pytest.mark.parametrize("profile,log_re", [(0, np.log(4.0)), (1, np.log(6.0)), (0, np.log(15.0))])
def test_close_to_phase_shift_for_smooth_models(tables, psf0, profile, log_re):
    """For models that are smooth on the pixel scale (the PSF has sigma
    1.5 px) the Lanczos and Fourier-phase shifts agree to interpolation
    error: within 1e-2 of the peak (measured up to 3.9e-3).  The periodic,
    normalised convolution keeps the patch sum of the integer-offset model
    exactly."""
    g = _gal(x=0.37, y=-0.29, e1=0.15, e2=0.1, log_re=log_re, profile=profile, sersic_n=1.0 if profile == 0 else 4.0)
    a = L.render_lanczos(g, psf0.image, psf0.mog, tables)
    b = R.render(g, psf0.image, psf0.mog, tables)
    assert np.max(np.abs(a - b)) < 1e-2 * np.max(b)
    c = R.render(dict(g, x=0.0, y=0.0), psf0.image, psf0.mog, tables)
    assert abs(a.sum() - c.sum()) < 1e-12 * abs(c.sum())
