"""Pins of the oracle's derivatives of the Lanczos sub-pixel-shift model
(Section 2, Step 8 variant) against FP64 central finite differences of the
oracle's own forward Lanczos model, and of the kernel derivative against the
kernel (no GPU)."""

import numpy as np
import pytest

from oracle import lanczos as L
from oracle import render as R
from workloads import single_galaxy_64


def test_kernel_derivative_matches_differences():
    # away from the kinks at |t| = 3 and including t near 0, where L' -> 0
    t = np.concatenate([np.linspace(-2.95, 2.95, 119) + 0.0037, [1e-5, -2e-4, 0.01]])
    h = 1e-6
    fd = (L.lanczos3(t + h) - L.lanczos3(t - h)) / (2 * h)
    np.testing.assert_allclose(L.lanczos3_derivative(t), fd, atol=1e-8)
    assert L.lanczos3_derivative(0.0) == 0.0
    assert np.all(L.lanczos3_derivative(np.array([3.0, -3.5, 4.2])) == 0.0)
    # closed form: L'(1) = sinc'(1) sinc(1/3) = -sinc(1/3) (cos(pi) - 0) ... = -(3 sqrt(3) / (2 pi))
    assert abs(L.lanczos3_derivative(1.0) + 3.0 * np.sqrt(3.0) / (2.0 * np.pi)) < 1e-14


@pytest.mark.parametrize("d", [-0.5, -0.31, 0.0, 0.12, 0.4999])
def test_weight_derivatives(d):
    # at d = 0 the end taps sit at |t| = 3, where L is C^1 but L'' jumps, so a
    # central difference there is off by O(h): a small step keeps that below
    # the tolerance
    h = 2e-8 if d == 0.0 else 1e-6
    fd = (L.lanczos_weights(d + h) - L.lanczos_weights(d - h)) / (2 * h)
    dw = L.lanczos_weights_derivative(d)
    np.testing.assert_allclose(dw, fd, atol=1e-8)
    # the weights sum to one for every d, so their derivatives sum to zero
    assert abs(dw.sum()) < 1e-14


CASES = [
    # (log r_e, profile, e1, e2, x, y, N): all-Fourier, real-space / ramp, Sersic, offsets beyond a pixel
    (np.log(3.0), 0, 0.2, -0.1, 0.3, -0.2, 64),
    (np.log(9.0), 1, 0.3, -0.25, -0.4, 0.1, 64),
    (np.log(4.2), 2, 0.1, 0.1, 2.37, -1.61, 32),
    (np.log(0.4), 1, 0.5, 0.2, -0.3, 0.45, 32),
]


@pytest.mark.parametrize("case", CASES)
def test_jacobian_matches_central_differences(case, tables, psf0):
    lre, prof, e1, e2, x, y, n = case
    g = single_galaxy_64().row(0)
    g.update(log_re=lre, profile=prof, sersic_n=2.7 if prof == 2 else 1.0, e1=e1, e2=e2, x=x, y=y,
             flux=4.3, size=n)
    ph = R.psf_spectrum(psf0.image, n)
    jac = L.jacobian_lanczos(g, ph, psf0.mog, tables)
    names = ("flux", "x", "y", "log_re", "e1", "e2")
    for k, p in enumerate(names):
        h = 1e-5 * g["flux"] if p == "flux" else 1e-5
        gp, gm = dict(g), dict(g)
        gp[p] += h
        gm[p] -= h
        fd = (L.render_lanczos(gp, None, psf0.mog, tables, psf_hat=ph) -
              L.render_lanczos(gm, None, psf0.mog, tables, psf_hat=ph)) / (2 * h)
        assert np.max(np.abs(jac[k] - fd)) < 1e-6 * np.abs(fd).max(), p


def test_sersic_derivative_matches_central_differences(tables, psf0):
    g = single_galaxy_64().row(0)
    g.update(log_re=np.log(5.0), profile=2, sersic_n=2.6, e1=0.2, e2=0.1, x=0.27, y=-0.38, size=64)
    ph = R.psf_spectrum(psf0.image, 64)
    d = L.sersic_derivative_lanczos(g, ph, psf0.mog, tables)
    h = 1e-5
    gp, gm = dict(g), dict(g)
    gp["sersic_n"] += h
    gm["sersic_n"] -= h
    fd = (L.render_lanczos(gp, None, psf0.mog, tables, psf_hat=ph) -
          L.render_lanczos(gm, None, psf0.mog, tables, psf_hat=ph)) / (2 * h)
    assert np.max(np.abs(d - fd)) < 1e-6 * np.abs(fd).max()


def test_vjp_reduces_to_the_phase_model_at_integer_offsets(tables, psf0):
    # at d = 0 the weights are the identity, so every gradient but x and y is
    # the phase-shift model's; x and y then come from the weights' slope at
    # d = 0 applied to the same image
    from oracle import adjoint as A
    g = single_galaxy_64().row(0)
    g.update(x=2.0, y=-1.0)
    ph = R.psf_spectrum(psf0.image, 64)
    rng = np.random.default_rng(5)
    gp = rng.normal(size=(64, 64))
    vl = L.vjp_lanczos(g, ph, psf0.mog, tables, gp)
    va = A.vjp(g, ph, psf0.mog, tables, gp)
    np.testing.assert_allclose(vl[[0, 3, 4, 5]], va[[0, 3, 4, 5]], rtol=1e-12)
