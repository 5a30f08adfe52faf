"""Pins of the oracle's analytic derivatives against FP64 central finite
differences of the oracle's forward model (no GPU)."""

import numpy as np
import pytest

from oracle import adjoint as A
from oracle import render as R
from workloads import single_galaxy_64

CASES = [
    # (log r_e, profile, e1, e2, x, y, N): all-Fourier, ramp, real-space, tiny
    (np.log(3.0), 0, 0.2, -0.1, 0.3, -0.2, 64),
    (np.log(9.0), 1, 0.3, -0.25, -0.4, 0.1, 64),
    (np.log(12.0), 0, -0.2, 0.35, 0.05, 0.45, 64),
    (np.log(6.5), 0, 0.001, 0.0005, 0.2, 0.2, 64),
    (np.log(0.4), 1, 0.5, 0.2, -0.3, -0.5, 32),
    (np.log(4.2), 2, 0.1, 0.1, 0.1, -0.1, 32),
]


@pytest.mark.parametrize("case", CASES)
def test_jacobian_matches_central_differences(case, tables, psf0):
    lre, prof, e1, e2, x, y, n = case
    g = single_galaxy_64().row(0)
    g.update(log_re=lre, profile=prof, sersic_n=2.7 if prof == 2 else 1.0, e1=e1, e2=e2, x=x, y=y,
             flux=4.3, size=n)
    ph = R.psf_spectrum(psf0.image, n)
    jac = A.jacobian(g, ph, psf0.mog, tables)
    # near e = 0 the curvature in (e1, e2) grows like 1/e: shrink the step
    step = 1e-5 if np.hypot(e1, e2) > 0.01 else 1e-7
    fd = A.finite_difference(g, ph, psf0.mog, tables, step=step)
    for k in range(6):
        scale = np.abs(fd[k]).max()
        assert np.max(np.abs(jac[k] - fd[k])) < 1e-6 * scale, A.PARAMS[k]


def test_vjp_is_jacobian_contraction(tables, psf0):
    g = single_galaxy_64().row(0)
    ph = R.psf_spectrum(psf0.image, 64)
    rng = np.random.default_rng(3)
    gp = rng.normal(size=(64, 64))
    v = A.vjp(g, ph, psf0.mog, tables, gp)
    fd = A.finite_difference(g, ph, psf0.mog, tables, step=1e-6)
    want = np.tensordot(fd, gp, axes=([1, 2], [0, 1]))
    np.testing.assert_allclose(v, want, rtol=1e-6, atol=1e-9 * np.abs(want).max())


def test_shape_derivatives_match_differences():
    for lre, e1, e2 in [(0.3, 0.2, -0.1), (1.7, -0.45, 0.3), (-0.5, 0.01, 0.002)]:
        ds = A.shape_derivatives(lre, e1, e2)
        h = 1e-6
        args = [lre, e1, e2]
        for k in range(3):
            up, dn = list(args), list(args)
            up[k] += h
            dn[k] -= h
            fd = (R.ellipse_covariance(np.exp(up[0]), up[1], up[2]) -
                  R.ellipse_covariance(np.exp(dn[0]), dn[1], dn[2])) / (2 * h)
            np.testing.assert_allclose(ds[k], fd, rtol=1e-7, atol=1e-8 * np.abs(fd).max())


def test_subpixel_motion_is_smooth_for_point_source(tables, psf0):
    """Section 1's point-source thought experiment: with this method the image
    of a tiny galaxy moves smoothly; d pixel / dx exists and matches FD at
    every subpixel phase."""
    ph = R.psf_spectrum(psf0.image, 64)
    for x in np.linspace(-0.5, 0.5, 5):
        g = single_galaxy_64().row(0)
        g.update(log_re=np.log(1e-3), x=x, e1=0.1, e2=0.05)
        jac = A.jacobian(g, ph, psf0.mog, tables)
        fd = A.finite_difference(g, ph, psf0.mog, tables, step=1e-5)
        assert np.max(np.abs(jac[1] - fd[1])) < 1e-6 * np.abs(fd[1]).max()


@pytest.mark.parametrize("cd", [np.array([[0.8, 0.25], [-0.15, 1.2]]), np.array([[-1.1, 0.4], [0.3, 0.9]])])
def test_jacobian_with_wcs_matrix(cd, tables, psf0):
    """A general WCS matrix (Appendix A): the analytic Jacobian against central
    differences of the forward model rendered with the same CD."""
    for lre, prof in ((np.log(3.0), 0), (np.log(9.0), 1)):
        g = single_galaxy_64().row(0)
        g.update(log_re=lre, profile=prof, sersic_n=4.0 if prof == 1 else 1.0, e1=0.25, e2=-0.2, x=0.3, y=-0.1,
                 flux=2.0, size=64)
        ph = R.psf_spectrum(psf0.image, 64)
        jac = A.jacobian(g, ph, psf0.mog, tables, cd=cd)
        fd = A.finite_difference(g, ph, psf0.mog, tables, step=1e-5, cd=cd)
        for k in range(6):
            scale = np.abs(fd[k]).max()
            assert np.max(np.abs(jac[k] - fd[k])) < 1e-6 * scale, A.PARAMS[k]


@pytest.mark.parametrize("sn,lre,n", [(2.6, np.log(3.0), 64), (4.375, np.log(9.0), 64), (1.13, np.log(14.0), 32),
                                       (5.3, np.log(0.6), 32)])
def test_sersic_derivative_matches_central_differences(sn, lre, n, tables, psf0):
    """d pixel / d n through the interpolated Sersic table (all-Fourier, ramp
    and real-space cases), against central differences in n away from the
    table's nodes (n = 0.5 + 0.25 k)."""
    g = single_galaxy_64().row(0)
    g.update(profile=2, sersic_n=sn, log_re=lre, e1=0.2, e2=-0.15, x=0.3, y=-0.2, flux=3.0, size=n)
    ph = R.psf_spectrum(psf0.image, n)
    got = A.sersic_derivative(g, ph, psf0.mog, tables)
    h = 1e-5
    gp, gm = dict(g, sersic_n=sn + h), dict(g, sersic_n=sn - h)
    fd = (R.render(gp, None, psf0.mog, tables, psf_hat=ph) - R.render(gm, None, psf0.mog, tables, psf_hat=ph)) / (2 * h)
    assert np.max(np.abs(got - fd)) < 1e-6 * np.abs(fd).max()


def test_sersic_derivative_zero_for_fixed_profiles_and_outside_the_table(tables, psf0):
    g = single_galaxy_64().row(0)
    ph = R.psf_spectrum(psf0.image, 64)
    for prof, sn in ((0, 1.0), (1, 4.0), (2, 6.7), (2, 0.2)):
        g.update(profile=prof, sersic_n=sn, log_re=np.log(6.0))
        assert np.all(A.sersic_derivative(g, ph, psf0.mog, tables) == 0.0)
