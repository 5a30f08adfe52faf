"""FP64 oracle of rendering with a spatially varying (eigen-)PSF (Section 2,
Step 2: the PSF at an image position is a polynomial-weighted sum of
pixelized components, so its FFT is the same weighted sum of the
components' FFTs).

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

Readings (the paper describes the model only in words):
* Position (u, v) in image pixels; X = (u - u0) / su, Y = (v - v0) / sv; the
  polynomial terms of total degree <= D in the order 1, X, Y, X^2, X Y, Y^2.
* The pixelized PSF at (u, v) is sum_c m_c E_c; the oracle forms it in pixel
  space and then takes Steps 1-2 as for a constant PSF (the weighted sum of
  the component FFTs is the same by linearity).
* The real-space half needs a Gaussian mixture of that PSF: the components'
  mixtures share their shapes (mean, covariance) and the amplitudes vary with
  the same polynomial terms, so the mixture at (u, v) has amplitudes
  sum_c m_c A[c, j].
"""

import numpy as np

from .render import render


def monomials(u, v, degree, norm):
    """Polynomial terms 1, X, Y, X^2, X Y, Y^2, ... of total degree <= degree."""
    u0, v0, su, sv = norm
    X = (float(u) - u0) / su
    Y = (float(v) - v0) / sv
    out = []
    for t in range(degree + 1):
        for j in range(t + 1):
            out.append(X ** (t - j) * Y ** j)
    return np.array(out)


def psf_at(eig, u, v):
    """(image, mixture rows (w, mx, my, vxx, vxy, vyy)) of the PSF at (u, v)."""
    m = monomials(u, v, eig.degree, eig.norm)
    comps = np.asarray(eig.components, dtype=np.float64)
    assert len(m) == len(comps)
    image = np.tensordot(m, comps, axes=1)
    amps = m @ np.asarray(eig.mog_amp, dtype=np.float64)
    mog = np.column_stack([amps, np.asarray(eig.mog_shape, dtype=np.float64)])
    return image, mog


def render_eigen(gal, eig, u, v, tables, n=None):
    """Steps 1-8 for one galaxy at image position (u, v)."""
    image, mog = psf_at(eig, u, v)
    return render(gal, image, mog, tables, n=n)
