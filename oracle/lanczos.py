"""FP64 oracle of the Lanczos sub-pixel-shift variant (Section 2, Step 8:
the sub-pixel shift done by Lanczos convolution of the final pixel-space
model instead of by the Fourier phase of Eq. onegaussian).

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

Readings (the paper names the Lanczos convolution but not its details):
* Lanczos order 3: L(t) = sinc(t) sinc(t/3) for |t| < 3, else 0, with
  sinc(t) = sin(pi t) / (pi t).
* The offset x splits into an integer part n = floor(x + 1/2), applied
  exactly (Fourier phase of an integer shift, real-space centre at N/2 + n),
  and a fraction d = x - n in [-1/2, 1/2), applied by the convolution.
* Shifting by d: J(x) = sum_{a=-3..3} w_a I(x - a), w_a = L(a - d) / sum_b
  L(b - d) (weights normalised, so flux is kept), separably along x and y.
* The patch is treated as periodic (indices mod N), as the inverse FFT's
  output is.
* The convolution is applied to the whole model, Fourier part plus the
  real-space terms (Step 8 adds the real-space terms first).
"""

import numpy as np

from .render import render, psf_spectrum

TAPS = np.arange(-3, 4)


def sinpi(t):
    """sin(pi t) with the reduction t = k + r, k = round(t), done exactly:
    sin(pi t) = (-1)^k sin(pi r), so integers give exactly 0."""
    t = np.asarray(t, dtype=np.float64)
    k = np.rint(t)
    return np.where(np.mod(k, 2.0) == 0.0, 1.0, -1.0) * np.sin(np.pi * (t - k))


def lanczos3(t):
    """L(t) = sinc(t) sinc(t/3) on |t| < 3, zero outside; L(0) = 1."""
    t = np.asarray(t, dtype=np.float64)
    safe = np.where(t == 0.0, 1.0, t)
    v = 3.0 * sinpi(safe) * sinpi(safe / 3.0) / (np.pi * np.pi * safe * safe)
    return np.where(t == 0.0, 1.0, np.where(np.abs(t) < 3.0, v, 0.0))


def lanczos_weights(d):
    """Normalised weights w_a, a = -3..3, of a shift by d."""
    w = lanczos3(TAPS - d)
    return w / w.sum()


def lanczos_shift(img, dx, dy):
    """Periodic separable Lanczos-3 shift of an image indexed [y, x] by
    (dx, dy): the content moves towards +x by dx and +y by dy."""
    img = np.asarray(img, dtype=np.float64)
    wx, wy = lanczos_weights(dx), lanczos_weights(dy)
    tmp = np.zeros_like(img)
    for a, w in zip(TAPS, wx):
        tmp += w * np.roll(img, a, axis=1)      # I[y, x - a]
    out = np.zeros_like(img)
    for b, w in zip(TAPS, wy):
        out += w * np.roll(tmp, b, axis=0)      # tmp[y - b, x]
    return out


def split_offset(x):
    """(n, d): x = n + d with n = floor(x + 1/2) and d in [-1/2, 1/2)."""
    n = float(np.floor(x + 0.5))
    return n, float(x) - n


def render_lanczos(gal, psf_image, psf_mog, tables, n=None, psf_hat=None):
    """The model of ``oracle.render.render`` with its sub-pixel shift done by
    Lanczos convolution: Steps 1-8 at the integer offset, then the shift by
    the fractional part."""
    nx, dx = split_offset(gal["x"])
    ny, dy = split_offset(gal["y"])
    g = dict(gal)
    g["x"], g["y"] = nx, ny
    return lanczos_shift(render(g, psf_image, psf_mog, tables, n=n, psf_hat=psf_hat), dx, dy)


def render_batch_lanczos(gals, psfs, tables):
    """``render_lanczos`` for every galaxy of a ``workloads.Galaxies`` batch."""
    cache = {}
    out = []
    for i in range(len(gals)):
        g = gals.row(i)
        key = (g["psf"], g["size"])
        if key not in cache:
            cache[key] = psf_spectrum(psfs[g["psf"]].image, g["size"])
        out.append(render_lanczos(g, None, psfs[g["psf"]].mog, tables, psf_hat=cache[key]))
    return out


# ----------------------------------------------------------------------------
# Derivatives of the Lanczos variant (its adjoint).  J = Lz_d(I_n): the model
# I rendered at the integer offset n, convolved with the normalised weights
# of the fraction d.  Parameters other than the offset enter through I only;
# the offset enters through d only (n is piecewise constant), so
#   dJ/dtheta = Lz_d(dI/dtheta)              (flux, log r_e, e1, e2, Sersic n)
#   dJ/dx     = (dLz/d d_x)(I_n),  dJ/dy = (dLz/d d_y)(I_n).
# ----------------------------------------------------------------------------

def lanczos3_derivative(t):
    """L'(t): with sinc'(t) = (cos(pi t) - sinc(t)) / t,
    L'(t) = sinc'(t) sinc(t/3) + sinc(t) (cos(pi t / 3) - sinc(t/3)) / t on
    0 < |t| < 3; L'(0) = 0 (L is even) and L' = 0 for |t| >= 3 (continuous
    there, since sinc(+-3) = sinc(+-1) = 0)."""
    t = np.asarray(t, dtype=np.float64)
    safe = np.where(t == 0.0, 1.0, t)
    s1 = sinpi(safe) / (np.pi * safe)
    s3 = 3.0 * sinpi(safe / 3.0) / (np.pi * safe)
    c1, c3 = np.cos(np.pi * safe), np.cos(np.pi * safe / 3.0)
    v = ((c1 - s1) * s3 + s1 * (c3 - s3)) / safe
    return np.where(t == 0.0, 0.0, np.where(np.abs(t) < 3.0, v, 0.0))


def lanczos_weights_derivative(d):
    """d w_a / d d of the normalised weights w_a = L(a - d) / sum_b L(b - d):
    (-L'(a - d) S + L(a - d) sum_b L'(b - d)) / S^2, S = sum_b L(b - d)."""
    lv, dv = lanczos3(TAPS - d), lanczos3_derivative(TAPS - d)
    s = lv.sum()
    return (-dv * s + lv * dv.sum()) / (s * s)


def lanczos_conv(img, wx, wy):
    """Periodic separable convolution with weights wx (along x) and wy
    (along y), taps a = -3..3: out[y, x] = sum wy_b wx_a img[y - b, x - a]."""
    img = np.asarray(img, dtype=np.float64)
    tmp = np.zeros_like(img)
    for a, w in zip(TAPS, wx):
        tmp += w * np.roll(img, a, axis=1)
    out = np.zeros_like(img)
    for b, w in zip(TAPS, wy):
        out += w * np.roll(tmp, b, axis=0)
    return out


def jacobian_lanczos(gal, psf_hat, psf_mog, tables, n=None):
    """(6, n, n): d pixel / d (flux, x, y, log r_e, e1, e2) of the Lanczos
    model (``render_lanczos``)."""
    from .adjoint import jacobian
    nx, dx = split_offset(gal["x"])
    ny, dy = split_offset(gal["y"])
    g = dict(gal)
    g["x"], g["y"] = nx, ny
    jac = jacobian(g, psf_hat, psf_mog, tables, n)
    img = render(g, None, psf_mog, tables, n=n, psf_hat=psf_hat)
    wx, wy = lanczos_weights(dx), lanczos_weights(dy)
    out = np.stack([lanczos_conv(j, wx, wy) for j in jac])
    out[1] = lanczos_conv(img, lanczos_weights_derivative(dx), wy)
    out[2] = lanczos_conv(img, wx, lanczos_weights_derivative(dy))
    return out


def vjp_lanczos(gal, psf_hat, psf_mog, tables, grad_pix, n=None):
    """sum_p grad_pix[p] d pixel[p] / d theta of the Lanczos model."""
    return np.tensordot(jacobian_lanczos(gal, psf_hat, psf_mog, tables, n), grad_pix, axes=([1, 2], [0, 1]))


def sersic_derivative_lanczos(gal, psf_hat, psf_mog, tables, n=None):
    """(n, n) d pixel / d sersic_n of the Lanczos model: the shift of the
    integer-offset derivative."""
    from .adjoint import sersic_derivative
    nx, dx = split_offset(gal["x"])
    ny, dy = split_offset(gal["y"])
    g = dict(gal)
    g["x"], g["y"] = nx, ny
    return lanczos_conv(sersic_derivative(g, psf_hat, psf_mog, tables, n), lanczos_weights(dx), lanczos_weights(dy))
