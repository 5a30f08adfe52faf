"""Sersic radial profiles and their Gaussian-mixture least-squares fits.

Part of the FP64 oracle (test infrastructure; see ``oracle/__init__.py``).

The surface brightness of the model galaxies is I(r) proportional to
exp(-k(n) r^(1/n)) (Section 1, Eq. 1), with r in units of the effective radius
and k(n) chosen so that half the light falls within r <= 1.  For a 2-D profile
the light inside radius R is proportional to the lower incomplete gamma
function gamma(2n, k R^(1/n)), so k(n) is the root of P(2n, k) = 1/2 with P the
regularised lower incomplete gamma function.

A mixture of Gaussians (Section 1, footnote) sum_i a_i N(0, v_i I) with
sum_i a_i = 1 approximates the unit-flux profile.  The fit used here is the
reading recorded in the design notes: weighted least squares of the mixture
against the unit-flux profile over 0 < r <= 8, with weight r dr (the 2-D area
element), amplitudes and variances free (fitted in log space), then the
amplitudes renormalised to sum to one.
"""

import numpy as np
from scipy.optimize import least_squares
from scipy.special import gammaincinv, gammaln


def sersic_k(n):
    """k(n) with P(2n, k) = 1/2 (half the light within r_e)."""
    return float(gammaincinv(2.0 * n, 0.5))


def sersic_profile(r, n):
    """Unit-flux 2-D Sersic surface brightness at radius r (r_e units):
    exp(-k r^(1/n)) * k^(2n) / (2 pi n Gamma(2n))."""
    k = sersic_k(n)
    r = np.asarray(r, dtype=np.float64)
    lognorm = 2.0 * n * np.log(k) - np.log(2.0 * np.pi * n) - gammaln(2.0 * n)
    return np.exp(lognorm - k * r ** (1.0 / n))


def mog_profile(r, a, v):
    """sum_i a_i exp(-r^2 / (2 v_i)) / (2 pi v_i): the 2-D isotropic mixture."""
    r = np.asarray(r, dtype=np.float64)[..., None]
    return np.sum(a * np.exp(-0.5 * r * r / v) / (2.0 * np.pi * v), axis=-1)


def fit_grid(rmax=8.0, npts=800, rmin=1e-4):
    lr = np.linspace(np.log(rmin), np.log(rmax), npts)
    r = np.exp(lr)
    dlr = lr[1] - lr[0]
    w = 2.0 * np.pi * r * r * dlr       # 2 pi r dr with dr = r dlnr
    return r, w


def fit_mog(n, k, init=None, rmax=8.0):
    """Least-squares fit of a k-component mixture to the unit-flux Sersic
    profile of index n.  ``init`` = (a, v) starts the fit (used to continue a
    fit from a neighbouring n).  Returns (a, v) sorted by decreasing variance,
    with sum(a) = 1."""
    r, w = fit_grid(rmax)
    target = sersic_profile(r, n)
    sw = np.sqrt(w)
    if init is None:
        v0 = np.geomspace(1e-4 * n ** 1.5, 2.0 / n ** 0.3, k)
        a0 = np.full(k, 1.0 / k)
    else:
        a0, v0 = init
    lo = np.concatenate([np.full(k, -40.0), np.full(k, np.log(1e-10))])
    hi = np.concatenate([np.full(k, 1.0), np.full(k, np.log(100.0))])
    p0 = np.concatenate([np.log(np.maximum(a0, 1e-12)), np.log(v0)])
    p0 = np.clip(p0, lo + 1e-9, hi - 1e-9)

    def resid(p):
        a, v = np.exp(p[:k]), np.exp(p[k:])
        return sw * (mog_profile(r, a, v) - target)

    res = least_squares(resid, p0, bounds=(lo, hi), method="trf",
                        xtol=1e-14, ftol=1e-14, gtol=1e-14, max_nfev=5000)
    a, v = np.exp(res.x[:k]), np.exp(res.x[k:])
    order = np.argsort(-v)
    a, v = a[order], v[order]
    return a / a.sum(), v


def fit_error(n, a, v, rmax=8.0):
    """Relative L2 (area-weighted) error of the fit and the enclosed-flux
    error at r_e (should be 1/2 for the profile)."""
    r, w = fit_grid(rmax)
    t = sersic_profile(r, n)
    m = mog_profile(r, a, v)
    l2 = np.sqrt(np.sum(w * (m - t) ** 2) / np.sum(w * t * t))
    half = np.sum(a * (1.0 - np.exp(-0.5 / v)))   # mixture light inside r = 1
    return l2, half
