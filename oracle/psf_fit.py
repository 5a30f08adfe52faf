"""FP64 oracle of fitting a Gaussian mixture to a pixelized PSF (the input of
the real-space half: Section 2, Step 4 uses a Gaussian approximation of the
PSF; Section 1 describes fitting mixtures by chi-squared minimisation).

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

Definition (the readings in the design notes): minimise
    chi^2 = sum_pixels (sum_j w_j N(p - c - m_j; V_j) - image[p])^2
over k components, p the pixel centres, c = (w//2, h//2) the PSF centre,
with w_j = exp(lw_j) > 0 and V_j = L L^T, L = [[a, 0], [b, c']],
a = exp(la), c' = exp(lc) (positive definite by construction).  Start:
s = sqrt(max(sum image r^2 / (2 sum image), 1/4)), widths s (0.6, 1.1, 2.2,
4.0), weights (0.55, 0.35, 0.08, 0.015) of the image sum, means 0.  The fit
is a local minimisation (Levenberg-Marquardt, scipy's MINPACK driver); rows
(w, mx, my, vxx, vxy, vyy) sorted by decreasing weight.
"""

import numpy as np
from scipy.optimize import least_squares

SCALES = (0.6, 1.1, 2.2, 4.0)
WEIGHTS = (0.55, 0.35, 0.08, 0.015)


def initial_parameters(image, k):
    image = np.asarray(image, dtype=np.float64)
    h, w = image.shape
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    dx, dy = xx - w // 2, yy - h // 2
    tot = image.sum()
    s = np.sqrt(max((image * (dx * dx + dy * dy)).sum() / (2.0 * tot), 0.25))
    wts = np.array(WEIGHTS[:k])
    wts = wts / wts.sum() * tot
    p = []
    for j in range(k):
        p += [np.log(wts[j]), 0.0, 0.0, np.log(s * SCALES[j]), 0.0, np.log(s * SCALES[j])]
    return np.array(p)


def mixture_rows(p):
    k = len(p) // 6
    rows = []
    for j in range(k):
        lw, mx, my, la, b, lc = p[6 * j:6 * j + 6]
        a, c = np.exp(la), np.exp(lc)
        rows.append([np.exp(lw), mx, my, a * a, a * b, b * b + c * c])
    return np.array(rows)


def mixture_image(rows, h, w):
    """The mixture sampled at the pixel centres of an h x w image."""
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    out = np.zeros((h, w))
    for wt, mx, my, vxx, vxy, vyy in rows:
        ex, ey = xx - w // 2 - mx, yy - h // 2 - my
        det = vxx * vyy - vxy * vxy
        out += wt * np.exp(-0.5 * (vyy * ex * ex - 2 * vxy * ex * ey + vxx * ey * ey) / det) / (2 * np.pi * np.sqrt(det))
    return out


def chi2(rows, image):
    image = np.asarray(image, dtype=np.float64)
    return float(((mixture_image(rows, *image.shape) - image) ** 2).sum())


def fit_mog(image, k=3):
    """(k, 6) rows of the fitted mixture, and its chi^2."""
    image = np.asarray(image, dtype=np.float64)
    h, w = image.shape

    def resid(p):
        return (mixture_image(mixture_rows(p), h, w) - image).ravel()

    res = least_squares(resid, initial_parameters(image, k), method="lm", xtol=1e-14, ftol=1e-14, gtol=1e-14,
                        max_nfev=20000)
    rows = mixture_rows(res.x)
    rows = rows[np.argsort(-rows[:, 0])]
    return rows, chi2(rows, image)
