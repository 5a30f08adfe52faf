"""FP64 oracle: the forward model, Section 2 Steps 1-8 in the paper's order.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``): only tests, the smoke check
and the benchmark's CPU leg use it.

Conventions (the readings recorded in the design notes):
* Patch N x N, pixel (i, j) = (column x, row y) with its centre at integer
  coordinates; images are indexed [y, x].
* The galaxy centre is (x0, y0) = (N/2 + x, N/2 + y), (x, y) the offset.
* Frequencies: nu = k/N, k = 0..N/2 (rfft half, along x); omega = l/N in FFT
  order, l = 0..N/2-1, -N/2..-1 (along y).  Spectra are indexed [l, k].
* The PSF centre pixel (h//2, w//2) is embedded at the patch centre, larger
  PSFs are cropped (no renormalisation), then moved to index 0 (Step 1).
* The inverse transform is the real inverse DFT of the rfft half-spectrum
  (Hermitian extension along x; the self-conjugate bins contribute their real
  part only), which is what ``numpy.fft.irfft2`` computes.
* Aliasing split (Step 4): n_sigma_i = (N/2) / sqrt(trace C_i); components
  with n_sigma >= 4 are Fourier only, <= 3 real only, and in between both,
  weighted w_F = 3t^2 - 2t^3 (t = n_sigma - 3) and w_R = 1 - w_F, which is
  C^1 (the paper asks for continuous first derivatives).
* Real-space components are convolved analytically with the PSF's Gaussian
  mixture and point-sampled at pixel centres.
"""

import numpy as np

RAMP_LO = 3.0
RAMP_HI = 4.0


# --------------------------------------------------------------------------
# Steps 1-2: embed the pixelized PSF and take its FFT.
# --------------------------------------------------------------------------

def embed_psf(psf, n):
    """Step 1: place the PSF so that its centre pixel (h//2, w//2) lands on
    the patch centre (n//2, n//2); pad with zeros or crop."""
    psf = np.asarray(psf, dtype=np.float64)
    h, w = psf.shape
    out = np.zeros((n, n))
    cy, cx = h // 2, w // 2
    for yy in range(n):
        sy = yy - n // 2 + cy
        if not 0 <= sy < h:
            continue
        for xx in range(n):
            sx = xx - n // 2 + cx
            if 0 <= sx < w:
                out[yy, xx] = psf[sy, sx]
    return out


def frequencies(n):
    """(nu[k], omega[l]): rfft frequencies along x, full FFT order along y."""
    return np.fft.rfftfreq(n), np.fft.fftfreq(n)


def psf_spectrum(psf, n):
    """Step 2: FFT of the padded PSF with its centre moved to index 0.
    Returns the complex half-spectrum P[l, k] of shape (n, n//2 + 1)."""
    return np.fft.rfft2(np.fft.ifftshift(embed_psf(psf, n)))


# --------------------------------------------------------------------------
# Step 3: galaxy mixture -> pixel-space Gaussians (Eqs. 2-7, Appendix A).
# --------------------------------------------------------------------------

def ellipse_covariance(r_e, e1, e2, cd=None):
    """Pixel-space covariance per unit profile variance, C / v (Appendix A).

    With [[t, u], [v, w]] = CD, c = cos(theta), s = sin(theta):
      f   = (r_e / (t w - u v))^2
      C11 = beta^2 (w^2 c^2 + 2uw cs + u^2 s^2) + u^2 c^2 - 2uw cs + w^2 s^2
      C12 = -beta^2 (vw c^2 + (uv + tw) cs + tu s^2) - tu c^2 + (uv + tw) cs - vw s^2
      C22 = beta^2 (v^2 c^2 + 2tv cs + t^2 s^2) + t^2 c^2 - 2tv cs + v^2 s^2
    and c^2 = (1 + e1/e)/2, s^2 = (1 - e1/e)/2, cs = e2 / (2e).
    The printed C12 has (uv + tv) inside the beta^2 bracket; expanding
    A V A^T with A = CD^-1 E gives (uv + tw), which is used here.
    At e = 0 the shape is round and theta is arbitrary; theta = 0 is used.
    """
    if cd is None:
        cd = np.eye(2)
    t, u = float(cd[0][0]), float(cd[0][1])
    v, w = float(cd[1][0]), float(cd[1][1])
    e = np.hypot(e1, e2)
    beta = (1.0 - e) / (1.0 + e)
    if e > 0:
        c2 = 0.5 * (1.0 + e1 / e)
        s2 = 0.5 * (1.0 - e1 / e)
        cs = e2 / (2.0 * e)
    else:
        c2, s2, cs = 1.0, 0.0, 0.0
    b2 = beta * beta
    f = (r_e / (t * w - u * v)) ** 2
    c11 = b2 * (w * w * c2 + 2 * u * w * cs + u * u * s2) + u * u * c2 - 2 * u * w * cs + w * w * s2
    c12 = (-b2 * (v * w * c2 + (u * v + t * w) * cs + t * u * s2)
           - t * u * c2 + (u * v + t * w) * cs - v * w * s2)
    c22 = b2 * (v * v * c2 + 2 * t * v * cs + t * t * s2) + t * t * c2 - 2 * t * v * cs + v * v * s2
    return f * np.array([[c11, c12], [c12, c22]])


def profile_mixture(table, n):
    """Mixture (a_i, v_i) of a profile table at Sersic index n: linear
    interpolation of a_i and of log v_i between the two bracketing nodes
    (Section 3); fixed profiles have one node.  Zero-amplitude slots are
    dropped."""
    nodes = table.nodes
    if len(nodes) == 1:
        a, v = table.amp[0].copy(), table.var[0].copy()
    else:
        nn = min(max(float(n), nodes[0]), nodes[-1])
        j = min(int(np.searchsorted(nodes, nn, side="right")) - 1, len(nodes) - 2)
        tt = (nn - nodes[j]) / (nodes[j + 1] - nodes[j])
        a = (1 - tt) * table.amp[j] + tt * table.amp[j + 1]
        v = np.exp((1 - tt) * np.log(table.var[j]) + tt * np.log(table.var[j + 1]))
    keep = a > 0
    return a[keep], v[keep]


# --------------------------------------------------------------------------
# Step 4: aliasing test and ramp.
# --------------------------------------------------------------------------

def n_sigma(cov, n):
    """Number of sigmas from the centre to the edge of an n-pixel patch:
    (n/2) / sqrt(trace C)."""
    return 0.5 * n / np.sqrt(cov[0, 0] + cov[1, 1])


def ramp(ns, lo=RAMP_LO, hi=RAMP_HI):
    """Fourier weight: 1 for ns >= hi, 0 for ns <= lo, C^1 smoothstep between."""
    t = np.clip((ns - lo) / (hi - lo), 0.0, 1.0)
    return t * t * (3.0 - 2.0 * t)


def ramp_slope(ns, lo=RAMP_LO, hi=RAMP_HI):
    t = (ns - lo) / (hi - lo)
    if t <= 0.0 or t >= 1.0:
        return 0.0
    return 6.0 * t * (1.0 - t) / (hi - lo)


# --------------------------------------------------------------------------
# Steps 5-6: Fourier transform of the mixture on the (nu, omega) grid.
# --------------------------------------------------------------------------

def fourier_gaussian(cov, x0, y0, nu, om):
    """Eq. onegaussian: FT of a unit-flux Gaussian with covariance
    [[a, b], [b, d]] centred at (x0, y0):
      exp(-2 pi i (x0 nu + y0 om)) exp(-2 pi^2 (a nu^2 + 2 b nu om + d om^2)).
    ``nu`` and ``om`` broadcast."""
    a, b, d = cov[0, 0], cov[0, 1], cov[1, 1]
    phase = np.exp(-2j * np.pi * (x0 * nu + y0 * om))
    return phase * np.exp(-2.0 * np.pi ** 2 * (a * nu * nu + 2 * b * nu * om + d * om * om))


def fourier_mixture(amps, covs, x0, y0, n):
    """M[l, k] = sum_i A_i G_i(nu_k, omega_l): the mixture's transform
    evaluated on the FFT grid of an n-pixel patch (Step 6)."""
    nu, om = frequencies(n)
    NU, OM = nu[None, :], om[:, None]
    m = np.zeros((n, n // 2 + 1), dtype=np.complex128)
    for amp, cov in zip(amps, covs):
        if amp != 0.0:
            m += amp * fourier_gaussian(cov, x0, y0, NU, OM)
    return m


# --------------------------------------------------------------------------
# Step 8: real-space components.
# --------------------------------------------------------------------------

def gaussian_2d(cov, mx, my, xx, yy):
    """Unit-flux 2-D Gaussian density of covariance [[a, b], [b, d]] at
    (xx, yy), centred at (mx, my) (Section 2, the pixel-space g(x, y))."""
    a, b, d = cov[0, 0], cov[0, 1], cov[1, 1]
    det = a * d - b * b
    dx, dy = xx - mx, yy - my
    return np.exp(-(d * dx * dx - 2 * b * dx * dy + a * dy * dy) / (2 * det)) / (2 * np.pi * np.sqrt(det))


def real_space(amps, covs, x0, y0, psf_mog, n):
    """sum_i A_i sum_j pi_j N(p; (x0, y0) + m_j, C_i + P_j) at the pixel
    centres of an n x n patch."""
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64)
    out = np.zeros((n, n))
    for amp, cov in zip(amps, covs):
        if amp == 0.0:
            continue
        for w, mx, my, pxx, pxy, pyy in psf_mog:
            tot = cov + np.array([[pxx, pxy], [pxy, pyy]])
            out += amp * w * gaussian_2d(tot, x0 + mx, y0 + my, xx, yy)
    return out


# --------------------------------------------------------------------------
# The whole method for one galaxy.
# --------------------------------------------------------------------------

def galaxy_components(gal, tables, n, cd=None):
    """Steps 3-4 for one galaxy: per component amplitude A_i = flux a_i,
    pixel covariance C_i = v_i S, and the Fourier / real weights."""
    a, v = profile_mixture(tables[int(gal["profile"])], gal["sersic_n"])
    s = ellipse_covariance(np.exp(gal["log_re"]), gal["e1"], gal["e2"], cd)
    covs = [vi * s for vi in v]
    ns = np.array([n_sigma(c, n) for c in covs])
    wf = ramp(ns)
    return gal["flux"] * a, covs, wf, 1.0 - wf, s, v, ns


def render(gal, psf_image, psf_mog, tables, n=None, cd=None, psf_hat=None):
    """The PSF-convolved n x n image of one galaxy (Section 2, Steps 1-8).

    ``gal`` is a dict with flux, x, y, log_re, e1, e2, sersic_n, profile and
    size; ``psf_mog`` rows are (w, mx, my, vxx, vxy, vyy)."""
    n = int(gal["size"]) if n is None else int(n)
    if psf_hat is None:
        psf_hat = psf_spectrum(psf_image, n)                       # Steps 1-2
    amps, covs, wf, wr, *_ = galaxy_components(gal, tables, n, cd)  # Steps 3-4
    x0 = 0.5 * n + gal["x"]
    y0 = 0.5 * n + gal["y"]
    m = fourier_mixture(amps * wf, covs, x0, y0, n)                 # Steps 5-6
    pix = np.fft.irfft2(psf_hat * m, s=(n, n))                      # Step 7
    pix += real_space(amps * wr, covs, x0, y0, psf_mog, n)          # Step 8
    return pix


def render_batch(gals, psfs, tables, cd=None):
    """Renders every galaxy of a ``workloads.Galaxies`` batch; returns a list
    of images.  ``psfs`` is a list of ``workloads.PsfInput``."""
    cache = {}
    out = []
    for i in range(len(gals)):
        g = gals.row(i)
        key = (g["psf"], g["size"])
        if key not in cache:
            cache[key] = psf_spectrum(psfs[g["psf"]].image, g["size"])
        out.append(render(g, None, psfs[g["psf"]].mog, tables, cd=cd, psf_hat=cache[key]))
    return out
