"""FP64 oracle: derivatives of the rendered patch w.r.t. the galaxy parameters
theta = (flux, x, y, log r_e, e1, e2).

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

The paper has no gradients; they follow from differentiating its forward
model.  Every step after the Fourier evaluation is linear, so with
X = P_hat * M the pixel Jacobian is irfft2(P_hat * dM/dtheta) plus the
derivative of the real-space sum.  From Eq. onegaussian:
  dM/dflux = M / flux,  dM/dx = -2 pi i nu M,  dM/dy = -2 pi i omega M,
  dG_i/dS_ab = -2 pi^2 v_i (dq/dS_ab) G_i with q = S11 nu^2 + 2 S12 nu om + S22 om^2,
plus the ramp weights' dependence on n_sigma_i = (N/2) / sqrt(v_i trace S).
The real-space Gaussian N(d; Sigma) has dN/dmu = N Sigma^-1 d and
dN/dSigma = N (Sigma^-1 d d^T Sigma^-1 - Sigma^-1) / 2.
S(log r_e, e1, e2) is the CD = I covariance of Appendix A:
  S11 = r^2 (h + G e1), S12 = -r^2 G e2, S22 = r^2 (h - G e1),
  h = (1 + beta^2)/2, G = (beta^2 - 1)/(2e), beta = (1 - e)/(1 + e).
S is not differentiable at e = 0 (beta depends on |e|), so e > 0 is required.
The Sersic index n moves the mixture itself (amplitudes a_i(n) and variances
v_i(n), interpolated in the profile table): ``sersic_derivative``.
With a WCS matrix CD the pixel covariance is A S A^T with A = CD^-1
(Appendix A), which is linear in S, so its derivatives are A dS A^T.
"""

import numpy as np

from . import render as R

PARAMS = ("flux", "x", "y", "log_re", "e1", "e2")


def shape_derivatives(log_re, e1, e2):
    """dS/d(log r_e), dS/de1, dS/de2 as three 2x2 matrices (CD = I)."""
    r2 = np.exp(2.0 * log_re)
    e = np.hypot(e1, e2)
    if not e > 0:
        raise ValueError("the covariance is not differentiable at e = 0")
    beta = (1 - e) / (1 + e)
    dbeta = -2.0 / (1 + e) ** 2
    h = 0.5 * (1 + beta * beta)
    g = (beta * beta - 1) / (2 * e)
    dh = beta * dbeta
    dg = beta * dbeta / e - (beta * beta - 1) / (2 * e * e)
    s = r2 * np.array([[h + g * e1, -g * e2], [-g * e2, h - g * e1]])
    de1, de2 = e1 / e, e2 / e
    d1 = r2 * np.array([[dh * de1 + dg * de1 * e1 + g, -dg * de1 * e2],
                        [-dg * de1 * e2, dh * de1 - dg * de1 * e1 - g]])
    d2 = r2 * np.array([[dh * de2 + dg * de2 * e1, -(dg * de2 * e2 + g)],
                        [-(dg * de2 * e2 + g), dh * de2 - dg * de2 * e1]])
    return [2.0 * s, d1, d2]


def jacobian(gal, psf_hat, psf_mog, tables, n=None, cd=None):
    """(6, n, n) array: d pixel / d theta for one galaxy (WCS matrix ``cd``,
    identity when None)."""
    n = int(gal["size"]) if n is None else int(n)
    amps, covs, wf, wr, s, v, ns = R.galaxy_components(gal, tables, n, cd)
    flux = gal["flux"]
    x0, y0 = 0.5 * n + gal["x"], 0.5 * n + gal["y"]
    nu, om = R.frequencies(n)
    NU, OM = nu[None, :], om[:, None]
    tr = s[0, 0] + s[1, 1]
    dq = {(0, 0): NU * NU, (0, 1): 2 * NU * OM, (1, 1): OM * OM}
    slopes = np.array([R.ramp_slope(x) for x in ns])
    dns = {(0, 0): -0.5 * ns / tr, (0, 1): np.zeros_like(ns), (1, 1): -0.5 * ns / tr}

    # Fourier part: spectra of each derivative.
    shape = (n, n // 2 + 1)
    m = np.zeros(shape, complex)
    dm_s = {ab: np.zeros(shape, complex) for ab in dq}
    for i, (amp, cov) in enumerate(zip(amps, covs)):
        gi = R.fourier_gaussian(cov, x0, y0, NU, OM)
        m += amp * wf[i] * gi
        for ab in dq:
            dm_s[ab] += amp * gi * (slopes[i] * dns[ab][i] - wf[i] * 2 * np.pi ** 2 * v[i] * dq[ab])
    dm = [m / flux, -2j * np.pi * NU * m, -2j * np.pi * OM * m]
    ds = shape_derivatives(gal["log_re"], gal["e1"], gal["e2"])
    if cd is not None:
        a = np.linalg.inv(np.asarray(cd, dtype=np.float64))
        ds = [a @ d @ a.T for d in ds]
    for d in ds:
        dm.append(d[0, 0] * dm_s[(0, 0)] + d[0, 1] * dm_s[(0, 1)] + d[1, 1] * dm_s[(1, 1)])
    jac = np.stack([np.fft.irfft2(psf_hat * d, s=(n, n)) for d in dm])

    # Real-space part.
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64)
    rj = np.zeros((6, n, n))
    for i, (amp, cov) in enumerate(zip(amps, covs)):
        for w, mx, my, pxx, pxy, pyy in psf_mog:
            sig = cov + np.array([[pxx, pxy], [pxy, pyy]])
            nij = w * R.gaussian_2d(sig, x0 + mx, y0 + my, xx, yy)
            inv = np.linalg.inv(sig)
            dx, dy = xx - x0 - mx, yy - y0 - my
            ux = inv[0, 0] * dx + inv[0, 1] * dy
            uy = inv[1, 0] * dx + inv[1, 1] * dy
            q = {(0, 0): 0.5 * (ux * ux - inv[0, 0]),
                 (0, 1): 2 * 0.5 * (ux * uy - inv[0, 1]),
                 (1, 1): 0.5 * (uy * uy - inv[1, 1])}
            rj[0] += amp / flux * wr[i] * nij
            rj[1] += amp * wr[i] * nij * ux
            rj[2] += amp * wr[i] * nij * uy
            for k, d in enumerate(ds):
                acc = 0.0
                for ab in q:
                    dsab = d[ab]
                    acc = acc + dsab * (-slopes[i] * dns[ab][i] + wr[i] * v[i] * q[ab])
                rj[3 + k] += amp * nij * acc
    return jac + rj


def vjp(gal, psf_hat, psf_mog, tables, grad_pix, n=None, cd=None):
    """sum_p grad_pix[p] * d pixel[p] / d theta: the six gradients."""
    return np.tensordot(jacobian(gal, psf_hat, psf_mog, tables, n, cd), grad_pix, axes=([1, 2], [0, 1]))


def finite_difference(gal, psf_hat, psf_mog, tables, step=1e-6, n=None, cd=None):
    """Central finite differences of the forward model: absolute step for
    x, y, log r_e, e1, e2 and relative step (step * flux) for flux."""
    out = []
    for p in PARAMS:
        h = step * gal["flux"] if p == "flux" else step
        gp, gm = dict(gal), dict(gal)
        gp[p] = gal[p] + h
        gm[p] = gal[p] - h
        ip = R.render(gp, None, psf_mog, tables, n=n, psf_hat=psf_hat, cd=cd)
        im = R.render(gm, None, psf_mog, tables, n=n, psf_hat=psf_hat, cd=cd)
        out.append((ip - im) / (2 * h))
    return np.stack(out)


def profile_mixture_dn(table, n):
    """(a, v, da/dn, dv/dn) of every slot of a profile table at Sersic index
    n: a and log v are linear in n between the bracketing nodes (Section 3),
    so da/dn = (a_{j+1} - a_j) / dn and dv/dn = v (log v_{j+1} - log v_j) / dn
    inside the node range; zero outside it and for one-node tables.  Slots
    with a = 0 and da/dn = 0 are dropped."""
    nodes = table.nodes
    if len(nodes) == 1:
        a, v = table.amp[0].copy(), table.var[0].copy()
        da, dv = np.zeros_like(a), np.zeros_like(v)
    else:
        inside = nodes[0] <= float(n) <= nodes[-1]
        nn = min(max(float(n), nodes[0]), nodes[-1])
        j = min(int(np.searchsorted(nodes, nn, side="right")) - 1, len(nodes) - 2)
        h = nodes[j + 1] - nodes[j]
        tt = (nn - nodes[j]) / h
        la, lb = np.log(table.var[j]), np.log(table.var[j + 1])
        a = (1 - tt) * table.amp[j] + tt * table.amp[j + 1]
        v = np.exp((1 - tt) * la + tt * lb)
        da = (table.amp[j + 1] - table.amp[j]) / h if inside else np.zeros_like(a)
        dv = v * (lb - la) / h if inside else np.zeros_like(v)
    keep = (a > 0) | (da != 0)
    return a[keep], v[keep], da[keep], dv[keep]


def sersic_derivative(gal, psf_hat, psf_mog, tables, n=None, cd=None):
    """(n, n) d pixel / d sersic_n: the mixture's amplitudes and variances
    move with n, through the Fourier Gaussians, the ramp weights and the
    real-space Gaussians (dN/dv = N (u^T S u - tr(Sigma^-1 S)) / 2 with
    u = Sigma^-1 d, Sigma = v S + P)."""
    n = int(gal["size"]) if n is None else int(n)
    a, v, da, dv = profile_mixture_dn(tables[int(gal["profile"])], gal["sersic_n"])
    s = R.ellipse_covariance(np.exp(gal["log_re"]), gal["e1"], gal["e2"], cd)
    flux = gal["flux"]
    x0, y0 = 0.5 * n + gal["x"], 0.5 * n + gal["y"]
    nu, om = R.frequencies(n)
    NU, OM = nu[None, :], om[:, None]
    q = s[0, 0] * NU * NU + 2 * s[0, 1] * NU * OM + s[1, 1] * OM * OM
    dm = np.zeros((n, n // 2 + 1), complex)
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64)
    real = np.zeros((n, n))
    for ai, vi, dai, dvi in zip(a, v, da, dv):
        cov = vi * s
        ns = R.n_sigma(cov, n)
        wf, dwf = R.ramp(ns), R.ramp_slope(ns)
        dns = -0.5 * ns / vi * dvi            # d n_sigma / dn
        gi = R.fourier_gaussian(cov, x0, y0, NU, OM)
        dm += flux * (dai * wf + ai * dwf * dns) * gi + flux * ai * wf * dvi * (-2 * np.pi ** 2 * q) * gi
        for w, mx, my, pxx, pxy, pyy in psf_mog:
            sig = cov + np.array([[pxx, pxy], [pxy, pyy]])
            nij = w * R.gaussian_2d(sig, x0 + mx, y0 + my, xx, yy)
            inv = np.linalg.inv(sig)
            dx, dy = xx - x0 - mx, yy - y0 - my
            ux = inv[0, 0] * dx + inv[0, 1] * dy
            uy = inv[1, 0] * dx + inv[1, 1] * dy
            usu = s[0, 0] * ux * ux + 2 * s[0, 1] * ux * uy + s[1, 1] * uy * uy
            trs = np.trace(inv @ s)
            real += flux * nij * ((dai * (1 - wf) - ai * dwf * dns) + ai * (1 - wf) * dvi * 0.5 * (usu - trs))
    return np.fft.irfft2(psf_hat * dm, s=(n, n)) + real
