"""Pins of the FP64 oracle against things other than itself: closed forms,
invariants, limits and brute force (no GPU)."""

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import gammainc

from oracle import render as R
from oracle import sersic as S
from workloads import single_galaxy_64, gaussian_mixture_psf

# ----------------------------------------------------------------------------
# Helpers that restate the continuous quantities independently of the oracle.
# ----------------------------------------------------------------------------


def _direct_cov(r_e, e1, e2, cd):
    """C / v = A A^T with A = CD^-1 E and E from theta = atan2(e2, e1)/2
    (Eqs. 2-7) computed with explicit cos and sin."""
    theta = 0.5 * np.arctan2(e2, e1)
    e = np.hypot(e1, e2)
    beta = (1 - e) / (1 + e)
    c, s = np.cos(theta), np.sin(theta)
    E = r_e * np.array([[beta * c, s], [-beta * s, c]])
    A = np.linalg.inv(cd) @ E
    return A @ A.T


def _gauss(cov, mx, my, xx, yy):
    inv = np.linalg.inv(cov)
    dx, dy = xx - mx, yy - my
    q = inv[0, 0] * dx * dx + 2 * inv[0, 1] * dx * dy + inv[1, 1] * dy * dy
    return np.exp(-0.5 * q) / (2 * np.pi * np.sqrt(np.linalg.det(cov)))


def _mog_conv_mog(gal, tables, psf_mog, n):
    """Continuous PSF (x) galaxy for mixtures on both sides (Section 1): a
    mixture of all pairs with summed covariances, sampled at pixel centres."""
    a, v = R.profile_mixture(tables[gal["profile"]], gal["sersic_n"])
    Sx = _direct_cov(np.exp(gal["log_re"]), gal["e1"], gal["e2"], np.eye(2))
    yy, xx = np.mgrid[0:n, 0:n].astype(float)
    out = np.zeros((n, n))
    for ai, vi in zip(a, v):
        for w, mx, my, pxx, pxy, pyy in psf_mog:
            cov = vi * Sx + np.array([[pxx, pxy], [pxy, pyy]])
            out += gal["flux"] * ai * w * _gauss(cov, n / 2 + gal["x"] + mx, n / 2 + gal["y"] + my, xx, yy)
    return out


def _gal(**kw):
    g = single_galaxy_64().row(0)
    g.update(kw)
    return g


# ----------------------------------------------------------------------------
# Eq. onegaussian: closed form vs the DFT of a finely sampled Gaussian.
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("cov,x0,y0", [
    (np.array([[9.0, 3.5], [3.5, 16.0]]), 120.3, 131.7),
    (np.array([[12.0, -5.0], [-5.0, 10.0]]), 127.0, 125.45),
])
def test_fourier_gaussian_matches_dft(cov, x0, y0):
    n = 256
    yy, xx = np.mgrid[0:n, 0:n].astype(float)
    img = _gauss(cov, x0, y0, xx, yy)
    dft = np.fft.rfft2(img)
    nu, om = np.fft.rfftfreq(n), np.fft.fftfreq(n)
    closed = R.fourier_gaussian(cov, x0, y0, nu[None, :], om[:, None])
    assert np.max(np.abs(dft - closed)) < 1e-12


def test_fourier_gaussian_sign_conventions():
    # A wrong sign of b or of the phase fails this.
    cov = np.array([[4.0, 1.5], [1.5, 3.0]])
    nu, om = 0.1, 0.2
    g = R.fourier_gaussian(cov, 2.0, 0.0, nu, om)
    assert np.isclose(np.angle(g), np.angle(np.exp(-2j * np.pi * 0.2)))
    assert np.isclose(abs(g), np.exp(-2 * np.pi ** 2 * (4 * nu * nu + 3.0 * nu * om + 3 * om * om)))


# ----------------------------------------------------------------------------
# Appendix A covariance vs the direct matrix product.
# ----------------------------------------------------------------------------

def test_covariance_appendix_a_matches_direct_product():
    rng = np.random.default_rng(5)
    for _ in range(200):
        r_e = np.exp(rng.uniform(-2, 3))
        e = rng.uniform(0.01, 0.9)
        phi = rng.uniform(0, np.pi)
        e1, e2 = e * np.cos(2 * phi), e * np.sin(2 * phi)
        cd = rng.normal(size=(2, 2))
        got = R.ellipse_covariance(r_e, e1, e2, cd)
        want = _direct_cov(r_e, e1, e2, cd)
        np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-12 * np.abs(want).max())


def test_covariance_printed_c12_typo_is_wrong():
    """The printed C12 bracket (uv + tv) disagrees with A V A^T for a generic
    CD; the corrected (uv + tw) agrees (previous test)."""
    r_e, e1, e2 = 2.0, 0.3, 0.2
    cd = np.array([[0.7, 0.2], [-0.3, 1.1]])
    t, u, v, w = cd.ravel()
    e = np.hypot(e1, e2)
    b2 = ((1 - e) / (1 + e)) ** 2
    c2, s2, cs = 0.5 * (1 + e1 / e), 0.5 * (1 - e1 / e), e2 / (2 * e)
    printed = -b2 * (v * w * c2 + (u * v + t * v) * cs + t * u * s2) - t * u * c2 + (u * v + t * w) * cs - v * w * s2
    f = (r_e / (t * w - u * v)) ** 2
    want = _direct_cov(r_e, e1, e2, cd)[0, 1]
    assert abs(f * printed - want) > 1e-3
    assert np.isclose(R.ellipse_covariance(r_e, e1, e2, cd)[0, 1], want)


def test_covariance_invariants_cd_identity():
    rng = np.random.default_rng(6)
    for _ in range(50):
        r_e = np.exp(rng.uniform(-1, 3))
        e1, e2 = rng.uniform(-0.45, 0.45, 2)
        s = R.ellipse_covariance(r_e, e1, e2)
        e = np.hypot(e1, e2)
        beta = (1 - e) / (1 + e)
        assert np.isclose(np.linalg.det(s), r_e ** 4 * beta ** 2, rtol=1e-12)
        assert np.isclose(np.trace(s), r_e ** 2 * (1 + beta ** 2), rtol=1e-12)
    assert np.allclose(R.ellipse_covariance(2.0, 0.0, 0.0), 4.0 * np.eye(2))


# ----------------------------------------------------------------------------
# Step 7: inverse real FFT vs a brute-force Hermitian-extended DFT.
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("n", [8, 16])
def test_inverse_real_transform_matches_direct_sum(n):
    rng = np.random.default_rng(n)
    X = rng.normal(size=(n, n // 2 + 1)) + 1j * rng.normal(size=(n, n // 2 + 1))
    got = np.fft.irfft2(X, s=(n, n))
    ck = np.full(n // 2 + 1, 2.0)
    ck[0] = ck[n // 2] = 1.0
    want = np.zeros((n, n))
    for y in range(n):
        for x in range(n):
            acc = 0.0
            for l in range(n):
                for k in range(n // 2 + 1):
                    acc += ck[k] * (X[l, k] * np.exp(2j * np.pi * (k * x + l * y) / n)).real
            want[y, x] = acc / n / n
    np.testing.assert_allclose(got, want, atol=1e-12)


def test_psf_embedding_pad_crop_and_centre():
    psf = np.arange(64 * 64, dtype=float).reshape(64, 64)
    e128 = R.embed_psf(psf, 128)
    assert e128[64, 64] == psf[32, 32] and e128[32, 32] == psf[0, 0] and e128[31, 31] == 0
    e32 = R.embed_psf(psf, 32)
    assert e32[16, 16] == psf[32, 32] and e32[0, 0] == psf[16, 16] and e32[31, 31] == psf[47, 47]
    delta = np.zeros((64, 64))
    delta[32, 32] = 1.0
    assert np.allclose(R.psf_spectrum(delta, 64), 1.0)


# ----------------------------------------------------------------------------
# Invariants and limits of the whole method.
# ----------------------------------------------------------------------------

def test_flux_invariant_all_fourier(tables, psf0):
    for x, y in [(0.0, 0.0), (0.37, -0.21), (3.3, 5.9)]:
        g = _gal(x=x, y=y, log_re=np.log(1.5), flux=7.5)
        ph = R.psf_spectrum(psf0.image, 64)
        _, _, wf, *_ = R.galaxy_components(g, tables, 64)
        assert np.all(wf == 1.0)
        img = R.render(g, psf0.image, psf0.mog, tables)
        assert abs(img.sum() - 7.5 * ph[0, 0].real) < 1e-12 * 7.5


def test_point_source_integer_shift_is_a_roll(tables, psf0):
    g = _gal(log_re=np.log(1e-7), x=2.0, y=-3.0, flux=2.0)
    img = R.render(g, psf0.image, psf0.mog, tables)
    want = 2.0 * np.roll(R.embed_psf(psf0.image, 64), (-3, 2), axis=(0, 1))
    assert np.max(np.abs(img - want)) < 1e-12


def test_point_source_subpixel_shift_is_band_limited_interpolation(tables):
    """A point source convolved with a well-sampled Gaussian PSF must equal
    that Gaussian sampled at the shifted centre (the perfect low-pass of
    Section 2, Step 6), up to the PSF's own aliasing exp(-2 pi^2 s^2 / 4)."""
    sig = 2.5
    img_psf, mog = gaussian_mixture_psf([1.0], [sig], 64)
    yy, xx = np.mgrid[0:64, 0:64].astype(float)
    for x, y in [(0.3, -0.2), (-0.45, 0.5), (0.1, 0.0)]:
        g = _gal(log_re=np.log(1e-7), x=x, y=y, flux=1.0)
        img = R.render(g, img_psf.astype(np.float64), mog, tables)
        want = _gauss(sig * sig * np.eye(2), 32 + x, 32 + y, xx, yy)
        want /= _gauss(sig * sig * np.eye(2), 32, 32, xx, yy).sum()
        assert np.max(np.abs(img - want)) < 1e-9


def test_hybrid_equals_analytic_mog_convolution(tables, psf0):
    """With an exact Gaussian-mixture PSF the continuous answer is the
    mixture of all (galaxy, PSF) pairs.  All-Fourier galaxies agree to the
    pixelized PSF's Nyquist leakage; all-real galaxies agree to rounding when
    the real-space path is given the exact PSF mixture."""
    g = _gal()
    img = R.render(g, psf0.image, psf0.mog_exact, tables)
    truth = _mog_conv_mog(g, tables, psf0.mog_exact, 64)
    assert np.max(np.abs(img - truth)) < 1e-6 * truth.max()
    # r_e = 20 px: three components real, three Fourier, none in the ramp
    big = _gal(log_re=np.log(20.0), flux=3.0, x=0.2, y=0.4)
    _, _, wf, *_ = R.galaxy_components(big, tables, 64)
    img = R.render(big, psf0.image, psf0.mog_exact, tables)
    truth = _mog_conv_mog(big, tables, psf0.mog_exact, 64)
    assert (wf == 0.0).sum() == 3 and (wf == 1.0).sum() == 3
    assert np.max(np.abs(img - truth)) < 1e-6 * truth.max()


def _supersampled(gal, tables, psf_mog_iso, n, ss):
    """Brute force: the galaxy mixture point-sampled on an ss x ss sub-pixel
    grid, each sample convolved with the continuous isotropic PSF mixture
    (separably) and summed."""
    a, v = R.profile_mixture(tables[gal["profile"]], gal["sersic_n"])
    Sx = _direct_cov(np.exp(gal["log_re"]), gal["e1"], gal["e2"], np.eye(2))
    sub = (np.arange(n * ss) + 0.5) / ss - 0.5
    SY, SX = np.meshgrid(sub, sub, indexing="ij")
    x0, y0 = n / 2 + gal["x"], n / 2 + gal["y"]
    galimg = np.zeros_like(SX)
    for ai, vi in zip(a, v):
        galimg += gal["flux"] * ai * _gauss(vi * Sx, x0, y0, SX, SY)
    galimg /= ss * ss
    pix = np.arange(n, dtype=float)
    out = np.zeros((n, n))
    for w, _, _, pxx, _, _ in psf_mog_iso:
        k = np.exp(-0.5 * (pix[:, None] - sub[None, :]) ** 2 / pxx) / np.sqrt(2 * np.pi * pxx)
        out += w * k @ galimg @ k.T
    return out


def test_brute_force_supersampling_converges_to_method(tables, psf0):
    """16 x 16 supersampled brute force converges to the analytic mixture
    convolution; the method (pixelized PSF, perfect low-pass at its Nyquist
    frequency) agrees with it to the PSF's Nyquist leakage
    exp(-2 pi^2 sigma^2 / 4) = 1.5e-5 for sigma = 1.5 px, while 1x and 2x
    supersampling are far off."""
    g = _gal(log_re=np.log(2.0), e1=0.25, e2=0.1, x=0.31, y=-0.27)
    n = 32
    img = R.render(dict(g, size=n), psf0.image, psf0.mog_exact, tables, n=n)
    truth = _mog_conv_mog(g, tables, psf0.mog_exact, n)
    peak = truth.max()
    brute = {ss: _supersampled(g, tables, psf0.mog_exact, n, ss) for ss in (1, 2, 16)}
    assert np.max(np.abs(brute[16] - truth)) < 1e-7 * peak
    err = {ss: np.max(np.abs(b - img)) for ss, b in brute.items()}
    assert err[16] < 2e-5 * peak
    assert err[1] > err[2] > 100 * err[16]


def test_wraparound_hybrid_vs_large_fourier(tables, psf0):
    """Fig. wrap: a 32 x 32 hybrid render matches the centre of a 128 x 128
    all-Fourier render; the 32 x 32 all-Fourier render does not."""
    g = _gal(log_re=np.log(5.0), e1=0.1, e2=0.05, x=0.2, y=-0.1)
    _, _, wf32, *_ = R.galaxy_components(g, tables, 32)
    _, _, wf128, *_ = R.galaxy_components(g, tables, 128)
    assert np.all(wf128 == 1.0) and np.any(wf32 < 1.0)
    big = R.render(g, psf0.image, psf0.mog_exact, tables, n=128)[48:80, 48:80]
    hyb = R.render(g, psf0.image, psf0.mog_exact, tables, n=32)
    amps, covs, *_ = R.galaxy_components(g, tables, 32)
    m = R.fourier_mixture(amps, covs, 16 + g["x"], 16 + g["y"], 32)
    four = np.fft.irfft2(R.psf_spectrum(psf0.image, 32) * m, s=(32, 32))
    e_h = np.max(np.abs(hyb - big))
    e_f = np.max(np.abs(four - big))
    assert e_f > 100 * e_h
    assert e_h < 2e-3 * big.max()


def test_naive_rendering_aliases_more_than_method(tables, psf0):
    """Fig. aliasing: an exponential galaxy with r_e = 4 px rendered naively
    (profile point-sampled at pixel centres, then convolved) or at 2x
    resolution differs from the converged brute force far more than the
    method does."""
    g = _gal(log_re=np.log(4.0), e1=0.0, e2=0.0, x=0.0, y=0.0)
    n = 64
    ref = _supersampled(g, tables, psf0.mog_exact, n, 16)
    method = R.render(dict(g, size=n), psf0.image, psf0.mog_exact, tables, n=n)
    naive = _supersampled(g, tables, psf0.mog_exact, n, 1)
    double = _supersampled(g, tables, psf0.mog_exact, n, 2)
    e_m, e_n, e_d = (np.max(np.abs(x - ref)) for x in (method, naive, double))
    assert e_n > e_d > 100 * e_m


def test_symmetries(tables):
    img_psf, mog = gaussian_mixture_psf([0.7, 0.3], [1.4, 2.8], 64)
    g = _gal(x=0.0, y=0.0, e1=0.3, e2=0.0, log_re=np.log(6.0), profile=1, sersic_n=4.0)
    img = R.render(g, img_psf, mog, tables)
    inner = img[1:, 1:]
    assert np.max(np.abs(inner - inner[::-1, ::-1])) < 1e-12 * img.max()
    # (e2, y) -> (-e2, -y) mirrors the image in y about the patch centre, up
    # to the Nyquist row omega = -1/2, which the rfft half-spectrum evaluates
    # on one side only (the PSF's power there is ~1e-4 of its total)
    g1 = _gal(x=0.2, y=0.3, e1=0.1, e2=0.25, log_re=np.log(5.0))
    g2 = dict(g1, y=-0.3, e2=-0.25)
    a = R.render(g1, img_psf, mog, tables)[1:, :]
    b = R.render(g2, img_psf, mog, tables)[1:, :][::-1, :]
    assert np.max(np.abs(a - b)) < 1e-6 * a.max()


# ----------------------------------------------------------------------------
# Step 4 ramp.
# ----------------------------------------------------------------------------

def test_ramp_values_and_c1_continuity():
    assert R.ramp(3.0) == 0.0 and R.ramp(4.0) == 1.0 and R.ramp(3.5) == 0.5
    assert R.ramp(2.0) == 0.0 and R.ramp(9.0) == 1.0
    h = 1e-7
    for b in (3.0, 4.0):
        left = (R.ramp(b) - R.ramp(b - h)) / h
        right = (R.ramp(b + h) - R.ramp(b)) / h
        assert abs(left) < 1e-6 and abs(right) < 1e-6
    for x in (3.2, 3.5, 3.9):
        fd = (R.ramp(x + h) - R.ramp(x - h)) / (2 * h)
        assert np.isclose(fd, R.ramp_slope(x), rtol=1e-6)


def test_n_sigma_definition():
    cov = np.array([[9.0, 2.0], [2.0, 16.0]])
    assert np.isclose(R.n_sigma(cov, 64), 32.0 / 5.0)


# ----------------------------------------------------------------------------
# Sersic profiles and the committed mixture tables.
# ----------------------------------------------------------------------------

def test_sersic_k_half_light():
    for n in (0.5, 1.0, 2.5, 4.0, 6.0):
        k = S.sersic_k(n)
        inner = quad(lambda r: 2 * np.pi * r * np.exp(-k * r ** (1 / n)), 0, 1, limit=200)[0]
        total = quad(lambda r: 2 * np.pi * r * np.exp(-k * r ** (1 / n)), 0, np.inf, limit=400)[0]
        assert np.isclose(inner / total, 0.5, rtol=1e-7)
        assert np.isclose(gammainc(2 * n, k), 0.5)
    assert np.isclose(S.sersic_k(0.5), np.log(2.0))
    assert np.isclose(S.sersic_k(1.0), 1.67835, atol=1e-5)
    assert np.isclose(S.sersic_k(4.0), 7.66925, atol=1e-5)


def test_sersic_profile_unit_flux():
    for n in (0.5, 1.0, 4.0):
        tot = quad(lambda r: 2 * np.pi * r * S.sersic_profile(r, n), 0, np.inf, limit=400)[0]
        assert np.isclose(tot, 1.0, rtol=1e-7)


def test_tables_normalised_and_sorted(tables):
    for t in tables.values():
        for j in range(len(t.nodes)):
            a, v = t.amp[j], t.var[j]
            assert np.isclose(a.sum(), 1.0, atol=1e-12)
            assert np.all(a >= 0) and np.all(v > 0)
            act = v[: t.k[j]]
            assert np.all(np.diff(act) < 0)
    assert tables[0].k[0] == 6 and tables[1].k[0] == 10
    ks = tables[2].k
    assert ks.min() == 8 and ks.max() == 12 and len(tables[2].nodes) == 23


def test_sersic_table_half_node_is_one_gaussian(tables):
    a, v = R.profile_mixture(tables[2], 0.5)
    r = np.linspace(0.0, 4.0, 200)
    want = np.exp(-0.5 * r * r * 2 * np.log(2)) * 2 * np.log(2) / (2 * np.pi)
    assert np.max(np.abs(S.mog_profile(r, a, v) - want)) < 1e-6 * want.max()


def test_table_interpolation_hits_nodes_and_is_continuous(tables):
    t = tables[2]
    for j in (0, 5, 13, 22):
        a, v = R.profile_mixture(t, t.nodes[j])
        keep = t.amp[j] > 0
        np.testing.assert_allclose(a, t.amp[j][keep], rtol=1e-12)
        np.testing.assert_allclose(v, t.var[j][keep], rtol=1e-12)
    r = np.geomspace(1e-3, 6, 100)
    for n0 in (1.0, 2.0, 3.0, 4.5):
        lo = S.mog_profile(r, *R.profile_mixture(t, n0 - 1e-9))
        hi = S.mog_profile(r, *R.profile_mixture(t, n0 + 1e-9))
        assert np.max(np.abs(lo - hi) / hi) < 1e-6


def test_exp_table_fit_quality(tables):
    a, v = R.profile_mixture(tables[0], 1.0)
    l2, half = S.fit_error(1.0, a, v)
    assert l2 < 5e-3 and abs(half - 0.5) < 2e-3
