"""Seeded galaxy populations shaped like survey forward-modelling workloads.

The paper's own workload is the DESI Legacy Surveys forward modelling
(Section 3); those images are not available, so these generators stand in
for it with fixed distributions and seeds.  Parameters per galaxy:

* ``flux``   total flux of the profile (the mixture amplitudes sum to 1),
* ``x, y``   offset of the galaxy centre from the patch centre (N/2, N/2), px,
* ``log_re`` natural log of the effective radius in pixels,
* ``e1, e2`` ellipticity components (Section 2, Step 3),
* ``sersic_n`` Sersic index used to interpolate the Sersic table,
* ``profile`` profile-table id (exp / deV / Sersic),
* ``psf``    PSF id, ``size`` output patch side N.
"""

from dataclasses import dataclass, field

import numpy as np

PROFILE_EXP = 0
PROFILE_DEV = 1
PROFILE_SERSIC = 2
SIZE_BUCKETS = (32, 64, 128, 256)


@dataclass
class Galaxies:
    flux: np.ndarray
    x: np.ndarray
    y: np.ndarray
    log_re: np.ndarray
    e1: np.ndarray
    e2: np.ndarray
    sersic_n: np.ndarray
    profile: np.ndarray
    psf: np.ndarray
    size: np.ndarray
    meta: dict = field(default_factory=dict)

    FLOAT_FIELDS = ("flux", "x", "y", "log_re", "e1", "e2", "sersic_n")
    INT_FIELDS = ("profile", "psf", "size")

    def __len__(self):
        return int(self.flux.shape[0])

    def subset(self, idx):
        idx = np.asarray(idx)
        kw = {f: getattr(self, f)[idx] for f in self.FLOAT_FIELDS + self.INT_FIELDS}
        return Galaxies(meta=dict(self.meta), **kw)

    def row(self, i):
        return {f: getattr(self, f)[i].item() for f in self.FLOAT_FIELDS + self.INT_FIELDS}

    def params6(self):
        """(G, 6) float64 array of the differentiable parameters
        (flux, x, y, log_re, e1, e2)."""
        return np.stack([self.flux, self.x, self.y, self.log_re, self.e1, self.e2], axis=1).astype(np.float64)

    def with_params6(self, p):
        p = np.asarray(p)
        out = self.subset(np.arange(len(self)))
        out.flux, out.x, out.y, out.log_re, out.e1, out.e2 = (p[:, j].astype(self.flux.dtype) for j in range(6))
        return out


def _cast(**kw):
    f = {k: np.ascontiguousarray(kw[k], dtype=np.float32) for k in Galaxies.FLOAT_FIELDS}
    i = {k: np.ascontiguousarray(kw[k], dtype=np.int32) for k in Galaxies.INT_FIELDS}
    return Galaxies(**f, **i)


def bucket_size(r_e, buckets=SIZE_BUCKETS, factor=8.0):
    """Smallest patch side in ``buckets`` that is >= factor * r_e (the largest
    bucket when none is)."""
    r_e = np.asarray(r_e, dtype=np.float64)
    b = np.asarray(buckets)
    need = factor * r_e
    idx = np.searchsorted(b, need, side="left")
    return b[np.minimum(idx, len(b) - 1)].astype(np.int32)


def _shapes(rng, g, emax=0.6):
    emag = rng.uniform(0.0, emax, g)
    phi = rng.uniform(0.0, np.pi, g)
    return emag * np.cos(2 * phi), emag * np.sin(2 * phi)


def single_galaxy_64():
    """One exponential galaxy: r_e = 3 px, e = (0.2, -0.1), flux 1, offset
    (0.3, -0.2), 64x64 patch, PSF 0."""
    return _cast(flux=[1.0], x=[0.3], y=[-0.2], log_re=[np.log(3.0)], e1=[0.2], e2=[-0.1],
                 sersic_n=[1.0], profile=[PROFILE_EXP], psf=[0], size=[64])


def fixed_galaxies_64(g=100_000, seed=1, size=64):
    """Fixed-size batch: 50/50 exp/deV, r_e log-uniform 0.3-20 px, |e| uniform
    <= 0.6 at a uniform angle, flux log-uniform 1-1e4, offsets uniform in
    [-0.5, 0.5)^2, one shared PSF, N x N patches."""
    rng = np.random.default_rng(seed)
    prof = np.where(rng.uniform(size=g) < 0.5, PROFILE_EXP, PROFILE_DEV)
    log_re = rng.uniform(np.log(0.3), np.log(20.0), g)
    e1, e2 = _shapes(rng, g)
    flux = np.exp(rng.uniform(0.0, np.log(1e4), g))
    x = rng.uniform(-0.5, 0.5, g)
    y = rng.uniform(-0.5, 0.5, g)
    n = np.where(prof == PROFILE_EXP, 1.0, 4.0)
    return _cast(flux=flux, x=x, y=y, log_re=log_re, e1=e1, e2=e2, sersic_n=n, profile=prof,
                 psf=np.zeros(g), size=np.full(g, size))


def mixed_galaxies(g=200_000, seed=2, n_psf=64):
    """Uneven sizes: Sersic n uniform 0.5-6, r_e log-uniform 0.3-20 px, patch
    side the smallest of {32, 64, 128, 256} >= 8 r_e, PSF id uniform over
    ``n_psf`` PSFs; other parameters as in ``fixed_galaxies_64``."""
    rng = np.random.default_rng(seed)
    n = rng.uniform(0.5, 6.0, g)
    log_re = rng.uniform(np.log(0.3), np.log(20.0), g)
    e1, e2 = _shapes(rng, g)
    flux = np.exp(rng.uniform(0.0, np.log(1e4), g))
    x = rng.uniform(-0.5, 0.5, g)
    y = rng.uniform(-0.5, 0.5, g)
    psf = rng.integers(0, n_psf, g)
    size = bucket_size(np.exp(log_re))
    return _cast(flux=flux, x=x, y=y, log_re=log_re, e1=e1, e2=e2, sersic_n=n,
                 profile=np.full(g, PROFILE_SERSIC), psf=psf, size=size)


def fit_problem(g=50_000, seed=3):
    """Differentiation workload.  Returns ``(model, truth, noise_unit)``:
    ``model`` are the parameters the gradient is taken at (drawn as in
    ``fixed_galaxies_64``), ``truth`` are perturbed parameters the synthetic
    data image is rendered from (flux x(1 + 0.05 z), x, y += 0.1 z px,
    log r_e += 0.05 z, e1, e2 += 0.02 z with |e| clipped to 0.6), and
    ``noise_unit`` is a standard-normal field (G, N, N) that the caller scales
    by sigma = 0.01 * peak of each rendered truth patch."""
    model = fixed_galaxies_64(g, seed)
    rng = np.random.default_rng(seed + 1000)
    z = rng.standard_normal((g, 6))
    t = model.params6()
    t[:, 0] *= 1.0 + 0.05 * z[:, 0]
    t[:, 1] += 0.1 * z[:, 1]
    t[:, 2] += 0.1 * z[:, 2]
    t[:, 3] += 0.05 * z[:, 3]
    t[:, 4] += 0.02 * z[:, 4]
    t[:, 5] += 0.02 * z[:, 5]
    emag = np.hypot(t[:, 4], t[:, 5])
    scale = np.where(emag > 0.6, 0.6 / np.maximum(emag, 1e-30), 1.0)
    t[:, 4] *= scale
    t[:, 5] *= scale
    truth = model.with_params6(t)
    n = int(model.size[0])
    noise = rng.standard_normal((g, n, n)).astype(np.float32)
    return model, truth, noise


def serving_workload(n_fits=1000, per_fit=512, seed=4, rate_per_ms=20_000.0, duration_ms=1000.0,
                     max_size=512, n_psf=64, max_side=256, request_seed=None):
    """Serving workload: ``n_fits`` concurrent fits of ``per_fit`` galaxies
    each (drawn as in ``mixed_galaxies``, patch sides <= max_side), and
    requests of 1..``max_size`` galaxies (uniform) arriving as a Poisson
    process of ``rate_per_ms`` galaxies per millisecond for ``duration_ms``.
    A request names a fit, a contiguous range of its galaxies and their
    current parameters: the fit's values perturbed as in
    ``fit_problem``.  Returns ``(fits, arrival_ms, requests)`` with
    requests a list of (fit, first, params (count, 6) float32).
    ``request_seed`` (default ``seed``) seeds the request stream alone, so
    that streams of other rates share the same fits."""
    rng = np.random.default_rng(seed if request_seed is None else request_seed)
    pool = mixed_galaxies(int(n_fits * per_fit * 1.6) + 64, seed + 1, n_psf=n_psf)
    keep = np.nonzero(pool.size <= max_side)[0][:n_fits * per_fit]
    pool = pool.subset(keep)
    fits = [pool.subset(np.arange(f * per_fit, (f + 1) * per_fit)) for f in range(n_fits)]
    mean = 0.5 * (1 + max_size)
    n_req = int(np.ceil(rate_per_ms / mean * duration_ms))
    arrival = np.cumsum(rng.exponential(mean / rate_per_ms, n_req))
    sizes = rng.integers(1, max_size + 1, n_req)
    fit_id = rng.integers(0, n_fits, n_req)
    params6 = [f.params6() for f in fits]
    requests = []
    for r in range(n_req):
        c = int(min(sizes[r], per_fit))
        first = int(rng.integers(0, per_fit - c + 1))
        p = params6[fit_id[r]][first:first + c].copy()
        z = rng.standard_normal((c, 6))
        p[:, 0] *= 1.0 + 0.05 * z[:, 0]
        p[:, 1:3] += 0.1 * z[:, 1:3]
        p[:, 3] += 0.05 * z[:, 3]
        p[:, 4:6] += 0.02 * z[:, 4:6]
        emag = np.hypot(p[:, 4], p[:, 5])
        scale = np.where(emag > 0.6, 0.6 / np.maximum(emag, 1e-30), 1.0)
        p[:, 4] *= scale
        p[:, 5] *= scale
        requests.append((int(fit_id[r]), first, p.astype(np.float32)))
    return fits, arrival, requests


def composite_galaxies(g=100_000, seed=7, sizes=SIZE_BUCKETS):
    """Bulge + disk composites (Section 1: a linear combination of n = 1 and
    n = 4 profiles with one centre).  Returns ``(disk, bulge)`` batches that
    share offsets, PSF and patch side: disk exponential with r_e log-uniform
    0.5-15 px and |e| <= 0.6; bulge de Vaucouleurs with r_e = U(0.2, 0.6) x
    the disk's and |e| <= 0.3; bulge fraction U(0, 1) of a total flux
    log-uniform 1-1e4; offsets U[-0.5, 0.5)^2; PSF 0; side the smallest of
    ``sizes`` >= 8 r_e(disk)."""
    rng = np.random.default_rng(seed)
    re_d = np.exp(rng.uniform(np.log(0.5), np.log(15.0), g))
    re_b = re_d * rng.uniform(0.2, 0.6, g)
    frac = rng.uniform(0.0, 1.0, g)
    flux = np.exp(rng.uniform(0.0, np.log(1e4), g))
    e1d, e2d = _shapes(rng, g, 0.6)
    e1b, e2b = _shapes(rng, g, 0.3)
    x = rng.uniform(-0.5, 0.5, g)
    y = rng.uniform(-0.5, 0.5, g)
    size = bucket_size(re_d, sizes)
    common = dict(x=x, y=y, psf=np.zeros(g), size=size)
    disk = _cast(flux=(1.0 - frac) * flux, log_re=np.log(re_d), e1=e1d, e2=e2d, sersic_n=np.ones(g),
                 profile=np.full(g, PROFILE_EXP), **common)
    bulge = _cast(flux=frac * flux, log_re=np.log(re_b), e1=e1b, e2=e2b, sersic_n=np.full(g, 4.0),
                  profile=np.full(g, PROFILE_DEV), **common)
    return disk, bulge
