"""GPU parity of the Lanczos sub-pixel-shift variant (mog_render_batch_lanczos,
Section 2 Step 8) against the FP64 oracle: max |d pixel| <= 2e-6 flux,
|d flux| / flux <= 1e-5, as for the phase-shift path."""

import numpy as np
import pytest

from oracle import lanczos as L
from oracle import render as R
from parity import check_parity
from workloads import Galaxies, single_galaxy_64, fixed_galaxies_64, mixed_galaxies, PROFILE_DEV, PROFILE_SERSIC

pytestmark = pytest.mark.gpu


def _gals(rows):
    keys = Galaxies.FLOAT_FIELDS + Galaxies.INT_FIELDS
    cols = {k: np.array([r[k] for r in rows]) for k in keys}
    f = {k: cols[k].astype(np.float32) for k in Galaxies.FLOAT_FIELDS}
    i = {k: cols[k].astype(np.int32) for k in Galaxies.INT_FIELDS}
    return Galaxies(**f, **i)


def _row(**kw):
    r = single_galaxy_64().row(0)
    r.update(kw)
    return r


def lanczos_gpu(renderer, gals, shift="lanczos"):
    import torch
    from paper_2012_15797_gb300.renderer import patches, to_device
    b = to_device(gals)
    out = torch.full((b.total,), float("nan"), dtype=torch.float32, device="cuda")
    renderer.render(b, out, shift=shift)
    renderer.sync_status()
    return [p.double().cpu().numpy() for p in patches(out, b)], out, b


def lanczos_oracle(gals, psfs, tables):
    cache, out = {}, []
    for i in range(len(gals)):
        g = gals.row(i)
        key = (g["psf"], g["size"])
        if key not in cache:
            cache[key] = R.psf_spectrum(psfs[g["psf"]].image, g["size"])
        out.append(L.render_lanczos(g, None, psfs[g["psf"]].mog, tables, psf_hat=cache[key]))
    return out


EDGE = [
    dict(),                                                   # the single 64x64 galaxy as drawn
    dict(x=0.5, y=-0.5), dict(x=-0.5, y=0.4999), dict(x=0.0, y=0.0),
    dict(x=3.7, y=-6.2),                                      # integer part beyond a pixel
    dict(log_re=np.log(1e-4)),                                # point-source limit
    dict(log_re=np.log(20.0), profile=PROFILE_DEV, sersic_n=4.0, x=0.31, y=-0.27),   # real-space terms
    dict(log_re=np.log(12.0), e1=0.5, e2=-0.3, x=-0.45, y=0.2),                     # elongated, real space
    dict(profile=PROFILE_SERSIC, sersic_n=6.0, log_re=np.log(9.0), x=0.12, y=0.44, psf=2),
    dict(flux=1e4, x=-0.21, y=0.33),
]


@pytest.mark.parametrize("size", [32, 64, 128, 256])
def test_lanczos_edge_cases_each_size(gpu_renderer, tables, size):
    gals = _gals([_row(size=size, **e) for e in EDGE])
    gpu, _, _ = lanczos_gpu(gpu_renderer, gals)
    check_parity(gpu, lanczos_oracle(gals, gpu_renderer.psfs, tables), gals)


def test_lanczos_batch_fixed_size(gpu_renderer, tables):
    """The 64x64 fixed-size distribution, 160 galaxies (many CTAs, ragged)."""
    gals = fixed_galaxies_64(160, seed=41)
    gpu, _, _ = lanczos_gpu(gpu_renderer, gals)
    check_parity(gpu, lanczos_oracle(gals, gpu_renderer.psfs, tables), gals)


def test_lanczos_batch_mixed_sizes(gpu_renderer, tables):
    gals = mixed_galaxies(150, seed=42, n_psf=5)
    assert set(np.unique(gals.size)) == {32, 64, 128, 256}
    gpu, _, _ = lanczos_gpu(gpu_renderer, gals)
    check_parity(gpu, lanczos_oracle(gals, gpu_renderer.psfs, tables), gals)


def test_integer_offsets_equal_the_phase_path(gpu_renderer):
    """With integer offsets the Lanczos weights are a unit impulse, so the two
    entry points give the same bits (real-space terms included)."""
    rows = [_row(size=s, x=float(x), y=float(y), **e)
            for s in (32, 64, 128, 256) for x, y in ((0, 0), (2, -1))
            for e in (dict(), dict(log_re=np.log(18.0), profile=PROFILE_DEV, sersic_n=4.0))]
    gals = _gals(rows)
    a, _, _ = lanczos_gpu(gpu_renderer, gals, "lanczos")
    b, _, _ = lanczos_gpu(gpu_renderer, gals, "phase")
    for i in range(len(gals)):
        assert np.array_equal(a[i], b[i]), i


def test_lanczos_full_100k_sampled(gpu_renderer, tables):
    """100k galaxies at 64^2 in one Lanczos call, 32 sampled patches."""
    gals = fixed_galaxies_64()
    gpu, _, _ = lanczos_gpu(gpu_renderer, gals)
    idx = np.sort(np.random.default_rng(5).choice(len(gals), 32, replace=False))
    ora = lanczos_oracle(gals.subset(idx), gpu_renderer.psfs, tables)
    check_parity([gpu[i] for i in idx], ora, gals, idx)
