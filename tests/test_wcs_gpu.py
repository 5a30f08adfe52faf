"""GPU parity with a per-galaxy WCS matrix CD (batch field cd, Appendix A:
pixel covariance CD^-1 S CD^-T): forward render and adjoint against the FP64
oracle with the same CD, at the tolerances of the constant-CD tests."""

import numpy as np
import pytest

from oracle import adjoint as A
from oracle import render as R
from parity import check_parity
from workloads import Galaxies, single_galaxy_64, mixed_galaxies, PROFILE_DEV

pytestmark = pytest.mark.gpu

# rotations, shears, a flip (det < 0) and sky-like scales (coordinates in
# units of ~0.3 pixel or ~1.5 pixels)
CDS = [np.array(m, dtype=np.float64) for m in (
    [[0.262, 0.0], [0.0, 0.262]],
    [[0.8, 0.25], [-0.15, 1.2]],
    [[-1.1, 0.4], [0.3, 0.9]],
    [[np.cos(0.7), -np.sin(0.7)], [np.sin(0.7), np.cos(0.7)]],
    [[1.5, 0.0], [0.6, 1.4]],
)]


def _gals(rows):
    f = {k: np.array([r[k] for r in rows]).astype(np.float32) for k in Galaxies.FLOAT_FIELDS}
    i = {k: np.array([r[k] for r in rows]).astype(np.int32) for k in Galaxies.INT_FIELDS}
    return Galaxies(**f, **i)


def _row(**kw):
    r = single_galaxy_64().row(0)
    r.update(kw)
    return r


def _cds(n, seed):
    rng = np.random.default_rng(seed)
    return np.stack([CDS[k] for k in rng.integers(0, len(CDS), n)]).astype(np.float32)


def gpu_render(renderer, gals, cd):
    import torch
    from paper_2012_15797_gb300.renderer import patches, to_device
    b = to_device(gals, cd=cd)
    out = torch.full((b.total,), float("nan"), dtype=torch.float32, device="cuda")
    renderer.render(b, out)
    renderer.sync_status()
    return [p.double().cpu().numpy() for p in patches(out, b)]


def oracle_render(gals, cd, psfs, tables):
    out = []
    for i in range(len(gals)):
        g = gals.row(i)
        p = psfs[g["psf"]]
        out.append(R.render(g, p.image, p.mog, tables, cd=cd[i].astype(np.float64)))
    return out


@pytest.mark.parametrize("size", [32, 64, 128, 256])
def test_wcs_forward_each_size(gpu_renderer, tables, size):
    rows = [_row(size=size, **e) for e in (
        dict(), dict(e1=0.5, e2=-0.3, x=0.4, y=-0.2), dict(log_re=np.log(1e-4)),
        dict(log_re=np.log(6.0), profile=PROFILE_DEV, sersic_n=4.0, x=-0.3, y=0.45),
        dict(log_re=np.log(2.5), e1=-0.2, e2=0.35, psf=2))]
    gals = _gals(rows)
    cd = np.stack(CDS).astype(np.float32)
    check_parity(gpu_render(gpu_renderer, gals, cd), oracle_render(gals, cd, gpu_renderer.psfs, tables), gals)


def test_wcs_forward_mixed_batch(gpu_renderer, tables):
    gals = mixed_galaxies(120, seed=61, n_psf=5)
    cd = _cds(len(gals), 62)
    check_parity(gpu_render(gpu_renderer, gals, cd), oracle_render(gals, cd, gpu_renderer.psfs, tables), gals)


def test_identity_matrix_gives_the_same_bits(gpu_renderer):
    gals = mixed_galaxies(60, seed=63, n_psf=5)
    eye = np.tile(np.eye(2, dtype=np.float32), (len(gals), 1, 1))
    a = gpu_render(gpu_renderer, gals, eye)
    b = gpu_render(gpu_renderer, gals, None)
    for i in range(len(gals)):
        assert np.array_equal(a[i], b[i]), i


def test_singular_matrix_reported(gpu_renderer):
    import torch
    from paper_2012_15797_gb300.capi import MogError, MOG_ERR_DEVICE
    from paper_2012_15797_gb300.renderer import to_device
    gals = _gals([_row(), _row()])
    cd = np.array([np.eye(2), [[1.0, 2.0], [0.5, 1.0]]], dtype=np.float32)
    b = to_device(gals, cd=cd)
    out = torch.full((b.total,), -3.0, dtype=torch.float32, device="cuda")
    gpu_renderer.render(b, out)
    with pytest.raises(MogError) as ei:
        gpu_renderer.sync_status()
    assert ei.value.status == MOG_ERR_DEVICE
    o = out.cpu().numpy().reshape(2, -1)
    assert np.all(np.isfinite(o[0])) and np.all(o[1] == -3.0)
    gpu_renderer.sync_status()


def test_wcs_adjoint(gpu_renderer, tables):
    """Gradients w.r.t. (flux, x, y, log r_e, e1, e2) with a WCS matrix, against
    the oracle's analytic vector-Jacobian product with the same CD."""
    import torch
    from paper_2012_15797_gb300.renderer import to_device
    rows = [_row(size=s, **e) for s in (32, 64, 128, 256) for e in (
        dict(e1=0.3, e2=-0.2), dict(log_re=np.log(7.0), profile=PROFILE_DEV, sersic_n=4.0, e1=-0.25, e2=0.1))]
    gals = _gals(rows)
    cd = _cds(len(gals), 64)
    rng = np.random.default_rng(65)
    grad_pix = [rng.normal(size=(int(n), int(n))) for n in gals.size]
    b = to_device(gals, cd=cd)
    go = torch.from_numpy(np.concatenate([g.ravel() for g in grad_pix]).astype(np.float32)).cuda()
    gp = torch.full((len(gals), 6), float("nan"), device="cuda")
    gpu_renderer.render_backward(b, go, gp)
    gpu_renderer.sync_status()
    gpu = gp.double().cpu().numpy()
    for i in range(len(gals)):
        g = gals.row(i)
        p = gpu_renderer.psfs[g["psf"]]
        ora = A.vjp(g, R.psf_spectrum(p.image, g["size"]), p.mog, tables, grad_pix[i], cd=cd[i].astype(np.float64))
        flux = float(gals.flux[i])
        scale = np.array([1.0, flux, flux, flux, flux, flux]) * np.abs(grad_pix[i]).sum()
        err = np.abs(gpu[i] - ora)
        assert np.all(err <= 1e-4 * np.abs(ora) + 1e-5 * scale), (i, gpu[i], ora)
