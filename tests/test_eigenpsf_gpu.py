"""GPU parity of rendering with a spatially varying (eigen-)PSF
(mog_create_eigen_psf, Section 2 Step 2) against the FP64 oracle: max
|d pixel| <= 2e-6 flux, |d flux| / flux <= 1e-5."""

import numpy as np
import pytest

from oracle import eigenpsf as E
from oracle import lanczos as L
from oracle import render as R
from parity import check_parity
from workloads import (Galaxies, single_galaxy_64, fixed_galaxies_64, mixed_galaxies, eigen_psf, eigen_positions,
                       PROFILE_DEV)
from workloads.psf import EigenPsfInput

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eig():
    return eigen_psf()


@pytest.fixture(scope="module")
def eig_renderer(tables, psf0, eig):
    """PSF 0: the constant 2-Gaussian PSF; PSF 1: the eigen-PSF model;
    PSF 2: a degree-0 eigen-PSF equal to PSF 0."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_15797_gb300.build import build
    build()
    from paper_2012_15797_gb300.renderer import Renderer
    const0 = EigenPsfInput(components=psf0.image[None], degree=0, norm=(0.0, 0.0, 1.0, 1.0),
                           mog_shape=psf0.mog[:, 1:], mog_amp=psf0.mog[None, :, 0])
    r = Renderer(tables, [psf0, eig, const0])
    yield r
    r.close()


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


def gpu_render(renderer, gals, pos, shift="phase"):
    import torch
    from paper_2012_15797_gb300.renderer import patches, to_device
    b = to_device(gals, positions=pos)
    out = torch.full((b.total,), float("nan"), dtype=torch.float32, device="cuda")
    renderer.render(b, out, shift=shift)
    renderer.sync_status()
    return [p.double().cpu().numpy() for p in patches(out, b)]


def oracle_render(gals, pos, eig, psf0, tables, shift="phase"):
    out = []
    for i in range(len(gals)):
        g = gals.row(i)
        if g["psf"] == 1:
            img, mog = E.psf_at(eig, float(pos[0][i]), float(pos[1][i]))
        else:
            img, mog = psf0.image, psf0.mog
        out.append(R.render(g, img, mog, tables) if shift == "phase" else L.render_lanczos(g, img, mog, tables))
    return out


@pytest.mark.parametrize("size", [32, 64, 128, 256])
def test_eigen_edge_cases_each_size(eig_renderer, eig, psf0, tables, size):
    rows = [_row(size=size, psf=1, **e) for e in (
        dict(), dict(x=0.5, y=-0.5), dict(log_re=np.log(1e-4)),
        dict(log_re=np.log(20.0), profile=PROFILE_DEV, sersic_n=4.0, x=0.31, y=-0.27),
        dict(log_re=np.log(10.0), e1=0.5, e2=-0.3, x=-0.45, y=0.2))]
    gals = _gals(rows)
    # positions at the corners, the centre and the edges of the image
    pos = (np.array([0.0, 4096.0, 2048.0, 4096.0, 100.0], np.float32),
           np.array([0.0, 4096.0, 2048.0, 0.0, 3900.0], np.float32))
    check_parity(gpu_render(eig_renderer, gals, pos), oracle_render(gals, pos, eig, psf0, tables), gals)


def test_eigen_mixed_batch(eig_renderer, eig, psf0, tables):
    """Mixed sizes, eigen-PSF and constant-PSF galaxies interleaved."""
    gals = mixed_galaxies(120, seed=51, n_psf=2)   # psf ids 0 and 1
    pos = eigen_positions(len(gals), seed=52)
    check_parity(gpu_render(eig_renderer, gals, pos), oracle_render(gals, pos, eig, psf0, tables), gals)


def test_eigen_with_lanczos_shift(eig_renderer, eig, psf0, tables):
    gals = mixed_galaxies(60, seed=53, n_psf=2)
    pos = eigen_positions(len(gals), seed=54)
    check_parity(gpu_render(eig_renderer, gals, pos, "lanczos"),
                 oracle_render(gals, pos, eig, psf0, tables, "lanczos"), gals)


def test_degree_zero_equals_the_constant_psf(eig_renderer):
    rows = [_row(size=s, psf=p, **e) for p in (0, 2) for s in (32, 64, 128, 256)
            for e in (dict(), dict(log_re=np.log(18.0), profile=PROFILE_DEV, sersic_n=4.0))]
    gals = _gals(rows)
    pos = (np.full(len(gals), 77.0, np.float32), np.full(len(gals), 5.0, np.float32))
    got = gpu_render(eig_renderer, gals, pos)
    half = len(gals) // 2
    for i in range(half):
        assert np.array_equal(got[i], got[half + i]), i


def test_missing_positions_reported(eig_renderer):
    import torch
    from paper_2012_15797_gb300.capi import MogError, MOG_ERR_DEVICE
    from paper_2012_15797_gb300.renderer import to_device
    gals = _gals([_row(psf=0), _row(psf=1)])
    b = to_device(gals)   # no positions
    out = torch.full((b.total,), -3.0, dtype=torch.float32, device="cuda")
    eig_renderer.render(b, out)
    with pytest.raises(MogError) as ei:
        eig_renderer.sync_status()
    assert ei.value.status == MOG_ERR_DEVICE
    o = out.cpu().numpy().reshape(2, -1)
    assert np.all(np.isfinite(o[0])) and np.all(o[1] == -3.0)
    eig_renderer.sync_status()


def test_eigen_full_batch_sampled(eig_renderer, eig, psf0, tables):
    """100k 64^2 galaxies of the fixed-size distribution on the eigen-PSF,
    24 sampled patches."""
    gals = fixed_galaxies_64()
    gals.psf[:] = 1
    pos = eigen_positions(len(gals), seed=55)
    got = gpu_render(eig_renderer, gals, pos)
    idx = np.sort(np.random.default_rng(6).choice(len(gals), 24, replace=False))
    sub = gals.subset(idx)
    ora = oracle_render(sub, (pos[0][idx], pos[1][idx]), eig, psf0, tables)
    check_parity([got[i] for i in idx], ora, gals, idx)


def test_eigen_capable_kernels_match_for_constant_psfs(eig_renderer, gpu_renderer):
    """A context with an eigen-PSF launches the kernels that handle one; on
    constant-PSF galaxies they give the same bits as the plain kernels."""
    gals = mixed_galaxies(80, seed=56, n_psf=1)
    pos = eigen_positions(len(gals), seed=57)
    a = gpu_render(eig_renderer, gals, pos)
    b = gpu_render(gpu_renderer, gals, pos)
    for i in range(len(gals)):
        assert np.array_equal(a[i], b[i]), i


@pytest.mark.parametrize("size", [32, 64, 128, 256])
def test_eigen_adjoint_each_size(eig_renderer, eig, psf0, tables, size):
    """Gradients (and the Sersic-index gradient) with the PSF formed at each
    galaxy's position, against the oracle's analytic vector-Jacobian product
    with that PSF."""
    import torch
    from oracle import adjoint as A
    from paper_2012_15797_gb300.renderer import to_device
    rows = [_row(size=size, psf=p, **e) for p in (1, 0) for e in (
        dict(e1=0.3, e2=-0.2), dict(log_re=np.log(7.0), profile=2, sersic_n=2.6, e1=-0.25, e2=0.1))]
    gals = _gals(rows)
    pos = (np.array([300.0, 3900.0, 2048.0, 10.0], np.float32), np.array([4000.0, 150.0, 2048.0, 900.0], np.float32))
    rng = np.random.default_rng(111 + size)
    grad = [rng.normal(size=(size, size)) for _ in range(len(gals))]
    b = to_device(gals, positions=pos)
    go = torch.from_numpy(np.concatenate([g.ravel() for g in grad]).astype(np.float32)).cuda()
    got = eig_renderer.render_backward(b, go, sersic=True)
    eig_renderer.sync_status()
    got = got.double().cpu().numpy()
    for i in range(len(gals)):
        g = gals.row(i)
        if g["psf"] == 1:
            img, mog = E.psf_at(eig, float(pos[0][i]), float(pos[1][i]))
        else:
            img, mog = psf0.image, psf0.mog
        ph = R.psf_spectrum(img, size)
        ora = np.append(A.vjp(g, ph, mog, tables, grad[i]), np.sum(A.sersic_derivative(g, ph, mog, tables) * grad[i]))
        flux = float(gals.flux[i])
        scale = np.array([1.0] + [flux] * 6) * np.abs(grad[i]).sum()
        assert np.all(np.abs(got[i] - ora) <= 1e-4 * np.abs(ora) + 1e-5 * scale), (i, got[i], ora)
