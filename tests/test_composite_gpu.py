"""GPU composite (bulge + disk) galaxies through mog_render_batch_ex
(MOG_RENDER_ADD) against the FP64 oracle: max |d pixel| <= 2e-6 of the
composite's total flux, |d sum| <= 1e-5 of it; and the add mode itself."""

import numpy as np
import pytest

from oracle import composite as C
from oracle import render as R
from parity import FLUX_TOL, PIX_TOL
from workloads import composite_galaxies

pytestmark = pytest.mark.gpu


def _device(gals):
    from paper_2012_15797_gb300.renderer import to_device
    return to_device(gals)


def gpu_composite(renderer, disk, bulge, shift="phase"):
    import torch
    from paper_2012_15797_gb300.renderer import patches
    bd, bb = _device(disk), _device(bulge)
    out = torch.full((bd.total,), float("nan"), dtype=torch.float32, device="cuda")
    renderer.render_composite(bd, bb, out, shift=shift)
    renderer.sync_status()
    return [p.double().cpu().numpy() for p in patches(out, bd)]


def check(gpu, disk, bulge, psfs, tables, shift="phase"):
    for i in range(len(disk)):
        d, b = disk.row(i), bulge.row(i)
        p = psfs[d["psf"]]
        ora = C.render_composite(d, b, p.image, p.mog, tables, shift=shift)
        tot = d["flux"] + b["flux"]
        assert np.all(np.isfinite(gpu[i]))
        assert np.max(np.abs(gpu[i] - ora)) <= PIX_TOL * tot, (i, d, b, np.max(np.abs(gpu[i] - ora)) / tot)
        assert abs(gpu[i].sum() - ora.sum()) <= FLUX_TOL * tot, i


@pytest.mark.parametrize("size", [32, 64, 128, 256])
def test_composite_each_size(gpu_renderer, tables, size):
    disk, bulge = composite_galaxies(12, seed=80 + size, sizes=(size,))
    disk.size[:] = size
    bulge.size[:] = size
    check(gpu_composite(gpu_renderer, disk, bulge), disk, bulge, gpu_renderer.psfs, tables)


def test_composite_mixed_sizes(gpu_renderer, tables):
    disk, bulge = composite_galaxies(150, seed=91)
    assert {32, 64, 128} <= set(np.unique(disk.size).tolist())
    check(gpu_composite(gpu_renderer, disk, bulge), disk, bulge, gpu_renderer.psfs, tables)


def test_composite_lanczos(gpu_renderer, tables):
    disk, bulge = composite_galaxies(80, seed=92)
    check(gpu_composite(gpu_renderer, disk, bulge, "lanczos"), disk, bulge, gpu_renderer.psfs, tables, "lanczos")


@pytest.mark.parametrize("shift", ["phase", "lanczos"])
def test_add_mode_adds_to_the_patch(gpu_renderer, shift):
    """out + model with the same bits as adding the plain render on the host
    (every size, 256 included, whose kernel then works in a scratch)."""
    import torch
    from paper_2012_15797_gb300.renderer import patches
    disk, _ = composite_galaxies(60, seed=93)
    b = _device(disk)
    model = gpu_renderer.render(b, shift=shift)
    base = torch.from_numpy(np.random.default_rng(94).normal(size=b.total).astype(np.float32)).cuda()
    out = base.clone()
    gpu_renderer.render(b, out, shift=shift, add=True)
    gpu_renderer.sync_status()
    assert torch.equal(out, base + model)


def test_composite_gradients_are_the_parts(gpu_renderer, tables):
    """The adjoint of a composite is the adjoint of each part with the same
    upstream gradient (the shared offset's gradient is their sum)."""
    import torch
    from oracle import adjoint as A
    disk, bulge = composite_galaxies(8, seed=95, sizes=(64,))
    disk.e1[:] = np.where(np.abs(disk.e1) < 1e-3, 0.1, disk.e1)
    bulge.e1[:] = np.where(np.abs(bulge.e1) < 1e-3, 0.1, bulge.e1)
    rng = np.random.default_rng(96)
    grad = [rng.normal(size=(64, 64)) for _ in range(len(disk))]
    go = torch.from_numpy(np.concatenate([g.ravel() for g in grad]).astype(np.float32)).cuda()
    for part in (disk, bulge):
        gp = torch.full((len(part), 6), float("nan"), device="cuda")
        gpu_renderer.render_backward(_device(part), go, gp)
        gpu_renderer.sync_status()
        got = gp.double().cpu().numpy()
        for i in range(len(part)):
            g = part.row(i)
            p = gpu_renderer.psfs[g["psf"]]
            ora = A.vjp(g, R.psf_spectrum(p.image, 64), p.mog, tables, grad[i])
            flux = max(float(part.flux[i]), 1e-3)
            scale = np.array([1.0, flux, flux, flux, flux, flux]) * np.abs(grad[i]).sum()
            assert np.all(np.abs(got[i] - ora) <= 1e-4 * np.abs(ora) + 1e-5 * scale), (i, got[i], ora)
