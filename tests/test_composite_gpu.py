"""GPU composite (bulge + disk) galaxies against the FP64 oracle, max
|d pixel| <= 2e-6 of the composite's total flux and |d sum| <= 1e-5 of it,
in both forms: one pass (mog_render_composite: both profiles' mixtures on
one grid, one transform) and two (mog_render_batch_ex, MOG_RENDER_ADD); the
two forms against each other; the one-pass form's checks (profiles that
disagree, counts, eigen-PSFs); and the add mode itself."""

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


def gpu_composite(renderer, disk, bulge, shift="phase", fused=True):
    import torch
    from paper_2012_15797_gb300.renderer import patches
    bd, bb = _device(disk), _device(bulge)
    out = torch.full((bd.total,), float("nan"), dtype=torch.float32, device="cuda")
    renderer.render_composite(bd, bb, out, shift=shift, fused=fused)
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


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("size", [32, 64, 128, 256])
def test_composite_each_size(gpu_renderer, tables, size, fused):
    disk, bulge = composite_galaxies(12, seed=80 + size, sizes=(size,))
    disk.size[:] = size
    bulge.size[:] = size
    check(gpu_composite(gpu_renderer, disk, bulge, fused=fused), disk, bulge, gpu_renderer.psfs, tables)


@pytest.mark.parametrize("fused", [True, False])
def test_composite_mixed_sizes(gpu_renderer, tables, fused):
    disk, bulge = composite_galaxies(150, seed=91)
    assert {32, 64, 128} <= set(np.unique(disk.size).tolist())
    check(gpu_composite(gpu_renderer, disk, bulge, fused=fused), disk, bulge, gpu_renderer.psfs, tables)


@pytest.mark.parametrize("size", [32, 64, 128, 256])
def test_one_pass_equals_two_passes(gpu_renderer, size):
    """Many composites, Sersic profiles of every index on both parts (up to
    24 components with real-space terms), several PSFs: the one-pass form
    within float rounding of the two-pass form."""
    disk, bulge = composite_galaxies(1500 if size < 256 else 200, seed=100 + size, sizes=(size,))
    rng = np.random.default_rng(size)
    for part in (disk, bulge):
        part.size[:] = size
        part.profile[:] = 2
        part.sersic_n[:] = rng.uniform(0.5, 6.0, len(part)).astype(np.float32)
    disk.psf[:] = bulge.psf[:] = np.arange(len(disk)) % 5
    tot = (disk.flux + bulge.flux).astype(np.float64)
    for shift in ("phase", "lanczos"):
        one = np.stack(gpu_composite(gpu_renderer, disk, bulge, shift, fused=True))
        two = np.stack(gpu_composite(gpu_renderer, disk, bulge, shift, fused=False))
        d = np.abs(one - two).reshape(len(disk), -1).max(axis=1)
        assert np.all(d <= 0.25 * PIX_TOL * tot), (shift, float(np.max(d / tot)))


def test_one_pass_checks(gpu_renderer, tables):
    import torch
    from paper_2012_15797_gb300 import capi
    from paper_2012_15797_gb300.renderer import patches
    disk, bulge = composite_galaxies(40, seed=97)
    bulge.x[3] += 0.25                   # centres differ
    bulge.psf[5] = 1                     # PSFs differ
    bulge.log_re[7] = np.nan             # one profile invalid
    bd, bb = _device(disk), _device(bulge)
    out = torch.full((bd.total,), -9.0, dtype=torch.float32, device="cuda")
    gpu_renderer.render_composite(bd, bb, out)
    with pytest.raises(capi.MogError) as ei:
        gpu_renderer.sync_status()
    assert ei.value.status == capi.MOG_ERR_DEVICE
    got = [p.double().cpu().numpy() for p in patches(out, bd)]
    for i in range(len(disk)):
        if i in (3, 5, 7):
            assert np.all(got[i] == -9.0)
    keep = [i for i in range(len(disk)) if i not in (3, 5, 7)]
    check([got[i] for i in keep], disk.subset(keep), bulge.subset(keep), gpu_renderer.psfs, tables)
    short = capi.make_batch(len(disk) - 1, bb.ptrs(), 0)
    first = capi.make_batch(bd.count, bd.ptrs(), bd.size_mask())
    with pytest.raises(capi.MogError):
        capi.mog_render_composite(gpu_renderer.ctx, first, short, out.data_ptr(), 0)
    with pytest.raises(capi.MogError):                      # unknown flags
        capi.mog_render_composite(gpu_renderer.ctx, first, capi.make_batch(bb.count, bb.ptrs(), 0), out.data_ptr(),
                                  0, capi.MOG_RENDER_ADD)


def test_one_pass_rejects_eigen_psf_galaxies(tables, psf0):
    import torch
    from paper_2012_15797_gb300 import capi
    from paper_2012_15797_gb300.renderer import Renderer, patches
    from workloads import eigen_psf
    r = Renderer(tables, [psf0, eigen_psf()])
    try:
        disk, bulge = composite_galaxies(10, seed=98, sizes=(64,))
        disk.size[:] = bulge.size[:] = 64
        disk.psf[2] = bulge.psf[2] = 1
        bd, bb = _device(disk), _device(bulge)
        out = torch.full((bd.total,), -9.0, dtype=torch.float32, device="cuda")
        r.render_composite(bd, bb, out)
        with pytest.raises(capi.MogError):
            r.sync_status()
        got = [p.double().cpu().numpy() for p in patches(out, bd)]
        assert np.all(got[2] == -9.0)
        keep = [i for i in range(10) if i != 2]
        check([got[i] for i in keep], disk.subset(keep), bulge.subset(keep), [psf0], tables)
    finally:
        r.close()


@pytest.mark.parametrize("fused", [True, False])
def test_composite_lanczos(gpu_renderer, tables, fused):
    disk, bulge = composite_galaxies(80, seed=92)
    check(gpu_composite(gpu_renderer, disk, bulge, "lanczos", fused), disk, bulge, gpu_renderer.psfs, tables,
          "lanczos")


@pytest.mark.parametrize("size", [32, 64, 128, 256])
def test_composite_lanczos_each_size(gpu_renderer, tables, size):
    disk, bulge = composite_galaxies(10, seed=120 + size, sizes=(size,))
    disk.size[:] = bulge.size[:] = size
    disk.x[:] = bulge.x[:] = np.linspace(-2.6, 3.4, 10).astype(np.float32)   # integer parts and fractions
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
    grads = gpu_renderer.render_composite_backward(_device(disk), _device(bulge), go)
    gpu_renderer.sync_status()
    for part, gp in zip((disk, bulge), grads):
        got = gp.double().cpu().numpy()
        for i in range(len(part)):
            g = part.row(i)
            p = gpu_renderer.psfs[g["psf"]]
            ora = A.vjp(g, R.psf_spectrum(p.image, 64), p.mog, tables, grad[i])
            flux = max(float(part.flux[i]), 1e-3)
            scale = np.array([1.0, flux, flux, flux, flux, flux]) * np.abs(grad[i]).sum()
            assert np.all(np.abs(got[i] - ora) <= 1e-4 * np.abs(ora) + 1e-5 * scale), (i, got[i], ora)
