"""mog_render_chi2: render and loss in one pass.  The gradient patches, chi2
and optional model equal mog_render_batch followed by mog_chi2_gradient (the
model and gradient bit for bit, chi2 up to the order of its sum) at every
side, on mixed sizes and PSFs, with eigen-PSFs in the context; skipped
galaxies get chi2 NaN; arguments are checked."""

import numpy as np
import pytest
import torch

from workloads import fixed_galaxies_64, mixed_galaxies

pytestmark = pytest.mark.gpu


def _data_like(model, seed):
    g = torch.Generator(device="cpu").manual_seed(seed)
    noise = torch.randn(model.numel(), generator=g).to(model.device)
    return (model * 1.01 + 0.05 * noise).contiguous()


def _reference(r, b, data, ivar):
    model = r.render(b)
    grad, chi2 = r.chi2_gradient(b, model, data, ivar)
    r.sync_status()
    return model, grad, chi2


def _check(r, gals, seed):
    from paper_2012_15797_gb300.renderer import to_device
    b = to_device(gals)
    ref_model = r.render(b)
    data = _data_like(ref_model, seed)
    ivar = torch.from_numpy(np.random.default_rng(seed).uniform(0.5, 3.0, len(gals)).astype(np.float32)).cuda()
    model, grad_ref, chi2_ref = _reference(r, b, data, ivar)
    mdl = torch.full_like(model, -1.0)
    grad, chi2 = r.render_chi2(b, data, ivar, model=mdl)
    r.sync_status()
    assert torch.equal(mdl, model)
    assert torch.equal(grad, grad_ref)
    assert torch.allclose(chi2, chi2_ref, rtol=2e-5, atol=0.0)
    grad2, chi2b = r.render_chi2(b, data, ivar)       # without the model output
    r.sync_status()
    assert torch.equal(grad2, grad_ref) and torch.equal(chi2b, chi2)


def test_fixed_size(gpu_renderer):
    _check(gpu_renderer, fixed_galaxies_64(3000, seed=81), 1)


def test_mixed_sizes_and_psfs(gpu_renderer):
    _check(gpu_renderer, mixed_galaxies(2500, seed=82, n_psf=5), 2)


def test_eigen_psf_context(tables, psf0):
    from paper_2012_15797_gb300.renderer import Renderer
    from workloads import eigen_psf
    r = Renderer(tables, [psf0, eigen_psf()])
    try:
        _check(r, mixed_galaxies(800, seed=83, n_psf=1), 3)
    finally:
        r.close()


def test_skipped_galaxy_and_arguments(gpu_renderer):
    from paper_2012_15797_gb300 import capi
    from paper_2012_15797_gb300.renderer import to_device
    gals = fixed_galaxies_64(50, seed=84)
    gals.flux[7] = np.nan
    gals.size[11] = 48                     # a side no kernel renders
    b = to_device(gals)
    data = torch.zeros(b.total, device="cuda")
    ivar = torch.ones(len(gals), device="cuda")
    grad, chi2 = gpu_renderer.render_chi2(b, data, ivar)
    with pytest.raises(capi.MogError):
        gpu_renderer.sync_status()
    c = chi2.cpu().numpy()
    assert np.isnan(c[7]) and np.isnan(c[11]) and np.all(np.isfinite(np.delete(c, [7, 11])))
    bb = capi.make_batch(b.count, b.ptrs(), b.size_mask())
    with pytest.raises(capi.MogError):
        capi.mog_render_chi2(gpu_renderer.ctx, bb, 0, ivar.data_ptr(), grad.data_ptr(), chi2.data_ptr())
    with pytest.raises(capi.MogError):
        capi.mog_render_chi2(gpu_renderer.ctx, bb, data.data_ptr() + 4, ivar.data_ptr(), grad.data_ptr(),
                             chi2.data_ptr())
