"""The fit loss and its gradient on the device (mog_chi2_gradient):
chi^2 = ivar sum (model - data)^2 per galaxy and d chi^2 / d model =
2 ivar (model - data), against the same sums in float64 on the host, for
mixed patch sides, in place over the model, and unsupported sides skipped."""

import numpy as np
import pytest

from workloads import mixed_galaxies

pytestmark = pytest.mark.gpu


def test_chi2_gradient_matches_float64(gpu_renderer):
    import torch
    from paper_2012_15797_gb300.renderer import patches, to_device
    gals = mixed_galaxies(300, seed=71, n_psf=5)
    b = to_device(gals)
    model = gpu_renderer.render(b)
    gen = torch.Generator(device="cuda").manual_seed(3)
    data = model + 1e-3 * torch.randn(model.shape, device="cuda", generator=gen)
    ivar = torch.from_numpy(np.random.default_rng(4).uniform(0.5, 2.0, len(gals)).astype(np.float32)).cuda()
    grad, chi2 = gpu_renderer.chi2_gradient(b, model, data, ivar)
    gpu_renderer.sync_status()
    m, d, g = (patches(t, b) for t in (model, data, grad))
    for i in range(len(gals)):
        r = m[i].double() - d[i].double()
        iv = float(ivar[i])
        want_c = iv * float((r * r).sum())
        assert abs(float(chi2[i]) - want_c) <= 1e-5 * want_c
        torch.testing.assert_close(g[i].double(), 2.0 * iv * r, rtol=1e-6, atol=1e-9)
    # in place over the model
    grad2, _ = gpu_renderer.chi2_gradient(b, model, data, ivar, grad_pix=model)
    gpu_renderer.sync_status()
    assert torch.equal(grad2, grad)


def test_chi2_gradient_skips_unsupported_sides(gpu_renderer):
    import torch
    from paper_2012_15797_gb300 import capi
    from paper_2012_15797_gb300.renderer import to_device
    gals = mixed_galaxies(20, seed=72, n_psf=5)
    b = to_device(gals)
    model = torch.ones(b.total, device="cuda")
    data = torch.zeros_like(model)
    ivar = torch.ones(len(gals), device="cuda")
    b.tensors["size"][3] = 48
    grad = torch.full_like(model, -7.0)
    chi2 = torch.zeros(len(gals), device="cuda")
    capi.mog_chi2_gradient(gpu_renderer.ctx, capi.make_batch(b.count, b.ptrs()), model.data_ptr(), data.data_ptr(),
                           ivar.data_ptr(), grad.data_ptr(), chi2.data_ptr())
    torch.cuda.synchronize()
    assert torch.isnan(chi2[3]) and torch.all(torch.isfinite(chi2[torch.arange(20, device="cuda") != 3]))
    o, n = int(b.offsets[3]), int(gals.size[3]) ** 2
    assert torch.all(grad[o:o + n] == -7.0)
