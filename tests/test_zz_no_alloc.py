"""The allocation-free render entry point, for callers that cannot let the
library allocate device memory while they render (processes serving every
buffer from a pre-reserved arena; latency-critical loops that cannot take
cudaMalloc's possible device synchronisation).  It must give the same patches
as mog_render_batch, call after call, although its fixed scratch array keeps
the previous call's contents.

This file is collected last so that a failure here leaves every other test
already run."""

import numpy as np
import pytest

from parity import PIX_TOL
from workloads import fixed_galaxies_64, mixed_galaxies

pytestmark = pytest.mark.gpu


def _render_both(renderer, gals):
    import torch
    from paper_2012_15797_gb300 import capi
    from paper_2012_15797_gb300.renderer import to_device
    b = to_device(gals)
    ref = torch.full((b.total,), float("nan"), device="cuda")
    renderer.render(b, ref)
    got = torch.full((b.total,), float("nan"), device="cuda")
    capi.mog_render_batch_noalloc(renderer.ctx, capi.make_batch(b.count, b.ptrs(), b.size_mask()), got.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
    renderer.sync_status()
    return ref.cpu().numpy(), got.cpu().numpy(), b


def _check(ref, got, b, gals):
    assert np.all(np.isfinite(got))
    for i in range(b.count):
        o, n = int(b.offsets[i]), int(b.sizes[i]) ** 2
        assert np.max(np.abs(got[o:o + n] - ref[o:o + n])) <= PIX_TOL * float(gals.flux[i])


def test_noalloc_matches_render_batch_two_calls(gpu_renderer):
    # first call: mixed sizes and PSFs; second call: a smaller batch, so stale
    # scratch from the first call would show up if it were read
    g1 = mixed_galaxies(3000, seed=41, n_psf=5)
    g2 = fixed_galaxies_64(700, seed=42)
    for gals in (g1, g2):
        ref, got, b = _render_both(gpu_renderer, gals)
        _check(ref, got, b, gals)


def test_noalloc_rejects_oversized_batch(gpu_renderer):
    import torch
    from paper_2012_15797_gb300 import capi
    from paper_2012_15797_gb300.renderer import to_device
    gals = fixed_galaxies_64(capi.MOG_NOALLOC_MAX_GALAXIES + 1, seed=43)
    b = to_device(gals)
    out = torch.empty(b.total, device="cuda")
    with pytest.raises(capi.MogError) as ei:
        capi.mog_render_batch_noalloc(gpu_renderer.ctx, capi.make_batch(b.count, b.ptrs()), out.data_ptr())
    assert ei.value.status == capi.MOG_ERR_ARG
    assert "at most" in str(ei.value)


def test_noalloc_call_allocates_nothing(gpu_renderer):
    # the device's free memory is the same before and after calls made once
    # the kernels are loaded: no call allocates (or frees) device memory
    import torch
    from paper_2012_15797_gb300 import capi
    from paper_2012_15797_gb300.renderer import to_device
    b = to_device(mixed_galaxies(2000, seed=44, n_psf=5))
    out = torch.empty(b.total, device="cuda")
    batch = capi.make_batch(b.count, b.ptrs(), b.size_mask())
    stream = torch.cuda.current_stream().cuda_stream
    capi.mog_render_batch_noalloc(gpu_renderer.ctx, batch, out.data_ptr(), stream)
    gpu_renderer.sync_status()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        capi.mog_render_batch_noalloc(gpu_renderer.ctx, batch, out.data_ptr(), stream)
    gpu_renderer.sync_status()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_skips_eigen_psf_galaxies(tables, psf0):
    # an eigen-PSF galaxy has no place for its per-galaxy PSF terms in the
    # fixed array: it is reported as MOG_ERR_DEVICE and its patch is left
    # untouched, while the other galaxies of the call render as usual
    import torch
    from paper_2012_15797_gb300 import capi
    from paper_2012_15797_gb300.renderer import Renderer, to_device
    from workloads import eigen_positions, eigen_psf
    r = Renderer(tables, [psf0, eigen_psf()])
    try:
        gals = fixed_galaxies_64(64, seed=45)
        gals.psf[5] = 1
        gals.psf[40] = 1
        b = to_device(gals, positions=eigen_positions(len(gals)))
        ref = torch.full((b.total,), float("nan"), device="cuda")
        r.render(b, ref)
        r.sync_status()
        got = torch.full((b.total,), float("nan"), device="cuda")
        capi.mog_render_batch_noalloc(r.ctx, capi.make_batch(b.count, b.ptrs(), b.size_mask()), got.data_ptr(),
                                      torch.cuda.current_stream().cuda_stream)
        with pytest.raises(capi.MogError) as ei:
            r.sync_status()
        assert ei.value.status == capi.MOG_ERR_DEVICE
        ref, got = ref.cpu().numpy(), got.cpu().numpy()
        for i in range(b.count):
            o, n = int(b.offsets[i]), int(b.sizes[i]) ** 2
            if gals.psf[i] == 1:
                assert np.all(np.isnan(got[o:o + n]))
            else:
                assert np.max(np.abs(got[o:o + n] - ref[o:o + n])) <= PIX_TOL * float(gals.flux[i])
    finally:
        r.close()
