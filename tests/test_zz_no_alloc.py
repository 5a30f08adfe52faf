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
from workloads import config1_galaxies, config2_galaxies

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
    g1 = config2_galaxies(3000, seed=41, n_psf=5)
    g2 = config1_galaxies(700, seed=42)
    for gals in (g1, g2):
        ref, got, b = _render_both(gpu_renderer, gals)
        _check(ref, got, b, gals)


def test_noalloc_rejects_oversized_batch(gpu_renderer):
    import torch
    from paper_2012_15797_gb300 import capi
    from paper_2012_15797_gb300.renderer import to_device
    gals = config1_galaxies(capi.MOG_NOALLOC_MAX_GALAXIES + 1, seed=43)
    b = to_device(gals)
    out = torch.empty(b.total, device="cuda")
    with pytest.raises(capi.MogError) as ei:
        capi.mog_render_batch_noalloc(gpu_renderer.ctx, capi.make_batch(b.count, b.ptrs()), out.data_ptr())
    assert ei.value.status == capi.MOG_ERR_ARG
    assert "at most" in str(ei.value)
