"""mog_render_batch_host: parameters and patches in host memory, chunks
pipelined over two streams.  The chunks run the same kernels as the device
entry point, so the patches must equal mog_render_batch's bit for bit, for
any chunking (one chunk, many chunks over both lanes, a ragged last chunk),
both shift modes, pinned and pageable memory; a few galaxies are also checked
against the FP64 oracle with the method's tolerance."""

import numpy as np
import pytest

from oracle import render as R
from workloads import fixed_galaxies_64, mixed_galaxies

pytestmark = pytest.mark.gpu


def _device_render(r, gals, shift="phase"):
    from paper_2012_15797_gb300.renderer import to_device
    b = to_device(gals)
    out = r.render(b, shift=shift)
    r.sync_status()
    return out.cpu().numpy()


def _host_render(r, gals, chunk=0, shift="phase", pin=True):
    from paper_2012_15797_gb300.renderer import host_batch
    got = r.render_host(host_batch(gals, pin=pin), chunk=chunk, shift=shift)
    r.sync_status()
    return got.numpy()


@pytest.mark.parametrize("chunk", [0, 1, 257, 1000])
def test_fixed_size_equals_device_render(gpu_renderer, chunk):
    gals = fixed_galaxies_64(2500, seed=71)
    assert np.array_equal(_host_render(gpu_renderer, gals, chunk), _device_render(gpu_renderer, gals))


def test_mixed_sizes_and_psfs_equal_device_render(gpu_renderer):
    gals = mixed_galaxies(3000, seed=72, n_psf=5)
    want = _device_render(gpu_renderer, gals)
    assert np.array_equal(_host_render(gpu_renderer, gals, chunk=333), want)
    assert np.array_equal(_host_render(gpu_renderer, gals, chunk=0), want)


def test_lanczos_and_pageable_memory(gpu_renderer):
    gals = mixed_galaxies(800, seed=73, n_psf=5)
    want = _device_render(gpu_renderer, gals, shift="lanczos")
    assert np.array_equal(_host_render(gpu_renderer, gals, chunk=100, shift="lanczos"), want)
    assert np.array_equal(_host_render(gpu_renderer, gals, chunk=100, shift="lanczos", pin=False), want)


def test_matches_the_oracle(gpu_renderer, tables):
    gals = fixed_galaxies_64(40, seed=74)
    got = _host_render(gpu_renderer, gals, chunk=7)
    off = 0
    for i in range(len(gals)):
        g = gals.row(i)
        n = int(g["size"])
        p = gpu_renderer.psfs[g["psf"]]
        ref = R.render(g, p.image, p.mog, tables)
        img = got[off:off + n * n].reshape(n, n).astype(np.float64)
        off += n * n
        assert np.max(np.abs(img - ref)) <= 2e-6 * g["flux"], i
        assert abs(img.sum() - ref.sum()) <= 1e-5 * g["flux"], i


def test_rejects_bad_layouts(gpu_renderer):
    import torch
    from paper_2012_15797_gb300 import capi
    from paper_2012_15797_gb300.renderer import host_batch
    gals = fixed_galaxies_64(10, seed=75)
    t, total = host_batch(gals)
    out = torch.empty(total, dtype=torch.float32)

    def call(tt, flags=0):
        b = capi.make_batch(len(tt["flux"]), {k: v.data_ptr() for k, v in tt.items()})
        capi.mog_render_batch_host(gpu_renderer.ctx, b, out.data_ptr(), 0, flags)

    gapped = dict(t)
    gapped["offset"] = t["offset"].clone()
    gapped["offset"][5:] += 16   # a gap between patches 4 and 5
    with pytest.raises(capi.MogError):
        call(gapped)
    bad_size = dict(t)
    bad_size["size"] = t["size"].clone()
    bad_size["size"][3] = 48
    with pytest.raises(capi.MogError):
        call(bad_size)
    with pytest.raises(capi.MogError):
        call(t, flags=capi.MOG_RENDER_ADD)
    call(t)   # the context still works after the rejected calls
