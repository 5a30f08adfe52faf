"""Every transform schedule of the forward render (the autotuner's choice
per patch side: radix 32 = 8*4 or 8*2*2, 64 = 8*8 or 8*4*2, 128 = 8*8*2 or
8*4*4, 256 = 8*8*4 or 8*4*8, and for 64 x 64 a warp per galaxy with
register-resident transforms) against the FP64 oracle: max |d pixel|
<= 2e-6 flux, |d flux| / flux <= 1e-5."""

import numpy as np
import pytest

from parity import check_parity, gpu_patches, oracle_patches
from test_render_gpu import EDGE, _gals, _row
from workloads import fixed_galaxies_64, mixed_galaxies

pytestmark = pytest.mark.gpu

CASES = [(32, 0), (32, 1), (64, 0), (64, 1), (64, 2), (128, 0), (128, 1), (128, 2), (256, 0), (256, 1)]


@pytest.fixture(scope="module")
def sched_renderer(tables, psf0):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_15797_gb300.build import build
    build()
    from paper_2012_15797_gb300.renderer import Renderer
    from workloads import psf_set
    psfs = [psf0] + psf_set(4)
    r = Renderer(tables, psfs)
    r.psfs = psfs
    yield r
    r.close()


def _use(renderer, n, schedule, chunk=8):
    from paper_2012_15797_gb300 import capi
    for m in (32, 64, 128, 256):
        capi.mog_set_launch_shape(renderer.ctx, 0, m, 0, chunk, schedule if m == n else 0)


@pytest.mark.parametrize("n,schedule", CASES)
def test_schedule_parity(sched_renderer, tables, n, schedule):
    _use(sched_renderer, n, schedule)
    gals = mixed_galaxies(1500, seed=91 + schedule, n_psf=5)
    sub = gals.subset(np.flatnonzero(gals.size == n)[:12])
    gpu, _, _ = gpu_patches(sched_renderer, sub)
    ora = oracle_patches(sub, sched_renderer.psfs, tables)
    check_parity(gpu, ora, sub)
    rows = [_row(size=n, **e) for e in EDGE]
    edge = _gals(rows)
    gpu, _, _ = gpu_patches(sched_renderer, edge)
    check_parity(gpu, oracle_patches(edge, sched_renderer.psfs, tables), edge)


def test_warp_kernel_sampled_fixed_size_batch_and_add_mode(sched_renderer, tables):
    # the 64 x 64 warp kernel on the fixed-size distribution (exp / deV, one
    # PSF), a ragged count, with queue chunks of 1 and 32; and adding to
    # what the patches hold gives the plain render plus the old contents
    import torch
    from paper_2012_15797_gb300.renderer import patches, to_device
    gals = fixed_galaxies_64(3001, seed=95)
    idx = np.arange(0, 3001, 150)
    for chunk in (1, 32):
        _use(sched_renderer, 64, 2, chunk)
        gpu, out, b = gpu_patches(sched_renderer, gals)
        sub = gals.subset(idx)
        check_parity([gpu[i] for i in idx], oracle_patches(sub, sched_renderer.psfs, tables), sub)
    base = torch.randn(b.total, device="cuda")
    added = base.clone()
    sched_renderer.render(b, added, add=True)
    sched_renderer.sync_status()
    torch.testing.assert_close(added, base + out, rtol=0, atol=1e-6 * float(gals.flux.max()))


def test_launch_shape_arguments_checked(sched_renderer):
    from paper_2012_15797_gb300 import capi
    for bad in [(2, 64, 0, 8, 0), (0, 48, 0, 8, 0), (0, 64, 0, 0, 0), (0, 64, 0, 8, 3), (0, 32, 0, 8, 2),
                (0, 256, 0, 8, 2), (0, 128, 0, 8, 3), (1, 64, 0, 8, 1), (1, 128, 0, 8, 2)]:
        with pytest.raises(capi.MogError):
            capi.mog_set_launch_shape(sched_renderer.ctx, *bad)
