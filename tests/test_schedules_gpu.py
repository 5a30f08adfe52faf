"""Both radix schedules of the forward transforms (the autotuner's choice
per patch side: 32 = 8*4 or 8*2*2, 64 = 8*8 or 8*4*2, 128 = 8*8*2 or 8*4*4,
256 = 8*8*4 or 8*4*8) against the FP64 oracle at every side: max |d pixel|
<= 2e-6 flux, |d flux| / flux <= 1e-5."""

import numpy as np
import pytest

from parity import check_parity, gpu_patches, oracle_patches
from workloads import config2_galaxies

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sched_renderer(tables, psf0):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_15797_gb300.build import build
    build()
    from paper_2012_15797_gb300.renderer import Renderer
    from workloads import config2_psfs
    psfs = [psf0] + config2_psfs(4)
    r = Renderer(tables, psfs)
    r.psfs = psfs
    yield r
    r.close()


@pytest.mark.parametrize("schedule", [0, 1])
def test_schedule_parity_every_side(sched_renderer, tables, schedule):
    from paper_2012_15797_gb300 import capi
    for n in (32, 64, 128, 256):
        capi.mog_set_launch_shape(sched_renderer.ctx, 0, n, 0, 8, schedule)
    gals = config2_galaxies(1500, seed=91 + schedule, n_psf=5)
    idx = []
    for n in (32, 64, 128, 256):
        idx += list(np.flatnonzero(gals.size == n)[:6])
    sub = gals.subset(np.array(idx))
    gpu, _, _ = gpu_patches(sched_renderer, sub)
    ora = oracle_patches(sub, sched_renderer.psfs, tables)
    check_parity(gpu, ora, sub)


def test_launch_shape_arguments_checked(sched_renderer):
    from paper_2012_15797_gb300 import capi
    for bad in [(2, 64, 0, 8, 0), (0, 48, 0, 8, 0), (0, 64, 0, 0, 0), (0, 64, 0, 8, 2), (1, 64, 0, 8, 1)]:
        with pytest.raises(capi.MogError):
            capi.mog_set_launch_shape(sched_renderer.ctx, *bad)
