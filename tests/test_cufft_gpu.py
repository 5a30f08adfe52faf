"""mog_render_batch_cufft, the library comparator (spectra written out, one
batched cuFFT inverse real transform, real-space add): parity with the FP64
oracle at every side (edge cases, ragged batches, several PSFs) within the
render's tolerance, agreement with the fused render to float rounding, and
its argument and status checks."""

import numpy as np
import pytest
import torch

from parity import PIX_TOL, check_parity, oracle_patches
from workloads import Galaxies, fixed_galaxies_64, single_galaxy_64, PROFILE_DEV, PROFILE_SERSIC

pytestmark = pytest.mark.gpu

SIDES = [32, 64, 128, 256]


def _cufft_patches(r, gals):
    from paper_2012_15797_gb300.renderer import patches, to_device
    b = to_device(gals)
    out = torch.full((b.total,), float("nan"), dtype=torch.float32, device="cuda")
    r.render_cufft(b, out)
    r.sync_status()
    return [p.double().cpu().numpy() for p in patches(out, b)], out, b


def _gals(rows):
    cols = {k: np.array([r[k] for r in rows]) for k in Galaxies.FLOAT_FIELDS + Galaxies.INT_FIELDS}
    return Galaxies(**{k: cols[k].astype(np.float32) for k in Galaxies.FLOAT_FIELDS},
                    **{k: cols[k].astype(np.int32) for k in Galaxies.INT_FIELDS})


EDGE = [
    dict(), dict(e1=0.0, e2=0.0), dict(e1=0.6 * np.cos(1.0), e2=0.6 * np.sin(1.0)),
    dict(x=0.5, y=-0.5), dict(x=3.7, y=-6.2), dict(log_re=np.log(1e-4)),
    dict(log_re=np.log(20.0), profile=PROFILE_DEV, sersic_n=4.0),
    dict(profile=PROFILE_SERSIC, sersic_n=0.5), dict(profile=PROFILE_SERSIC, sersic_n=4.375, psf=3),
]


@pytest.mark.parametrize("size", SIDES)
def test_edge_cases_against_oracle(gpu_renderer, tables, size):
    base = single_galaxy_64().row(0)
    gals = _gals([{**base, "size": size, **e} for e in EDGE])
    gpu, _, _ = _cufft_patches(gpu_renderer, gals)
    check_parity(gpu, oracle_patches(gals, gpu_renderer.psfs, tables), gals)


@pytest.mark.parametrize("size,count", [(32, 517), (64, 333), (128, 129), (256, 37)])
def test_ragged_batch_against_oracle_and_fused(gpu_renderer, tables, size, count):
    gals = fixed_galaxies_64(count, seed=90 + size, size=size)
    gals.psf[:] = np.arange(count) % 5                     # several PSFs in one batch
    gpu, out, b = _cufft_patches(gpu_renderer, gals)
    idx = list(range(0, count, max(1, count // 12))) + [count - 1]
    check_parity([gpu[i] for i in idx], oracle_patches(gals, gpu_renderer.psfs, tables, idx), gals, idx)
    fused = gpu_renderer.render(b)
    gpu_renderer.sync_status()
    d = (out - fused).abs().view(count, -1).amax(dim=1).cpu().numpy()
    assert np.all(d <= 0.25 * PIX_TOL * gals.flux), float(np.max(d / gals.flux))


def test_full_100k_64_sampled(gpu_renderer, tables):
    """The 100k 64 x 64 workload: every patch against the fused render, a
    sample against the oracle."""
    gals = fixed_galaxies_64(100_000, seed=1)
    gpu, out, b = _cufft_patches(gpu_renderer, gals)
    idx = [0, 1, 4999, 31337, 77777, 99_999]
    check_parity([gpu[i] for i in idx], oracle_patches(gals, gpu_renderer.psfs, tables, idx), gals, idx)
    fused = gpu_renderer.render(b)
    gpu_renderer.sync_status()
    d = (out - fused).abs().view(len(gals), -1).amax(dim=1).cpu().numpy()
    assert np.all(d <= 0.25 * PIX_TOL * gals.flux), float(np.max(d / gals.flux))


def test_arguments_and_status(gpu_renderer):
    from paper_2012_15797_gb300 import capi
    from paper_2012_15797_gb300.renderer import to_device
    gals = fixed_galaxies_64(6, seed=97)
    gals.size[4] = 32                                       # another side in the batch
    gals.flux[2] = np.nan                                   # an invalid galaxy
    b = to_device(gals)
    out = torch.full((b.total,), -5.0, dtype=torch.float32, device="cuda")
    with pytest.raises(capi.MogError):                      # the mask names two sides
        gpu_renderer.render_cufft(b, out)
    bb = capi.make_batch(b.count, b.ptrs(), 0x2)            # render the 64 x 64 galaxies only
    capi.mog_render_batch_cufft(gpu_renderer.ctx, bb, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    with pytest.raises(capi.MogError):
        gpu_renderer.sync_status()
    gpu_renderer.sync_status()                              # cleared
    offs = b.tensors["offset"].cpu().numpy()
    o = out.cpu().numpy()
    for g in range(6):
        p = o[offs[g]:offs[g] + gals.size[g] ** 2]
        if g in (2, 4):
            assert np.all(p == -5.0)                        # skipped, untouched
        else:
            assert np.all(np.isfinite(p)) and not np.any(p == -5.0)
    for mask in (0, 0x3, 0x10):
        bad = capi.make_batch(b.count, b.ptrs(), mask)
        with pytest.raises(capi.MogError):
            capi.mog_render_batch_cufft(gpu_renderer.ctx, bad, out.data_ptr(), 0)
    with pytest.raises(capi.MogError):                      # misaligned output
        capi.mog_render_batch_cufft(gpu_renderer.ctx, bb, out.data_ptr() + 4, 0)
    empty = to_device(fixed_galaxies_64(0))
    gpu_renderer.render_cufft(empty, torch.empty(0, device="cuda"))


def test_eigen_psf_galaxies_skipped_and_plan_rebuilt(tables, psf0):
    """Galaxies on an eigen-PSF are skipped with MOG_ERR_DEVICE (the others
    render); calls of different counts and sides re-plan and stay correct."""
    from paper_2012_15797_gb300 import capi
    from paper_2012_15797_gb300.renderer import Renderer, patches, to_device
    from workloads import eigen_positions, eigen_psf
    r = Renderer(tables, [psf0, eigen_psf()])
    try:
        gals = fixed_galaxies_64(12, seed=98)
        gals.psf[[3, 8]] = 1
        b = to_device(gals, positions=eigen_positions(len(gals)))
        out = torch.full((b.total,), -4.0, dtype=torch.float32, device="cuda")
        r.render_cufft(b, out)
        with pytest.raises(capi.MogError):
            r.sync_status()
        got = [p.double().cpu().numpy() for p in patches(out, b)]
        keep = [i for i in range(len(gals)) if i not in (3, 8)]
        assert np.all(got[3] == -4.0) and np.all(got[8] == -4.0)
        check_parity([got[i] for i in keep], oracle_patches(gals, [psf0], tables, keep), gals, keep)
        for n, count in ((32, 7), (64, 19), (32, 7)):
            g2 = fixed_galaxies_64(count, seed=99 + n + count, size=n)
            one, _, b2 = _cufft_patches(r, g2)
            fused = r.render(b2)
            r.sync_status()
            d = max(float(np.max(np.abs(one[i] - p.double().cpu().numpy()))) / float(g2.flux[i])
                    for i, p in enumerate(patches(fused, b2)))
            assert d <= 0.25 * PIX_TOL, d
    finally:
        r.close()
