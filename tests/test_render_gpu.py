"""GPU parity of the fused forward render (through the C-ABI) against the
FP64 oracle: max |d pixel| <= 2e-6 flux, |d flux| / flux <= 1e-5."""

import numpy as np
import pytest

from parity import check_parity, gpu_patches, oracle_patches
from workloads import (Galaxies, single_galaxy_64, fixed_galaxies_64, mixed_galaxies,
                       PROFILE_EXP, PROFILE_DEV, PROFILE_SERSIC)

pytestmark = pytest.mark.gpu


def _gals(rows):
    keys = Galaxies.FLOAT_FIELDS + Galaxies.INT_FIELDS
    cols = {k: np.array([r[k] for r in rows]) for k in keys}
    f = {k: cols[k].astype(np.float32) for k in Galaxies.FLOAT_FIELDS}
    i = {k: cols[k].astype(np.int32) for k in Galaxies.INT_FIELDS}
    return Galaxies(**f, **i)


def _row(**kw):
    r = single_galaxy_64().row(0)
    r.update(kw)
    return r


def test_single_galaxy_64(gpu_renderer, tables):
    gals = single_galaxy_64()
    gpu, _, _ = gpu_patches(gpu_renderer, gals)
    ora = oracle_patches(gals, gpu_renderer.psfs, tables)
    check_parity(gpu, ora, gals)


EDGE = [
    dict(),                                                  # the single 64x64 galaxy as drawn
    dict(e1=0.0, e2=0.0),                                     # round
    dict(e1=0.6 * np.cos(1.0), e2=0.6 * np.sin(1.0)),         # |e| = 0.6
    dict(flux=1e4), dict(x=0.5, y=-0.5), dict(x=-0.5, y=0.4999),
    dict(log_re=np.log(1e-4)),                                # point-source limit
    dict(log_re=np.log(20.0), profile=PROFILE_DEV, sersic_n=4.0),   # mostly real space
    dict(log_re=np.log(0.3), profile=PROFILE_DEV, sersic_n=4.0),
    dict(profile=PROFILE_SERSIC, sersic_n=0.5), dict(profile=PROFILE_SERSIC, sersic_n=6.0),
    dict(profile=PROFILE_SERSIC, sersic_n=2.6), dict(profile=PROFILE_SERSIC, sersic_n=4.375, psf=3),
    dict(x=3.7, y=-6.2),                                      # offsets beyond a pixel
]


@pytest.mark.parametrize("size", [32, 64, 128, 256])
def test_edge_cases_each_size(gpu_renderer, tables, size):
    rows = [_row(size=size, **e) for e in EDGE]
    gals = _gals(rows)
    gpu, _, _ = gpu_patches(gpu_renderer, gals)
    ora = oracle_patches(gals, gpu_renderer.psfs, tables)
    check_parity(gpu, ora, gals)


@pytest.mark.parametrize("size", [32, 64, 128, 256])
def test_ramp_boundaries(gpu_renderer, tables, size):
    """Galaxies whose largest exp component sits at n_sigma = 2.9, 3, 3.5, 4
    and 4.1 (the aliasing split of Step 4 and its ramp)."""
    a, v = tables[PROFILE_EXP].amp[0], tables[PROFILE_EXP].var[0]
    vmax = v[0]
    rows = []
    for ns in (2.9, 3.0, 3.2, 3.5, 3.8, 4.0, 4.1):
        # round galaxy: trace(v S) = 2 v r_e^2 -> r_e = (N/2) / (ns sqrt(2 v))
        r_e = 0.5 * size / (ns * np.sqrt(2 * vmax))
        rows.append(_row(size=size, e1=0.0, e2=0.0, log_re=np.log(r_e)))
    gals = _gals(rows)
    gpu, _, _ = gpu_patches(gpu_renderer, gals)
    ora = oracle_patches(gals, gpu_renderer.psfs, tables)
    check_parity(gpu, ora, gals)


def test_batch_fixed_size_ragged(gpu_renderer, tables):
    """333 config-1 galaxies (many CTAs, a ragged last chunk)."""
    gals = fixed_galaxies_64(333, seed=11)
    gpu, _, _ = gpu_patches(gpu_renderer, gals)
    ora = oracle_patches(gals, gpu_renderer.psfs, tables)
    check_parity(gpu, ora, gals)


def test_batch_mixed_sizes_and_psfs(gpu_renderer, tables):
    gals = mixed_galaxies(301, seed=12, n_psf=5)
    assert set(np.unique(gals.size)) == {32, 64, 128, 256}
    gpu, _, _ = gpu_patches(gpu_renderer, gals)
    ora = oracle_patches(gals, gpu_renderer.psfs, tables)
    check_parity(gpu, ora, gals)


def test_batch_equals_single(gpu_renderer):
    gals = mixed_galaxies(64, seed=13, n_psf=5)
    full, _, _ = gpu_patches(gpu_renderer, gals)
    big = int(np.nonzero(gals.size == 256)[0][0])
    for i in (0, 5, big, len(gals) - 1):
        one, _, _ = gpu_patches(gpu_renderer, gals.subset([i]))
        assert np.array_equal(one[0], full[i])


def test_every_pixel_written_once_and_gaps_untouched(gpu_renderer):
    import torch
    from paper_2012_15797_gb300.renderer import to_device
    gals = fixed_galaxies_64(50, seed=14)
    b = to_device(gals)
    # spread the patches out with 4-float gaps filled with a canary
    off = np.arange(50, dtype=np.int64) * (64 * 64 + 4)
    b.tensors["offset"] = torch.from_numpy(off).cuda()
    out = torch.full((50 * (64 * 64 + 4),), -7.0, dtype=torch.float32, device="cuda")
    gpu_renderer.render(b, out)
    gpu_renderer.sync_status()
    o = out.cpu().numpy().reshape(50, 64 * 64 + 4)
    assert np.all(o[:, -4:] == -7.0)
    assert not np.any(o[:, :-4] == -7.0)


def test_empty_batch(gpu_renderer):
    gals = fixed_galaxies_64(0)
    gpu, out, _ = gpu_patches(gpu_renderer, gals)
    assert gpu == [] and out.numel() == 0


def test_invalid_galaxy_reports_status_and_skips(gpu_renderer):
    import torch
    from paper_2012_15797_gb300.capi import MogError, MOG_ERR_DEVICE
    from paper_2012_15797_gb300.renderer import to_device
    gals = fixed_galaxies_64(3, seed=15)
    gals.log_re[1] = np.nan
    b = to_device(gals)
    out = torch.full((b.total,), -3.0, dtype=torch.float32, device="cuda")
    gpu_renderer.render(b, out)
    with pytest.raises(MogError) as ei:
        gpu_renderer.sync_status()
    assert ei.value.status == MOG_ERR_DEVICE
    o = out.cpu().numpy().reshape(3, -1)
    assert np.all(o[1] == -3.0) and np.all(np.isfinite(o[0])) and np.all(np.isfinite(o[2]))
    gpu_renderer.sync_status()   # cleared


def test_unsupported_size_reports_status(gpu_renderer):
    import torch
    from paper_2012_15797_gb300.capi import MogError
    from paper_2012_15797_gb300.renderer import to_device
    gals = fixed_galaxies_64(2, seed=16, size=48)
    b = to_device(gals)
    out = torch.zeros(b.total, dtype=torch.float32, device="cuda")
    gpu_renderer.render(b, out)
    with pytest.raises(MogError):
        gpu_renderer.sync_status()


def test_full_100k_64_sampled(gpu_renderer, tables):
    """100k galaxies at 64^2 in one call (the benchmark's launch), 48 sampled
    patches checked against the oracle."""
    gals = fixed_galaxies_64()
    gpu, _, _ = gpu_patches(gpu_renderer, gals.subset(np.arange(len(gals))))
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(len(gals), 48, replace=False))
    ora = oracle_patches(gals, gpu_renderer.psfs, tables, idx)
    check_parity([gpu[i] for i in idx], ora, gals, idx)
