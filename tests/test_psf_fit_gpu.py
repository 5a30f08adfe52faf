"""On-device Gaussian-mixture fits of pixelized PSFs (mog_fit_psf_mixture)
against the FP64 oracle fit: exact mixtures recovered, and for real
(Moffat-winged) PSFs a chi^2 within 2% of the oracle's local minimum from the
same start."""

import numpy as np
import pytest

from oracle import psf_fit as F
from workloads import psf_set

pytestmark = pytest.mark.gpu


def _gauss_image(rows, n):
    return F.mixture_image(np.asarray(rows, dtype=np.float64), n, n)


def gpu_fit(renderer, images, k, iters=400):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(np.stack(images), dtype=np.float32)).cuda()
    rows, chi2 = renderer.fit_psf_mixtures(t, k=k, iters=iters)
    renderer.sync_status()
    return rows.double().cpu().numpy(), chi2.double().cpu().numpy()


TRUTHS = [
    [[0.8, 0.0, 0.0, 2.25, 0.0, 2.25], [0.2, 0.0, 0.0, 9.0, 0.0, 9.0]],
    [[0.6, 0.25, -0.15, 2.0, 0.5, 1.6], [0.3, -0.1, 0.2, 6.0, -1.2, 4.5], [0.1, 0.0, 0.0, 20.0, 0.0, 20.0]],
]


@pytest.mark.parametrize("n", [32, 64])
@pytest.mark.parametrize("truth", TRUTHS)
def test_exact_mixture_recovered(gpu_renderer, n, truth):
    truth = np.array(truth)
    rows, chi2 = gpu_fit(gpu_renderer, [_gauss_image(truth, n)], k=len(truth))
    want = truth[np.argsort(-truth[:, 0])]
    assert np.max(np.abs(rows[0] - want) / np.maximum(np.abs(want), 0.05)) < 2e-3, (rows[0], want)
    assert chi2[0] < 1e-10


def test_winged_psfs_match_the_oracle_fit(gpu_renderer):
    psfs = [p.image.astype(np.float64) for p in psf_set(6, seed=31, fit=False)]
    rows, chi2 = gpu_fit(gpu_renderer, psfs, k=3)
    for i, img in enumerate(psfs):
        ora_rows, ora_chi2 = F.fit_mog(img, 3)
        start = F.chi2(F.mixture_rows(F.initial_parameters(img, 3)), img)
        got = F.chi2(rows[i], img)   # the GPU mixture's chi^2, recomputed in FP64
        assert got <= 1.02 * ora_chi2 + 1e-14, (i, got, ora_chi2)
        assert got < 1e-2 * start
        assert abs(chi2[i] - got) <= 1e-3 * got + 1e-14


def test_batch_equals_single_calls(gpu_renderer):
    psfs = [p.image for p in psf_set(5, seed=32, fit=False)]
    rows, chi2 = gpu_fit(gpu_renderer, psfs, k=3)
    for i in (0, 3):
        r1, c1 = gpu_fit(gpu_renderer, [psfs[i]], k=3)
        assert np.array_equal(r1[0], rows[i]) and np.array_equal(c1[0], chi2[i])


def test_rejects_bad_arguments(gpu_renderer):
    import torch
    from paper_2012_15797_gb300 import capi
    t = torch.zeros(1, 16, 16, device="cuda")
    out = torch.zeros(1, 5, 6, device="cuda")
    with pytest.raises(capi.MogError):
        capi.mog_fit_psf_mixture(gpu_renderer.ctx, t.data_ptr(), 1, 16, 16, 5, 10, out.data_ptr())
    with pytest.raises(capi.MogError):
        capi.mog_fit_psf_mixture(gpu_renderer.ctx, t.data_ptr(), 1, 16, 16, 3, 0, out.data_ptr())
