"""The library's render of the single 64x64 galaxy against the stored
oracle values of tests/golden/single_galaxy_64.txt: sampled pixels within
the parity tolerance (2e-6 of the flux), the sum and first moments."""

import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_render_matches_the_stored_oracle_values(gpu_renderer):
    from paper_2012_15797_gb300.renderer import patches, to_device
    from workloads import single_galaxy_64
    stored = {}
    with open(os.path.join(HERE, "golden", "single_galaxy_64.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                stored[k] = float(v)
    b = to_device(single_galaxy_64())
    img = patches(gpu_renderer.render(b), b)[0].double().cpu().numpy()
    gpu_renderer.sync_status()
    for k, v in stored.items():
        if k.startswith("pixel_"):
            _, y, x = k.split("_")
            assert abs(img[int(y), int(x)] - v) <= 2e-6, k
    assert abs(img.sum() - stored["sum"]) <= 1e-5
    yy, xx = np.mgrid[0:64, 0:64]
    assert (img * xx).sum() / img.sum() == pytest.approx(stored["mean_x"], abs=1e-4)
    assert (img * yy).sum() / img.sum() == pytest.approx(stored["mean_y"], abs=1e-4)
