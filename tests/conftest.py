import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def tables():
    from workloads import load_profile_tables
    return load_profile_tables()


@pytest.fixture(scope="session")
def psf0():
    from workloads import single_psf
    return single_psf()


@pytest.fixture(scope="session")
def gpu_renderer(tables, psf0):
    """A library context with the profile tables, PSF 0 = the 2-Gaussian
    PSF and PSFs 1..4 = Moffat-winged PSFs."""
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
