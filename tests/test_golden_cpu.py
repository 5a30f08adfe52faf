"""tests/golden/single_galaxy_64.txt: the oracle still reproduces its stored
rendering and gradients of the single 64x64 galaxy (a regression fixture
written by tests/golden/make_golden.py from the oracle alone), and the
stored values satisfy what the mathematics fixes independently of any
code: the flux is kept (sum = flux, the PSF being normalised), the first
moments are the patch centre plus the offset (a centred symmetric PSF and
an elliptical profile: Eq. onegaussian's phase is the only shift), and the
patch sum depends on the flux alone (its gradient w.r.t. position and shape
vanishes, w.r.t. flux equals the sum over the flux)."""

import os
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))


def _stored():
    vals = {}
    with open(os.path.join(HERE, "golden", "single_galaxy_64.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split()
            vals[k] = float(v)
    return vals


def test_stored_values_satisfy_the_invariants():
    v = _stored()
    assert v["sum"] == pytest.approx(1.0, abs=1e-7)                 # flux 1, normalised PSF
    assert v["mean_x"] == pytest.approx(32 + 0.3, abs=1e-6)         # centre N/2 + offset
    assert v["mean_y"] == pytest.approx(32 - 0.2, abs=1e-6)
    assert v["grad_sum_flux"] == pytest.approx(v["sum"], rel=1e-12)  # sum is linear in flux (flux = 1)
    for k in ("x", "y", "log_re", "e1", "e2"):
        assert abs(v[f"grad_sum_{k}"]) < 1e-12
    assert v["var_x"] > 3.6 and v["var_y"] > 3.6                    # wider than the PSF alone (0.8 1.5^2 + 0.2 3^2)
    assert v["pixel_32_32"] == v["peak"]


def test_oracle_reproduces_the_fixture():
    import make_golden
    now = make_golden.compute()
    stored = _stored()
    assert set(now) == set(stored)
    for k, want in stored.items():
        assert float(now[k]) == pytest.approx(want, rel=1e-10, abs=1e-15), k
