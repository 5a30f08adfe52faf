"""Writes tests/golden/single_galaxy_64.txt: the oracle's rendering of the
single 64 x 64 exponential galaxy (r_e = 3 px, e = (0.2, -0.1), flux 1,
offset (0.3, -0.2), PSF 0.8 N(1.5) + 0.2 N(3.0) with its 3-Gaussian fit):
Section 2, Steps 1-8, and the gradients of sum(patch) and of a fixed
weighted sum of the patch with respect to (flux, x, y, log r_e, e1, e2)
(the analytic derivatives of Eq. onegaussian and of the real-space terms).

Calls only oracle/ (inputs from the seeded generators in workloads/).  The
paper prints no worked example with numbers, so this fixture pins the
oracle against itself over time (a regression fixture), not against the
paper; the pins against the paper and the mathematics are the CPU tests
test_oracle_*.py.

    python tests/golden/make_golden.py
"""

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import adjoint as A  # noqa: E402
from oracle import render as R  # noqa: E402
from workloads import load_profile_tables, single_galaxy_64, single_psf  # noqa: E402

OUT = os.path.join(HERE, "single_galaxy_64.txt")
SAMPLE = [(32, 32), (32, 33), (30, 35), (0, 0), (63, 63), (10, 50), (45, 20), (31, 40)]   # (y, x)


def weights(n=64):
    """A fixed, non-symmetric weighting of the patch (the upstream gradient
    of the second VJP)."""
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    return np.cos(0.1 * x) + 0.5 * np.sin(0.07 * y + 0.3) + 0.01 * x


def compute():
    tables = load_profile_tables()
    psf = single_psf()
    g = single_galaxy_64().row(0)
    img = R.render(g, psf.image, psf.mog, tables)
    hat = R.psf_spectrum(psf.image, 64)
    vjp_sum = A.vjp(g, hat, psf.mog, tables, np.ones((64, 64)))
    vjp_w = A.vjp(g, hat, psf.mog, tables, weights())
    yy, xx = np.mgrid[0:64, 0:64].astype(np.float64)
    tot = img.sum()
    mx, my = (img * xx).sum() / tot, (img * yy).sum() / tot
    return {
        "sum": tot, "peak": img.max(), "peak_index": int(np.argmax(img)),
        "mean_x": mx, "mean_y": my,
        "var_x": (img * (xx - mx) ** 2).sum() / tot, "var_y": (img * (yy - my) ** 2).sum() / tot,
        "cov_xy": (img * (xx - mx) * (yy - my)).sum() / tot,
        **{f"pixel_{y}_{x}": img[y, x] for y, x in SAMPLE},
        **{f"grad_sum_{k}": v for k, v in zip(("flux", "x", "y", "log_re", "e1", "e2"), vjp_sum)},
        **{f"grad_weighted_{k}": v for k, v in zip(("flux", "x", "y", "log_re", "e1", "e2"), vjp_w)},
    }


def main():
    vals = compute()
    with open(OUT, "w") as f:
        f.write("# The oracle's single 64x64 galaxy (Section 2, Steps 1-8) and gradients of its\n")
        f.write("# patch sums; written by tests/golden/make_golden.py (oracle only).  name value\n")
        for k, v in vals.items():
            f.write(f"{k} {float(v):.17g}\n")


if __name__ == "__main__":
    main()
