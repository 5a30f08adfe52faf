"""FP64 oracle of composite (bulge + disk) galaxies: Section 1 names the
linear combination of an n = 1 and an n = 4 profile with one centre; the
method is linear in the model, so the composite's image is the sum of the
two profiles' images (Steps 1-8 for each), and with the Lanczos variant the
shift of the sum.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).
"""

from .lanczos import lanczos_shift, split_offset
from .render import render


def render_composite(disk, bulge, psf_image, psf_mog, tables, shift="phase", psf_hat=None):
    """``disk`` and ``bulge`` are galaxy dicts with the same x, y, psf and
    size; returns the composite's patch."""
    assert (disk["x"], disk["y"], disk["size"]) == (bulge["x"], bulge["y"], bulge["size"])
    if shift == "phase":
        return (render(disk, psf_image, psf_mog, tables, psf_hat=psf_hat)
                + render(bulge, psf_image, psf_mog, tables, psf_hat=psf_hat))
    nx, dx = split_offset(disk["x"])
    ny, dy = split_offset(disk["y"])
    d, b = dict(disk, x=nx, y=ny), dict(bulge, x=nx, y=ny)
    both = render(d, psf_image, psf_mog, tables, psf_hat=psf_hat) + render(b, psf_image, psf_mog, tables, psf_hat=psf_hat)
    return lanczos_shift(both, dx, dy)
