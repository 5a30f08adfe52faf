"""Pins of the composite-galaxy oracle: the combination is linear, so it must
reduce to the single-profile method exactly where one part vanishes or both
parts are the same profile."""

import numpy as np

from oracle import composite as C
from oracle import lanczos as L
from oracle import render as R
from workloads import composite_galaxies


def _pair(i=3):
    d, b = composite_galaxies(8, seed=71)
    return d.row(i), b.row(i)


def test_vanishing_bulge_is_the_disk(tables, psf0):
    d, b = _pair()
    b["flux"] = 0.0
    got = C.render_composite(d, b, psf0.image, psf0.mog, tables)
    assert np.array_equal(got, R.render(d, psf0.image, psf0.mog, tables) + 0.0 * got)


def test_two_equal_parts_add_their_fluxes(tables, psf0):
    d, _ = _pair()
    half = dict(d, flux=0.5 * d["flux"])
    got = C.render_composite(half, dict(half), psf0.image, psf0.mog, tables)
    want = R.render(d, psf0.image, psf0.mog, tables)
    assert np.max(np.abs(got - want)) < 1e-12 * d["flux"]


def test_lanczos_composite_is_the_shift_of_the_phase_parts_at_integer_offsets(tables, psf0):
    d, b = _pair(5)
    for x, y in ((0.0, 0.0), (2.0, -1.0)):
        dd, bb = dict(d, x=x, y=y), dict(b, x=x, y=y)
        a = C.render_composite(dd, bb, psf0.image, psf0.mog, tables, shift="lanczos")
        p = C.render_composite(dd, bb, psf0.image, psf0.mog, tables)
        assert np.array_equal(a, p)
    got = C.render_composite(d, b, psf0.image, psf0.mog, tables, shift="lanczos")
    want = (L.render_lanczos(d, psf0.image, psf0.mog, tables) + L.render_lanczos(b, psf0.image, psf0.mog, tables))
    assert np.max(np.abs(got - want)) < 1e-12 * (d["flux"] + b["flux"])


def test_generator_shares_layout(tables):
    d, b = composite_galaxies(50, seed=72)
    for f in ("x", "y", "psf", "size"):
        assert np.array_equal(getattr(d, f), getattr(b, f))
    assert np.all(np.exp(b.log_re) < np.exp(d.log_re)) and np.all(b.profile == 1) and np.all(d.profile == 0)
