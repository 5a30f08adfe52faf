"""GPU gradient w.r.t. the Sersic index (mog_render_backward_ex with
MOG_GRAD_SERSIC) against the FP64 oracle's analytic derivative, with the
adjoint tests' tolerance: |d g_k| <= 1e-4 |g_k| + 1e-5 ||dL/dpix||_1 s_k
(s = 1 for flux, s = flux otherwise, the Sersic index included)."""

import numpy as np
import pytest

from oracle import adjoint as A
from oracle import render as R
from workloads import Galaxies, single_galaxy_64, mixed_galaxies, PROFILE_DEV, PROFILE_EXP, PROFILE_SERSIC

pytestmark = pytest.mark.gpu


def _gals(rows):
    f = {k: np.array([r[k] for r in rows]).astype(np.float32) for k in Galaxies.FLOAT_FIELDS}
    i = {k: np.array([r[k] for r in rows]).astype(np.int32) for k in Galaxies.INT_FIELDS}
    return Galaxies(**f, **i)


def _row(**kw):
    r = single_galaxy_64().row(0)
    r.update(profile=PROFILE_SERSIC, e1=0.2, e2=-0.15)
    r.update(kw)
    return r


def gpu_grads(renderer, gals, grad_pix, sersic=True):
    import torch
    from paper_2012_15797_gb300.renderer import to_device
    b = to_device(gals)
    go = torch.from_numpy(np.concatenate([g.ravel() for g in grad_pix]).astype(np.float32)).cuda()
    gp = renderer.render_backward(b, go, sersic=sersic)
    renderer.sync_status()
    return gp.double().cpu().numpy()


def check(gpu, gals, psfs, tables, grad_pix):
    for i in range(len(gals)):
        g = gals.row(i)
        p = psfs[g["psf"]]
        ph = R.psf_spectrum(p.image, g["size"])
        ora = np.append(A.vjp(g, ph, p.mog, tables, grad_pix[i]),
                        np.sum(A.sersic_derivative(g, ph, p.mog, tables) * grad_pix[i]))
        flux = float(gals.flux[i])
        scale = np.array([1.0] + [flux] * 6) * np.abs(grad_pix[i]).sum()
        err = np.abs(gpu[i] - ora)
        assert np.all(err <= 1e-4 * np.abs(ora) + 1e-5 * scale), (i, g, gpu[i], ora, err)


CASES = [dict(sersic_n=2.6), dict(sersic_n=4.375, log_re=np.log(7.0)), dict(sersic_n=1.13, log_re=np.log(14.0)),
         dict(sersic_n=5.3, log_re=np.log(0.6), x=0.45, y=-0.3), dict(sersic_n=0.8, log_re=np.log(2.0), psf=2),
         dict(sersic_n=3.1, log_re=np.log(20.0), e1=-0.4, e2=0.3)]


@pytest.mark.parametrize("size", [32, 64, 128, 256])
def test_sersic_gradient_each_size(gpu_renderer, tables, size):
    gals = _gals([_row(size=size, **c) for c in CASES])
    rng = np.random.default_rng(101 + size)
    grad = [rng.normal(size=(size, size)) for _ in range(len(gals))]
    check(gpu_grads(gpu_renderer, gals, grad), gals, gpu_renderer.psfs, tables, grad)


def test_sersic_gradient_mixed_batch(gpu_renderer, tables):
    gals = mixed_galaxies(60, seed=102, n_psf=5)
    rng = np.random.default_rng(103)
    grad = [rng.normal(size=(int(n), int(n))) for n in gals.size]
    check(gpu_grads(gpu_renderer, gals, grad), gals, gpu_renderer.psfs, tables, grad)


def test_first_six_equal_the_plain_adjoint_and_fixed_profiles_give_zero(gpu_renderer):
    rows = [_row(size=s, **c) for s in (32, 64, 128, 256) for c in CASES[:3]]
    rows += [_row(size=64, profile=PROFILE_EXP, sersic_n=1.0), _row(size=64, profile=PROFILE_DEV, sersic_n=4.0),
             _row(size=64, sersic_n=7.5)]   # outside the table's nodes
    gals = _gals(rows)
    rng = np.random.default_rng(104)
    grad = [rng.normal(size=(int(n), int(n))) for n in gals.size]
    a = gpu_grads(gpu_renderer, gals, grad, sersic=True)
    b = gpu_grads(gpu_renderer, gals, grad, sersic=False)
    assert np.array_equal(a[:, :6], b)
    assert np.all(a[-3:, 6] == 0.0)
