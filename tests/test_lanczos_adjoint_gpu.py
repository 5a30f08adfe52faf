"""GPU adjoint of the Lanczos sub-pixel-shift variant (mog_render_backward_ex
with MOG_GRAD_LANCZOS) against the FP64 oracle's vector-Jacobian product of
the Lanczos model (itself pinned by central differences), at every patch
side, with the adjoint's tolerance: |d g_k| <= 1e-4 |g_k| +
1e-5 ||dL/dpix||_1 s_k (s_k = 1 for flux, flux otherwise)."""

import numpy as np
import pytest

from oracle import lanczos as L
from oracle import render as R
from test_adjoint_gpu import _gals, _random_grad, _row, check
from workloads import mixed_galaxies

pytestmark = pytest.mark.gpu

EDGE = [
    dict(), dict(e1=0.5, e2=-0.3, x=0.49, y=-0.49), dict(flux=1e4, x=2.3, y=-1.7), dict(log_re=np.log(0.4), x=-0.05),
    dict(log_re=np.log(12.0), profile=1, sersic_n=4.0, x=0.21), dict(log_re=np.log(20.0), y=0.37),
    dict(profile=2, sersic_n=2.6, psf=2, x=-0.33, y=0.12), dict(x=1.0, y=-2.0),
]


def gpu_grads_lanczos(renderer, gals, grad_pix, sersic=False):
    import torch
    from paper_2012_15797_gb300.renderer import to_device
    b = to_device(gals)
    go = torch.from_numpy(np.concatenate([g.ravel() for g in grad_pix]).astype(np.float32)).cuda()
    gp = torch.full((len(gals), 7 if sersic else 6), float("nan"), device="cuda")
    renderer.render_backward(b, go, gp, sersic=sersic, shift="lanczos")
    renderer.sync_status()
    return gp.double().cpu().numpy()


def oracle_grads_lanczos(gals, psfs, tables, grad_pix):
    out = []
    for i in range(len(gals)):
        g = gals.row(i)
        ph = R.psf_spectrum(psfs[g["psf"]].image, g["size"])
        out.append(L.vjp_lanczos(g, ph, psfs[g["psf"]].mog, tables, grad_pix[i]))
    return np.array(out)


@pytest.mark.parametrize("size", [32, 64, 128, 256])
def test_lanczos_adjoint_every_side(gpu_renderer, tables, size):
    gals = _gals([_row(size=size, **e) for e in EDGE])
    gp = _random_grad(gals, 300 + size)
    check(gpu_grads_lanczos(gpu_renderer, gals, gp), oracle_grads_lanczos(gals, gpu_renderer.psfs, tables, gp),
          gals, gp)


def test_lanczos_adjoint_mixed_batch(gpu_renderer, tables):
    gals = mixed_galaxies(160, seed=301, n_psf=5)
    gp = _random_grad(gals, 302)
    gpu = gpu_grads_lanczos(gpu_renderer, gals, gp)
    idx = [int(i) for n in (32, 64, 128, 256) for i in np.flatnonzero(gals.size == n)[:3]]
    sub = gals.subset(np.array(idx))
    ora = oracle_grads_lanczos(sub, gpu_renderer.psfs, tables, [gp[i] for i in idx])
    check(gpu[idx], ora, sub, [gp[i] for i in idx])


def test_lanczos_adjoint_sersic_gradient(gpu_renderer, tables):
    gals = _gals([_row(size=64, profile=2, sersic_n=n, x=0.3, y=-0.2) for n in (1.3, 2.6, 4.4)])
    gp = _random_grad(gals, 303)
    gpu = gpu_grads_lanczos(gpu_renderer, gals, gp, sersic=True)
    for i in range(len(gals)):
        g = gals.row(i)
        ph = R.psf_spectrum(gpu_renderer.psfs[0].image, 64)
        dn = float(np.sum(L.sersic_derivative_lanczos(g, ph, gpu_renderer.psfs[0].mog, tables) * gp[i]))
        tol = 1e-4 * abs(dn) + 1e-5 * np.abs(gp[i]).sum() * float(gals.flux[i])
        assert abs(gpu[i, 6] - dn) <= tol, (i, gpu[i, 6], dn)
    check(gpu[:, :6], oracle_grads_lanczos(gals, gpu_renderer.psfs, tables, gp), gals, gp)


def test_lanczos_adjoint_at_integer_offsets_is_the_phase_adjoint(gpu_renderer):
    # at integer offsets the weights are the identity: every gradient but x
    # and y equals the plain adjoint's (to rounding: the upstream patch went
    # through the transposed convolution with weights 0 and 1)
    import torch
    from paper_2012_15797_gb300.renderer import to_device
    gals = mixed_galaxies(200, seed=304, n_psf=5)
    gals.x[:] = np.round(gals.x * 4)
    gals.y[:] = np.round(gals.y * 4)
    b = to_device(gals)
    go = torch.randn(b.total, device="cuda")
    lz = gpu_renderer.render_backward(b, go, shift="lanczos")
    ph = gpu_renderer.render_backward(b, go)
    gpu_renderer.sync_status()
    cols = [0, 3, 4, 5]
    torch.testing.assert_close(lz[:, cols], ph[:, cols], rtol=1e-5, atol=1e-6 * float(go.abs().max()))
