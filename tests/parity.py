"""Shared parity helpers: GPU render through the C-ABI vs the FP64 oracle."""

import numpy as np

from oracle import render as R

PIX_TOL = 2e-6    # max |d pixel| <= PIX_TOL * flux
FLUX_TOL = 1e-5   # |d sum| <= FLUX_TOL * flux


def oracle_patches(gals, psfs, tables, idx=None):
    idx = range(len(gals)) if idx is None else idx
    cache = {}
    out = []
    for i in idx:
        g = gals.row(i)
        key = (g["psf"], g["size"])
        if key not in cache:
            cache[key] = R.psf_spectrum(psfs[g["psf"]].image, g["size"])
        out.append(R.render(g, None, psfs[g["psf"]].mog, tables, psf_hat=cache[key]))
    return out


def gpu_patches(renderer, gals):
    import torch
    from paper_2012_15797_gb300.renderer import patches, to_device
    b = to_device(gals)
    out = torch.full((b.total,), float("nan"), dtype=torch.float32, device="cuda")
    renderer.render(b, out)
    renderer.sync_status()
    return [p.double().cpu().numpy() for p in patches(out, b)], out, b


def check_parity(gpu, ora, gals, idx=None):
    """Element-wise parity; returns the worst (pixel, flux) relative errors."""
    idx = range(len(gals)) if idx is None else idx
    worst_p = worst_f = 0.0
    for k, i in enumerate(idx):
        flux = float(gals.flux[i])
        g, o = gpu[k], ora[k]
        assert g.shape == o.shape
        assert np.all(np.isfinite(g)), f"galaxy {i}: non-finite output"
        dp = np.max(np.abs(g - o)) / flux
        df = abs(g.sum() - o.sum()) / flux
        worst_p, worst_f = max(worst_p, dp), max(worst_f, df)
        assert dp <= PIX_TOL, f"galaxy {i} {gals.row(i)}: max|dpix|/flux = {dp:.3e}"
        assert df <= FLUX_TOL, f"galaxy {i} {gals.row(i)}: |dflux|/flux = {df:.3e}"
    return worst_p, worst_f
