"""Batching feature: the autotuner's launch shapes and the captured CUDA
graph give exactly the eager default render (each galaxy is computed the
same way whichever CTA takes it)."""

import numpy as np
import pytest

from workloads import fixed_galaxies_64, mixed_galaxies

pytestmark = pytest.mark.gpu


def test_autotune_keeps_results(tables, psf0):
    # the launch shape does not change a galaxy's result; the radix schedule
    # changes its rounding only (each schedule is at oracle parity,
    # test_schedules_gpu.py), so the tuned render equals the default one to
    # the parity tolerance, and equals itself bit for bit call after call
    import torch
    from paper_2012_15797_gb300.renderer import Renderer, to_device
    from parity import PIX_TOL
    from workloads import psf_set
    r = Renderer(tables, [psf0] + psf_set(4))
    try:
        gals = mixed_galaxies(4000, seed=51, n_psf=5)
        b = to_device(gals)
        ref = r.render(b)
        out = torch.empty_like(ref)
        shapes = r.autotune(b, out, reps=1)
        assert isinstance(shapes.pop("serial"), bool)
        assert set(n for d, n in shapes) == {32, 64, 128, 256}
        for (d, n), (c, ch, sc) in shapes.items():
            assert c >= 1 and ch in (1, 2, 4, 8, 16, 32) and sc in (range(3) if n in (64, 128) else (0, 1))
        again = r.render(b)
        r.sync_status()
        flux = torch.from_numpy(np.repeat(gals.flux.astype(np.float64), b.sizes.astype(np.int64) ** 2)).cuda()
        assert torch.all((again.double() - ref.double()).abs() <= PIX_TOL * flux)
        assert torch.equal(r.render(b), again)
    finally:
        r.close()


def test_autotune_adjoint(gpu_renderer):
    import torch
    from paper_2012_15797_gb300.renderer import to_device
    gals = fixed_galaxies_64(3000, seed=52)
    b = to_device(gals)
    go = torch.randn(b.total, device="cuda")
    ref = gpu_renderer.render_backward(b, go)
    out = torch.empty(b.total, device="cuda")
    gp = torch.empty_like(ref)
    shapes = gpu_renderer.autotune(b, out, go, gp, reps=1)
    assert ("bwd", 64) in shapes and ("fwd", 64) in shapes
    assert shapes[("bwd", 64)][2] == 0
    again = gpu_renderer.render_backward(b, go)
    gpu_renderer.sync_status()
    assert torch.equal(again, ref)


def test_graph_launch_matches_eager_and_sees_new_inputs(gpu_renderer):
    import torch
    from paper_2012_15797_gb300.renderer import to_device
    gals = mixed_galaxies(3000, seed=53, n_psf=5)
    b = to_device(gals)
    ref = gpu_renderer.render(b)
    out = torch.full_like(ref, float("nan"))
    g = gpu_renderer.graph(b, out)
    out.fill_(float("nan"))
    g.launch()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    # new contents of the same buffers are picked up by the next launch
    b.tensors["flux"].mul_(2.0)
    g.launch()
    ref2 = gpu_renderer.render(b)
    gpu_renderer.sync_status()
    assert torch.equal(out, ref2)
    assert torch.allclose(ref2, 2.0 * ref, rtol=1e-5, atol=1e-6)
    g.close()


def test_full_mixed_200k_graph_sampled(tables):
    """The benchmark's mixed-size launch at full size: 200k galaxies (Sersic n
    0.5-6, N = 32..256) with 64 Moffat-winged PSFs, launch shapes from the
    autotuner, one CUDA-graph launch; every pixel written, and 32 sampled
    patches (eight per patch side) within the method's tolerance of the FP64
    oracle."""
    import torch
    from parity import check_parity, oracle_patches
    from paper_2012_15797_gb300.renderer import Renderer, to_device
    from workloads import psf_set
    psfs = psf_set(64)
    r = Renderer(tables, psfs)
    try:
        gals = mixed_galaxies()
        b = to_device(gals)
        out = torch.empty(b.total, dtype=torch.float32, device="cuda")
        r.autotune(b, out, reps=1)
        g = r.graph(b, out)
        out.fill_(float("nan"))
        g.launch()
        torch.cuda.synchronize()
        r.sync_status()
        g.close()
        assert not torch.isnan(out).any()
        rng = np.random.default_rng(7)
        idx = np.sort(np.concatenate([rng.choice(np.flatnonzero(gals.size == n), 8, replace=False)
                                      for n in (32, 64, 128, 256)]))
        gpu = []
        for i in idx:
            n, o = int(b.sizes[i]), int(b.offsets[i])
            gpu.append(out[o:o + n * n].view(n, n).double().cpu().numpy())
        check_parity(gpu, oracle_patches(gals, psfs, tables, idx), gals, idx)
    finally:
        r.close()
