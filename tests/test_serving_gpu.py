"""Serving runtime: continuous batching of render + gradient requests from
several fits.  Each request's result is the same alone and in the mix
(within the gradient tolerance) and equals the direct render -> chi^2
gradient -> adjoint computation; admission by memory serialises requests
under a tiny budget without changing results."""

import numpy as np
import pytest

from workloads import mixed_galaxies

pytestmark = pytest.mark.gpu


def _fits(n_fits=3, per_fit=300, seed=61):
    fits = []
    for f in range(n_fits):
        g = mixed_galaxies(per_fit, seed=seed + f, n_psf=5)
        fits.append(g)
    return fits


def _requests(fits, n=40, seed=7):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        f = int(rng.integers(len(fits)))
        cnt = int(rng.integers(1, 65))
        first = int(rng.integers(0, len(fits[f]) - cnt + 1))
        p = fits[f].params6()[first:first + cnt].copy()
        p[:, 0] *= 1.0 + 0.05 * rng.standard_normal(cnt)
        p[:, 1:3] += 0.1 * rng.standard_normal((cnt, 2))
        p[:, 3] += 0.05 * rng.standard_normal(cnt)
        out.append((f, first, p.astype(np.float32)))
    return out


@pytest.fixture(scope="module")
def setup(gpu_renderer):
    from paper_2012_15797_gb300.serving import make_fits
    fits = _fits()
    state = make_fits(gpu_renderer, fits)
    return fits, state, _requests(fits)


def _serve(renderer, state, reqs, **cfg):
    from paper_2012_15797_gb300.serving import Server
    srv = Server(renderer, **cfg)
    for st in state:
        srv.add_fit(**st)
    tickets, keeps = srv.replay(reqs, np.zeros(len(reqs)))
    lat = srv.wait_replayed(tickets, keeps)
    stats = srv.stats()
    srv.close()
    return [(k[1].copy(), k[2].copy()) for k in keeps], lat, stats


def _direct(renderer, fits, state, req):
    """Plain API: render, residual gradient with torch, adjoint."""
    import torch
    from paper_2012_15797_gb300.renderer import to_device
    f, first, p = req
    g = fits[f].subset(np.arange(first, first + len(p))).with_params6(p.astype(np.float64))
    b = to_device(g)
    model = renderer.render(b)
    st = state[f]
    data = torch.cat([st["data"][int(st["data_offset"][first + k]):int(st["data_offset"][first + k]) + int(n) ** 2]
                      for k, n in enumerate(g.size)])
    ivar = torch.repeat_interleave(st["ivar"][first:first + len(p)],
                                   torch.from_numpy(np.asarray(g.size, np.int64) ** 2).cuda())
    r = model - data
    gp = renderer.render_backward(b, (2.0 * ivar * r).contiguous())
    chi2 = torch.stack([(ivar * r * r)[int(o):int(o) + int(n) ** 2].sum() for o, n in zip(b.offsets, g.size)])
    renderer.sync_status()
    return gp.cpu().numpy(), chi2.cpu().numpy()


def test_mix_equals_alone_equals_direct(gpu_renderer, setup):
    fits, state, reqs = setup
    mixed, lat_mix, st_mix = _serve(gpu_renderer, state, reqs, budget_bytes=1 << 30, lanes=3,
                                    max_batch_galaxies=4096)
    alone, lat_alone, st_alone = _serve(gpu_renderer, state, reqs, budget_bytes=1 << 30, lanes=1,
                                        max_batch_galaxies=0)
    assert st_alone["batches"] == len(reqs)
    assert st_mix["batches"] < len(reqs)          # requests really were batched together
    for (gm, cm), (ga, ca) in zip(mixed, alone):
        assert np.all(np.isfinite(gm)) and np.all(np.isfinite(cm))
        np.testing.assert_array_equal(gm, ga)
        np.testing.assert_array_equal(cm, ca)
    for i in (0, 7, len(reqs) - 1):
        gd, cd = _direct(gpu_renderer, fits, state, reqs[i])
        gm, cm = mixed[i]
        scale = np.abs(gd).max(axis=0, keepdims=True)
        assert np.all(np.abs(gm - gd) <= 1e-4 * np.abs(gd) + 1e-5 * scale)
        np.testing.assert_allclose(cm, cd, rtol=1e-4)
    assert np.all(lat_mix > 0) and np.all(lat_alone > 0)


def test_admission_by_memory(gpu_renderer, setup):
    """A budget that fits about one request at a time still serves them all,
    one micro-batch each, with unchanged results."""
    fits, state, reqs = setup
    reqs = reqs[:12]
    ref, _, _ = _serve(gpu_renderer, state, reqs, budget_bytes=1 << 30, lanes=1, max_batch_galaxies=0)
    out, _, st = _serve(gpu_renderer, state, reqs, budget_bytes=(4 << 20) + 128 * 64 * 64 * 4 * 64 // 8,
                        lanes=4, max_batch_galaxies=4096)
    assert st["requests"] == len(reqs)
    for (g1, c1), (g2, c2) in zip(ref, out):
        np.testing.assert_array_equal(g1, g2)
        np.testing.assert_array_equal(c1, c2)


def test_trace_rows_account_for_every_batch(gpu_renderer, setup):
    """The per micro-batch trace has one row per batch, its galaxies add up
    to the requests', its times are ordered (admission <= completion) and a
    timing reset clears it."""
    from paper_2012_15797_gb300.serving import Server
    fits, state, reqs = setup
    srv = Server(gpu_renderer, budget_bytes=1 << 30, lanes=2, max_batch_galaxies=512)
    for st in state:
        srv.add_fit(**st)
    tickets, keeps = srv.replay(reqs, np.arange(len(reqs)) * 2e-4)
    srv.wait_replayed(tickets, keeps)
    stats = srv.stats()
    tr = srv.trace()
    assert tr.shape == (stats["batches"], len(Server.TRACE_KEYS))
    col = {k: i for i, k in enumerate(Server.TRACE_KEYS)}
    assert int(tr[:, col["galaxies"]].sum()) == sum(len(q[2]) for q in reqs)
    assert np.all(tr[:, col["admit_ms"]] >= 0)
    assert np.all(tr[:, col["done_ms"]] >= tr[:, col["admit_ms"]])
    assert np.all(tr[:, col["device_ms"]] > 0)
    assert np.all(tr[:, col["launch_host_ms"]] >= 0)
    assert set(np.unique(tr[:, col["lane"]]).astype(int)) <= {0, 1}
    assert np.all((tr[:, col["lanes_busy"]] >= 1) & (tr[:, col["lanes_busy"]] <= 2))
    assert np.all(tr[:, col["backlog_galaxies"]] >= 0)
    srv.timing(reset=True)
    assert srv.trace().shape[0] == 0
    srv.close()


def test_many_small_batches_match_one_per_launch(gpu_renderer, setup):
    """Hundreds of micro-batches over four lanes (small batch limit, requests
    arriving faster than they are served, then slower): every request's
    gradients and chi2 equal the one-request-per-launch results bit for bit,
    so no lane is reused while its batch still runs."""
    fits, state, _ = setup
    reqs = _requests(fits, n=400, seed=17)
    ref, _, st_ref = _serve(gpu_renderer, state, reqs, budget_bytes=1 << 30, lanes=1, max_batch_galaxies=0)
    from paper_2012_15797_gb300.serving import Server
    srv = Server(gpu_renderer, budget_bytes=1 << 30, lanes=4, max_batch_galaxies=96)
    for st in state:
        srv.add_fit(**st)
    times = np.concatenate([np.zeros(200), 0.004 * np.arange(1, 201)])   # a burst, then one every 4 ms
    tickets, keeps = srv.replay(reqs, times)
    srv.wait_replayed(tickets, keeps)
    stats = srv.stats()
    srv.close()
    assert stats["batches"] > 150
    for (g1, c1), k in zip(ref, keeps):
        np.testing.assert_array_equal(g1, k[1])
        np.testing.assert_array_equal(c1, k[2])


def test_add_fits_while_serving(gpu_renderer, setup):
    """Fits added while micro-batches are in flight (the device fit table
    grows from 64 to 128 entries under load): the requests in flight and the
    requests on the new fits are answered, and a new fit holding the same
    state as fit 0 answers as fit 0 does."""
    from paper_2012_15797_gb300.serving import Server
    fits, state, _ = setup
    reqs = _requests(fits, n=300, seed=23)
    srv = Server(gpu_renderer, budget_bytes=1 << 30, lanes=4, max_batch_galaxies=128)
    for st in state:
        srv.add_fit(**st)
    tickets, keeps = srv.replay(reqs, 0.002 * np.arange(len(reqs)))
    ids = [srv.add_fit(**state[0]) for _ in range(100)]
    srv.wait_replayed(tickets, keeps)
    assert ids == list(range(len(state), len(state) + 100))
    p = _requests(fits, n=1, seed=29)[0][2]
    first = 0
    while len(p) > len(fits[0]) - first:
        p = p[:-1]
    g0, c0, _ = srv.wait(srv.submit(0, first, p))
    g1, c1, _ = srv.wait(srv.submit(ids[-1], first, p))
    srv.close()
    np.testing.assert_array_equal(g0, g1)
    np.testing.assert_array_equal(c0, c1)
    assert all(np.all(np.isfinite(k[1])) for k in keeps)
