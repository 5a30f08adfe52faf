"""Failure detection without a GPU fault: the serving runtime's failure
paths driven by host-side injection (a dropped completion, a failing launch,
a failing allocation, malformed requests and fits, unknown and repeated
tickets) and a bounded device wait made to run out.  Every failure surfaces
as a status within its limit, and the server and context keep working."""

import numpy as np
import pytest

from workloads import mixed_galaxies

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def served(gpu_renderer):
    from paper_2012_15797_gb300.serving import make_fits
    fits = [mixed_galaxies(200, seed=81 + f, n_psf=5) for f in range(2)]
    return fits, make_fits(gpu_renderer, fits)


def _server(renderer, state, **cfg):
    from paper_2012_15797_gb300.serving import Server
    srv = Server(renderer, **({"budget_bytes": 1 << 30, "lanes": 2, "max_batch_galaxies": 0} | cfg))
    for st in state:
        srv.add_fit(**st)
    return srv


def _params(fits, f, first, count):
    return fits[f].params6()[first:first + count].astype(np.float32)


def _reference(renderer, state, fits):
    """Each fit's first 8 galaxies served once without faults."""
    srv = _server(renderer, state)
    try:
        out = [srv.wait(srv.submit(f, 0, _params(fits, f, 0, 8)))[0].copy() for f in range(2)]
    finally:
        srv.close()
    return out


def test_dropped_completion_times_out_and_server_continues(gpu_renderer, served):
    from paper_2012_15797_gb300 import capi
    fits, state = served
    ref = _reference(gpu_renderer, state, fits)
    srv = _server(gpu_renderer, state)
    try:
        srv.inject_fault(capi.MOG_FAULT_DROP, 2)
        t1 = srv.submit(0, 0, _params(fits, 0, 0, 8))
        g1 = srv.wait(t1)[0].copy()
        t2 = srv.submit(1, 0, _params(fits, 1, 0, 8))   # the second admitted: its completion is lost
        with pytest.raises(capi.MogError) as ei:
            srv.wait(t2, timeout=0.5)
        assert ei.value.status == capi.MOG_ERR_TIMEOUT
        t3 = srv.submit(1, 0, _params(fits, 1, 0, 8))
        g3 = srv.wait(t3)[0].copy()
        np.testing.assert_array_equal(g1, ref[0])
        np.testing.assert_array_equal(g3, ref[1])
    finally:
        srv.close()


@pytest.mark.parametrize("kind,status", [("LAUNCH", "MOG_ERR_CUDA"), ("NOMEM", "MOG_ERR_NOMEM")])
def test_failed_batch_reports_status_and_server_continues(gpu_renderer, served, kind, status):
    from paper_2012_15797_gb300 import capi
    fits, state = served
    ref = _reference(gpu_renderer, state, fits)
    srv = _server(gpu_renderer, state)
    try:
        srv.inject_fault(getattr(capi, f"MOG_FAULT_{kind}"), 1)
        t1 = srv.submit(0, 0, _params(fits, 0, 0, 8))
        with pytest.raises(capi.MogError) as ei:
            srv.wait(t1, timeout=10.0)
        assert ei.value.status == getattr(capi, status)
        t2 = srv.submit(1, 0, _params(fits, 1, 0, 8))
        np.testing.assert_array_equal(srv.wait(t2)[0], ref[1])
        assert srv.stats()["pending"] == 0
    finally:
        srv.close()


def test_unknown_and_repeated_tickets_are_rejected(gpu_renderer, served):
    from paper_2012_15797_gb300 import capi
    fits, state = served
    srv = _server(gpu_renderer, state)
    try:
        t = srv.submit(0, 0, _params(fits, 0, 0, 4))
        srv.wait(t)
        for bad in (t, t + 1000):   # already collected; never issued
            st = capi.library().mog_server_wait(srv.handle, bad, 0.1, None)
            assert st == capi.MOG_ERR_ARG
    finally:
        srv.close()


@pytest.mark.parametrize("field,value", [("flux", np.nan), ("x", np.inf), ("e1", 0.9), ("log_re", 40.0)])
def test_malformed_request_rejected_at_submission(gpu_renderer, served, field, value):
    from paper_2012_15797_gb300 import capi
    fits, state = served
    srv = _server(gpu_renderer, state)
    try:
        p = _params(fits, 0, 0, 4)
        col = {"flux": 0, "x": 1, "y": 2, "log_re": 3, "e1": 4, "e2": 5}[field]
        p[2, col] = value
        if field == "e1":
            p[2, 5] = 0.9
        with pytest.raises(capi.MogError) as ei:
            srv.submit(0, 0, p)
        assert ei.value.status == capi.MOG_ERR_ARG
        with pytest.raises(capi.MogError):
            srv.submit(0, 195, _params(fits, 0, 0, 10))   # beyond the fit's 200 galaxies
        with pytest.raises(capi.MogError):
            srv.submit(7, 0, _params(fits, 0, 0, 2))      # no such fit
        assert srv.stats()["pending"] == 0
        t = srv.submit(0, 0, _params(fits, 0, 0, 4))      # still serving
        assert np.all(np.isfinite(srv.wait(t)[0]))
    finally:
        srv.close()


@pytest.mark.parametrize("field,value", [("size", 48), ("psf", 1000), ("psf", -1), ("profile", 7), ("sersic_n", np.nan),
                                         ("data_offset", 2)])
def test_malformed_fit_rejected(gpu_renderer, served, field, value):
    from paper_2012_15797_gb300 import capi
    from paper_2012_15797_gb300.serving import Server
    _, state = served
    st = dict(state[0])
    t = st[field].clone()
    t[3] = value
    st[field] = t
    srv = Server(gpu_renderer, budget_bytes=1 << 30, lanes=1, max_batch_galaxies=0)
    try:
        with pytest.raises(capi.MogError) as ei:
            srv.add_fit(**st)
        assert ei.value.status == capi.MOG_ERR_ARG
    finally:
        srv.close()


def test_bounded_device_wait_runs_out_and_context_stays_usable(gpu_renderer):
    import time
    import torch
    from paper_2012_15797_gb300 import capi
    from paper_2012_15797_gb300.renderer import to_device
    from workloads import fixed_galaxies_64
    gpu_renderer.sync_status()
    t0 = time.perf_counter()
    capi.mog_check_wait_timeout(gpu_renderer.ctx, 0.05, torch.cuda.current_stream().cuda_stream)
    with pytest.raises(capi.MogError) as ei:
        gpu_renderer.sync_status()
    elapsed = time.perf_counter() - t0
    assert ei.value.status == capi.MOG_ERR_TIMEOUT
    assert 0.04 <= elapsed < 5.0
    gpu_renderer.sync_status()   # the status word was cleared
    b = to_device(fixed_galaxies_64(50, seed=83))
    out = gpu_renderer.render(b)
    gpu_renderer.sync_status()
    assert torch.isfinite(out).all()
    with pytest.raises(capi.MogError):
        capi.mog_check_wait_timeout(gpu_renderer.ctx, 5.0)
