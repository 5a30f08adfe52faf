"""Python handle of the library's serving runtime (continuous batching of
render + gradient requests from many fits).  Marshalling only: scheduling,
admission, batching and all device work run in the library (server.cu)."""

import ctypes

import numpy as np
import torch

from . import capi


class Server:
    def __init__(self, renderer, budget_bytes=16 << 30, lanes=4, max_batch_galaxies=32768):
        self.renderer = renderer
        cfg = capi.mog_server_config(int(budget_bytes), int(lanes), int(max_batch_galaxies))
        h = ctypes.c_void_p()
        capi._check(renderer.ctx, capi.library().mog_server_create(renderer.ctx, ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h
        self._fits = []       # keep device tensors alive
        self._live = {}       # ticket -> (params, grads, chi2)

    def add_fit(self, sersic_n, profile, psf, size, data_offset, data, ivar, _keep=None):
        """Device tensors of one fit: float32 sersic_n, int32 profile, psf,
        size, int64 data_offset, float32 data (packed patches), float32 ivar."""
        t = dict(sersic_n=sersic_n, profile=profile, psf=psf, size=size, data_offset=data_offset, data=data, ivar=ivar)
        for k, v in t.items():
            assert v.is_cuda and v.is_contiguous(), k
        fs = capi.mog_fit_state(int(size.numel()), *(t[k].data_ptr() for k in
                                                     ("sersic_n", "profile", "psf", "size", "data_offset", "data",
                                                      "ivar")))
        fid = ctypes.c_int(-1)
        capi._check(self.renderer.ctx, capi.library().mog_server_add_fit(self.handle, ctypes.byref(fs), ctypes.byref(fid)))
        self._fits.append((t, _keep))
        return fid.value

    def _request(self, fit, first, params):
        params = np.ascontiguousarray(params, dtype=np.float32).reshape(-1, 6)
        grads = np.full(params.shape, np.nan, dtype=np.float32)
        chi2 = np.full(params.shape[0], np.nan, dtype=np.float32)
        req = capi.mog_request(int(fit), int(first), int(params.shape[0]), params.ctypes.data, grads.ctypes.data,
                               chi2.ctypes.data)
        return req, (params, grads, chi2)

    def submit(self, fit, first, params):
        req, keep = self._request(fit, first, params)
        t = ctypes.c_uint64()
        capi._check(self.renderer.ctx, capi.library().mog_server_submit(self.handle, ctypes.byref(req), ctypes.byref(t)))
        self._live[t.value] = keep
        return t.value

    def wait(self, ticket, timeout=60.0):
        """Returns (grads (count, 6), chi2 (count,), latency seconds)."""
        lat = ctypes.c_double()
        st = capi.library().mog_server_wait(self.handle, ctypes.c_uint64(ticket), float(timeout), ctypes.byref(lat))
        # a request that timed out is still the server's: keep its buffers
        keep = self._live.get(ticket) if st == capi.MOG_ERR_TIMEOUT else self._live.pop(ticket, None)
        capi._check(self.renderer.ctx, st)
        return keep[1], keep[2], lat.value

    def inject_fault(self, kind, nth):
        """Arms a host-side fault (capi.MOG_FAULT_DROP / _LAUNCH / _NOMEM) for
        the nth request admitted or micro-batch launched from now on."""
        capi._check(self.renderer.ctx, capi.library().mog_server_inject_fault(self.handle, int(kind), int(nth)))

    def replay(self, requests, arrival_s):
        """requests: list of (fit, first, params (count, 6)); submitted by a
        library thread at arrival_s[i] seconds from now.  Returns the ticket
        array (filled as requests are submitted) and the kept buffers."""
        n = len(requests)
        arr = (capi.mog_request * n)()
        keeps = []
        for i, (fit, first, params) in enumerate(requests):
            arr[i], keep = self._request(fit, first, params)
            keeps.append(keep)
        times = np.ascontiguousarray(arrival_s, dtype=np.float64)
        tickets = np.zeros(n, dtype=np.uint64)
        capi._check(self.renderer.ctx, capi.library().mog_server_replay(
            self.handle, arr, times.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n,
            tickets.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
        self._replay_keep = (arr, times, tickets, keeps)
        return tickets, keeps

    def replay_join(self):
        capi._check(self.renderer.ctx, capi.library().mog_server_replay_join(self.handle))

    def wait_replayed(self, tickets, keeps, timeout=120.0):
        """Waits for every replayed request; returns their latencies."""
        self.replay_join()
        lat = np.zeros(len(tickets))
        for i, t in enumerate(tickets):
            if int(t) == 0:
                raise RuntimeError(f"replayed request {i} was not submitted")
            l = ctypes.c_double()
            capi._check(self.renderer.ctx, capi.library().mog_server_wait(self.handle, ctypes.c_uint64(int(t)),
                                                                           float(timeout), ctypes.byref(l)))
            lat[i] = l.value
        return lat

    def stats(self):
        out = (ctypes.c_int64 * 6)()
        capi._check(self.renderer.ctx, capi.library().mog_server_stats(self.handle, out))
        keys = ("requests", "galaxies", "batches", "max_batch_galaxies", "max_lanes_in_flight", "pending")
        return dict(zip(keys, list(out)))

    def timing(self, reset=False):
        """(p50, p99, max) in ms of micro-batch launch (host) and device
        times and of request queue wait and service times."""
        out = (ctypes.c_double * 12)()
        capi._check(self.renderer.ctx, capi.library().mog_server_timing(self.handle, out, 1 if reset else 0))
        keys = ("launch_host", "device", "queue_wait", "service")
        return {k: {"p50_ms": out[3 * i], "p99_ms": out[3 * i + 1], "max_ms": out[3 * i + 2]} for i, k in enumerate(keys)}

    TRACE_KEYS = ("admit_ms", "launch_host_ms", "device_ms", "done_ms", "galaxies", "lane", "backlog_galaxies",
                  "lanes_busy")

    def trace(self):
        """Per micro-batch rows (completion order) since the server started
        or the last ``timing(reset=True)``: an (n, 8) float64 array with
        columns ``TRACE_KEYS``."""
        lib = capi.library()
        n = ctypes.c_int64()
        capi._check(self.renderer.ctx, lib.mog_server_trace(self.handle, None, 0, ctypes.byref(n)))
        out = np.zeros((max(n.value, 0), capi.MOG_TRACE_COLS), dtype=np.float64)
        if n.value:
            got = ctypes.c_int64()
            capi._check(self.renderer.ctx, lib.mog_server_trace(
                self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n.value, ctypes.byref(got)))
            out = out[:min(n.value, got.value)]
        return out

    def close(self):
        if self.handle is not None:
            capi.library().mog_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_fits(renderer, fits_gals, noise_seed=0, sigma_frac=0.01):
    """Device fit state for a list of ``workloads.Galaxies`` (one per fit):
    observed patches rendered from the galaxies' parameters (the fits'
    'truth') plus Gaussian noise of sigma_frac times each patch's peak, and
    ivar = 1 / sigma^2 per patch.  All fits are rendered in one batch; each
    fit's state is a set of views into the shared device tensors.  Returns a
    list of dicts of device tensors."""
    from .renderer import to_device
    from workloads import Galaxies
    counts = [len(g) for g in fits_gals]
    allg = Galaxies(**{f: np.concatenate([getattr(g, f) for g in fits_gals])
                       for f in Galaxies.FLOAT_FIELDS + Galaxies.INT_FIELDS})
    b = to_device(allg)
    img = renderer.render(b)
    npix = torch.from_numpy(np.asarray(b.sizes, np.int64) ** 2).cuda()
    peaks = torch.segment_reduce(img, "max", lengths=npix)
    sigma = sigma_frac * peaks
    gen = torch.Generator(device="cuda").manual_seed(noise_seed)
    data = img + torch.repeat_interleave(sigma, npix) * torch.randn(img.shape, device="cuda", generator=gen)
    ivar = (1.0 / sigma ** 2).float().contiguous()
    del img
    out = []
    start = 0
    for c in counts:
        sl = slice(start, start + c)
        base = int(b.offsets[start])
        out.append(dict(sersic_n=b.tensors["sersic_n"][sl], profile=b.tensors["profile"][sl],
                        psf=b.tensors["psf"][sl], size=b.tensors["size"][sl],
                        data_offset=(b.tensors["offset"][sl] - base).contiguous(),
                        data=data[base:], ivar=ivar[sl]))
        start += c
    out_keep = (b, data, ivar)
    for d in out:
        d["_keep"] = out_keep
    return out
