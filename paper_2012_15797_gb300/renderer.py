"""PyTorch marshalling around the C-ABI: device memory and streams come from
torch, every computation runs in the library's kernels."""

from dataclasses import dataclass

import numpy as np
import torch

from . import capi

FLOAT_FIELDS = ("flux", "x", "y", "log_re", "e1", "e2", "sersic_n")
INT_FIELDS = ("profile", "psf", "size")


@dataclass
class DeviceBatch:
    """A batch of galaxies resident on the device (structure of arrays) plus
    the packed-output layout: galaxy g owns out[offset[g] : offset[g] + size[g]^2]."""
    tensors: dict
    count: int
    total: int           # output elements
    sizes: np.ndarray    # host copy of the patch sides
    offsets: np.ndarray  # host copy of the offsets

    def ptrs(self):
        return {k: v.data_ptr() for k, v in self.tensors.items()}

    def size_mask(self):
        # computed once per batch: the sides do not change, and for batches of
        # 10^5 galaxies recomputing it every call cost more host time than the
        # render took on the device
        m = self.__dict__.get("_size_mask")
        if m is None:
            m = self.__dict__["_size_mask"] = size_mask(self.sizes)
        return m


SIDES = (32, 64, 128, 256)


def size_mask(sizes):
    """Bitmask of the patch sides present (bit b: N = 32 << b); 0 when a
    side is not one of them (the library then reports it)."""
    sizes = np.asarray(sizes)
    hit = [bool(np.any(sizes == n)) for n in SIDES]
    if sum(int(np.count_nonzero(sizes == n)) for n, h in zip(SIDES, hit) if h) != sizes.size:
        return 0
    return sum(1 << b for b, h in enumerate(hit) if h)


def pack_offsets(sizes):
    sizes = np.asarray(sizes, dtype=np.int64)
    area = sizes * sizes
    off = np.zeros(len(sizes), dtype=np.int64)
    if len(sizes) > 1:
        off[1:] = np.cumsum(area)[:-1]
    return off, int(area.sum())


def host_batch(gals, pin=False, positions=None, cd=None):
    """Host tensors (optionally pinned) of a ``workloads.Galaxies`` batch;
    ``positions`` = (img_x, img_y) image positions, needed by galaxies whose
    PSF is an eigen-PSF; ``cd`` = (G, 2, 2) or (G, 4) WCS matrices (None:
    pixel units)."""
    t = {}
    for f in FLOAT_FIELDS:
        t[f] = torch.from_numpy(np.ascontiguousarray(getattr(gals, f), dtype=np.float32))
    for f in INT_FIELDS:
        t[f] = torch.from_numpy(np.ascontiguousarray(getattr(gals, f), dtype=np.int32))
    off, total = pack_offsets(gals.size)
    t["offset"] = torch.from_numpy(off)
    if positions is not None:
        t["img_x"] = torch.from_numpy(np.ascontiguousarray(positions[0], dtype=np.float32))
        t["img_y"] = torch.from_numpy(np.ascontiguousarray(positions[1], dtype=np.float32))
    if cd is not None:
        t["cd"] = torch.from_numpy(np.ascontiguousarray(np.asarray(cd).reshape(len(gals), 4), dtype=np.float32))
    if pin:
        t = {k: v.pin_memory() for k, v in t.items()}
    return t, total


def to_device(gals, device="cuda", positions=None, cd=None):
    t, total = host_batch(gals, positions=positions, cd=cd)
    dev = {k: v.to(device) for k, v in t.items()}
    return DeviceBatch(dev, len(gals), total, np.asarray(gals.size).copy(), t["offset"].numpy().copy())


class Renderer:
    """Owns a library context with its profile tables and PSFs."""

    def __init__(self, tables, psfs, device=0):
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        self.ctx = capi.mog_create_context(device)
        for pid, t in tables.items():
            capi.mog_set_profile_table(self.ctx, pid, t.nodes, t.amp, t.var)
        self.psf_ids = [capi.mog_create_psf(self.ctx, p.image, p.mog) if hasattr(p, "image")
                        else capi.mog_create_eigen_psf(self.ctx, p.components, p.degree, p.norm, p.mog_shape,
                                                       p.mog_amp)
                        for p in psfs]
        if self.psf_ids != list(range(len(psfs))):
            raise RuntimeError("fresh context expected PSF ids 0..P-1")

    def close(self):
        if self.ctx is not None:
            capi.mog_destroy_context(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def render(self, batch, out=None, stream=None, shift="phase", add=False):
        """Renders a DeviceBatch into a flat float32 device tensor.  ``shift``
        selects how the sub-pixel offset is applied: "phase" (Fourier shift
        phase) or "lanczos" (Lanczos-3 convolution of the final model).  With
        ``add`` the models are added to what ``out`` holds."""
        if shift not in ("phase", "lanczos"):
            raise ValueError(f"unknown shift {shift!r}")
        if add and out is None:
            raise ValueError("add=True needs an output to add to")
        if out is None:
            out = torch.empty(batch.total, dtype=torch.float32, device=self.device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        b = capi.make_batch(batch.count, batch.ptrs(), batch.size_mask())
        if add:
            flags = capi.MOG_RENDER_ADD | (capi.MOG_RENDER_LANCZOS if shift == "lanczos" else 0)
            capi.mog_render_batch_ex(self.ctx, b, out.data_ptr(), s.cuda_stream, flags)
            return out
        fn = capi.mog_render_batch if shift == "phase" else capi.mog_render_batch_lanczos
        fn(self.ctx, b, out.data_ptr(), s.cuda_stream)
        return out

    def render_cufft(self, batch, out=None, stream=None):
        """The library comparator of ``render`` (mog_render_batch_cufft): the
        same patches through written-out spectra, a batched cuFFT inverse
        real transform and a real-space pass.  One patch side per batch."""
        if out is None:
            out = torch.empty(batch.total, dtype=torch.float32, device=self.device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        b = capi.make_batch(batch.count, batch.ptrs(), batch.size_mask())
        capi.mog_render_batch_cufft(self.ctx, b, out.data_ptr(), s.cuda_stream)
        return out

    def render_host(self, host, out=None, chunk=0, shift="phase"):
        """Renders a batch held in host memory, ``host`` = ``host_batch(...)``
        (tensors, pinned for asynchronous copies; packed offsets), into a host
        float32 tensor (allocated pinned when ``out`` is None) through
        mog_render_batch_host: chunks of at most ``chunk`` galaxies (0: about
        64 MiB of patches), copies overlapping renders on two streams.
        Synchronous."""
        if shift not in ("phase", "lanczos"):
            raise ValueError(f"unknown shift {shift!r}")
        t, total = host
        if out is None:
            out = torch.empty(total, dtype=torch.float32).pin_memory()
        if out.device.type != "cpu" or out.dtype != torch.float32 or out.numel() < total:
            raise ValueError("out must be a host float32 tensor of the batch's total size")
        # no size mask: the library works out each chunk's buckets itself
        b = capi.make_batch(len(t["flux"]), {k: v.data_ptr() for k, v in t.items()})
        capi.mog_render_batch_host(self.ctx, b, out.data_ptr(), chunk,
                                   capi.MOG_RENDER_LANCZOS if shift == "lanczos" else 0)
        return out

    def render_composite(self, disk, bulge, out=None, stream=None, shift="phase", fused=True):
        """Composite (bulge + disk) galaxies: the sum of two profiles sharing
        the patch layout, PSF and centre.  ``disk`` and ``bulge`` are
        DeviceBatches with the same sizes, offsets, PSFs and (x, y).  With
        ``fused`` one call renders both profiles (mog_render_composite: one
        transform per galaxy); otherwise the disks are rendered and the
        bulges added (mog_render_batch_ex, add mode)."""
        if shift not in ("phase", "lanczos"):
            raise ValueError(f"unknown shift {shift!r}")
        if fused:
            if out is None:
                out = torch.empty(disk.total, dtype=torch.float32, device=self.device)
            s = stream if stream is not None else torch.cuda.current_stream(self.device)
            capi.mog_render_composite(self.ctx, capi.make_batch(disk.count, disk.ptrs(), disk.size_mask()),
                                      capi.make_batch(bulge.count, bulge.ptrs(), 0), out.data_ptr(), s.cuda_stream,
                                      capi.MOG_RENDER_LANCZOS if shift == "lanczos" else 0)
            return out
        out = self.render(disk, out, stream, shift)
        return self.render(bulge, out, stream, shift, add=True)

    def render_composite_backward(self, disk, bulge, grad_out, stream=None, sersic=False, shift="phase"):
        """Gradients of a composite's loss with respect to each profile's
        parameters, ((count, k), (count, k)): the adjoint of a sum is each
        part's adjoint with the same upstream gradient.  The shared centre's
        gradient is the sum of the two x (and y) columns."""
        return (self.render_backward(disk, grad_out, stream=stream, sersic=sersic, shift=shift),
                self.render_backward(bulge, grad_out, stream=stream, sersic=sersic, shift=shift))

    def render_backward(self, batch, grad_out, grad_params=None, stream=None, sersic=False, shift="phase"):
        """Gradients (count, 6) of L w.r.t. (flux, x, y, log_re, e1, e2)
        given grad_out = dL/d(packed output); with ``sersic`` (count, 7), the
        last column d L / d sersic_n.  ``shift``: the model differentiated,
        "phase" (Fourier shift phase) or "lanczos" (the Lanczos-3 variant)."""
        if shift not in ("phase", "lanczos"):
            raise ValueError(f"unknown shift {shift!r}")
        k = 7 if sersic else 6
        if grad_params is None:
            grad_params = torch.empty(batch.count, k, dtype=torch.float32, device=self.device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        b = capi.make_batch(batch.count, batch.ptrs(), batch.size_mask())
        flags = (capi.MOG_GRAD_SERSIC if sersic else 0) | (capi.MOG_GRAD_LANCZOS if shift == "lanczos" else 0)
        if flags:
            capi.mog_render_backward_ex(self.ctx, b, grad_out.data_ptr(), grad_params.data_ptr(), s.cuda_stream,
                                        flags)
        else:
            capi.mog_render_backward(self.ctx, b, grad_out.data_ptr(), grad_params.data_ptr(), s.cuda_stream)
        return grad_params

    def chi2_gradient(self, batch, model, data, ivar, grad_pix=None, chi2=None, stream=None):
        """d chi^2 / d model = 2 ivar (model - data) on every patch (the
        upstream gradient of render_backward) and chi^2 per galaxy;
        ``ivar`` (count,) float32.  Returns (grad_pix, chi2)."""
        if grad_pix is None:
            grad_pix = torch.empty_like(model)
        if chi2 is None:
            chi2 = torch.empty(batch.count, dtype=torch.float32, device=self.device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        b = capi.make_batch(batch.count, batch.ptrs(), batch.size_mask())
        capi.mog_chi2_gradient(self.ctx, b, model.data_ptr(), data.data_ptr(), ivar.contiguous().data_ptr(),
                               grad_pix.data_ptr(), chi2.data_ptr(), s.cuda_stream)
        return grad_pix, chi2

    def render_chi2(self, batch, data, ivar, grad_pix=None, chi2=None, model=None, stream=None):
        """Render and loss in one pass (mog_render_chi2): returns (grad_pix,
        chi2) with grad_pix = 2 ivar (model - data) on every patch and chi2 =
        ivar sum (model - data)^2 per galaxy; the model is written into
        ``model`` too when a tensor is given."""
        if grad_pix is None:
            grad_pix = torch.empty(batch.total, dtype=torch.float32, device=self.device)
        if chi2 is None:
            chi2 = torch.empty(batch.count, dtype=torch.float32, device=self.device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        b = capi.make_batch(batch.count, batch.ptrs(), batch.size_mask())
        capi.mog_render_chi2(self.ctx, b, data.data_ptr(), ivar.contiguous().data_ptr(), grad_pix.data_ptr(),
                             chi2.data_ptr(), model.data_ptr() if model is not None else 0, s.cuda_stream)
        return grad_pix, chi2

    def fit_psf_mixtures(self, images, k=3, iters=400, stream=None):
        """Gaussian-mixture fits of a (count, h, w) float32 device tensor of
        PSF images: returns ((count, k, 6) rows, (count,) chi^2)."""
        images = images.contiguous()
        count, h, w = images.shape
        rows = torch.empty(count, k, 6, dtype=torch.float32, device=self.device)
        chi2 = torch.empty(count, dtype=torch.float32, device=self.device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        capi.mog_fit_psf_mixture(self.ctx, images.data_ptr(), count, h, w, k, iters, rows.data_ptr(), chi2.data_ptr(),
                                 s.cuda_stream)
        return rows, chi2

    def autotune(self, batch, out, grad_out=None, grad_params=None, reps=3, stream=None):
        """Times every launch shape per size bucket and keeps the fastest
        (forward, and the adjoint when gradient buffers are given)."""
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        b = capi.make_batch(batch.count, batch.ptrs(), batch.size_mask())
        return capi.mog_autotune(self.ctx, b, out.data_ptr(), grad_out.data_ptr() if grad_out is not None else 0,
                                 grad_params.data_ptr() if grad_params is not None else 0, s.cuda_stream, reps)

    def graph(self, batch, out):
        """A captured CUDA graph rendering `batch` into `out` on every launch."""
        return Graph(self, batch, out)

    def sync_status(self, stream=None):
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        capi.mog_sync_status(self.ctx, s.cuda_stream)


class Graph:
    def __init__(self, renderer, batch, out):
        self.renderer, self.batch, self.out = renderer, batch, out
        self._b = capi.make_batch(batch.count, batch.ptrs(), batch.size_mask())
        self.handle = capi.mog_graph_capture(renderer.ctx, self._b, out.data_ptr())

    def launch(self, stream=None):
        s = stream if stream is not None else torch.cuda.current_stream(self.renderer.device)
        capi.mog_graph_launch(self.handle, s.cuda_stream)
        return self.out

    def close(self):
        if self.handle is not None:
            capi.mog_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def patches(out, batch):
    """List of (N, N) views of a packed output."""
    o = out.reshape(-1)
    return [o[int(batch.offsets[i]):int(batch.offsets[i]) + int(batch.sizes[i]) ** 2].view(
        int(batch.sizes[i]), int(batch.sizes[i])) for i in range(batch.count)]


PARAM_FIELDS = ("flux", "x", "y", "log_re", "e1", "e2")


class _Render(torch.autograd.Function):
    """theta (6, G) float32 CUDA tensor, rows (flux, x, y, log_re, e1, e2);
    returns the packed patches.  Backward runs the library's adjoint kernel."""

    @staticmethod
    def forward(ctx, theta, renderer, batch):
        theta = theta.contiguous()
        tensors = dict(batch.tensors)
        for k, name in enumerate(PARAM_FIELDS):
            tensors[name] = theta[k]
        b = DeviceBatch(tensors, batch.count, batch.total, batch.sizes, batch.offsets)
        out = renderer.render(b)
        ctx.renderer = renderer
        ctx.batch = b
        ctx.save_for_backward(theta)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        grad_out = grad_out.contiguous()
        g = ctx.renderer.render_backward(ctx.batch, grad_out)
        return g.t(), None, None


def render(theta, renderer, batch):
    """Differentiable batched render: theta (6, G) -> packed patches."""
    return _Render.apply(theta, renderer, batch)


def theta_of(batch):
    """(6, G) tensor of the differentiable parameters of a DeviceBatch."""
    return torch.stack([batch.tensors[k] for k in PARAM_FIELDS])
