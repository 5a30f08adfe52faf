"""ctypes binding of the C-ABI declared in include/mogconv.h.

Argument marshalling only: every function here forwards to the entry point of
the same name in lib/libmogconv.so and raises ``MogError`` on a non-zero
status.  Device pointers are passed as integers (e.g. ``tensor.data_ptr()``),
streams as the integer handle of a ``torch.cuda.Stream`` (``.cuda_stream``).
The library must have been built (``paper_2012_15797_gb300.build.build()``);
importing this module without it raises.
"""

import ctypes
import os

import numpy as np

from .build import LIB

MOG_OK = 0
MOG_ERR_ARG = -1
MOG_ERR_CUDA = -2
MOG_ERR_NOMEM = -3
MOG_ERR_STATE = -4
MOG_ERR_TIMEOUT = -5
MOG_ERR_DEVICE = -6
MOG_MAX_COMPONENTS = 12
MOG_MAX_PSF_COMPONENTS = 4
MOG_MAX_PSFS = 1024
MOG_MAX_PROFILES = 8
MOG_MAX_NODES = 64

EXPORTED = (
    "mog_create_context", "mog_destroy_context", "mog_last_error", "mog_set_profile_table",
    "mog_create_psf", "mog_destroy_psf", "mog_render_batch", "mog_sync_status",
    "mog_set_timing", "mog_read_timing", "mog_render_backward", "mog_render_batch_noalloc",
    "mog_autotune", "mog_graph_capture", "mog_graph_launch", "mog_graph_destroy",
    "mog_server_create", "mog_server_add_fit", "mog_server_submit", "mog_server_wait", "mog_server_replay",
    "mog_server_replay_join", "mog_server_stats", "mog_server_destroy", "mog_render_batch_lanczos",
    "mog_create_eigen_psf", "mog_render_batch_ex", "mog_render_backward_ex", "mog_fit_psf_mixture",
    "mog_render_batch_host", "mog_measure_pipe_rates", "mog_server_inject_fault", "mog_check_wait_timeout",
    "mog_set_launch_shape", "mog_chi2_gradient", "mog_server_timing", "mog_server_trace", "mog_render_chi2",
    "mog_render_batch_cufft", "mog_render_composite",
)
MOG_TRACE_COLS = 8
MOG_NOALLOC_MAX_GALAXIES = 16384


class MogError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"mogconv error {status}: {msg}")
        self.status = status


class mog_batch(ctypes.Structure):
    _fields_ = [
        ("count", ctypes.c_int64),
        ("flux", ctypes.c_void_p), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
        ("log_re", ctypes.c_void_p), ("e1", ctypes.c_void_p), ("e2", ctypes.c_void_p),
        ("sersic_n", ctypes.c_void_p), ("profile", ctypes.c_void_p), ("psf", ctypes.c_void_p),
        ("size", ctypes.c_void_p), ("offset", ctypes.c_void_p),
        ("size_mask", ctypes.c_uint32),
        ("img_x", ctypes.c_void_p), ("img_y", ctypes.c_void_p), ("cd", ctypes.c_void_p),
    ]


class mog_server_config(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("lanes", ctypes.c_int), ("max_batch_galaxies", ctypes.c_int64)]


class mog_fit_state(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int64), ("sersic_n", ctypes.c_void_p), ("profile", ctypes.c_void_p),
                ("psf", ctypes.c_void_p), ("size", ctypes.c_void_p), ("data_offset", ctypes.c_void_p),
                ("data", ctypes.c_void_p), ("ivar", ctypes.c_void_p)]


class mog_request(ctypes.Structure):
    _fields_ = [("fit", ctypes.c_int32), ("first", ctypes.c_int64), ("count", ctypes.c_int64),
                ("params", ctypes.c_void_p), ("grads", ctypes.c_void_p), ("chi2", ctypes.c_void_p)]


def _load():
    if not os.path.exists(LIB):
        raise ImportError(f"CUDA library not built: {LIB} is missing (run paper_2012_15797_gb300.build.build())")
    lib = ctypes.CDLL(LIB)
    P, I, VP = ctypes.POINTER, ctypes.c_int, ctypes.c_void_p
    FP = P(ctypes.c_float)
    sig = {
        "mog_create_context": ([P(VP), I], I),
        "mog_destroy_context": ([VP], I),
        "mog_last_error": ([VP], ctypes.c_char_p),
        "mog_set_profile_table": ([VP, I, I, FP, FP, FP], I),
        "mog_create_psf": ([VP, FP, I, I, FP, I, P(I)], I),
        "mog_create_eigen_psf": ([VP, FP, I, I, I, I, FP, FP, FP, I, P(I)], I),
        "mog_destroy_psf": ([VP, I], I),
        "mog_render_batch": ([VP, P(mog_batch), VP, VP], I),
        "mog_render_batch_lanczos": ([VP, P(mog_batch), VP, VP], I),
        "mog_render_batch_ex": ([VP, P(mog_batch), VP, VP, ctypes.c_uint], I),
        "mog_render_backward": ([VP, P(mog_batch), VP, VP, VP], I),
        "mog_render_backward_ex": ([VP, P(mog_batch), VP, VP, VP, ctypes.c_uint], I),
        "mog_fit_psf_mixture": ([VP, VP, I, I, I, I, I, VP, VP, VP], I),
        "mog_render_batch_noalloc": ([VP, P(mog_batch), VP, VP], I),
        "mog_render_batch_host": ([VP, P(mog_batch), VP, ctypes.c_int64, ctypes.c_uint], I),
        "mog_autotune": ([VP, P(mog_batch), VP, VP, VP, VP, I, P(I)], I),
        "mog_graph_capture": ([VP, P(mog_batch), VP, P(VP)], I),
        "mog_graph_launch": ([VP, VP], I),
        "mog_graph_destroy": ([VP], I),
        "mog_server_create": ([VP, P(mog_server_config), P(VP)], I),
        "mog_server_add_fit": ([VP, P(mog_fit_state), P(I)], I),
        "mog_server_submit": ([VP, P(mog_request), P(ctypes.c_uint64)], I),
        "mog_server_wait": ([VP, ctypes.c_uint64, ctypes.c_double, P(ctypes.c_double)], I),
        "mog_server_replay": ([VP, P(mog_request), P(ctypes.c_double), ctypes.c_int64, P(ctypes.c_uint64)], I),
        "mog_server_replay_join": ([VP], I),
        "mog_server_stats": ([VP, P(ctypes.c_int64)], I),
        "mog_server_destroy": ([VP], I),
        "mog_sync_status": ([VP, VP], I),
        "mog_set_timing": ([VP, I], I),
        "mog_read_timing": ([VP, P(ctypes.c_double), P(ctypes.c_int64)], I),
        "mog_measure_pipe_rates": ([VP, I, P(ctypes.c_double), P(ctypes.c_double)], I),
        "mog_server_inject_fault": ([VP, I, ctypes.c_int64], I),
        "mog_check_wait_timeout": ([VP, ctypes.c_double, VP], I),
        "mog_set_launch_shape": ([VP, I, I, I, I, I], I),
        "mog_chi2_gradient": ([VP, P(mog_batch), VP, VP, VP, VP, VP, VP], I),
        "mog_server_timing": ([VP, P(ctypes.c_double), I], I),
        "mog_server_trace": ([VP, P(ctypes.c_double), ctypes.c_int64, P(ctypes.c_int64)], I),
        "mog_render_chi2": ([VP, P(mog_batch), VP, VP, VP, VP, VP, VP], I),
        "mog_render_batch_cufft": ([VP, P(mog_batch), VP, VP], I),
        "mog_render_composite": ([VP, P(mog_batch), P(mog_batch), VP, VP, ctypes.c_uint], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()


def library():
    return _lib


def _check(ctx, status):
    if status != MOG_OK:
        msg = _lib.mog_last_error(ctx).decode() if ctx else ""
        raise MogError(status, msg)


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def mog_create_context(device=0):
    h = ctypes.c_void_p()
    _check(None, _lib.mog_create_context(ctypes.byref(h), int(device)))
    return h


def mog_destroy_context(ctx):
    _check(None, _lib.mog_destroy_context(ctx))


def mog_last_error(ctx):
    return _lib.mog_last_error(ctx).decode()


def mog_set_profile_table(ctx, profile_id, nodes, amp, var):
    nodes = np.ascontiguousarray(nodes, dtype=np.float32)
    amp = np.ascontiguousarray(amp, dtype=np.float32)
    var = np.ascontiguousarray(var, dtype=np.float32)
    n = nodes.shape[0]
    assert amp.size == n * MOG_MAX_COMPONENTS and var.size == n * MOG_MAX_COMPONENTS
    _check(ctx, _lib.mog_set_profile_table(ctx, int(profile_id), n, _fptr(nodes), _fptr(amp), _fptr(var)))


def mog_create_psf(ctx, pixels, mog):
    pixels = np.ascontiguousarray(pixels, dtype=np.float32)
    mog = np.ascontiguousarray(mog, dtype=np.float32)
    h, w = pixels.shape
    k = mog.shape[0]
    assert mog.shape == (k, 6)
    out = ctypes.c_int(-1)
    _check(ctx, _lib.mog_create_psf(ctx, _fptr(pixels), h, w, _fptr(mog), k, ctypes.byref(out)))
    return out.value


def mog_create_eigen_psf(ctx, components, degree, norm, mog_shape, mog_amp):
    comps = np.ascontiguousarray(components, dtype=np.float32)
    K, h, w = comps.shape
    norm = np.ascontiguousarray(norm, dtype=np.float32)
    shape = np.ascontiguousarray(mog_shape, dtype=np.float32)
    amp = np.ascontiguousarray(mog_amp, dtype=np.float32)
    k = shape.shape[0]
    assert norm.shape == (4,) and shape.shape == (k, 5) and amp.shape == (K, k)
    out = ctypes.c_int(-1)
    _check(ctx, _lib.mog_create_eigen_psf(ctx, _fptr(comps), K, h, w, int(degree), _fptr(norm), _fptr(shape),
                                          _fptr(amp), k, ctypes.byref(out)))
    return out.value


def mog_destroy_psf(ctx, psf_id):
    _check(ctx, _lib.mog_destroy_psf(ctx, int(psf_id)))


def make_batch(count, ptrs, size_mask=0):
    """``ptrs``: dict of device pointers (ints) for every batch field;
    ``size_mask``: optional bitmask of the patch sides present."""
    b = mog_batch()
    b.count = int(count)
    for f, kind in mog_batch._fields_[1:]:
        if kind is ctypes.c_void_p:
            setattr(b, f, ctypes.c_void_p(int(ptrs[f])) if ptrs.get(f) is not None else None)
    b.size_mask = int(size_mask)
    return b


def mog_render_batch(ctx, batch, out_ptr, stream=0):
    _check(ctx, _lib.mog_render_batch(ctx, ctypes.byref(batch), ctypes.c_void_p(int(out_ptr)),
                                      ctypes.c_void_p(int(stream))))


def mog_render_batch_lanczos(ctx, batch, out_ptr, stream=0):
    _check(ctx, _lib.mog_render_batch_lanczos(ctx, ctypes.byref(batch), ctypes.c_void_p(int(out_ptr)),
                                              ctypes.c_void_p(int(stream))))


MOG_RENDER_LANCZOS, MOG_RENDER_ADD = 1, 2


def mog_render_batch_ex(ctx, batch, out_ptr, stream=0, flags=0):
    _check(ctx, _lib.mog_render_batch_ex(ctx, ctypes.byref(batch), ctypes.c_void_p(int(out_ptr)),
                                         ctypes.c_void_p(int(stream)), ctypes.c_uint(int(flags))))


def mog_render_composite(ctx, first, second, out_ptr, stream=0, flags=0):
    """Composite galaxies in one pass (see include/mogconv.h): galaxy g of
    ``first`` and of ``second`` are the two profiles of one galaxy; flags 0
    or MOG_RENDER_LANCZOS."""
    _check(ctx, _lib.mog_render_composite(ctx, ctypes.byref(first), ctypes.byref(second),
                                          ctypes.c_void_p(int(out_ptr)), ctypes.c_void_p(int(stream)),
                                          ctypes.c_uint(int(flags))))


def mog_render_batch_cufft(ctx, batch, out_ptr, stream=0):
    """The library comparator of mog_render_batch (see include/mogconv.h):
    spectra, one batched cuFFT inverse real transform, real-space add; the
    batch's size_mask names its one patch side."""
    _check(ctx, _lib.mog_render_batch_cufft(ctx, ctypes.byref(batch), ctypes.c_void_p(int(out_ptr)),
                                            ctypes.c_void_p(int(stream))))


def mog_render_batch_host(ctx, batch, out_ptr, chunk=0, flags=0):
    """Render of a batch held in host memory into a host output (see
    include/mogconv.h): packed patches, chunks pipelined over two streams;
    returns when the patches are in the output."""
    _check(ctx, _lib.mog_render_batch_host(ctx, ctypes.byref(batch), ctypes.c_void_p(int(out_ptr)),
                                           ctypes.c_int64(int(chunk)), ctypes.c_uint(int(flags))))


def mog_render_batch_noalloc(ctx, batch, out_ptr, stream=0):
    """The allocation-free render (see include/mogconv.h): at most
    MOG_NOALLOC_MAX_GALAXIES galaxies, calls that overlap on the GPU race."""
    _check(ctx, _lib.mog_render_batch_noalloc(ctx, ctypes.byref(batch), ctypes.c_void_p(int(out_ptr)),
                                              ctypes.c_void_p(int(stream))))


def mog_render_backward(ctx, batch, grad_out_ptr, grad_params_ptr, stream=0):
    _check(ctx, _lib.mog_render_backward(ctx, ctypes.byref(batch), ctypes.c_void_p(int(grad_out_ptr)),
                                         ctypes.c_void_p(int(grad_params_ptr)), ctypes.c_void_p(int(stream))))


MOG_GRAD_SERSIC = 1
MOG_GRAD_LANCZOS = 2
MOG_FAULT_DROP, MOG_FAULT_LAUNCH, MOG_FAULT_NOMEM = 1, 2, 3


def mog_render_backward_ex(ctx, batch, grad_out_ptr, grad_params_ptr, stream=0, flags=0):
    _check(ctx, _lib.mog_render_backward_ex(ctx, ctypes.byref(batch), ctypes.c_void_p(int(grad_out_ptr)),
                                            ctypes.c_void_p(int(grad_params_ptr)), ctypes.c_void_p(int(stream)),
                                            ctypes.c_uint(int(flags))))


def mog_fit_psf_mixture(ctx, images_ptr, count, h, w, k, iters, rows_ptr, chi2_ptr=0, stream=0):
    _check(ctx, _lib.mog_fit_psf_mixture(ctx, ctypes.c_void_p(int(images_ptr)), int(count), int(h), int(w), int(k),
                                         int(iters), ctypes.c_void_p(int(rows_ptr)),
                                         ctypes.c_void_p(int(chi2_ptr)) if chi2_ptr else None,
                                         ctypes.c_void_p(int(stream))))


MOG_AUTOTUNE_REPORT = 2 * 4 * 3 + 1


def mog_autotune(ctx, batch, out_ptr, grad_out_ptr=0, grad_params_ptr=0, stream=0, reps=3):
    """Returns {("fwd"|"bwd", N): (ctas_per_sm, chunk, schedule)} for the
    tuned buckets and {"serial": bool} (size kernels one after the other
    rather than forked)."""
    rep = (ctypes.c_int * MOG_AUTOTUNE_REPORT)()
    _check(ctx, _lib.mog_autotune(ctx, ctypes.byref(batch), ctypes.c_void_p(int(out_ptr)),
                                  ctypes.c_void_p(int(grad_out_ptr)), ctypes.c_void_p(int(grad_params_ptr)),
                                  ctypes.c_void_p(int(stream)), int(reps), rep))
    out = {}
    for d, name in enumerate(("fwd", "bwd")):
        for b in range(4):
            c, ch, sc = rep[(d * 4 + b) * 3], rep[(d * 4 + b) * 3 + 1], rep[(d * 4 + b) * 3 + 2]
            if c:
                out[(name, 32 << b)] = (c, ch, sc)
    out["serial"] = bool(rep[MOG_AUTOTUNE_REPORT - 1])
    return out


def mog_set_launch_shape(ctx, direction, n, ctas_per_sm=0, chunk=8, schedule=0):
    """direction: 0 render, 1 adjoint."""
    _check(ctx, _lib.mog_set_launch_shape(ctx, int(direction), int(n), int(ctas_per_sm), int(chunk), int(schedule)))


def mog_render_chi2(ctx, batch, data_ptr, ivar_ptr, grad_ptr, chi2_ptr, model_ptr=0, stream=0):
    _check(ctx, _lib.mog_render_chi2(ctx, ctypes.byref(batch), ctypes.c_void_p(int(data_ptr)),
                                     ctypes.c_void_p(int(ivar_ptr)), ctypes.c_void_p(int(grad_ptr)),
                                     ctypes.c_void_p(int(chi2_ptr)), ctypes.c_void_p(int(model_ptr)),
                                     ctypes.c_void_p(int(stream))))


def mog_chi2_gradient(ctx, batch, model_ptr, data_ptr, ivar_ptr, grad_ptr, chi2_ptr=0, stream=0):
    _check(ctx, _lib.mog_chi2_gradient(ctx, ctypes.byref(batch), ctypes.c_void_p(int(model_ptr)),
                                       ctypes.c_void_p(int(data_ptr)), ctypes.c_void_p(int(ivar_ptr)),
                                       ctypes.c_void_p(int(grad_ptr)), ctypes.c_void_p(int(chi2_ptr)),
                                       ctypes.c_void_p(int(stream))))


def mog_graph_capture(ctx, batch, out_ptr):
    g = ctypes.c_void_p()
    _check(ctx, _lib.mog_graph_capture(ctx, ctypes.byref(batch), ctypes.c_void_p(int(out_ptr)), ctypes.byref(g)))
    return g


def mog_graph_launch(graph, stream=0):
    _check(None, _lib.mog_graph_launch(graph, ctypes.c_void_p(int(stream))))


def mog_graph_destroy(graph):
    _check(None, _lib.mog_graph_destroy(graph))


def mog_set_timing(ctx, enable):
    _check(ctx, _lib.mog_set_timing(ctx, 1 if enable else 0))


def mog_read_timing(ctx):
    """Returns (ms[4], launches[4]) per patch side 32, 64, 128, 256."""
    ms = (ctypes.c_double * 4)()
    n = (ctypes.c_int64 * 4)()
    _check(ctx, _lib.mog_read_timing(ctx, ms, n))
    return list(ms), list(n)


def mog_measure_pipe_rates(ctx, reps=100):
    """(ex2 per second, FP32 FMA per second) measured on the context's device."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(ctx, _lib.mog_measure_pipe_rates(ctx, int(reps), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def mog_check_wait_timeout(ctx, limit_s, stream=0):
    _check(ctx, _lib.mog_check_wait_timeout(ctx, float(limit_s), ctypes.c_void_p(int(stream))))


def mog_sync_status(ctx, stream=0):
    _check(ctx, _lib.mog_sync_status(ctx, ctypes.c_void_p(int(stream))))
