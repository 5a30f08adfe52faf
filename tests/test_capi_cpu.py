"""Host-side checks of the C-ABI library (no GPU): it builds, loads, exports
every entry point that include/mogconv.h declares, and rejects bad arguments
before touching the device."""

import ctypes
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"^\s*(?:mog_status|const char\*)\s+(mog_\w+)\s*\(", src, re.M))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2012_15797_gb300.build import build
    lib = ctypes.CDLL(build())
    names = _declared()
    assert len(names) >= 8
    for n in names:
        assert hasattr(lib, n), n
    from paper_2012_15797_gb300 import capi
    assert set(capi.EXPORTED) <= names


def test_null_arguments_rejected_without_device():
    from paper_2012_15797_gb300 import capi
    lib = capi.library()
    assert lib.mog_create_context(None, 0) == capi.MOG_ERR_ARG
    assert lib.mog_destroy_context(None) == capi.MOG_ERR_ARG
    assert lib.mog_render_batch(None, None, None, None) == capi.MOG_ERR_ARG
    assert lib.mog_sync_status(None, None) == capi.MOG_ERR_ARG
    assert lib.mog_render_composite(None, None, None, None, None, 0) == capi.MOG_ERR_ARG
    assert lib.mog_render_batch_cufft(None, None, None, None) == capi.MOG_ERR_ARG
    assert lib.mog_render_chi2(None, None, None, None, None, None, None, None) == capi.MOG_ERR_ARG
    assert lib.mog_last_error(None) == b"null context"


def test_pack_offsets():
    from paper_2012_15797_gb300.renderer import pack_offsets
    off, total = pack_offsets([32, 64, 32])
    assert list(off) == [0, 1024, 1024 + 4096] and total == 1024 + 4096 + 1024
    assert np.all(off % 4 == 0)
