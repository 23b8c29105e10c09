"""The C ABI builds for sm_103a, loads, and exports every declared symbol.

No compute call is made here (there is no GPU on the build host)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "icr.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(icr_[a-z_A-Z0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libicr():
    from paper_2306_06946_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("icr_set_system", "icr_set_mapping", "icr_update_directions", "icr_build_WH", "icr_update_W",
                 "icr_solve_friction", "icr_update_proximity", "icr_correct_motion", "icr_get"):
        assert name in syms


def test_library_exports_every_declared_symbol(libicr):
    missing = [s for s in declared_symbols() if not hasattr(libicr, s)]
    assert not missing


def test_binding_covers_every_declared_symbol():
    from paper_2306_06946_gb300 import icr
    assert sorted(icr.EXPORTS) == declared_symbols()


def test_last_error_is_callable_without_gpu(libicr):
    libicr.icr_last_error.restype = ctypes.c_char_p
    assert isinstance(libicr.icr_last_error(), bytes)


def test_null_arguments_are_rejected_without_gpu(libicr):
    # argument checks run before any CUDA call
    libicr.icr_ctx_create.restype = ctypes.c_int
    assert libicr.icr_ctx_create(None, 0, None, ctypes.c_uint64(0)) == 1        # ICR_EINVAL
    libicr.icr_build_WH.restype = ctypes.c_int
    assert libicr.icr_build_WH(None) == 1


def test_kernels_are_built_for_sm103a():
    from paper_2306_06946_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_batch_calls_reject_null_arguments_without_gpu(libicr):
    # every batch entry point checks its arguments before any CUDA call
    for name in ("icr_batch_create", "icr_batch_launch", "icr_batch_info", "icr_batch_profile"):
        getattr(libicr, name).restype = ctypes.c_int
    assert libicr.icr_batch_create(None, None, 0, 1, 1) == 1            # ICR_EINVAL
    out = ctypes.c_void_p()
    assert libicr.icr_batch_create(ctypes.byref(out), None, 1, 1, 1) == 1
    assert libicr.icr_batch_launch(None) == 1
    assert libicr.icr_batch_info(None, None) == 1
    n = ctypes.c_int32()
    assert libicr.icr_batch_profile(None, None, 0, ctypes.byref(n)) == 1
    libicr.icr_batch_destroy.restype = ctypes.c_int
    assert libicr.icr_batch_destroy(None) == 0                          # ICR_OK: nothing to free
