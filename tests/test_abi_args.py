"""Argument checks of the C ABI run on the host before any CUDA call: NULL handles or buffers and
bad sizes return GWE_ERR_ARG (1) with a message in gwe_last_error, here without a GPU."""
import ctypes

import pytest

import paper_2201_11133_gb300 as gwe

ARG = 1
FAKE = 0x1000          # a non-NULL pointer that no check dereferences


def _lib():
    gwe.build()
    return gwe.load()


def _expect_arg(status):
    assert status == ARG
    assert len(_lib().gwe_last_error()) > 0


def test_forward_entry_points_reject_bad_arguments():
    lib = _lib()
    _expect_arg(lib.gwe_forward(None, FAKE, FAKE, 8192, 4096, 2048, None, 0, FAKE, None))
    _expect_arg(lib.gwe_forward_logits(None, FAKE, FAKE, 4, 4096, FAKE, None))
    _expect_arg(lib.gwe_forward_static(None, FAKE, FAKE, 8192, 4096, 2048, FAKE, None, None))
    seg = (ctypes.c_int64 * 1)(0)
    _expect_arg(lib.gwe_forward_segments(None, FAKE, FAKE, seg, seg, 1, 4096, 2048, None, 0, FAKE, None))


def test_backward_rejects_bad_arguments():
    lib = _lib()
    _expect_arg(lib.gwe_backward(None, 0, FAKE, FAKE, 4, 4096, FAKE, FAKE, None, None, None))


@pytest.mark.parametrize("window,stride,coinc", [(0, 1, 0), (4096, 0, 0), (4096, 8192, 0), (4096, 2048, -1)])
def test_triggers_reject_bad_geometry(window, stride, coinc):
    lib = _lib()
    n_out = ctypes.c_int64(0)
    _expect_arg(lib.gwe_triggers(FAKE, 4, 1, 10, window, stride, 0.5, 2048.0, coinc, 0, None, 0,
                                 ctypes.byref(n_out), None))


def test_triggers_reject_null_buffers():
    lib = _lib()
    n_out = ctypes.c_int64(0)
    _expect_arg(lib.gwe_triggers(None, 4, 1, 10, 4096, 2048, 0.5, 2048.0, 2048, 0, None, 0,
                                 ctypes.byref(n_out), None))
    _expect_arg(lib.gwe_triggers(FAKE, 4, 1, 10, 4096, 2048, 0.5, 2048.0, 2048, 0, None, 5,
                                 ctypes.byref(n_out), None))      # cap > 0 without an output array


@pytest.mark.parametrize("n,fs,seg", [(100000, 0.0, 16384), (100000, 4096.0, 1000), (1000, 4096.0, 16384)])
def test_whiten_rejects_bad_arguments(n, fs, seg):
    lib = _lib()
    _expect_arg(lib.gwe_whiten(FAKE, n, fs, seg, 0, FAKE + 64, None))
    _expect_arg(lib.gwe_whiten(FAKE, 100000, 4096.0, 16384, 0, FAKE, None))   # out aliases strain


def test_plan_and_search_reject_null_handles():
    lib = _lib()
    out = ctypes.c_void_p(0)
    seg = (ctypes.c_int64 * 1)(0)
    _expect_arg(lib.gwe_plan_create(None, FAKE, FAKE, seg, seg, 1, 4096, 2048, None, 0, FAKE, 0,
                                    ctypes.byref(out), None))
    _expect_arg(lib.gwe_plan_execute(None, None))
    _expect_arg(lib.gwe_search_create(None, None, ctypes.byref(out)))
    n_out = ctypes.c_int64(0)
    _expect_arg(lib.gwe_search_run(None, FAKE, FAKE, 0, 0, None, 0, ctypes.byref(n_out), None))
    _expect_arg(lib.gwe_sync(None, None))
