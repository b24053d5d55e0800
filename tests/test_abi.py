"""CPU checks of the C ABI: the library loads and exports every declared call.

No kernel runs here (no GPU is needed): only calls that fail argument checks
before touching CUDA, and the static string functions.
"""
import ctypes

import pytest


@pytest.fixture(scope="module")
def rfim():
    from paper_2001_03389_gb300 import build

    build.build()
    from paper_2001_03389_gb300 import rfim as r

    return r


def test_exports_every_header_function(rfim):
    names = rfim.header_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(rfim._lib, n), f"{n} declared in include/rfim.h but not exported"


def test_static_strings(rfim):
    assert rfim.rfim_version().decode().startswith("rfim-gb300")
    assert rfim.rfim_status_str(rfim.OK).decode() == "ok"
    assert rfim.rfim_status_str(rfim.ERR_TIMEOUT).decode() == "device-side wait timed out"
    assert rfim.rfim_status_str(99).decode() == "unknown status"


def test_null_context_is_rejected(rfim):
    blk = rfim.rfim_block()
    cut = rfim.make_cut(3.0)
    assert rfim.rfim_tdsc(None, ctypes.byref(blk), ctypes.byref(cut), None) == rfim.ERR_ARG
    assert rfim.rfim_fdsc(None, ctypes.byref(blk), ctypes.byref(cut), None) == rfim.ERR_ARG
    assert rfim.rfim_clean(None, ctypes.byref(blk), ctypes.byref(cut), None, None) == rfim.ERR_ARG
    assert rfim.rfim_set_option(None, b"schedule", 1) == rfim.ERR_ARG
    assert rfim.rfim_destroy(None) == rfim.OK
    assert rfim.rfim_create(None, 0, 0, None) == rfim.ERR_ARG


def test_struct_layout_matches_header(rfim):
    # rfim_cut: double, int, enum, int; rfim_block: 3 pointers, 6 ints
    assert ctypes.sizeof(rfim.rfim_cut) == 24
    assert ctypes.sizeof(rfim.rfim_block) == 3 * 8 + 6 * 4 + 0  # 48 bytes, no padding
