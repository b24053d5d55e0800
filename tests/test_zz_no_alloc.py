"""The no-allocation entry point against the regular one (GPU, through the C ABI).

rfim_clean_noalloc serves callers that may not allocate device memory (a
real-time pipeline with a fixed memory budget, a plugin without a context);
it keeps its work-queue counters in a fixed device array that every call
shares and clears.  Two calls in a row must each give the same output and
flags as rfim_clean (bit-exact for uint8), and oversize batches are refused.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_matches_rfim_clean_twice():
    import torch

    from paper_2001_03389_gb300 import build

    build.build()
    from paper_2001_03389_gb300 import rfim, synth

    torch.cuda.set_device(0)
    dev = torch.device("cuda:0")
    x = torch.from_numpy(synth.make_beams(synth.ARTS, beams=[0, 1])[:, :, :3001].copy()).to(dev)  # 2 x 1536 x 3001
    B, C, T = x.shape
    td = rfim.make_cut(3.0, 2, "median")
    fd = rfim.make_cut(3.0, 2, "median", 32)

    ctx = rfim.Context(0)
    ref = torch.empty_like(x)
    ref_mask = torch.zeros(rfim.mask_words(C, T, B), dtype=torch.int32, device=dev)
    ctx.clean(ctx.block(x, ref, ref_mask, "bct", "bits"), td, fd)
    torch.cuda.synchronize()
    ctx.close()

    for call in range(2):
        out = torch.full_like(x, 7)
        mask = torch.full((rfim.mask_words(C, T, B),), -1, dtype=torch.int32, device=dev)
        blk = rfim.Context.block(x, out, mask, "bct", "bits")
        st = rfim.rfim_clean_noalloc(ctypes.byref(blk), ctypes.byref(td), ctypes.byref(fd), None)
        assert st == rfim.OK, f"call {call}: status {st}"
        torch.cuda.synchronize()
        assert torch.equal(out, ref), f"call {call}: output differs from rfim_clean"
        assert torch.equal(mask, ref_mask), f"call {call}: mask differs from rfim_clean"

    # single-method calls through the same scratch
    out = torch.empty_like(x)
    blk = rfim.Context.block(x, out, None, "bct", None)
    assert rfim.rfim_clean_noalloc(ctypes.byref(blk), ctypes.byref(td), None, None) == rfim.OK
    torch.cuda.synchronize()
    ctx = rfim.Context(0)
    ref2 = torch.empty_like(x)
    ctx.tdsc(ctx.block(x, ref2), td)
    torch.cuda.synchronize()
    ctx.close()
    assert torch.equal(out, ref2)


@pytest.mark.parametrize("dtype", ["u8", "f32"])
def test_noalloc_fused_long_rows_twice(dtype):
    # Rows longer than ~3,150 samples take the fused schedule (one launch whose
    # FDSC items wait for their beam's TDSC rows through the shared counters):
    # whole ARTS beams (uint8) and float32 blocks, two calls in a row, each equal
    # to rfim_clean (uint8 bit for bit; float32 too, as both calls run the same
    # kernels on the same data).  The status query reads no timeout.
    import torch

    from paper_2001_03389_gb300 import build

    build.build()
    from paper_2001_03389_gb300 import rfim, synth

    torch.cuda.set_device(0)
    dev = torch.device("cuda:0")
    if dtype == "u8":
        x = torch.from_numpy(synth.make_beams(synth.ARTS, beams=[2, 3])).to(dev)  # 2 x 1536 x 12500
        td = rfim.make_cut(3.0, 2, "median")
        fd = rfim.make_cut(3.0, 2, "median", 32)
    else:
        g = torch.Generator(device=dev)
        g.manual_seed(7)
        x = synth.torch_beam_f32(g, 512, 4100, synth.fp32_model(), dev)[None].repeat(2, 1, 1)  # 2 x 512 x 4100
        td = rfim.make_cut(2.5, 3, "mean")
        fd = rfim.make_cut(2.5, 3, "mean", 32)
    B, C, T = x.shape
    ctx = rfim.Context(0)
    ref = torch.empty_like(x)
    ref_mask = torch.zeros(rfim.mask_words(C, T, B), dtype=torch.int32, device=dev)
    ctx.clean(ctx.block(x, ref, ref_mask, "bct", "bits"), td, fd)
    torch.cuda.synchronize()
    ctx.close()
    for call in range(2):
        out = torch.full_like(x, 3)
        mask = torch.full((rfim.mask_words(C, T, B),), -1, dtype=torch.int32, device=dev)
        blk = rfim.Context.block(x, out, mask, "bct", "bits")
        st = rfim.rfim_clean_noalloc(ctypes.byref(blk), ctypes.byref(td), ctypes.byref(fd), None)
        assert st == rfim.OK, f"call {call}: status {st}"
        assert rfim.rfim_noalloc_status(None) == rfim.OK
        assert torch.equal(out, ref), f"call {call}: output differs from rfim_clean"
        assert torch.equal(mask, ref_mask), f"call {call}: mask differs from rfim_clean"


def test_noalloc_rejects_oversize_batch():
    import torch

    from paper_2001_03389_gb300 import rfim

    n = rfim.RFIM_NOALLOC_MAX_BEAMS + 1 if hasattr(rfim, "RFIM_NOALLOC_MAX_BEAMS") else 161
    x = torch.zeros((n, 2, 64), dtype=torch.uint8, device="cuda:0")
    out = torch.empty_like(x)
    blk = rfim.Context.block(x, out)
    cut = rfim.make_cut(3.0)
    assert rfim.rfim_clean_noalloc(ctypes.byref(blk), ctypes.byref(cut), None, None) == rfim.ERR_RANGE
