"""Ragged batching: one persistent launch over beams of uneven shapes.

rfim_clean_batch must give, bit for bit, what separate rfim_clean calls give,
with and without CUDA-graph capture and with the autotuner; sampled beams are
also checked against the CPU oracle.  Shapes follow the ragged workload
(channel counts from {384, 768, 1536, 4096}, uneven sample counts), scaled so
that the oracle finishes in seconds.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2001_03389_gb300 import build

    build.build()
    from paper_2001_03389_gb300 import rfim

    c = rfim.Context(0)
    yield c
    c.close()


def _blocks(rfim, beams, mask_fmt="bits"):
    import torch

    outs, masks, blks = [], [], []
    for x in beams:
        C, T = x.shape
        out = torch.full_like(x, 0x5A)
        mask = torch.full((rfim.mask_words(C, T),), -1, dtype=torch.int32, device=x.device)
        outs.append(out)
        masks.append(mask)
        blks.append(rfim.Context.block(x[None], out[None], mask, "bct", mask_fmt))
    return outs, masks, blks


CUTS = dict(tdsc=dict(k=3.0, iterations=2, replace="median"), fdsc=dict(k=3.0, iterations=2, replace="median", bin=32))


def test_batch_equals_per_beam_and_oracle(ctx, oracle):
    import torch

    from gpu_util import unpack_bits
    from paper_2001_03389_gb300 import rfim, synth

    shapes = [(384, 1000), (768, 2500), (1536, 1333), (4096, 1200), (384, 3001), (768, 1021), (1536, 777),
              (4096, 515), (384, 25000), (768, 4096)]
    beams = synth.torch_ragged_batch(shapes, seed=synth.RAGGED_SEED, device="cuda:0")
    td, fd = rfim.make_cut(**CUTS["tdsc"]), rfim.make_cut(**CUTS["fdsc"])
    # reference: one rfim_clean per beam
    ref_o, ref_m, ref_b = _blocks(rfim, beams)
    for b in ref_b:
        ctx.clean(b, td, fd)
    torch.cuda.synchronize()
    for flags in (0, rfim.BATCH_GRAPH, rfim.BATCH_GRAPH, rfim.BATCH_AUTOTUNE | rfim.BATCH_GRAPH):
        o, m, b = _blocks(rfim, beams)
        ctx.clean_batch(b, td, fd, flags=flags)
        torch.cuda.synchronize()
        for i in range(len(beams)):
            assert torch.equal(o[i], ref_o[i]), (flags, i, shapes[i])
            assert torch.equal(m[i], ref_m[i]), (flags, i, shapes[i])
    assert ctx.device_status() == rfim.OK
    # oracle on three beams (a short, a 4096-channel and a 25000-sample one)
    for i in (0, 3, 8):
        x = beams[i].cpu().numpy()[None]
        want, wf = oracle.clean(x, "bct", tdsc=CUTS["tdsc"], fdsc=CUTS["fdsc"])
        C, T = shapes[i]
        assert np.array_equal(ref_o[i].cpu().numpy()[None], want), shapes[i]
        assert np.array_equal(unpack_bits(ref_m[i].cpu().numpy(), C, T)[None], wf > 0), shapes[i]


def test_batch_single_methods_and_byte_masks(ctx, oracle):
    import torch

    from paper_2001_03389_gb300 import rfim, synth

    shapes = [(96, 700), (130, 333), (64, 2048)]
    beams = synth.torch_ragged_batch(shapes, seed=7, device="cuda:0")
    for td, fd in ((CUTS["tdsc"], None), (None, dict(CUTS["fdsc"], bin=16))):
        o = [torch.empty_like(x) for x in beams]
        masks = [torch.zeros_like(x) for x in beams]
        b = [rfim.Context.block(x[None], oo[None], mm[None], "bct", "bytes") for x, oo, mm in zip(beams, o, masks)]
        ctx.clean_batch(b, td and rfim.make_cut(**td), fd and rfim.make_cut(**fd), flags=rfim.BATCH_GRAPH)
        torch.cuda.synchronize()
        for i, x in enumerate(beams):
            want, wf = oracle.clean(x.cpu().numpy()[None], "bct", tdsc=td, fdsc=fd)
            assert np.array_equal(o[i].cpu().numpy()[None], want)
            assert np.array_equal(masks[i].cpu().numpy()[None], wf)


def test_fdsc_channel_limit(ctx):
    import torch

    from paper_2001_03389_gb300 import rfim

    x = torch.zeros((1, 120000, 8), dtype=torch.uint8, device="cuda:0")  # beyond the column-at-a-time layout too
    with pytest.raises(rfim.RfimError) as e:
        ctx.fdsc(ctx.block(x, torch.empty_like(x)), rfim.make_cut(3.0, bin=32))
    assert e.value.status == rfim.ERR_RANGE


def test_batch_rejects_mixed_dtypes(ctx):
    import torch

    from paper_2001_03389_gb300 import rfim

    a = torch.zeros((1, 8, 64), dtype=torch.uint8, device="cuda:0")
    b = torch.zeros((1, 8, 64), dtype=torch.float32, device="cuda:0")
    blks = [rfim.Context.block(a, torch.empty_like(a)), rfim.Context.block(b, torch.empty_like(b))]
    with pytest.raises(rfim.RfimError):
        ctx.clean_batch(blks, rfim.make_cut(3.0), None)


def test_batch_graph_interleaved(ctx, oracle):
    # graph capture of interleaved rounds (two launches per round per beam group)
    import torch

    from gpu_util import unpack_bits
    from paper_2001_03389_gb300 import rfim, synth

    shapes = [(96, 700), (130, 333), (64, 2048)]
    beams = synth.torch_ragged_batch(shapes, seed=19, device="cuda:0")
    td = dict(k=2.5, iterations=3, replace="median")
    fd = dict(k=2.5, iterations=2, replace="mean", bin=32)
    try:
        ctx.set_option("order", 1)
        for _ in range(2):  # capture, then replay
            o, m, b = _blocks(rfim, beams)
            ctx.clean_batch(b, rfim.make_cut(**td), rfim.make_cut(**fd), flags=rfim.BATCH_GRAPH)
            torch.cuda.synchronize()
            for i, x in enumerate(beams):
                C, T = shapes[i]
                want, wf = oracle.clean(x.cpu().numpy()[None], "bct", tdsc=td, fdsc=fd, order="interleaved")
                assert np.array_equal(o[i].cpu().numpy()[None], want)
                assert np.array_equal(unpack_bits(m[i].cpu().numpy(), C, T)[None], wf > 0)
        assert ctx.device_status() == rfim.OK
    finally:
        ctx.set_option("order", 0)


def test_ragged_batch_full_size(ctx, oracle):
    # The ragged configuration at full size: 200 beams, C from {384, 768, 1536,
    # 4096}, T uniform in [1000, 25000] (4.16 GB), drawn on the device.
    # One graph-captured, autotuned rfim_clean_batch equals 200 separate
    # rfim_clean calls bit for bit (a replay too), and three beams -- the first,
    # the longest, and the shortest 4096-channel one -- equal the oracle.
    import torch

    from gpu_util import unpack_bits
    from paper_2001_03389_gb300 import rfim, synth

    shapes = synth.ragged_shapes(200)
    beams = synth.torch_ragged_batch(shapes, seed=synth.RAGGED_SEED, device="cuda:0")
    assert sum(c * t for c, t in shapes) > 4e9
    td, fd = rfim.make_cut(**CUTS["tdsc"]), rfim.make_cut(**CUTS["fdsc"])
    ref_o, ref_m, ref_b = _blocks(rfim, beams)
    for b in ref_b:
        ctx.clean(b, td, fd)
    torch.cuda.synchronize()
    for _ in range(2):  # capture (after tuning), then replay
        o, m, b = _blocks(rfim, beams)
        ctx.clean_batch(b, td, fd, flags=rfim.BATCH_GRAPH | rfim.BATCH_AUTOTUNE)
        torch.cuda.synchronize()
        for i in range(len(beams)):
            assert torch.equal(o[i], ref_o[i]), (i, shapes[i])
            assert torch.equal(m[i], ref_m[i]), (i, shapes[i])
        del o, m, b
    assert ctx.device_status() == rfim.OK
    longest = max(range(200), key=lambda i: shapes[i][1])
    wide = min((i for i in range(200) if shapes[i][0] == 4096), key=lambda i: shapes[i][1])
    for i in (0, longest, wide):
        C, T = shapes[i]
        x = beams[i].cpu().numpy()[None]
        want, wf = oracle.clean(x, "bct", tdsc=CUTS["tdsc"], fdsc=CUTS["fdsc"])
        assert np.array_equal(ref_o[i].cpu().numpy()[None], want), shapes[i]
        assert np.array_equal(unpack_bits(ref_m[i].cpu().numpy(), C, T)[None], wf > 0), shapes[i]
