"""GPU parity of random replacement (Sec. IV, last paragraph) against the oracle.

A flagged sample takes the value of an unflagged sample of its row (TDSC) or
bin (FDSC), drawn by the counter-based rule both sides implement from its
definition (SplitMix64 output function over beam, line, index, method,
iteration and attempt).  uint8: bit-exact, values and masks.  float32: the
margin tolerance of the float32 tests; a sample both sides replace holds the
same copied value.
"""
import numpy as np
import pytest

from gpu_util import noise_u8, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch  # noqa: F401

    from paper_2001_03389_gb300 import build

    build.build()
    from paper_2001_03389_gb300 import rfim

    c = rfim.Context(0)
    yield c
    c.close()


def check_u8(oracle, ctx, x, td=None, fd=None, order="blocked", mask_fmt="bits", **kw):
    layout = kw.get("layout", "bct")
    want, wf = oracle.clean(x, layout, tdsc=td, fdsc=fd, order=order)
    got, gf = run_gpu(ctx, x, tdsc=td, fdsc=fd, mask_fmt=mask_fmt, **kw)
    bad = np.argwhere(got != want)
    assert bad.size == 0, f"{len(bad)} samples differ, first at {bad[:3].tolist()}"
    if mask_fmt == "bits":
        assert np.array_equal(gf, wf > 0), f"mask differs at {np.argwhere(gf != (wf > 0))[:3].tolist()}"
    elif mask_fmt == "bytes":
        assert np.array_equal(gf, wf), f"byte mask differs at {np.argwhere(gf != wf)[:3].tolist()}"
    return want, wf


def rfi_u8(rng, shape, frac=0.03):
    """Noise with a few percent of bright samples, so that rows and bins have flags."""
    x = noise_u8(rng, shape, rfi=False)
    flat = x.reshape(-1)
    idx = rng.integers(0, flat.size, max(1, int(flat.size * frac)))
    flat[idx] = rng.integers(220, 256, idx.size).astype(np.uint8)
    return x


# warp rows, CTA rows (from 10210 samples: more than 640 chunks), ragged ends,
# the longest staged row, and rows beyond the stage (flag bitmaps, rows read
# from memory) up to the longest uint8 row
@pytest.mark.parametrize("C,T", [(1, 1), (3, 5), (7, 31), (37, 32), (64, 100), (100, 257), (33, 4099),
                                 (5, 10209), (4, 10210), (3, 12500), (2, 25000), (1, 78609), (1, 78610),
                                 (2, 100003), (1, 372181)])
def test_tdsc_random_u8(oracle, ctx, C, T):
    rng = np.random.default_rng(C * 7919 + T)
    x = rfi_u8(rng, (2, C, T))
    for it, k in [(1, 3.0), (3, 2.0)]:
        want, wf = check_u8(oracle, ctx, x, td=dict(k=k, iterations=it, replace="random"), api="tdsc")
    if x.size > 1000:
        assert (wf & 1).any()


# fast 32-channel bins, word bins, byte bins, ragged last bins, bins of one channel
@pytest.mark.parametrize("C,T,bin", [(1, 40, 1), (4, 33, 4), (32, 64, 32), (37, 70, 32), (64, 31, 7),
                                     (100, 50, 3), (96, 97, 32), (130, 200, 16), (1536, 40, 32), (200, 33, 200)])
def test_fdsc_random_u8(oracle, ctx, C, T, bin):
    rng = np.random.default_rng(C * 31 + T * 7 + bin)
    x = rfi_u8(rng, (2, C, T))
    for it, k in [(1, 3.0), (2, 2.0)]:
        check_u8(oracle, ctx, x, fd=dict(k=k, iterations=it, replace="random", bin=bin), api="fdsc")


@pytest.mark.parametrize("mask_fmt", ["bits", "bytes"])
def test_clean_random_u8(oracle, ctx, mask_fmt):
    rng = np.random.default_rng(5)
    x = rfi_u8(rng, (3, 96, 1000))
    td = dict(k=2.5, iterations=2, replace="random")
    fd = dict(k=2.5, iterations=2, replace="random", bin=32)
    check_u8(oracle, ctx, x, td=td, fd=fd, mask_fmt=mask_fmt)
    # random in one method only
    check_u8(oracle, ctx, x, td=td, fd=dict(fd, replace="median"), mask_fmt=mask_fmt)
    check_u8(oracle, ctx, x, td=dict(td, replace="mean"), fd=fd, mask_fmt=mask_fmt)


def test_random_u8_misaligned_in_place_btc(oracle, ctx):
    rng = np.random.default_rng(6)
    td = dict(k=2.5, iterations=2, replace="random")
    fd = dict(k=2.5, iterations=2, replace="random", bin=16)
    x = rfi_u8(rng, (2, 70, 333))
    check_u8(oracle, ctx, x, td=td, fd=fd, in_off=3, out_off=5)
    check_u8(oracle, ctx, x, td=td, fd=fd, in_place=True, in_off=1)
    xb = rfi_u8(rng, (2, 333, 70))
    check_u8(oracle, ctx, xb, td=td, fd=fd, layout="btc")


def test_random_u8_interleaved(oracle, ctx):
    rng = np.random.default_rng(7)
    x = rfi_u8(rng, (2, 64, 700))
    td = dict(k=2.5, iterations=3, replace="random")
    fd = dict(k=2.5, iterations=3, replace="random", bin=32)
    try:
        ctx.set_option("order", 1)
        check_u8(oracle, ctx, x, td=td, fd=fd, order="interleaved")
    finally:
        ctx.set_option("order", 0)


def test_random_u8_full_beam(oracle, ctx):
    # two whole beams of the ARTS batch (1536 x 12500), both methods random
    from paper_2001_03389_gb300 import synth

    x = synth.make_beams(synth.ARTS, beams=[0, 7])
    spec = synth.WORKLOADS[synth.ARTS]
    td = dict(spec["tdsc"], replace="random")
    fd = dict(spec["fdsc"], replace="random")
    want, wf = check_u8(oracle, ctx, x, td=td, fd=fd)
    assert (wf & 1).any() and (wf & 2).any()


def test_random_row_limits(ctx):
    import torch

    from paper_2001_03389_gb300 import rfim

    # uint8: random replacement reaches the exactness bound of every uint8 row
    x = torch.zeros((1, 1, 372182), dtype=torch.uint8, device="cuda:0")
    with pytest.raises(rfim.RfimError) as e:
        ctx.tdsc(ctx.block(x, torch.empty_like(x)), rfim.make_cut(3.0, replace="random"))
    assert e.value.status == rfim.ERR_RANGE
    # float32: rows beyond the stage keep two flag bitmaps in shared memory
    y = torch.zeros((1, 1, 921600), dtype=torch.float32, device="cuda:0")
    ctx.tdsc(ctx.block(y, torch.empty_like(y)), rfim.make_cut(3.0, replace="random"))
    torch.cuda.synchronize()
    y = torch.zeros((1, 1, 921601), dtype=torch.float32, device="cuda:0")
    with pytest.raises(rfim.RfimError) as e:
        ctx.tdsc(ctx.block(y, torch.empty_like(y)), rfim.make_cut(3.0, replace="random"))
    assert e.value.status == rfim.ERR_ARG
    assert ctx.device_status() == rfim.OK


@pytest.mark.parametrize("mask_fmt", ["bits", "bytes"])
def test_random_long_rows_misaligned_in_place(oracle, ctx, mask_fmt):
    # rows beyond the stage: misaligned input and output, in place, both mask
    # formats, and the fused launch with FDSC after them
    rng = np.random.default_rng(404)
    x = rfi_u8(rng, (2, 3, 100003))
    td = dict(k=2.5, iterations=3, replace="random")
    check_u8(oracle, ctx, x, td=td, mask_fmt=mask_fmt, in_off=5, out_off=11, api="tdsc")
    check_u8(oracle, ctx, x, td=td, mask_fmt=mask_fmt, in_place=True, in_off=3, api="tdsc")
    check_u8(oracle, ctx, x, td=td, fd=dict(k=2.5, iterations=2, replace="random", bin=3), mask_fmt=mask_fmt)
    if mask_fmt == "bits":  # (the float32 checker reads bit masks)
        y = chi2_f32(rng, (2, 3, 60001))
        check_f32(oracle, ctx, y, td=td, in_place=True, api="tdsc")
        check_f32(oracle, ctx, y, td=td, fd=dict(k=2.5, iterations=2, replace="random", bin=3))


# ---- float32

MARGIN = 1e-9
REL = 1e-6


def check_f32(oracle, ctx, x, td=None, fd=None, **kw):
    want, wf, margin = oracle.clean_f32_margin(x, "bct", tdsc=td, fdsc=fd)
    got, gf = run_gpu(ctx, x, tdsc=td, fdsc=fd, **kw)
    wflag = wf > 0
    dis = gf != wflag
    bad = dis & ~(margin <= MARGIN)
    assert not bad.any(), f"{int(bad.sum())} mask disagreements away from the threshold"
    ok = np.ones_like(wflag)
    for b, c, t in np.argwhere(dis):  # a disagreement changes its row's and column's draws
        ok[b, c, :] = False
        ok[b, :, t] = False
    keep = ok & ~wflag & ~gf
    assert np.array_equal(got[keep].view(np.uint32), x[keep].view(np.uint32)), "unflagged samples changed"
    both = ok & wflag & gf
    err = np.abs(got[both].astype(np.float64) - want[both].astype(np.float64))
    assert np.all(err <= REL * np.maximum(np.abs(want[both].astype(np.float64)), 1e-30)), "replaced values differ"
    return int(dis.sum()), wf


def chi2_f32(rng, shape):
    x = (rng.standard_exponential(shape) * 2.0).astype(np.float32)
    flat = x.reshape(-1)
    idx = rng.integers(0, flat.size, max(1, flat.size // 30))
    flat[idx] *= 8.0
    return x


@pytest.mark.parametrize("C,T", [(1, 1), (3, 7), (17, 129), (64, 1000), (5, 12500), (2, 40000), (1, 52001),
                                 (2, 150000)])
def test_tdsc_random_f32(oracle, ctx, C, T):
    rng = np.random.default_rng(C + 13 * T)
    x = chi2_f32(rng, (2, C, T))
    for it, k in [(1, 3.0), (3, 2.0)]:
        nd, wf = check_f32(oracle, ctx, x, td=dict(k=k, iterations=it, replace="random"), api="tdsc")
        assert nd <= max(2, x.size // 100000)


@pytest.mark.parametrize("C,T,bin", [(4, 9, 4), (64, 33, 32), (100, 20, 7), (1536, 16, 32), (200, 9, 200)])
def test_fdsc_random_f32(oracle, ctx, C, T, bin):
    rng = np.random.default_rng(C + 7 * T + bin)
    x = chi2_f32(rng, (2, C, T))
    for it, k in [(1, 3.0), (2, 2.0)]:
        nd, wf = check_f32(oracle, ctx, x, fd=dict(k=k, iterations=it, replace="random", bin=bin), api="fdsc")
        assert nd <= max(2, x.size // 100000)


def test_clean_random_f32(oracle, ctx):
    rng = np.random.default_rng(9)
    x = chi2_f32(rng, (2, 96, 700))
    nd, wf = check_f32(oracle, ctx, x, td=dict(k=2.5, iterations=2, replace="random"),
                       fd=dict(k=2.5, iterations=2, replace="random", bin=32))
    assert (wf & 1).any() and (wf & 2).any()


def test_random_through_batch_graph_and_noalloc(oracle, ctx):
    # the draws are keyed by the beam's index within its block: a ragged batch
    # of one-beam blocks and one three-beam block, eager, captured, replayed and
    # autotuned, and the allocation-free entry point, all match the oracle
    import ctypes

    import torch

    from gpu_util import unpack_bits
    from paper_2001_03389_gb300 import rfim

    rng = np.random.default_rng(21)
    td = dict(k=2.5, iterations=2, replace="random")
    fd = dict(k=2.5, iterations=2, replace="random", bin=32)
    xs = [rfi_u8(rng, (1, 384, 1000)), rfi_u8(rng, (3, 96, 2500)), rfi_u8(rng, (1, 768, 13001)),
          rfi_u8(rng, (1, 64, 333))]
    wants = [oracle.clean(x, "bct", tdsc=td, fdsc=fd) for x in xs]
    dev = torch.device("cuda:0")
    tdc, fdc = rfim.make_cut(**td), rfim.make_cut(**fd)
    for flags in (0, rfim.BATCH_GRAPH, rfim.BATCH_GRAPH, rfim.BATCH_AUTOTUNE | rfim.BATCH_GRAPH):
        ins = [torch.from_numpy(x).to(dev) for x in xs]
        outs = [torch.full_like(x, 0x5A) for x in ins]
        masks = [torch.full((rfim.mask_words(x.shape[1], x.shape[2], x.shape[0]),), -1, dtype=torch.int32,
                            device=dev) for x in ins]
        blks = [rfim.Context.block(i, o, m, "bct", "bits") for i, o, m in zip(ins, outs, masks)]
        ctx.clean_batch(blks, tdc, fdc, flags=flags)
        torch.cuda.synchronize()
        for x, o, m, (want, wf) in zip(xs, outs, masks, wants):
            B, C, T = x.shape
            assert np.array_equal(o.cpu().numpy(), want), (flags, x.shape)
            assert np.array_equal(unpack_bits(m.cpu().numpy(), B * C, T).reshape(x.shape), wf > 0), (flags, x.shape)
    assert ctx.device_status() == rfim.OK
    # allocation-free entry point, the three-beam block
    x, (want, wf) = xs[1], wants[1]
    xin = torch.from_numpy(x).to(dev)
    out = torch.full_like(xin, 7)
    mask = torch.full((rfim.mask_words(x.shape[1], x.shape[2], x.shape[0]),), -1, dtype=torch.int32, device=dev)
    blk = rfim.Context.block(xin, out, mask, "bct", "bits")
    assert rfim.rfim_clean_noalloc(ctypes.byref(blk), ctypes.byref(tdc), ctypes.byref(fdc), None) == rfim.OK
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), want)
    assert np.array_equal(unpack_bits(mask.cpu().numpy(), x.shape[0] * x.shape[1], x.shape[2]).reshape(x.shape),
                          wf > 0)


def test_random_f32_btc(oracle, ctx):
    # float32 BTC blocks go through the BCT scratch: the draws keep the beam,
    # channel and sample indices of the block
    rng = np.random.default_rng(31)
    x = np.ascontiguousarray(chi2_f32(rng, (2, 96, 300)).transpose(0, 2, 1))  # (B, T, C)
    td = dict(k=2.5, iterations=2, replace="random")
    fd = dict(k=2.5, iterations=2, replace="random", bin=32)
    want, wf, margin = oracle.clean_f32_margin(x, "btc", tdsc=td, fdsc=fd)
    got, gf = run_gpu(ctx, x, layout="btc", tdsc=td, fdsc=fd)
    dis = gf != (wf > 0)
    assert not (dis & ~(margin <= MARGIN)).any()
    if not dis.any():
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
