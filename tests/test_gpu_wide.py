"""FDSC on columns wider than the on-chip tile (Sec. IV, FDSC paragraph).

Such beams clean their columns one time sample at a time (the column gathered
into shared memory); the results must be those of the oracle: bit-exact for
uint8, within the float32 margin tolerance for float32.  Shapes: 32-channel
bins over 20,000 and 30,000 channels, two-channel bins over several thousand
channels, ragged last bins, every replacement, both mask formats, FDSC alone
and after TDSC in the fused launch.
"""
import numpy as np
import pytest

from gpu_util import noise_u8, run_gpu

pytestmark = pytest.mark.gpu

MARGIN = 1e-9


@pytest.fixture(scope="module")
def ctx():
    from paper_2001_03389_gb300 import build

    build.build()
    from paper_2001_03389_gb300 import rfim

    c = rfim.Context(0)
    yield c
    c.close()


def rfi_cols_u8(rng, shape):
    """Noise with bright channels and samples, so that wide columns carry flags."""
    x = noise_u8(rng, shape, rfi=False)
    B, C, T = shape
    ch = rng.integers(0, C, max(1, C // 50))
    x[:, ch, :] = np.clip(x[:, ch, :].astype(np.int32) + 70, 0, 255).astype(np.uint8)
    flat = x.reshape(-1)
    idx = rng.integers(0, flat.size, flat.size // 200)
    flat[idx] = 250
    return x


def check_u8(oracle, ctx, x, td, fd, mask_fmt="bits", api="clean"):
    want, wf = oracle.clean(x, "bct", tdsc=td, fdsc=fd)
    got, gf = run_gpu(ctx, x, tdsc=td, fdsc=fd, mask_fmt=mask_fmt, api=api)
    bad = np.argwhere(got != want)
    assert bad.size == 0, f"{len(bad)} samples differ, first at {bad[:3].tolist()}"
    if mask_fmt == "bits":
        assert np.array_equal(gf, wf > 0)
    else:
        assert np.array_equal(gf, wf)
    return wf


@pytest.mark.parametrize("C,T,bin", [(20000, 70, 32), (20007, 33, 32), (6000, 40, 2), (9001, 36, 7)])
@pytest.mark.parametrize("rep", ["median", "mean", "random"])
def test_wide_fdsc_u8(oracle, ctx, C, T, bin, rep):
    rng = np.random.default_rng(C + T + bin)
    x = rfi_cols_u8(rng, (2, C, T))
    fd = dict(k=2.5, iterations=2, replace=rep, bin=bin)
    wf = check_u8(oracle, ctx, x, None, fd, api="fdsc")
    assert (wf & 2).any()


@pytest.mark.parametrize("mask_fmt", ["bits", "bytes"])
def test_wide_clean_u8(oracle, ctx, mask_fmt):
    # TDSC then FDSC in one launch (rows of 3,300 samples take warps, so the
    # launch is fused): the FDSC items wait for their beam's rows
    rng = np.random.default_rng(77)
    x = rfi_cols_u8(rng, (2, 16500, 3300))
    wf = check_u8(oracle, ctx, x, dict(k=3.0, iterations=2, replace="median"),
                  dict(k=3.0, iterations=2, replace="median", bin=32), mask_fmt=mask_fmt)
    assert (wf & 1).any() and (wf & 2).any()


def test_wide_btc_and_interleaved_u8(oracle, ctx):
    # tall columns through the BTC scratch copy, and in the interleaved order
    # (one iteration of each method per round, single-iteration launches)
    rng = np.random.default_rng(91)
    x = rfi_cols_u8(rng, (2, 16000, 48))
    td = dict(k=2.5, iterations=2, replace="median")
    fd = dict(k=2.5, iterations=2, replace="median", bin=32)
    want, wf = oracle.clean(x, "bct", tdsc=td, fdsc=fd)
    xt = np.ascontiguousarray(x.transpose(0, 2, 1))
    got, gf = run_gpu(ctx, xt, layout="btc", tdsc=td, fdsc=fd, mask_fmt="bytes")
    assert np.array_equal(got.transpose(0, 2, 1), want)
    assert np.array_equal(gf.transpose(0, 2, 1), wf)
    try:
        ctx.set_option("order", 1)
        want, wf = oracle.clean(x, "bct", tdsc=td, fdsc=fd, order="interleaved")
        got, gf = run_gpu(ctx, x, tdsc=td, fdsc=fd)
        assert np.array_equal(got, want)
        assert np.array_equal(gf, wf > 0)
    finally:
        ctx.set_option("order", 0)


def check_f32(oracle, ctx, x, td, fd, api="clean"):
    want, wf, margin = oracle.clean_f32_margin(x, "bct", tdsc=td, fdsc=fd)
    got, gf = run_gpu(ctx, x, tdsc=td, fdsc=fd, api=api)
    wflag = wf > 0
    dis = gf != wflag
    assert not (dis & ~(margin <= MARGIN)).any(), "mask disagreements away from the threshold"
    # a disagreement changes its column's later statistics (and its row's, with TDSC)
    ok = np.ones_like(wflag)
    for b, c, t in np.argwhere(dis):
        ok[b, :, t] = False
        ok[b, c, :] = False
    keep = ok & ~wflag & ~gf
    assert np.array_equal(got[keep].view(np.uint32), x[keep].view(np.uint32))
    both = ok & wflag & gf
    err = np.abs(got[both].astype(np.float64) - want[both].astype(np.float64))
    assert np.all(err <= 1e-6 * np.maximum(np.abs(want[both].astype(np.float64)), 1e-30))
    return int(dis.sum()), wf


@pytest.mark.parametrize("C,T,bin", [(30000, 40, 32), (14000, 33, 2), (30011, 9, 64)])
@pytest.mark.parametrize("rep", ["mean", "median", "random"])
def test_wide_fdsc_f32(oracle, ctx, C, T, bin, rep):
    rng = np.random.default_rng(C * 3 + T + bin)
    x = (rng.standard_exponential((2, C, T)) * 2.0).astype(np.float32)
    x[:, rng.integers(0, C, C // 50), :] *= 6.0
    nd, wf = check_f32(oracle, ctx, x, None, dict(k=2.5, iterations=2, replace=rep, bin=bin), api="fdsc")
    assert nd <= max(2, x.size // 100000)
    assert (wf & 2).any()


def test_wide_clean_f32(oracle, ctx):
    rng = np.random.default_rng(78)
    x = (rng.standard_exponential((2, 30000, 64)) * 2.0).astype(np.float32)
    x[:, rng.integers(0, 30000, 600), :] *= 6.0
    nd, wf = check_f32(oracle, ctx, x, dict(k=2.5, iterations=2, replace="mean"),
                       dict(k=2.5, iterations=2, replace="mean", bin=32))
    assert nd <= max(2, x.size // 100000)
    assert (wf & 1).any() and (wf & 2).any()


def test_wide_limits(ctx):
    import torch

    from paper_2001_03389_gb300 import rfim

    x = torch.zeros((1, 120000, 8), dtype=torch.uint8, device="cuda:0")
    with pytest.raises(rfim.RfimError) as e:
        ctx.fdsc(ctx.block(x, torch.empty_like(x)), rfim.make_cut(3.0, bin=32))
    assert e.value.status == rfim.ERR_RANGE
    y = torch.zeros((1, 60000, 4), dtype=torch.float32, device="cuda:0")
    with pytest.raises(rfim.RfimError) as e:
        ctx.fdsc(ctx.block(y, torch.empty_like(y)), rfim.make_cut(3.0, bin=32))
    assert e.value.status == rfim.ERR_RANGE
    assert ctx.device_status() == rfim.OK
