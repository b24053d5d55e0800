"""GPU parity of the float32 path against the CPU oracle.

Tolerance (float32): a mask disagreement is allowed only where the oracle's
decision lies within 1e-9 relative of its threshold, |(|x - mu| - k sigma)| <=
1e-9 k sigma (the oracle reports that distance per sample); such
disagreements are counted (tests/conftest.py prints the tally).  Samples
neither side flags must be bit-identical to the input; samples both sides
replace must agree within 1e-6 relative.

A disagreement changes the later statistics of its own row (TDSC) or column
(FDSC) only, so the value checks leave out just that row or column.  A fused
clean (TDSC then FDSC) is checked method by method: the library's TDSC output
against the oracle's TDSC on the input (rows), the library's FDSC of that
output against the oracle's FDSC of the same output (columns), and the fused
launch against the two separate launches, bit for bit.
"""
import numpy as np
import pytest

from conftest import F32_TALLY
from gpu_util import run_gpu

pytestmark = pytest.mark.gpu

MARGIN = 1e-9
REL = 1e-6


@pytest.fixture(scope="module")
def ctx():
    import torch  # noqa: F401

    from paper_2001_03389_gb300 import build

    build.build()
    from paper_2001_03389_gb300 import rfim

    c = rfim.Context(0)
    yield c
    c.close()


def _gpu_flags(got, gf, x, mask_fmt):
    if mask_fmt == "bits":
        return gf
    if mask_fmt == "bytes":
        return gf > 0
    return got != x  # no mask: changed samples (a replaced value can equal the original)


def compare_f32(x, want, wf, margin, got, gflag, line_axes, mask_fmt="bits", byte_flags=None):
    """One method's output against the oracle's on the same input.  line_axes:
    the axes that index a line of that method (a disagreement excludes its
    line from the value checks).  Returns the number of mask disagreements."""
    wflag = wf > 0
    if mask_fmt is None:
        dis = np.zeros_like(wflag)
    elif byte_flags is not None:
        dis = byte_flags != wf
    else:
        dis = gflag != wflag
    nd = int(dis.sum())
    ok = np.ones_like(wflag)
    if nd:
        bad = dis & ~(margin <= MARGIN)
        assert not bad.any(), (f"{int(bad.sum())} mask disagreements farther than {MARGIN} from the threshold, "
                               f"first at {np.argwhere(bad)[:3].tolist()}, margins {margin[bad][:3]}")
        for idx in np.argwhere(dis):
            sel = tuple(int(idx[a]) if a in line_axes else slice(None) for a in range(3))
            ok[sel] = False
    keep = ok & ~wflag & ~gflag if mask_fmt is not None else ok & ~wflag
    assert np.array_equal(got[keep].view(np.uint32), x[keep].view(np.uint32)), "unflagged samples changed"
    both = ok & wflag & (gflag if mask_fmt is not None else True)
    if both.any():
        err = np.abs(got[both].astype(np.float64) - want[both].astype(np.float64))
        tol = REL * np.maximum(np.abs(want[both].astype(np.float64)), 1e-30)
        assert np.all(err <= tol), f"replaced values differ: max rel {np.max(err / tol) * REL:.3g}"
    F32_TALLY["checks"] += 1
    F32_TALLY["decisions"] += int(x.size)
    F32_TALLY["disagreements"] += nd
    return nd


def check_f32(oracle, ctx, x, td=None, fd=None, mask_fmt="bits", layout="bct", **kw):
    """Clean x on the GPU with the given cuts and check it against the oracle.
    Returns the number of (allowed) mask disagreements."""
    rows = (0, 1) if layout == "bct" else (0, 2)  # (beam, channel) indexes a TDSC row
    cols = (0, 2) if layout == "bct" else (0, 1)  # (beam, time) indexes an FDSC column
    api = kw.pop("api", "clean" if td and fd else ("tdsc" if td else "fdsc"))
    if td and fd and api == "clean":
        # the two methods one at a time, each on its own input
        got_t, bt = run_gpu(ctx, x, layout=layout, tdsc=td, mask_fmt="bytes", api="tdsc")
        want_t, wft, mt = oracle.clean_f32_margin(x, layout, tdsc=td)
        nd = compare_f32(x, want_t, wft, mt, got_t, bt > 0, rows, "bytes", byte_flags=bt)
        got_f, bf = run_gpu(ctx, got_t, layout=layout, fdsc=fd, mask_fmt="bytes", api="fdsc")
        want_f, wff, mf = oracle.clean_f32_margin(got_t, layout, fdsc=fd)
        nd += compare_f32(got_t, want_f, wff, mf, got_f, bf > 0, cols, "bytes", byte_flags=bf)
        # the fused launch equals the two launches
        got, gf = run_gpu(ctx, x, layout=layout, tdsc=td, fdsc=fd, mask_fmt=mask_fmt, **kw)
        assert np.array_equal(got.view(np.uint32), got_f.view(np.uint32)), "fused clean differs from TDSC then FDSC"
        if mask_fmt == "bits":
            assert np.array_equal(gf, (bt | bf) > 0)
        elif mask_fmt == "bytes":
            assert np.array_equal(gf, bt | bf)
        return nd
    want, wf, margin = oracle.clean_f32_margin(x, layout, tdsc=td, fdsc=fd)
    got, gf = run_gpu(ctx, x, layout=layout, tdsc=td, fdsc=fd, mask_fmt=mask_fmt, api=api, **kw)
    return compare_f32(x, want, wf, margin, got, _gpu_flags(got, gf, x, mask_fmt), rows if td else cols, mask_fmt,
                       byte_flags=gf if mask_fmt == "bytes" else None)


def chi2_block(rng, B, C, T, gain=True):
    g = np.exp(rng.uniform(np.log(0.5), np.log(2.0), size=(B, C, 1))) if gain else np.ones((B, C, 1))
    x = (rng.standard_exponential((B, C, T)) * 2.0 * g).astype(np.float32)
    if x.size > 16:
        flat = x.reshape(-1)
        idx = rng.integers(0, flat.size, max(1, flat.size // 100))
        flat[idx] *= 6.0
        if C > 4:
            x[:, C // 3, :] += 8.0 * g[:, C // 3]  # a narrowband channel
    return x


@pytest.mark.parametrize("C,T", [(1, 1), (1, 5), (3, 7), (5, 33), (37, 64), (64, 100), (100, 257), (33, 1031),
                                 (4, 8192), (2, 20001)])
@pytest.mark.parametrize("rep", ["mean", "median"])
def test_tdsc_f32_shapes(oracle, ctx, C, T, rep):
    rng = np.random.default_rng(C * 1000 + T + 7)
    x = chi2_block(rng, 2, C, T)
    for it, k in [(1, 3.0), (3, 2.5)]:
        check_f32(oracle, ctx, x, td=dict(k=k, iterations=it, replace=rep), api="tdsc")


@pytest.mark.parametrize("C,T", [(1, 52001), (2, 100003)])
@pytest.mark.parametrize("rep", ["mean", "median"])
def test_tdsc_f32_long_rows(oracle, ctx, C, T, rep):
    # rows beyond the on-chip stage (52,000 samples): read from memory in every
    # pass, the earlier iterations replayed; misaligned, in place, byte masks
    rng = np.random.default_rng(C * 31 + T)
    x = chi2_block(rng, 2, C, T)
    for it, k in [(1, 3.0), (3, 2.5)]:
        check_f32(oracle, ctx, x, td=dict(k=k, iterations=it, replace=rep), api="tdsc")
    td = dict(k=2.5, iterations=2, replace=rep)
    check_f32(oracle, ctx, x, td=td, fd=dict(k=2.5, iterations=2, replace="mean", bin=C), in_off=4, out_off=12)
    check_f32(oracle, ctx, x, td=td, api="tdsc", in_place=True, in_off=8)
    check_f32(oracle, ctx, x, td=td, api="tdsc", mask_fmt="bytes")


@pytest.mark.parametrize("C,T,bin", [(1, 40, 1), (4, 33, 4), (32, 64, 32), (37, 70, 32), (64, 31, 7),
                                     (100, 50, 3), (130, 96, 32), (96, 40, 96), (4096, 40, 32), (257, 33, 16)])
@pytest.mark.parametrize("rep", ["mean", "median"])
def test_fdsc_f32_shapes(oracle, ctx, C, T, bin, rep):
    rng = np.random.default_rng(C * 7 + T + bin)
    x = chi2_block(rng, 2, C, T)
    for it, k in [(1, 3.0), (3, 2.5)]:
        check_f32(oracle, ctx, x, fd=dict(k=k, iterations=it, replace=rep, bin=bin), api="fdsc")


@pytest.mark.parametrize("C,T", [(64, 2048), (100, 777), (1536, 96), (48, 5003)])
def test_clean_f32_fused(oracle, ctx, C, T):
    rng = np.random.default_rng(C + T)
    x = chi2_block(rng, 3, C, T)
    for rep in ("mean", "median"):
        td = dict(k=2.5, iterations=3, replace=rep)
        fd = dict(k=2.5, iterations=3, replace=rep, bin=32)
        check_f32(oracle, ctx, x, td=td, fd=fd)
        check_f32(oracle, ctx, x, td=td, fd=fd, mask_fmt="bytes")
        check_f32(oracle, ctx, x, td=td, fd=fd, mask_fmt=None)


@pytest.mark.parametrize("in_off,out_off", [(4, 0), (12, 8), (8, 8), (0, 4)])
def test_f32_misaligned_and_in_place(oracle, ctx, in_off, out_off):
    rng = np.random.default_rng(in_off * 31 + out_off)
    x = chi2_block(rng, 2, 40, 301)
    td = dict(k=2.5, iterations=2, replace="median")
    fd = dict(k=2.5, iterations=2, replace="mean", bin=8)
    check_f32(oracle, ctx, x, td=td, fd=fd, in_off=in_off, out_off=out_off)
    check_f32(oracle, ctx, x, td=td, fd=fd, in_place=True, in_off=in_off)


def test_f32_value_distributions(oracle, ctx):
    rng = np.random.default_rng(77)
    td = dict(k=3.0, iterations=3, replace="mean")
    fd = dict(k=3.0, iterations=3, replace="mean", bin=32)
    cases = [
        rng.normal(128.0, 16.0, (2, 64, 500)),          # offset data, mean/sigma = 8
        rng.normal(0.0, 1.0, (2, 64, 500)),             # signed, zero mean
        rng.normal(1.0e4, 1.0, (1, 64, 300)),           # mean/sigma = 1e4: the FP64 two-pass
        rng.standard_cauchy((1, 64, 300)) * 10.0,       # heavy tails
        np.round(rng.normal(100.0, 3.0, (1, 64, 300))),  # integer-valued with ties
    ]
    for x in cases:
        check_f32(oracle, ctx, x.astype(np.float32), td=td, fd=fd)
        check_f32(oracle, ctx, x.astype(np.float32), td=dict(td, replace="median"), fd=dict(fd, replace="median"))


def test_f32_degenerate(oracle, ctx):
    x = np.full((1, 16, 64), 2.5, np.float32)
    check_f32(oracle, ctx, x, td=dict(k=3.0, iterations=3), fd=dict(k=3.0, iterations=3, bin=4))
    x = np.zeros((1, 8, 40), np.float32)
    check_f32(oracle, ctx, x, td=dict(k=1.0, iterations=2), fd=dict(k=1.0, iterations=2, bin=8))
    x = np.tile(np.array([-1.0, 1.0], np.float32), (1, 6, 20))
    check_f32(oracle, ctx, x, td=dict(k=0.5, iterations=2, replace="median"), fd=dict(k=0.6, iterations=2, bin=2))
    x = np.zeros((1, 4, 10), np.float32)
    x[0, :, 3] = -0.0
    x[0, 1, :] = 7.0
    check_f32(oracle, ctx, x, td=dict(k=0.3, iterations=2, replace="median"), fd=dict(k=0.4, iterations=2, bin=2))


def test_f32_many_k(oracle, ctx):
    rng = np.random.default_rng(5)
    x = chi2_block(rng, 1, 24, 600)
    for k in (0.3, 0.999, 1.0, 1.5, 2.0, 2.5, 3.25, 4.0, 7.5, 100.0):
        check_f32(oracle, ctx, x, td=dict(k=k, iterations=2, replace="median"), fd=dict(k=k, iterations=2, bin=5))


@pytest.mark.parametrize("k", [1e-300, 1e-40, 1e-12, 1e-3, 5e5, 2e6, 1e39, 1e300])
def test_f32_extreme_k(oracle, ctx, k):
    rng = np.random.default_rng(int(abs(np.log10(k))) + 5)
    x = chi2_block(rng, 2, 40, 300)
    x[0, 3, :] = 1.5  # constant row
    for rep in ("mean", "median"):
        check_f32(oracle, ctx, x, td=dict(k=k, iterations=2, replace=rep), fd=dict(k=k, iterations=2, replace=rep,
                                                                                  bin=16))


def test_fp32_workload_full_beam(oracle, ctx):
    # one full beam of the float32 configuration: 4096 x 8192, fused, k = 2.5, 3 iterations, mean
    from paper_2001_03389_gb300 import synth

    spec = synth.WORKLOADS[synth.FP32]
    x = synth.make_beams(synth.FP32, beams=[0])
    nd = check_f32(oracle, ctx, x, td=spec["tdsc"], fd=spec["fdsc"])
    print(f"float32 workload, beam 0: {nd} allowed mask disagreements")


def test_fp32_workload_full_launch_sampled(oracle, ctx):
    # The float32 configuration at full size, in the launch the benchmark times:
    # 32 beams x 4096 channels x 8192 samples drawn on the device, one fused
    # rfim_clean (k = 2.5, 3 iterations, mean).  Beams 0 and 31 of that launch
    # equal TDSC then FDSC launched on the beam alone, bit for bit, and those
    # two launches match the oracle within the float32 tolerance.
    import torch

    from gpu_util import unpack_bits
    from paper_2001_03389_gb300 import rfim, synth

    spec = synth.WORKLOADS[synth.FP32]
    dev = torch.device("cuda:0")
    xin = synth.torch_make_beams(synth.FP32, spec["B"], synth.seed_of(synth.FP32), dev)
    B, C, T = xin.shape
    out = torch.empty_like(xin)
    mask = torch.zeros(rfim.mask_words(C, T, B), dtype=torch.int32, device=dev)
    ctx.clean(ctx.block(xin, out, mask, "bct", "bits"), spec["tdsc"], spec["fdsc"])
    torch.cuda.synchronize()
    assert ctx.device_status() == rfim.OK
    nd = 0
    for b in (0, B - 1):
        x = xin[b:b + 1].cpu().numpy()
        got = out[b:b + 1].cpu().numpy()
        gm = unpack_bits(mask.view(B, -1)[b].cpu().numpy(), C, T)[None]
        got_t, bt = run_gpu(ctx, x, tdsc=spec["tdsc"], mask_fmt="bytes", api="tdsc")
        got_f, bf = run_gpu(ctx, got_t, fdsc=spec["fdsc"], mask_fmt="bytes", api="fdsc")
        assert np.array_equal(got.view(np.uint32), got_f.view(np.uint32)), b
        assert np.array_equal(gm, (bt | bf) > 0), b
        want_t, wft, mt = oracle.clean_f32_margin(x, "bct", tdsc=spec["tdsc"])
        nd += compare_f32(x, want_t, wft, mt, got_t, bt > 0, (0, 1), "bytes", byte_flags=bt)
        want_f, wff, mf = oracle.clean_f32_margin(got_t, "bct", fdsc=spec["fdsc"])
        nd += compare_f32(got_t, want_f, wff, mf, got_f, bf > 0, (0, 2), "bytes", byte_flags=bf)
    print(f"float32 workload, beams 0 and {B - 1} of the full launch: {nd} allowed mask disagreements")
    assert nd <= 4


@pytest.mark.parametrize("rep", ["mean", "median"])
def test_f32_cut_records(oracle, ctx, rep):
    # Option f32_records: fused TDSC rows record their cuts instead of writing
    # the row, and FDSC items replay them on the input.  The fused launch must
    # equal TDSC then FDSC launched separately (bit for bit), in place and
    # misaligned too, with rows beyond the stage among them.
    rng = np.random.default_rng(3)
    try:
        ctx.set_option("f32_records", 1)
        for C, T in [(64, 2048), (130, 333), (3, 52003)]:
            x = chi2_block(rng, 2, C, T)
            td = dict(k=2.5, iterations=3, replace=rep)
            fd = dict(k=2.5, iterations=2, replace="mean", bin=min(32, C))
            check_f32(oracle, ctx, x, td=td, fd=fd)
            check_f32(oracle, ctx, x, td=td, fd=fd, in_place=True, in_off=4)
            check_f32(oracle, ctx, x, td=dict(td, iterations=5), fd=fd, in_off=8, out_off=12)
    finally:
        ctx.set_option("f32_records", 0)


def test_f32_tile_widths(oracle, ctx):
    rng = np.random.default_rng(21)
    x = chi2_block(rng, 2, 300, 203)
    td = dict(k=2.5, iterations=2, replace="mean")
    fd = dict(k=2.5, iterations=2, replace="mean", bin=32)
    try:
        for ws in (8, 4, 2, 1):
            ctx.set_option("tile_samples", ws)
            check_f32(oracle, ctx, x, td=td, fd=fd)
        ctx.set_option("tile_samples", 0)
        for sch in (1, 2):
            ctx.set_option("schedule", sch)
            check_f32(oracle, ctx, x, td=td, fd=fd)
    finally:
        ctx.set_option("tile_samples", 0)
        ctx.set_option("schedule", 0)


def test_f32_validation(ctx):
    import torch

    from paper_2001_03389_gb300 import rfim

    row = torch.zeros((1, 1, 921601), dtype=torch.float32, device="cuda:0")
    with pytest.raises(rfim.RfimError) as e:  # random replacement: the row's flag bitmaps do not fit
        ctx.tdsc(ctx.block(row, torch.empty_like(row)), rfim.make_cut(3.0, replace="random"))
    assert e.value.status == rfim.ERR_ARG
    big = torch.zeros((1, 60000, 4), dtype=torch.float32, device="cuda:0")  # beyond the column-at-a-time layout too
    with pytest.raises(rfim.RfimError) as e:
        ctx.fdsc(ctx.block(big, torch.empty_like(big)), rfim.make_cut(3.0, bin=32))
    assert e.value.status == rfim.ERR_RANGE


@pytest.mark.parametrize("C,T", [(3, 7), (40, 301), (96, 64), (257, 129)])
def test_f32_btc_layout(oracle, ctx, C, T):
    rng = np.random.default_rng(C + 5 * T)
    xb = chi2_block(rng, 2, C, T)
    x = np.ascontiguousarray(xb.transpose(0, 2, 1))
    td = dict(k=2.5, iterations=3, replace="mean")
    fd = dict(k=2.5, iterations=3, replace="median", bin=min(32, C))
    for kw in (dict(), dict(in_place=True), dict(mask_fmt="bytes")):
        check_f32(oracle, ctx, x, td=td, fd=fd, layout="btc", **kw)


def test_f32_interleaved_order(oracle, ctx):
    rng = np.random.default_rng(17)
    x = chi2_block(rng, 2, 96, 403)
    td = dict(k=2.5, iterations=3, replace="mean")
    fd = dict(k=2.5, iterations=2, replace="median", bin=32)
    want, wf = oracle.clean(x, "bct", tdsc=td, fdsc=fd, order="interleaved")
    try:
        ctx.set_option("order", 1)
        for mf in ("bits", "bytes"):
            got, gf = run_gpu(ctx, x, tdsc=td, fdsc=fd, mask_fmt=mf)
            gflag = gf if mf == "bits" else gf > 0
            if np.array_equal(gflag, wf > 0):
                keep = ~(wf > 0)
                assert np.array_equal(got[keep].view(np.uint32), x[keep].view(np.uint32))
                both = wf > 0
                assert np.all(np.abs(got[both].astype(np.float64) - want[both]) <= REL * np.abs(want[both]) + 1e-30)
            else:
                pytest.fail("interleaved float32 masks differ from the oracle")
    finally:
        ctx.set_option("order", 0)
