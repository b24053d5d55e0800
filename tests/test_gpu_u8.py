"""GPU parity of the uint8 path against the CPU oracle (bit-exact).

Every case runs through the C ABI (librfim.so) and compares the cleaned block
and the flag mask with the oracle element by element, at sizes the oracle
finishes in seconds that still span several tiles and ragged tails, plus the
full-size ARTS configuration on whole beams of the launch the benchmark times.
"""
import numpy as np
import pytest

from gpu_util import noise_u8, run_gpu, unpack_bits

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


def check(oracle, ctx, x, td=None, fd=None, mask_fmt="bits", **kw):
    want, wf = oracle.clean(x, kw.get("layout", "bct"), tdsc=td, fdsc=fd)
    got, gf = run_gpu(ctx, x, tdsc=td, fdsc=fd, mask_fmt=mask_fmt, **kw)
    bad = np.argwhere(got != want)
    assert bad.size == 0, f"{len(bad)} samples differ, first at {bad[:3].tolist()}"
    if mask_fmt == "bits":
        assert np.array_equal(gf, wf > 0), f"mask differs at {np.argwhere(gf != (wf > 0))[:3].tolist()}"
    elif mask_fmt == "bytes":
        assert np.array_equal(gf, wf), f"byte mask differs at {np.argwhere(gf != wf)[:3].tolist()}"


def test_small_paper_canvas(oracle, ctx):
    from paper_2001_03389_gb300 import synth

    x = synth.make_beams(synth.SMALL)
    spec = synth.WORKLOADS[synth.SMALL]
    check(oracle, ctx, x, td=spec["tdsc"], api="tdsc")
    check(oracle, ctx, x, td=spec["tdsc"])


@pytest.mark.parametrize("C,T", [(1, 1), (1, 33), (3, 5), (7, 31), (37, 32), (64, 100), (100, 257), (130, 1000),
                                 (37, 1250), (5, 3169), (5, 3170),
                                 (33, 4099), (5, 12500), (3, 12769), (3, 12770), (2, 25000), (1, 98273),
                                 (1, 98274), (2, 131073), (1, 372181)])
@pytest.mark.parametrize("rep", ["mean", "median"])
def test_tdsc_shapes(oracle, ctx, C, T, rep):
    rng = np.random.default_rng(C * 1000 + T)
    x = noise_u8(rng, (2, C, T))
    for it, k in [(1, 3.0), (3, 2.0)]:
        check(oracle, ctx, x, td=dict(k=k, iterations=it, replace=rep), api="tdsc")


@pytest.mark.parametrize("C,T,bin", [(1, 40, 1), (4, 33, 4), (32, 64, 32), (37, 70, 32), (64, 31, 7), (100, 50, 3),
                                     (130, 96, 32), (96, 40, 96), (1536, 65, 32), (257, 33, 16)])
@pytest.mark.parametrize("rep", ["mean", "median"])
def test_fdsc_shapes(oracle, ctx, C, T, bin, rep):
    rng = np.random.default_rng(C * 7 + T + bin)
    x = noise_u8(rng, (2, C, T))
    if C > 8:
        x[:, C // 3, :] = np.clip(x[:, C // 3, :].astype(int) + 70, 0, 255)  # narrowband channel
    for it, k in [(1, 3.0), (2, 2.5)]:
        check(oracle, ctx, x, fd=dict(k=k, iterations=it, replace=rep, bin=bin), api="fdsc")


@pytest.mark.parametrize("C,T", [(64, 2048), (100, 777), (1536, 200), (48, 5000)])
def test_clean_fused(oracle, ctx, C, T):
    rng = np.random.default_rng(C + T)
    x = noise_u8(rng, (3, C, T))
    x[:, 5, :] = np.clip(x[:, 5, :].astype(int) + 60, 0, 255)
    x[:, :, T // 3] = 250
    for rep in ("mean", "median"):
        td = dict(k=3.0, iterations=2, replace=rep)
        fd = dict(k=3.0, iterations=2, replace=rep, bin=32)
        check(oracle, ctx, x, td=td, fd=fd)
        check(oracle, ctx, x, td=td, fd=fd, mask_fmt="bytes")
        check(oracle, ctx, x, td=td, fd=fd, mask_fmt=None)


@pytest.mark.parametrize("in_off,out_off", [(1, 0), (3, 7), (5, 5), (15, 2)])
def test_misaligned_buffers(oracle, ctx, in_off, out_off):
    rng = np.random.default_rng(in_off * 31 + out_off)
    x = noise_u8(rng, (2, 40, 301))
    td = dict(k=2.5, iterations=2, replace="median")
    fd = dict(k=2.5, iterations=2, replace="mean", bin=8)
    check(oracle, ctx, x, td=td, fd=fd, in_off=in_off, out_off=out_off)
    check(oracle, ctx, x, td=td, fd=fd, in_off=in_off, out_off=out_off, mask_fmt="bytes")


def test_in_place(oracle, ctx):
    rng = np.random.default_rng(5)
    x = noise_u8(rng, (2, 64, 999))
    td = dict(k=3.0, iterations=3, replace="mean")
    fd = dict(k=2.75, iterations=3, replace="median", bin=32)
    check(oracle, ctx, x, td=td, fd=fd, in_place=True)
    check(oracle, ctx, x, td=td, api="tdsc", in_place=True)
    check(oracle, ctx, x, fd=fd, api="fdsc", in_place=True)


@pytest.mark.parametrize("T", [1250, 3169, 12500])
def test_schedules_agree_by_row_mode(oracle, ctx, T):
    # automatic (separate launches when every row takes a quarter warp), fused
    # and separate schedules all match the oracle
    rng = np.random.default_rng(T)
    x = noise_u8(rng, (3, 64, T))
    x[:, 9, :] = np.clip(x[:, 9, :].astype(int) + 60, 0, 255)
    td = dict(k=3.0, iterations=2, replace="median")
    fd = dict(k=3.0, iterations=2, replace="median", bin=32)
    try:
        for sched in (0, 1, 2):
            ctx.set_option("schedule", sched)
            check(oracle, ctx, x, td=td, fd=fd)
            check(oracle, ctx, x, td=dict(td, replace="mean"), fd=dict(fd, replace="mean"), mask_fmt="bytes")
    finally:
        ctx.set_option("schedule", 0)


def test_long_rows_read_from_memory(oracle, ctx):
    # rows beyond the on-chip stage (98,273 samples): every pass reads the row
    # from memory; misaligned, in place, byte masks, fused with FDSC
    import torch

    from paper_2001_03389_gb300 import rfim

    rng = np.random.default_rng(17)
    x = noise_u8(rng, (2, 3, 200003))
    x[:, 1, 5000:5100] = 255
    td = dict(k=2.5, iterations=3, replace="median")
    fd = dict(k=2.5, iterations=2, replace="mean", bin=2)
    check(oracle, ctx, x, td=td, fd=fd, in_off=3, out_off=9)
    check(oracle, ctx, x, td=dict(td, replace="mean"), api="tdsc", in_place=True, in_off=1)
    check(oracle, ctx, x, td=td, fd=fd, mask_fmt="bytes", in_off=7)
    # the exactness bound of the uint8 decisions: (255 T)^2 < 2^53
    y = torch.zeros((1, 1, 372182), dtype=torch.uint8, device="cuda:0")
    with pytest.raises(rfim.RfimError) as e:
        ctx.tdsc(ctx.block(y, torch.empty_like(y)), rfim.make_cut(3.0))
    assert e.value.status == rfim.ERR_RANGE


def test_degenerate_rows(oracle, ctx):
    # constant rows and columns (sigma = 0) flag nothing; k < 1 may flag everything
    x = np.full((1, 16, 64), 77, np.uint8)
    check(oracle, ctx, x, td=dict(k=3.0, iterations=3), fd=dict(k=3.0, iterations=3, bin=4))
    x = np.zeros((1, 4, 4), np.uint8)
    x[:, :, 2:] = 1
    check(oracle, ctx, x, td=dict(k=0.5, iterations=1), api="tdsc")
    x = np.tile(np.array([0, 255], np.uint8), (1, 3, 20))
    check(oracle, ctx, x, td=dict(k=1.0, iterations=2, replace="median"), fd=dict(k=0.6, iterations=2, bin=2))


def test_many_k_values(oracle, ctx):
    rng = np.random.default_rng(9)
    x = noise_u8(rng, (1, 24, 600))
    for k in (0.3, 0.999, 1.0, 1.5, 2.0, 2.25, 2.75, 3.25, 4.0, 7.5, 100.0):
        check(oracle, ctx, x, td=dict(k=k, iterations=2, replace="median"), fd=dict(k=k, iterations=2, bin=5))


@pytest.mark.parametrize("k", [1e-300, 1e-12, 1e-9, 3e-9, 1e-6, 1e-3, 0.05, 5e5, 1e6, 2e6, 1e20, 1e300])
def test_extreme_k(oracle, ctx, k):
    # any finite k > 0 is a valid cut (Sec. IV's n sigma); tiny k flags every
    # sample off the mean, huge k flags nothing
    rng = np.random.default_rng(int(abs(np.log10(k))) + 3)
    x = noise_u8(rng, (2, 40, 700))
    x[0, 5, :] = 77  # a constant row: sigma = 0 flags nothing for any k
    for rep in ("mean", "median", "random"):
        check(oracle, ctx, x, td=dict(k=k, iterations=2, replace=rep), fd=dict(k=k, iterations=2, replace=rep, bin=16),
              mask_fmt="bytes")


def test_arts_full_beam(oracle, ctx):
    # one full ARTS-shaped beam: 1536 x 12500, TDSC then FDSC, k=3, 2 iterations, median, bit mask
    from paper_2001_03389_gb300 import synth

    spec = synth.WORKLOADS[synth.ARTS]
    x = synth.make_beams(synth.ARTS, beams=[0])
    check(oracle, ctx, x, td=spec["tdsc"], fd=spec["fdsc"])


def test_arts_full_size_sampled(oracle, ctx):
    # all 12 beams in the launch the benchmark times; beams 0 and 11 against the oracle
    import torch

    from gpu_util import unpack_bits
    from paper_2001_03389_gb300 import rfim, synth

    spec = synth.WORKLOADS[synth.ARTS]
    x = synth.make_beams(synth.ARTS)
    B, C, T = x.shape
    dev = torch.device("cuda:0")
    xin = torch.from_numpy(x).to(dev)
    out = torch.empty_like(xin)
    mask = torch.zeros(rfim.mask_words(C, T, B), dtype=torch.int32, device=dev)
    blk = ctx.block(xin, out, mask, "bct", "bits")
    ctx.clean(blk, spec["tdsc"], spec["fdsc"])
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    gm = unpack_bits(mask.cpu().numpy(), B * C, T).reshape(B, C, T)
    for b in (0, B - 1):
        want, wf = oracle.clean(x[b:b + 1], "bct", tdsc=spec["tdsc"], fdsc=spec["fdsc"])
        assert np.array_equal(got[b:b + 1], want)
        assert np.array_equal(gm[b:b + 1], wf > 0)


def test_schedules_agree(oracle, ctx):
    rng = np.random.default_rng(12)
    x = noise_u8(rng, (4, 96, 1500))
    td = dict(k=3.0, iterations=2, replace="median")
    fd = dict(k=3.0, iterations=2, replace="median", bin=32)
    want, wf = oracle.clean(x, "bct", tdsc=td, fdsc=fd)
    try:
        for opts in ({"schedule": 2}, {"schedule": 1, "fused_lag": 0}, {"schedule": 1, "fused_lag": 3},
                     {"tile_samples": 8}, {"tile_samples": 16}, {"ctas_per_sm": 1}, {"smem_target": 40000}):
            for k, v in opts.items():
                ctx.set_option(k, v)
            got, gf = run_gpu(ctx, x, tdsc=td, fdsc=fd)
            assert np.array_equal(got, want), opts
            assert np.array_equal(gf, wf > 0), opts
            for k in opts:
                ctx.set_option(k, {"schedule": 0, "fused_lag": 1, "tile_samples": 0, "ctas_per_sm": 0,
                                   "smem_target": 113 * 1024}[k])
    finally:
        for k, v in {"schedule": 0, "fused_lag": 1, "tile_samples": 0, "ctas_per_sm": 0,
                     "smem_target": 113 * 1024}.items():
            ctx.set_option(k, v)


def test_validation_errors(ctx):
    import torch

    from paper_2001_03389_gb300 import rfim

    x = torch.zeros((1, 8, 64), dtype=torch.uint8, device="cuda:0")
    out = torch.zeros_like(x)
    blk = ctx.block(x, out)
    for bad_k in (0.0, -1.0, float("inf"), float("nan")):
        with pytest.raises(rfim.RfimError) as e:
            ctx.tdsc(blk, rfim.make_cut(bad_k))
        assert e.value.status == rfim.ERR_ARG
    with pytest.raises(rfim.RfimError) as e:
        ctx.fdsc(blk, rfim.make_cut(3.0, bin=9))
    assert e.value.status == rfim.ERR_ARG
    with pytest.raises(rfim.RfimError) as e:
        ctx.tdsc(blk, rfim.make_cut(3.0, iterations=17))
    assert e.value.status == rfim.ERR_ARG
    big = torch.zeros(400, dtype=torch.uint8, device="cuda:0")
    blk2 = rfim.rfim_block(big.data_ptr(), big.data_ptr() + 10, None, 1, 1, 100, rfim.U8, rfim.LAYOUT_BCT, 0)
    with pytest.raises(rfim.RfimError) as e:
        ctx.tdsc(blk2, rfim.make_cut(3.0))
    assert e.value.status == rfim.ERR_ARG  # partial overlap of out and in
    long_row = torch.zeros((1, 1, 372200), dtype=torch.uint8, device="cuda:0")
    with pytest.raises(rfim.RfimError) as e:
        ctx.tdsc(ctx.block(long_row, torch.empty_like(long_row)), rfim.make_cut(3.0))
    assert e.value.status == rfim.ERR_RANGE


def test_allocation_failure_is_reported():
    # Host-side fault injection: the "fail_alloc_after" hook refuses the
    # context's device and pinned-host allocations.  Every call that needs one
    # returns RFIM_ERR_OOM without launching, and once the hook is off the same
    # calls succeed on the same context with the results of a plain launch.
    import torch

    from paper_2001_03389_gb300 import rfim

    rng = np.random.default_rng(11)
    B, C, T = 2, 96, 700
    x = torch.from_numpy(noise_u8(rng, (B, C, T))).cuda()
    td, fd = rfim.make_cut(3.0, 2, "median"), rfim.make_cut(3.0, 2, "median", 32)
    ref = torch.empty_like(x)
    ref_mask = torch.zeros(rfim.mask_words(C, T, B), dtype=torch.int32, device="cuda:0")
    c = rfim.Context(0)
    try:
        c.clean(rfim.Context.block(x, ref, ref_mask, "bct", "bits"), td, fd)
        torch.cuda.synchronize()
        xt = x.transpose(1, 2).contiguous()  # BTC copy of the same beams
        hin = x.cpu().pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        hmask = torch.zeros(rfim.mask_words(C, T, B), dtype=torch.int32).pin_memory()
        hblk = rfim.rfim_block(hin.data_ptr(), hout.data_ptr(), hmask.data_ptr(), B, C, T, rfim.U8,
                               rfim.LAYOUT_BCT, rfim.MASK_BITS)

        def calls():
            out_t = torch.empty_like(xt)
            m_t = torch.empty_like(xt)  # byte mask: the BTC path takes a data and a mask scratch
            yield "btc", lambda: c.clean(rfim.Context.block(xt, out_t, m_t, "btc", "bytes"), td, fd), (out_t, m_t)
            o = torch.empty_like(x)
            yield "graph", lambda: c.clean_batch([rfim.Context.block(x, o)], td, fd, flags=rfim.BATCH_GRAPH), o
            yield "host", lambda: c.clean_host(hblk, td, fd), None
            yield "stream", lambda: c.stream_open(4, C, T, rfim.U8, td, fd), None

        for after in (0, 1):
            for name, call, _ in calls():
                c.set_option("fail_alloc_after", after)
                if name == "graph" and after == 1:
                    continue  # the graph takes a single allocation
                with pytest.raises(rfim.RfimError) as e:
                    call()
                assert e.value.status == rfim.ERR_OOM, name
                assert c.last_error(), name
        c.set_option("fail_alloc_after", -1)
        for name, call, out in calls():
            call()
            torch.cuda.synchronize()
            if name == "btc":
                assert torch.equal(out[0].transpose(1, 2), ref)
                flagged = unpack_bits(ref_mask.cpu().numpy(), B * C, T).reshape(B, C, T)
                assert np.array_equal(out[1].transpose(1, 2).cpu().numpy() != 0, flagged)
            elif name == "graph":
                assert torch.equal(out, ref)
            elif name == "host":
                assert torch.equal(hout, ref.cpu()) and torch.equal(hmask, ref_mask.cpu())
            else:
                c.stream_close()
        assert c.device_status() == rfim.OK
    finally:
        c.close()


def test_device_wait_timeout_is_reported(ctx):
    # The test hook withholds beam 0's TDSC completion: its FDSC items must give
    # up after the spin limit, report RFIM_ERR_TIMEOUT, and leave the context usable.
    import torch

    from paper_2001_03389_gb300 import rfim

    rng = np.random.default_rng(3)
    x = torch.from_numpy(noise_u8(rng, (2, 64, 500))).cuda()
    out = torch.empty_like(x)
    blk = ctx.block(x, out)
    try:
        ctx.set_option("spin_limit_us", 20000)
        ctx.set_option("schedule", 1)
        ctx.set_option("withhold_tdsc_done", 1)
        ctx.clean(blk, rfim.make_cut(3.0), rfim.make_cut(3.0, bin=32))
        assert ctx.device_status() == rfim.ERR_TIMEOUT
    finally:
        ctx.set_option("withhold_tdsc_done", 0)
        ctx.set_option("spin_limit_us", 2000000)
        ctx.set_option("schedule", 0)
    ctx.clean(blk, rfim.make_cut(3.0), rfim.make_cut(3.0, bin=32))
    assert ctx.device_status() == rfim.OK


@pytest.mark.parametrize("C,T", [(1, 1), (7, 33), (40, 301), (100, 64), (1536, 97), (33, 1250)])
def test_btc_layout(oracle, ctx, C, T):
    # time-major blocks (B, T, C): every method and mask format, against the oracle's BTC path
    rng = np.random.default_rng(C * 3 + T)
    x = np.ascontiguousarray(noise_u8(rng, (2, C, T)).transpose(0, 2, 1))
    td = dict(k=3.0, iterations=2, replace="median")
    fd = dict(k=2.5, iterations=2, replace="mean", bin=min(32, C))
    check(oracle, ctx, x, td=td, fd=fd, layout="btc")
    check(oracle, ctx, x, td=td, fd=fd, layout="btc", mask_fmt="bytes")
    check(oracle, ctx, x, td=td, api="tdsc", layout="btc")
    check(oracle, ctx, x, fd=fd, api="fdsc", layout="btc", mask_fmt=None)
    check(oracle, ctx, x, td=td, fd=fd, layout="btc", in_place=True)
    check(oracle, ctx, x, td=td, fd=fd, layout="btc", in_off=3, out_off=5)


def test_btc_batch(oracle, ctx):
    import torch

    from gpu_util import unpack_bits
    from paper_2001_03389_gb300 import rfim

    rng = np.random.default_rng(44)
    shapes = [(96, 300), (40, 129), (1536, 64)]
    xs = [np.ascontiguousarray(noise_u8(rng, (1, C, T)).transpose(0, 2, 1)) for C, T in shapes]
    td = dict(k=3.0, iterations=2, replace="median")
    fd = dict(k=3.0, iterations=2, replace="median", bin=32)
    dev = [torch.from_numpy(x).cuda() for x in xs]
    outs = [torch.empty_like(d) for d in dev]
    # BTC bit masks: one row of ceil(C / 32) words per time sample
    masks = [torch.zeros(T * ((C + 31) // 32), dtype=torch.int32, device="cuda:0") for C, T in shapes]
    blks = [ctx.block(d, o, m, "btc", "bits") for d, o, m in zip(dev, outs, masks)]
    ctx.clean_batch(blks, rfim.make_cut(**td), rfim.make_cut(**fd), flags=rfim.BATCH_GRAPH)
    torch.cuda.synchronize()
    for x, o, m, (C, T) in zip(xs, outs, masks, shapes):
        want, wf = oracle.clean(x, "btc", tdsc=td, fdsc=fd)
        assert np.array_equal(o.cpu().numpy(), want)
        # BTC bit mask: rows are time samples, bits along channels
        assert np.array_equal(unpack_bits(m.cpu().numpy(), T, C)[None], wf > 0)


def test_interleaved_order(oracle, ctx):
    # round i: TDSC iteration i on every row, then FDSC iteration i on every column
    from paper_2001_03389_gb300 import rfim

    rng = np.random.default_rng(31)
    x = noise_u8(rng, (3, 96, 777))
    x[:, 5, :] = np.clip(x[:, 5, :].astype(int) + 60, 0, 255)
    cases = [(dict(k=2.5, iterations=3, replace="median"), dict(k=2.5, iterations=2, replace="median", bin=32)),
             (dict(k=2.0, iterations=2, replace="mean"), dict(k=2.0, iterations=3, replace="mean", bin=16))]
    try:
        ctx.set_option("order", 1)
        for td, fd in cases:
            want, wf = oracle.clean(x, "bct", tdsc=td, fdsc=fd, order="interleaved")
            for mf in ("bits", "bytes"):
                got, gf = run_gpu(ctx, x, tdsc=td, fdsc=fd, mask_fmt=mf)
                assert np.array_equal(got, want)
                assert np.array_equal(gf, wf > 0) if mf == "bits" else np.array_equal(gf, wf)
            got, gf = run_gpu(ctx, x, tdsc=td, fdsc=fd, in_place=True)
            assert np.array_equal(got, want) and np.array_equal(gf, wf > 0)
        with pytest.raises(rfim.RfimError):
            ctx.set_option("order", 2)
    finally:
        ctx.set_option("order", 0)
