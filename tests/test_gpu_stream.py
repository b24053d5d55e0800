"""Streaming service (continuous batching): results, admission and the C ABI.

A chunk is one batch (Sec. IV): its result must be the same whether it is
cleaned alone or inside a mixed micro-batch, bit for bit (uint8), and equal to
rfim_clean of the same chunk and to the CPU oracle.
"""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TD = dict(k=3.0, iterations=2, replace="median")
FD = dict(k=3.0, iterations=2, replace="median", bin=32)


@pytest.fixture(scope="module")
def lib():
    from paper_2001_03389_gb300 import build

    build.build()
    from paper_2001_03389_gb300 import rfim

    return rfim


def chunks_u8(n, C, T, seed):
    import torch

    from paper_2001_03389_gb300 import synth

    return synth.torch_ragged_batch([(C, T)] * n, seed=seed, device="cuda:0")


def result(rfim, ctx, ticket, C, T, dtype):
    """(output bytes, mask words) of a completed ticket, copied to the host."""
    from gpu_util import device_bytes

    got = ctx.stream_poll(ticket, wait_us=5_000_000)
    assert got is not None, "chunk not done within 5 s"
    out_p, mask_p = got
    es = 1 if dtype == rfim.U8 else 4
    W = (T + 31) // 32
    out = device_bytes(out_p, C * T * es).cpu().numpy()
    mask = device_bytes(mask_p, C * W * 4).cpu().numpy().view(np.int32)
    return out, mask


def reference(rfim, ctx, x):
    import torch

    C, T = x.shape
    out = torch.empty_like(x)
    mask = torch.zeros(rfim.mask_words(C, T), dtype=torch.int32, device=x.device)
    ctx.clean(ctx.block(x[None], out[None], mask, "bct", "bits"), rfim.make_cut(**TD), rfim.make_cut(**FD))
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(-1).view(np.uint8), mask.cpu().numpy()


def test_stream_alone_equals_mixed_and_clean(lib, oracle):
    import torch

    from gpu_util import unpack_bits

    rfim = lib
    C, T = 96, 1250
    ctx = rfim.Context(0)
    try:
        ctx.stream_open(8, C, T, rfim.U8, rfim.make_cut(**TD), rfim.make_cut(**FD))
        pool = chunks_u8(40, C, T, seed=11)
        x = pool[7]
        # alone
        t = ctx.stream_push(3, x, time.monotonic())
        alone = result(rfim, ctx, t, C, T, rfim.U8)
        ctx.stream_release(t)
        # in a burst of 40 chunks of 8 beams (several micro-batches), x in the middle
        tickets, results = [], {}
        for i in range(40):
            tk = None
            while tk is None:
                tk = ctx.stream_push(i % 8, pool[i], time.monotonic())
                if tk is None:  # no slot: finish the oldest
                    j, tj = tickets.pop(0)
                    results[j] = result(rfim, ctx, tj, C, T, rfim.U8)
                    ctx.stream_release(tj)
            tickets.append((i, tk))
        for i, tk in tickets:
            results[i] = result(rfim, ctx, tk, C, T, rfim.U8)
            ctx.stream_release(tk)
        assert sorted(results) == list(range(40))
        for i, r in results.items():
            want = reference(rfim, ctx, pool[i])
            assert np.array_equal(r[0], want[0]) and np.array_equal(r[1], want[1]), f"chunk {i} != rfim_clean"
        mixed = results[7]
        assert np.array_equal(alone[0], mixed[0]) and np.array_equal(alone[1], mixed[1])
        # and the oracle
        xo = x.cpu().numpy()[None]
        wo, wf = oracle.clean(xo, "bct", tdsc=TD, fdsc=FD)
        assert np.array_equal(alone[0].reshape(1, C, T), wo)
        assert np.array_equal(unpack_bits(alone[1], C, T)[None], wf > 0)
        st = ctx.stream_stats()
        assert st["chunks"] == 41 and st["p50_s"] > 0 and st["p99_s"] >= st["p50_s"]
        ctx.stream_close()
    finally:
        ctx.close()


def test_stream_host_chunks_and_f32(lib, oracle):
    import torch

    rfim = lib
    C, T = 64, 700
    ctx = rfim.Context(0)
    try:
        ctx.stream_open(2, C, T, rfim.U8, rfim.make_cut(**TD), rfim.make_cut(**FD))
        dev = chunks_u8(3, C, T, seed=5)
        host = [d.cpu().numpy() for d in dev]
        tks = [ctx.stream_push(i % 2, host[i].ctypes.data, time.monotonic()) for i in range(3)]
        for i, tk in enumerate(tks):
            r = result(rfim, ctx, tk, C, T, rfim.U8)
            want = reference(rfim, ctx, dev[i])
            assert np.array_equal(r[0], want[0]) and np.array_equal(r[1], want[1])
            ctx.stream_release(tk)
        ctx.stream_close()
        # float32 chunks: equal to rfim_clean of the same chunk
        td = dict(k=2.5, iterations=3, replace="mean")
        fd = dict(k=2.5, iterations=3, replace="mean", bin=32)
        ctx.stream_open(2, C, T, rfim.F32, rfim.make_cut(**td), rfim.make_cut(**fd))
        g = torch.Generator(device="cuda:0")
        g.manual_seed(3)
        xs = [torch.empty((C, T), device="cuda:0").exponential_(1.0, generator=g) * 2.0 for _ in range(4)]
        tks = [ctx.stream_push(i % 2, xs[i], time.monotonic()) for i in range(4)]
        for i, tk in enumerate(tks):
            r = result(rfim, ctx, tk, C, T, rfim.F32)
            out = torch.empty_like(xs[i])
            mask = torch.zeros(rfim.mask_words(C, T), dtype=torch.int32, device="cuda:0")
            ctx.clean(ctx.block(xs[i][None], out[None], mask, "bct", "bits"), rfim.make_cut(**td), rfim.make_cut(**fd))
            torch.cuda.synchronize()
            assert np.array_equal(r[0].view(np.float32), out.cpu().numpy().reshape(-1))
            assert np.array_equal(r[1], mask.cpu().numpy())
            ctx.stream_release(tk)
        ctx.stream_close()
    finally:
        ctx.close()


def test_stream_admission_and_errors(lib):
    rfim = lib
    C, T = 32, 256
    slot = C * T + 256 + ((C * ((T + 31) // 32) * 4 + 255) // 256) * 256
    ctx = rfim.Context(0, hbm_budget=3 * slot)
    try:
        with pytest.raises(rfim.RfimError) as e:
            ctx.stream_push(0, 1, 0.0)
        assert e.value.status == rfim.ERR_STATE
        ctx.stream_open(4, C, T, rfim.U8, rfim.make_cut(3.0), None)
        with pytest.raises(rfim.RfimError) as e:
            ctx.stream_open(4, C, T, rfim.U8, rfim.make_cut(3.0), None)
        assert e.value.status == rfim.ERR_STATE
        pool = chunks_u8(4, C, T, seed=2)
        tks = [ctx.stream_push(0, pool[i], time.monotonic()) for i in range(3)]
        assert all(t is not None for t in tks)
        assert ctx.stream_push(1, pool[3], time.monotonic()) is None  # no slot free: RFIM_ERR_BUSY
        with pytest.raises(rfim.RfimError) as e:
            ctx.stream_push(9, pool[3], time.monotonic())
        assert e.value.status == rfim.ERR_ARG
        with pytest.raises(rfim.RfimError) as e:
            ctx.stream_poll(123456)
        assert e.value.status == rfim.ERR_ARG
        assert ctx.stream_poll(tks[0], wait_us=5_000_000) is not None
        ctx.stream_release(tks[0])
        assert ctx.stream_push(1, pool[3], time.monotonic()) is not None  # a slot is free again
        ctx.stream_close()
        with pytest.raises(rfim.RfimError) as e:
            ctx.stream_close()
        assert e.value.status == rfim.ERR_STATE
    finally:
        ctx.close()


def test_stream_replay_schedule(lib):
    rfim = lib
    C, T = 256, 1250
    ctx = rfim.Context(0)
    try:
        ctx.stream_open(16, C, T, rfim.U8, rfim.make_cut(**TD), rfim.make_cut(**FD))
        pool = chunks_u8(16, C, T, seed=9)
        rng = np.random.default_rng(1)
        n = 2000
        gaps = rng.exponential(1.0 / 20000.0, n)  # Poisson arrivals at 20k chunks/s
        t0 = time.monotonic() + 0.01
        arr = t0 + np.cumsum(gaps)
        beams = np.arange(n) % 16
        ctx.stream_replay(beams, [pool[b].data_ptr() for b in beams], arr)
        st = ctx.stream_stats(reset=True)
        assert st["chunks"] == n
        assert 0 < st["p50_s"] <= st["p99_s"] <= st["p999_s"] < 1.0
        assert st["gbps"] > 0
        assert ctx.device_status() == rfim.OK
        ctx.stream_close()
    finally:
        ctx.close()


def test_stream_random_replacement_matches_oracle(lib, oracle):
    # random replacement through the service: each chunk is a block of one
    # beam (index 0 for the draws), alone or inside a micro-batch
    import torch

    from gpu_util import unpack_bits

    rfim = lib
    C, T = 64, 1250
    td = dict(k=2.5, iterations=2, replace="random")
    fd = dict(k=2.5, iterations=2, replace="random", bin=32)
    ctx = rfim.Context(0)
    try:
        ctx.stream_open(4, C, T, rfim.U8, rfim.make_cut(**td), rfim.make_cut(**fd))
        pool = chunks_u8(12, C, T, seed=23)
        results, tickets = {}, []
        for i in range(12):
            tk = None
            while tk is None:
                tk = ctx.stream_push(i % 4, pool[i], time.monotonic())
                if tk is None:  # no slot: finish the oldest
                    j, tj = tickets.pop(0)
                    results[j] = result(rfim, ctx, tj, C, T, rfim.U8)
                    ctx.stream_release(tj)
            tickets.append((i, tk))
        for i, tk in tickets:
            results[i] = result(rfim, ctx, tk, C, T, rfim.U8)
            ctx.stream_release(tk)
        assert sorted(results) == list(range(12))
        for i, (out, mask) in results.items():
            want, wf = oracle.clean(pool[i].cpu().numpy()[None], "bct", tdsc=td, fdsc=fd)
            assert np.array_equal(out.reshape(1, C, T), want), i
            assert np.array_equal(unpack_bits(mask, C, T)[None], wf > 0), i
        torch.cuda.synchronize()
    finally:
        ctx.stream_close()
        ctx.close()


def test_stream_per_beam_device_state(lib):
    # Each beam keeps its latest completed chunk on the device: the cleaned
    # data, mask and per-channel sums of the chunk's input.  The sums are the
    # plain totals of the input (checked against numpy); they never enter a
    # decision (the results above equal rfim_clean of the chunk alone).
    from gpu_util import device_bytes

    rfim = lib
    C, T = 128, 1250
    ctx = rfim.Context(0)
    try:
        ctx.stream_open(3, C, T, rfim.U8, rfim.make_cut(**TD), rfim.make_cut(**FD))
        pool = chunks_u8(9, C, T, seed=31)
        assert ctx.stream_beam_state(0, C) is None  # nothing completed yet
        last = {}
        for i in range(9):
            b = i % 3
            tk = ctx.stream_push(b, pool[i], time.monotonic())
            assert tk is not None
            out, mask = result(rfim, ctx, tk, C, T, rfim.U8)
            ctx.stream_release(tk)
            last[b] = (i // 3, pool[i].cpu().numpy().astype(np.int64), out, mask)
        for b, (idx, x, out, mask) in last.items():
            got = ctx.stream_beam_state(b, C)
            assert got is not None
            gi, stats, op, mp = got
            assert gi == idx
            assert np.array_equal(stats[:, 0], x.sum(axis=1).astype(np.float64))
            assert np.array_equal(stats[:, 1], (x * x).sum(axis=1).astype(np.float64))
            # the retained slot still holds that chunk's cleaned data and mask
            assert np.array_equal(device_bytes(op, C * T).cpu().numpy(), out)
            W = (T + 31) // 32
            assert np.array_equal(device_bytes(mp, C * W * 4).cpu().numpy().view(np.int32), mask)
        assert ctx.device_status() == rfim.OK
        ctx.stream_close()
    finally:
        ctx.close()


def test_stream_batch_timeout_is_reported(lib):
    # A device-side wait that gives up inside a streaming batch: the test hook
    # withholds the TDSC completion of the batch's first beam, so its FDSC
    # items wait out a short spin limit.  The chunks of that batch complete
    # with RFIM_ERR_TIMEOUT, rfim_device_status reports it once, and the
    # context and the service stay usable.
    rfim = lib
    C, T = 64, 4000  # rows longer than ~3,150 samples: one fused launch per batch
    ctx = rfim.Context(0)
    try:
        ctx.set_option("withhold_tdsc_done", 1)
        ctx.set_option("spin_limit_us", 20000)
        ctx.stream_open(2, C, T, rfim.U8, rfim.make_cut(**TD), rfim.make_cut(**FD))
        pool = chunks_u8(2, C, T, seed=41)
        tk = ctx.stream_push(0, pool[0], time.monotonic())
        with pytest.raises(rfim.RfimError) as e:
            ctx.stream_poll(tk, wait_us=5_000_000)
        assert e.value.status == rfim.ERR_TIMEOUT
        ctx.stream_release(tk)
        assert ctx.device_status() == rfim.ERR_TIMEOUT
        assert ctx.device_status() == rfim.OK  # reported once
        ctx.stream_close()
        # a new service without the hook cleans normally
        ctx.set_option("withhold_tdsc_done", 0)
        ctx.set_option("spin_limit_us", 2000000)
        ctx.stream_open(2, C, T, rfim.U8, rfim.make_cut(**TD), rfim.make_cut(**FD))
        tk = ctx.stream_push(1, pool[1], time.monotonic())
        out, _ = result(rfim, ctx, tk, C, T, rfim.U8)
        ctx.stream_release(tk)
        ref, _ = reference(rfim, ctx, pool[1])
        assert np.array_equal(out, ref)
        assert ctx.device_status() == rfim.OK
        ctx.stream_close()
    finally:
        ctx.close()
