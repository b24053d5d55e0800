"""Randomised sweeps against the oracle (Sec. IV, both methods).

Two hundred seeded cases draw a shape, a layout, a mask format, the entry point,
buffer offsets and in-place use, and for each method a threshold, an
iteration count, a replacement and (FDSC) a bin size, in blocked or
interleaved order.  uint8 results must equal the oracle's bit for bit, so
every combination the planner can reach is checked exactly, including the
ones no hand-written case lists.  Eighty float32 cases do the same for one
method at a time under the float32 tolerance, and twenty ragged uint8
batches go through rfim_clean_batch, eager or captured.
"""
import numpy as np
import pytest

from gpu_util import noise_u8, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2001_03389_gb300 import build

    build.build()
    from paper_2001_03389_gb300 import rfim

    c = rfim.Context(0)
    yield c
    c.set_option("order", 0)
    c.close()


def draw_case(seed):
    r = np.random.default_rng(seed)
    B = int(r.integers(1, 4))
    C = int(r.choice([1, 2, 3, 5, 17, 31, 32, 33, 64, 96, 130, 257, 300]))
    T = int(r.choice([1, 2, 7, 31, 32, 33, 100, 257, 1000, 1250, 1501, 3001, 3999]))
    api = str(r.choice(["clean", "clean", "tdsc", "fdsc"]))
    cut = lambda: dict(k=float(r.choice([1.5, 2.0, 2.5, 3.0, 4.0])), iterations=int(r.integers(1, 4)),
                       replace=str(r.choice(["mean", "median", "random"])))
    td = cut() if api in ("clean", "tdsc") else None
    fd = None
    if api in ("clean", "fdsc"):
        fd = cut()
        fd["bin"] = int(min(C, r.choice([1, 2, 3, 7, 16, 32, 32, C])))
    if api == "clean" and td is None:
        td = cut()
    order = "interleaved" if api == "clean" and r.random() < 0.25 else "blocked"
    layout = "btc" if r.random() < 0.2 else "bct"
    mask_fmt = str(r.choice(["bits", "bits", "bytes", "none"]))
    in_place = bool(r.random() < 0.2)
    in_off = int(r.integers(0, 8)) if r.random() < 0.3 else 0
    out_off = int(r.integers(0, 8)) if r.random() < 0.3 else 0
    return dict(B=B, C=C, T=T, api=api, td=td, fd=fd, order=order, layout=layout, mask_fmt=mask_fmt,
                in_place=in_place, in_off=in_off, out_off=out_off)


@pytest.mark.parametrize("seed", range(200))
def test_uint8_sweep(oracle, ctx, seed):
    case = draw_case(9000 + seed)
    B, C, T = case["B"], case["C"], case["T"]
    rng = np.random.default_rng(seed)
    x = noise_u8(rng, (B, C, T))
    if case["layout"] == "btc":
        x = np.ascontiguousarray(x.transpose(0, 2, 1))
    want, wf = oracle.clean(x, case["layout"], tdsc=case["td"], fdsc=case["fd"], order=case["order"])
    try:
        ctx.set_option("order", 1 if case["order"] == "interleaved" else 0)
        mf = None if case["mask_fmt"] == "none" else case["mask_fmt"]
        got, gf = run_gpu(ctx, x, layout=case["layout"], tdsc=case["td"], fdsc=case["fd"], mask_fmt=mf,
                          in_place=case["in_place"], in_off=case["in_off"], out_off=case["out_off"], api=case["api"])
    finally:
        ctx.set_option("order", 0)
    bad = np.argwhere(got != want)
    assert bad.size == 0, f"{case}: {len(bad)} samples differ, first at {bad[:3].tolist()}"
    if case["mask_fmt"] == "bits":
        assert np.array_equal(gf, wf > 0), case
    elif case["mask_fmt"] == "bytes":
        assert np.array_equal(gf, wf), case


MARGIN = 1e-9


@pytest.mark.parametrize("seed", range(80))
def test_float32_sweep(oracle, ctx, seed):
    # One method per case (a mask disagreement near a threshold then changes
    # only its own row or column): decisions may differ from the oracle's only
    # within 1e-9 relative of the threshold; values away from disagreements
    # match, unflagged ones bit for bit and replaced ones within 1e-6.
    r = np.random.default_rng(7000 + seed)
    B = int(r.integers(1, 3))
    C = int(r.choice([1, 3, 17, 32, 33, 96, 130, 300]))
    T = int(r.choice([1, 7, 33, 100, 257, 1000, 3001]))
    api = str(r.choice(["tdsc", "fdsc"]))
    cut = dict(k=float(r.choice([2.0, 2.5, 3.0])), iterations=int(r.integers(1, 4)),
               replace=str(r.choice(["mean", "median", "random"])))
    if api == "fdsc":
        cut["bin"] = int(min(C, r.choice([1, 2, 7, 16, 32, C])))
    td, fd = (cut, None) if api == "tdsc" else (None, cut)
    layout = "btc" if r.random() < 0.2 else "bct"
    in_place = bool(r.random() < 0.2)
    x = (r.standard_exponential((B, C, T)) * 2.0).astype(np.float32)
    x.reshape(-1)[r.integers(0, x.size, max(1, x.size // 40))] *= 8.0
    if layout == "btc":
        x = np.ascontiguousarray(x.transpose(0, 2, 1))
    want, wf, margin = oracle.clean_f32_margin(x, layout, tdsc=td, fdsc=fd)
    got, gf = run_gpu(ctx, x, layout=layout, tdsc=td, fdsc=fd, api=api, in_place=in_place)
    wflag = wf > 0
    dis = gf != wflag
    assert not (dis & ~(margin <= MARGIN)).any(), "mask disagreements away from the threshold"
    # axes of the line a disagreement affects: TDSC rows are (beam, channel),
    # FDSC columns (beam, time); BTC blocks hold (beam, time, channel)
    ok = np.ones_like(wflag)
    for b, i, j in np.argwhere(dis):
        if (api == "tdsc") == (layout == "bct"):
            ok[b, i, :] = False
        else:
            ok[b, :, j] = False
    keep = ok & ~wflag & ~gf
    assert np.array_equal(got[keep].view(np.uint32), x[keep].view(np.uint32)), "unflagged samples changed"
    both = ok & wflag & gf
    err = np.abs(got[both].astype(np.float64) - want[both].astype(np.float64))
    assert np.all(err <= 1e-6 * np.maximum(np.abs(want[both].astype(np.float64)), 1e-30)), "replaced values differ"


@pytest.mark.parametrize("seed", range(20))
def test_batch_sweep(oracle, ctx, seed):
    # ragged uint8 batches through rfim_clean_batch (eager or captured, each
    # block its own shape and beam count) against the oracle block by block
    import torch

    from gpu_util import unpack_bits
    from paper_2001_03389_gb300 import rfim

    r = np.random.default_rng(5000 + seed)
    n = int(r.integers(1, 7))
    shapes = [(int(r.integers(1, 3)), int(r.choice([3, 32, 64, 96, 200])), int(r.choice([5, 64, 500, 1250, 3000])))
              for _ in range(n)]
    rep = str(r.choice(["mean", "median", "random"]))
    td = dict(k=float(r.choice([2.0, 3.0])), iterations=int(r.integers(1, 3)), replace=rep)
    fd = dict(k=float(r.choice([2.0, 3.0])), iterations=int(r.integers(1, 3)), replace=rep, bin=3)
    flags = rfim.BATCH_GRAPH if r.random() < 0.5 else 0
    xs = [noise_u8(np.random.default_rng(seed * 31 + i), s) for i, s in enumerate(shapes)]
    dev = torch.device("cuda:0")
    ins = [torch.from_numpy(x).to(dev) for x in xs]
    outs = [torch.empty_like(t) for t in ins]
    masks = [torch.full((rfim.mask_words(s[1], s[2], s[0]),), -1, dtype=torch.int32, device=dev) for s in shapes]
    blks = [rfim.Context.block(i, o, m, "bct", "bits") for i, o, m in zip(ins, outs, masks)]
    ctx.clean_batch(blks, rfim.make_cut(**td), rfim.make_cut(**fd), flags=flags)
    torch.cuda.synchronize()
    for x, o, m, (B, C, T) in zip(xs, outs, masks, shapes):
        want, wf = oracle.clean(x, "bct", tdsc=td, fdsc=fd)
        assert np.array_equal(o.cpu().numpy(), want), (seed, B, C, T)
        assert np.array_equal(unpack_bits(m.cpu().numpy(), B * C, T).reshape(B, C, T), wf > 0), (seed, B, C, T)
    assert ctx.device_status() == rfim.OK
