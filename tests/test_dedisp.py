"""The accuracy claim of Sec. V-A on its simulated canvas (Figs. 4-6): a faint
dispersed FRB (DM 500, dedispersed S/N 15) drowned by bright low-DM broadband
and narrowband RFI falls below the detection threshold (S/N 8) when
dedispersed, and rises above it after TDSC (3.25 sigma) and FDSC (bin 32,
2.75 sigma) -- here checked on the CPU oracle and, marked gpu, on the library."""
import numpy as np
import pytest

from dedisp_util import dedisperse, snr_at

THRESHOLD = 8.0  # detection threshold of the ARTS pipeline (Sec. V-A)
TD = dict(k=3.25, iterations=1, replace="mean")
FD = dict(k=2.75, iterations=1, replace="mean", bin=32)


def _frb():
    from paper_2001_03389_gb300 import synth

    p = synth.FRB_CANVAS
    return p["frb_dm"], p["frb_t0"]


@pytest.fixture(scope="module")
def canvas():
    from paper_2001_03389_gb300 import synth

    return synth.frb_canvas()


def test_canvas_snr_without_rfi():
    from paper_2001_03389_gb300 import synth

    dm, t0 = _frb()
    s = dedisperse(synth.frb_canvas(rfi=False), dm)
    assert 12.0 < snr_at(s, t0) < 18.0  # the injected S/N 15, up to the noise
    assert int(np.argmax(s)) == t0


def test_oracle_cleaning_restores_the_frb(oracle, canvas):
    dm, t0 = _frb()
    dirty = dedisperse(canvas, dm)
    assert snr_at(dirty, t0) < THRESHOLD  # not detected with the RFI in place
    out, fl = oracle.clean(canvas[None], "bct", tdsc=TD, fdsc=FD)
    clean = dedisperse(out[0], dm)
    assert snr_at(clean, t0) > THRESHOLD
    assert int(np.argmax(clean)) == t0  # the FRB is the brightest dedispersed sample
    assert (fl > 0).mean() < 0.02


@pytest.mark.gpu
def test_library_cleaning_restores_the_frb(oracle, canvas):
    import torch

    from paper_2001_03389_gb300 import build

    build.build()
    from paper_2001_03389_gb300 import rfim

    dm, t0 = _frb()
    ctx = rfim.Context(0)
    try:
        x = torch.from_numpy(canvas[None].copy()).cuda()
        out = torch.empty_like(x)
        ctx.clean(ctx.block(x, out), rfim.make_cut(**TD), rfim.make_cut(**FD))
        torch.cuda.synchronize()
        got = out.cpu().numpy()[0]
    finally:
        ctx.close()
    want, _ = oracle.clean(canvas[None], "bct", tdsc=TD, fdsc=FD)
    clean = dedisperse(got, dm)
    assert snr_at(clean, t0) > THRESHOLD and int(np.argmax(clean)) == t0
    assert abs(snr_at(clean, t0) - snr_at(dedisperse(want[0], dm), t0)) < 1e-3
