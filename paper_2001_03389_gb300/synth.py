"""Seeded synthetic filterbanks shaped like the paper's ARTS data.

This module only draws inputs; it holds none of the cleaning arithmetic, so
both the GPU path and the CPU oracle can be fed from it.

Recipe (the paper's own data are not available; these stand in for them):
  * Noise: uint8 blocks are round(N(128, 16^2)) clipped to [0, 255]; float32
    blocks are g_c * chi^2_2 with a per-channel bandpass gain g_c drawn
    log-uniform in [0.5, 2] (sigma_c = 2 g_c).  The paper's own simulation
    (Sec. V-A) uses N(0, 1) on an ARTS-shaped canvas.
  * Narrowband RFI (Sec. V-A: "narrow-band periodic pulses"): a fraction of
    channels carries +A_nb * (1 + 0.5 sin(2 pi t / P + phi)) for every t,
    P ~ U[500, 5000] samples, phi ~ U[0, 2 pi); optionally constant (no sine).
  * Broadband RFI (Sec. V-A: "bright low-DM broadband pulses"): a set of time
    samples carries +A_bb in every channel; bursts are `bb_width` samples wide.
  * One faint dispersed pulse (Sec. V-A, the FRB stand-in): +A_disp, one
    sample wide per channel, delayed per Eq. 2, delay(nu) proportional to
    nu^-2 - nu_hi^-2 over the Apertif band (1250-1550 MHz, channel 0 the
    highest frequency), scaled so the lowest channel lags by `disp_span`
    samples.
  * ARTS shapes: 1536 channels, 81.92 us sampling (Sec. V-A footnote),
    12 beams per node (Sec. V-B).
Seeds: each workload has its own SeedSequence (2001033891 for the small
canvas, ...92 for the ARTS batch, ...93 for the float32 batch, ...94 for the
ragged batch, ...95 for streaming chunks); beam j draws from child j of that
sequence, so any subset of beams can be regenerated alone.
"""
from __future__ import annotations

import dataclasses

import numpy as np

SEED_BASE = 2001033890
F_HI_MHZ = 1550.0
BW_MHZ = 300.0


@dataclasses.dataclass
class RFIModel:
    nb_frac: float = 0.02        # fraction of channels with narrowband RFI
    nb_count: int | None = None  # exact number of narrowband channels (overrides nb_frac)
    nb_amp: float = 60.0         # narrowband amplitude (uint8 units or sigma_c multiples)
    nb_sine: bool = True         # sinusoidal amplitude drift
    bb_frac: float = 0.01        # fraction of time samples hit by broadband bursts
    bb_count: int | None = None  # exact number of bursts (overrides bb_frac)
    bb_width: int = 1            # samples per burst
    bb_amp: float = 90.0
    disp_amp: float = 20.0       # dispersed pulse amplitude (0 disables)
    disp_span: int = 300         # delay of the lowest channel, samples


def _dispersion_delays(C: int, span: int) -> np.ndarray:
    """Per-channel delay in samples following Eq. 2 (delay ~ nu^-2 - nu_hi^-2)."""
    nu = F_HI_MHZ - BW_MHZ * (np.arange(C) + 0.5) / C
    d = nu ** -2 - F_HI_MHZ ** -2
    d = d / d.max() if d.max() > 0 else d
    return np.rint(d * span).astype(np.int64)


def _beam_rng(seed: int, beam: int) -> np.random.Generator:
    ss = np.random.SeedSequence(seed, spawn_key=(beam,))
    return np.random.Generator(np.random.PCG64(ss))


def _rfi_offsets(rng, C: int, T: int, m: RFIModel, scale: np.ndarray | float):
    """Additive RFI for one beam, as a float32 (C, T) array in units of `scale`."""
    add = np.zeros((C, T), dtype=np.float32)
    n_nb = m.nb_count if m.nb_count is not None else int(round(m.nb_frac * C))
    if n_nb > 0:
        chans = rng.choice(C, size=min(n_nb, C), replace=False)
        t = np.arange(T, dtype=np.float64)
        for c in chans:
            if m.nb_sine:
                P = rng.uniform(500.0, 5000.0)
                phi = rng.uniform(0.0, 2 * np.pi)
                add[c] += (m.nb_amp * (1.0 + 0.5 * np.sin(2 * np.pi * t / P + phi))).astype(np.float32)
            else:
                add[c] += m.nb_amp
    n_bb = m.bb_count if m.bb_count is not None else int(round(m.bb_frac * T / max(m.bb_width, 1)))
    if n_bb > 0:
        starts = rng.choice(max(T - m.bb_width + 1, 1), size=min(n_bb, max(T - m.bb_width + 1, 1)), replace=False)
        for s in starts:
            add[:, s:s + m.bb_width] += m.bb_amp
    if m.disp_amp:
        t0 = int(rng.integers(0, max(T // 2, 1)))
        delays = _dispersion_delays(C, m.disp_span)
        ts = t0 + delays
        ok = ts < T
        add[np.arange(C)[ok], ts[ok]] += m.disp_amp
    return add * scale


def beam_u8(seed: int, beam: int, C: int, T: int, model: RFIModel, layout: str = "bct") -> np.ndarray:
    """One uint8 beam: round(N(128,16^2) + RFI) clipped to [0,255]; (C,T) or (T,C)."""
    rng = _beam_rng(seed, beam)
    x = rng.standard_normal((C, T), dtype=np.float32)
    x *= 16.0
    x += 128.0
    x += _rfi_offsets(rng, C, T, model, 1.0)
    np.rint(x, out=x)
    np.clip(x, 0, 255, out=x)
    out = x.astype(np.uint8)
    return np.ascontiguousarray(out.T) if layout == "btc" else out


def beam_f32(seed: int, beam: int, C: int, T: int, model: RFIModel, layout: str = "bct") -> np.ndarray:
    """One float32 beam: g_c chi^2_2 noise plus RFI in multiples of sigma_c = 2 g_c."""
    rng = _beam_rng(seed, beam)
    g = np.exp(rng.uniform(np.log(0.5), np.log(2.0), size=C)).astype(np.float32)
    x = rng.standard_exponential((C, T), dtype=np.float32)
    x *= 2.0                       # chi^2 with 2 degrees of freedom
    x += _rfi_offsets(rng, C, T, model, 2.0)  # amplitudes in sigma units (sigma of chi^2_2 is 2)
    x *= g[:, None]
    return np.ascontiguousarray(x.T) if layout == "btc" else x


# ---------------------------------------------------------------------------
# The paper-shaped workloads.
# ---------------------------------------------------------------------------

def small_canvas_model() -> RFIModel:
    # 3 persistent narrowband channels at +60, 5 broadband impulses 4 samples wide at +90,
    # one dispersed pulse at +20.
    return RFIModel(nb_count=3, nb_amp=60.0, nb_sine=False, bb_count=5, bb_width=4, bb_amp=90.0,
                    disp_amp=20.0, disp_span=300)


def arts_model() -> RFIModel:
    # 2% of channels sinusoidal narrowband around +60, 1% of samples broadband +90, one pulse.
    return RFIModel(nb_frac=0.02, nb_amp=60.0, nb_sine=True, bb_frac=0.01, bb_width=1, bb_amp=90.0,
                    disp_amp=20.0, disp_span=300)


def fp32_model() -> RFIModel:
    # Same mix at 5x density, amplitudes as multiples of sigma_c: 60/16 = 3.75, 90/16 = 5.625, 20/16 = 1.25.
    return RFIModel(nb_frac=0.10, nb_amp=3.75, nb_sine=True, bb_frac=0.05, bb_width=1, bb_amp=5.625,
                    disp_amp=1.25, disp_span=300)


# The workloads, named by what they are: a small uint8 canvas for TDSC, the
# ARTS batch (12 beams of 1536 channels x 12,500 samples, Sec. V-B), and a
# float32 batch of the same cut at larger size.
SMALL = "tdsc_1x64x2048_u8"
ARTS = "arts_12x1536x12500_u8"
FP32 = "fp32_32x4096x8192"
WORKLOADS = {
    SMALL: dict(name=SMALL, dtype="u8", B=1, C=64, T=2048, model=small_canvas_model, seed=SEED_BASE + 1,
                tdsc=dict(k=3.0, iterations=1, replace="mean"), fdsc=None),
    ARTS: dict(name=ARTS, dtype="u8", B=12, C=1536, T=12500, model=arts_model, seed=SEED_BASE + 2,
               tdsc=dict(k=3.0, iterations=2, replace="median"),
               fdsc=dict(k=3.0, iterations=2, replace="median", bin=32)),
    FP32: dict(name=FP32, dtype="f32", B=32, C=4096, T=8192, model=fp32_model, seed=SEED_BASE + 3,
               tdsc=dict(k=2.5, iterations=3, replace="mean"),
               fdsc=dict(k=2.5, iterations=3, replace="mean", bin=32)),
}
RAGGED_SEED = SEED_BASE + 4  # the ragged batch
STREAM_SEED = SEED_BASE + 5  # streaming chunks


def seed_of(workload: str) -> int:
    return WORKLOADS[workload]["seed"]


def make_beams(workload: str, beams=None, layout: str = "bct"):
    """Generate beams of a fixed-shape workload as one (b, C, T) array."""
    spec = WORKLOADS[workload]
    ids = list(range(spec["B"])) if beams is None else list(beams)
    fn = beam_u8 if spec["dtype"] == "u8" else beam_f32
    model = spec["model"]()
    return np.stack([fn(spec["seed"], j, spec["C"], spec["T"], model, layout) for j in ids])


def ragged_shapes(n: int = 200, seed: int | None = None):
    """Shapes of the ragged batch: C from {384, 768, 1536, 4096}, T ~ U[1000, 25000]."""
    rng = np.random.Generator(np.random.PCG64(RAGGED_SEED if seed is None else seed))
    Cs = rng.choice([384, 768, 1536, 4096], size=n)
    Ts = rng.integers(1000, 25001, size=n)
    return [(int(c), int(t)) for c, t in zip(Cs, Ts)]


def ragged_beam(j: int, C: int, T: int, layout: str = "bct") -> np.ndarray:
    """Beam j of the ragged batch, ARTS noise and RFI model."""
    return beam_u8(RAGGED_SEED, j, C, T, arts_model(), layout)


def stream_chunk(beam: int, chunk: int, C: int = 1536, T: int = 1250) -> np.ndarray:
    """Chunk `chunk` of streaming beam `beam` (ARTS model), shape (C, T)."""
    rng_seed = STREAM_SEED * 1_000_003 + beam
    return beam_u8(rng_seed, chunk, C, T, arts_model())


# ---------------------------------------------------------------------------
# On-device generation for the multi-gigabyte workloads (ragged batch,
# streaming): the same noise and RFI model, drawn with a seeded torch CUDA
# generator so that gigabytes need not be produced on the host.  (Different
# numbers than the numpy recipe above; results are checked against the CPU
# oracle on copies of these bytes.)
# ---------------------------------------------------------------------------

def _torch_rfi(gen, C: int, T: int, model: RFIModel, device):
    """Additive RFI of one beam as a float32 (C, T) device tensor (the RFIModel recipe)."""
    import math

    import torch

    add = torch.zeros((C, T), device=device, dtype=torch.float32)
    n_nb = model.nb_count if model.nb_count is not None else int(round(model.nb_frac * C))
    if n_nb > 0:
        chans = torch.randperm(C, generator=gen, device=device)[:n_nb]
        t = torch.arange(T, device=device, dtype=torch.float32)
        if model.nb_sine:
            P = 500.0 + 4500.0 * torch.rand((n_nb, 1), generator=gen, device=device)
            phi = 2 * math.pi * torch.rand((n_nb, 1), generator=gen, device=device)
            add[chans] += model.nb_amp * (1.0 + 0.5 * torch.sin(2 * math.pi * t[None, :] / P + phi))
        else:
            add[chans] += model.nb_amp
    n_bb = model.bb_count if model.bb_count is not None else int(round(model.bb_frac * T / max(model.bb_width, 1)))
    if n_bb > 0:
        starts = torch.randperm(max(T - model.bb_width + 1, 1), generator=gen, device=device)[:n_bb]
        for w in range(model.bb_width):
            add[:, starts + w] += model.bb_amp
    if model.disp_amp:
        t0 = int(torch.randint(0, max(T // 2, 1), (1,), generator=gen, device=device).item())
        ts = t0 + torch.from_numpy(_dispersion_delays(C, model.disp_span)).to(device)
        ok = ts < T
        add[torch.arange(C, device=device)[ok], ts[ok]] += model.disp_amp
    return add


def torch_beam_u8(gen, C: int, T: int, model: RFIModel, device):
    """One uint8 beam (C, T) on `device`: round(N(128, 16^2) + RFI) clipped."""
    import torch

    x = torch.randn((C, T), generator=gen, device=device, dtype=torch.float32)
    x.mul_(16.0).add_(128.0).add_(_torch_rfi(gen, C, T, model, device))
    return x.round_().clamp_(0, 255).to(torch.uint8)


def torch_beam_f32(gen, C: int, T: int, model: RFIModel, device):
    """One float32 beam (C, T) on `device`: g_c (chi^2_2 noise + RFI in sigma units)."""
    import math

    import torch

    g = torch.exp(math.log(0.5) + (math.log(2.0) - math.log(0.5)) * torch.rand((C, 1), generator=gen, device=device))
    x = torch.empty((C, T), device=device, dtype=torch.float32).exponential_(1.0, generator=gen)
    x.mul_(2.0).add_(_torch_rfi(gen, C, T, model, device), alpha=2.0)
    return x.mul_(g)


def torch_make_beams(workload: str, beams: int, seed: int, device):
    """A (beams, C, T) device block of a fixed-shape workload, drawn on the device."""
    import torch

    spec = WORKLOADS[workload]
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    fn = torch_beam_u8 if spec["dtype"] == "u8" else torch_beam_f32
    dt = torch.uint8 if spec["dtype"] == "u8" else torch.float32
    out = torch.empty((beams, spec["C"], spec["T"]), dtype=dt, device=device)
    for b in range(beams):
        out[b] = fn(gen, spec["C"], spec["T"], spec["model"](), device)
    return out


def torch_ragged_batch(shapes, seed: int, device, layout: str = "bct"):
    """Beams of the given (C, T) shapes, ARTS model, as separate device tensors."""
    import torch

    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    out = []
    for C, T in shapes:
        b = torch_beam_u8(gen, C, T, arts_model(), device)
        out.append(b.t().contiguous() if layout == "btc" else b)
    return out


# ---------------------------------------------------------------------------
# The simulated accuracy canvas of Sec. V-A (Figs. 4-6): Gaussian noise
# (mu = 0, sigma = 1) on the ARTS band, a faint dispersed FRB and bright RFI.
# ---------------------------------------------------------------------------
K_DM = 4.15e3          # MHz^2 pc^-1 cm^3 s (Eq. 2)
T_SAMP = 81.92e-6      # s (Sec. V-A)


def dm_delays(C: int, dm: float, f_hi: float = F_HI_MHZ, bw: float = BW_MHZ, dt: float = T_SAMP) -> np.ndarray:
    """Per-channel delay in samples of a pulse of dispersion measure dm (Eq. 2),
    channel 0 the highest frequency."""
    f = f_hi - bw * (np.arange(C) + 0.5) / C
    return np.rint(K_DM * (f ** -2.0 - f_hi ** -2.0) * dm / dt).astype(np.int64)


FRB_CANVAS = dict(frb_dm=500.0, frb_t0=488, frb_snr=15.0,            # Fig. 4 caption; t0 = 0.04 s
                  bb=((1.0, 2000, 100.0), (10.0, 6500, 150.0)),       # (DM, start, amplitude in sigma)
                  nb=((300, 10), (900, 15)), nb_amp=125.0, nb_period=400, nb_width=16)


def frb_canvas(C: int = 1536, T: int = 8192, seed: int = SEED_BASE + 6, frb: bool = True, rfi: bool = True):
    """float32 (C, T) block: N(0, 1) noise, a one-sample FRB at DM 500 whose
    dedispersed S/N is 15 (amplitude 15 / sqrt(C) per channel), two bright
    low-DM broadband pulses (DM 1 and 10, 100 and 150 sigma per channel) and two
    periodic narrowband pulses (125 sigma in 10 and 15 channels)."""
    p = FRB_CANVAS
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((C, T)).astype(np.float32)
    ch = np.arange(C)

    def sweep(dm, t0, amp):
        ts = t0 + dm_delays(C, dm)
        ok = ts < T
        x[ch[ok], ts[ok]] += np.float32(amp)

    if frb:
        sweep(p["frb_dm"], p["frb_t0"], p["frb_snr"] / np.sqrt(C))
    if rfi:
        for dm, t0, amp in p["bb"]:
            sweep(dm, t0, amp)
        for c0, n in p["nb"]:
            for t in range(100, T, p["nb_period"]):
                x[c0:c0 + n, t:t + p["nb_width"]] += np.float32(p["nb_amp"])
    return x
