"""Benchmark: cleaned-filterbank throughput of the fused TDSC+FDSC path on GB300.

Workload (one step): the ARTS-shaped batch of 12 beams x 1536 channels x 12500
time samples, uint8, BCT layout; TDSC then FDSC, k = 3, 2 iterations each,
median replacement, bit-mask output (Sec. IV and V of arXiv:2001.03389 give the
method; beams, channels and the sampling come from its ARTS description).
Inputs are synthetic (seeded noise + RFI, see paper_2001_03389_gb300/synth.py).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints ONE JSON line on rank 0.  `value` = input bytes cleaned per second over
all ranks (each rank cleans its own batch: weak scaling, no collective on the
data path).  `roofline` compares the engine kernel's algorithmic bytes
(1 read + 1 write + 1/8 mask byte per sample) per launch with the measured
HBM copy peak.  `e2e` measures the same metric through rfim_clean_host with
pinned host buffers (copies inside the timed region).  `cpu_baseline` times
the CPU oracle (test infrastructure) on whole beams on the host cores, one
core and all cores, and `parity` compares those beams with the GPU's output.

At one GPU the line also carries `configs`: the float32 workload (32 x 4096 x
8192, the largest dense configuration) with its own value, roofline, e2e,
cpu_baseline and parity, and the ragged 200-beam batch timed as one
graph-captured, autotuned rfim_clean_batch against 200 plain rfim_clean
launches on the same inputs, and the ARTS batch in BTC layout beside BCT;
and `streaming`, the service at 10-100 x the ARTS rate.  `--impl reference` times the oracle alone, as the reference arm.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ARTS = "arts_12x1536x12500_u8"  # the reported workload: the ARTS batch
FP32 = "fp32_32x4096x8192"  # the float32 workload
RAGGED = "ragged_200_u8"  # the ragged batch (sub-record only)
WORKLOAD = ARTS
METRIC = "cleaned filterbank GB/s (TDSC+FDSC) & % HBM peak; p99 chunk latency"
UNIT = "GB/s"
NOMINAL_HBM_GBS = 8000.0
F32_MARGIN = 1e-9  # float32 parity: mask disagreements allowed within this relative distance of the threshold
F32_REL = 1e-6     # float32 parity: replaced values agree within this relative tolerance


def alg_bytes_per_sample(dtype):
    """Read + write of the sample plus its mask bit: 2.125 B (uint8), 8.125 B (float32)."""
    es = 1 if dtype == "u8" else 4
    return es + es + 1 / 8


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_spec(name):
    from paper_2001_03389_gb300 import synth

    return dict(synth.WORKLOADS[name])


def config_json(spec, n):
    es = 1 if spec["dtype"] == "u8" else 4
    mb = spec["B"] * spec["C"] * spec["T"] * es / 1e6
    return {
        "workload": f"{spec['name']}_bct_tdsc_then_fdsc",
        "beams": spec["B"], "channels": spec["C"], "samples": spec["T"], "dtype": spec["dtype"], "layout": "BCT",
        "tdsc": spec["tdsc"], "fdsc": spec["fdsc"], "mask": "bits",
        "global_batch": spec["B"] * n, "parallelism": f"replicas{n}" if n > 1 else "single",
        "l2": f"inputs larger than L2 ({mb:.1f} MB read + {mb:.1f} MB written per step vs 135.5 MB L2)",
    }


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"rfim_bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        for r in rows:
            for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                                 r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows), "power_w_max": max(pw) if pw else None}


# ---------------------------------------------------------------------------
# CPU oracle legs (cpu_baseline, parity, and the reference arm)
# ---------------------------------------------------------------------------
def _oracle_clean_beam(args):
    """One beam through the CPU oracle (worker of the all-cores leg)."""
    x, tdsc, fdsc = args
    from oracle import oracle

    t0 = time.perf_counter()
    out, fl = oracle.clean(x[None], "bct", tdsc=tdsc, fdsc=fdsc)
    return time.perf_counter() - t0, out[0], fl[0]


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(spec, beams_np, budget_s=15.0, all_cores=True):
    """The oracle on whole beams of the batch.  (i) one core: beams one after
    another until about `budget_s` seconds of CPU work; (ii) all cores in the
    affinity set: one beam per core in spawned worker processes, all at once.
    Returns (record, {beam: (out, flags)}) -- the outputs serve the parity check."""
    from oracle import oracle

    outs = {}
    tot_t, tot_b, nb = 0.0, 0, 0
    while nb < len(beams_np) and tot_t < budget_s:
        x = beams_np[nb]
        t0 = time.perf_counter()
        out, fl = oracle.clean(x[None], "bct", tdsc=spec["tdsc"], fdsc=spec["fdsc"])
        tot_t += time.perf_counter() - t0
        tot_b += x.nbytes
        outs[nb] = (out[0], fl[0])
        nb += 1
    rec = {"value": tot_b / tot_t / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{nb} of {spec['B']} beams x {spec['C']} channels x {spec['T']} samples, full TDSC+FDSC, "
                     f"single-threaded C oracle, {tot_t:.1f} s"}
    if all_cores:
        import multiprocessing as mp

        cores = _cores()
        n = min(cores, len(beams_np))
        oracle.build()
        ctx = mp.get_context("spawn")  # never fork a process that holds a CUDA context
        t0 = time.perf_counter()
        with ctx.Pool(n) as pool:
            res = pool.map(_oracle_clean_beam, [(beams_np[i], spec["tdsc"], spec["fdsc"]) for i in range(n)])
        wall = time.perf_counter() - t0
        for i, (_, o, f) in enumerate(res):
            outs.setdefault(i, (o, f))
        bytes_all = sum(beams_np[i].nbytes for i in range(n))
        rec["all_cores"] = {"value": bytes_all / wall / 1e9, "unit": UNIT, "cores": n, "kind": "oracle",
                            "sample": f"{n} beams at once, one per spawned process, on {cores} host cores; "
                                      f"wall time {wall:.1f} s including process start"}
    return rec, outs


def parity_u8(got, gflags, outs):
    """Bit-exact comparison of GPU beams with the oracle's."""
    bad = [b for b, (o, f) in outs.items()
           if not (np.array_equal(got[b], o) and np.array_equal(gflags[b], f > 0))]
    return {"beams_checked": sorted(outs), "bit_exact": not bad, "mismatched_beams": bad}


def parity_f32(x, got, gflags, spec, beams):
    """float32 parity on sampled beams: mask disagreements (each must lie within
    1e-9 relative of its threshold, by the oracle's own margin) and replaced
    values within 1e-6 relative outside the rows and columns of a disagreement."""
    from oracle import oracle

    dis_total, beyond, val_bad = 0, 0, 0
    for b in beams:
        want, wf, margin = oracle.clean_f32_margin(x[b:b + 1], "bct", tdsc=spec["tdsc"], fdsc=spec["fdsc"])
        want, wf, margin = want[0], wf[0] > 0, margin[0]
        dis = gflags[b] != wf
        dis_total += int(dis.sum())
        beyond += int((dis & ~(margin <= F32_MARGIN)).sum())
        ok = np.ones_like(wf)
        for c, t in np.argwhere(dis):
            ok[c, :] = False
            ok[:, t] = False
        keep = ok & ~wf & ~gflags[b]
        val_bad += int((got[b][keep].view(np.uint32) != x[b][keep].view(np.uint32)).sum())
        both = ok & wf & gflags[b]
        err = np.abs(got[b][both].astype(np.float64) - want[both].astype(np.float64))
        val_bad += int((err > F32_REL * np.maximum(np.abs(want[both].astype(np.float64)), 1e-30)).sum())
    return {"beams_checked": list(beams), "f32_disagreements": dis_total, "beyond_margin": beyond,
            "values_out_of_tolerance": val_bad, "margin": F32_MARGIN, "rel": F32_REL}


def oracle_time_sample(x_beam, spec, T_sample):
    """Run the CPU oracle on one beam restricted to T_sample time samples."""
    from oracle import oracle

    xs = x_beam[:, :, :T_sample].copy()
    t0 = time.perf_counter()
    oracle.clean(xs, "bct", tdsc=spec["tdsc"], fdsc=spec["fdsc"])
    return time.perf_counter() - t0, xs.nbytes


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    spec = workload_spec(WORKLOAD)
    from paper_2001_03389_gb300 import synth

    x = synth.make_beams(WORKLOAD, beams=[0])
    K, W = args.steps, args.warmup
    # size each step so the whole run stays within about two minutes
    t_small, b_small = oracle_time_sample(x, spec, 128)
    rate = b_small / t_small
    per_step_s = max(0.05, min(5.0, 120.0 / max(1, K + W)))
    T_s = int(min(spec["T"], max(64, rate * per_step_s / spec["C"])))
    for _ in range(W):
        oracle_time_sample(x, spec, T_s)
    tot_t, tot_b = 0.0, 0
    for _ in range(K):
        dt, nb = oracle_time_sample(x, spec, T_s)
        tot_t += dt
        tot_b += nb
    v = tot_b / tot_t / 1e9
    out = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
           "ms_per_step": tot_t / K * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": spec["dtype"], "data": "synthetic", "impl": "reference",
           "config": config_json(spec, 1),
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"per step: 1 beam x {spec['C']} channels x {T_s} samples, full TDSC+FDSC"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# GPU measurements
# ---------------------------------------------------------------------------
def timed_launches(step, stream, K):
    """Run `step` K times on `stream`; per-step CUDA-event times (ms) and the total."""
    import torch

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t_start.record(stream)
    for i in range(K):
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    t_end.record(stream)
    t_end.synchronize()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev], t_start.elapsed_time(t_end)


def roofline(spec, avg_launch_ms, workload):
    peak, peak_kind = peaks()
    B, C, T = spec["B"], spec["C"], spec["T"]
    alg = alg_bytes_per_sample(spec["dtype"]) * B * C * T
    achieved = alg / (avg_launch_ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": profiled_traffic(workload),
            "peak_kind": f"{peak_kind} copy (MEASURED_PEAKS.json hbm_gbs)",
            "frac_of_nominal_8tbs": achieved / NOMINAL_HBM_GBS,
            "kernel": PROFILES[workload][2], "alg_bytes_per_launch": alg, "avg_launch_ms": avg_launch_ms}


def e2e_host(rfim, ctx, x, B, C, T, dt, td, fd, Ke, out_dev, ws=1):
    """The same clean through rfim_clean_host: pinned host in/out/mask, the
    host<->device copies inside the timed region."""
    import torch

    hin = torch.from_numpy(x).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    hmask = torch.empty(rfim.mask_words(C, T, B), dtype=torch.int32).pin_memory()
    hblk = rfim.rfim_block(hin.data_ptr(), hout.data_ptr(), hmask.data_ptr(), B, C, T, dt, rfim.LAYOUT_BCT,
                           rfim.MASK_BITS)
    for _ in range(2):
        ctx.clean_host(hblk, td, fd)
    if ws > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(Ke):
        ctx.clean_host(hblk, td, fd)
    e2e_s = time.perf_counter() - t0
    if ws > 1:
        t = torch.tensor([e2e_s], device=out_dev.device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(t.item())
    nbytes = x.nbytes
    rec = {"value": nbytes * Ke * ws / e2e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes + hmask.numel() * 4, "api": "rfim_clean_host", "steps": Ke}
    ok = bool(torch.equal(hout, out_dev.cpu()))
    del hin, hout, hmask
    return rec, ok


def unpack_mask(mask_words, B, C, T):
    w = mask_words.cpu().numpy().view(np.uint32).reshape(B * C, -1)
    b = np.unpackbits(w.view(np.uint8), axis=-1, bitorder="little")[:, :T]
    return b.reshape(B, C, T).astype(bool)


def measure_fixed(rfim, synth, dev, spec, workload, K, W, args, ws=1, rank=0, with_clocks=True,
                  cpu_budget_s=15.0, cpu_all_cores=True, parity_beams=None):
    """One fixed-shape workload: device-timed steps, roofline, e2e, CPU legs, parity."""
    import torch

    B, C, T = spec["B"], spec["C"], spec["T"]
    if spec["dtype"] == "u8":
        x = synth.make_beams(workload, beams=range(B))
        xin = torch.from_numpy(x).to(dev)
    else:
        # 4.3 GB: drawn on the device with the same model
        xin = synth.torch_make_beams(workload, B, synth.seed_of(workload), dev)
        x = xin.cpu().numpy()
    out = torch.empty_like(xin)
    mask = torch.zeros(rfim.mask_words(C, T, B), dtype=torch.int32, device=dev)
    ctx = rfim.Context(dev.index or 0)
    dt = rfim.U8 if spec["dtype"] == "u8" else rfim.F32
    td, fd = rfim.make_cut(**spec["tdsc"]), rfim.make_cut(**spec["fdsc"])
    blk = ctx.block(xin, out, mask, "bct", "bits")
    stream = torch.cuda.Stream(device=dev)

    def step():
        ctx.clean(blk, td, fd, stream)

    with torch.cuda.stream(stream):
        for _ in range(max(3, W)):
            step()
    stream.synchronize()
    st = ctx.device_status(stream)
    if st != rfim.OK:
        raise RuntimeError(f"device status {st}: {ctx.last_error()}")
    clocks = Clocks(dev.index or 0) if with_clocks and rank == 0 else None
    if clocks:
        clocks.start()
    if ws > 1:
        torch.distributed.barrier()
    per_launch, total_ms = timed_launches(step, stream, K)
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop() if clocks else None
    st = ctx.device_status(stream)
    if st != rfim.OK:
        raise RuntimeError(f"device status {st}: {ctx.last_error()}")
    if ws > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    avg_launch_ms = sum(per_launch) / len(per_launch)
    rec = {"value": x.nbytes * K * ws / (total_ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": total_ms / K,
           "steps": K, "samples_per_s": B * C * T * K * ws / (total_ms * 1e-3),
           "roofline": roofline(spec, avg_launch_ms, workload), "gpu_launches": K}
    if clk:
        rec["clocks"] = clk
    e2e, ok = e2e_host(rfim, ctx, x, B, C, T, dt, td, fd, max(3, min(K, 30)), out, ws)
    rec["e2e"] = e2e
    rec["e2e_matches_device"] = ok
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        pb = parity_beams if parity_beams is not None else [0, B - 1]
        if spec["dtype"] == "u8":
            cb, outs = cpu_baseline(spec, [x[b] for b in range(B)], cpu_budget_s, cpu_all_cores)
            rec["cpu_baseline"] = cb
            got = out.cpu().numpy()
            rec["parity"] = parity_u8(got, unpack_mask(mask, B, C, T), outs)
        else:
            cb, _ = cpu_baseline(spec, [x[b] for b in range(min(B, _cores()))], cpu_budget_s, cpu_all_cores)
            rec["cpu_baseline"] = cb
            rec["parity"] = parity_f32(x, out.cpu().numpy(), unpack_mask(mask, B, C, T), spec, pb)
    ctx.close()
    del xin, out, mask
    torch.cuda.empty_cache()
    return rec


def measure_ragged(rfim, synth, dev, K=20, W=3):
    """The ragged 200-beam batch: one graph-captured, autotuned rfim_clean_batch
    per step against 200 plain rfim_clean launches per step, on the same inputs
    and outputs; bit-exact agreement of the two is reported."""
    import torch

    shapes = synth.ragged_shapes(200)
    beams = synth.torch_ragged_batch(shapes, seed=synth.RAGGED_SEED, device=dev)
    nbytes = sum(c * t for c, t in shapes)
    spec = workload_spec(ARTS)
    td, fd = rfim.make_cut(**spec["tdsc"]), rfim.make_cut(**spec["fdsc"])

    def blocks():
        outs = [torch.empty_like(x) for x in beams]
        masks = [torch.zeros(rfim.mask_words(*x.shape), dtype=torch.int32, device=dev) for x in beams]
        blks = [rfim.Context.block(x[None], o[None], m, "bct", "bits") for x, o, m in zip(beams, outs, masks)]
        return outs, masks, blks

    ctx = rfim.Context(dev.index or 0)
    stream = torch.cuda.Stream(device=dev)
    o_b, m_b, b_b = blocks()
    o_p, m_p, b_p = blocks()

    def batched():
        ctx.clean_batch(b_b, td, fd, flags=rfim.BATCH_GRAPH | rfim.BATCH_AUTOTUNE, stream=stream)

    def plain():
        for b in b_p:
            ctx.clean(b, td, fd, stream)

    res = {}
    for name, fn in (("batched", batched), ("plain", plain)):
        with torch.cuda.stream(stream):
            for _ in range(W):
                fn()
        stream.synchronize()
        per, total = timed_launches(fn, stream, K)
        res[name] = {"value": nbytes * K / (total * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": total / K}
    st = ctx.device_status(stream)
    equal = all(torch.equal(a, b) for a, b in zip(o_b, o_p)) and all(torch.equal(a, b) for a, b in zip(m_b, m_p))
    ctx.close()
    del beams, o_b, m_b, b_b, o_p, m_p, b_p
    torch.cuda.empty_cache()
    return {"workload": "200 beams, C from {384, 768, 1536, 4096}, T uniform in [1000, 25000], uint8, "
                        "TDSC then FDSC k=3 median 2+2 iterations, bit mask",
            "bytes_per_step": nbytes, "steps": K,
            "batched": dict(res["batched"], api="rfim_clean_batch(GRAPH|AUTOTUNE)"),
            "plain": dict(res["plain"], api="200 x rfim_clean"),
            "speedup": res["plain"]["ms_per_step"] / res["batched"]["ms_per_step"],
            "batched_equals_plain": bool(equal), "device_status_ok": st == rfim.OK}


def measure_btc(rfim, synth, dev, K=30, W=3):
    """The ARTS batch in BTC layout ([beam][time][channel], channels fastest)
    through rfim_clean, against the same batch in BCT, on the same data; the
    results must agree (the BTC output transposed equals the BCT output)."""
    import torch

    spec = workload_spec(ARTS)
    B, C, T = spec["B"], spec["C"], spec["T"]
    x = torch.from_numpy(synth.make_beams(ARTS, beams=range(B))).to(dev)
    xt = x.transpose(1, 2).contiguous()
    td, fd = rfim.make_cut(**spec["tdsc"]), rfim.make_cut(**spec["fdsc"])
    ctx = rfim.Context(dev.index or 0)
    stream = torch.cuda.Stream(device=dev)
    res = {}
    outs = {}
    for layout, xin in (("bct", x), ("btc", xt)):
        out = torch.empty_like(xin)
        rows, fast = (B * C, T) if layout == "bct" else (B * T, C)
        mask = torch.zeros(rows * ((fast + 31) // 32), dtype=torch.int32, device=dev)
        blk = ctx.block(xin, out, mask, layout, "bits")

        def step():
            ctx.clean(blk, td, fd, stream)

        with torch.cuda.stream(stream):
            for _ in range(W):
                step()
        stream.synchronize()
        per, total = timed_launches(step, stream, K)
        res[layout] = {"value": x.numel() * K / (total * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": total / K}
        outs[layout] = out
    same = bool(torch.equal(outs["btc"].transpose(1, 2), outs["bct"]))
    st = ctx.device_status(stream)
    ctx.close()
    del x, xt, outs
    torch.cuda.empty_cache()
    return {"workload": "ARTS batch 12 x 1536 x 12500 uint8, TDSC then FDSC k=3 median 2+2, bit mask",
            "bct": res["bct"], "btc": dict(res["btc"], path="on-device transposition into BCT scratch, "
                                                           "BCT engine, transposition back"),
            "btc_over_bct": res["btc"]["value"] / res["bct"]["value"], "btc_equals_bct": same,
            "device_status_ok": st == rfim.OK, "steps": K}


def run_gpu(args):
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    from paper_2001_03389_gb300 import build

    if rank == 0 or ws == 1:
        build.build()
    if ws > 1:
        torch.distributed.barrier()
    from paper_2001_03389_gb300 import rfim, synth

    spec = workload_spec(WORKLOAD)
    if args.beams:
        spec["B"] = args.beams  # a smaller batch of the same beams (profiling captures)

    if args.profile:
        # profiling mode: W warm-up steps, K plain steps, nothing else
        B, C, T = spec["B"], spec["C"], spec["T"]
        if spec["dtype"] == "u8":
            xin = torch.from_numpy(synth.make_beams(WORKLOAD, beams=range(B))).to(dev)
        else:
            xin = synth.torch_make_beams(WORKLOAD, B, synth.seed_of(WORKLOAD), dev)
        out = torch.empty_like(xin)
        mask = torch.zeros(rfim.mask_words(C, T, B), dtype=torch.int32, device=dev)
        ctx = rfim.Context(local)
        blk = ctx.block(xin, out, mask, "bct", "bits")
        td, fd = rfim.make_cut(**spec["tdsc"]), rfim.make_cut(**spec["fdsc"])
        stream = torch.cuda.Stream(device=dev)
        for _ in range(max(3, args.warmup) + args.steps):
            ctx.clean(blk, td, fd, stream)
        stream.synchronize()
        print(json.dumps({"profile_run": True, "steps": args.steps, "status": ctx.device_status(stream),
                          "source_hash": source_hash(WORKLOAD)}), flush=True)
        ctx.close()
        return

    main = measure_fixed(rfim, synth, dev, spec, WORKLOAD, args.steps, args.warmup, args, ws, rank)
    if rank == 0:
        res = {
            "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": spec["dtype"], "data": "synthetic", "config": config_json(spec, ws),
            "samples_per_s": main["samples_per_s"], "roofline": main["roofline"], "e2e": main["e2e"],
            "e2e_matches_device": main["e2e_matches_device"], "gpu_launches": main["gpu_launches"],
        }
        for k in ("clocks", "cpu_baseline", "parity"):
            if k in main:
                res[k] = main[k]
        if ws == 1 and not args.main_only and WORKLOAD == ARTS:
            configs = {}
            fspec = workload_spec(FP32)
            configs[FP32] = dict(measure_fixed(rfim, synth, dev, fspec, FP32, args.steps_fp32, 3, args,
                                               cpu_budget_s=8.0), config=config_json(fspec, 1))
            configs[RAGGED] = measure_ragged(rfim, synth, dev)
            configs["arts_btc_layout"] = measure_btc(rfim, synth, dev)
            res["configs"] = configs
            res["gpu_launches"] += configs[FP32]["gpu_launches"]
        if ws == 1 and not args.no_stream and WORKLOAD == ARTS:
            res["streaming"] = run_stream_bench(rfim, synth, dev, duration_s=args.stream_seconds)
        print(json.dumps(res), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


# per workload: the committed ncu summary of its kernel, the kernel's sources, its name
PROFILES = {
    ARTS: ("engine_u8_arts12.md", ("common.cuh", "engine.h", "engine_u8_impl.cuh", "engine_u8.cu"),
           "k_engine_u8 (fused TDSC->FDSC persistent work queue)"),
    FP32: ("engine_f32_fp32x32.md", ("common.cuh", "engine.h", "engine_f32.cu"),
           "k_engine_f32 (fused TDSC->FDSC persistent work queue)"),
}


# ---------------------------------------------------------------------------
# streaming service: Poisson arrivals of 1536 x 1250 uint8 chunks from 480 beams
# ---------------------------------------------------------------------------
def run_stream_bench(rfim, synth, dev, rates=(10, 25, 50, 100), duration_s=5.0, seed=2001033895):
    """Latency percentiles and sustained GB/s of the streaming service at m x the
    ARTS input rate of 73 Gb/s (480 beams of 1536 channels sampled every
    81.92 us; a 1250-sample chunk lasts 102.4 ms).  Chunks come from a pool of 4
    per beam resident in HBM (device ingest, read in place by the kernels)."""
    import torch

    n_beams, C, T = 480, 1536, 1250
    per_beam = 4
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    pool = torch.empty((n_beams * per_beam, C, T), dtype=torch.uint8, device=dev)
    model = synth.arts_model()
    for i in range(pool.shape[0]):
        pool[i] = synth.torch_beam_u8(gen, C, T, model, dev)
    torch.cuda.synchronize()
    base = pool.data_ptr()
    cb = C * T
    ctx = rfim.Context(dev.index or 0)
    td = rfim.make_cut(3.0, 2, "median")
    fd = rfim.make_cut(3.0, 2, "median", 32)
    ctx.stream_open(n_beams, C, T, rfim.U8, td, fd)
    rng = np.random.default_rng(seed)
    chunk_rate = 73e9 / (8 * C * T)  # ARTS input rate, 73 Gb/s (Sec. I), in 1536 x 1250 chunks: 4753 /s

    def replay(m, dur):
        n = max(1, int(m * chunk_rate * dur))
        arr = time.monotonic() + 0.02 + np.cumsum(rng.exponential(1.0 / (m * chunk_rate), n))
        beams = np.arange(n) % n_beams
        ptrs = base + (beams * per_beam + (np.arange(n) // n_beams) % per_beam) * cb
        ctx.stream_replay(beams, ptrs, arr)
        return ctx.stream_stats(reset=True)

    replay(10, 0.1)  # warm-up
    out = []
    for m in rates:
        st = replay(m, duration_s)
        out.append({"rate_x_arts": m, "offered_chunks_per_s": m * chunk_rate,
                    "offered_gbps": m * chunk_rate * cb / 1e9, "gbps": st["gbps"], "chunks": st["chunks"],
                    "p50_ms": st["p50_s"] * 1e3, "p99_ms": st["p99_s"] * 1e3, "p999_ms": st["p999_s"] * 1e3,
                    "sustained": bool(st["gbps"] >= 0.95 * m * chunk_rate * cb / 1e9 and st["p99_s"] < 0.1024)})
    state = ctx.stream_beam_state(0, C)
    ctx.stream_close()
    ctx.close()
    del pool
    torch.cuda.empty_cache()
    return {"workload": "480 beams x 1536 ch x 1250-sample uint8 chunks, Poisson arrivals, TDSC+FDSC k=3 median",
            "ingest": "device (chunks read in place from an HBM pool of 4 per beam)",
            "latency": "scheduled arrival -> completion seen by the host", "budget_ms": 102.4,
            "duration_s_per_rate": duration_s, "rates": out,
            "per_beam_state": {"kept": state is not None,
                               "what": "latest completed chunk per beam resident on the device: cleaned data, "
                                       "mask, per-channel input sum and sum of squares"}}


def profiled_traffic(workload):
    """DRAM bytes per launch of the engine kernel from the committed ncu summary,
    or None when the kernel sources changed since that capture."""
    prof = os.path.join(ROOT, "profiles", PROFILES[workload][0])
    if not os.path.exists(prof):
        return None
    vals = {}
    with open(prof) as fh:
        for line in fh:
            if line.startswith("traffic:"):
                for kv in line.split()[1:]:
                    if "=" in kv:
                        k, v = kv.split("=", 1)
                        vals[k] = v
    if vals.get("source_hash") != source_hash(workload):
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def source_hash(workload):
    """Hash of the sources the engine kernel of the workload is compiled from."""
    import hashlib

    h = hashlib.sha256()
    cs = os.path.join(ROOT, "paper_2001_03389_gb300", "csrc")
    for f in PROFILES[workload][1]:
        with open(os.path.join(cs, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default 2000, or 300 for the float32 workload)")
    ap.add_argument("--workload", default=ARTS, choices=[ARTS, FP32],
                    help=f"{ARTS}: the ARTS uint8 batch (the reported workload); {FP32}: the float32 workload alone")
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--steps-fp32", type=int, default=100, help="timed steps of the float32 sub-record")
    ap.add_argument("--beams", type=int, default=None, help="clean only the first N beams (profiling captures)")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-stream", action="store_true", help="skip the streaming-service measurement")
    ap.add_argument("--stream-seconds", type=float, default=5.0, help="duration of each streaming rate")
    ap.add_argument("--main-only", action="store_true", help="skip the float32 and ragged sub-records")
    ap.add_argument("--profile", action="store_true", help="warm-up and plain steps only (for ncu captures)")
    args = ap.parse_args()
    global WORKLOAD
    WORKLOAD = args.workload
    if args.steps is None:
        args.steps = 2000 if WORKLOAD == ARTS else 300
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
