"""Helpers for the GPU parity tests: run the library through its C ABI and
unpack its masks.  (No cleaning arithmetic lives here.)"""
import numpy as np


def unpack_bits(words: np.ndarray, rows: int, n: int) -> np.ndarray:
    """uint32 words (rows x ceil(n/32)) -> bool (rows x n), bit i%32 of word i/32."""
    w = np.ascontiguousarray(words).view(np.uint32).reshape(rows, -1)
    b = np.unpackbits(w.view(np.uint8), axis=-1, bitorder="little")
    return b[:, :n].astype(bool)


GUARD = 64


def run_gpu(ctx, x, layout="bct", tdsc=None, fdsc=None, mask_fmt="bits", in_place=False, in_off=0, out_off=0,
            api="clean", stream=None):
    """Clean the numpy block x ((B, C, T) for 'bct', (B, T, C) for 'btc') on the
    GPU through the C ABI.  in_off / out_off shift the device pointers by that
    many bytes (misaligned buffers; multiples of 4 for float32).  Guard bytes
    around the output and the mask are checked for stray writes.  Returns
    (out, flags): flags is bool for 'bits', the flag bytes for 'bytes'."""
    import torch

    from paper_2001_03389_gb300 import rfim

    dev = torch.device("cuda:0")
    B = x.shape[0]
    C, T = (x.shape[1], x.shape[2]) if layout == "bct" else (x.shape[2], x.shape[1])
    n = x.size
    es = x.itemsize
    tdt = torch.uint8 if x.dtype == np.uint8 else torch.float32
    host = torch.from_numpy(np.ascontiguousarray(x).reshape(-1).view(np.uint8))
    raw_in = torch.zeros(n * es + 2 * GUARD, dtype=torch.uint8, device=dev)
    raw_in[GUARD + in_off:GUARD + in_off + n * es].copy_(host.to(dev))
    xin = raw_in[GUARD + in_off:GUARD + in_off + n * es].view(tdt).view(x.shape)
    if in_place:
        raw_out, oo, out = raw_in, GUARD + in_off, xin
    else:
        raw_out = torch.full((n * es + 2 * GUARD,), 0xAB, dtype=torch.uint8, device=dev)
        oo = GUARD + out_off
        out = raw_out[oo:oo + n * es].view(tdt).view(x.shape)
    rows = B * (C if layout == "bct" else T)
    fast = T if layout == "bct" else C
    W = (fast + 31) // 32
    if mask_fmt == "bits":
        raw_mask = torch.full((rows * W + 2 * GUARD,), -1, dtype=torch.int32, device=dev)
        mask = raw_mask[GUARD:GUARD + rows * W]
    elif mask_fmt == "bytes":
        raw_mask = torch.full((n + 2 * GUARD,), 0xEE, dtype=torch.uint8, device=dev)
        mask = raw_mask[GUARD:GUARD + n]
    else:
        raw_mask = mask = None
    blk = rfim.Context.block(xin, out, mask, layout, mask_fmt)
    if api == "clean":
        ctx.clean(blk, tdsc, fdsc, stream)
    elif api == "tdsc":
        ctx.tdsc(blk, tdsc, stream)
    elif api == "fdsc":
        ctx.fdsc(blk, fdsc, stream)
    else:
        raise ValueError(api)
    torch.cuda.synchronize()
    ro = raw_out.cpu().numpy()
    got = ro[oo:oo + n * es].view(x.dtype).reshape(x.shape).copy()
    if not in_place:
        assert np.all(ro[:oo] == 0xAB) and np.all(ro[oo + n * es:] == 0xAB), "output written outside its buffer"
    else:
        assert np.all(ro[:oo] == 0) and np.all(ro[oo + n * es:] == 0), "data written outside its buffer"
    flags = None
    if mask_fmt == "bits":
        m = raw_mask.cpu().numpy()
        assert np.all(m[:GUARD] == -1) and np.all(m[GUARD + rows * W:] == -1), "bit mask written outside its buffer"
        words = m[GUARD:GUARD + rows * W].view(np.uint32).reshape(rows, W)
        if fast % 32:
            assert np.all((words[:, -1] >> (fast % 32)) == 0), "padding bits set"
        flags = unpack_bits(words, rows, fast).reshape(x.shape)
    elif mask_fmt == "bytes":
        m = raw_mask.cpu().numpy()
        assert np.all(m[:GUARD] == 0xEE) and np.all(m[GUARD + n:] == 0xEE), "byte mask written outside its buffer"
        flags = m[GUARD:GUARD + n].reshape(x.shape).copy()
    return got, flags


def noise_u8(rng, shape, rfi=True):
    """Small uint8 test blocks: N(128, 16^2) with bright samples and channels."""
    x = np.clip(np.rint(rng.normal(128, 16, shape)), 0, 255).astype(np.uint8)
    if rfi and x.size > 8:
        flat = x.reshape(-1)
        idx = rng.integers(0, flat.size, max(1, flat.size // 200))
        flat[idx] = rng.integers(200, 256, idx.size).astype(np.uint8)
        flat[rng.integers(0, flat.size, max(1, flat.size // 500))] = 0
    return x


class _RawDevice:
    def __init__(self, ptr, nbytes):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (int(ptr), False),
                                         "version": 3}


def device_bytes(ptr, nbytes):
    """A uint8 torch view of nbytes of device memory at a raw pointer (no copy)."""
    import torch

    return torch.as_tensor(_RawDevice(ptr, nbytes), device="cuda")
