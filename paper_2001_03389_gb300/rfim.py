"""Thin Python binding of librfim.so (ctypes).

Functions carry the C ABI's names and only marshal arguments; every step of
the cleaning runs in the library's CUDA kernels.  PyTorch is used for device
memory and streams only.  Importing this module loads the in-tree
librfim.so and raises ImportError if it is missing (build it with
`python -m paper_2001_03389_gb300.build`): there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librfim.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "rfim.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2001_03389_gb300.build`")
_lib = ctypes.CDLL(LIB_PATH)

# ---- enums (include/rfim.h)
OK, ERR_ARG, ERR_RANGE, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_BUSY, ERR_STATE = range(8)
U8, F32 = 0, 1
LAYOUT_BCT, LAYOUT_BTC = 0, 1
REPLACE_MEAN, REPLACE_MEDIAN, REPLACE_RANDOM = 0, 1, 2
MASK_NONE, MASK_BITS, MASK_BYTES = 0, 1, 2
BATCH_GRAPH, BATCH_AUTOTUNE = 1, 2
RFIM_NOALLOC_MAX_BEAMS = 160

_LAYOUTS = {"bct": LAYOUT_BCT, "btc": LAYOUT_BTC}
_REPLACE = {"mean": REPLACE_MEAN, "median": REPLACE_MEDIAN, "random": REPLACE_RANDOM}
_MASKS = {None: MASK_NONE, "none": MASK_NONE, "bits": MASK_BITS, "bytes": MASK_BYTES}


class rfim_cut(ctypes.Structure):
    _fields_ = [("k", ctypes.c_double), ("iterations", ctypes.c_int), ("replace", ctypes.c_int),
                ("fdsc_bin", ctypes.c_int)]


class rfim_block(ctypes.Structure):
    _fields_ = [("in_", ctypes.c_void_p), ("out", ctypes.c_void_p), ("mask", ctypes.c_void_p),
                ("beams", ctypes.c_int), ("channels", ctypes.c_int), ("samples", ctypes.c_int),
                ("dtype", ctypes.c_int), ("layout", ctypes.c_int), ("mask_fmt", ctypes.c_int)]


_vp = ctypes.c_void_p
_cutp = ctypes.POINTER(rfim_cut)
_blkp = ctypes.POINTER(rfim_block)
_SIGS = {
    "rfim_create": ([ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_size_t, ctypes.c_char_p], ctypes.c_int),
    "rfim_destroy": ([_vp], ctypes.c_int),
    "rfim_set_option": ([_vp, ctypes.c_char_p, ctypes.c_longlong], ctypes.c_int),
    "rfim_tdsc": ([_vp, _blkp, _cutp, _vp], ctypes.c_int),
    "rfim_fdsc": ([_vp, _blkp, _cutp, _vp], ctypes.c_int),
    "rfim_clean": ([_vp, _blkp, _cutp, _cutp, _vp], ctypes.c_int),
    "rfim_clean_batch": ([_vp, _blkp, ctypes.c_int, _cutp, _cutp, ctypes.c_uint, _vp], ctypes.c_int),
    "rfim_clean_host": ([_vp, _blkp, _cutp, _cutp], ctypes.c_int),
    "rfim_device_status": ([_vp, _vp], ctypes.c_int),
    "rfim_clean_noalloc": ([_blkp, _cutp, _cutp, _vp], ctypes.c_int),
    "rfim_noalloc_status": ([_vp], ctypes.c_int),
    "rfim_stream_open": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _cutp, _cutp], ctypes.c_int),
    "rfim_stream_push": ([_vp, ctypes.c_int, _vp, ctypes.c_double, ctypes.POINTER(ctypes.c_ulonglong)], ctypes.c_int),
    "rfim_stream_poll": ([_vp, ctypes.c_ulonglong, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_int], ctypes.c_int),
    "rfim_stream_release": ([_vp, ctypes.c_ulonglong], ctypes.c_int),
    "rfim_stream_beam_state": ([_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(_vp), ctypes.POINTER(_vp)], ctypes.c_int),
    "rfim_stream_replay": ([_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_vp),
                            ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "rfim_stream_stats": ([_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_ulonglong), ctypes.c_int], ctypes.c_int),
    "rfim_stream_close": ([_vp], ctypes.c_int),
    "rfim_status_str": ([ctypes.c_int], ctypes.c_char_p),
    "rfim_last_error": ([_vp], ctypes.c_char_p),
    "rfim_version": ([], ctypes.c_char_p),
}
for _name, (_args, _res) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = _res
    globals()[_name] = _fn


def header_functions():
    """Names of the functions declared in include/rfim.h."""
    with open(HEADER) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rfim_[a-z_0-9]+)\s*\(", text)))


class RfimError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{rfim_status_str(status).decode()}: {msg}")
        self.status = status


def make_cut(k, iterations=1, replace="mean", bin=0):
    return rfim_cut(float(k), int(iterations), _REPLACE[replace] if isinstance(replace, str) else int(replace), int(bin))


def _cut_arg(c):
    if c is None:
        return None
    if isinstance(c, dict):
        c = make_cut(c["k"], c.get("iterations", 1), c.get("replace", "mean"), c.get("bin", 0))
    return ctypes.byref(c)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Context:
    """An rfim_ctx on one device; methods take torch tensors (device memory)."""

    def __init__(self, device: int = 0, hbm_budget: int = 0, tune_cache: str | None = None):
        h = _vp()
        st = rfim_create(ctypes.byref(h), int(device), int(hbm_budget),
                         tune_cache.encode() if tune_cache else None)
        if st != OK:
            raise RfimError(st, f"rfim_create(device={device})")
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            rfim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != OK:
            raise RfimError(st, f"{what}: {rfim_last_error(self.h).decode()}")

    def set_option(self, key: str, value: int):
        self._check(rfim_set_option(self.h, key.encode(), int(value)), f"set_option({key})")

    @staticmethod
    def block(x, out=None, mask=None, layout="bct", mask_fmt=None):
        """rfim_block for a 3-D tensor x shaped (B, C, T) ('bct') or (B, T, C) ('btc')."""
        import torch

        if x.dim() != 3:
            raise ValueError("expected a (beams, channels, samples) tensor")
        if x.dtype == torch.uint8:
            dt = U8
        elif x.dtype == torch.float32:
            dt = F32
        else:
            raise TypeError(f"unsupported dtype {x.dtype}")
        B = x.shape[0]
        C, T = (x.shape[1], x.shape[2]) if layout == "bct" else (x.shape[2], x.shape[1])
        mf = _MASKS[mask_fmt] if mask is not None else MASK_NONE
        return rfim_block(_ptr(x), _ptr(out if out is not None else x), _ptr(mask), B, C, T, dt, _LAYOUTS[layout], mf)

    def tdsc(self, blk, cut, stream=None):
        self._check(rfim_tdsc(self.h, ctypes.byref(blk), _cut_arg(cut), _stream_ptr(stream)), "rfim_tdsc")

    def fdsc(self, blk, cut, stream=None):
        self._check(rfim_fdsc(self.h, ctypes.byref(blk), _cut_arg(cut), _stream_ptr(stream)), "rfim_fdsc")

    def clean(self, blk, tdsc=None, fdsc=None, stream=None):
        self._check(rfim_clean(self.h, ctypes.byref(blk), _cut_arg(tdsc), _cut_arg(fdsc), _stream_ptr(stream)),
                    "rfim_clean")

    def clean_batch(self, blocks, tdsc=None, fdsc=None, flags=0, stream=None):
        arr = (rfim_block * len(blocks))(*blocks)
        self._check(rfim_clean_batch(self.h, arr, len(blocks), _cut_arg(tdsc), _cut_arg(fdsc), int(flags),
                                     _stream_ptr(stream)), "rfim_clean_batch")

    def clean_host(self, blk, tdsc=None, fdsc=None):
        self._check(rfim_clean_host(self.h, ctypes.byref(blk), _cut_arg(tdsc), _cut_arg(fdsc)), "rfim_clean_host")

    def device_status(self, stream=None):
        return rfim_device_status(self.h, _stream_ptr(stream))

    # ---- streaming service
    def stream_open(self, n_beams, channels, chunk_samples, dtype=U8, tdsc=None, fdsc=None):
        self._check(rfim_stream_open(self.h, int(n_beams), int(channels), int(chunk_samples), int(dtype),
                                     _cut_arg(tdsc), _cut_arg(fdsc)), "rfim_stream_open")

    def stream_push(self, beam, chunk, arrival_s):
        """Returns the ticket, or None when no slot is free (RFIM_ERR_BUSY)."""
        t = ctypes.c_ulonglong()
        st = rfim_stream_push(self.h, int(beam), _ptr(chunk), float(arrival_s), ctypes.byref(t))
        if st == ERR_BUSY:
            return None
        self._check(st, "rfim_stream_push")
        return t.value

    def stream_poll(self, ticket, wait_us=0):
        """(out_ptr, mask_ptr) when done, None while in flight."""
        o, m = _vp(), _vp()
        st = rfim_stream_poll(self.h, ticket, ctypes.byref(o), ctypes.byref(m), int(wait_us))
        if st == ERR_BUSY:
            return None
        self._check(st, "rfim_stream_poll")
        return o.value, m.value

    def stream_release(self, ticket):
        self._check(rfim_stream_release(self.h, ticket), "rfim_stream_release")

    def stream_beam_state(self, beam, channels):
        """(chunk index, stats (channels x 2: input sum, sum of squares), out_ptr,
        mask_ptr) of the beam's latest completed chunk, or None before its first."""
        import numpy as np

        idx = ctypes.c_ulonglong()
        stats = np.zeros((channels, 2), dtype=np.float64)
        o, m = _vp(), _vp()
        st = rfim_stream_beam_state(self.h, int(beam), ctypes.byref(idx),
                                    stats.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(o),
                                    ctypes.byref(m))
        if st == ERR_BUSY:
            return None
        self._check(st, "rfim_stream_beam_state")
        return idx.value, stats, o.value, m.value

    def stream_replay(self, beams, chunk_ptrs, arrivals):
        import numpy as np

        b = np.ascontiguousarray(beams, dtype=np.int32)
        c = np.ascontiguousarray(chunk_ptrs, dtype=np.uint64)
        a = np.ascontiguousarray(arrivals, dtype=np.float64)
        n = int(b.shape[0])
        if c.shape[0] != n or a.shape[0] != n:
            raise ValueError("beams, chunk_ptrs and arrivals differ in length")
        self._check(rfim_stream_replay(self.h, n, b.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                       ctypes.cast(c.ctypes.data, ctypes.POINTER(_vp)),
                                       a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "rfim_stream_replay")

    def stream_stats(self, reset=False):
        p50, p99, p999, g = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_ulonglong()
        self._check(rfim_stream_stats(self.h, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(p999),
                                      ctypes.byref(g), ctypes.byref(n), int(bool(reset))), "rfim_stream_stats")
        return {"p50_s": p50.value, "p99_s": p99.value, "p999_s": p999.value, "gbps": g.value, "chunks": n.value}

    def stream_close(self):
        self._check(rfim_stream_close(self.h), "rfim_stream_close")

    def last_error(self) -> str:
        return rfim_last_error(self.h).decode()


def mask_words(C: int, T: int, B: int = 1) -> int:
    """uint32 words of a BCT bit mask."""
    return B * C * ((T + 31) // 32)
