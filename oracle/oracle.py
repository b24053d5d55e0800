"""ctypes binding of the CPU oracle (rfim_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
benchmark's CPU-baseline leg may import this module.  It never imports the
GPU package and the GPU package never imports it.

`build()` compiles rfim_oracle.c with gcc (-O2 -ffp-contract=off, so each
floating-point operation is one IEEE rounding on every host architecture).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rfim_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

LAYOUT = {"bct": 0, "btc": 1}
REPLACE = {"mean": 0, "median": 1, "random": 2}


class OrcCut(ctypes.Structure):
    _fields_ = [
        ("enabled", ctypes.c_int),
        ("k", ctypes.c_double),
        ("iterations", ctypes.c_int),
        ("replace", ctypes.c_int),
        ("bin", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (skipped when up to date)."""
    deps = [SRC, os.path.join(HERE, "rfim_oracle.h")]
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(d) for d in deps):
        return LIB
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        f32p = ctypes.POINTER(ctypes.c_float)
        i64 = ctypes.c_int64
        cutp = ctypes.POINTER(OrcCut)
        L.orc_clean_u8.argtypes = [u8p, u8p, u8p, i64, i64, i64, ctypes.c_int, cutp, cutp]
        L.orc_clean_u8.restype = ctypes.c_int
        L.orc_clean_f32.argtypes = [f32p, f32p, u8p, i64, i64, i64, ctypes.c_int, cutp, cutp]
        L.orc_clean_f32.restype = ctypes.c_int
        L.orc_clean_u8_interleaved.argtypes = [u8p, u8p, u8p, i64, i64, i64, ctypes.c_int, cutp, cutp]
        L.orc_clean_u8_interleaved.restype = ctypes.c_int
        L.orc_clean_f32_interleaved.argtypes = [f32p, f32p, u8p, i64, i64, i64, ctypes.c_int, cutp, cutp]
        L.orc_clean_f32_interleaved.restype = ctypes.c_int
        L.orc_mix64.argtypes = [ctypes.c_uint64]
        L.orc_mix64.restype = ctypes.c_uint64
        L.orc_draw.argtypes = [ctypes.c_int, ctypes.c_int, i64, i64, i64, ctypes.c_int, i64]
        L.orc_draw.restype = i64
        f64p = ctypes.POINTER(ctypes.c_double)
        L.orc_clean_f32m.argtypes = [f32p, f32p, u8p, f64p, i64, i64, i64, ctypes.c_int, cutp, cutp]
        L.orc_clean_f32m.restype = ctypes.c_int
        L.orc_tdsc_row_u8.argtypes = [u8p, u8p, i64, ctypes.c_double, ctypes.c_int, ctypes.c_int]
        L.orc_fdsc_col_u8.argtypes = [u8p, u8p, i64, ctypes.c_double, ctypes.c_int, ctypes.c_int, i64]
        L.orc_tdsc_row_f32.argtypes = [f32p, u8p, i64, ctypes.c_double, ctypes.c_int, ctypes.c_int]
        L.orc_fdsc_col_f32.argtypes = [f32p, u8p, i64, ctypes.c_double, ctypes.c_int, ctypes.c_int, i64]
        L.orc_lower_median_u8.argtypes = [u8p, i64]
        L.orc_lower_median_u8.restype = ctypes.c_uint8
        L.orc_lower_median_f32.argtypes = [f32p, i64]
        L.orc_lower_median_f32.restype = ctypes.c_float
        _lib = L
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def make_cut(cut: dict | None, bin_default: int = 0) -> OrcCut:
    if cut is None:
        return OrcCut(0, 0.0, 0, 0, 0)
    return OrcCut(
        1,
        float(cut["k"]),
        int(cut.get("iterations", 1)),
        REPLACE[cut.get("replace", "mean")],
        int(cut.get("bin", bin_default) or bin_default),
    )


class OracleError(RuntimeError):
    def __init__(self, rc):
        super().__init__(f"oracle returned {rc}")
        self.rc = rc


def clean(x: np.ndarray, layout: str = "bct", tdsc: dict | None = None, fdsc: dict | None = None,
          order: str = "blocked"):
    """Clean a 3-D filterbank block.

    x: uint8 or float32 array shaped (B, C, T) for layout 'bct' or (B, T, C)
    for 'btc'.  tdsc / fdsc: dicts with k, iterations, replace ('mean' or
    'median') and, for fdsc, bin (defaults to 32 capped at C).
    order: 'blocked' (all TDSC iterations, then all FDSC iterations) or
    'interleaved' (TDSC iteration i, then FDSC iteration i, per round).
    Returns (out, flags) where flags holds bit 0 = TDSC, bit 1 = FDSC.
    """
    if order not in ("blocked", "interleaved"):
        raise ValueError(order)
    x = np.ascontiguousarray(x)
    if layout == "bct":
        B, C, T = x.shape
    else:
        B, T, C = x.shape
    tc = make_cut(tdsc)
    fc = make_cut(fdsc, bin_default=min(32, C))
    out = np.empty_like(x)
    flags = np.zeros(x.shape, dtype=np.uint8)
    L = lib()
    il = order == "interleaved"
    if x.dtype == np.uint8:
        fn = L.orc_clean_u8_interleaved if il else L.orc_clean_u8
        rc = fn(_ptr(x, ctypes.c_uint8), _ptr(out, ctypes.c_uint8), _ptr(flags, ctypes.c_uint8),
                B, C, T, LAYOUT[layout], ctypes.byref(tc), ctypes.byref(fc))
    elif x.dtype == np.float32:
        fn = L.orc_clean_f32_interleaved if il else L.orc_clean_f32
        rc = fn(_ptr(x, ctypes.c_float), _ptr(out, ctypes.c_float), _ptr(flags, ctypes.c_uint8),
                B, C, T, LAYOUT[layout], ctypes.byref(tc), ctypes.byref(fc))
    else:
        raise TypeError(f"unsupported dtype {x.dtype}")
    if rc != 0:
        raise OracleError(rc)
    return out, flags


def tdsc_row(row: np.ndarray, k: float, iterations: int = 1, replace: str = "mean"):
    """TDSC on one row (uint8 or float32).  Returns (cleaned row, flags)."""
    v = np.array(row, copy=True)
    f = np.zeros(v.shape[0], dtype=np.uint8)
    L = lib()
    if v.dtype == np.uint8:
        L.orc_tdsc_row_u8(_ptr(v, ctypes.c_uint8), _ptr(f, ctypes.c_uint8), v.shape[0], k, iterations, REPLACE[replace])
    else:
        v = v.astype(np.float32)
        L.orc_tdsc_row_f32(_ptr(v, ctypes.c_float), _ptr(f, ctypes.c_uint8), v.shape[0], k, iterations, REPLACE[replace])
    return v, f


def fdsc_col(col: np.ndarray, k: float, iterations: int = 1, replace: str = "mean", bin: int = 32):
    """FDSC on one column of channels (uint8 or float32).  Returns (cleaned, flags)."""
    v = np.array(col, copy=True)
    f = np.zeros(v.shape[0], dtype=np.uint8)
    L = lib()
    if v.dtype == np.uint8:
        L.orc_fdsc_col_u8(_ptr(v, ctypes.c_uint8), _ptr(f, ctypes.c_uint8), v.shape[0], k, iterations, REPLACE[replace], bin)
    else:
        v = v.astype(np.float32)
        L.orc_fdsc_col_f32(_ptr(v, ctypes.c_float), _ptr(f, ctypes.c_uint8), v.shape[0], k, iterations, REPLACE[replace], bin)
    return v, f


def lower_median(v: np.ndarray):
    v = np.ascontiguousarray(v)
    L = lib()
    if v.dtype == np.uint8:
        return int(L.orc_lower_median_u8(_ptr(v, ctypes.c_uint8), v.shape[0]))
    v = v.astype(np.float32)
    return float(L.orc_lower_median_f32(_ptr(v, ctypes.c_float), v.shape[0]))


def clean_f32_margin(x: np.ndarray, layout: str = "bct", tdsc: dict | None = None, fdsc: dict | None = None):
    """clean() of a float32 block that also returns, per sample, the relative
    distance |(|x - mu| - k sigma)| / (k sigma) of its closest decision (inf
    where sigma = 0): the measure the float32 tolerance is stated in."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    if layout == "bct":
        B, C, T = x.shape
    else:
        B, T, C = x.shape
    tc = make_cut(tdsc)
    fc = make_cut(fdsc, bin_default=min(32, C))
    out = np.empty_like(x)
    flags = np.zeros(x.shape, dtype=np.uint8)
    margin = np.empty(x.shape, dtype=np.float64)
    rc = lib().orc_clean_f32m(_ptr(x, ctypes.c_float), _ptr(out, ctypes.c_float), _ptr(flags, ctypes.c_uint8),
                              _ptr(margin, ctypes.c_double), B, C, T, LAYOUT[layout], ctypes.byref(tc),
                              ctypes.byref(fc))
    if rc != 0:
        raise OracleError(rc)
    return out, flags, margin


def mix64(z: int) -> int:
    """SplitMix64 output function of the random-replacement draws."""
    return int(lib().orc_mix64(z & 0xFFFFFFFFFFFFFFFF))


def draw(method: int, it: int, beam: int, line: int, index: int, attempt: int, n: int) -> int:
    """Position in [0, n) of a random-replacement attempt (see rfim_oracle.h)."""
    return int(lib().orc_draw(method, it, beam, line, index, attempt, n))
