"""Arithmetic identities the uint8 kernels rely on, checked on the CPU.

These are not pins of the oracle: they check, by brute force over random and
edge-case bytes, two shortcuts the FDSC item takes on 32-channel bins, so a
reader can see that they decide exactly what the definition decides.

1. The flag pass.  A byte x of a bin with sum S is flagged iff |32 x - S| > A
   (the exact keep rule for 32-channel bins when every bin has 32 channels,
   Sec. IV FDSC paragraph with the integer reading of the sigma test), so the
   bin holds a flagged byte iff 32 max - S > A or S - 32 min > A.
2. The byte extremes.  The maximum (minimum) of two unsigned 16-bit lanes has
   the larger (smaller) high byte, so the 16-bit lane extremes of the words
   carry the extremes of bytes 1 and 3 in their high bytes, and those of the
   words shifted up one byte carry the extremes of bytes 0 and 2.
"""
import numpy as np


def bins(rng, n):
    """n bins of 32 bytes: noise, bins with outliers, constant bins, extremes."""
    x = np.clip(np.rint(rng.normal(128, 16, size=(n, 32))), 0, 255).astype(np.int64)
    k = n // 4
    x[:k, rng.integers(0, 32, k)] = rng.integers(0, 256, k)  # one bright or dark byte
    x[k:2 * k] = rng.integers(0, 256, size=(k, 32))           # uniform bytes
    x[2 * k:2 * k + 8] = rng.integers(0, 256, size=(8, 1))     # constant bins
    x[2 * k + 8] = 0
    x[2 * k + 9] = 255
    x[2 * k + 10, ::2] = 0
    x[2 * k + 10, 1::2] = 255
    return x


def test_bin_flag_test_from_extremes():
    rng = np.random.default_rng(2001033890)
    x = bins(rng, 4000)
    S = x.sum(axis=1)
    for A in [0, 1, 15, 31, 32, 33, 100, 480, 1536, 4000, 8160, 8161]:
        flagged = np.abs(32 * x - S[:, None]) > A                  # the definition, byte by byte
        any_def = flagged.any(axis=1)
        mx, mn = x.max(axis=1), x.min(axis=1)
        any_ext = (32 * mx - S > A) | (S - 32 * mn > A)            # the two comparisons
        assert np.array_equal(any_def, any_ext), A


def vmax2(a, b):
    """Unsigned 16-bit lane maximum of two uint32 words (numpy model)."""
    lo = np.maximum(a & 0xFFFF, b & 0xFFFF)
    hi = np.maximum(a >> 16, b >> 16)
    return (hi << 16) | lo


def vmin2(a, b):
    lo = np.minimum(a & 0xFFFF, b & 0xFFFF)
    hi = np.minimum(a >> 16, b >> 16)
    return (hi << 16) | lo


def extremes_from_words(w):
    """The kernel's reduction over the 8 words of a bin (w: (n, 8) uint32)."""
    w = w.astype(np.uint64)
    u = (w << 8) & 0xFFFFFFFF
    hx, lx, hn, ln = w[:, 0], u[:, 0], w[:, 0], u[:, 0]
    for i in range(1, 8):
        hx, lx = vmax2(hx, w[:, i]), vmax2(lx, u[:, i])
        hn, ln = vmin2(hn, w[:, i]), vmin2(ln, u[:, i])
    x, n = vmax2(hx, lx), vmin2(hn, ln)
    mx = np.maximum(x >> 24, (x >> 8) & 0xFF)
    mn = np.minimum(n >> 24, (n >> 8) & 0xFF)
    return mx.astype(np.int64), mn.astype(np.int64)


def test_byte_extremes_from_16bit_lanes():
    rng = np.random.default_rng(7)
    x = bins(rng, 4000).astype(np.uint8)
    # all orders of one extreme byte over the 32 positions, on a flat background
    for v, bg in [(255, 0), (0, 255), (200, 17), (3, 250)]:
        b = np.full((32, 32), bg, dtype=np.uint8)
        b[np.arange(32), np.arange(32)] = v
        x = np.concatenate([x, b])
    w = x.reshape(-1, 8, 4).astype(np.uint32)
    words = w[..., 0] | (w[..., 1] << 8) | (w[..., 2] << 16) | (w[..., 3] << 24)  # little-endian bytes
    mx, mn = extremes_from_words(words)
    assert np.array_equal(mx, x.max(axis=1))
    assert np.array_equal(mn, x.min(axis=1))
