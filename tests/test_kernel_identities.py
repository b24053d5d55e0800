"""Arithmetic identities the uint8 kernels rely on, checked on the CPU.

These are not pins of the oracle: they check, by brute force over random and
edge-case bytes, the shortcuts the kernels take, so a reader can see that
they decide exactly what the definition decides.

1. The flag pass.  A byte x of a bin with sum S is flagged iff |32 x - S| > A
   (the exact keep rule for 32-channel bins when every bin has 32 channels,
   Sec. IV FDSC paragraph with the integer reading of the sigma test), so the
   bin holds a flagged byte iff 32 max - S > A or S - 32 min > A.
2. The byte extremes.  The maximum (minimum) of two unsigned 16-bit lanes has
   the larger (smaller) high byte, so the 16-bit lane extremes of the words
   carry the extremes of bytes 1 and 3 in their high bytes, and those of the
   words shifted up one byte carry the extremes of bytes 0 and 2.
3. The median window.  Both median searches (TDSC rows, FDSC bins) start
   inside [floor(mu - sigma) - 1, ceil(mu + sigma) + 1], which holds the
   lower median because any median is within one population sigma of the
   mean.
4. Counting by sums of absolute differences.  With f(p) the sum of |x - p|,
   #(x <= p) = (n + f(p + 1) - f(p)) / 2, which is how both searches count.
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


def lower_median(x):
    """Rank floor((n - 1) / 2) (0-based) of each row, the lower median."""
    return np.sort(x, axis=1)[:, (x.shape[1] - 1) // 2]


def test_median_window_holds_the_lower_median():
    # Both median searches start from the window [floor(mu - sigma) - 1,
    # ceil(mu + sigma) + 1]: any median m minimises E|x - c|, so
    # |mu - m| <= E|x - m| <= E|x - mu| <= sigma (population sigma).
    rng = np.random.default_rng(11)
    for n in [1, 2, 3, 4, 7, 31, 32, 33, 100, 1250]:
        x = np.clip(np.rint(rng.normal(128, 16, size=(300, n))), 0, 255).astype(np.int64)
        x[:100] = rng.integers(0, 256, size=(100, n))                         # uniform rows
        x[100:150, : max(1, n // 3)] = 255                                    # a third of the row bright
        x[150:200] = np.where(rng.random((50, n)) < 0.5, 0, 255)               # two-valued rows
        m = lower_median(x)
        mu = x.mean(axis=1)
        sd = np.sqrt(((x - mu[:, None]) ** 2).mean(axis=1))
        assert np.all(np.abs(m - mu) <= sd + 1e-9), n
        assert np.all((np.floor(mu - sd) - 1 <= m) & (m <= np.ceil(mu + sd) + 1)), n


def test_counts_from_sums_of_absolute_differences():
    # f(p) = sum |x - p| over n bytes; for p <= 254, #(x <= p) = (n + f(p + 1) - f(p)) / 2,
    # so the lower median is min{p : f(p + 1) - f(p) >= 2 * need - n}, need = floor((n + 1) / 2).
    rng = np.random.default_rng(12)
    x = bins(rng, 500)
    for p in [0, 1, 100, 127, 128, 200, 254]:
        f = np.abs(x - p).sum(axis=1)
        f1 = np.abs(x - (p + 1)).sum(axis=1)
        assert np.array_equal((32 + f1 - f) // 2, (x <= p).sum(axis=1)), p
        assert np.all((32 + f1 - f) % 2 == 0), p
    need = (32 + 1) // 2
    med = np.array([min(p for p in range(256) if (row <= p).sum() >= need) for row in x])
    assert np.array_equal(med, lower_median(x))
