"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself.  The pins are:
  * hand-worked rows/columns (tests/golden, derivations in the files);
  * brute force against exact rational arithmetic (fractions.Fraction) of the
    definitions in Sec. IV -- a formulation with real mu and sigma^2, not the
    scaled-integer form the oracle evaluates;
  * closed-form tail fractions on clean noise;
  * invariants (idempotence, range, untouched unflagged samples) and special
    cases that reduce one method to another (FDSC with one bin == TDSC on the
    column; float32 == uint8 on integer-valued data with median replacement);
  * the qualitative results of Sec. V-A on the paper-shaped synthetic canvas.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from conftest import read_golden
from paper_2001_03389_gb300 import synth

# ---------------------------------------------------------------------------
# exact-rational restatements of Sec. IV (used only as pins)
# ---------------------------------------------------------------------------


def _frac_k2(k):
    return Fraction(k) ** 2  # k is a binary double; its square is an exact rational


M64 = (1 << 64) - 1


def py_mix64(z):
    """SplitMix64 output function (Steele, Lea, Flood 2014), restated from the
    published definition: add the golden-ratio increment, then two
    xor-shift-multiply rounds and a final xor-shift."""
    z = (z + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def py_draw(method, it, beam, line, index, attempt, n):
    """Position in [0, n) of a random-replacement attempt (the library's
    documented key: method 1 = TDSC, 2 = FDSC; it = the iteration)."""
    h = py_mix64(py_mix64(py_mix64(py_mix64(beam) ^ line) ^ index) ^ (method << 8 | it << 16 | attempt << 24))
    return ((h >> 32) * n) >> 32


def _random_pick(x, hit, method, it, beam, line, index, lo, n):
    """Value taken by flagged sample `index`: the first of 32 draws over
    positions lo .. lo + n - 1 that lands on an unflagged sample (unflagged
    values do not change within an iteration), else its own value."""
    for a in range(32):
        u = lo + py_draw(method, it, beam, line, index, a, n)
        if not hit[u]:
            return x[u]
    return x[index]


def _round_f32(q):
    """(float) of the double nearest to the rational q: the float32 replacement
    value is the float32 rounding of the double mean."""
    return Fraction(float(np.float32(float(q))))


def rational_tdsc(row, k, iterations, replace, beam=0, line=0, it0=0, f32=False):
    """TDSC on exact rationals: mu = mean, sigma^2 = population variance.
    Returns (values, flags, ties) where ties counts exact |x - mu| = k sigma
    decisions (decided by rounding in a floating-point evaluation)."""
    x = [Fraction(float(v)) if f32 else Fraction(int(v)) for v in row]
    n = len(x)
    flags = [0] * n
    ties = 0
    k2 = _frac_k2(k)
    for i in range(iterations):
        mu = sum(x) / n
        var = sum((v - mu) ** 2 for v in x) / n
        if replace == "mean":
            r = _round_f32(mu) if f32 else Fraction(math.floor(mu + Fraction(1, 2)))  # round half up
        else:
            r = sorted(x)[(n - 1) // 2]
        hit = [(v - mu) ** 2 > k2 * var for v in x]
        ties += sum(1 for v in x if var > 0 and (v - mu) ** 2 == k2 * var)
        new = list(x)
        for t, h in enumerate(hit):
            if h:
                new[t] = _random_pick(x, hit, 1, it0 + i, beam, line, t, 0, n) if replace == "random" else r
                flags[t] = 1
        x = new
    vals = [float(v) for v in x] if f32 else [int(v) for v in x]
    return vals, flags, ties


def rational_fdsc(col, k, iterations, replace, bin, beam=0, line=0, it0=0, f32=False):
    """FDSC on exact rationals: bin means, corrected values d, mu', sigma'.
    Returns (values, flags, ties) as rational_tdsc."""
    x = [Fraction(float(v)) if f32 else Fraction(int(v)) for v in col]
    n = len(x)
    flags = [0] * n
    ties = 0
    k2 = _frac_k2(k)
    bins = [list(range(s, min(s + bin, n))) for s in range(0, n, bin)]
    for i in range(iterations):
        m = {}
        rep = {}
        for b in bins:
            mb = sum(x[c] for c in b) / len(b)
            for c in b:
                m[c] = mb
            if replace == "mean":
                rep[b[0]] = _round_f32(mb) if f32 else Fraction(math.floor(mb + Fraction(1, 2)))
            else:
                rep[b[0]] = sorted(x[c] for c in b)[(len(b) - 1) // 2]
        d = [x[c] - m[c] for c in range(n)]
        mu = sum(d) / n
        var = sum((v - mu) ** 2 for v in d) / n
        hit = [(d[c] - mu) ** 2 > k2 * var for c in range(n)]
        ties += sum(1 for c in range(n) if var > 0 and (d[c] - mu) ** 2 == k2 * var)
        new = list(x)
        for b in bins:
            for c in b:
                if hit[c]:
                    if replace == "random":
                        new[c] = _random_pick(x, hit, 2, it0 + i, beam, line, c, b[0], len(b))
                    else:
                        new[c] = rep[b[0]]
                    flags[c] = 1
        x = new
    vals = [float(v) for v in x] if f32 else [int(v) for v in x]
    return vals, flags, ties


def rational_clean(x, tdsc=None, fdsc=None, order="blocked"):
    """A (B, C, T) block cleaned on exact rationals, per the order readings:
    blocked = every TDSC iteration on each row, then every FDSC iteration on
    each column; interleaved = round r runs TDSC iteration r on every row, then
    FDSC iteration r on every column (random draws keyed by r), the method with
    more iterations running alone in the last rounds.  Flags: bit 0 TDSC,
    bit 1 FDSC.  Returns (out, flags, ties)."""
    f32 = x.dtype == np.float32
    out = x.astype(np.float64 if f32 else np.int64).copy()
    flags = np.zeros(x.shape, np.uint8)
    B, C, T = x.shape
    it_t = tdsc["iterations"] if tdsc else 0
    it_f = fdsc["iterations"] if fdsc else 0
    if order == "blocked":
        passes = [("t", 0, it_t)] if it_t else []
        passes += [("f", 0, it_f)] if it_f else []
    else:
        passes = []
        for r in range(max(it_t, it_f)):
            if r < it_t:
                passes.append(("t", r, 1))
            if r < it_f:
                passes.append(("f", r, 1))
    ties = 0
    for kind, it0, n_it in passes:
        for b in range(B):
            if kind == "t":
                for c in range(C):
                    v, f, tz = rational_tdsc(out[b, c], tdsc["k"], n_it, tdsc["replace"], b, c, it0, f32)
                    out[b, c] = v
                    flags[b, c] |= np.array(f, np.uint8)
                    ties += tz
            else:
                for t in range(T):
                    v, f, tz = rational_fdsc(out[b, :, t], fdsc["k"], n_it, fdsc["replace"], fdsc["bin"], b, t, it0,
                                             f32)
                    out[b, :, t] = v
                    flags[b, :, t] |= np.array(f, np.uint8) << 1
                    ties += tz
    return out.astype(x.dtype), flags, ties


# ---------------------------------------------------------------------------
# hand-worked fixtures
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("case", read_golden("tdsc_u8_handworked.txt"), ids=lambda c: str(c["params"]))
def test_tdsc_u8_handworked(oracle, case):
    p = case["params"]
    row = np.array(case["in"], dtype=np.uint8)
    out, fl = oracle.tdsc_row(row, float(p["k"]), int(p["iterations"]), p["replace"])
    assert out.tolist() == [int(v) for v in case["out"]]
    assert fl.tolist() == [int(v) for v in case["flag"]]


@pytest.mark.parametrize("case", read_golden("fdsc_u8_handworked.txt"), ids=lambda c: str(c["params"]))
def test_fdsc_u8_handworked(oracle, case):
    p = case["params"]
    col = np.array(case["in"], dtype=np.uint8)
    out, fl = oracle.fdsc_col(col, float(p["k"]), int(p["iterations"]), p["replace"], int(p["bin"]))
    assert out.tolist() == [int(v) for v in case["out"]]
    assert (fl > 0).astype(int).tolist() == [int(v) for v in case["flag"]]


@pytest.mark.parametrize("case", read_golden("tdsc_f32_handworked.txt"), ids=lambda c: str(c["params"]))
def test_tdsc_f32_handworked(oracle, case):
    p = case["params"]
    row = np.array(case["in"], dtype=np.float32)
    out, fl = oracle.tdsc_row(row, float(p["k"]), int(p["iterations"]), p["replace"])
    assert out.tolist() == [float(v) for v in case["out"]]
    assert fl.tolist() == [int(v) for v in case["flag"]]


# ---------------------------------------------------------------------------
# brute force against exact rationals
# ---------------------------------------------------------------------------

KS = [0.75, 1.0, 1.5, 2.0, 2.5, 2.75, 3.0, 3.25]


def test_tdsc_u8_bruteforce_vs_rational(oracle):
    rng = np.random.default_rng(11)
    for trial in range(1500):
        n = int(rng.integers(1, 13))
        if trial % 2:
            row = rng.choice([0, 1, 2, 255], size=n).astype(np.uint8)
        else:
            row = rng.integers(0, 256, size=n).astype(np.uint8)
        k = float(rng.choice(KS))
        it = int(rng.integers(1, 4))
        rep = "mean" if trial % 3 else "median"
        out, fl = oracle.tdsc_row(row, k, it, rep)
        r_out, r_fl, _ = rational_tdsc(row, k, it, rep)
        assert out.tolist() == r_out, (row, k, it, rep)
        assert fl.tolist() == r_fl, (row, k, it, rep)


def test_fdsc_u8_bruteforce_vs_rational(oracle):
    rng = np.random.default_rng(12)
    for trial in range(800):
        n = int(rng.integers(1, 17))
        bin = int(rng.integers(1, n + 1))
        if trial % 2:
            col = rng.choice([0, 3, 128, 255], size=n).astype(np.uint8)
        else:
            col = rng.integers(0, 256, size=n).astype(np.uint8)
        k = float(rng.choice(KS))
        it = int(rng.integers(1, 4))
        rep = "mean" if trial % 3 else "median"
        out, fl = oracle.fdsc_col(col, k, it, rep, bin)
        r_out, r_fl, _ = rational_fdsc(col, k, it, rep, bin)
        assert out.tolist() == r_out, (col, k, it, rep, bin)
        assert (fl > 0).astype(int).tolist() == r_fl, (col, k, it, rep, bin)


def test_fdsc_u8_larger_columns_vs_rational(oracle):
    # ARTS-like column lengths with a short last bin, one iteration each.
    rng = np.random.default_rng(13)
    for n, bin in [(100, 32), (96, 32), (61, 7), (64, 64)]:
        col = np.clip(np.rint(rng.normal(128, 16, n)), 0, 255).astype(np.uint8)
        col[rng.integers(0, n, 3)] = 250
        for k in (2.0, 3.0):
            out, fl = oracle.fdsc_col(col, k, 2, "mean", bin)
            r_out, r_fl, _ = rational_fdsc(col, k, 2, "mean", bin)
            assert out.tolist() == r_out
            assert (fl > 0).astype(int).tolist() == r_fl


# ---------------------------------------------------------------------------
# closed-form tail fractions on clean noise (first iteration)
# ---------------------------------------------------------------------------


def _binom_band(p, n, z=5.0):
    s = math.sqrt(p * (1 - p) / n)
    return p - z * s, p + z * s


def _ncdf(z):
    return 0.5 * math.erfc(-z / math.sqrt(2))


@pytest.mark.parametrize("k", [2.5, 3.0, 4.0])
def test_tdsc_u8_gaussian_tail_fraction(oracle, k):
    # uint8 N(128, 16^2) rounded: the expected fraction sums the discretised pmf
    # over the integers outside mu +- k sigma of that pmf.
    rng = np.random.default_rng(21)
    n_rows, T = 24, 50000
    x = np.clip(np.rint(rng.normal(128, 16, (n_rows, T))), 0, 255).astype(np.uint8)
    _, fl = oracle.clean(x[None], "bct", tdsc=dict(k=k, iterations=1, replace="mean"))
    frac = fl.mean()
    # The cut sits between integers, so the expectation is taken per row at
    # that row's own sample mean and deviation (population form).
    v = np.arange(256)
    pmf = np.array([_ncdf((u + 0.5 - 128) / 16) - _ncdf((u - 0.5 - 128) / 16) for u in v])
    xs = x.astype(np.float64)
    mus, sds = xs.mean(axis=1), xs.std(axis=1)
    expect = np.mean([pmf[np.abs(v - m) > k * s].sum() for m, s in zip(mus, sds)])
    lo, hi = _binom_band(expect, fl.size)
    assert lo < frac < hi, (frac, expect)
    if k == 4.0:
        # the loose 4-sigma cut of Sec. V-A changes almost nothing on clean data
        assert frac < 2e-4


@pytest.mark.parametrize("k", [2.0, 2.5, 3.0])
def test_tdsc_f32_chi2_tail_fraction(oracle, k):
    # chi^2_2 scaled by any gain g: mu = sigma = 2 g; only the upper tail exists,
    # P(x > (1 + k) 2 g) = exp(-(1 + k)).
    rng = np.random.default_rng(22)
    n_rows, T = 16, 40000
    g = np.exp(rng.uniform(np.log(0.5), np.log(2.0), n_rows))[:, None]
    x = (rng.standard_exponential((n_rows, T)) * 2.0 * g).astype(np.float32)
    _, fl = oracle.clean(x[None], "bct", tdsc=dict(k=k, iterations=1, replace="mean"))
    expect = math.exp(-(1 + k))
    lo, hi = _binom_band(expect, fl.size)
    assert lo < fl.mean() < hi, (fl.mean(), expect)


def test_fdsc_u8_gaussian_tail_fraction(oracle):
    # One bin equal to the whole column: the corrected values are x - mean, so
    # the flagged fraction follows the same discretised-normal tail as TDSC.
    rng = np.random.default_rng(23)
    C, T = 4096, 300
    x = np.clip(np.rint(rng.normal(128, 16, (1, C, T))), 0, 255).astype(np.uint8)
    _, fl = oracle.clean(x, "bct", fdsc=dict(k=3.0, iterations=1, replace="mean", bin=C))
    v = np.arange(256)
    pmf = np.array([_ncdf((u + 0.5 - 128) / 16) - _ncdf((u - 0.5 - 128) / 16) for u in v])
    xs = x[0].astype(np.float64)
    mus, sds = xs.mean(axis=0), xs.std(axis=0)  # per column (time sample)
    expect = np.mean([pmf[np.abs(v - m) > 3.0 * s].sum() for m, s in zip(mus, sds)])
    lo, hi = _binom_band(expect, fl.size)
    assert lo < (fl > 0).mean() < hi, ((fl > 0).mean(), expect)


# ---------------------------------------------------------------------------
# invariants and reductions
# ---------------------------------------------------------------------------


def test_tdsc_invariants(oracle):
    rng = np.random.default_rng(31)
    x = np.clip(np.rint(rng.normal(128, 16, (2, 40, 3000))), 0, 255).astype(np.uint8)
    x[:, :, rng.integers(0, 3000, 30)] = 250
    for rep in ("mean", "median"):
        out, fl = oracle.clean(x, "bct", tdsc=dict(k=3.0, iterations=3, replace=rep))
        # unflagged samples are byte-identical; changed samples are flagged
        assert np.array_equal(out[fl == 0], x[fl == 0])
        assert np.all(fl[out != x] == 1)
        # the output stays inside each row's input range
        assert np.all(out.min(axis=2) >= x.min(axis=2)) and np.all(out.max(axis=2) <= x.max(axis=2))
        # run to convergence, then one more iteration flags nothing
        conv, _ = oracle.clean(x, "bct", tdsc=dict(k=3.0, iterations=16, replace=rep))
        again, fl2 = oracle.clean(conv, "bct", tdsc=dict(k=3.0, iterations=16, replace=rep))
        if rep == "median":
            # the lower median is unchanged by replacing values with it, so the
            # median cut converges; the mean cut may keep moving by rounding
            rows_done = np.array([[not np.any(oracle.tdsc_row(conv[b, c], 3.0, 1, rep)[1]) for c in range(40)] for b in range(2)])
            assert rows_done.mean() > 0.9
        assert np.array_equal(again[fl2 == 0], conv[fl2 == 0])


def test_fdsc_single_bin_equals_tdsc_on_column(oracle):
    # bin == C: the corrected value is x - column mean and mu' = 0, so FDSC on a
    # column is TDSC on that column read as a row (same rounding of the mean).
    rng = np.random.default_rng(32)
    for dtype in (np.uint8, np.float32):
        for rep in ("mean", "median"):
            C = 97
            if dtype == np.uint8:
                col = np.clip(np.rint(rng.normal(128, 16, C)), 0, 255).astype(np.uint8)
            else:
                col = (rng.standard_exponential(C) * 3.0).astype(np.float32)
            col[[5, 50]] = col.max() * 2 if dtype == np.float32 else 255
            a, fa = oracle.fdsc_col(col, 2.5, 3, rep, C)
            b, fb = oracle.tdsc_row(col, 2.5, 3, rep)
            assert np.array_equal(a, b)
            assert np.array_equal(fa > 0, fb > 0)


def test_fdsc_flagged_value_is_bin_statistic(oracle):
    # Fig. 3: an outlier's original value is replaced by its bin's mean (median).
    rng = np.random.default_rng(33)
    C, bin = 64, 16
    col = np.clip(np.rint(rng.normal(100, 5, C)), 0, 255).astype(np.uint8)
    col[[3, 40]] = [250, 0]
    for rep in ("mean", "median"):
        out, fl = oracle.fdsc_col(col, 3.0, 1, rep, bin)
        for c in np.nonzero(fl)[0]:
            b = col[(c // bin) * bin:(c // bin + 1) * bin].astype(np.int64)
            want = (2 * b.sum() + len(b)) // (2 * len(b)) if rep == "mean" else np.sort(b)[(len(b) - 1) // 2]
            assert out[c] == want


def test_f32_matches_u8_on_integer_data(oracle):
    # Independent arithmetic: exact integers (uint8) vs two-pass IEEE double
    # (float32) reach the same decisions on integer-valued data; with median
    # replacement the outputs coincide.  Exact ties of |x-mu| = k sigma are
    # excluded by construction (they would be decided by rounding).
    rng = np.random.default_rng(34)
    x = np.clip(np.rint(rng.normal(128, 16, (2, 48, 1000))), 0, 255).astype(np.uint8)
    x[:, :, rng.integers(0, 1000, 10)] = 240
    x[:, 7, :] = np.clip(x[:, 7, :].astype(int) + 60, 0, 255)
    td = dict(k=2.75, iterations=2, replace="median")
    fd = dict(k=2.75, iterations=2, replace="median", bin=16)
    ou, fu = oracle.clean(x, "bct", tdsc=td, fdsc=fd)
    of, ff = oracle.clean(x.astype(np.float32), "bct", tdsc=td, fdsc=fd)
    assert np.array_equal(ou.astype(np.float32), of)
    assert np.array_equal(fu, ff)


def test_layouts_agree(oracle):
    rng = np.random.default_rng(35)
    x = np.clip(np.rint(rng.normal(128, 16, (2, 40, 300))), 0, 255).astype(np.uint8)
    x[:, 3, :] = 200
    td = dict(k=3.0, iterations=2, replace="median")
    fd = dict(k=3.0, iterations=2, replace="mean", bin=8)
    a, fa = oracle.clean(x, "bct", tdsc=td, fdsc=fd)
    b, fb = oracle.clean(np.ascontiguousarray(x.transpose(0, 2, 1)), "btc", tdsc=td, fdsc=fd)
    assert np.array_equal(a, b.transpose(0, 2, 1))
    assert np.array_equal(fa, fb.transpose(0, 2, 1))


def test_combined_is_tdsc_then_fdsc(oracle):
    rng = np.random.default_rng(36)
    x = np.clip(np.rint(rng.normal(128, 16, (1, 64, 700))), 0, 255).astype(np.uint8)
    td = dict(k=3.0, iterations=2, replace="median")
    fd = dict(k=3.0, iterations=2, replace="median", bin=32)
    both, fb = oracle.clean(x, "bct", tdsc=td, fdsc=fd)
    t, ft = oracle.clean(x, "bct", tdsc=td)
    f, ff = oracle.clean(t, "bct", fdsc=fd)
    assert np.array_equal(both, f)
    assert np.array_equal(fb, ft | ff)
    assert set(np.unique(ft)) <= {0, 1} and set(np.unique(ff)) <= {0, 2}


def test_in_place(oracle):
    rng = np.random.default_rng(37)
    x = np.clip(np.rint(rng.normal(128, 16, (1, 16, 200))), 0, 255).astype(np.uint8)
    out, fl = oracle.clean(x, "bct", tdsc=dict(k=2.0, iterations=2, replace="mean"))
    assert fl.any()


# ---------------------------------------------------------------------------
# medians
# ---------------------------------------------------------------------------


def test_lower_median_rank_property(oracle):
    rng = np.random.default_rng(41)
    for n in list(range(1, 20)) + [255, 256, 1000, 12500]:
        for dtype in (np.uint8, np.float32):
            v = rng.integers(0, 256, n).astype(dtype) if dtype == np.uint8 else rng.normal(0, 1, n).astype(np.float32)
            m = oracle.lower_median(v)
            r = (n - 1) // 2
            assert np.sum(v < m) <= r < np.sum(v <= m)
            assert m in v


def test_lower_median_signed_zero(oracle):
    v = np.array([0.0, -0.0, 1.0, -0.0], dtype=np.float32)  # sorted: -0 -0 0 1, rank 1 -> -0
    assert math.copysign(1.0, oracle.lower_median(v)) == -1.0
    v = np.array([0.0, -0.0, 0.0], dtype=np.float32)        # sorted: -0 0 0, rank 1 -> +0
    assert math.copysign(1.0, oracle.lower_median(v)) == 1.0


def test_median_invariant_under_replacement(oracle):
    # Replacing any subset of values by the lower median keeps the lower median.
    rng = np.random.default_rng(42)
    for _ in range(300):
        n = int(rng.integers(1, 40))
        v = rng.integers(0, 256, n).astype(np.uint8)
        m = oracle.lower_median(v)
        w = v.copy()
        w[rng.random(n) < 0.3] = m
        assert oracle.lower_median(w) == m


# ---------------------------------------------------------------------------
# argument validation
# ---------------------------------------------------------------------------


def test_validation(oracle):
    x = np.zeros((1, 4, 8), np.uint8)
    for bad in (dict(k=0.0), dict(k=float("nan")), dict(k=3.0, iterations=0), dict(k=3.0, iterations=17)):
        with pytest.raises(oracle.OracleError):
            oracle.clean(x, "bct", tdsc=bad)
    with pytest.raises(oracle.OracleError):
        oracle.clean(x, "bct", fdsc=dict(k=3.0, bin=5))
    # exactness range: (255 T)^2 must stay below 2^53
    big = np.zeros((1, 1, 372200), np.uint8)
    with pytest.raises(oracle.OracleError) as e:
        oracle.clean(big, "bct", tdsc=dict(k=3.0))
    assert e.value.rc == 2


# ---------------------------------------------------------------------------
# the qualitative results of Sec. V-A on the paper-shaped 1 x 64 x 2048 canvas
# ---------------------------------------------------------------------------


def _small_canvas_truth():
    """Recreate the small canvas's RFI positions from the generator's own draws."""
    spec = synth.WORKLOADS[synth.SMALL]
    m = spec["model"]()
    rng = synth._beam_rng(synth.seed_of(synth.SMALL), 0)
    rng.standard_normal((spec["C"], spec["T"]), dtype=np.float32)
    chans = rng.choice(spec["C"], size=m.nb_count, replace=False)
    starts = rng.choice(spec["T"] - m.bb_width + 1, size=m.bb_count, replace=False)
    t0 = int(rng.integers(0, spec["T"] // 2))
    delays = synth._dispersion_delays(spec["C"], m.disp_span)
    return chans, starts, t0 + delays


def test_paper_accuracy_claims_small_canvas(oracle):
    x = synth.make_beams(synth.SMALL)
    C, T = x.shape[1:]
    chans, starts, pulse_t = _small_canvas_truth()
    bb = np.zeros(T, bool)
    for s in starts:
        bb[s:s + 4] = True
    td = dict(k=3.0, iterations=1, replace="mean")
    # FDSC at the paper's 2.75 sigma with bin 32 (Fig. 5), three iterations (Sec. V-A)
    fd = dict(k=2.75, iterations=3, replace="mean", bin=32)
    _, ft = oracle.clean(x, "bct", tdsc=td)
    _, ff = oracle.clean(x, "bct", fdsc=fd)
    ft = ft[0] > 0
    ff = ff[0] > 0
    quiet = np.setdiff1d(np.arange(C), chans)
    # TDSC removes the bright broadband impulses (+90 = 5.6 sigma) ...
    assert ft[np.ix_(quiet, np.nonzero(bb)[0])].mean() > 0.97
    # ... but not the persistent narrowband channels (their own mean absorbs them)
    assert ft[chans][:, ~bb].mean() < 0.05
    # FDSC removes most of the narrowband samples (+60 = 3.75 sigma, far fainter
    # than the paper's SNR-125 pulses) while touching almost no clean channel
    assert ff[chans][:, ~bb].mean() > 0.7
    assert ff[quiet][:, ~bb].mean() < 0.01
    # the faint dispersed pulse (+20 = 1.25 sigma) survives both methods almost untouched
    ok = pulse_t < T
    cs = np.arange(C)[ok]
    ps = pulse_t[ok]
    on_bb = bb[ps]
    assert ft[cs[~on_bb], ps[~on_bb]].mean() < 0.2
    assert ff[cs[~on_bb], ps[~on_bb]].mean() < 0.2


def test_f32_margin_diagnostic(oracle):
    # Row [0, 0, 0, 4], k = 1, one iteration: mu = 1, sigma = sqrt(3) (population).
    # |x - mu| is 1 for the zeros and 3 for the 4, so the relative distances from
    # k sigma are |1 - sqrt 3| / sqrt 3 and |3 - sqrt 3| / sqrt 3; the 4 is flagged.
    import math

    x = np.array([[[0, 0, 0, 4]]], np.float32)
    out, fl, mg = oracle.clean_f32_margin(x, "bct", tdsc=dict(k=1.0, iterations=1))
    s3 = math.sqrt(3.0)
    assert np.allclose(mg[0, 0], [abs(1 - s3) / s3] * 3 + [abs(3 - s3) / s3], rtol=1e-12)
    assert fl[0, 0].tolist() == [0, 0, 0, 1]
    want, wf = oracle.clean(x, "bct", tdsc=dict(k=1.0, iterations=1))
    assert np.array_equal(out, want) and np.array_equal(fl, wf)
    # a constant column: sigma = 0, no decision has a finite margin
    y = np.full((1, 4, 3), 2.5, np.float32)
    _, fl2, mg2 = oracle.clean_f32_margin(y, "bct", fdsc=dict(k=2.0, iterations=2, bin=2))
    assert np.all(np.isinf(mg2)) and not fl2.any()


def test_interleaved_order(oracle):
    # Interleaved order (one TDSC iteration, then one FDSC iteration, per round)
    # equals blocked order when each method runs once, equals the explicit
    # sequence of single-iteration calls, and differs from blocked order on
    # data where an FDSC replacement changes a later TDSC decision.
    rng = np.random.default_rng(8)
    td1 = dict(k=2.0, iterations=1, replace="mean")
    fd1 = dict(k=2.0, iterations=1, replace="mean", bin=4)
    x = noise_u8_local(rng, (2, 12, 40))
    a = oracle.clean(x, "bct", tdsc=td1, fdsc=fd1)
    b = oracle.clean(x, "bct", tdsc=td1, fdsc=fd1, order="interleaved")
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    td2, fd2 = dict(td1, iterations=2), dict(fd1, iterations=2)
    y = x.copy()
    fl = np.zeros_like(x)
    for _ in range(2):
        y, f = oracle.clean(y, "bct", tdsc=td1, fdsc=fd1)
        fl |= f
    got, gf = oracle.clean(x, "bct", tdsc=td2, fdsc=fd2, order="interleaved")
    assert np.array_equal(got, y) and np.array_equal(gf, fl)
    differs = False
    for s in range(20):
        z = noise_u8_local(np.random.default_rng(100 + s), (1, 8, 24))
        if not np.array_equal(oracle.clean(z, "bct", tdsc=td2, fdsc=fd2)[0],
                              oracle.clean(z, "bct", tdsc=td2, fdsc=fd2, order="interleaved")[0]):
            differs = True
            break
    assert differs
    with pytest.raises(ValueError):
        oracle.clean(x, "bct", tdsc=td1, order="sideways")


def noise_u8_local(rng, shape):
    x = np.clip(np.rint(rng.normal(128, 16, shape)), 0, 255).astype(np.uint8)
    flat = x.reshape(-1)
    flat[rng.integers(0, flat.size, max(1, flat.size // 30))] = 250
    return x


def test_random_replacement_generator(oracle):
    # SplitMix64 (Steele, Lea, Flood 2014) seeded with 0: its first two outputs
    assert oracle.mix64(0) == 0xE220A8397B1DCDAF
    assert oracle.mix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4
    # draws fall in [0, n) and spread over it
    seen = {oracle.draw(1, 0, 3, 7, i, 0, 10) for i in range(400)}
    assert seen == set(range(10))


def test_random_replacement_takes_unflagged_values(oracle):
    # one iteration: a flagged sample takes the value of an unflagged sample of
    # the same row (TDSC) or bin (FDSC) -- the first draw that hits one
    rng = np.random.default_rng(12)
    x = noise_u8_local(rng, (2, 16, 300))
    td = dict(k=1.5, iterations=1, replace="random")
    out, fl = oracle.clean(x, "bct", tdsc=td)
    for b in range(2):
        for c in range(16):
            row, o, f = x[b, c], out[b, c], fl[b, c] > 0
            assert f.any() and (~f).any()
            assert np.array_equal(o[~f], row[~f])
            for t in np.flatnonzero(f):
                for a in range(32):
                    u = oracle.draw(1, 0, b, c, t, a, row.size)
                    if not f[u]:
                        assert o[t] == row[u]
                        break
                else:
                    assert o[t] == row[t]
    fd = dict(k=1.5, iterations=1, replace="random", bin=8)
    out, fl = oracle.clean(x, "bct", fdsc=fd)
    for b in range(2):
        for t in range(0, 300, 37):
            col, o, f = x[b, :, t], out[b, :, t], fl[b, :, t] > 0
            assert np.array_equal(o[~f], col[~f])
            for c in np.flatnonzero(f):
                g0 = (c // 8) * 8
                for a in range(32):
                    u = g0 + oracle.draw(2, 0, b, t, c, a, 8)
                    if not f[u]:
                        assert o[c] == col[u]
                        break
                else:
                    assert o[c] == col[c]


def test_random_replacement_statistics_and_edge_cases(oracle):
    # the replaced values average to the mean of the kept samples
    rng = np.random.default_rng(4)
    x = np.clip(np.rint(rng.normal(100, 10, (1, 4, 20000))), 0, 255).astype(np.uint8)
    x[0, :, ::50] = 250
    out, fl = oracle.clean(x, "bct", tdsc=dict(k=3.0, iterations=1, replace="random"))
    f = fl[0] > 0
    assert abs(out[0][f].astype(float).mean() - x[0][~f].astype(float).mean()) < 1.0
    # everything flagged (|x - mu| = sigma > k sigma for k < 1): nothing to draw, values stay
    z = np.tile(np.array([0, 255], np.uint8), (1, 2, 50))
    out, fl = oracle.clean(z, "bct", tdsc=dict(k=0.5, iterations=2, replace="random"))
    assert np.array_equal(out, z) and (fl == 1).all()
    # float32 follows the same rule
    y = z.astype(np.float32)
    out32, fl32 = oracle.clean(y, "bct", tdsc=dict(k=0.5, iterations=1, replace="random"))
    assert np.array_equal(out32, y) and (fl32 == 1).all()
    xf = x.astype(np.float32)
    o8, f8 = oracle.clean(x, "bct", tdsc=dict(k=3.0, iterations=2, replace="random"),
                          fdsc=dict(k=3.0, iterations=2, replace="random", bin=2))
    o32, f32 = oracle.clean(xf, "bct", tdsc=dict(k=3.0, iterations=2, replace="random"),
                            fdsc=dict(k=3.0, iterations=2, replace="random", bin=2))
    assert np.array_equal(f8, f32) and np.array_equal(o8.astype(np.float32), o32)


# ---------------------------------------------------------------------------
# float32 FDSC over several bins, random draws keyed by the iteration, and the
# interleaved order, each against the exact-rational restatements above
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("case", read_golden("fdsc_f32_handworked.txt"), ids=lambda c: str(c["params"]))
def test_fdsc_f32_handworked(oracle, case):
    p = case["params"]
    col = np.array(case["in"], dtype=np.float32)
    out, fl = oracle.fdsc_col(col, float(p["k"]), int(p["iterations"]), p["replace"], int(p["bin"]))
    assert out.tolist() == [float(v) for v in case["out"]]
    assert (fl > 0).astype(int).tolist() == [int(v) for v in case["flag"]]


def test_py_draw_restates_splitmix64(oracle):
    # the test's own SplitMix64 gives the published first outputs of seed 0,
    # and the oracle's draws equal the test's draws
    assert py_mix64(0) == 0xE220A8397B1DCDAF
    assert py_mix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4
    rng = np.random.default_rng(5)
    for _ in range(300):
        m, it, b, line, idx, a = (int(rng.integers(1, 3)), int(rng.integers(0, 16)), int(rng.integers(0, 200)),
                                  int(rng.integers(0, 30000)), int(rng.integers(0, 30000)), int(rng.integers(0, 32)))
        n = int(rng.integers(1, 5000))
        assert oracle.draw(m, it, b, line, idx, a, n) == py_draw(m, it, b, line, idx, a, n)


def _dyadic_f32(rng, n):
    # small integers over small powers of two: sums and means of up to 16
    # values stay exact in double, so only exact ties are decided by rounding
    return (rng.integers(0, 40, n) / rng.choice([1, 2, 4, 8], n)).astype(np.float32)


@pytest.mark.parametrize("replace", ["mean", "median", "random"])
def test_fdsc_f32_bruteforce_vs_rational(oracle, replace):
    # several bins, a partial last bin, 1-3 iterations (Sec. IV FDSC, Fig. 3)
    rng = np.random.default_rng(61)
    run = 0
    for trial in range(400):
        n = int(rng.integers(2, 17))
        bin = int(rng.integers(1, n + 1))
        col = _dyadic_f32(rng, n)
        col[rng.integers(0, n)] = float(rng.choice([60.0, 100.5, 0.0]))
        k = float(rng.choice([0.75, 1.0, 1.5, 2.0, 2.5]))
        it = int(rng.integers(1, 4))
        r_out, r_fl, ties = rational_fdsc(col, k, it, replace, bin, f32=True)
        if ties:
            continue  # an exact tie: the double evaluation may go either way
        run += 1
        x = col[None, :, None]
        out, fl = oracle.clean(x, "bct", fdsc=dict(k=k, iterations=it, replace=replace, bin=bin))
        assert out[0, :, 0].tolist() == r_out, (col, k, it, bin)
        assert (fl[0, :, 0] > 0).astype(int).tolist() == r_fl, (col, k, it, bin)
    assert run > 300


@pytest.mark.parametrize("replace", ["mean", "median", "random"])
def test_tdsc_f32_bruteforce_vs_rational(oracle, replace):
    rng = np.random.default_rng(62)
    run = 0
    for trial in range(400):
        n = int(rng.integers(2, 17))
        row = _dyadic_f32(rng, n)
        row[rng.integers(0, n)] = float(rng.choice([60.0, 100.5, 0.0]))
        k = float(rng.choice([0.75, 1.0, 1.5, 2.0, 2.5]))
        it = int(rng.integers(1, 4))
        r_out, r_fl, ties = rational_tdsc(row, k, it, replace, f32=True)
        if ties:
            continue
        run += 1
        out, fl = oracle.clean(row[None, None, :], "bct", tdsc=dict(k=k, iterations=it, replace=replace))
        assert out[0, 0].tolist() == r_out, (row, k, it)
        assert fl[0, 0].astype(int).tolist() == r_fl, (row, k, it)
    assert run > 300


def test_random_u8_bruteforce_vs_rational(oracle):
    # random replacement over several iterations: iteration i draws with it = i
    rng = np.random.default_rng(63)
    for trial in range(300):
        B, C, T = 2, int(rng.integers(2, 9)), int(rng.integers(2, 13))
        x = rng.integers(0, 256, (B, C, T)).astype(np.uint8)
        x[rng.random(x.shape) < 0.1] = 250
        k = float(rng.choice([0.75, 1.0, 1.5, 2.0]))
        td = dict(k=k, iterations=int(rng.integers(1, 4)), replace="random")
        fd = dict(k=k, iterations=int(rng.integers(1, 4)), replace="random", bin=int(rng.integers(1, C + 1)))
        want, wf, _ = rational_clean(x, td, fd)
        got, gf = oracle.clean(x, "bct", tdsc=td, fdsc=fd)
        assert np.array_equal(got, want) and np.array_equal(gf, wf), (x, td, fd)


@pytest.mark.parametrize("replace", ["mean", "median", "random"])
def test_interleaved_vs_rational(oracle, replace):
    # Interleaved order with equal and unequal iteration counts: round r is
    # iteration r of each method (random draws keyed by r); the method with
    # more iterations runs alone in the last rounds.
    rng = np.random.default_rng(64)
    for trial in range(150):
        B, C, T = int(rng.integers(1, 3)), int(rng.integers(2, 7)), int(rng.integers(2, 9))
        x = rng.integers(0, 256, (B, C, T)).astype(np.uint8)
        x[rng.random(x.shape) < 0.1] = 250
        k = float(rng.choice([0.75, 1.0, 1.5, 2.0]))
        td = dict(k=k, iterations=int(rng.integers(1, 4)), replace=replace)
        fd = dict(k=k, iterations=int(rng.integers(1, 4)), replace=replace, bin=int(rng.integers(1, C + 1)))
        want, wf, _ = rational_clean(x, td, fd, order="interleaved")
        got, gf = oracle.clean(x, "bct", tdsc=td, fdsc=fd, order="interleaved")
        assert np.array_equal(got, want) and np.array_equal(gf, wf), (x, td, fd)


def test_interleaved_f32_vs_rational(oracle):
    rng = np.random.default_rng(65)
    run = 0
    for trial in range(120):
        C, T = int(rng.integers(2, 6)), int(rng.integers(2, 8))
        x = _dyadic_f32(rng, C * T).reshape(1, C, T)
        k = float(rng.choice([0.75, 1.0, 1.5]))
        rep = ["mean", "median", "random"][trial % 3]
        td = dict(k=k, iterations=int(rng.integers(1, 4)), replace=rep)
        fd = dict(k=k, iterations=int(rng.integers(1, 4)), replace=rep, bin=int(rng.integers(1, C + 1)))
        want, wf, ties = rational_clean(x, td, fd, order="interleaved")
        if ties:
            continue
        run += 1
        got, gf = oracle.clean(x, "bct", tdsc=td, fdsc=fd, order="interleaved")
        assert np.array_equal(got, want) and np.array_equal(gf, wf), (x, td, fd)
    assert run > 60


@pytest.mark.parametrize("case", read_golden("interleaved_u8_handworked.txt"), ids=lambda c: str(c["params"]))
def test_interleaved_handworked(oracle, case):
    p = case["params"]
    C, T = int(p["C"]), int(p["T"])
    x = np.array(case["in"], dtype=np.uint8).reshape(1, C, T)
    td = dict(k=float(p["tdsc_k"]), iterations=int(p["tdsc_it"]), replace="mean")
    fd = dict(k=float(p["fdsc_k"]), iterations=int(p["fdsc_it"]), replace="mean", bin=int(p["bin"]))
    out, fl = oracle.clean(x, "bct", tdsc=td, fdsc=fd, order="interleaved")
    assert out.reshape(-1).tolist() == [int(v) for v in case["out"]]
    assert fl.reshape(-1).tolist() == [int(v) for v in case["flag"]]
    # the blocked order differs on this block (TDSC's second iteration runs before FDSC)
    _, fb = oracle.clean(x, "bct", tdsc=td, fdsc=fd)
    assert fb.reshape(-1).tolist() != [int(v) for v in case["flag"]]
