"""Incoherent dedispersion and time-series S/N for the accuracy checks of
Sec. V-A (test harness only: the detection side, not the cleaning)."""
import numpy as np


def dedisperse(x, dm):
    """Sum of the channels of a (C, T) block shifted by their Eq. 2 delays."""
    from paper_2001_03389_gb300 import synth

    C, T = x.shape
    d = synth.dm_delays(C, dm)
    L = T - int(d.max())
    s = np.zeros(L, np.float64)
    for c in range(C):
        s += x[c, d[c]:d[c] + L]
    return s


def snr_at(series, t):
    """S/N of the sample at t: (s[t] - mean) / std over the whole series."""
    return float((series[t] - series.mean()) / series.std())
