"""Oracle pins for the gather of Algorithm 1 and its mean padding.

Algorithm 1 builds the demodulated series as S'_j = S[idx_j]; where idx_j falls
outside the observed series the paper pads with the series mean (Sec. 2.8, mean
padding).  These checks fail for the plausible slips in that step: filling 0
instead of the mean, an off-by-one range test (idx <= n, idx > 0), a fill taken
from the first or last sample, or a mean that is not the FP64 mean of all samples.
"""
import math

import numpy as np


def test_series_mean_is_the_exact_mean(orc):
    rng = np.random.default_rng(17)
    for n in [1, 2, 3, 1000, 65537]:
        x = (rng.standard_normal(n) * 3.0 + 7.25).astype(np.float32)
        exact = math.fsum(float(v) for v in x) / n
        got = orc.series_mean(x)
        # sequential FP64 summation of n float32 values: error <= n eps sum|x|
        assert abs(got - exact) <= n * 2.3e-16 * float(np.sum(np.abs(x), dtype=np.float64)) / n + 1e-300
    assert orc.series_mean(np.array([5.0], np.float32)) == 5.0
    assert orc.series_mean(np.array([1.0, 2.0, 4.0, 8.0], np.float32)) == 3.75


def test_resample_in_range_and_mean_padding(orc):
    n = 257
    x = (np.arange(n, dtype=np.float32) * np.float32(0.5) - np.float32(20.0))
    fill = orc.series_mean(x)
    assert fill == float(np.mean(x.astype(np.float64)))
    edges = [-(1 << 40), -1000, -2, -1, 0, 1, n - 2, n - 1, n, n + 1, n + 1000, 1 << 40]
    rest = list(np.random.default_rng(3).integers(-n, 2 * n, n - len(edges)))
    idx = np.array(edges + rest, np.int64)
    out = orc.resample(x, idx, fill)
    for j, i in enumerate(idx):
        if 0 <= i < n:
            assert out[j] == float(x[i]), (j, i)
        else:
            assert out[j] == fill, (j, i)
    # the two range ends exactly: x[0] and x[n-1] are kept, -1 and n are padded
    assert out[edges.index(0)] == float(x[0]) and out[edges.index(n - 1)] == float(x[n - 1])
    assert out[edges.index(-1)] == fill and out[edges.index(n)] == fill
    assert fill not in (float(x[0]), float(x[n - 1]), 0.0)


def test_search_pads_with_the_series_mean(orc):
    """End to end: an orbit whose map leaves the series at the end gives the spectrum
    of the mean-padded series (and not of a zero- or edge-padded one)."""
    n, ts = 1 << 14, 64e-6
    x = (np.random.default_rng(8).standard_normal(n) + 4.0).astype(np.float32)
    tmpl = (0.9, 0.004, 3.0, 0.0, 0.0)  # tau/t_s = 62.5 samples, period 0.9 s
    idx, _, _ = orc.index_map(tmpl, n, ts)
    outside = (idx < 0) | (idx >= n)
    assert outside.sum() > 10
    mean = orc.series_mean(x)
    r = orc.search_template(x, ts, tmpl, whiten_block=256, want_arrays=True)
    r_mean = orc.search_template(x, ts, tmpl, whiten_block=256, want_arrays=True, fill=mean)
    assert np.array_equal(r["Pw"], r_mean["Pw"])
    # the same spectrum rebuilt from the primitives with explicit mean padding
    xr = np.where(outside, mean, x[np.clip(idx, 0, n - 1)].astype(np.float64))
    Pw_ref, _ = orc.whiten(orc.power_spectrum(xr), 256)
    assert np.array_equal(r["Pw"], Pw_ref)
    # zero padding or edge padding would change it
    for other in (0.0, float(x[-1])):
        r_o = orc.search_template(x, ts, tmpl, whiten_block=256, want_arrays=True, fill=other)
        assert np.max(np.abs(r_o["Pw"] - r["Pw"])) > 1e-3
