"""Oracle pins: radix-2 FFT, power spectrum, de-reddening, harmonic sums and
thresholds.

Pins:
  * the FFT equals the brute-force DFT X_k = sum_j x_j e^{-2 pi i jk/N}
    (N <= 1024, relative 1e-12), Parseval, a pure tone gives one spike, and
    numpy's pocketfft agrees at N = 2^16 (an independent library);
  * whitened noise is Exp(1): in every block exactly floor((W-1)/2) bins lie
    below ln 2 (lower median), the result is invariant to scaling the series,
    and the tail follows e^{-x} (Sec. 2.1: chi^2 with 2 dof);
  * harmonic sums collect a comb of n harmonics into n at the n-th harmonic
    bin, S_1 = Pw, and whitened noise follows the Gamma(n, 1) tail (chi^2 with
    2^{L+1} dof, Sec. 2.1) checked with scipy;
  * thresholds: n = 1 is -ln p exactly; Q(n, thr) = p against scipy; P_min
    and S/N_min closed forms (Sec. 2.1).
"""
import math

import numpy as np
import pytest
import scipy.special as sp
import scipy.stats as st


def test_fft_bruteforce(orc):
    rng = np.random.default_rng(5)
    for n in [1, 2, 4, 8, 64, 1024]:
        z = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        j = np.arange(n)
        D = np.exp(-2j * np.pi * np.outer(j, j) / n)
        ref = D @ z
        got = orc.fft(z)
        assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_fft_parseval_and_tone(orc):
    rng = np.random.default_rng(6)
    n = 1 << 14
    z = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    X = orc.fft(z)
    assert abs(np.sum(np.abs(z) ** 2) - np.sum(np.abs(X) ** 2) / n) <= 1e-12 * np.sum(np.abs(z) ** 2)
    k0 = 777
    tone = np.exp(2j * np.pi * k0 * np.arange(n) / n)
    T = orc.fft(tone)
    assert abs(T[k0] - n) < 1e-8
    T[k0] = 0
    assert np.max(np.abs(T)) < 1e-8


def test_fft_vs_numpy_large(orc):
    rng = np.random.default_rng(7)
    n = 1 << 16
    z = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    a = orc.fft(z)
    b = np.fft.fft(z)
    assert np.max(np.abs(a - b)) <= 1e-11 * np.max(np.abs(b))


def test_power_spectrum_real_input(orc):
    rng = np.random.default_rng(8)
    x = rng.standard_normal(4096)
    P = orc.power_spectrum(x)
    assert P.size == 2048 and P[0] == 0.0
    ref = np.abs(np.fft.fft(x)[:2048]) ** 2
    ref[0] = 0
    assert np.max(np.abs(P - ref)) <= 1e-10 * ref.max()


def test_whiten_lower_median_and_scale(orc):
    rng = np.random.default_rng(9)
    x = rng.standard_normal(1 << 16)
    P = orc.power_spectrum(x)
    W = 1024
    Pw, med = orc.whiten(P, W)
    for b in range(P.size // W):
        blk = Pw[b * W:(b + 1) * W]
        assert np.sum(blk < math.log(2)) == (W - 1) // 2
        assert np.isclose(np.sort(P[b * W:(b + 1) * W])[(W - 1) // 2], med[b], rtol=0, atol=0)
    Pw2, _ = orc.whiten(orc.power_spectrum(3.7 * x), W)
    assert np.max(np.abs(Pw2 - Pw)) <= 1e-12 * Pw.max()


def test_whiten_zero_block(orc):
    Pw, med = orc.whiten(np.zeros(2048), 1024)
    assert np.all(Pw == 0) and np.all(med == 0)


def test_whitened_noise_is_exp1(orc):
    rng = np.random.default_rng(10)
    x = rng.standard_normal(1 << 20).astype(np.float32)
    Pw, _ = orc.whiten(orc.power_spectrum(x.astype(np.float64)), 1024)
    v = Pw[1:]
    assert abs(v.mean() - 1.0) < 0.01
    for thr in [1.0, 3.0, 6.0]:
        frac = np.mean(v > thr)
        expect = math.exp(-thr)
        assert abs(frac - expect) < 5 * math.sqrt(expect / v.size) + 2e-3 * expect


def test_harmonic_sum_comb(orc):
    nb, base = 1 << 14, 300
    Pw = np.zeros(nb)
    Pw[base * np.arange(1, 17)] = 1.0
    S = orc.harmonic_sums(Pw, 5)
    assert np.array_equal(S[0], Pw)
    for L in range(5):
        n = 1 << L
        assert S[L, n * base] == n
        assert S[L, 0] == 0.0
        assert S[L].max() == n


def test_harmonic_sum_rounding_rule(orc):
    """Harmonic h of top-harmonic bin k maps to round-half-up(k h / n)."""
    nb = 64
    for L, n in enumerate([1, 2, 4, 8, 16]):
        for h in range(1, n + 1):
            for k in range(1, nb):
                Pw = np.zeros(nb)
                target = math.floor(k * h / n + 0.5)
                Pw[target] = 1.0
                S = orc.harmonic_sums(Pw, L + 1)
                hits = sum(1 for hh in range(1, n + 1) if math.floor(k * hh / n + 0.5) == target)
                assert S[L, k] == hits


def test_harmonic_sums_gamma_tail(orc):
    rng = np.random.default_rng(11)
    Pw = rng.exponential(1.0, 1 << 20)
    S = orc.harmonic_sums(Pw, 5)
    for L in range(5):
        n = 1 << L
        v = S[L, 4096:]  # bins whose harmonics are all distinct
        for q in [0.5, 0.05, 0.001]:
            x = st.gamma.isf(q, n)
            frac = np.mean(v > x)
            assert abs(frac - q) < 6 * math.sqrt(q / v.size * n) + 1e-3 * q, (n, q, frac)


def test_thresholds(orc):
    for sigma in [3.0, 5.0, 6.0, 8.0]:
        p = 0.5 * math.erfc(sigma / math.sqrt(2))
        assert abs(orc.threshold(1, sigma) + math.log(p)) < 1e-9
        for n in [1, 2, 4, 8, 16]:
            thr = orc.threshold(n, sigma)
            assert abs(sp.gammaincc(n, thr) - p) < 1e-9 * p
            assert abs(orc.gamma_q(n, thr) - sp.gammaincc(n, thr)) < 1e-12
    assert abs(orc.threshold(1, 6.0) - 20.7368) < 1e-4


def test_pmin_snmin(orc):
    assert abs(orc.pmin(2 ** 23) - math.log(2 ** 24)) < 1e-12
    assert abs(orc.snmin(math.exp(math.pi / 4))) < 1e-12
    n = 2.0 ** 23 * 5 * 4096
    v = (math.sqrt(math.log(n)) - math.sqrt(math.pi / 4)) / math.sqrt(1 - math.pi / 4)
    assert abs(orc.snmin(n) - v) < 1e-12
