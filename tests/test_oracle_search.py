"""Oracle pins on the whole per-template path (App. A, Algorithm 1 + Sec. 2.1).

  * an injected pulsar is recovered under its true orbit at
    k = round(n f0 T) (+-1) for every harmonic level n, circular and
    elliptical, and the true orbit beats the zero orbit and every random
    template of the bank;
  * the candidate set is invariant to scaling the series (whitening);
  * on noise alone the false-alarm count per level matches (N/2) Q(n, thr).
"""
import math

import numpy as np
import pytest

import synth


def _check_recovery(orc, x, tsamp, p, tmpl, nlevels=5):
    n = x.size
    T = n * tsamp
    r = orc.search_template(x, tsamp, tmpl, want_arrays=True, nharm_max=1 << (nlevels - 1))
    S = r["S"]
    for L in range(nlevels):
        nh = 1 << L
        k_best = int(np.argmax(S[L]))
        k_true = round(nh * T / p.period_s)
        # fundamental may be out-scored by a stronger harmonic at n = 1, 2
        if nh >= 4:
            assert abs(k_best - k_true) <= 1, (nh, k_best, k_true)
        assert S[L, k_true - 1:k_true + 2].max() >= r["thr"][L]
    return S


def test_circular_pulsar_recovered(orc):
    ts, n = 64e-6, 1 << 18
    p = synth.Pulsar(period_s=0.02, porb_s=30.0, tau_lts=0.2, phi_rad=1.0, amp=0.4)
    x = synth.inject(synth.noise(n, 20), ts, p)
    S_true = _check_recovery(orc, x, ts, p, p.orbit())
    S_zero = orc.search_template(x, ts, (p.porb_s, 0.0, 0.0), want_arrays=True)["S"]
    assert S_true[4].max() > 3.0 * S_zero[4].max()


def test_elliptical_pulsar_recovered(orc):
    ts, n = 64e-6, 1 << 18
    p = synth.Pulsar(period_s=0.02, porb_s=25.0, tau_lts=0.3, phi_rad=2.0,
                     omega_rad=1.1, ecc=0.3, amp=0.4)
    x = synth.inject(synth.noise(n, 21), ts, p)
    S_true = _check_recovery(orc, x, ts, p, p.orbit())
    # the same orbit without eccentricity loses the signal
    wrong = (p.porb_s, p.tau_lts, p.phi_rad, p.omega_rad, 0.0)
    S_wrong = orc.search_template(x, ts, wrong, want_arrays=True)["S"]
    assert S_true[4].max() > 3.0 * S_wrong[4].max()


def test_true_template_best_in_bank(orc):
    w = synth.plain_circular(n=1 << 18, K=12)
    cands, counts, _ = orc.search(w.series, w.tsamp, w.bank)
    best = {}
    for c in cands[cands["nharm"] == 16]:
        best[c["template_idx"]] = max(best.get(c["template_idx"], 0.0), c["power"])
    assert max(best, key=best.get) == w.true_idx[0]


def test_candidates_scale_invariant(orc):
    w = synth.plain_circular(n=1 << 16, K=2)
    a = orc.search_template(w.series, w.tsamp, w.bank[w.true_idx[0]])["cands"]
    b = orc.search_template(w.series * np.float32(4.0), w.tsamp, w.bank[w.true_idx[0]])["cands"]
    assert np.array_equal(a[["nharm", "bin"]], b[["nharm", "bin"]])


def test_noise_false_alarm_rate(orc):
    n = 1 << 18
    x = synth.noise(n, 33)
    sigma = 3.0
    r = orc.search_template(x, 64e-6, (400.0, 0.1, 0.5), sigma=sigma, cap=1 << 20)
    c = r["cands"]
    p = 0.5 * math.erfc(sigma / math.sqrt(2))
    for L in range(5):
        nh = 1 << L
        got = np.sum((c["nharm"] == nh) & (c["bin"] >= 64))
        expect = (n // 2 - 64) * p
        assert abs(got - expect) < 6 * math.sqrt(expect) + 0.05 * expect, (nh, got, expect)
