"""Candidate distillation (bps_distill, host routine): repeated detections of one
signal -- same fundamental frequency under several templates or levels, or a
small-integer harmonic ratio of it -- collapse into one group led by the most
significant member (false-alarm exponent -ln Q(n, S) of the Gamma(n, 1) tail)."""
import math

import numpy as np
import pytest
import scipy.special as sp


@pytest.fixture(scope="module")
def bps():
    from paper_2112_11991_b300 import build
    build.build()
    import paper_2112_11991_b300 as m
    m.lib()
    return m


def _cands(bps, rows):
    a = np.zeros(len(rows), bps.CAND_DTYPE)
    for i, (t, n, k, s) in enumerate(rows):
        a[i] = (t, n, 0, k, s)
    return a


N, TS = 1 << 20, 64e-6
T = N * TS


def test_groups_duplicates_and_harmonics(bps):
    f0 = 41.7  # Hz, fundamental of a "pulsar"
    k = lambda f, n: int(round(f * n * T))
    rows = [
        (3, 16, k(f0, 16), 300.0),      # strongest: the true orbit, 16 harmonics
        (4, 16, k(f0, 16) + 1, 250.0),  # neighbouring template, next bin
        (7, 8, k(f0, 8), 120.0),        # same signal at 8 harmonics
        (3, 4, k(2 * f0, 4), 90.0),     # second harmonic seen as a fundamental
        (9, 2, k(1.5 * f0, 2), 60.0),   # 3/2 ratio
        (5, 16, k(f0 * math.pi, 16), 80.0),  # unrelated (irrational ratio)
    ]
    out = bps.distill(_cands(bps, rows), N, TS, tol_bins=1.5, max_ratio=16)
    assert out.size == 2
    assert out[0]["template_idx"] == 3 and out[0]["nharm"] == 16 and out[0]["flags"] == 5
    assert out[1]["template_idx"] == 5 and out[1]["flags"] == 1


def test_significance_order_matches_gamma_tail(bps):
    rows = [(0, 1, 1000, 30.0), (1, 16, 5001, 70.0), (2, 4, 7777, 40.0), (3, 8, 9999, 50.0)]
    out = bps.distill(_cands(bps, rows), N, TS, tol_bins=0.01, max_ratio=1)
    ref = sorted(rows, key=lambda r: -(-math.log(sp.gammaincc(r[1], r[3]))))
    assert [int(c["template_idx"]) for c in out] == [r[0] for r in ref]


def test_invalid_and_empty(bps):
    assert bps.distill(np.zeros(0, bps.CAND_DTYPE), N, TS).size == 0
    with pytest.raises(bps.BpsError):
        bps.distill(_cands(bps, [(0, 1, 5, 30.0)]), N, TS, tol_bins=0.0)


def test_distill_oracle_candidates(bps, orc):
    """Candidates of a noise + pulsar series under a few templates (FP64 oracle) distil
    to a leading group at a small-integer ratio of the pulsar's frequency."""
    import synth
    ts, n = 64e-6, 1 << 18
    p = synth.Pulsar(period_s=0.02, porb_s=30.0, tau_lts=0.2, phi_rad=1.0, amp=0.4)
    x = synth.inject(synth.noise(n, 20), ts, p)
    bank = np.array([p.orbit(), (30.0, 0.21, 1.0, 0, 0), (30.0, 0.19, 1.02, 0, 0)])
    oc, _, _ = orc.search(x, ts, bank)
    c = np.zeros(oc.size, bps.CAND_DTYPE)
    for f in ("template_idx", "nharm", "bin", "power"):
        c[f] = oc[f]
    out = bps.distill(c, n, ts, tol_bins=2.0, max_ratio=16)
    assert out.size < oc.size / 10
    lead = out[0]
    f = float(lead["bin"]) / (float(lead["nharm"]) * n * ts)
    r = f * p.period_s
    assert any(abs(r - a / b) < 2.0 / (n * ts) * p.period_s * 16 for a in range(1, 17)
               for b in range(1, 17))
