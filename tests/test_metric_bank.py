"""Random template banks from the frequency-projected metric (bps_metric_*, host code).

Pins:
* the projected-metric density against a 40-digit evaluation of the definition with
  numerically differentiated phase (oracle/metric.py), circular and elliptical;
* the long-observation limit T >> P_orb of the circular density, where the time
  averages have the closed form sqrt(det gamma) = (2 pi f)^3 tau^2 T / sqrt(96);
* the paper's printed circular bank size for its Table 1 region (tests/golden/
  bank_counts.txt);
* exact scalings (density ~ f_max^n) and the N_R formula from the returned volume;
* probabilistic coverage: points drawn with the same density lie within the nominal
  mismatch of some template for a fraction close to eta.
"""
import math
import os

import numpy as np
import pytest

from oracle import metric as orc_metric

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def bps():
    from paper_2112_11991_b300 import build
    build.build()
    import paper_2112_11991_b300 as m
    m.lib()
    return m


def _golden_counts():
    out = {}
    for line in open(os.path.join(HERE, "golden", "bank_counts.txt")):
        if line.strip() and not line.startswith("#"):
            name, dims, count = line.split()
            out[name] = (int(dims), int(count))
    return out


@pytest.mark.parametrize("tmpl,ell", [((8 * 3600.0, 3.0, 1.0, 0.7, 0.05), True),
                                      ((6.5 * 3600, 6.0, 4.0, 2.0, 0.09), True),
                                      ((11 * 3600.0, 0.5, 0.2, 5.0, 0.01), True),
                                      ((9 * 3600.0, 2.0, 5.5, 0.0, 0.0), False),
                                      ((6 * 3600.0, 7.0, 0.1, 0.0, 0.0), False)])
def test_density_matches_high_precision_definition(bps, tmpl, ell):
    sp = bps.default_bank_spec(n_time=32, ecc_max=0.1 if ell else 0.0)
    got = bps.metric_density(sp, np.array([tmpl]))[0]
    ref = orc_metric.projected_sqrt_det(sp.tobs_s, sp.f_max_hz, sp.n_time, tmpl, ell)
    assert got == pytest.approx(ref, rel=1e-7)


@pytest.mark.parametrize("tau,alpha", [(0.5, 0.3), (2.0, 2.0), (1.0, 4.0)])
def test_long_observation_closed_form(bps, tau, alpha):
    P, f = 100.0, 50.0
    T = 200 * P
    sp = bps.default_bank_spec(ecc_max=0.0, tobs_s=T, f_max_hz=f, porb_min_s=P, porb_max_s=P,
                               tau_max_lts=3.0, n_time=16384)
    d = bps.metric_density(sp, np.array([[P, tau, alpha, 0.0, 0.0]]))[0]
    assert d == pytest.approx((2 * math.pi * f) ** 3 * tau ** 2 * T / math.sqrt(96), rel=1e-3)


def test_paper_circular_bank_size(bps):
    dims, count = _golden_counts()["circular"]
    sp = bps.default_bank_spec(ecc_max=0.0, n_time=128, n_volume=100000)
    _, V, N = bps.metric_bank(sp, seed=1, count_only=True)
    assert dims == 3 and N == pytest.approx(count, rel=0.03)


def test_scalings_and_count_formula(bps):
    for ecc in (0.0, 0.1):
        n = 5 if ecc else 3
        a = bps.default_bank_spec(ecc_max=ecc, n_time=64, n_volume=2000)
        b = bps.default_bank_spec(ecc_max=ecc, n_time=64, n_volume=2000, f_max_hz=2 * a.f_max_hz)
        _, Va, Na = bps.metric_bank(a, seed=7, count_only=True)
        _, Vb, _ = bps.metric_bank(b, seed=7, count_only=True)
        assert Vb / Va == pytest.approx(2.0 ** n, rel=1e-9)
        Cn = math.pi ** (n / 2) / math.gamma(n / 2 + 1)
        assert Na == pytest.approx(math.log(1 - a.coverage) /
                                   math.log1p(-a.mismatch ** (n / 2) * Cn / Va), rel=1e-12)
    # the e -> 0 edge: the omega direction shrinks with e, so the density is ~ e
    sp = bps.default_bank_spec(n_time=64)
    d = bps.metric_density(sp, np.array([[8 * 3600.0, 3.0, 1.0, 0.7, e] for e in (0.002, 0.004)]))
    assert d[1] / d[0] == pytest.approx(2.0, rel=0.02)


def test_bank_coverage(bps):
    """T = 2 h, P_orb in [1800, 1900] s, tau <= 0.1 lt-s, f_max 30 Hz: the mismatch
    ellipsoids are small against the region, so the random-bank count gives close to
    the requested coverage eta = 0.9."""
    kw = dict(ecc_max=0.0, tobs_s=7200.0, porb_min_s=1800.0, porb_max_s=1900.0, tau_max_lts=0.1,
              f_max_hz=30.0, n_time=64, n_volume=20000)
    sp = bps.default_bank_spec(**kw)
    bank, V, N = bps.metric_bank(sp, seed=3)
    assert len(bank) == math.ceil(N) and 5000 < len(bank) < 30000
    assert np.all((bank[:, 0] >= 1800) & (bank[:, 0] <= 1900) & (bank[:, 1] >= 0) &
                  (bank[:, 1] <= 0.1) & (bank[:, 2] >= 0) & (bank[:, 2] < 2 * math.pi))
    pts, _, _ = bps.metric_bank(bps.default_bank_spec(**kw, mismatch=0.9), seed=99)
    pts = pts[:300]

    def coords(b):
        return np.stack([b[:, 1], 2 * np.pi / b[:, 0], b[:, 2]], 1)

    cb = coords(bank)
    ms = []
    for p in pts:
        G = bps.metric_projected(sp, p)
        d = cb - coords(p[None])[0]
        d[:, 2] = (d[:, 2] + np.pi) % (2 * np.pi) - np.pi
        ms.append(np.einsum("ki,ij,kj->k", d, G, d).min())
    cov = float(np.mean(np.array(ms) <= sp.mismatch))
    assert 0.8 <= cov <= 0.96, cov


def test_determinism_and_arguments(bps):
    sp = bps.default_bank_spec(ecc_max=0.0, tobs_s=7200.0, porb_min_s=1800.0, porb_max_s=1850.0,
                               tau_max_lts=0.05, f_max_hz=20.0, n_time=32, n_volume=500)
    a, _, _ = bps.metric_bank(sp, seed=5)
    assert a.shape[0] > 50
    b, _, _ = bps.metric_bank(sp, seed=5)
    c, _, _ = bps.metric_bank(sp, seed=6)
    assert a.size > 0 and np.array_equal(a, b) and not np.array_equal(a, c)
    with pytest.raises(bps.BpsError) as e:
        bps.metric_bank(sp, seed=5, cap=max(1, a.shape[0] - 1))
    assert e.value.code == bps.BPS_ERR_CAND_OVERFLOW
    for bad in (dict(mismatch=0.0), dict(coverage=1.0), dict(porb_min_s=-1.0), dict(n_time=4),
                dict(ecc_max=1.0), dict(tau_max_lts=0.0, m_comp_max_msun=0.0)):
        with pytest.raises(bps.BpsError):
            bps.metric_bank(bps.default_bank_spec(**bad), seed=1, count_only=True)
    with pytest.raises(bps.BpsError):
        bps.metric_density(sp, np.array([[-5.0, 1.0, 0.0, 0.0, 0.0]]))
