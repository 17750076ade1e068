"""Oracle pins: Kepler's equation, BT Roemer delay and the Algorithm 1 index map.

Pins (arXiv:2112.11991):
  * Kepler residual |E - e sin E - M| <= 1e-12 (Sec. 2.1, Kepler's equation);
  * the printed App. B series for cos E and sqrt(1-e^2) sin E agree with the
    Newton solution to O(e^7) (tests/golden/appb_coefficients.txt);
  * e = 0 reduces the BT delay to the circular model tau sin(Omega t + alpha)
    (Sec. 2.1, circular phase model), and an e = 0 elliptical template with
    (phi, omega) equals the circular template with phase phi + omega;
  * tau = 0 and Omega -> 0 give the identity index map; idx_0 = 0 (zero offset
    of Algorithm 1); the map moves by at most one sample per step.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden", "appb_coefficients.txt")


def _appb():
    C, S = {}, {}
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        s, k, p, num, den = line.split()
        d = C if s == "C" else S
        d.setdefault(int(k), {})[int(p)] = Fraction(int(num), int(den))
    return C, S


def test_kepler_residual_grid(orc):
    worst = 0.0
    for e in [0.0, 1e-6, 0.01, 0.05, 0.1, 0.3, 0.6, 0.9, 0.97]:
        for M in np.linspace(-7.0, 13.0, 401):
            E = orc.kepler(M, e)
            worst = max(worst, abs(E - e * math.sin(E) - M))
    assert worst <= 1e-12


def test_kepler_special_values(orc):
    assert orc.kepler(0.0, 0.5) == 0.0
    assert abs(orc.kepler(math.pi, 0.7) - math.pi) < 1e-14
    for M in [0.3, 1.7, 2.9]:
        assert orc.kepler(M, 0.0) == M
        assert abs(orc.kepler(-M, 0.4) + orc.kepler(M, 0.4)) < 1e-14


@pytest.mark.parametrize("e", [0.01, 0.05, 0.1])
def test_appb_series_matches_newton(orc, e):
    C, S = _appb()
    worst_c = worst_s = 0.0
    for M in np.linspace(0.0, 2 * math.pi, 257):
        E = orc.kepler(M, e)
        cs = sum(float(sum(c * Fraction(e) ** p for p, c in C[k].items())) * math.cos(k * M)
                 for k in C)
        ss = sum(float(sum(c * Fraction(e) ** p for p, c in S[k].items())) * math.sin(k * M)
                 for k in S)
        worst_c = max(worst_c, abs(cs - math.cos(E)))
        worst_s = max(worst_s, abs(ss - math.sqrt(1 - e * e) * math.sin(E)))
    bound = 10 * e ** 7
    assert worst_c <= bound, (worst_c, bound)
    assert worst_s <= bound, (worst_s, bound)


def test_appb_error_shrinks_like_e7(orc):
    """Halving e must shrink the truncation error by ~2^7 (a wrong coefficient
    would leave an error of lower order)."""
    C, S = _appb()

    def err(e):
        w = 0.0
        for M in np.linspace(0.0, 2 * math.pi, 129):
            E = orc.kepler(M, e)
            cs = sum(float(sum(c * Fraction(e) ** p for p, c in C[k].items())) * math.cos(k * M)
                     for k in C)
            w = max(w, abs(cs - math.cos(E)))
        return w

    r = err(0.2) / err(0.1)
    assert 2 ** 6 < r < 2 ** 8, r


def test_bt_circular_closed_form(orc):
    for (porb, tau, phi) in [(400.0, 0.2, 1.0), (1610.0, 3.0, 5.5), (3e4, 20.0, 0.1)]:
        om = 2 * math.pi / porb
        for t in np.linspace(0.0, 600.0, 31):
            d = orc.roemer_bt(t, (porb, tau, phi, 0.0, 0.0))
            assert abs(d - tau * math.sin(om * t + phi)) <= 1e-12 * max(1.0, tau)


def test_bt_e0_elliptical_equals_circular(orc):
    n, ts = 1 << 12, 64e-6
    a = orc.index_map((50.0, 0.7, 0.4, 1.9, 0.0), n, ts)[0]
    b = orc.index_map((50.0, 0.7, 0.4 + 1.9, 0.0, 0.0), n, ts)[0]
    assert np.array_equal(a, b)


def test_bt_periodic_in_orbit(orc):
    tm = (300.0, 1.3, 0.8, 2.2, 0.4)
    for t in [0.0, 17.0, 123.4]:
        assert abs(orc.roemer_bt(t, tm) - orc.roemer_bt(t + 300.0, tm)) < 1e-10


def test_index_map_identity_cases(orc):
    n, ts = 1 << 14, 64e-6
    for tm in [(400.0, 0.0, 1.0, 0.0, 0.0), (400.0, 0.0, 2.0, 1.0, 0.3),
               (1e12, 5.0, 0.7, 0.0, 0.0), (1e13, 5.0, 0.7, 1.2, 0.1)]:
        idx, off, near = orc.index_map(tm, n, ts)
        assert np.array_equal(idx, np.arange(n))


def test_index_map_zero_offset_and_steps(orc):
    n, ts = 1 << 15, 64e-6
    for tm in [(400.0, 0.2, 1.0, 0.0, 0.0), (90.0, 0.4, 4.0, 1.0, 0.5)]:
        idx, off, near = orc.index_map(tm, n, ts)
        assert idx[0] == 0 and off[0] == 0.0
        steps = np.diff(idx)
        assert steps.min() >= 0 and steps.max() <= 2


def test_index_map_follows_velocity(orc):
    """d off / dj = -tau Omega t_s cos(M) / t_s (circular): the map drifts
    against the line-of-sight velocity, sign fixed by Algorithm 1."""
    n, ts = 1 << 16, 64e-6
    porb, tau, phi = 40.0, 0.3, 0.0  # cos(phi) = 1: delay grows at t = 0
    idx, off, near = orc.index_map((porb, tau, phi, 0.0, 0.0), n, ts)
    slope = (off[1000] - off[0]) / 1000.0
    expect = -tau * (2 * math.pi / porb)
    assert abs(slope - expect) < 1e-3 * abs(expect)
