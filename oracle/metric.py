"""High-precision oracle of the template-bank metric (TEST INFRASTRUCTURE ONLY: used by
``tests/``; the product package never imports it).

Definitions (arXiv:2112.11991):
* phase of a pulsar in a binary, Phi(t) = 2 pi f0 (t - Delta_R(t)), with the BT Roemer
  delay Delta_R = tau [(cos E - e) sin omega + sqrt(1 - e^2) sin E cos omega] and
  Kepler's equation E - e sin E = Omega t + alpha (Sec. 2.1, App. A);
* metric g_ab = <d_a Phi d_b Phi>_T - <d_a Phi>_T <d_b Phi>_T (Sec. 2.3, "Definition of
  Metric and Mismatch"), here with the time average taken by the midpoint rule over
  n_time points of [0, T] (the same quadrature the library uses, so the two agree to
  rounding);
* frequency-projected metric gamma_ab = g_ab - g_fa g_fb / g_ff (Sec. 2.4), coordinates
  (tau, Omega, alpha[, omega, e]).

Derivatives are taken numerically (mpmath's differentiation of Phi itself, at 40
digits), not from hand-derived formulas, and the determinant in 40-digit arithmetic.
"""
from __future__ import annotations

import mpmath as mp


def _phase(lam, t, elliptical):
    f0, tau, om, al = lam[0], lam[1], lam[2], lam[3]
    w, e = (lam[4], lam[5]) if elliptical else (mp.mpf(0), mp.mpf(0))
    M = om * t + al
    E = M + e * mp.sin(M)
    for _ in range(60):
        E = E - (E - e * mp.sin(E) - M) / (1 - e * mp.cos(E))
    delta = tau * ((mp.cos(E) - e) * mp.sin(w) + mp.sqrt(1 - e * e) * mp.sin(E) * mp.cos(w))
    return 2 * mp.pi * f0 * (t - delta)


def projected_sqrt_det(tobs_s, f_max_hz, n_time, template, elliptical, dps=40):
    """sqrt(det gamma) at template (porb_s, tau_lts, alpha, omega, e)."""
    with mp.workdps(dps):
        porb, tau, al, w, e = (mp.mpf(float(x)) for x in template)
        lam = [mp.mpf(float(f_max_hz)), tau, 2 * mp.pi / porb, al]
        if elliptical:
            lam += [w, e]
        d = len(lam)
        T = mp.mpf(float(tobs_s))
        rows = []
        for i in range(n_time):
            t = (i + mp.mpf("0.5")) * T / n_time
            row = []
            for a in range(d):
                def phi_a(x, a=a):
                    l2 = list(lam)
                    l2[a] = x
                    return _phase(l2, t, elliptical)
                row.append(mp.diff(phi_a, lam[a]))
            rows.append(row)
        mean = [sum(r[a] for r in rows) / n_time for a in range(d)]
        g = mp.matrix(d, d)
        for a in range(d):
            for b in range(d):
                g[a, b] = sum((r[a] - mean[a]) * (r[b] - mean[b]) for r in rows) / n_time
        gam = mp.matrix(d - 1, d - 1)
        for a in range(1, d):
            for b in range(1, d):
                gam[a - 1, b - 1] = g[a, b] - g[a, 0] * g[b, 0] / g[0, 0]
        return float(mp.sqrt(mp.det(gam)))
