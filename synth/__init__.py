"""Seeded synthetic inputs shared by the tests, ``bench.py`` and ``smoke()``.

This module holds none of the search's arithmetic (no index map, FFT,
whitening, harmonic sum or threshold).  It draws:

* white Gaussian noise N(0, 1) in float32 (numpy PCG64, fixed seeds);
* uniform random orbital template banks over the prior boxes of the
  workloads (the paper's random-template-bank prior ranges, Sec. 2.3 and
  Table 1), with the true orbits of the injected pulsars placed at seeded
  indices;
* injected pulsars: a periodic Gaussian pulse (FWHM = duty x period) emitted
  at rest-frame time t' and received at t = t' + Delta(0) - Delta(t') (solved
  exactly on a grid fine enough for 1e-13 s interpolation error), the
  exact inverse of the paper's nearest-neighbour demodulation map
  (Algorithm 1, App. A) and, to first order in tau*Omega, the paper's
  phase model Phi(t) = 2 pi f0 t + phi_D(t) (Sec. 2.1).  The orbit is
  evaluated with its own Kepler solver (a plain fixed-point iteration
  E <- M + e sin E, deliberately not the Newton iteration used by either
  the oracle or the CUDA path) so that no orbit code is shared.

Projected semi-major axes come from Kepler's third law with the paper's
mass limits (Sec. 2.6): tau_max = theta G^(1/3) Omega^(-2/3) m_c /
(c (m_p + m_c)^(2/3)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

G_SI = 6.67430e-11
C_SI = 299792458.0
MSUN_KG = 1.98847e30
TWO_PI = 2.0 * math.pi


def noise(n: int, seed: int) -> np.ndarray:
    """N(0,1) white noise, float32, from a fixed seed."""
    return np.random.default_rng(seed).standard_normal(n, dtype=np.float32)


def tau_max(porb_s, m_p=1.4, m_c=8.0, theta=1.0):
    """Largest projected semi-major axis [lt-s] (Kepler III, Sec. 2.6)."""
    om = TWO_PI / np.asarray(porb_s, np.float64)
    gm13 = (G_SI * MSUN_KG) ** (1.0 / 3.0)
    return theta * gm13 * om ** (-2.0 / 3.0) * m_c / (C_SI * (m_p + m_c) ** (2.0 / 3.0))


@dataclass
class Pulsar:
    period_s: float
    porb_s: float
    tau_lts: float
    phi_rad: float
    omega_rad: float = 0.0
    ecc: float = 0.0
    amp: float = 0.3
    duty: float = 0.05
    phase0: float = 0.0

    def orbit(self):
        return (self.porb_s, self.tau_lts, self.phi_rad, self.omega_rad, self.ecc)


def _ecc_anomaly_fixed_point(M: np.ndarray, e: float, E0=None) -> np.ndarray:
    """E - e sin E = M by the fixed-point iteration E <- M + e sin E (contraction
    factor e), started from E0 when given (a nearby earlier solution)."""
    E = M.copy() if E0 is None else E0.copy()
    if e == 0.0:
        return M.copy()
    for _ in range(4000):
        En = M + e * np.sin(E)
        if np.max(np.abs(En - E)) < 1e-15:
            return En
        E = En
    return E


def _orbit_delay(t: np.ndarray, p: Pulsar, E0=None):
    """Orbital light-travel delay of the pulsar at emission time t [s], and the
    eccentric anomaly it used."""
    M = (TWO_PI / p.porb_s) * t + p.phi_rad
    E = _ecc_anomaly_fixed_point(M, p.ecc, E0)
    e = p.ecc
    d = p.tau_lts * ((np.cos(E) - e) * math.sin(p.omega_rad)
                     + math.sqrt(1.0 - e * e) * np.sin(E) * math.cos(p.omega_rad))
    return d, E


def _emission_times_exact(t: np.ndarray, p: Pulsar) -> np.ndarray:
    """Rest-frame time t' of the signal received at t, solving
    t = t' + Delta(0) - Delta(t') by fixed-point iteration (|dDelta/dt| << 1)."""
    d0 = float(_orbit_delay(np.zeros(1), p)[0][0])
    tp = t.copy()
    E = None
    for _ in range(200):
        d, E = _orbit_delay(tp, p, E)
        tn = t - d0 + d
        done = np.max(np.abs(tn - tp)) < 1e-12
        tp = tn
        if done:
            break
    return tp


def emission_times(n: int, tsamp: float, p: Pulsar, chunk: int = 1 << 22) -> np.ndarray:
    """Rest-frame time t' of the signal received at t = i*tsamp.  t'(t) is smooth on
    orbital time scales: it is solved exactly on a grid of every `stride` samples
    and interpolated linearly in between, with stride the largest power of two
    <= 64 whose interpolation error bound (stride t_s)^2/8 * tau Omega^2 / (1-e)^3
    stays below 1e-13 s (stride 1, no interpolation, for fast orbits)."""
    om = TWO_PI / p.porb_s
    curv = p.tau_lts * om * om / (1.0 - p.ecc) ** 3
    stride = 64
    while stride > 1 and (stride * tsamp) ** 2 / 8.0 * curv > 1e-13:
        stride //= 2
    out = np.empty(n, np.float64)
    if stride == 1:
        for s in range(0, n, chunk):
            t = np.arange(s, min(n, s + chunk), dtype=np.float64) * tsamp
            out[s:s + t.size] = _emission_times_exact(t, p)
        return out
    grid = np.arange(0, n + stride, stride, dtype=np.float64) * tsamp
    tg = np.empty_like(grid)
    for s in range(0, grid.size, chunk):
        tg[s:s + chunk] = _emission_times_exact(grid[s:s + chunk], p)
    t = np.arange(n, dtype=np.float64) * tsamp
    return np.interp(t, grid, tg)


def inject(x: np.ndarray, tsamp: float, p: Pulsar) -> np.ndarray:
    """Add a Gaussian pulse train (FWHM = duty periods, peak amp) in place."""
    tp = emission_times(x.size, tsamp, p)
    ph = tp / p.period_s + p.phase0
    fr = ph - np.floor(ph) - 0.5
    w = p.duty / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    x += (p.amp * np.exp(-(fr * fr) / (2.0 * w * w))).astype(np.float32)
    return x


def uniform_bank(K: int, seed: int, porb=(200.0, 670.0), tau=(0.0, 0.4),
                 ecc=None, true_orbits=(), true_seed=None) -> tuple[np.ndarray, list[int]]:
    """K templates as a (K, 5) float64 array (porb_s, tau_lts, phi_rad, omega_rad, ecc).
    Circular when ecc is None (omega = e = 0).  True orbits replace the random
    template at seeded distinct indices, which are returned."""
    rng = np.random.default_rng(seed)
    b = np.zeros((K, 5), np.float64)
    b[:, 0] = rng.uniform(porb[0], porb[1], K)
    b[:, 1] = rng.uniform(tau[0], tau[1], K)
    b[:, 2] = rng.uniform(0.0, TWO_PI, K)
    if ecc is not None:
        b[:, 3] = rng.uniform(0.0, TWO_PI, K)
        b[:, 4] = rng.uniform(ecc[0], ecc[1], K)
    where = []
    if true_orbits:
        r2 = np.random.default_rng(seed + 7919 if true_seed is None else true_seed)
        where = sorted(r2.choice(K, size=len(true_orbits), replace=False).tolist())
        for w, o in zip(where, true_orbits):
            b[w] = o
    return b, where


@dataclass
class Workload:
    name: str
    n: int
    tsamp: float
    bank: np.ndarray
    pulsars: list = field(default_factory=list)
    true_idx: list = field(default_factory=list)
    seed: int = 1
    nharm_max: int = 16
    whiten_block: int = 1024
    sigma: float = 6.0
    series: np.ndarray | None = None

    def describe(self) -> dict:
        return {"workload": self.name, "n_samples": self.n, "tsamp_s": self.tsamp,
                "templates": int(self.bank.shape[0]), "nharm_max": self.nharm_max,
                "whiten_block": self.whiten_block, "sigma": self.sigma,
                "seed": self.seed, "pulsars": [asdict(p) for p in self.pulsars],
                "true_template_idx": list(self.true_idx)}


def plain_circular(n: int = 1 << 20, K: int = 32, seed: int = 1, with_series=True) -> Workload:
    """2^20 samples at 64 us, N(0,1) + one pulsar (P = 20 ms, 5 % duty, A = 0.3)
    in a circular orbit Porb = 400 s, tau = 0.2 lt-s, phi = 1.0 rad; K-1 random
    templates Porb U[200,670] s, tau U[0,0.4] lt-s, phi U[0,2pi) + the true orbit."""
    tsamp = 64e-6
    p = Pulsar(period_s=0.020, porb_s=400.0, tau_lts=0.2, phi_rad=1.0)
    bank, where = uniform_bank(K, seed + 100, (200.0, 670.0), (0.0, 0.4),
                               true_orbits=[p.orbit()])
    w = Workload("plain circular search 2^%d x %d templates" % (int(math.log2(n)), K),
                 n, tsamp, bank, [p], where, seed)
    if with_series:
        x = noise(n, seed)
        w.series = inject(x, tsamp, p)
    return w


def htru_circular(n: int = 1 << 23, K: int = 4096, seed: int = 2, with_series=True,
                  amp: float = 0.02) -> Workload:
    """HTRU-like: 2^23 samples at 64 us (537 s), N(0,1) + 3 pulsar-BH binaries
    (P U[20,100] ms, m_p 1.4, m_c 10 Msun, Porb U[3T,10T], cos i U[0,1),
    tau = tau_max sin i, peak amplitude 0.02 sigma: the single-pulse S/N of the
    paper's simulations, Table 2); K-3 templates Porb U[3T,10T], tau U[0,3] lt-s,
    phi U."""
    tsamp = 64e-6
    T = n * tsamp
    rng = np.random.default_rng(seed + 200)
    pulsars = []
    for _ in range(3):
        porb = rng.uniform(3 * T, 10 * T)
        cosi = rng.uniform(0.0, 1.0)
        tau = float(tau_max(porb, 1.4, 10.0)) * math.sqrt(1.0 - cosi * cosi)
        pulsars.append(Pulsar(period_s=rng.uniform(0.020, 0.100), porb_s=porb,
                              tau_lts=tau, phi_rad=rng.uniform(0.0, TWO_PI), amp=amp))
    bank, where = uniform_bank(K, seed + 100, (3 * T, 10 * T), (0.0, 3.0),
                               true_orbits=[p.orbit() for p in pulsars])
    w = Workload("HTRU-like circular search 2^%d x %d templates" % (int(math.log2(n)), K),
                 n, tsamp, bank, pulsars, where, seed)
    if with_series:
        x = noise(n, seed)
        for p in pulsars:
            inject(x, tsamp, p)
        w.series = x
    return w


def equal_snr_amp(n: int, amp_2p23: float = 0.02) -> float:
    """Peak amplitude that gives a pulse train in n samples the per-harmonic signal-to-noise
    of amplitude amp_2p23 in 2^23 samples (the coherent power grows as amp^2 n)."""
    return amp_2p23 * math.sqrt((1 << 23) / n)


def pulsar_bh_series(n: int, tsamp: float, seed: int, amp: float = 0.02):
    """N(0,1) series with one pulsar-BH binary drawn as in htru_circular (P U[20,100] ms,
    m_c 10 Msun, Porb U[3T,10T], tau = tau_max sin i).  Returns (series, Pulsar)."""
    T = n * tsamp
    rng = np.random.default_rng(seed + 700)
    porb = rng.uniform(3 * T, 10 * T)
    cosi = rng.uniform(0.0, 1.0)
    p = Pulsar(period_s=rng.uniform(0.020, 0.100), porb_s=porb,
               tau_lts=float(tau_max(porb, 1.4, 10.0)) * math.sqrt(1.0 - cosi * cosi),
               phi_rad=rng.uniform(0.0, TWO_PI), amp=amp)
    x = noise(n, seed)
    inject(x, tsamp, p)
    return x, p


def elliptical_imbh(n: int = 1 << 25, K: int = 2048, seed: int = 3, with_series=True,
                    amp: float = 0.02) -> Workload:
    """Elliptical IMBH-in-globular-cluster: 2^25 samples at 128 us, 2 pulsars with
    e = 0.05 and 0.09 (P U[20,40] ms, peak amplitude 0.02 sigma as in Table 2);
    K-2 templates Porb U[5T,10T], tau U[0,20], phi, omega U[0,2pi), e U[0,0.1]."""
    tsamp = 128e-6
    T = n * tsamp
    rng = np.random.default_rng(seed + 200)
    pulsars = []
    for e in (0.05, 0.09):
        pulsars.append(Pulsar(period_s=rng.uniform(0.020, 0.040),
                              porb_s=rng.uniform(5 * T, 10 * T),
                              tau_lts=rng.uniform(0.0, 20.0),
                              phi_rad=rng.uniform(0.0, TWO_PI),
                              omega_rad=rng.uniform(0.0, TWO_PI), ecc=e, amp=amp))
    bank, where = uniform_bank(K, seed + 100, (5 * T, 10 * T), (0.0, 20.0),
                               ecc=(0.0, 0.1), true_orbits=[p.orbit() for p in pulsars])
    w = Workload("elliptical IMBH search 2^%d x %d templates" % (int(math.log2(n)), K),
                 n, tsamp, bank, pulsars, where, seed)
    if with_series:
        x = noise(n, seed)
        for p in pulsars:
            inject(x, tsamp, p)
        w.series = x
    return w
