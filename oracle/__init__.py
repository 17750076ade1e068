"""FP64 CPU oracle for the coherent template-bank binary-pulsar search.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference leg of ``bench.py``; the product package
``paper_2112_11991_b300`` never imports it.  The arithmetic lives in
``oracle/bps_oracle.c`` (plain C, FP64), compiled with gcc by :func:`build`;
this module only marshals numpy arrays through ctypes.

Paper anchors (arXiv:2112.11991): Kepler's equation and the detection
statistic (Sec. 2.1), the BT Roemer delay and Algorithm 1 (App. A),
the incoherent harmonic sum and its chi^2 statistics (Sec. 2.1).

``oracle/metric.py`` evaluates the template-bank metric (Sec. 2.3-2.4) at 40 digits
with numerically differentiated phase, for the tests of the bank generator.

Parity pinned by ``tests/test_oracle_*.py`` against closed forms, brute force
and the paper's printed App. B coefficients; the whitening rule, harmonic bin
map, threshold statistic and out-of-range fill are readings of the paper
(it does not define them) -- "parity unpinned by the paper" for those four,
which are pinned only to the noise statistics they are designed to produce.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bps_oracle.c")
_LIB = os.path.join(_HERE, "_bps_oracle.so")
_lib = None


class Template(C.Structure):
    _fields_ = [("porb_s", C.c_double), ("tau_lts", C.c_double),
                ("phi_rad", C.c_double), ("omega_rad", C.c_double),
                ("ecc", C.c_double)]


class Candidate(C.Structure):
    _fields_ = [("template_idx", C.c_int64), ("nharm", C.c_int32),
                ("near_thr", C.c_int32), ("bin", C.c_int64),
                ("power", C.c_double)]


def build(force: bool = False) -> str:
    """Compile bps_oracle.c into _bps_oracle.so with gcc (-O2, FP64, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-D_GNU_SOURCE", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        d, i64, i32, vp = C.c_double, C.c_int64, C.c_int, C.c_void_p
        L.orc_kepler.restype = d
        L.orc_kepler.argtypes = [d, d]
        L.orc_mean_anomaly.restype = d
        L.orc_mean_anomaly.argtypes = [d, C.POINTER(Template)]
        L.orc_roemer_bt.restype = d
        L.orc_roemer_bt.argtypes = [d, C.POINTER(Template)]
        L.orc_index_map.restype = None
        L.orc_index_map.argtypes = [C.POINTER(Template), i64, d, vp, vp, vp]
        L.orc_resample.restype = None
        L.orc_resample.argtypes = [vp, i64, vp, d, vp]
        L.orc_mean.restype = d
        L.orc_mean.argtypes = [vp, i64]
        L.orc_fft.restype = None
        L.orc_fft.argtypes = [vp, vp, i64]
        L.orc_power_spectrum.restype = None
        L.orc_power_spectrum.argtypes = [vp, i64, vp]
        L.orc_whiten.restype = None
        L.orc_whiten.argtypes = [vp, i64, i64, vp, vp]
        L.orc_harmonic_sums.restype = None
        L.orc_harmonic_sums.argtypes = [vp, i64, i32, vp]
        L.orc_gamma_q.restype = d
        L.orc_gamma_q.argtypes = [i32, d]
        L.orc_threshold.restype = d
        L.orc_threshold.argtypes = [i32, d]
        L.orc_pmin.restype = d
        L.orc_pmin.argtypes = [d]
        L.orc_snmin.restype = d
        L.orc_snmin.argtypes = [d]
        L.orc_search_template.restype = i64
        L.orc_search_template.argtypes = [vp, i64, d, d, C.POINTER(Template), i64,
                                          i32, i64, vp, vp, i64, vp, vp, vp, vp, vp]
        L.orc_search.restype = i32
        L.orc_search.argtypes = [vp, i64, d, d, vp, vp, i64, i32, i64, vp,
                                 vp, i64, vp, vp, i32]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def as_template(t) -> Template:
    """Accept a Template, a 5-sequence (porb, tau, phi, omega, ecc) or a mapping."""
    if isinstance(t, Template):
        return t
    if isinstance(t, dict):
        return Template(t["porb_s"], t["tau_lts"], t["phi_rad"],
                        t.get("omega_rad", 0.0), t.get("ecc", 0.0))
    v = [float(x) for x in t]
    v += [0.0] * (5 - len(v))
    return Template(*v[:5])


def bank_array(bank) -> np.ndarray:
    """(K, 5) float64 array in the order porb_s, tau_lts, phi_rad, omega_rad, ecc."""
    a = np.ascontiguousarray(np.asarray(bank, dtype=np.float64).reshape(-1, 5))
    return a


# --- single steps ------------------------------------------------------------

def kepler(M: float, e: float) -> float:
    return lib().orc_kepler(float(M), float(e))


def mean_anomaly(t: float, tmpl) -> float:
    return lib().orc_mean_anomaly(float(t), C.byref(as_template(tmpl)))


def roemer_bt(t: float, tmpl) -> float:
    return lib().orc_roemer_bt(float(t), C.byref(as_template(tmpl)))


def index_map(tmpl, n: int, tsamp: float):
    """Returns (idx int64[n], off float64[n], near bool[n])  (Algorithm 1)."""
    idx = np.empty(n, np.int64)
    off = np.empty(n, np.float64)
    near = np.empty(n, np.uint8)
    lib().orc_index_map(C.byref(as_template(tmpl)), n, float(tsamp),
                        _ptr(idx), _ptr(off), _ptr(near))
    return idx, off, near.astype(bool)


def series_mean(x: np.ndarray) -> float:
    x = np.ascontiguousarray(x, np.float32)
    return lib().orc_mean(_ptr(x), x.size)


def resample(x: np.ndarray, idx: np.ndarray, fill: float) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float32)
    idx = np.ascontiguousarray(idx, np.int64)
    out = np.empty(x.size, np.float64)
    lib().orc_resample(_ptr(x), x.size, _ptr(idx), float(fill), _ptr(out))
    return out


def fft(z: np.ndarray) -> np.ndarray:
    """Forward unnormalised DFT by the oracle's own radix-2 FFT (complex in, complex out)."""
    z = np.asarray(z, np.complex128)
    re = np.ascontiguousarray(z.real, np.float64).copy()
    im = np.ascontiguousarray(z.imag, np.float64).copy()
    lib().orc_fft(_ptr(re), _ptr(im), re.size)
    return re + 1j * im


def power_spectrum(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float64)
    P = np.empty(x.size // 2, np.float64)
    lib().orc_power_spectrum(_ptr(x), x.size, _ptr(P))
    return P


def whiten(P: np.ndarray, W: int):
    """Returns (Pw, med) -- block lower-median de-reddening."""
    P = np.ascontiguousarray(P, np.float64)
    Pw = np.empty_like(P)
    med = np.empty((P.size + W - 1) // W, np.float64)
    lib().orc_whiten(_ptr(P), P.size, int(W), _ptr(Pw), _ptr(med))
    return Pw, med


def harmonic_sums(Pw: np.ndarray, nlevels: int) -> np.ndarray:
    """(nlevels, nbins): row L holds S_{2^L}."""
    Pw = np.ascontiguousarray(Pw, np.float64)
    S = np.empty((nlevels, Pw.size), np.float64)
    lib().orc_harmonic_sums(_ptr(Pw), Pw.size, int(nlevels), _ptr(S))
    return S


def gamma_q(n: int, x: float) -> float:
    return lib().orc_gamma_q(int(n), float(x))


def threshold(n: int, sigma: float) -> float:
    return lib().orc_threshold(int(n), float(sigma))


def thresholds(nlevels: int, sigma: float) -> np.ndarray:
    return np.array([threshold(1 << L, sigma) for L in range(nlevels)], np.float64)


def pmin(nsamp: float) -> float:
    return lib().orc_pmin(float(nsamp))


def snmin(ntrials: float) -> float:
    return lib().orc_snmin(float(ntrials))


def nlevels_for(nharm_max: int) -> int:
    return int(nharm_max).bit_length()


# --- whole path -----------------------------------------------------------------

def search_template(x, tsamp, tmpl, *, nharm_max=16, whiten_block=1024,
                    sigma=6.0, thr=None, fill=None, template_idx=0,
                    cap=1 << 20, want_arrays=False, idx_in=None):
    """One template through the whole path.  Returns a dict with 'cands'
    (structured numpy array: template_idx, nharm, near_thr, bin, power),
    'n_found', 'n_near' and, if want_arrays, 'idx', 'Pw', 'S'.  idx_in replaces
    the index map (a map validated against index_map(), see bps_oracle.c)."""
    x = np.ascontiguousarray(x, np.float32)
    n = x.size
    nl = nlevels_for(nharm_max)
    thr = thresholds(nl, sigma) if thr is None else np.ascontiguousarray(thr, np.float64)
    fill = series_mean(x) if fill is None else float(fill)
    out = (Candidate * cap)()
    n_near = C.c_int64(0)
    idx = np.empty(n, np.int64) if want_arrays else None
    Pw = np.empty(n // 2, np.float64) if want_arrays else None
    S = np.empty((nl, n // 2), np.float64) if want_arrays else None
    found = lib().orc_search_template(
        _ptr(x), n, float(tsamp), fill, C.byref(as_template(tmpl)), int(template_idx),
        nl, int(whiten_block), _ptr(thr), C.cast(out, C.c_void_p), cap,
        _ptr(idx) if want_arrays else None, _ptr(Pw) if want_arrays else None,
        _ptr(S) if want_arrays else None, C.byref(n_near),
        _ptr(np.ascontiguousarray(idx_in, np.int64)) if idx_in is not None else None)
    cands = _cands_to_numpy(out, min(found, cap))
    res = {"cands": cands, "n_found": int(found), "n_near": int(n_near.value), "thr": thr}
    if want_arrays:
        res.update(idx=idx, Pw=Pw, S=S)
    return res


CAND_DTYPE = np.dtype([("template_idx", np.int64), ("nharm", np.int32),
                       ("near_thr", np.int32), ("bin", np.int64), ("power", np.float64)])


def _cands_to_numpy(buf, count) -> np.ndarray:
    a = np.frombuffer(buf, dtype=CAND_DTYPE, count=len(buf))[:count].copy()
    return a


def search(x, tsamp, bank, *, nharm_max=16, whiten_block=1024, sigma=6.0,
           thr=None, template_ids=None, cap_per=4096, nthreads=None):
    """Whole bank over a pthread pool.  Returns (cands sorted by template, nharm,
    bin; per-template true counts; per-template near-boundary sample counts)."""
    x = np.ascontiguousarray(x, np.float32)
    b = bank_array(bank)
    K = b.shape[0]
    nl = nlevels_for(nharm_max)
    thr = thresholds(nl, sigma) if thr is None else np.ascontiguousarray(thr, np.float64)
    tidx = None if template_ids is None else np.ascontiguousarray(template_ids, np.int64)
    out = (Candidate * (K * cap_per))()
    counts = np.zeros(K, np.int64)
    n_near = np.zeros(K, np.int64)
    nthreads = nthreads or os.cpu_count() or 1
    lib().orc_search(_ptr(x), x.size, float(tsamp), series_mean(x), _ptr(b),
                     _ptr(tidx) if tidx is not None else None, K, nl,
                     int(whiten_block), _ptr(thr), C.cast(out, C.c_void_p), cap_per,
                     _ptr(counts), _ptr(n_near), int(nthreads))
    allc = np.frombuffer(out, dtype=CAND_DTYPE).reshape(K, cap_per)
    parts = [allc[t, :min(counts[t], cap_per)] for t in range(K)]
    cands = np.concatenate(parts) if parts else np.zeros(0, CAND_DTYPE)
    cands = np.sort(cands, order=["template_idx", "nharm", "bin"])
    return cands, counts, n_near
