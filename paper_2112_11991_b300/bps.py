"""ctypes binding of ``libbps.so`` (C ABI in include/bps.h).

Argument marshalling only: every step of the search runs in the library's CUDA
kernels.  There is no CPU fallback -- if the library is missing or no CUDA
device is present the calls raise :class:`BpsError`.

Functions keep the C names (``bps_create`` ...); :class:`Context` wraps them.
Arrays may be numpy arrays (host) or torch tensors (host or CUDA; a CUDA float32
tensor is passed by device pointer).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libbps.so")
_lib = None

BPS_OK = 0
BPS_ERR_INVALID_ARG = -1
BPS_ERR_OUT_OF_MEMORY = -2
BPS_ERR_NOT_READY = -3
BPS_ERR_CAND_OVERFLOW = -4
BPS_ERR_TIMEOUT = -5
BPS_ERR_CUDA = -6
BPS_ERR_UNSUPPORTED = -7

BPS_F32 = 0
BPS_F16_SCALED = 1
BPS_MODE_FUSED = 0
BPS_MODE_PLAIN = 1
BPS_PASS1_AUTO = 0
BPS_PASS1_FUSED = 1
BPS_PASS1_WARPSPEC = 2
BPS_PASS1_ASYNC = 3
BPS_POWER_AUTO = 0
BPS_POWER_BINS = 1
BPS_POWER_ROWS = 2
BPS_PASS2_AUTO = 0
BPS_PASS2_FUSED = 1
BPS_PASS2_TMA = 2

EXPORTED = ["bps_default_params", "bps_create", "bps_destroy", "bps_load_series",
            "bps_load_bank", "bps_search", "bps_query", "bps_fetch_candidates",
            "bps_unload", "bps_last_error", "bps_index_map", "bps_whitened_spectrum",
            "bps_harmonic_sums", "bps_thresholds", "bps_set_profiling",
            "bps_request_stats", "bps_whitened_spectrum_noalloc", "bps_server_create",
            "bps_server_destroy", "bps_server_submit", "bps_server_result", "bps_server_stats",
            "bps_server_last_error", "bps_autotune", "bps_distill", "bps_series_update",
            "bps_graph_create", "bps_graph_launch", "bps_graph_fetch", "bps_default_bank_spec",
            "bps_metric_density", "bps_metric_projected", "bps_metric_bank",
            "bps_selftest_bounded_wait", "bps_whiten", "bps_server_load_series",
            "bps_server_submit_series", "bps_server_unload_series", "bps_server_series_info"]
STAGES = ["anchors", "pass1", "pass2", "power", "median", "harmsum"]


class BpsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("bps error %d: %s" % (code, msg))
        self.code = code


class bps_template(C.Structure):
    _fields_ = [("porb_s", C.c_double), ("tau_lts", C.c_double), ("phi_rad", C.c_double),
                ("omega_rad", C.c_double), ("ecc", C.c_double)]


class bps_candidate(C.Structure):
    _fields_ = [("template_idx", C.c_uint32), ("nharm", C.c_uint16), ("flags", C.c_uint16),
                ("bin", C.c_uint32), ("power", C.c_float)]


class bps_bank_spec(C.Structure):
    _fields_ = [("tobs_s", C.c_double), ("f_max_hz", C.c_double), ("mismatch", C.c_double),
                ("coverage", C.c_double), ("porb_min_s", C.c_double), ("porb_max_s", C.c_double),
                ("tau_max_lts", C.c_double), ("m_pulsar_min_msun", C.c_double),
                ("m_comp_max_msun", C.c_double), ("ecc_max", C.c_double), ("n_time", C.c_int32),
                ("n_volume", C.c_int32)]


class bps_search_params(C.Structure):
    _fields_ = [("nharm_max", C.c_int32), ("whiten_block", C.c_int32), ("sigma_thr", C.c_double),
                ("auto_thr", C.c_int32), ("mode", C.c_int32), ("cand_cap", C.c_int64),
                ("precision", C.c_int32), ("batch", C.c_int32), ("log_tile", C.c_int32),
                ("log_tile2", C.c_int32), ("log_cols", C.c_int32), ("pass1_kind", C.c_int32),
                ("power_layout", C.c_int32), ("pass2_kind", C.c_int32)]


class bps_server_config(C.Structure):
    _fields_ = [("max_active", C.c_int32), ("groups_in_flight", C.c_int32),
                ("hbm_budget", C.c_int64)]


class bps_stats(C.Structure):
    _fields_ = [("templates", C.c_int64), ("batch", C.c_int32), ("anchor_block", C.c_int32),
                ("launches", C.c_int32), ("profiled", C.c_int32),
                ("stage_launches", C.c_int32 * 8), ("stage_ms", C.c_float * 8)]


CAND_DTYPE = np.dtype([("template_idx", np.uint32), ("nharm", np.uint16), ("flags", np.uint16),
                       ("bin", np.uint32), ("power", np.float32)])


def library_path() -> str:
    return _LIB_PATH


def lib():
    """Load libbps.so (raises BpsError when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise BpsError(BPS_ERR_UNSUPPORTED,
                           "libbps.so not built (run paper_2112_11991_b300/build.py)")
        L = C.CDLL(_LIB_PATH)
        vp, i64, i32, P = C.c_void_p, C.c_int64, C.c_int, C.POINTER
        L.bps_default_params.restype = None
        L.bps_default_params.argtypes = [P(bps_search_params)]
        L.bps_create.restype = i32
        L.bps_create.argtypes = [P(vp), i32]
        L.bps_destroy.restype = None
        L.bps_destroy.argtypes = [vp]
        L.bps_load_series.restype = i32
        L.bps_load_series.argtypes = [vp, vp, i64, C.c_double, i32, i32, P(i64)]
        L.bps_load_bank.restype = i32
        L.bps_load_bank.argtypes = [vp, vp, i64, P(i64)]
        L.bps_search.restype = i32
        L.bps_search.argtypes = [vp, i64, i64, P(bps_search_params), vp, P(i64)]
        L.bps_query.restype = i32
        L.bps_query.argtypes = [vp, i64, P(i32)]
        L.bps_fetch_candidates.restype = i32
        L.bps_fetch_candidates.argtypes = [vp, i64, vp, i64, P(i64), P(i64)]
        L.bps_unload.restype = i32
        L.bps_unload.argtypes = [vp, i64]
        L.bps_last_error.restype = C.c_char_p
        L.bps_last_error.argtypes = [vp]
        L.bps_index_map.restype = i32
        L.bps_index_map.argtypes = [vp, i64, i64, i64, vp, P(i64)]
        L.bps_whitened_spectrum.restype = i32
        L.bps_whitened_spectrum.argtypes = [vp, i64, i64, i64, i64, P(bps_search_params), vp]
        L.bps_harmonic_sums.restype = i32
        L.bps_harmonic_sums.argtypes = [vp, i64, i64, i64, P(bps_search_params), vp]
        L.bps_set_profiling.restype = i32
        L.bps_set_profiling.argtypes = [vp, i32]
        L.bps_request_stats.restype = i32
        L.bps_request_stats.argtypes = [vp, i64, P(bps_stats)]
        L.bps_whitened_spectrum_noalloc.restype = i32
        L.bps_whitened_spectrum_noalloc.argtypes = [vp, i64, C.c_double, C.c_double,
                                                    P(bps_template), i32, vp, vp]
        L.bps_server_create.restype = i32
        L.bps_server_create.argtypes = [vp, P(bps_server_config), P(vp)]
        L.bps_server_destroy.restype = None
        L.bps_server_destroy.argtypes = [vp]
        L.bps_server_submit.restype = i32
        L.bps_server_submit.argtypes = [vp, vp, i64, C.c_double, i32, vp, i64,
                                        P(bps_search_params), P(i64)]
        L.bps_server_result.restype = i32
        L.bps_server_result.argtypes = [vp, i64, C.c_int32, vp, i64, P(i64), P(i64),
                                        P(C.c_double)]
        L.bps_server_load_series.restype = i32
        L.bps_server_load_series.argtypes = [vp, vp, i64, C.c_double, i32, P(i64)]
        L.bps_server_submit_series.restype = i32
        L.bps_server_submit_series.argtypes = [vp, i64, vp, i64, P(bps_search_params), P(i64)]
        L.bps_server_unload_series.restype = i32
        L.bps_server_unload_series.argtypes = [vp, i64]
        L.bps_server_series_info.restype = i32
        L.bps_server_series_info.argtypes = [vp, i64, P(C.c_int32), P(i64)]
        L.bps_server_stats.restype = i32
        L.bps_server_stats.argtypes = [vp, P(i64), P(i64), P(i64), P(i64)]
        L.bps_server_last_error.restype = C.c_char_p
        L.bps_server_last_error.argtypes = [vp]
        L.bps_autotune.restype = i32
        L.bps_autotune.argtypes = [vp, i64, i64, P(bps_search_params), i64, P(bps_search_params),
                                   P(C.c_double)]
        L.bps_distill.restype = i32
        L.bps_distill.argtypes = [vp, i64, i64, C.c_double, C.c_double, C.c_int32, vp, i64,
                                  P(i64)]
        L.bps_thresholds.restype = i32
        L.bps_thresholds.argtypes = [P(bps_search_params), i64, i64, vp]
        L.bps_series_update.restype = i32
        L.bps_series_update.argtypes = [vp, i64, vp, i32]
        L.bps_graph_create.restype = i32
        L.bps_graph_create.argtypes = [vp, i64, vp, vp, P(bps_search_params), P(i64)]
        L.bps_graph_launch.restype = i32
        L.bps_graph_launch.argtypes = [vp, i64, vp]
        L.bps_graph_fetch.restype = i32
        L.bps_graph_fetch.argtypes = [vp, i64, i64, vp, i64, P(i64), P(i64)]
        L.bps_selftest_bounded_wait.restype = i32
        L.bps_selftest_bounded_wait.argtypes = [vp, i32, P(i32)]
        L.bps_whiten.restype = i32
        L.bps_whiten.argtypes = [vp, vp, i64, i64, i32, vp, vp, vp]
        L.bps_default_bank_spec.restype = None
        L.bps_default_bank_spec.argtypes = [P(bps_bank_spec)]
        L.bps_metric_density.restype = i32
        L.bps_metric_density.argtypes = [P(bps_bank_spec), vp, i64, vp]
        L.bps_metric_projected.restype = i32
        L.bps_metric_projected.argtypes = [P(bps_bank_spec), vp, vp]
        L.bps_metric_bank.restype = i32
        L.bps_metric_bank.argtypes = [P(bps_bank_spec), C.c_uint64, vp, i64, P(i64),
                                      P(C.c_double), P(C.c_double)]
        _lib = L
    return _lib


def default_params(**kw) -> bps_search_params:
    p = bps_search_params()
    lib().bps_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError("unknown search parameter %r" % k)
        setattr(p, k, v)
    return p


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(int(stream.cuda_stream))


def distill(cands: np.ndarray, n_samples: int, tsamp: float, tol_bins: float = 1.5,
            max_ratio: int = 16) -> np.ndarray:
    """Group repeated / harmonically related detections (bps_distill); returns the group
    leaders, most significant first, with flags = group size."""
    c = np.ascontiguousarray(cands, CAND_DTYPE)
    out = np.zeros(max(1, c.size), CAND_DTYPE)
    n = C.c_int64()
    rc = lib().bps_distill(_np_ptr(c), c.size, int(n_samples), float(tsamp), float(tol_bins),
                           int(max_ratio), _np_ptr(out), out.size, C.byref(n))
    if rc:
        raise BpsError(rc, "bps_distill: invalid arguments")
    return out[:n.value]


def default_bank_spec(**kw) -> bps_bank_spec:
    """Template-bank search region (Table 1 defaults), fields overridden by keyword."""
    sp = bps_bank_spec()
    lib().bps_default_bank_spec(C.byref(sp))
    for k, v in kw.items():
        if not hasattr(sp, k):
            raise TypeError("unknown bank spec field %r" % k)
        setattr(sp, k, v)
    return sp


def _bank_array(bank) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(bank, np.float64).reshape(-1, 5))


def metric_density(spec: bps_bank_spec, bank) -> np.ndarray:
    """sqrt(det) of the frequency-projected metric at each template (K x 5 array)."""
    b = _bank_array(bank)
    out = np.zeros(b.shape[0], np.float64)
    rc = lib().bps_metric_density(C.byref(spec), _np_ptr(b), b.shape[0], _np_ptr(out))
    if rc:
        raise BpsError(rc, "bps_metric_density: invalid spec or template")
    return out


def metric_projected(spec: bps_bank_spec, template) -> np.ndarray:
    """The frequency-projected metric (n x n, n = 3 circular / 5 elliptical) at one template."""
    b = _bank_array(template)
    n = 5 if spec.ecc_max > 0 else 3
    out = np.zeros((n, n), np.float64)
    rc = lib().bps_metric_projected(C.byref(spec), _np_ptr(b), _np_ptr(out))
    if rc:
        raise BpsError(rc, "bps_metric_projected: invalid spec or template")
    return out


def metric_bank(spec: bps_bank_spec, seed: int = 0, cap: int = 1 << 24, count_only=False):
    """Random template bank of the region (bps_metric_bank): returns (bank K x 5 array,
    proper volume, expected template count N_R); count_only skips drawing the bank.  The
    count is computed first (the same seed gives the same volume), then exactly that many
    rows are allocated; more than cap templates raises BPS_ERR_CAND_OVERFLOW."""
    n = C.c_int64()
    vol, nexp = C.c_double(), C.c_double()
    rc = lib().bps_metric_bank(C.byref(spec), int(seed), None, 0, C.byref(n), C.byref(vol),
                               C.byref(nexp))
    if rc:
        raise BpsError(rc, "bps_metric_bank: invalid spec" if rc == BPS_ERR_INVALID_ARG else
                       "bps_metric_bank failed (%d)" % rc)
    if count_only:
        return np.zeros((0, 5), np.float64), vol.value, nexp.value
    if n.value > cap:
        raise BpsError(BPS_ERR_CAND_OVERFLOW, "bps_metric_bank: bank of %d templates exceeds cap %d"
                       % (n.value, cap))
    out = np.zeros((max(1, n.value), 5), np.float64)
    rc = lib().bps_metric_bank(C.byref(spec), int(seed), _np_ptr(out), out.shape[0], C.byref(n),
                               C.byref(vol), C.byref(nexp))
    if rc:
        raise BpsError(rc, "bps_metric_bank failed (%d)" % rc)
    return out[:n.value].copy(), vol.value, nexp.value


def thresholds(params: bps_search_params, n_samples: int, n_templates: int) -> np.ndarray:
    nlev = int(params.nharm_max).bit_length()
    out = np.zeros(5, np.float64)
    rc = lib().bps_thresholds(C.byref(params), int(n_samples), int(n_templates), _np_ptr(out))
    if rc:
        raise BpsError(rc, "invalid search parameters")
    return out[:nlev]


class Context:
    """One library context on one CUDA device (wraps bps_create / bps_destroy)."""

    def __init__(self, device: int = 0):
        h = C.c_void_p()
        rc = lib().bps_create(C.byref(h), int(device))
        if rc:
            raise BpsError(rc, "bps_create(device=%d) failed: no usable CUDA device" % device)
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            lib().bps_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc, what):
        if rc:
            raise BpsError(rc, "%s: %s" % (what, lib().bps_last_error(self.h).decode()))

    # --- residency ------------------------------------------------------------
    def load_series(self, x, tsamp: float, dtype: int = BPS_F32) -> int:
        sid = C.c_int64()
        on_dev = 0
        keep = x
        if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
            if str(x.dtype) != "torch.float32":
                raise TypeError("series tensor must be float32")
            x = x.contiguous()
            keep = x
            if x.is_cuda:
                ptr, on_dev = C.c_void_p(x.data_ptr()), 1
            else:
                ptr = C.c_void_p(x.data_ptr())
            n = x.numel()
        else:
            keep = np.ascontiguousarray(x, np.float32)
            ptr, n = _np_ptr(keep), keep.size
        rc = lib().bps_load_series(self.h, ptr, n, float(tsamp), int(dtype), on_dev, C.byref(sid))
        self._check(rc, "bps_load_series")
        if on_dev and dtype == BPS_F32:
            # borrowed device memory: keep the tensor alive with the id
            self.__dict__.setdefault("_borrowed", {})[sid.value] = keep
        return sid.value

    def update_series(self, series_id: int, x):
        """Replace the samples of a loaded series in place (same length and storage type);
        ids, banks and graphs that use it stay valid."""
        if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
            if str(x.dtype) != "torch.float32":
                raise TypeError("series tensor must be float32")
            x = x.contiguous()
            ptr, on_dev, keep = C.c_void_p(x.data_ptr()), int(bool(x.is_cuda)), x
        else:
            keep = np.ascontiguousarray(x, np.float32)
            ptr, on_dev = _np_ptr(keep), 0
        self._check(lib().bps_series_update(self.h, int(series_id), ptr, on_dev), "bps_series_update")
        del keep

    def load_bank(self, bank) -> int:
        b = np.ascontiguousarray(np.asarray(bank, np.float64).reshape(-1, 5))
        bid = C.c_int64()
        rc = lib().bps_load_bank(self.h, _np_ptr(b), b.shape[0], C.byref(bid))
        self._check(rc, "bps_load_bank")
        return bid.value

    def unload(self, id_: int):
        rc = lib().bps_unload(self.h, int(id_))
        self._check(rc, "bps_unload")
        self.__dict__.get("_borrowed", {}).pop(int(id_), None)

    # --- search ------------------------------------------------------------------
    def search(self, series_id: int, bank_id: int, params: bps_search_params | None = None,
               stream=None) -> int:
        params = params or default_params()
        rid = C.c_int64()
        rc = lib().bps_search(self.h, int(series_id), int(bank_id), C.byref(params),
                              _stream_ptr(stream), C.byref(rid))
        self._check(rc, "bps_search")
        return rid.value

    def query(self, req_id: int) -> bool:
        d = C.c_int32()
        self._check(lib().bps_query(self.h, int(req_id), C.byref(d)), "bps_query")
        return bool(d.value)

    def fetch_candidates(self, req_id: int, cap: int | None = None, allow_overflow=False):
        """Returns (candidates structured array sorted by template, nharm, bin; n_total)."""
        nw, nt = C.c_int64(), C.c_int64()
        rc = lib().bps_fetch_candidates(self.h, int(req_id), None, 0, C.byref(nw), C.byref(nt))
        if rc and not (rc == BPS_ERR_CAND_OVERFLOW and allow_overflow):
            self._check(rc, "bps_fetch_candidates")
        total = nt.value
        n = total if cap is None else min(cap, total)
        out = np.zeros(n, CAND_DTYPE)
        rc = lib().bps_fetch_candidates(self.h, int(req_id), _np_ptr(out) if n else None, n,
                                        C.byref(nw), C.byref(nt))
        if rc and not (rc == BPS_ERR_CAND_OVERFLOW and allow_overflow):
            self._check(rc, "bps_fetch_candidates")
        return out[:nw.value], nt.value

    def autotune(self, series_id: int, bank_id: int, params: bps_search_params | None = None,
                 sample_templates: int = 64):
        """Time the launch shapes on a sample of the bank; returns (best params, ms per
        template).  The context remembers the choice for this series length."""
        params = params or default_params()
        best = bps_search_params()
        ms = C.c_double()
        rc = lib().bps_autotune(self.h, int(series_id), int(bank_id), C.byref(params),
                                int(sample_templates), C.byref(best), C.byref(ms))
        self._check(rc, "bps_autotune")
        return best, ms.value

    # --- CUDA graphs ----------------------------------------------------------------
    def graph_create(self, pairs, params: bps_search_params | None = None) -> int:
        """Capture the searches of [(series_id, bank_id), ...] into one CUDA graph."""
        params = params or default_params()
        sids = np.array([int(p[0]) for p in pairs], np.int64)
        bids = np.array([int(p[1]) for p in pairs], np.int64)
        gid = C.c_int64()
        rc = lib().bps_graph_create(self.h, sids.size, _np_ptr(sids), _np_ptr(bids),
                                    C.byref(params), C.byref(gid))
        self._check(rc, "bps_graph_create")
        return gid.value

    def graph_launch(self, graph_id: int, stream=None):
        self._check(lib().bps_graph_launch(self.h, int(graph_id), _stream_ptr(stream)),
                    "bps_graph_launch")

    def graph_fetch(self, graph_id: int, pair: int, allow_overflow=False):
        """(candidates of pair `pair` from the last replay, sorted as fetch_candidates; n_total)"""
        nw, nt = C.c_int64(), C.c_int64()
        rc = lib().bps_graph_fetch(self.h, int(graph_id), int(pair), None, 0, C.byref(nw),
                                   C.byref(nt))
        if rc and not (rc == BPS_ERR_CAND_OVERFLOW and allow_overflow):
            self._check(rc, "bps_graph_fetch")
        out = np.zeros(nt.value, CAND_DTYPE)
        rc = lib().bps_graph_fetch(self.h, int(graph_id), int(pair), _np_ptr(out) if out.size else None,
                                   out.size, C.byref(nw), C.byref(nt))
        if rc and not (rc == BPS_ERR_CAND_OVERFLOW and allow_overflow):
            self._check(rc, "bps_graph_fetch")
        return out[:nw.value], nt.value

    def selftest_bounded_wait(self, poll_limit: int = 1000) -> bool:
        """Run the bounded-wait self-test kernel; True when its wait expired as designed."""
        t = C.c_int32()
        self._check(lib().bps_selftest_bounded_wait(self.h, int(poll_limit), C.byref(t)),
                    "bps_selftest_bounded_wait")
        return bool(t.value)

    def whiten(self, power, whiten_block: int = 1024, stream=None, out=None):
        """Block-median whitening of caller-provided power spectra on the device
        (bps_whiten): power is a contiguous float32 CUDA tensor of shape (count, nbins)
        or (nbins,); returns (Pw, scale) with scale = ln2 / block median per block.
        out=power whitens in place.  Runs on `stream` (default: the current torch
        stream) and does not wait."""
        import torch
        if not (isinstance(power, torch.Tensor) and power.is_cuda and
                power.dtype == torch.float32 and power.is_contiguous()):
            raise TypeError("power must be a contiguous float32 CUDA tensor")
        pw2 = power.reshape(-1, power.shape[-1])
        count, nbins = pw2.shape
        pw = torch.empty_like(power) if out is None else out
        if not (pw.is_cuda and pw.dtype == torch.float32 and pw.is_contiguous() and
                pw.shape == power.shape):
            raise TypeError("out must match power")
        scale = torch.empty(power.shape[:-1] + (max(nbins // int(whiten_block), 1),),
                            dtype=torch.float32, device=power.device)
        if stream is None:
            stream = torch.cuda.current_stream(power.device)
        rc = lib().bps_whiten(self.h, C.c_void_p(power.data_ptr()), int(count), int(nbins),
                              int(whiten_block), C.c_void_p(pw.data_ptr()),
                              C.c_void_p(scale.data_ptr()), _stream_ptr(stream))
        self._check(rc, "bps_whiten")
        return pw, scale

    def set_profiling(self, on: bool):
        self._check(lib().bps_set_profiling(self.h, int(bool(on))), "bps_set_profiling")

    def request_stats(self, req_id: int) -> dict:
        st = bps_stats()
        self._check(lib().bps_request_stats(self.h, int(req_id), C.byref(st)), "bps_request_stats")
        return {"templates": st.templates, "batch": st.batch, "anchor_block": st.anchor_block,
                "launches": st.launches, "profiled": bool(st.profiled),
                "stage_launches": {STAGES[i]: st.stage_launches[i] for i in range(6)},
                "stage_ms": {STAGES[i]: float(st.stage_ms[i]) for i in range(6)}}

    # --- stage entry points --------------------------------------------------------
    def index_map(self, series_id: int, bank_id: int, template_idx: int, n: int):
        out = np.empty(n, np.int32)
        npre = C.c_int64()
        rc = lib().bps_index_map(self.h, int(series_id), int(bank_id), int(template_idx),
                                 _np_ptr(out), C.byref(npre))
        self._check(rc, "bps_index_map")
        return out, npre.value

    def whitened_spectrum(self, series_id: int, bank_id: int, t0: int, count: int, n: int,
                          params: bps_search_params | None = None):
        params = params or default_params()
        out = np.empty((count, n // 2), np.float32)
        rc = lib().bps_whitened_spectrum(self.h, int(series_id), int(bank_id), int(t0),
                                         int(count), C.byref(params), _np_ptr(out))
        self._check(rc, "bps_whitened_spectrum")
        return out

    def harmonic_sums(self, series_id: int, bank_id: int, template_idx: int, n: int,
                      params: bps_search_params | None = None):
        params = params or default_params()
        nlev = int(params.nharm_max).bit_length()
        out = np.empty((nlev, n // 2), np.float32)
        rc = lib().bps_harmonic_sums(self.h, int(series_id), int(bank_id), int(template_idx),
                                     C.byref(params), _np_ptr(out))
        self._check(rc, "bps_harmonic_sums")
        return out


class Server:
    """Continuously batched request loop on one context (bps_server_*): submit() returns
    a ticket at once; result() waits for it and returns (candidates, n_total, latency_s)."""

    def __init__(self, ctx: Context, max_active: int = 4, groups_in_flight: int = 2,
                 hbm_budget: int = 0):
        cfg = bps_server_config(max_active, groups_in_flight, hbm_budget)
        h = C.c_void_p()
        rc = lib().bps_server_create(ctx.h, C.byref(cfg), C.byref(h))
        if rc:
            raise BpsError(rc, "bps_server_create: %s" % lib().bps_last_error(ctx.h).decode())
        self.h = h
        self.ctx = ctx

    def close(self):
        if getattr(self, "h", None):
            lib().bps_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc, what, ok=()):
        if rc and rc not in ok:
            raise BpsError(rc, "%s: %s" % (what, lib().bps_server_last_error(self.h).decode()))

    def submit(self, series, tsamp: float, bank, params: bps_search_params | None = None,
               dtype: int = BPS_F32) -> int:
        params = params or default_params()
        x = np.ascontiguousarray(series, np.float32)
        b = np.ascontiguousarray(np.asarray(bank, np.float64).reshape(-1, 5))
        t = C.c_int64()
        rc = lib().bps_server_submit(self.h, _np_ptr(x), x.size, float(tsamp), int(dtype),
                                     _np_ptr(b), b.shape[0], C.byref(params), C.byref(t))
        self._check(rc, "bps_server_submit")
        return t.value

    def load_series(self, series, tsamp: float, dtype: int = BPS_F32) -> int:
        """Put a series into the server's resident store; returns its server series id."""
        x = np.ascontiguousarray(series, np.float32)
        sid = C.c_int64()
        self._check(lib().bps_server_load_series(self.h, _np_ptr(x), x.size, float(tsamp),
                                                 int(dtype), C.byref(sid)),
                    "bps_server_load_series")
        return sid.value

    def submit_series(self, series_id: int, bank, params: bps_search_params | None = None) -> int:
        """Submit a search over a resident series; returns a ticket."""
        params = params or default_params()
        b = np.ascontiguousarray(np.asarray(bank, np.float64).reshape(-1, 5))
        t = C.c_int64()
        self._check(lib().bps_server_submit_series(self.h, int(series_id), _np_ptr(b), b.shape[0],
                                                   C.byref(params), C.byref(t)),
                    "bps_server_submit_series")
        return t.value

    def unload_series(self, series_id: int):
        self._check(lib().bps_server_unload_series(self.h, int(series_id)), "bps_server_unload_series")

    def series_info(self, series_id: int) -> dict:
        r, n = C.c_int32(), C.c_int64()
        self._check(lib().bps_server_series_info(self.h, int(series_id), C.byref(r), C.byref(n)),
                    "bps_server_series_info")
        return {"resident": bool(r.value), "times_staged": n.value}

    def result(self, ticket: int, timeout_ms: int = -1, allow_overflow=False):
        nw, nt, lat = C.c_int64(), C.c_int64(), C.c_double()
        rc = lib().bps_server_result(self.h, int(ticket), int(timeout_ms), None, 0, C.byref(nw),
                                     C.byref(nt), C.byref(lat))
        if rc == BPS_ERR_NOT_READY:
            return None
        self._check(rc, "bps_server_result", ok=(BPS_ERR_CAND_OVERFLOW,) if allow_overflow else ())
        out = np.zeros(max(1, nt.value), CAND_DTYPE)
        rc = lib().bps_server_result(self.h, int(ticket), 0, _np_ptr(out), out.size, C.byref(nw),
                                     C.byref(nt), C.byref(lat))
        self._check(rc, "bps_server_result", ok=(BPS_ERR_CAND_OVERFLOW,) if allow_overflow else ())
        return out[:nw.value], nt.value, lat.value

    def stats(self) -> dict:
        q, a, f, by = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        self._check(lib().bps_server_stats(self.h, C.byref(q), C.byref(a), C.byref(f), C.byref(by)),
                    "bps_server_stats")
        return {"queued": q.value, "active": a.value, "finished": f.value, "bytes_held": by.value}


def __getattr__(name):
    """The C entry points under their own names (``bps.bps_search(...)`` and so on):
    module attributes that resolve to the library's typed ctypes functions."""
    if name in EXPORTED:
        return getattr(lib(), name)
    raise AttributeError("module %r has no attribute %r" % (__name__, name))


__all__ = ["Context", "Server", "distill", "bps_server_config", "bps_bank_spec",
           "default_bank_spec", "metric_density", "metric_projected", "metric_bank", "BpsError", "default_params", "thresholds", "CAND_DTYPE", "EXPORTED",
           "STAGES", "bps_template", "bps_candidate", "bps_search_params", "bps_stats"] + [
    n for n in dir() if n.startswith("BPS_")]
