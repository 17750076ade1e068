"""CPU checks of the C-ABI library: it builds, loads, exports every entry point
declared in include/bps.h, and its host-side logic (defaults, thresholds,
argument checks) is right.  No compute call needs a GPU here."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bps():
    from paper_2112_11991_b300 import build
    build.build()
    import paper_2112_11991_b300 as m
    m.lib()
    return m


def _declared():
    src = open(os.path.join(ROOT, "include", "bps.h")).read()
    return sorted(set(re.findall(r"\b(bps_[a-z_0-9]+)\s*\(", src)))


def test_header_symbols_exported(bps):
    L = bps.lib()
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(L, n), n
    assert sorted(bps.EXPORTED) == names


def test_struct_layouts(bps):
    assert C.sizeof(bps.bps_candidate) == 16
    assert C.sizeof(bps.bps_template) == 40
    # bps_search_params as include/bps.h lays it out: eleven int32 fields, one double
    # and one int64 (at offsets 8 and 24) -> 64 bytes (bps_default_params writes them all)
    assert C.sizeof(bps.bps_search_params) == 64
    assert bps.bps_search_params.sigma_thr.offset == 8
    assert bps.bps_search_params.cand_cap.offset == 24
    assert bps.bps_search_params.pass2_kind.offset == 60
    assert bps.CAND_DTYPE.itemsize == 16


def test_default_params(bps):
    p = bps.default_params()
    assert (p.nharm_max, p.whiten_block, p.sigma_thr, p.mode, p.batch) == (16, 1024, 6.0, 0, 0)
    assert p.cand_cap == 1 << 20


def test_thresholds_match_oracle(bps, orc):
    for sigma in [4.0, 6.0, 7.5]:
        p = bps.default_params(sigma_thr=sigma)
        got = bps.thresholds(p, 1 << 20, 32)
        ref = orc.thresholds(5, sigma)
        assert np.max(np.abs(got - ref) / ref) < 1e-10


def test_auto_threshold_uses_snmin(bps, orc):
    p = bps.default_params(auto_thr=1)
    n, K = 1 << 23, 4096
    got = bps.thresholds(p, n, K)
    sigma = orc.snmin((n // 2) * 5 * K)
    ref = orc.thresholds(5, sigma)
    assert np.max(np.abs(got - ref) / ref) < 1e-10


def test_threshold_argument_checks(bps):
    for kw in [dict(nharm_max=3), dict(whiten_block=1000), dict(whiten_block=16),
               dict(sigma_thr=-1.0), dict(cand_cap=0), dict(mode=7), dict(pass1_kind=4),
               dict(pass2_kind=3), dict(power_layout=3), dict(log_tile=12)]:
        p = bps.default_params(**kw)
        with pytest.raises(bps.BpsError):
            bps.thresholds(p, 1 << 20, 1)


def test_create_without_device_fails_loudly(bps):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(bps.BpsError):
        bps.Context(0)


def test_oracle_not_imported_by_package():
    """The product path never imports, links or runs the oracle."""
    pkg = os.path.join(ROOT, "paper_2112_11991_b300")
    pat = re.compile(r"^\s*(import|from)\s+oracle\b|_bps_oracle|bps_oracle\.c", re.M)
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                assert not pat.search(open(os.path.join(dirpath, f)).read()), f


def test_c_names_resolve_to_library_functions(bps):
    """The binding offers every entry point under its C name (argument marshalling only)."""
    L = bps.lib()
    for n in bps.EXPORTED:
        assert getattr(bps, n) is getattr(L, n), n
    p = bps.bps_search_params()
    bps.bps_default_params(C.byref(p))
    assert p.nharm_max == 16
    with pytest.raises(AttributeError):
        bps.bps_no_such_call
