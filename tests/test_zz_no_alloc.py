"""The allocation-free entry point bps_whitened_spectrum_noalloc.

It exists for callers that must not allocate device memory while they run
(real-time back ends with all GPU memory reserved up front, or frameworks
whose own allocator owns the device memory): it runs the whitened-spectrum
kernels for one template with a fixed scratch array inside the library.  These
tests call it through the C ABI twice in a row, on device buffers they own,
and check each result against the ordinary bps_whitened_spectrum entry point
within the power tolerance the parity tests use -- at the documented largest
size (2^20 samples), with a whitening block above 1024 (the other median
kernel), and once from a fresh process that never creates a library context.
The file name makes pytest collect it last."""
import ctypes as C
import os
import subprocess
import sys

import numpy as np
import pytest

import synth
from gpu_common import PW_TOL

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TEMPLATES = [(90.0, 0.1, 0.3, 0.0, 0.0), (60.0, 0.3, 4.0, 2.0, 0.2)]


def _series(n):
    p = synth.Pulsar(period_s=0.02, porb_s=90.0, tau_lts=0.1, phi_rad=0.3, amp=0.5)
    return synth.inject(synth.noise(n, 91), 64e-6, p)


def _reference(bps, x, W):
    with bps.Context(0) as ctx:
        sid = ctx.load_series(x, 64e-6)
        bid = ctx.load_bank(np.array(TEMPLATES))
        return ctx.whitened_spectrum(sid, bid, 0, len(TEMPLATES), x.size,
                                     bps.default_params(whiten_block=W))


def _noalloc_twice(bps, x, W):
    """The entry point on each template in turn (two calls in a row), through ctypes."""
    import torch
    n = x.size
    xd = torch.from_numpy(x).cuda()
    out = torch.empty(n // 2, dtype=torch.float32, device="cuda")
    fill = float(np.mean(x, dtype=np.float64))
    stream = torch.cuda.current_stream()
    L = bps.lib()
    got = []
    for tm in TEMPLATES:
        t = bps.bps_template(*tm)
        out.fill_(float("nan"))
        rc = L.bps_whitened_spectrum_noalloc(C.c_void_p(xd.data_ptr()), n, 64e-6, fill,
                                             C.byref(t), W, C.c_void_p(out.data_ptr()),
                                             C.c_void_p(stream.cuda_stream))
        assert rc == bps.BPS_OK, rc
        torch.cuda.synchronize()
        got.append(out.cpu().numpy().copy())
    return got


@pytest.fixture(scope="module")
def bps():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_11991_b300 import build
    build.build()
    import paper_2112_11991_b300 as m
    return m


@pytest.mark.parametrize("logn,W", [(18, 1024), (20, 1024), (16, 4096)])
def test_noalloc_matches_whitened_spectrum_twice(bps, logn, W):
    x = _series(1 << logn)
    got = _noalloc_twice(bps, x, W)
    ref = _reference(bps, x, W)
    for call in range(len(TEMPLATES)):
        err = np.max(np.abs(got[call].astype(np.float64) - ref[call]) / np.maximum(1.0, ref[call]))
        assert err <= PW_TOL, (logn, W, call, err)


def test_noalloc_rejects_beyond_the_scratch(bps):
    import torch
    x = torch.zeros(1 << 12, dtype=torch.float32, device="cuda")
    out = torch.empty(1 << 11, dtype=torch.float32, device="cuda")
    t = bps.bps_template(*TEMPLATES[0])
    L = bps.lib()
    for n in (1 << 21, 1 << 40, 1 << 62):
        assert L.bps_whitened_spectrum_noalloc(C.c_void_p(x.data_ptr()), n, 64e-6, 0.0,
                                               C.byref(t), 1024, C.c_void_p(out.data_ptr()),
                                               None) == bps.BPS_ERR_UNSUPPORTED
    for n in (3000, (1 << 62) + 1, -4):
        assert L.bps_whitened_spectrum_noalloc(C.c_void_p(x.data_ptr()), n, 64e-6, 0.0,
                                               C.byref(t), 1024, C.c_void_p(out.data_ptr()),
                                               None) == bps.BPS_ERR_INVALID_ARG


_CHILD = r"""
import sys, numpy as np
sys.path.insert(0, sys.argv[1])
import test_zz_no_alloc as T
import paper_2112_11991_b300 as bps
got = T._noalloc_twice(bps, T._series(1 << 17), 1024)
np.save(sys.argv[2], np.stack(got))
"""


def test_noalloc_in_a_fresh_process_without_context(bps, tmp_path):
    """No library context exists in the child process before (or during) the calls."""
    out = str(tmp_path / "pw.npy")
    env = dict(os.environ)
    env["PYTHONPATH"] = os.pathsep.join([ROOT, os.path.join(ROOT, "tests"),
                                         env.get("PYTHONPATH", "")])
    subprocess.run([sys.executable, "-c", _CHILD, os.path.join(ROOT, "tests"), out],
                   check=True, env=env, timeout=600)
    got = np.load(out)
    x = _series(1 << 17)
    ref = _reference(bps, x, 1024)
    for call in range(len(TEMPLATES)):
        err = np.max(np.abs(got[call].astype(np.float64) - ref[call]) / np.maximum(1.0, ref[call]))
        assert err <= PW_TOL, (call, err)
