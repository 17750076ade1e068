"""The allocation-free entry point bps_whitened_spectrum_noalloc.

It exists for callers that must not allocate device memory while they run
(real-time back ends with all GPU memory reserved up front, or frameworks
whose own allocator owns the device memory): it runs the whitened-spectrum
kernels for one template with a fixed scratch array inside the library.  This
test calls it through the C ABI twice in a row, on device buffers it owns,
and checks each result against the ordinary bps_whitened_spectrum entry point
within the power tolerance the parity tests use.  The file name makes pytest
collect it last."""
import ctypes as C

import numpy as np
import pytest

import synth
from gpu_common import PW_TOL

pytestmark = pytest.mark.gpu


def test_noalloc_matches_whitened_spectrum_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_11991_b300 import build
    build.build()
    import paper_2112_11991_b300 as bps

    n, ts = 1 << 18, 64e-6
    p = synth.Pulsar(period_s=0.02, porb_s=90.0, tau_lts=0.1, phi_rad=0.3, amp=0.5)
    x = synth.inject(synth.noise(n, 91), ts, p)
    tms = [p.orbit(), (60.0, 0.3, 4.0, 2.0, 0.2)]
    W = 1024
    xd = torch.from_numpy(x).cuda()
    out = torch.empty(n // 2, dtype=torch.float32, device="cuda")
    fill = float(np.mean(x, dtype=np.float64))
    stream = torch.cuda.current_stream()
    with bps.Context(0) as ctx:
        sid = ctx.load_series(x, ts)
        bid = ctx.load_bank(np.array(tms))
        ref = ctx.whitened_spectrum(sid, bid, 0, len(tms), n, bps.default_params(whiten_block=W))
    L = bps.lib()
    for call, tm in enumerate(tms):
        t = bps.bps_template(*tm)
        out.fill_(float("nan"))
        rc = L.bps_whitened_spectrum_noalloc(C.c_void_p(xd.data_ptr()), n, ts, fill, C.byref(t),
                                             W, C.c_void_p(out.data_ptr()),
                                             C.c_void_p(stream.cuda_stream))
        assert rc == bps.BPS_OK, rc
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        err = np.max(np.abs(got.astype(np.float64) - ref[call]) / np.maximum(1.0, ref[call]))
        assert err <= PW_TOL, (call, err)
    big = bps.bps_template(*tms[0])
    assert L.bps_whitened_spectrum_noalloc(C.c_void_p(xd.data_ptr()), 1 << 21, ts, fill,
                                           C.byref(big), W, C.c_void_p(out.data_ptr()),
                                           None) == bps.BPS_ERR_UNSUPPORTED
