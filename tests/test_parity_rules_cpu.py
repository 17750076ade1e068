"""CPU check of the end-to-end parity leg's deviation bound (tests/gpu_common.py).

A map that rounds some samples differently from the oracle's own (here: five samples
moved by one, standing in for the GPU's admissible roundings near a half-integer
offset) changes the whitened power and the candidates.  The bound the end-to-end leg
asserts -- every DFT bin moves by at most the summed change of the resampled samples,
the block median by at most its block's largest power change -- must hold for the
oracle's own spectra of the two maps, with no tolerance to spare."""
import numpy as np

import synth
from gpu_common import end_to_end_leg


def test_end_to_end_bound_holds_for_moved_samples(orc):
    n, ts = 1 << 16, 64e-6
    p = synth.Pulsar(period_s=0.02, porb_s=60.0, tau_lts=0.05, phi_rad=1.0, amp=0.4)
    x = synth.inject(synth.noise(n, 21), ts, p)
    tmpl = p.orbit()
    idx, _, _ = orc.index_map(tmpl, n, ts)
    moved = idx.copy()
    rng = np.random.default_rng(4)
    pos = rng.choice(n, 5, replace=False)
    moved[pos] += rng.choice([-1, 1], 5)
    thr = orc.thresholds(5, 4.0)
    r = orc.search_template(x, ts, tmpl, idx_in=moved, want_arrays=True, sigma=4.0)
    gc = r["cands"].copy()
    out = end_to_end_leg(orc, x, ts, tmpl, moved, r["Pw"].astype(np.float32), gc, thr,
                         W=1024, require_near=False)
    assert out["samples_rounded_differently"] == 5
    assert 0.0 < out["max_pw_dev"] <= out["max_pw_bound"]
    assert out["candidates_common"] > 0
