"""GPU parity at the full sizes, in the launch configuration bench.py times.

* HTRU-like circular search, 2^23 samples x 4096 templates (the benchmark
  workload, default batch and tiles): the whole bank is searched on the GPU and
  a sample of templates (the three true orbits and two random ones) is checked
  against the FP64 oracle, candidate by candidate, on the GPU's validated index
  maps; the three true orbits are also checked end to end, against the oracle on
  its own index maps (samples rounded differently counted, the power and
  candidate deviations they allow bounded); each injected pulsar is found under
  its true orbit at round(n T / P) for some harmonic level n.
* 2^24 samples (8192-point column FFTs): whitened spectrum of one template.
* 2^25 samples, the largest size (elliptical IMBH workload shape): whitened
  spectrum and candidates of the two true orbits and one random template; the same
  with FP16 series storage against the oracle's FP32-series result.
Tolerances: tests/gpu_common.py.
"""
import numpy as np
import pytest

import synth
from gpu_common import PW_TOL, compare_candidates, end_to_end_leg, oracle_on_gpu_maps, pw_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bps():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_11991_b300 import build
    build.build()
    import paper_2112_11991_b300 as m
    return m


@pytest.fixture(scope="module")
def ctx(bps):
    c = bps.Context(0)
    yield c
    c.close()


def _recovered(cands, T, period, thr):
    """True when some level n has its strongest candidate within one bin of
    round(n T / P) and above threshold."""
    for L, n in enumerate([1, 2, 4, 8, 16]):
        c = cands[cands["nharm"] == n]
        if c.size == 0:
            continue
        best = c[np.argmax(c["power"])]
        if abs(int(best["bin"]) - round(n * T / period)) <= 1 and best["power"] >= thr[L]:
            return True
    return False


def test_htru_2p23_full_bank_sampled(bps, ctx, orc):
    """The whole 2^23 x 4096 request in the launch configuration the benchmark times: the
    autotuner's choice on a 64-template sample (four-step split, tiles, batch -- and with
    them the power layout), which later searches of this size use."""
    w = synth.htru_circular()
    sid = ctx.load_series(w.series, w.tsamp)
    bid = ctx.load_bank(w.bank)
    prm = bps.default_params(cand_cap=1 << 24)
    best, _ = ctx.autotune(sid, bid, prm, sample_templates=64)
    print("\n[shape] 2^23 autotuned: C = 2^%d, tiles %d/%d, batch %d"
          % (best.log_cols, best.log_tile, best.log_tile2, best.batch))
    gc, total = ctx.fetch_candidates(ctx.search(sid, bid, prm))
    assert total == gc.size
    thr = bps.thresholds(prm, w.n, w.bank.shape[0])
    rng = np.random.default_rng(5)
    others = [int(t) for t in rng.choice(np.setdiff1d(np.arange(w.bank.shape[0]), w.true_idx), 2,
                                         replace=False)]
    sample = list(w.true_idx) + others
    sub = w.bank[sample]
    sbid = ctx.load_bank(sub)
    oc, res = oracle_on_gpu_maps(ctx, orc, sid, sbid, w.series, w.tsamp, sub)
    # relabel the oracle's template indices (0..4 in the sub-bank) to bank indices
    oc["template_idx"] = np.array(sample)[oc["template_idx"]]
    g_sub = gc[np.isin(gc["template_idx"], sample)]
    matched, excused = compare_candidates(g_sub, oc, thr)
    print("\n[parity] 2^23 GPU-map leg: %d candidates matched, %d excused at the threshold"
          % (matched, excused))
    # end to end: the oracle on its own index map for the three true orbits
    for i, ti in enumerate(w.true_idx):
        pw = ctx.whitened_spectrum(sid, bid, int(ti), 1, w.n, prm)[0]
        r = end_to_end_leg(orc, w.series, w.tsamp, w.bank[ti], res[i]["idx_gpu"], pw,
                           gc[gc["template_idx"] == ti], thr)
        print("[parity] 2^23 end-to-end leg, template %d: %s" % (ti, r))
    T = w.n * w.tsamp
    for ti, p in zip(w.true_idx, w.pulsars):
        assert _recovered(gc[gc["template_idx"] == ti], T, p.period_s, thr), ti


def test_2p24_whitened_spectrum(bps, ctx, orc):
    n, ts = 1 << 24, 64e-6
    p = synth.Pulsar(period_s=0.03, porb_s=6000.0, tau_lts=1.5, phi_rad=0.7, amp=0.05)
    x = synth.inject(synth.noise(n, 24), ts, p)
    sid = ctx.load_series(x, ts)
    bid = ctx.load_bank(np.array([p.orbit()]))
    pw = ctx.whitened_spectrum(sid, bid, 0, 1, n)
    _, res = oracle_on_gpu_maps(ctx, orc, sid, bid, x, ts, np.array([p.orbit()]),
                                want_arrays=True)
    e = pw_close(pw[0], res[0]["Pw"])
    print("\n[error] 2^24 FP32 whitened power vs FP64 oracle: %.3g" % e)
    assert e <= PW_TOL
    ctx.unload(sid)
    ctx.unload(bid)


def test_max_size_2p25_elliptical(bps, ctx, orc):
    w = synth.elliptical_imbh(K=3)
    sid = ctx.load_series(w.series, w.tsamp)
    bid = ctx.load_bank(w.bank)
    prm = bps.default_params()
    gc, _ = ctx.fetch_candidates(ctx.search(sid, bid, prm))
    pw = ctx.whitened_spectrum(sid, bid, 0, 1, w.n)
    oc, res = oracle_on_gpu_maps(ctx, orc, sid, bid, w.series, w.tsamp, w.bank,
                                 want_arrays=False)
    r0 = orc.search_template(w.series, w.tsamp, w.bank[0], want_arrays=True,
                             idx_in=ctx.index_map(sid, bid, 0, w.n)[0].astype(np.int64))
    e32 = pw_close(pw[0], r0["Pw"])
    print("\n[error] 2^25 FP32 whitened power vs FP64 oracle: %.3g" % e32)
    assert e32 <= PW_TOL
    compare_candidates(gc, oc, bps.thresholds(prm, w.n, w.bank.shape[0]))
    T = w.n * w.tsamp
    for ti, p in zip(w.true_idx, w.pulsars):
        assert _recovered(gc[gc["template_idx"] == ti], T, p.period_s,
                          bps.thresholds(prm, w.n, 3)), ti
    # the same search with FP16 series storage (scale per 4096 samples, FP32 FFT):
    # whitened power within 5e-3 of the FP64 oracle on the FP32 series, the strongest bin
    # of every harmonic level unchanged, each injected pulsar still found
    s16 = ctx.load_series(w.series, w.tsamp, dtype=bps.BPS_F16_SCALED)
    pw16 = ctx.whitened_spectrum(s16, bid, 0, 1, w.n)[0]
    err = np.abs(pw16 - r0["Pw"]) / np.maximum(1.0, r0["Pw"])
    print("[error] 2^25 FP16-storage whitened power vs FP64 oracle: %.3g" % err.max())
    assert err.max() < 5e-3, err.max()
    S16 = ctx.harmonic_sums(s16, bid, 0, w.n)
    sig = [float(np.max(np.abs(S16[L] - r0["S"][L]) / ((1 << L) + r0["S"][L]))) for L in range(5)]
    print("[error] 2^25 FP16-storage harmonic sums vs FP64 oracle, |dS|/(n+S) per level: %s"
          % ", ".join("%.2g" % v for v in sig))
    for L in range(5):
        assert int(np.argmax(S16[L])) == int(np.argmax(r0["S"][L]))
    g16, _ = ctx.fetch_candidates(ctx.search(s16, bid, prm))
    for ti, p in zip(w.true_idx, w.pulsars):
        assert _recovered(g16[g16["template_idx"] == ti], T, p.period_s,
                          bps.thresholds(prm, w.n, 3)), ti
    ctx.unload(s16)
    ctx.unload(sid)
    ctx.unload(bid)
