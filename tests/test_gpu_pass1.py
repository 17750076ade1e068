"""Pass-1 organisations and power layouts against the FP64 oracle.

* The warp-specialised pass 1 (producer warps run Algorithm 1's index map and gather
  into one shared-memory tile while consumer warps run the column FFTs of the other)
  gives the oracle's whitened power and candidates for every column length it is built
  for (R = 2^10, 2^11, 2^12) from 2^21 to 2^25 samples, with FP32 and FP16 series
  storage, and for batches whose tiles outnumber the CTAs (each CTA walks many tiles
  through its two buffers).
* The one-phase pass 1 with asynchronous gathers (2^13 tiles, two CTAs per SM) gives the
  oracle's whitened power and candidates for its splits, batched as well as per template;
  FP16 series, which it does not take, run the one-phase kernel with the same results.
* The TMA-fed pass 2 (one thread copies the next tile's rows into shared memory with
  bulk copies while the consumer warps transform the current tile) gives the oracle's
  whitened power and candidates for its splits (R, C in 2^10..2^12), alone and combined
  with the warp-specialised pass 1, in both power layouts, and over batches whose tiles
  outnumber the CTAs.
* The two power layouts of pass 2 (bins in order, or row-major blocks of 8 columns that
  the whitening kernel transposes) give bit-identical whitened spectra and candidates,
  at the smallest sizes where a pass-2 CTA holds one or two row pairs.
Tolerances: tests/gpu_common.py.
"""
import numpy as np
import pytest

import synth
from gpu_common import F16_TOL, PW_TOL, compare_candidates, oracle_on_gpu_maps, pw_close

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


def _workload(logn, seed, K=2, ecc=False):
    n, ts = 1 << logn, 64e-6
    T = n * ts
    p = synth.Pulsar(period_s=0.021, porb_s=5 * T, tau_lts=0.08, phi_rad=1.3,
                     omega_rad=0.7 if ecc else 0.0, ecc=0.06 if ecc else 0.0, amp=0.3)
    x = synth.inject(synth.noise(n, seed), ts, p)
    others = [(7 * T, 0.05, 2.2, 1.0 if ecc else 0.0, 0.03 if ecc else 0.0),
              (4 * T, 0.2, 4.1, 0.0, 0.0), (9 * T, 0.01, 0.4, 0.0, 0.0)]
    bank = np.array([p.orbit()] + others[:K - 1])
    return x, ts, bank


@pytest.mark.parametrize("logn,log_cols", [(21, 10), (21, 9), (22, 10), (22, 11), (23, 12),
                                           (23, 11), (23, 10), (24, 12), (24, 11)])
def test_warpspec_pass1_against_oracle(bps, ctx, orc, logn, log_cols):
    x, ts, bank = _workload(logn, 4000 + logn + log_cols, K=2 if logn <= 23 else 1,
                            ecc=(log_cols % 2 == 0))
    n = x.size
    sid = ctx.load_series(x, ts)
    bid = ctx.load_bank(bank)
    prm = bps.default_params(log_cols=log_cols, sigma_thr=5.0,
                             pass1_kind=bps.BPS_PASS1_WARPSPEC)
    pw = ctx.whitened_spectrum(sid, bid, 0, len(bank), n, prm)
    gc, _ = ctx.fetch_candidates(ctx.search(sid, bid, prm))
    oc, res = oracle_on_gpu_maps(ctx, orc, sid, bid, x, ts, bank, want_arrays=True, sigma=5.0)
    for t in range(len(bank)):
        e = pw_close(pw[t], res[t]["Pw"])
        assert e <= PW_TOL, (t, e)
    compare_candidates(gc, oc, bps.thresholds(prm, n, len(bank)))
    ctx.unload(sid)
    ctx.unload(bid)


def test_warpspec_pass1_max_size_and_fp16(bps, ctx, orc):
    """2^25 samples (R = C = 4096) with FP32 storage against the oracle, and FP16 storage
    against the oracle on the FP32 series at the FP16 tolerance."""
    x, ts, bank = _workload(25, 4100, K=1)
    n = x.size
    bid = ctx.load_bank(bank)
    prm = bps.default_params(log_cols=12, sigma_thr=5.0, pass1_kind=bps.BPS_PASS1_WARPSPEC)
    s32 = ctx.load_series(x, ts)
    pw = ctx.whitened_spectrum(s32, bid, 0, 1, n, prm)[0]
    oc, res = oracle_on_gpu_maps(ctx, orc, s32, bid, x, ts, bank, want_arrays=True, sigma=5.0)
    assert pw_close(pw, res[0]["Pw"]) <= PW_TOL
    gc, _ = ctx.fetch_candidates(ctx.search(s32, bid, prm))
    compare_candidates(gc, oc, bps.thresholds(prm, n, 1))
    s16 = ctx.load_series(x, ts, dtype=bps.BPS_F16_SCALED)
    pw16 = ctx.whitened_spectrum(s16, bid, 0, 1, n, prm)[0]
    e16 = pw_close(pw16, res[0]["Pw"])
    print("\n[error] 2^25 warp-specialised pass 1, FP16 storage, whitened power vs oracle: %.3g" % e16)
    assert e16 <= F16_TOL
    g16, _ = ctx.fetch_candidates(ctx.search(s16, bid, prm))
    compare_candidates(g16, oc, bps.thresholds(prm, n, 1), tol=F16_TOL)
    for i in (s32, s16, bid):
        ctx.unload(i)


def test_warpspec_pass1_many_tiles_per_cta(bps, ctx, orc):
    """24 templates of 2^21 samples at R = 2^10 (8 columns per tile): 24 x 128 tiles over
    at most one CTA per SM, so every CTA reuses both buffers many times; the batched
    search equals one template per launch and the oracle on sampled templates."""
    logn = 21
    n, ts = 1 << logn, 64e-6
    T = n * ts
    x, _, _ = _workload(logn, 4200)
    bank, where = synth.uniform_bank(24, 4201, (3 * T, 10 * T), (0.0, 0.3), ecc=(0.0, 0.1))
    sid = ctx.load_series(x, ts)
    bid = ctx.load_bank(bank)
    res = {}
    for batch in (24, 1, 7):
        prm = bps.default_params(log_cols=10, batch=batch, sigma_thr=4.5,
                                 pass1_kind=bps.BPS_PASS1_WARPSPEC)
        res[batch] = ctx.fetch_candidates(ctx.search(sid, bid, prm))[0]
    assert np.array_equal(res[24], res[1]) and np.array_equal(res[7], res[1])
    assert res[1].size > 0
    sample = [0, 11, 23]
    sbid = ctx.load_bank(bank[sample])
    oc, _ = oracle_on_gpu_maps(ctx, orc, sid, sbid, x, ts, bank[sample], sigma=4.5)
    oc["template_idx"] = np.array(sample)[oc["template_idx"]]
    prm = bps.default_params(log_cols=10, sigma_thr=4.5)
    compare_candidates(res[24][np.isin(res[24]["template_idx"], sample)], oc,
                       bps.thresholds(prm, n, 24))
    for i in (sid, bid, sbid):
        ctx.unload(i)


def test_warpspec_pass1_rejected_where_not_built(bps, ctx):
    x, ts, bank = _workload(16, 4300)
    sid = ctx.load_series(x, ts)
    bid = ctx.load_bank(bank)
    with pytest.raises(bps.BpsError) as e:
        ctx.search(sid, bid, bps.default_params(pass1_kind=bps.BPS_PASS1_WARPSPEC))
    assert e.value.code == bps.BPS_ERR_INVALID_ARG
    with pytest.raises(bps.BpsError):
        ctx.search(sid, bid, bps.default_params(pass1_kind=7))
    ctx.unload(sid)
    ctx.unload(bid)


@pytest.mark.parametrize("logn,log_cols,tile2,W", [(17, 11, 13, 32), (18, 12, 13, 32),
                                                   (18, 12, 14, 32), (19, 12, 13, 64),
                                                   (20, 11, 13, 256), (22, 11, 13, 1024)])
def test_power_layouts_identical(bps, ctx, orc, logn, log_cols, tile2, W):
    """Row-major power (the whitening kernel transposes blocks of 8 columns x W rows) and
    bin-order power give the same bits, where a pass-2 CTA holds NP = 2 (C = 2048,
    2^13 tiles; C = 4096, 2^14 tiles) or NP = 1 (C = 4096, 2^13 tiles) row pairs; the
    smallest series with those splits (R = 32 rows at C = 2048 and 4096) and whitening
    blocks from 32 bins up to all of a column's rows.  The medians are the oracle's on the same spectra
    (whitening is bit-exact, tests/test_gpu_whiten.py), checked here through the
    candidates against the oracle."""
    x, ts, bank = _workload(logn, 4400 + logn + W)
    n = x.size
    sid = ctx.load_series(x, ts)
    bid = ctx.load_bank(bank)
    out = {}
    for layout in (bps.BPS_POWER_BINS, bps.BPS_POWER_ROWS):
        prm = bps.default_params(log_cols=log_cols, log_tile2=tile2, whiten_block=W,
                                 sigma_thr=4.5, power_layout=layout)
        out[layout] = (ctx.whitened_spectrum(sid, bid, 0, len(bank), n, prm),
                       ctx.fetch_candidates(ctx.search(sid, bid, prm))[0])
    a, b = out[bps.BPS_POWER_BINS], out[bps.BPS_POWER_ROWS]
    assert np.array_equal(a[0].view(np.uint32), b[0].view(np.uint32))
    assert np.array_equal(a[1], b[1])
    oc, res = oracle_on_gpu_maps(ctx, orc, sid, bid, x, ts, bank, want_arrays=True, sigma=4.5,
                                 whiten_block=W)
    for t in range(len(bank)):
        assert pw_close(b[0][t], res[t]["Pw"]) <= PW_TOL
    compare_candidates(b[1], oc, bps.thresholds(prm, n, len(bank)))
    ctx.unload(sid)
    ctx.unload(bid)


def test_power_rows_rejected_where_not_possible(bps, ctx):
    x, ts, bank = _workload(18, 4500)
    sid = ctx.load_series(x, ts)
    bid = ctx.load_bank(bank)
    with pytest.raises(bps.BpsError):  # C = 512, 2^13 tiles: 8 row pairs per pass-2 CTA
        ctx.search(sid, bid, bps.default_params(log_cols=9, power_layout=bps.BPS_POWER_ROWS))
    ctx.unload(sid)
    ctx.unload(bid)


@pytest.mark.parametrize("logn,log_cols,p1", [(21, 10, 1), (22, 10, 1), (22, 11, 2), (23, 11, 1),
                                              (23, 12, 2), (23, 10, 1), (24, 12, 1), (24, 11, 2)])
def test_tma_pass2_against_oracle(bps, ctx, orc, logn, log_cols, p1):
    x, ts, bank = _workload(logn, 4600 + logn + log_cols, K=2 if logn <= 23 else 1,
                            ecc=(log_cols % 2 == 1))
    n = x.size
    sid = ctx.load_series(x, ts)
    bid = ctx.load_bank(bank)
    prm = bps.default_params(log_cols=log_cols, log_tile2=13, sigma_thr=5.0, pass1_kind=p1,
                             pass2_kind=bps.BPS_PASS2_TMA)
    pw = ctx.whitened_spectrum(sid, bid, 0, len(bank), n, prm)
    gc, _ = ctx.fetch_candidates(ctx.search(sid, bid, prm))
    oc, res = oracle_on_gpu_maps(ctx, orc, sid, bid, x, ts, bank, want_arrays=True, sigma=5.0)
    for t in range(len(bank)):
        e = pw_close(pw[t], res[t]["Pw"])
        assert e <= PW_TOL, (t, e)
    compare_candidates(gc, oc, bps.thresholds(prm, n, len(bank)))
    # the one-phase pass 2 in the same launch shape gives the same candidates set (both
    # within the power tolerance of the oracle)
    ref, _ = ctx.fetch_candidates(ctx.search(sid, bid, bps.default_params(
        log_cols=log_cols, log_tile2=13, sigma_thr=5.0, pass1_kind=p1, pass2_kind=bps.BPS_PASS2_FUSED)))
    compare_candidates(gc, ref, bps.thresholds(prm, n, len(bank)), max_excused=2)
    ctx.unload(sid)
    ctx.unload(bid)


def test_tma_pass2_many_tiles_and_rejects(bps, ctx, orc):
    """24 templates of 2^21 samples (C = R = 1024: 128 tiles each) on at most one CTA per
    SM: batched equals one template per launch and the oracle on sampled templates; the
    TMA-fed pass 2 is refused where it is not built."""
    logn = 21
    n, ts = 1 << logn, 64e-6
    T = n * ts
    x, _, _ = _workload(logn, 4700)
    bank, _ = synth.uniform_bank(24, 4701, (3 * T, 10 * T), (0.0, 0.3))
    sid = ctx.load_series(x, ts)
    bid = ctx.load_bank(bank)
    res = {}
    for batch in (24, 1, 5):
        prm = bps.default_params(log_cols=10, log_tile2=13, batch=batch, sigma_thr=4.5,
                                 pass2_kind=bps.BPS_PASS2_TMA)
        res[batch] = ctx.fetch_candidates(ctx.search(sid, bid, prm))[0]
    assert np.array_equal(res[24], res[1]) and np.array_equal(res[5], res[1])
    sample = [3, 17]
    sbid = ctx.load_bank(bank[sample])
    oc, _ = oracle_on_gpu_maps(ctx, orc, sid, sbid, x, ts, bank[sample], sigma=4.5)
    oc["template_idx"] = np.array(sample)[oc["template_idx"]]
    compare_candidates(res[24][np.isin(res[24]["template_idx"], sample)], oc,
                       bps.thresholds(prm, n, 24))
    with pytest.raises(bps.BpsError):  # 2^14 pass-2 tiles
        ctx.search(sid, bid, bps.default_params(log_cols=10, log_tile2=14,
                                                pass2_kind=bps.BPS_PASS2_TMA))
    with pytest.raises(bps.BpsError):  # C = 2^9
        ctx.search(sid, bid, bps.default_params(log_cols=9, pass2_kind=bps.BPS_PASS2_TMA))
    for i in (sid, bid, sbid):
        ctx.unload(i)


@pytest.mark.parametrize("logn,log_cols", [(21, 10), (22, 11), (23, 11), (23, 12), (24, 12)])
def test_async_pass1_against_oracle(bps, ctx, orc, logn, log_cols):
    x, ts, bank = _workload(logn, 4800 + logn + log_cols, K=2 if logn <= 23 else 1,
                            ecc=(log_cols % 2 == 0))
    n = x.size
    sid = ctx.load_series(x, ts)
    bid = ctx.load_bank(bank)
    prm = bps.default_params(log_cols=log_cols, sigma_thr=5.0, pass1_kind=bps.BPS_PASS1_ASYNC)
    pw = ctx.whitened_spectrum(sid, bid, 0, len(bank), n, prm)
    gc, _ = ctx.fetch_candidates(ctx.search(sid, bid, prm))
    oc, res = oracle_on_gpu_maps(ctx, orc, sid, bid, x, ts, bank, want_arrays=True, sigma=5.0)
    for t in range(len(bank)):
        e = pw_close(pw[t], res[t]["Pw"])
        assert e <= PW_TOL, (t, e)
    compare_candidates(gc, oc, bps.thresholds(prm, n, len(bank)))
    if logn == 21:
        # batched (many CTAs per SM) equals one template per launch; FP16 storage takes the
        # one-phase kernel and matches it
        b1 = ctx.fetch_candidates(ctx.search(sid, bid, bps.default_params(
            log_cols=log_cols, sigma_thr=5.0, pass1_kind=bps.BPS_PASS1_ASYNC, batch=1)))[0]
        assert np.array_equal(b1, gc)
        s16 = ctx.load_series(x, ts, dtype=bps.BPS_F16_SCALED)
        a16 = ctx.fetch_candidates(ctx.search(s16, bid, prm))[0]
        f16 = ctx.fetch_candidates(ctx.search(s16, bid, bps.default_params(
            log_cols=log_cols, sigma_thr=5.0, pass1_kind=bps.BPS_PASS1_FUSED)))[0]
        assert np.array_equal(a16, f16)
        ctx.unload(s16)
    ctx.unload(sid)
    ctx.unload(bid)
