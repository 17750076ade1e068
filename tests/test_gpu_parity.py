"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element
by element, on seeded inputs at sizes the oracle finishes in seconds (several
FFT tiles and anchor blocks, ragged orbits), plus edge cases.  Tolerances are
in tests/gpu_common.py."""
import math

import numpy as np
import pytest

import synth
from gpu_common import (PW_TOL, compare_candidates, oracle_on_gpu_maps, pw_close, s_close,
                        validated_gpu_map)

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


@pytest.fixture(scope="module")
def w1():
    return synth.plain_circular()


ORBITS = [
    (400.0, 0.2, 1.0, 0.0, 0.0),       # the injected orbit of the 2^20 workload
    (200.0, 0.4, 5.9, 0.0, 0.0),       # fastest / widest circular corner
    (670.0, 0.05, 3.3, 0.0, 0.0),
    (25.0, 0.3, 2.0, 1.1, 0.3),        # fast eccentric orbit
    (300.0, 0.5, 2.0, 1.1, 0.3),
    (5000.0, 20.0, 0.4, 4.0, 0.09),    # wide elliptical, large tau
    (400.0, 0.0, 1.0, 0.0, 0.0),       # tau = 0: identity
]


@pytest.mark.parametrize("logn,ts", [(11, 64e-6), (16, 64e-6), (20, 64e-6), (20, 128e-6)])
def test_index_map_bitexact(bps, ctx, orc, logn, ts):
    n = 1 << logn
    x = synth.noise(n, 3)
    sid = ctx.load_series(x, ts)
    bid = ctx.load_bank(np.array(ORBITS))
    for t, tm in enumerate(ORBITS):
        gi, nd = validated_gpu_map(ctx, orc, sid, bid, t, tm, n, ts)
        if tm[1] == 0.0:
            assert np.array_equal(gi, np.arange(n)) and nd == 0
    ctx.unload(sid)
    ctx.unload(bid)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("logn", [11, 14, 17, 20])
def test_whitened_spectrum_parity(bps, ctx, orc, logn, mode):
    n = 1 << logn
    ts = 64e-6
    p = synth.Pulsar(period_s=0.02, porb_s=90.0, tau_lts=0.1, phi_rad=0.3, amp=0.5)
    x = synth.inject(synth.noise(n, 40 + logn), ts, p)
    tms = [p.orbit(), (60.0, 0.3, 4.0, 2.0, 0.2), (1e4, 0.0, 0.0, 0.0, 0.0)]
    sid = ctx.load_series(x, ts)
    bid = ctx.load_bank(np.array(tms))
    W = min(1024, n // 2)
    prm = bps.default_params(whiten_block=W, mode=mode)
    pw = ctx.whitened_spectrum(sid, bid, 0, len(tms), n, prm)
    _, res = oracle_on_gpu_maps(ctx, orc, sid, bid, x, ts, np.array(tms), want_arrays=True,
                                whiten_block=W)
    for t in range(len(tms)):
        assert pw_close(pw[t], res[t]["Pw"]) <= PW_TOL, (t, pw_close(pw[t], res[t]["Pw"]))
    ctx.unload(sid)
    ctx.unload(bid)


@pytest.mark.parametrize("nharm", [1, 2, 4, 8, 16])
def test_harmonic_sums_parity(bps, ctx, orc, w1, nharm):
    n = 1 << 18
    x = w1.series[:n].copy()
    sid = ctx.load_series(x, w1.tsamp)
    tm = w1.pulsars[0].orbit()
    bid = ctx.load_bank(np.array([tm]))
    prm = bps.default_params(nharm_max=nharm)
    S = ctx.harmonic_sums(sid, bid, 0, n, prm)
    _, res = oracle_on_gpu_maps(ctx, orc, sid, bid, x, w1.tsamp, np.array([tm]), want_arrays=True,
                                nharm_max=nharm)
    r = res[0]
    for L in range(S.shape[0]):
        assert s_close(S[L], r["S"][L], 1 << L) <= PW_TOL, (L, s_close(S[L], r["S"][L], 1 << L))
    ctx.unload(sid)
    ctx.unload(bid)


@pytest.mark.parametrize("mode", [0, 1])
def test_search_candidates_workload_2p20(bps, ctx, orc, w1, mode):
    """The whole 2^20-sample, 32-template circular workload: GPU candidates equal
    the oracle's, and the injected pulsar is found under its true orbit."""
    sid = ctx.load_series(w1.series, w1.tsamp)
    bid = ctx.load_bank(w1.bank)
    prm = bps.default_params(mode=mode)
    rid = ctx.search(sid, bid, prm)
    gc, total = ctx.fetch_candidates(rid)
    assert total == gc.size
    oc, _ = oracle_on_gpu_maps(ctx, orc, sid, bid, w1.series, w1.tsamp, w1.bank)
    thr = bps.thresholds(prm, w1.n, w1.bank.shape[0])
    matched, excused = compare_candidates(gc, oc, thr)
    assert matched > 1000
    p = w1.pulsars[0]
    ti = w1.true_idx[0]
    top = gc[(gc["template_idx"] == ti) & (gc["nharm"] == 16)]
    kbest = int(top["bin"][np.argmax(top["power"])])
    assert abs(kbest - round(16 * w1.n * w1.tsamp / p.period_s)) <= 1
    best_t = {}
    for c in gc[gc["nharm"] == 16]:
        best_t[int(c["template_idx"])] = max(best_t.get(int(c["template_idx"]), 0), float(c["power"]))
    assert max(best_t, key=best_t.get) == ti
    ctx.unload(rid)
    ctx.unload(sid)
    ctx.unload(bid)


def test_batch_invariance(bps, ctx, w1):
    n = 1 << 18
    x = w1.series[:n].copy()
    sid = ctx.load_series(x, w1.tsamp)
    bid = ctx.load_bank(w1.bank[:7])
    res = []
    for b in [1, 3, 0]:
        rid = ctx.search(sid, bid, bps.default_params(batch=b))
        c, _ = ctx.fetch_candidates(rid)
        res.append(c)
        ctx.unload(rid)
    for c in res[1:]:
        assert np.array_equal(c, res[0])
    ctx.unload(sid)
    ctx.unload(bid)


@pytest.mark.parametrize("W,nharm,sigma", [(32, 4, 5.0), (8192, 16, 6.0), (256, 1, 4.5)])
def test_variants_parity(bps, ctx, orc, W, nharm, sigma):
    n = 1 << 17
    ts = 64e-6
    p = synth.Pulsar(period_s=0.03, porb_s=50.0, tau_lts=0.05, phi_rad=2.5, amp=0.5)
    x = synth.inject(synth.noise(n, 77), ts, p)
    bank = np.array([p.orbit(), (80.0, 0.1, 1.0, 0.0, 0.0), (40.0, 0.06, 2.0, 0.5, 0.05)])
    sid = ctx.load_series(x, ts)
    bid = ctx.load_bank(bank)
    prm = bps.default_params(whiten_block=W, nharm_max=nharm, sigma_thr=sigma)
    gc, _ = ctx.fetch_candidates(ctx.search(sid, bid, prm))
    oc, _ = oracle_on_gpu_maps(ctx, orc, sid, bid, x, ts, bank, nharm_max=nharm, whiten_block=W,
                               sigma=sigma)
    compare_candidates(gc, oc, bps.thresholds(prm, n, 3))
    ctx.unload(sid)
    ctx.unload(bid)


def test_minimum_size(bps, ctx, orc):
    n, ts = 1 << 11, 64e-6
    x = synth.noise(n, 5)
    x[::50] += 3.0
    bank = np.array([(30.0, 0.001, 1.0, 0.0, 0.0), (30.0, 0.0, 0.0, 0.0, 0.0)])
    sid = ctx.load_series(x, ts)
    bid = ctx.load_bank(bank)
    prm = bps.default_params(whiten_block=32, sigma_thr=4.0)
    gc, _ = ctx.fetch_candidates(ctx.search(sid, bid, prm))
    oc, res = oracle_on_gpu_maps(ctx, orc, sid, bid, x, ts, bank, want_arrays=True,
                                 whiten_block=32, sigma=4.0)
    m, _ = compare_candidates(gc, oc, bps.thresholds(prm, n, 2))
    assert m > 0
    pw = ctx.whitened_spectrum(sid, bid, 0, 2, n, prm)
    for t in range(2):
        assert pw_close(pw[t], res[t]["Pw"]) <= PW_TOL


def test_zero_series_has_no_candidates(bps, ctx):
    n = 1 << 14
    sid = ctx.load_series(np.zeros(n, np.float32), 64e-6)
    bid = ctx.load_bank(np.array([(100.0, 0.1, 0.0, 0.0, 0.0)]))
    gc, total = ctx.fetch_candidates(ctx.search(sid, bid))
    assert total == 0
    pw = ctx.whitened_spectrum(sid, bid, 0, 1, n)
    assert np.all(pw == 0)


def test_invalid_arguments(bps, ctx):
    with pytest.raises(bps.BpsError) as e:
        ctx.load_series(np.zeros(3000, np.float32), 64e-6)
    assert e.value.code == bps.BPS_ERR_INVALID_ARG
    with pytest.raises(bps.BpsError):
        ctx.load_series(np.zeros(1 << 10, np.float32), 64e-6)
    with pytest.raises(bps.BpsError):
        ctx.load_series(np.zeros(1 << 12, np.float32), 0.0)
    for bad in [(0.0, 0.1, 0, 0, 0), (100.0, -1.0, 0, 0, 0), (100.0, 0.1, 0, 0, 1.0),
                (100.0, 0.1, float("nan"), 0, 0)]:
        with pytest.raises(bps.BpsError):
            ctx.load_bank(np.array([bad]))
    sid = ctx.load_series(np.zeros(1 << 12, np.float32), 64e-6)
    bid = ctx.load_bank(np.array([(100.0, 0.1, 0, 0, 0)]))
    with pytest.raises(bps.BpsError):
        ctx.search(sid, 999999)
    with pytest.raises(bps.BpsError):
        ctx.search(sid, bid, bps.default_params(whiten_block=4096))  # > n/2
    fast = ctx.load_bank(np.array([(1.0, 50.0, 0, 0, 0)]))  # beyond the FP32 index-map envelope
    with pytest.raises(bps.BpsError) as e:
        ctx.search(sid, fast)
    assert e.value.code == bps.BPS_ERR_UNSUPPORTED
    with pytest.raises(bps.BpsError):
        ctx.unload(123456789)


def test_candidate_overflow(bps, ctx, w1):
    n = 1 << 18
    sid = ctx.load_series(w1.series[:n].copy(), w1.tsamp)
    bid = ctx.load_bank(w1.bank[:4])
    rid = ctx.search(sid, bid, bps.default_params(sigma_thr=3.0))
    full, total = ctx.fetch_candidates(rid)
    rid2 = ctx.search(sid, bid, bps.default_params(sigma_thr=3.0, cand_cap=10))
    with pytest.raises(bps.BpsError) as e:
        ctx.fetch_candidates(rid2)
    assert e.value.code == bps.BPS_ERR_CAND_OVERFLOW
    part, total2 = ctx.fetch_candidates(rid2, allow_overflow=True)
    assert total2 == total and part.size == 10
    assert set(map(tuple, part[["template_idx", "nharm", "bin"]].tolist())) <= \
        set(map(tuple, full[["template_idx", "nharm", "bin"]].tolist()))


def test_device_pointer_series_and_stream(bps, ctx, w1):
    import torch
    n = 1 << 18
    x = w1.series[:n].copy()
    bid = ctx.load_bank(w1.bank[:5])
    s_host = ctx.load_series(x, w1.tsamp)
    xt = torch.from_numpy(x).cuda()
    s_dev = ctx.load_series(xt, w1.tsamp)
    st = torch.cuda.Stream()
    a, _ = ctx.fetch_candidates(ctx.search(s_host, bid))
    rid = ctx.search(s_dev, bid, stream=st)
    b, _ = ctx.fetch_candidates(rid)
    assert np.array_equal(a, b)


def test_query_is_nonblocking_and_completes(bps, ctx, w1):
    import time
    sid = ctx.load_series(w1.series, w1.tsamp)
    bid = ctx.load_bank(w1.bank)
    rid = ctx.search(sid, bid)
    t0 = time.time()
    while not ctx.query(rid):
        assert time.time() - t0 < 60
        time.sleep(0.001)
    c, total = ctx.fetch_candidates(rid)
    assert total > 0


def test_fp16_storage_error_bounded(bps, ctx, orc, w1):
    """FP16 series with a power-of-two scale per 4096 samples, FP32 FFT: the
    whitened power differs from the FP64 oracle (fed the original FP32 series)
    by the FP16 rounding of the samples only; the pulsar's top candidates agree."""
    n = 1 << 20
    sid = ctx.load_series(w1.series, w1.tsamp, dtype=bps.BPS_F16_SCALED)
    ti = w1.true_idx[0]
    bid = ctx.load_bank(w1.bank[ti:ti + 1])
    pw = ctx.whitened_spectrum(sid, bid, 0, 1, n)[0]
    r = orc.search_template(w1.series, w1.tsamp, w1.bank[ti], want_arrays=True)
    err = np.abs(pw - r["Pw"]) / np.maximum(1.0, r["Pw"])
    assert err.max() < 5e-3, err.max()
    S = ctx.harmonic_sums(sid, bid, 0, n)
    for L in range(5):
        assert int(np.argmax(S[L])) == int(np.argmax(r["S"][L]))


def test_autotune_choice_and_invariance(bps, ctx, w1):
    n = 1 << 18
    x = w1.series[:n].copy()
    sid = ctx.load_series(x, w1.tsamp)
    bid = ctx.load_bank(w1.bank[:12])
    ref, _ = ctx.fetch_candidates(ctx.search(sid, bid, bps.default_params(log_tile=14, log_tile2=13,
                                                                        batch=8)))
    best, ms = ctx.autotune(sid, bid, bps.default_params(), sample_templates=8)
    assert best.log_tile in (13, 14) and best.log_tile2 in (12, 13, 14) and best.batch in (4, 8)
    # 2^18 samples: the default split (10) or one the autotuner also tries (-1, +1, +2)
    assert best.log_cols in (9, 10, 11, 12)
    assert ms > 0
    got, _ = ctx.fetch_candidates(ctx.search(sid, bid, bps.default_params()))  # uses the choice
    # the same launch shape given explicitly computes the same floats
    same, _ = ctx.fetch_candidates(ctx.search(sid, bid, bps.default_params(
        log_tile=best.log_tile, log_tile2=best.log_tile2, log_cols=best.log_cols, batch=best.batch)))
    assert np.array_equal(got, same)
    # another four-step split rounds differently: same candidates, powers within 1e-5
    key = ["template_idx", "nharm", "bin"]
    assert np.array_equal(got[key], ref[key])
    assert np.allclose(got["power"], ref["power"], rtol=1e-5, atol=0)


@pytest.mark.parametrize("logn", [16, 19, 21])
def test_pass1_tiles_identical(bps, ctx, logn):
    """Pass-1 tiles of 2^13 and 2^14 complex (G = 2^13/R and 2^14/R columns per CTA,
    different kernel instantiations) compute the same floats: every column FFT runs the
    same operations in the same order whatever the tile."""
    n, ts = 1 << logn, 64e-6
    T = n * ts
    p = synth.Pulsar(period_s=0.021, porb_s=5 * T, tau_lts=0.08, phi_rad=0.4, amp=0.3)
    x = synth.inject(synth.noise(n, 1000 + logn), ts, p)
    bank, _ = synth.uniform_bank(6, 2000 + logn, (3 * T, 10 * T), (0.0, 0.1),
                                 true_orbits=[p.orbit()])
    sid = ctx.load_series(x, ts)
    bid = ctx.load_bank(bank)
    res = {}
    for lt in (13, 14):
        prm = bps.default_params(log_tile=lt, log_tile2=13, sigma_thr=5.0)
        res[lt] = (ctx.whitened_spectrum(sid, bid, 0, 6, n, prm),
                   ctx.fetch_candidates(ctx.search(sid, bid, prm))[0])
    assert np.array_equal(res[13][0], res[14][0])
    assert np.array_equal(res[13][1], res[14][1]) and res[13][1].size > 0
    ctx.unload(sid)
    ctx.unload(bid)


@pytest.mark.parametrize("logn,log_cols", [(16, 0), (19, 0), (21, 0), (23, 11)])
def test_pass2_tiles_identical(bps, ctx, logn, log_cols):
    """Pass-2 tiles of 2^12, 2^13 and 2^14 complex (NP = tile / 2C row pairs per CTA, one,
    two or four CTAs per SM; row-major or bin-order power by NP) compute the same floats:
    every row FFT, split and power runs the same operations whatever the tile.  2^23 at
    C = 2048 is the benchmark's split (NP = 1, 2 and 4)."""
    n, ts = 1 << logn, 64e-6
    T = n * ts
    p = synth.Pulsar(period_s=0.023, porb_s=6 * T, tau_lts=0.06, phi_rad=1.4, amp=0.3)
    x = synth.inject(synth.noise(n, 1100 + logn), ts, p)
    K = 3 if logn >= 23 else 5
    bank, _ = synth.uniform_bank(K, 2100 + logn, (3 * T, 10 * T), (0.0, 0.1),
                                 true_orbits=[p.orbit()])
    sid = ctx.load_series(x, ts)
    bid = ctx.load_bank(bank)
    res = {}
    for t2 in (12, 13, 14):
        prm = bps.default_params(log_tile=14, log_tile2=t2, log_cols=log_cols, sigma_thr=5.0)
        res[t2] = (ctx.whitened_spectrum(sid, bid, 0, K, n, prm),
                   ctx.fetch_candidates(ctx.search(sid, bid, prm))[0])
    for t2 in (12, 14):
        assert np.array_equal(res[13][0].view(np.uint32), res[t2][0].view(np.uint32)), t2
        assert np.array_equal(res[13][1], res[t2][1]), t2
    assert res[13][1].size > 0
    ctx.unload(sid)
    ctx.unload(bid)


@pytest.mark.parametrize("logn", [17, 23])
def test_f16_uniform_scale_bit_exact(bps, ctx, logn):
    """FP16 storage with one power-of-two scale for all blocks (here 2^8: |x| < 4
    everywhere): the whitened power and the candidates equal, bit for bit, the FP32 path on
    the series quantised the same way in numpy, half(x / 2^8) * 2^8 (round-to-nearest-even
    FP16 conversion): the packing rounds like numpy and the FP16 gather dequantises
    exactly.  tau = 0 templates map every sample inside the series, so the fill value (the
    mean of the unquantised series for FP16 storage) plays no part."""
    n, ts = 1 << logn, 64e-6
    rng = np.random.default_rng(1200 + logn)
    x = np.clip(rng.standard_normal(n), -3.9, 3.9).astype(np.float32)
    xq = ((x / np.float32(256.0)).astype(np.float16).astype(np.float32) * np.float32(256.0))
    T = n * ts
    bank = np.array([[4.0 * T, 0.0, 0.3, 0.0, 0.0], [7.0 * T, 0.0, 2.1, 0.0, 0.0]])
    s16 = ctx.load_series(x, ts, bps.BPS_F16_SCALED)
    sq = ctx.load_series(xq, ts)
    bid = ctx.load_bank(bank)
    prm = bps.default_params(sigma_thr=5.0)
    a = ctx.whitened_spectrum(s16, bid, 0, 2, n, prm)
    b = ctx.whitened_spectrum(sq, bid, 0, 2, n, prm)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    ca, _ = ctx.fetch_candidates(ctx.search(s16, bid, prm))
    cb, _ = ctx.fetch_candidates(ctx.search(sq, bid, prm))
    assert np.array_equal(ca, cb)
    for i in (s16, sq, bid):
        ctx.unload(i)


def test_bounded_wait_expires_and_context_survives(bps, ctx, w1):
    """A kernel polling an mbarrier whose phase nothing completes gives up after its
    limit and reports it; the context keeps working (a search right after matches one
    before)."""
    n = 1 << 16
    sid = ctx.load_series(w1.series[:n].copy(), w1.tsamp)
    bid = ctx.load_bank(w1.bank[:2])
    before, _ = ctx.fetch_candidates(ctx.search(sid, bid, bps.default_params(sigma_thr=4.0)))
    assert ctx.selftest_bounded_wait(1000) is True
    after, _ = ctx.fetch_candidates(ctx.search(sid, bid, bps.default_params(sigma_thr=4.0)))
    assert np.array_equal(before, after)
    with pytest.raises(bps.BpsError):
        ctx.selftest_bounded_wait(0)
    ctx.unload(sid)
    ctx.unload(bid)


@pytest.mark.parametrize("logn,log_cols,W", [(16, 9, 1024), (18, 9, 1024), (18, 11, 1024),
                                             (20, 11, 1024), (20, 12, 1024), (21, 12, 256),
                                             (21, 12, 32), (22, 11, 1024), (22, 11, 64)])
def test_four_step_splits_against_oracle(bps, ctx, orc, logn, log_cols, W):
    """Other four-step splits N/2 = R x C (other radix structures of both FFT passes;
    where a pass-2 CTA holds one or two row pairs and W <= R -- 2^21 with C = 4096, 2^22
    with C = 2048 -- the grouped row-major power layout and the transposing median) give
    the oracle's whitened power and candidates."""
    n, ts = 1 << logn, 64e-6
    T = n * ts
    p = synth.Pulsar(period_s=0.023, porb_s=6 * T, tau_lts=0.06, phi_rad=0.9, amp=0.4)
    x = synth.inject(synth.noise(n, 3000 + logn), ts, p)
    bank = np.array([p.orbit(), (8 * T, 0.03, 2.0, 0.0, 0.0)])
    sid = ctx.load_series(x, ts)
    bid = ctx.load_bank(bank)
    prm = bps.default_params(log_cols=log_cols, sigma_thr=5.0, whiten_block=W)
    pw = ctx.whitened_spectrum(sid, bid, 0, 2, n, prm)
    gc, _ = ctx.fetch_candidates(ctx.search(sid, bid, prm))
    oc, res = oracle_on_gpu_maps(ctx, orc, sid, bid, x, ts, bank, want_arrays=True, sigma=5.0,
                                 whiten_block=W)
    for t in range(2):
        assert pw_close(pw[t], res[t]["Pw"]) <= PW_TOL, t
    compare_candidates(gc, oc, bps.thresholds(prm, n, 2))
    with pytest.raises(bps.BpsError):
        ctx.search(sid, bid, bps.default_params(log_cols=logn))  # R < 32
    ctx.unload(sid)
    ctx.unload(bid)


def test_fp16_storage_mixed_block_scales(bps, ctx, orc, w1):
    """FP16 storage of a series whose blocks need different scales (a burst 2^10 times
    louder in one 4096-sample block, so the per-block scales differ and every gathered
    sample takes its own block's scale): whitened power within 5e-3 of the oracle on the
    FP32 series, as for a series whose blocks share one scale."""
    n = 1 << 18
    x = w1.series[:n].copy()
    x[40960:45056] *= 1024.0
    ti = w1.true_idx[0]
    bank = w1.bank[ti:ti + 1]
    bid = ctx.load_bank(bank)
    r = orc.search_template(x, w1.tsamp, bank[0], want_arrays=True)
    for data in (x, w1.series[:n].copy()):
        r = orc.search_template(data, w1.tsamp, bank[0], want_arrays=True)
        sid = ctx.load_series(data, w1.tsamp, dtype=bps.BPS_F16_SCALED)
        pw = ctx.whitened_spectrum(sid, bid, 0, 1, n)[0]
        err = np.abs(pw - r["Pw"]) / np.maximum(1.0, r["Pw"])
        assert err.max() < 5e-3, err.max()
        ctx.unload(sid)
    ctx.unload(bid)
