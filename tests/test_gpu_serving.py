"""The continuously batched request loop (bps_server_*).

* every request's candidates are identical whether it runs alone or mixed with
  requests of other series lengths, banks and storage types (and identical to a
  plain bps_search of the same inputs);
* every request's candidates of its true orbit and one other template agree with the
  FP64 oracle (on the GPU's validated index maps; the FP16 request against the oracle
  on the FP32 series at the FP16 tolerance);
* with an HBM budget that fits about one request, later requests wait in the queue
  and all complete; a request larger than the budget is refused at submission;
* latencies are measured from submission to candidates on the host.
"""
import time

import numpy as np
import pytest

import synth
from gpu_common import F16_TOL, PW_TOL, compare_candidates, oracle_subset

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


def _requests(bps):
    out = []
    for i, (logn, K, ecc, f16) in enumerate([(16, 24, False, False), (18, 40, True, False),
                                             (20, 16, False, True), (17, 64, True, False),
                                             (19, 8, False, False)]):
        n, ts = 1 << logn, 64e-6
        T = n * ts
        p = synth.Pulsar(period_s=0.025, porb_s=4 * T, tau_lts=0.05, phi_rad=1.0 + i,
                         omega_rad=0.5 if ecc else 0.0, ecc=0.05 if ecc else 0.0, amp=0.3)
        x = synth.inject(synth.noise(n, 300 + i), ts, p)
        bank, where = synth.uniform_bank(K, 400 + i, (3 * T, 10 * T), (0.0, 0.1),
                                         ecc=(0.0, 0.1) if ecc else None, true_orbits=[p.orbit()])
        out.append((x, ts, bank, bps.BPS_F16_SCALED if f16 else bps.BPS_F32, int(where[0])))
    return out


def test_same_results_alone_and_in_the_mix(bps, ctx, orc):
    reqs = [r[:4] for r in _requests(bps)]
    truth = [r[4] for r in _requests(bps)]
    prm = bps.default_params(sigma_thr=5.0)
    with bps.Server(ctx, max_active=4, groups_in_flight=2) as srv:
        alone = []
        for x, ts, bank, dt in reqs:
            t = srv.submit(x, ts, bank, prm, dt)
            c, tot, lat = srv.result(t)
            assert tot == c.size and lat > 0
            alone.append(c)
        tickets = [srv.submit(x, ts, bank, prm, dt) for (x, ts, bank, dt) in reqs + reqs[::-1]]
        mixed = [srv.result(t)[0] for t in tickets]
    for i in range(len(reqs)):
        assert np.array_equal(mixed[i], alone[i]), i
        assert np.array_equal(mixed[2 * len(reqs) - 1 - i], alone[i]), i
    # served results against the FP64 oracle, two templates per request
    for (x, ts, bank, dt), ti, c in zip(reqs, truth, alone):
        sid = ctx.load_series(x, ts)
        sample = sorted({ti, (ti + 1) % len(bank)})
        oc, _ = oracle_subset(ctx, orc, sid, x, ts, bank, sample, sigma=5.0)
        ctx.unload(sid)
        tol = F16_TOL if dt == bps.BPS_F16_SCALED else PW_TOL
        compare_candidates(c[np.isin(c["template_idx"], sample)], oc,
                           bps.thresholds(prm, x.size, len(bank)), tol=tol)
    # the same kernels through the plain request path
    x, ts, bank, dt = reqs[1]
    sid = ctx.load_series(x, ts, dt)
    bid = ctx.load_bank(bank)
    c, _ = ctx.fetch_candidates(ctx.search(sid, bid, prm))
    assert np.array_equal(c, alone[1])
    assert sum(a.size for a in alone) > 0


def test_admission_queue_and_budget(bps, ctx):
    reqs = [r[:4] for r in _requests(bps)]
    prm = bps.default_params(sigma_thr=5.0, cand_cap=1 << 16)
    x, ts, bank, dt = reqs[2]  # 2^20 samples: the largest request
    with bps.Server(ctx, max_active=4, groups_in_flight=2, hbm_budget=160 << 20) as srv:
        tickets = [srv.submit(x, ts, bank, prm, dt) for _ in range(6)]
        seen_queued = srv.stats()["queued"] > 0
        res = [srv.result(t) for t in tickets]
        st = srv.stats()
    assert seen_queued
    assert all(np.array_equal(r[0], res[0][0]) for r in res)
    lat = [r[2] for r in res]
    assert lat == sorted(lat) or max(lat) > min(lat)  # later requests waited
    assert st["active"] == 0 and st["bytes_held"] == 0
    with bps.Server(ctx, max_active=1, hbm_budget=1 << 20) as small:
        with pytest.raises(bps.BpsError) as e:
            small.submit(x, ts, bank, prm, dt)
        assert e.value.code == bps.BPS_ERR_OUT_OF_MEMORY


def test_nonblocking_result_and_invalid(bps, ctx):
    reqs = [r[:4] for r in _requests(bps)]
    x, ts, bank, dt = reqs[0]
    with bps.Server(ctx, max_active=2) as srv:
        t = srv.submit(x, ts, bank, bps.default_params(), dt)
        r = srv.result(t, timeout_ms=0)
        t0 = time.time()
        while r is None:
            assert time.time() - t0 < 60
            r = srv.result(t, timeout_ms=10)
        with pytest.raises(bps.BpsError):
            srv.submit(x[:3000], ts, bank, bps.default_params(), dt)
        with pytest.raises(bps.BpsError):
            srv.result(987654)


def test_resident_series_same_results(bps, ctx):
    """Requests on series held in the server's resident store return exactly the
    candidates of requests that carry their own copy of the series; the series is staged
    once and stays on the device."""
    reqs = [r[:4] for r in _requests(bps)]
    prm = bps.default_params(sigma_thr=5.0)
    with bps.Server(ctx, max_active=4, groups_in_flight=2) as srv:
        ref = [srv.result(srv.submit(x, ts, bank, prm, dt))[0] for x, ts, bank, dt in reqs]
        ids = [srv.load_series(x, ts, dt) for x, ts, bank, dt in reqs]
        assert not srv.series_info(ids[0])["resident"]
        tickets = [srv.submit_series(i, bank, prm) for i, (_, _, bank, _) in zip(ids, reqs)]
        tickets += [srv.submit_series(i, bank, prm) for i, (_, _, bank, _) in zip(ids, reqs)][::-1]
        res = [srv.result(t)[0] for t in tickets]
        for i in range(len(reqs)):
            assert np.array_equal(res[i], ref[i]), i
            assert np.array_equal(res[2 * len(reqs) - 1 - i], ref[i]), i
        for i in ids:
            info = srv.series_info(i)
            assert info["resident"] and info["times_staged"] == 1
        srv.unload_series(ids[0])
        with pytest.raises(bps.BpsError):
            srv.submit_series(ids[0], reqs[0][2], prm)
        with pytest.raises(bps.BpsError):
            srv.series_info(987654)


def test_resident_series_lru_eviction(bps, ctx):
    """With an HBM budget that holds one 2^24-sample series beside a request but not two,
    alternating requests evict the least recently used idle series and stage it again
    from the server's host copy; results are unchanged."""
    n, ts, K = 1 << 24, 64e-6, 4
    T = n * ts
    xs = [synth.noise(n, 600 + i) for i in range(2)]
    bank, _ = synth.uniform_bank(K, 601, (3 * T, 10 * T), (0.0, 1.0))
    prm = bps.default_params(sigma_thr=5.0, batch=K, cand_cap=1 << 10, log_cols=11,
                             log_tile=14, log_tile2=13)
    M = n // 2
    # device bytes of one request (bank, workspace of K templates, candidates): the packed
    # FFT intermediate, the power in bin order and row-major (C = 2048, 2^13 pass-2 tiles),
    # anchors and block scales (< 1 MiB)
    req = (M + 1) * 8 * K + 2 * M * 4 * K + (1 << 20)
    ser = 4 * n
    with bps.Server(ctx, max_active=1, groups_in_flight=2, hbm_budget=req + ser + ser // 2) as srv:
        ids = [srv.load_series(x, ts) for x in xs]
        order = [0, 1, 0, 0, 1]
        out = [srv.result(srv.submit_series(ids[j], bank, prm))[0] for j in order]
        staged = [srv.series_info(i)["times_staged"] for i in ids]
        assert staged == [2, 2], staged
        assert srv.stats()["bytes_held"] == ser  # the last series used stays resident
    with bps.Server(ctx, max_active=1) as big:
        ref = [big.result(big.submit(x, ts, bank, prm))[0] for x in xs]
    for j, c in zip(order, out):
        assert np.array_equal(c, ref[j]), j


def test_resident_series_pinned_while_named(bps, ctx):
    """A series named by an unfinished request cannot be unloaded; once its requests are
    done it can, and then it can no longer be named."""
    n, ts = 1 << 22, 64e-6
    T = n * ts
    x = synth.noise(n, 650)
    bank, _ = synth.uniform_bank(2048, 651, (3 * T, 10 * T), (0.0, 1.0))  # ~50 ms of work
    prm = bps.default_params(cand_cap=1 << 12)
    with bps.Server(ctx, max_active=1) as srv:
        sid = srv.load_series(x, ts)
        t = srv.submit_series(sid, bank, prm)
        with pytest.raises(bps.BpsError):
            srv.unload_series(sid)
        srv.result(t, allow_overflow=True)
        srv.unload_series(sid)
        with pytest.raises(bps.BpsError):
            srv.submit_series(sid, bank, prm)
