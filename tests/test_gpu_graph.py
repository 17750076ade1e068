"""Many searches captured into one CUDA graph (bps_graph_*), and in-place series
updates (bps_series_update).

* a graph over pairs of different series lengths, banks (circular and eccentric) and
  storage types returns, per pair, exactly the candidates of a plain bps_search of
  the same pair; a second replay returns them again;
* per pair, the graph's candidates of the true orbit and one other template agree with
  the FP64 oracle (on the GPU's validated index maps; FP16 pairs against the oracle on
  the FP32 series at the FP16 tolerance);
* after bps_series_update of one series, a replay of the same graph returns the
  candidates of a fresh search of the new data (the other pairs unchanged);
* the plain form cannot be captured; a series or bank captured in a graph cannot be
  unloaded before the graph.
"""
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


def _pair(bps, ctx, logn, K, ecc, f16, seed):
    n, ts = 1 << logn, 64e-6
    T = n * ts
    p = synth.Pulsar(period_s=0.025, porb_s=4 * T, tau_lts=0.05, phi_rad=1.0 + seed,
                     omega_rad=0.5 if ecc else 0.0, ecc=0.05 if ecc else 0.0, amp=0.3)
    x = synth.inject(synth.noise(n, 700 + seed), ts, p)
    bank, where = synth.uniform_bank(K, 800 + seed, (3 * T, 10 * T), (0.0, 0.1),
                                     ecc=(0.0, 0.1) if ecc else None, true_orbits=[p.orbit()])
    dt = bps.BPS_F16_SCALED if f16 else bps.BPS_F32
    return ctx.load_series(x, ts, dt), ctx.load_bank(bank), x, ts, bank, dt, int(where[0])


SHAPES = [(16, 24, False, False), (18, 40, True, False), (20, 12, False, True),
          (17, 64, True, False), (19, 8, False, False), (16, 5, True, False)]


def test_graph_matches_search_and_update(bps, ctx, orc):
    import torch
    prm = bps.default_params(sigma_thr=5.0)
    pairs = [_pair(bps, ctx, *s, seed=i) for i, s in enumerate(SHAPES)]
    ref = [ctx.fetch_candidates(ctx.search(sid, bid, prm))[0] for sid, bid, *_ in pairs]
    gid = ctx.graph_create([(sid, bid) for sid, bid, *_ in pairs], prm)
    st = torch.cuda.Stream()
    for rep in range(2):
        ctx.graph_launch(gid, st if rep else None)
        for i in range(len(pairs)):
            c, tot = ctx.graph_fetch(gid, i)
            assert tot == c.size
            assert np.array_equal(c, ref[i]), (rep, i)
    assert sum(r.size for r in ref) > 0
    # the graph's candidates against the FP64 oracle on two templates per pair
    for i, (sid, bid, x, ts, bank, dt, ti) in enumerate(pairs):
        c, _ = ctx.graph_fetch(gid, i)
        sample = sorted({ti, (ti + 1) % len(bank)})
        oc, _ = oracle_subset(ctx, orc, sid, x, ts, bank, sample, sigma=5.0)
        tol = F16_TOL if dt == bps.BPS_F16_SCALED else PW_TOL
        compare_candidates(c[np.isin(c["template_idx"], sample)], oc,
                           bps.thresholds(prm, x.size, len(bank)), tol=tol)
    # new data for pairs 1 (FP32) and 2 (FP16): the same graph searches it
    for j in (1, 2):
        sid, bid, x, ts, bank, dt, _ = pairs[j]
        x2 = synth.noise(x.size, 900 + j) + np.float32(0.5) * np.sin(
            2 * np.pi * np.arange(x.size) * ts / 0.013).astype(np.float32)
        ctx.update_series(sid, x2 if j == 1 else torch.from_numpy(x2).cuda())
        fresh_sid = ctx.load_series(x2, ts, dt)
        ref[j] = ctx.fetch_candidates(ctx.search(fresh_sid, bid, prm))[0]
        ctx.unload(fresh_sid)
    ctx.graph_launch(gid)
    for i in range(len(pairs)):
        c, _ = ctx.graph_fetch(gid, i)
        assert np.array_equal(c, ref[i]), i
    with pytest.raises(bps.BpsError):
        ctx.unload(pairs[0][0])
    ctx.unload(gid)
    for sid, bid, *_ in pairs:
        ctx.unload(sid)
        ctx.unload(bid)


def test_graph_invalid(bps, ctx):
    sid, bid, *_ = _pair(bps, ctx, 16, 4, False, False, seed=20)
    with pytest.raises(bps.BpsError) as e:
        ctx.graph_create([(sid, bid)], bps.default_params(mode=bps.BPS_MODE_PLAIN))
    assert e.value.code == bps.BPS_ERR_UNSUPPORTED
    with pytest.raises(bps.BpsError):
        ctx.graph_create([(sid, 987654)])
    gid = ctx.graph_create([(sid, bid)])
    with pytest.raises(bps.BpsError):
        ctx.graph_fetch(gid, 0)  # not launched yet
    ctx.graph_launch(gid)
    with pytest.raises(bps.BpsError):
        ctx.graph_fetch(gid, 1)
    ctx.graph_fetch(gid, 0)
    ctx.unload(gid)
    with pytest.raises(bps.BpsError):
        ctx.graph_launch(gid)
    ctx.unload(sid)
    ctx.unload(bid)
