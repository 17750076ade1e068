"""Algorithm 1's index map at the edge of the planner's FP32 envelope.

The per-sample fast path evaluates the offset off(c + d) - I = f - inc(d) about an FP64
anchor c with the cubic Taylor polynomial inc(d) ~ L d + q2 d^2 + q3 d^3 in FP32; the
planner picks the anchor block B (h = B/2 = the largest |d|) so that, for every template
of the bank, |K g h| <= 128 samples, K g^2 h^2 <= 0.25 and K g^4 h^4 <= 1e-5, with
K = tau / t_s and g = Omega t_s / (1 - e).  The templates here sit just inside those
limits at B = 2^14 (d = +-8192 at every block edge): one where the linear term reaches
127.9 samples, one where the quadratic and quartic terms reach 0.2497 and 9e-6, for
e = 0.1 and e = 0.9, at 2^20, 2^23 and 2^25 samples.  The GPU map must equal the FP64
oracle's except at samples whose FP64 offset lies within 1e-6 of a rounding boundary,
where the two differ by one sample (the error budget of the fast path, about 3.3e-5
sample, stays inside its 1e-4 guard; samples inside the guard take the compensated
branch)."""
import math

import numpy as np
import pytest

from gpu_common import validated_gpu_map

pytestmark = pytest.mark.gpu

TS = 64e-6
H = 8192.0  # B / 2 at the largest anchor block


def edge_templates(e):
    """(linear-edge, quadratic/quartic-edge) templates at B = 2^14 for eccentricity e."""
    out = []
    for gh, K, phi, om in [(1.5e-3, 127.9 / 1.5e-3, 0.7, 1.9),    # K g h = 127.9
                           (6e-3, 0.2497 / 6e-3 ** 2, 2.3, 4.4)]:  # K (g h)^2 = 0.2497
        g = gh / H
        porb = 2.0 * math.pi * TS / (g * (1.0 - e))
        out.append((porb, K * TS, phi, om, e))
    return out


def planner_terms(t):
    K = t[1] / TS
    g = (2.0 * math.pi / t[0]) * TS / (1.0 - t[4])
    return K * g * H, K * (g * H) ** 2, K * (g * H) ** 4


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


def test_edge_templates_are_at_the_limits():
    for e in (0.1, 0.9):
        lin, quad = edge_templates(e)
        a = planner_terms(lin)
        b = planner_terms(quad)
        assert 127.0 < a[0] <= 128.0 and a[1] <= 0.25 and a[2] <= 1e-5
        assert b[0] <= 128.0 and 0.249 < b[1] <= 0.25 and 8e-6 < b[2] <= 1e-5


@pytest.mark.parametrize("logn", [20, 23, 25])
@pytest.mark.parametrize("e", [0.1, 0.9])
def test_index_map_at_the_envelope_edge(bps, ctx, orc, logn, e):
    n = 1 << logn
    x = np.zeros(n, np.float32)
    sid = ctx.load_series(x, TS)
    for t in edge_templates(e):
        bid = ctx.load_bank(np.array([t]))
        # the planner keeps B = 2^14 for this template
        rid = ctx.search(sid, bid, bps.default_params(nharm_max=1, whiten_block=1024))
        ctx.fetch_candidates(rid)
        assert ctx.request_stats(rid)["anchor_block"] == 1 << 14
        ctx.unload(rid)
        gi, nd = validated_gpu_map(ctx, orc, sid, bid, 0, t, n, TS)
        _, npre = ctx.index_map(sid, bid, 0, n)
        print("\n[envelope] 2^%d e=%.1f tau=%.4g Porb=%.5g: %d samples rounded the other way "
              "(inside the 1e-6 band), %d took the compensated branch" % (logn, e, t[1], t[0], nd, npre))
        ctx.unload(bid)
    ctx.unload(sid)
