"""bps_whiten against the oracle's block lower median (App. A, "Fourier de-reddening").

The median is an element of its block, so the scale ln2 / med (one FP32 division) and
Pw = P * scale (one FP32 product) are compared bit for bit.  The value distributions
reach every branch of the median kernels: noise power (one or two values share the
median's top 16 bits: the ballot gather), values quantised to a few levels (exact ties:
the gather with ties when at most 32 remain, the last two radix digits when more do),
values within one part in 2^8 of each other (all candidates: the radix digits on
distinct values), constant blocks, blocks whose median is 0, and values spread over
sixty binades; whitening blocks of 32 ... 8192 bins (warp kernels up to 1024, the
block kernel above)."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

LN2 = np.float32(np.log(2.0))


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


def power_values(kind: str, shape, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    e = rng.exponential(1.0, shape)
    if kind == "noise":
        trend = 1.0 + 0.5 * np.sin(np.linspace(0.0, 3.0, shape[-1]))
        v = e * trend
    elif kind == "ties_fine":
        v = np.round(e * 64.0) / 64.0
    elif kind == "ties_coarse":
        v = np.round(e * 4.0) / 4.0
    elif kind == "near":
        v = 1.0 + 2.0 ** -20 * rng.integers(0, 4096, shape)
    elif kind == "const":
        v = np.full(shape, 3.25)
    elif kind == "zero_median":
        # 60 % zeros in the first half (median 0), 30 % in the second
        pz = np.where(np.arange(shape[-1]) < shape[-1] // 2, 0.6, 0.3)
        v = np.where(rng.random(shape) < pz, 0.0, e)
    elif kind == "binades":
        v = 2.0 ** rng.uniform(-30.0, 30.0, shape)
    else:
        raise ValueError(kind)
    return v.astype(np.float32)


def expected(orc, P32: np.ndarray, W: int):
    """Scale and whitened power from the oracle's medians, in the kernels' FP32 steps."""
    sc_all, pw_all = [], []
    for row in P32:
        _, med = orc.whiten(row.astype(np.float64), W)
        m32 = med.astype(np.float32)
        assert np.array_equal(m32.astype(np.float64), med)  # the median is an element
        sc = np.zeros_like(m32)
        nz = m32 > 0
        sc[nz] = LN2 / m32[nz]
        sc_all.append(sc)
        pw_all.append(row * np.repeat(sc, W))
    return np.stack(sc_all), np.stack(pw_all)


KINDS = ["noise", "ties_fine", "ties_coarse", "near", "const", "zero_median", "binades"]


@pytest.mark.parametrize("W", [32, 64, 256, 1024, 2048, 8192])
@pytest.mark.parametrize("kind", KINDS)
def test_whiten_bitexact(bps, ctx, orc, kind, W):
    import torch
    nbins = 1 << 15
    P = power_values(kind, (3, nbins), 1000 + W + KINDS.index(kind))
    d = torch.from_numpy(P).cuda()
    pw, sc = ctx.whiten(d, W)
    torch.cuda.synchronize()
    sc_ref, pw_ref = expected(orc, P, W)
    got_sc = sc.cpu().numpy()
    assert np.array_equal(got_sc.view(np.uint32), sc_ref.view(np.uint32)), \
        np.argwhere(got_sc != sc_ref)[:5]
    assert np.array_equal(pw.cpu().numpy().view(np.uint32), pw_ref.view(np.uint32))
    assert torch.equal(d.cpu(), torch.from_numpy(P))  # input left unchanged


def test_whiten_in_place_and_single_spectrum(bps, ctx, orc):
    import torch
    P = power_values("noise", (1, 1 << 12), 7)
    d = torch.from_numpy(P[0].copy()).cuda()
    pw, sc = ctx.whiten(d, 1024, out=d)
    torch.cuda.synchronize()
    sc_ref, pw_ref = expected(orc, P, 1024)
    assert pw.data_ptr() == d.data_ptr()
    assert np.array_equal(d.cpu().numpy(), pw_ref[0])
    assert np.array_equal(sc.cpu().numpy(), sc_ref[0])


def test_whiten_many_spectra(bps, ctx, orc):
    """More spectra than one launch's grid height (65535): the call splits them."""
    import torch
    count, nbins, W = 70000, 64, 32
    P = power_values("noise", (count, nbins), 11)
    pw, sc = ctx.whiten(torch.from_numpy(P).cuda(), W)
    torch.cuda.synchronize()
    idx = [0, 1, 65534, 65535, 65536, count - 1]
    sc_ref, pw_ref = expected(orc, P[idx], W)
    assert np.array_equal(sc.cpu().numpy()[idx], sc_ref)
    assert np.array_equal(pw.cpu().numpy()[idx], pw_ref)


def test_whiten_arguments(bps, ctx):
    import torch
    d = torch.zeros(1 << 12, device="cuda")
    o = torch.empty_like(d)
    s = torch.empty(1 << 8, device="cuda")
    L = bps.lib()
    vp = C.c_void_p
    ok = dict(count=1, nbins=1 << 12, W=32)

    def call(src=d, out=o, scale=s, count=1, nbins=1 << 12, W=32):
        p = lambda t: vp(t.data_ptr()) if hasattr(t, "data_ptr") else t
        return L.bps_whiten(ctx.h, p(src), count, nbins, W, p(out), p(scale), None)

    assert call(**ok) == bps.BPS_OK
    for bad in (dict(W=16), dict(W=16384), dict(W=48), dict(nbins=16), dict(nbins=3000),
                dict(count=0), dict(count=1 << 61), dict(out=d[1:]), dict(scale=None)):
        assert call(**bad) == bps.BPS_ERR_INVALID_ARG, bad
    host = np.zeros(1 << 12, np.float32)
    assert call(src=host.ctypes.data_as(vp)) == bps.BPS_ERR_INVALID_ARG
    torch.cuda.synchronize()
