"""Helpers for the GPU parity tests: the library context and the comparison
rules between the CUDA path and the FP64 oracle.

Tolerances (written here once, used by every parity test):
  * index map: bit-exact except samples whose FP64 offset lies within 1e-6 of
    a rounding boundary (the oracle's ``near`` flag), which are counted;
  * whitened power: |Pw_gpu - Pw_orc| <= 1e-4 * max(1, Pw_orc);
  * harmonic sums: |S_gpu - S_orc| <= 1e-4 * (n + S_orc) (n terms, each within
    the power tolerance);
  * candidates (template, n, bin): identical sets, except candidates whose
    harmonic sum lies within 1e-4 relative of the threshold thr_n, which are
    excused and counted;
  * FP16 series storage, against the oracle on the FP32 series: the same rules
    with 5e-3 in place of 1e-4 (F16_TOL).

Two legs (Algorithm 1's index map has two admissible roundings for offsets
within 1e-6 of a half-integer):
  * oracle_on_gpu_maps: the oracle runs on the GPU's index map after checking it
    sample by sample, which isolates the FFT, whitening and harmonic-sum error;
  * end_to_end_leg: the oracle on its own index map; the samples the two maps
    round differently are counted and the power and candidate deviations they
    can cause are bounded and checked.
"""
import numpy as np

PW_TOL = 1e-4
F16_TOL = 5e-3
LN2 = float(np.log(2.0))


def pw_close(gpu, orc):
    err = np.abs(gpu.astype(np.float64) - orc) / np.maximum(1.0, orc)
    return float(err.max())


def s_close(gpu, orc, nharm):
    err = np.abs(gpu.astype(np.float64) - orc) / (nharm + orc)
    return float(err.max())


def cand_key_set(c):
    return set(zip(c["template_idx"].astype(np.int64).tolist(),
                   c["nharm"].astype(np.int64).tolist(),
                   c["bin"].astype(np.int64).tolist()))


def _cand_dict(c):
    return {k: float(p) for k, p in zip(zip(c["template_idx"].astype(np.int64).tolist(),
                                            c["nharm"].astype(np.int64).tolist(),
                                            c["bin"].astype(np.int64).tolist()), c["power"])}


def compare_candidates(gpu, orc, thr, max_excused=8, tol=PW_TOL):
    """gpu: bps CAND_DTYPE array, orc: oracle CAND_DTYPE array, thr[L] per level.
    Candidates in one set only must lie within tol relative of their level's threshold
    (excused and counted); common candidates agree within tol (n + S).
    Returns (n_matched, n_excused)."""
    g = _cand_dict(gpu)
    o = _cand_dict(orc)
    excused = 0
    for k in set(g) ^ set(o):
        n = k[1]
        t = thr[int(n).bit_length() - 1]
        s = g.get(k, o.get(k))
        assert abs(s - t) <= tol * t, ("candidate mismatch", k, s, t)
        excused += 1
    assert excused <= max_excused, excused
    both = set(g) & set(o)
    for k in both:
        n = k[1]
        assert abs(g[k] - o[k]) <= tol * (n + o[k]), ("power", k, g[k], o[k])
    return len(both), excused


def validated_gpu_map(ctx, orc, sid, bid, t, tmpl, n, ts):
    """The GPU's Algorithm 1 index map for template t, checked against the oracle:
    identical except at samples whose FP64 offset lies within 1e-6 of a rounding
    boundary, where the two differ by one sample.  Returns (map, n_differ)."""
    gi, _ = ctx.index_map(sid, bid, t, n)
    oi, off, near = orc.index_map(tmpl, n, ts)
    gi = gi.astype(np.int64)
    bad = gi != oi
    assert not np.any(bad & ~near), ("index map outside the band", t, np.flatnonzero(bad & ~near)[:8])
    assert np.all(np.abs(gi[bad] - oi[bad]) == 1)
    return gi, int(bad.sum())


def oracle_on_gpu_maps(ctx, orc, sid, bid, x, ts, bank, want_arrays=False, **kw):
    """Oracle run of every template with the validated GPU index map (the
    near-boundary samples take the GPU's admissible rounding).  Returns
    (candidates sorted by template, nharm, bin; per-template results)."""
    import concurrent.futures as cf
    import os
    n = x.size

    maps = []
    # the GPU calls are serialised by the library; run them first, then the oracle in threads
    for t in range(len(bank)):
        maps.append(validated_gpu_map(ctx, orc, sid, bid, t, bank[t], n, ts))

    def orc_one(t):
        r = orc.search_template(x, ts, bank[t], template_idx=t, idx_in=maps[t][0],
                                want_arrays=want_arrays, cap=1 << 20, **kw)
        r["n_differ"] = maps[t][1]
        r["idx_gpu"] = maps[t][0]
        return r

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        res = list(ex.map(orc_one, range(len(bank))))
    cands = np.concatenate([r["cands"] for r in res]) if res else None
    cands = np.sort(cands, order=["template_idx", "nharm", "bin"])
    return cands, res


def oracle_subset(ctx, orc, sid, x, ts, bank, sample, **kw):
    """The oracle on the GPU's validated maps for templates `sample` of `bank` (a
    sub-bank is loaded for the maps); candidates relabelled to bank indices."""
    sub = np.asarray(bank)[list(sample)]
    sbid = ctx.load_bank(sub)
    try:
        oc, res = oracle_on_gpu_maps(ctx, orc, sid, sbid, x, ts, sub, **kw)
    finally:
        ctx.unload(sbid)
    oc["template_idx"] = np.array(sample, np.int64)[oc["template_idx"]]
    return oc, res


def end_to_end_leg(orc, x, ts, tmpl, idx_gpu, pw_gpu, gpu_cands, thr, W=1024, nlev=5,
                   require_near=True):
    """The oracle on its OWN index map against the GPU (the second parity check).

    The two maps may round a near-boundary sample differently.  With delta_j the change
    of resampled sample j that this makes (gather with mean padding) and D = sum |delta_j|,
    every DFT bin moves by at most D, so |P' - P| <= eP = 2 sqrt(P) D + D^2; a block's
    lower median moves by at most the block's largest eP (the median is 1-Lipschitz in the
    max norm), and Pw = P ln2 / med moves by at most
        b = ln2 (eP / (med - emed) + P emed / (med (med - emed))).
    Checks |Pw_gpu - Pw_own| <= b + 1e-4 max(1, Pw_own) bin by bin, and that candidates in
    one set only lie within (harmonic sum of b) + 1e-4 (n + thr) of the threshold.
    Returns a dict with the counts and the largest deviation and bound."""
    x = np.ascontiguousarray(x, np.float32)
    n = x.size
    idx_own, _, near = orc.index_map(tmpl, n, ts)
    diff = idx_gpu != idx_own
    if require_near:
        assert not np.any(diff & ~near)
    mean = orc.series_mean(x)
    xr_own = orc.resample(x, idx_own, mean)
    xr_gpu = orc.resample(x, idx_gpu, mean)
    D = float(np.sum(np.abs(xr_gpu - xr_own)))
    P = orc.power_spectrum(xr_own)
    Pw_own, med = orc.whiten(P, W)
    eP = 2.0 * np.sqrt(P) * D + D * D
    emed = eP.reshape(-1, W).max(axis=1)
    m = np.repeat(med, W)
    em = np.repeat(emed, W)
    with np.errstate(divide="ignore", invalid="ignore"):
        b = np.where(m > em, LN2 * (eP / (m - em) + P * em / (m * (m - em))), np.inf)
    b[0] = 0.0 if med[0] > emed[0] else b[0]
    dev = np.abs(pw_gpu.astype(np.float64) - Pw_own)
    assert np.all(dev <= b + PW_TOL * np.maximum(1.0, Pw_own)), float(np.max(dev - b))
    S_own = orc.harmonic_sums(Pw_own, nlev)
    Sb = orc.harmonic_sums(np.where(np.isfinite(b), b, 1e30), nlev)
    own = {}
    for L in range(nlev):
        ks = np.flatnonzero(S_own[L] >= thr[L])
        ks = ks[ks >= 1]
        for k in ks.tolist():
            own[(1 << L, k)] = float(S_own[L, k])
    g = {(int(c["nharm"]), int(c["bin"])): float(c["power"]) for c in gpu_cands}
    differ = set(g) ^ set(own)
    for key in differ:
        n_h, k = key
        L = n_h.bit_length() - 1
        s = g.get(key, own.get(key))
        assert abs(s - thr[L]) <= Sb[L, k] + PW_TOL * (n_h + thr[L]), (key, s, thr[L], Sb[L, k])
    return {"samples_rounded_differently": int(diff.sum()), "near_band_samples": int(near.sum()),
            "sum_abs_delta": D, "max_pw_dev": float(dev.max()),
            "max_pw_bound": float(np.max(b[np.isfinite(b)])) if np.any(np.isfinite(b)) else 0.0,
            "candidates_common": len(set(g) & set(own)), "candidates_differ": len(differ)}
