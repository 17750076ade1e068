"""Helpers for the GPU parity tests: the library context and the comparison
rules between the CUDA path and the FP64 oracle.

Tolerances (written here once, used by every parity test):
  * index map: bit-exact except samples whose FP64 offset lies within 1e-6 of
    a rounding boundary (the oracle's ``near`` flag), which are counted;
  * whitened power: |Pw_gpu - Pw_orc| <= 1e-4 * max(1, Pw_orc);
  * harmonic sums: |S_gpu - S_orc| <= 1e-4 * (n + S_orc) (n terms, each within
    the power tolerance);
  * candidates (template, n, bin): identical sets, except candidates whose
    harmonic sum lies within the harmonic-sum tolerance of the threshold,
    which are excused and counted.
"""
import numpy as np

PW_TOL = 1e-4


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


def compare_candidates(gpu, orc, thr, max_excused=8):
    """gpu: bps CAND_DTYPE array, orc: oracle CAND_DTYPE array, thr[L] per level.
    Returns (n_matched, n_excused); asserts the parity rule."""
    g = {k: float(p) for k, p in zip(zip(gpu["template_idx"].astype(np.int64).tolist(),
                                        gpu["nharm"].astype(np.int64).tolist(),
                                        gpu["bin"].astype(np.int64).tolist()), gpu["power"])}
    o = {k: float(p) for k, p in zip(zip(orc["template_idx"].astype(np.int64).tolist(),
                                        orc["nharm"].astype(np.int64).tolist(),
                                        orc["bin"].astype(np.int64).tolist()), orc["power"])}
    excused = 0
    for k in set(g) ^ set(o):
        n = k[1]
        t = thr[int(n).bit_length() - 1]
        s = g.get(k, o.get(k))
        assert abs(s - t) <= 2 * PW_TOL * (n + t), ("candidate mismatch", k, s, t)
        excused += 1
    assert excused <= max_excused, excused
    both = set(g) & set(o)
    for k in both:
        n = k[1]
        assert abs(g[k] - o[k]) <= PW_TOL * (n + o[k]), ("power", k, g[k], o[k])
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
        return r

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        res = list(ex.map(orc_one, range(len(bank))))
    cands = np.concatenate([r["cands"] for r in res]) if res else None
    cands = np.sort(cands, order=["template_idx", "nharm", "bin"])
    return cands, res
