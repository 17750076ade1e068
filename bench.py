#!/usr/bin/env python
"""Benchmark of the coherent template-bank binary-pulsar search hot path.

One step = one search request: every orbital template of the bank through
index map -> gather -> FFT -> power -> de-reddening -> harmonic sum ->
threshold -> compaction, over one synthetic series already resident in HBM.
Default workload: HTRU-like circular search, 2^23 samples at 64 us, 4096
templates, 16 harmonics, 6 sigma (synthetic noise + 3 injected pulsars).

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
instead (the program the GPU results are checked against).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

HBM_FALLBACK_GBS = 6400.0
METRIC = "templates searched/sec at 2^23 samples vs plain GPU form; p50/p99 request latency"
UNIT = "templates/s"
# Algorithmic bytes per template per stage, in units of N (FP32 series):
#   pass1: series read 4N + packed-complex write 4N; pass2: 4N read + 2N power write;
#   median: 2N read + 2N whitened write; harmsum: 2N read.  Whole path (one series read,
#   whitened spectrum written once and read once): 8N.  With the FFT split into two
#   passes through device memory the packed intermediate adds a 4N write and a 4N read:
#   16N, the bound of a two-pass (out-of-core) FFT.
STAGE_BYTES_PER_N = {"pass1": 8.0, "pass2": 6.0, "median": 4.0, "harmsum": 2.0,
                     "power": 4.0 + 2.0, "anchors": 0.0}
PATH_BYTES_PER_N = 8.0
TWO_PASS_BYTES_PER_N = 16.0
CAND_CAP = 1 << 22


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--logn", type=int, default=23)
    ap.add_argument("--templates", type=int, default=4096)
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--log-tile", type=int, default=0)
    ap.add_argument("--log-tile2", type=int, default=0)
    ap.add_argument("--log-cols", type=int, default=0,
                    help="log2 of the four-step row length C (0 = library / autotuner)")
    ap.add_argument("--pass1-kind", type=int, default=0,
                    help="0 = library / autotuner, 1 = one-phase pass 1, 2 = warp-specialised")
    ap.add_argument("--pass2-kind", type=int, default=0,
                    help="0 = library / autotuner, 1 = one-phase pass 2, 2 = TMA-fed")
    ap.add_argument("--power-layout", type=int, default=0,
                    help="0 = library / autotuner, 1 = bin order, 2 = row-major blocks")
    ap.add_argument("--dtype", default="f32", choices=["f32", "f16"],
                    help="series storage on the device: f32, or f16 with a power-of-two "
                         "scale per 4096 samples (FFT arithmetic is FP32 either way)")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-f16", action="store_true",
                    help="skip the FP16-storage line of the same request")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-rates", default="1,2,5,10,20,50",
                    help="Poisson request rates (req/s) of the serving sweep")
    ap.add_argument("--serve-seconds", type=float, default=4.0,
                    help="arrival window per rate (requests = max(8, rate x seconds))")
    ap.add_argument("--no-uneven", action="store_true",
                    help="skip the batched uneven-length workload (CUDA graph)")
    ap.add_argument("--no-elliptical", action="store_true",
                    help="skip the 2^25-sample elliptical FP16 workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-templates", type=int, default=0)
    ap.add_argument("--cpu-threads", type=int, default=0)
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def kernel_source_hash():
    """Hash of the device-kernel sources (csrc/k_*.cu and the headers they include), the
    code the committed ncu traffic was captured on."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2112_11991_b300", "csrc")
    for f in sorted(os.listdir(d)):
        if (f.startswith("k_") and f.endswith(".cu")) or f.endswith(".cuh"):
            with open(os.path.join(d, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def geometry_key(logn, log_cols, log_tile, log_tile2, pass1_kind=0, pass2_kind=0):
    """Traffic key of a launch shape: four-step split and the two pass tiles (0 = the
    library's defaults: C = 2^min(10, log M - 5) raised to M / 2^12, tiles 14 / 13), with
    a suffix for the warp-specialised pass 1 and the TMA-fed pass 2."""
    logM = logn - 1
    lc = log_cols or (min(10, logM - 5) if logM - min(10, logM - 5) <= 12 else logM - 12)
    key = "c%d_t%d_%d" % (lc, log_tile or 14, log_tile2 or 13)
    if pass1_kind == 2:
        key += "_p1ws"
    if pass2_kind == 2:
        key += "_p2tma"
    return key


def ncu_traffic(stage, workload, templates_per_launch, geom):
    """DRAM bytes per launch of `stage` from the committed ncu summary for this launch
    shape, scaled from the captured launch's templates to this run's (the traffic of
    these kernels grows in proportion to the templates a launch processes), or None when
    absent, captured on another shape or on different kernel sources."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f)
        e = d[workload][geom][stage]
        if e.get("source_hash") != kernel_source_hash():
            return None
        return float(e["dram_bytes_per_launch"]) * templates_per_launch / float(e["templates_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu_id)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons, pw = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                pw.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_init(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=ws)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(ws, v):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(args, ws, rank):
    n = 1 << args.logn
    K = args.templates
    w = synth.htru_circular(n=n, K=K * ws, seed=2)
    bank = w.bank[rank * K:(rank + 1) * K]
    return w, bank


def oracle_rate(x, tsamp, bank, threads):
    import oracle
    t0 = time.perf_counter()
    oracle.search(x, tsamp, bank, nthreads=threads, cap_per=1 << 15)
    dt = time.perf_counter() - t0
    return bank.shape[0] / dt, dt


def f16_oracle_error(ctx, sid16, bid, w, bank, count=2):
    """Whitened-power and harmonic-sum error of the FP16-storage path against the FP64
    oracle on the FP32 series, for the first `count` injected orbits of the bank (the
    oracle on the GPU's index map), in the units of the parity tests: |dPw| / max(1, Pw)
    and |dS| / (n + S) per harmonic level."""
    import oracle
    n = w.n
    pw_err, s_err = 0.0, [0.0] * 5
    tis = [int(t) for t in w.true_idx if t < bank.shape[0]][:count]
    for ti in tis:
        gi = ctx.index_map(sid16, bid, ti, n)[0].astype(np.int64)
        r = oracle.search_template(w.series, w.tsamp, bank[ti], want_arrays=True, idx_in=gi)
        pw = ctx.whitened_spectrum(sid16, bid, ti, 1, n)[0].astype(np.float64)
        S = ctx.harmonic_sums(sid16, bid, ti, n).astype(np.float64)
        pw_err = max(pw_err, float(np.max(np.abs(pw - r["Pw"]) / np.maximum(1.0, r["Pw"]))))
        for L in range(5):
            s_err[L] = max(s_err[L], float(np.max(np.abs(S[L] - r["S"][L]) / ((1 << L) + r["S"][L]))))
    return {"templates": tis, "pw_rel_max": pw_err,
            "harmonic_sum_rel_max_per_level": dict(zip(["1", "2", "4", "8", "16"], s_err))}


def cpu_threads(args):
    c = os.cpu_count() or 1
    return args.cpu_threads or max(1, min(c, 32))


def run_reference(args, ws, rank):
    """FP64 CPU oracle on the host cores, each step a bounded sample of the workload."""
    if rank != 0:
        return
    w, bank = workload(args, 1, 0)
    thr = cpu_threads(args)
    per_step = args.cpu_templates or thr
    sel = np.linspace(0, bank.shape[0] - 1, per_step * (args.steps + 1)).astype(int)
    for i in range(args.warmup):
        oracle_rate(w.series, w.tsamp, bank[sel[i:i + 1]], 1)
    times = []
    for s in range(args.steps):
        b = bank[sel[s * per_step:(s + 1) * per_step]]
        _, dt = oracle_rate(w.series, w.tsamp, b, thr)
        times.append(dt)
    value = per_step * args.steps / sum(times)
    sample = "%d of %d templates per step (%d steps), 2^%d samples" % (
        per_step, bank.shape[0], args.steps, args.logn)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": config_of(w, args, ws),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def serving_pool(seed=5):
    """Seeded series for the serving sweep: three per length 2^20..2^24 at 64 us, the
    first with one injected pulsar-BH binary (0-1 pulsar per request)."""
    return {logn: [synth.pulsar_bh_series(1 << logn, 64e-6, 3000 + 10 * logn,
                                          amp=synth.equal_snr_amp(1 << logn))[0]] +
            [synth.noise(1 << logn, 3000 + 10 * logn + i) for i in (1, 2)]
            for logn in range(20, 25)}


def run_serving(bps, ctx, rate, nreq, pool, seed=5):
    """Poisson stream of search requests into the continuously batched server: series
    2^20..2^24 samples (log-uniform) at 64 us stored FP16 and held in the server's
    resident store (loaded once, before the stream), banks of 64..4096 (log-uniform)
    circular or elliptical (e <= 0.1) templates.  Returns throughput and p50/p99 latency
    (submission to candidates on the host)."""
    import threading
    rng = np.random.default_rng(seed + int(rate * 1000))
    reqs = []
    for i in range(nreq):
        logn = int(rng.integers(20, 25))
        ts = 64e-6
        T = (1 << logn) * ts
        K = int(2 ** rng.uniform(6, 12))
        ecc = (0.0, 0.1) if rng.random() < 0.5 else None
        bank, _ = synth.uniform_bank(K, 1000 + i, (3 * T, 10 * T), (0.0, 0.5), ecc=ecc)
        reqs.append(((logn, i % 3), bank))
    gaps = rng.exponential(1.0 / rate, nreq)
    prm = bps.default_params(cand_cap=1 << 16)
    lat, tickets = [], []
    with bps.Server(ctx, max_active=4, groups_in_flight=2) as srv:
        sids = {(logn, j): srv.load_series(x, 64e-6, bps.BPS_F16_SCALED)
                for logn, xs in pool.items() for j, x in enumerate(xs)}
        # stage every series once (one small request each) so the stream finds them resident
        warm = [srv.submit_series(sid, np.array([(1e4, 0.0, 0.0, 0.0, 0.0)]), prm)
                for sid in sids.values()]
        for t in warm:
            srv.result(t, allow_overflow=True)
        t_start = time.perf_counter()
        done = threading.Event()

        def collect():
            for i in range(nreq):
                while len(tickets) <= i:
                    time.sleep(0.0005)
                _, _, l = srv.result(tickets[i], allow_overflow=True)
                lat.append(l)
            done.set()

        th = threading.Thread(target=collect)
        th.start()
        t_next = t_start
        for (key, bank), g in zip(reqs, gaps):
            t_next += g
            d = t_next - time.perf_counter()
            if d > 0:
                time.sleep(d)
            tickets.append(srv.submit_series(sids[key], bank, prm))
        done.wait()
        th.join()
        wall = time.perf_counter() - t_start
    templates = sum(r[1].shape[0] for r in reqs)
    return {"rate_req_s": rate, "requests": nreq, "templates": templates,
            "templates_per_s": templates / wall, "wall_s": wall,
            "p50_ms": 1e3 * float(np.percentile(lat, 50)),
            "p99_ms": 1e3 * float(np.percentile(lat, 99))}


SERVING_WORKLOAD = ("Poisson arrivals; series 2^20-2^24 (log-uniform) x 64 us, FP16 storage, "
                    "resident in the server (15 series loaded and staged before the stream), "
                    "one in three with an injected pulsar-BH binary; "
                    "banks 64-4096 (log-uniform) circular or elliptical (e <= 0.1) templates; "
                    "server max_active 4, 2 launch groups in flight per request, HBM budget "
                    "0.9 x free; latency from submission to candidates on the host")


def run_uneven(bps, ctx, steps=2, warmup=1, seed=11):
    """Batched uneven search: 64 series of random length 2^21..2^24 at 64 us, each with
    one injected pulsar-BH binary (as in the 2^23 workload, peak amplitude 0.03 sqrt(2^23 / n):
    the same per-harmonic signal-to-noise at every length, 2.25 times the 2^23 workload's
    in power, so that scalloping and noise leave every pulsar detectable) and its own bank of
    256..2048 circular templates (Porb U[3T,10T], tau U[0,3] lt-s, phi U) that includes
    the true orbit; launch shapes autotuned per length, all 64 searches captured in one
    CUDA graph and replayed; device time per replay by CUDA events on the launching
    stream.  Also counts the pulsars whose true template has a candidate within one bin
    of n T / P at some harmonic level n."""
    import torch
    rng = np.random.default_rng(seed)
    pairs, K, n_of, truth, lens, bank_sizes = [], 0, {}, [], [], {}
    ids = []
    for i in range(64):
        logn = int(rng.integers(21, 25))
        n, ts = 1 << logn, 64e-6
        T = n * ts
        k = int(rng.integers(256, 2049))
        x, p = synth.pulsar_bh_series(n, ts, 6000 + i, amp=synth.equal_snr_amp(n, 0.03))
        bank, where = synth.uniform_bank(k, 5000 + i, (3 * T, 10 * T), (0.0, 3.0),
                                         true_orbits=[p.orbit()])
        sid = ctx.load_series(x, ts)
        bid = ctx.load_bank(bank)
        ids += [sid, bid]
        pairs.append((sid, bid))
        lens.append(logn)
        bank_sizes[(sid, bid)] = k
        truth.append((where[0], T, p.period_s))
        n_of[logn] = (sid, bid)
        K += k
    prm = bps.default_params(cand_cap=1 << 20)
    tuned, ms_t = {}, {}
    for logn, (sid, bid) in sorted(n_of.items()):
        best, ms = ctx.autotune(sid, bid, prm, sample_templates=64)
        tuned[logn] = [best.log_tile, best.log_tile2, best.batch, best.log_cols]
        ms_t[logn] = ms
    # the rate the mix would reach if every template ran at its length's uniform rate (the
    # autotuner's best time per template on a 64-template sample of that length)
    k_of = {}
    for (sid, bid), (ti, T, P), logn in zip(pairs, truth, lens):
        k_of[logn] = k_of.get(logn, 0) + bank_sizes[(sid, bid)]
    bound = K / (sum(k_of[l] * ms_t[l] for l in k_of) / 1e3)
    gid = ctx.graph_create(pairs, prm)
    st = torch.cuda.Stream()
    ms = []
    for i in range(warmup + steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st.synchronize()
        e0.record(st)
        ctx.graph_launch(gid, st)
        e1.record(st)
        st.synchronize()
        if i >= warmup:
            ms.append(e0.elapsed_time(e1))
    ncand, found = 0, 0
    for j, (ti, T, P) in enumerate(truth):
        c, tot = ctx.graph_fetch(gid, j, allow_overflow=True)
        ncand += tot
        c = c[c["template_idx"] == ti]
        found += any(abs(int(b) - round(int(h) * T / P)) <= 1 for b, h in zip(c["bin"], c["nharm"]))
    ctx.unload(gid)
    for x in ids:
        ctx.unload(x)
    return {"workload": "64 series of 2^21-2^24 samples (random) x 64 us, one injected pulsar-BH "
                        "binary each (peak amplitude 0.03 sqrt(2^23/n)), each with 256-2048 "
                        "circular templates (Porb U[3T,10T], "
                        "tau U[0,3] lt-s) including its true orbit; one CUDA graph over the 64 "
                        "searches (4 parallel branches), launch shapes autotuned per length",
            "templates": K, "value": K / (statistics.mean(ms) / 1e3), "unit": UNIT,
            "ms_per_graph": statistics.mean(ms), "steps": steps, "warmup": warmup,
            "autotuned": {"2^%d" % k: v for k, v in tuned.items()},
            "templates_per_length": {"2^%d" % k: v for k, v in sorted(k_of.items())},
            "uniform_ms_per_template": {"2^%d" % k: v for k, v in sorted(ms_t.items())},
            "uniform_rate_bound": bound, "fraction_of_uniform_rate_bound": (K / (statistics.mean(ms) / 1e3)) / bound,
            "candidates": int(ncand),
            "pulsars_found": "%d of 64" % found}


def run_elliptical_f16(bps, ctx, steps=2, warmup=1):
    """Elliptical IMBH search at 2^25 samples x 128 us, 2048 five-parameter templates,
    series stored FP16 with a power-of-two scale per 4096 samples, FP32 FFT.  Reports
    templates/s and the whitened-power difference from the FP32-storage path on the
    true orbits (the FP64-oracle comparison is in the GPU tests)."""
    import torch
    w = synth.elliptical_imbh()
    bid = ctx.load_bank(w.bank)
    sid16 = ctx.load_series(w.series, w.tsamp, bps.BPS_F16_SCALED)
    prm = bps.default_params(cand_cap=1 << 22)
    best, _ = ctx.autotune(sid16, bid, prm, sample_templates=32)
    st = torch.cuda.Stream()
    ms = []
    for i in range(warmup + steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st.synchronize()
        e0.record(st)
        rid = ctx.search(sid16, bid, prm, stream=st)
        e1.record(st)
        c, total = ctx.fetch_candidates(rid, allow_overflow=True)
        ctx.unload(rid)
        if i >= warmup:
            ms.append(e0.elapsed_time(e1))
    sid32 = ctx.load_series(w.series, w.tsamp)
    err = 0.0
    for ti in w.true_idx:
        a = ctx.whitened_spectrum(sid16, bid, int(ti), 1, w.n)[0]
        b = ctx.whitened_spectrum(sid32, bid, int(ti), 1, w.n)[0]
        err = max(err, float(np.max(np.abs(a - b) / np.maximum(1.0, b))))
    for x in (sid16, sid32, bid):
        ctx.unload(x)
    K = w.bank.shape[0]
    return {"workload": "elliptical IMBH: 2^25 samples x 128 us, %d templates (Porb U[5T,10T], "
                        "tau U[0,20] lt-s, e U[0,0.1]), FP16 series + scale per 4096, FP32 FFT" % K,
            "value": K / (statistics.mean(ms) / 1e3), "unit": UNIT,
            "ms_per_step": statistics.mean(ms), "steps": steps, "warmup": warmup,
            "autotuned": [best.log_tile, best.log_tile2, best.batch, best.log_cols],
            "candidates": int(total),
            "pw_max_rel_diff_vs_fp32_storage": err}


def config_of(w, args, ws):
    return {"workload": "HTRU-like circular search: 2^%d samples @ 64 us, %d circular templates "
                        "(Porb U[3T,10T], tau U[0,3] lt-s), 16 harmonics, 6 sigma, "
                        "3 injected P-BH pulsars" % (args.logn, args.templates),
            "n_samples": 1 << args.logn, "tsamp_s": w.tsamp, "templates_per_gpu": args.templates,
            "global_templates": args.templates * ws, "nharm_max": 16, "whiten_block": 1024,
            "sigma": 6.0, "parallelism": "template shards, replicas" if ws > 1 else "1 GPU",
            "l2": "flushed between timed steps (256 MiB write)"}


def main():
    args = parse()
    ws, rank, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    import torch

    import paper_2112_11991_b300 as bps
    from paper_2112_11991_b300 import build
    if rank == 0 or ws == 1:
        build.build()
    barrier(ws)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w, bank = workload(args, ws, rank)
    n = w.n
    K = bank.shape[0]
    ctx = bps.Context(local)
    # a real stream: the library runs on the stream it is given, and the CUDA events
    # below are recorded on the same one
    stream = torch.cuda.Stream(dev)
    sdt = bps.BPS_F16_SCALED if args.dtype == "f16" else bps.BPS_F32
    sid = ctx.load_series(w.series, w.tsamp, sdt)
    bid = ctx.load_bank(bank)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    # launch shapes of the fused form chosen by the library's autotuner on 64 templates
    tuned = None
    if (args.batch == 0 and args.log_tile == 0 and args.log_tile2 == 0 and args.log_cols == 0
            and args.pass1_kind == 0 and args.pass2_kind == 0 and args.power_layout == 0):
        best, ms_t = ctx.autotune(sid, bid, bps.default_params(cand_cap=CAND_CAP),
                                  sample_templates=min(64, K))
        tuned = {"log_tile": best.log_tile, "log_tile2": best.log_tile2, "batch": best.batch,
                 "log_cols": best.log_cols, "pass1_kind": best.pass1_kind,
                 "pass2_kind": best.pass2_kind,
                 "power_layout": best.power_layout,
                 "ms_per_template_sample": ms_t}

    def timed_steps(mode, steps, warmup, profile):
        prm = bps.default_params(mode=mode, batch=args.batch if mode == 0 else 0,
                                 cand_cap=CAND_CAP, log_tile=args.log_tile,
                                 log_tile2=args.log_tile2,
                                 log_cols=args.log_cols if mode == 0 else 0,
                                 pass1_kind=args.pass1_kind if mode == 0 else 0,
                                 pass2_kind=args.pass2_kind if mode == 0 else 0,
                                 power_layout=args.power_layout if mode == 0 else 0)
        ctx.set_profiling(False)
        for _ in range(warmup):
            rid = ctx.search(sid, bid, prm, stream=stream)
            ctx.fetch_candidates(rid, cap=0, allow_overflow=True)
            ctx.unload(rid)
        ctx.set_profiling(profile)
        ms, stats, ncand = [], [], 0
        barrier(ws)
        torch.cuda.synchronize(dev)
        for _ in range(steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            rid = ctx.search(sid, bid, prm, stream=stream)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
            stats.append(ctx.request_stats(rid))
            _, tot = ctx.fetch_candidates(rid, cap=0, allow_overflow=True)
            ncand = tot
            ctx.unload(rid)
        torch.cuda.synchronize(dev)
        barrier(ws)
        ctx.set_profiling(False)
        return ms, stats, ncand

    clocks = ClockSampler(local)
    clocks.start()
    ms, stats, ncand = timed_steps(0, args.steps, args.warmup, True)
    clk = clocks.stop()
    total_s = allmax(ws, sum(ms) / 1e3)
    value = K * ws * args.steps / total_s

    plain = None
    if not args.no_plain:
        pms, pstats, pc = timed_steps(1, max(2, min(args.steps, 3)), 1, True)
        ptot = allmax(ws, sum(pms) / 1e3)
        plain = {"value": K * ws * len(pms) / ptot, "unit": UNIT,
                 "ms_per_step": statistics.mean(pms), "candidates": pc,
                 "stage_ms_per_step": {k: sum(s["stage_ms"][k] for s in pstats) / len(pstats)
                                       for k in bps.STAGES},
                 "form": "index map + gather kernel -> cuFFT R2C -> power -> same median/harmonic-sum kernels, one template per launch"}

    # the mixed-precision form at the same request: the series stored FP16 with a
    # power-of-two scale per 4096 samples, FP32 FFT arithmetic (same kernels and shape)
    f16 = None
    if args.dtype == "f32" and not args.no_f16:
        sid16 = ctx.load_series(w.series, w.tsamp, bps.BPS_F16_SCALED)
        sid_main = sid
        sid = sid16
        hms, hstats, hc = timed_steps(0, args.steps, 2, True)
        sid = sid_main
        htot = allmax(ws, sum(hms) / 1e3)
        f16 = {"value": K * ws * len(hms) / htot, "unit": UNIT, "ms_per_step": statistics.mean(hms),
               "candidates": hc, "storage": "FP16 + power-of-two FP32 scale per 4096 samples",
               "arithmetic": "f32",
               "stage_ms_per_step": {k: sum(s_["stage_ms"][k] for s_ in hstats) / len(hstats)
                                     for k in bps.STAGES},
               "speedup_vs_plain": None, "speedup_vs_f32_storage": None}
        f16["speedup_vs_f32_storage"] = f16["value"] / value
        if plain:
            f16["speedup_vs_plain"] = f16["value"] / plain["value"]

    # end to end through the public API with host buffers: pinned series H2D, bank, search,
    # candidate D2H, unload -- every step.
    pinned = torch.from_numpy(w.series).pin_memory()
    e2e_ms = []
    d2h = 0
    prm = bps.default_params(batch=args.batch, cand_cap=CAND_CAP, log_tile=args.log_tile,
                             log_tile2=args.log_tile2, log_cols=args.log_cols,
                             pass1_kind=args.pass1_kind, pass2_kind=args.pass2_kind,
                             power_layout=args.power_layout)
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        s2 = ctx.load_series(pinned, w.tsamp, sdt)
        b2 = ctx.load_bank(bank)
        rid = ctx.search(s2, b2, prm, stream=stream)
        c, tot = ctx.fetch_candidates(rid, allow_overflow=True)
        ctx.unload(rid)
        ctx.unload(s2)
        ctx.unload(b2)
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e_ms.append(1e3 * (t1 - t0))
            d2h = c.nbytes + 8
    e2e_tot = allmax(ws, sum(e2e_ms) / 1e3)
    e2e = {"value": K * ws * len(e2e_ms) / e2e_tot, "unit": UNIT,
           "h2d_bytes_per_step": int(w.series.nbytes + bank.nbytes),
           "d2h_bytes_per_step": int(d2h),
           "ms_per_step": statistics.mean(e2e_ms),
           "p50_ms": float(np.percentile(e2e_ms, 50)), "p99_ms": float(np.percentile(e2e_ms, 99))}

    # roofline of the dominant kernel from the live stage events of the timed steps
    peak, peak_kind = peaks()
    stage_ms = {k: sum(s["stage_ms"][k] for s in stats) for k in bps.STAGES}
    stage_launch = {k: sum(s["stage_launches"][k] for s in stats) for k in bps.STAGES}
    dom = max(stage_ms, key=stage_ms.get)
    batch = stats[0]["batch"]
    per_launch_ms = stage_ms[dom] / max(1, stage_launch[dom])
    alg_bytes = STAGE_BYTES_PER_N[dom] * n * batch
    achieved = alg_bytes / (per_launch_ms * 1e-3) / 1e9
    if tuned:
        geom = geometry_key(args.logn, tuned["log_cols"], tuned["log_tile"], tuned["log_tile2"],
                            tuned["pass1_kind"], tuned["pass2_kind"])
    else:
        geom = geometry_key(args.logn, args.log_cols, args.log_tile, args.log_tile2,
                            args.pass1_kind, args.pass2_kind)
    traffic = ncu_traffic(dom, "htru_2p%d" % args.logn, batch, geom)
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
            "launch_shape": geom,
            "alg_bytes_per_launch": alg_bytes, "templates_per_launch": batch,
            "ms_per_launch": per_launch_ms}
    path_gbs = PATH_BYTES_PER_N * n * K * args.steps / (sum(ms) / 1e3) / 1e9
    two_pass_gbs = TWO_PASS_BYTES_PER_N * n * K * args.steps / (sum(ms) / 1e3) / 1e9
    # DRAM bytes the four kernels move per template (the committed ncu rows of this launch
    # shape, when all are current) over the whole step's time
    per_t = [ncu_traffic(k, "htru_2p%d" % args.logn, 1, geom)
             for k in ("pass1", "pass2", "median", "harmsum")]
    path_dram = None
    if all(v is not None for v in per_t):
        dram_gbs = sum(per_t) * K * args.steps / (sum(ms) / 1e3) / 1e9
        path_dram = {"dram_bytes_per_template": sum(per_t), "achieved": dram_gbs, "peak": peak,
                     "unit": "GB/s", "frac": dram_gbs / peak,
                     "source": "profiles/traffic.json rows of launch shape " + geom}
    stage_share = {k: v / max(1e-9, sum(stage_ms.values())) for k, v in stage_ms.items()}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        thr = cpu_threads(args)
        nt = args.cpu_templates or thr
        sel = np.linspace(0, K - 1, nt).astype(int)
        rate, dt = oracle_rate(w.series, w.tsamp, bank[sel], thr)
        cpu = {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": "%d of %d templates of the 2^%d-sample workload (%.1f s)" % (
                   nt, K, args.logn, dt)}
        if f16 is not None:
            f16["error_vs_oracle"] = f16_oracle_error(ctx, sid16, bid, w, bank)

    serving = None
    if not args.no_serving and ws == 1:
        pool = serving_pool()
        sweep = []
        for r in [float(v) for v in args.serve_rates.split(",") if v]:
            sweep.append(run_serving(bps, ctx, r, max(8, int(r * args.serve_seconds)), pool))
        serving = {"workload": SERVING_WORKLOAD, "sweep": sweep}
    uneven = run_uneven(bps, ctx) if (not args.no_uneven and ws == 1) else None
    elliptical = run_elliptical_f16(bps, ctx) if (not args.no_elliptical and ws == 1) else None

    launches = sum(s["launches"] for s in stats)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": statistics.mean(ms), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.dtype == "f32" else "f16-storage/f32",
           "data": "synthetic (seeded noise + injected pulsars)",
           "config": config_of(w, args, ws),
           "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
           "plain_form": plain,
           "speedup_vs_plain": (value / plain["value"]) if plain else None,
           "f16_headline": f16,
           "roofline": roof,
           "path_roofline": {"achieved": path_gbs, "peak": peak, "unit": "GB/s",
                             "frac": path_gbs / peak, "alg_bytes_per_template": PATH_BYTES_PER_N * n},
           "two_pass_roofline": {"achieved": two_pass_gbs, "peak": peak, "unit": "GB/s",
                                 "frac": two_pass_gbs / peak,
                                 "alg_bytes_per_template": TWO_PASS_BYTES_PER_N * n},
           "path_dram": path_dram,
           "stage_ms_per_step": {k: v / args.steps for k, v in stage_ms.items()},
           "stage_share": stage_share,
           "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": launches,
           "candidates_per_step": ncand, "anchor_block": stats[0]["anchor_block"],
           "serving": serving, "batched_uneven": uneven, "elliptical_f16": elliptical,
           "autotuned": tuned}
    if rank == 0:
        print(json.dumps(out), flush=True)
    ctx.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
