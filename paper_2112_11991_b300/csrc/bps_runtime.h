// bps_runtime.h -- host runtime internals shared by the C-ABI translation units
// (bps_api.cu: contexts, searches, graphs, autotuner, stage entry points; bps_server.cu:
// the serving loop): device-resident series and banks, request records, the planner,
// workspaces and the batched search job.
#pragma once

#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <array>
#include <map>
#include <mutex>
#include <memory>
#include <string>
#include <vector>

#include "../../include/bps.h"
#include "bps_internal.cuh"
#include "dev_template.h"

namespace bps {
namespace rt {


struct Series {
    int64_t n = 0;
    double tsamp = 0;
    int dtype = BPS_F32;
    float* f32 = nullptr;
    bool owned = false;
    uint16_t* f16 = nullptr;
    float* scale = nullptr;
    double mean = 0;
    double* d_sum = nullptr;  // FP64 sum of the samples (device)
    float* d_fill = nullptr;  // fill value (the mean) on the device, read by the gather
};

struct Bank {
    int64_t K = 0;
    DevTemplate* d = nullptr;
    std::vector<bps_template> h;
};


struct Request {
    int64_t series = 0, bank = 0, K = 0;
    int32_t batch = 0, logB = 0, launches = 0;
    int32_t stage_launches[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;  // (stage, start/stop)
    cudaEvent_t done = nullptr;
    Cand* d_cands = nullptr;
    unsigned long long* d_count = nullptr;
    int64_t cap = 0;
    bool synced = false;
    unsigned long long total = 0;
    unsigned long long status = 0;  // non-zero: a bounded device wait expired (bit 0 harmonic
                                    // sum, bit 1 warp-specialised pass 1, bit 2 TMA-fed pass 2)
    std::vector<bps_candidate> result;
};

struct FftKey {
    int64_t n;
    int nt;
    bool operator<(const FftKey& o) const { return n < o.n || (n == o.n && nt < o.nt); }
};


struct GraphObj;

}  // namespace rt
}  // namespace bps

struct bps_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    // stream-ordered device memory of workspaces and candidate buffers: a pool of the
    // context that keeps what is freed (release threshold: never), so after the first
    // request of a size no allocation reaches the driver
    cudaMemPool_t pool = nullptr;
    std::vector<cudaEvent_t> free_events;  // completion events for reuse
    std::recursive_mutex mu;
    std::string err = "";
    int64_t next_id = 1;
    std::map<int64_t, bps::rt::Series> series;
    std::map<int64_t, bps::rt::Bank> banks;
    std::map<int64_t, bps::rt::Request> reqs;
    std::map<bps::rt::FftKey, cufftHandle> ffts;
    float2* tw = nullptr;
    bool profiling = false;
    // autotuned launch shapes per (log2 n, mode, log2 nharm): tile1, tile2, batch, log C,
    // pass-1 kind, power layout, pass-2 kind
    std::map<int, std::array<int, 7>> tuned;
    std::map<int64_t, bps::rt::GraphObj*> graphs;
};

namespace bps {
namespace rt {


inline int fail(bps_ctx* c, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? BPS_ERR_OUT_OF_MEMORY     \
                                                             : BPS_ERR_CUDA,             \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,       \
                        __LINE__);                                                       \
    } while (0)

inline int ilog2(int64_t v)
{
    int l = 0;
    while ((1ll << l) < v) ++l;
    return l;
}

inline bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

// Gamma(n, 1) upper tail  Q(n, x) = e^{-x} sum_{m<n} x^m / m!  (chi^2 with 2n dof / 2).
inline double q_gamma(int n, double x)
{
    double term = 1.0, sum = 1.0;
    for (int m = 1; m < n; ++m) {
        term *= x / m;
        sum += term;
    }
    return std::exp(-x) * sum;
}

// Solve Q(n, x) = p (p in (0, 1)): Newton on log Q with a bisection bracket.
inline double solve_threshold(int n, double p)
{
    double lo = 0.0, hi = 1.0;
    while (q_gamma(n, hi) > p) hi *= 2.0;
    double x = 0.5 * (lo + hi);
    const double lp = std::log(p);
    for (int it = 0; it < 200; ++it) {
        const double q = q_gamma(n, x);
        if (q > p) lo = x; else hi = x;
        // d/dx log Q = -x^{n-1} e^{-x} / ((n-1)! Q)
        double dens = std::exp(-x + (n - 1) * std::log(std::max(x, 1e-300)) - std::lgamma((double)n));
        double step = (std::log(q) - lp) / (dens / q);
        double xn = x + step;
        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        if (std::fabs(xn - x) < 1e-13 * std::max(1.0, x)) {
            x = xn;
            break;
        }
        x = xn;
    }
    return x;
}

inline int check_params(bps_ctx* ctx, const bps_search_params* pr, int64_t n)
{
    if (!pr) return fail(ctx, BPS_ERR_INVALID_ARG, "params is NULL");
    if (!(pr->nharm_max == 1 || pr->nharm_max == 2 || pr->nharm_max == 4 ||
          pr->nharm_max == 8 || pr->nharm_max == 16))
        return fail(ctx, BPS_ERR_INVALID_ARG, "nharm_max must be 1, 2, 4, 8 or 16");
    if (!is_pow2(pr->whiten_block) || pr->whiten_block < 32 || pr->whiten_block > 8192 ||
        pr->whiten_block > n / 2)
        return fail(ctx, BPS_ERR_INVALID_ARG, "whiten_block must be a power of two in [32, min(8192, n/2)]");
    if (!pr->auto_thr && !(pr->sigma_thr > 0.0 && pr->sigma_thr < 38.0))
        return fail(ctx, BPS_ERR_INVALID_ARG, "sigma_thr must be in (0, 38)");
    if (pr->cand_cap < 1) return fail(ctx, BPS_ERR_INVALID_ARG, "cand_cap must be >= 1");
    if (pr->mode != BPS_MODE_FUSED && pr->mode != BPS_MODE_PLAIN)
        return fail(ctx, BPS_ERR_INVALID_ARG, "unknown mode %d", pr->mode);
    if (pr->batch < 0) return fail(ctx, BPS_ERR_INVALID_ARG, "batch must be >= 0");
    if ((pr->log_tile != 0 && pr->log_tile != 13 && pr->log_tile != 14) ||
        (pr->log_tile2 != 0 && (pr->log_tile2 < 12 || pr->log_tile2 > 14)))
        return fail(ctx, BPS_ERR_INVALID_ARG, "log_tile must be 0, 13 or 14, log_tile2 0 or 12..14");
    if (pr->log_cols != 0 && !log_cols_ok(ilog2(n) - 1, pr->log_cols))
        return fail(ctx, BPS_ERR_INVALID_ARG, "log_cols %d is not a valid split of %lld samples",
                    pr->log_cols, (long long)n);
    if (pr->pass1_kind < BPS_PASS1_AUTO || pr->pass1_kind > BPS_PASS1_ASYNC)
        return fail(ctx, BPS_ERR_INVALID_ARG, "unknown pass1_kind %d", pr->pass1_kind);
    if (pr->power_layout < BPS_POWER_AUTO || pr->power_layout > BPS_POWER_ROWS)
        return fail(ctx, BPS_ERR_INVALID_ARG, "unknown power_layout %d", pr->power_layout);
    if (pr->pass2_kind < BPS_PASS2_AUTO || pr->pass2_kind > BPS_PASS2_TMA)
        return fail(ctx, BPS_ERR_INVALID_ARG, "unknown pass2_kind %d", pr->pass2_kind);
    return BPS_OK;
}

inline void thresholds(const bps_search_params* pr, int64_t n, int64_t K, double* out)
{
    const int nlev = ilog2(pr->nharm_max) + 1;
    double sigma = pr->sigma_thr;
    if (pr->auto_thr) {
        // S/N_min of Sec. 2.1 with n_trials = n_samp/2 bins * levels * orbital templates
        const double ntr = (double)(n / 2) * nlev * (double)std::max<int64_t>(K, 1);
        sigma = (std::sqrt(std::log(ntr)) - std::sqrt(M_PI / 4.0)) / std::sqrt(1.0 - M_PI / 4.0);
    }
    const double p = 0.5 * std::erfc(sigma / std::sqrt(2.0));
    for (int L = 0; L < nlev; ++L) out[L] = solve_threshold(1 << L, p);
}

inline int tune_key(int logn, int mode, int lognh) { return (logn << 8) | (mode << 4) | lognh; }

// Geometry (plan_geometry) + anchor block length (plan_anchor_block).  Tiles not given in
// the parameters come from the context's autotuned entry for this size, else 14 / 13.
inline int make_plan(bps_ctx* ctx, const Series& s, const Bank& b, const bps_search_params& pr,
              Plan& p)
{
    p.n = s.n;
    p.logn = ilog2(s.n);
    p.M = s.n / 2;
    p.logM = p.logn - 1;
    int t1 = 14, t2 = 13, lc = 0, p1k = BPS_PASS1_FUSED, pl = BPS_POWER_AUTO, p2k = BPS_PASS2_FUSED;
    bool tuned = false;
    if (ctx) {
        auto it = ctx->tuned.find(tune_key(ilog2(s.n), pr.mode, ilog2(pr.nharm_max)));
        if (it != ctx->tuned.end()) {
            t1 = it->second[0];
            t2 = it->second[1];
            lc = it->second[3];
            p1k = it->second[4];
            pl = it->second[5];
            p2k = it->second[6];
            tuned = true;
        }
    }
    plan_geometry(p, pr.log_tile ? pr.log_tile : t1, pr.log_tile2 ? pr.log_tile2 : t2,
                  pr.log_cols ? pr.log_cols : lc);
    p.logW = ilog2(pr.whiten_block);
    // pass-1 organisation: the caller's, else the autotuned one (when the caller left the
    // split and tiles to the library too), else the one-phase kernel
    int kind = pr.pass1_kind;
    if (kind == BPS_PASS1_AUTO)
        kind = (tuned && !pr.log_cols && !pr.log_tile) ? p1k : BPS_PASS1_FUSED;
    if (pr.mode == BPS_MODE_FUSED && (kind == BPS_PASS1_WARPSPEC || kind == BPS_PASS1_ASYNC)) {
        if (!ws_pass1_built(p.logR, p.logC)) {
            if (pr.pass1_kind == kind)
                return fail(ctx, BPS_ERR_INVALID_ARG,
                            "this pass-1 form is not built for R = 2^%d, C = 2^%d", p.logR, p.logC);
        } else if (kind == BPS_PASS1_WARPSPEC) {
            p.p1ws = 1;
        } else {
            p.p1async = 1;
        }
    }
    // pass-2 organisation, chosen like pass 1's
    int kind2 = pr.pass2_kind;
    if (kind2 == BPS_PASS2_AUTO)
        kind2 = (tuned && !pr.log_cols && !pr.log_tile2) ? p2k : BPS_PASS2_FUSED;
    if (pr.mode == BPS_MODE_FUSED && kind2 == BPS_PASS2_TMA) {
        if (!tma_pass2_built(p.logR, p.logC, p.logTile2)) {
            if (pr.pass2_kind == BPS_PASS2_TMA)
                return fail(ctx, BPS_ERR_INVALID_ARG,
                            "the TMA-fed pass 2 is built for 2^13 tiles and R, C in 2^10..2^12");
        } else {
            p.p2tma = 1;
        }
    }
    // row-major power (in groups of NP rows) when a pass-2 CTA holds at most two row pairs,
    // whose bin-order stores would be runs of one or two words, a whitening block lies
    // within one k2 (W <= R) and the warp median applies (W <= 1024).  Measured at 2^23,
    // C = 2048: NP = 2 pass 2 + median 14.5 + 7.7 us (bin order 21.1 + 5.4); NP = 4
    // 17.0 + 7.4 (bin order 18.5 + 5.4).
    const bool rows_ok = pr.mode == BPS_MODE_FUSED && p.logW <= 10 && p.logW <= p.logR && p.logNP <= 1;
    int layout = pr.power_layout;
    if (layout == BPS_POWER_AUTO && tuned && !pr.log_cols && !pr.log_tile2) layout = pl;
    if (layout == BPS_POWER_ROWS && !rows_ok) {
        if (pr.power_layout == BPS_POWER_ROWS)
            return fail(ctx, BPS_ERR_INVALID_ARG,
                        "row-major power needs at most two row pairs per pass-2 CTA, W <= R and W <= 1024");
        layout = BPS_POWER_AUTO;
    }
    p.ptrans = layout == BPS_POWER_BINS ? 0 : (layout == BPS_POWER_ROWS ? 1 : (rows_ok ? 1 : 0));
    p.nharm = pr.nharm_max;
    p.lognh = ilog2(pr.nharm_max);
    p.nlev = p.lognh + 1;
    p.tsamp = s.tsamp;
    p.inv_tsamp = 1.0 / s.tsamp;
    // per template: K = tau/t_s, g = Omega t_s / (1 - e) (bound on dE/dsample)
    double kg1 = 0.0, kg2 = 0.0, kg4 = 0.0, Kmax = 0.0, gmax = 0.0;
    for (const auto& t : b.h) {
        const double K = t.tau_lts / s.tsamp;
        const double g = (2.0 * M_PI / t.porb_s) * s.tsamp / (1.0 - t.ecc);
        kg1 = std::max(kg1, K * g);
        kg2 = std::max(kg2, K * g * g);
        kg4 = std::max(kg4, K * g * g * g * g);
        Kmax = std::max(Kmax, K);
        gmax = std::max(gmax, K > 0 ? g : 0.0);
    }
    const int logB = plan_anchor_block(kg1, kg2, kg4, p.logn);
    if (logB < 6)
        return fail(ctx, BPS_ERR_UNSUPPORTED,
                    "orbit too fast for the FP32 index map (tau/t_s = %.3g, Omega t_s/(1-e) = %.3g)",
                    Kmax, gmax);
    p.logB = logB;
    p.nanchor = s.n >> logB;
    return BPS_OK;
}

inline SeriesView view_of(const Series& s)
{
    SeriesView v;
    v.f32 = s.dtype == BPS_F32 ? s.f32 : nullptr;
    v.f16 = s.dtype == BPS_F16_SCALED ? s.f16 : nullptr;
    v.scale = s.scale;
    v.uscalep = s.scale ? s.scale + ((s.n + 4095) >> 12) : nullptr;
    v.uscale = 0.f;
    v.fill = (float)s.mean;
    v.fillp = s.d_fill;
    return v;
}

inline int default_batch(const Plan& p, int64_t K, int mode)
{
    if (mode == BPS_MODE_PLAIN) return 1;
    int64_t nt = std::max<int64_t>(1, (1ll << 27) / p.M);
    nt = std::min<int64_t>(nt, 64);
    return (int)std::min<int64_t>(nt, std::max<int64_t>(K, 1));
}

struct Workspace {
    Anchor* anc = nullptr;
    float2* Y = nullptr;   // fused: M complex per template; plain: R2C output (M+1)
    float* x = nullptr;    // plain: resampled series
    float* P = nullptr;    // power, then the whitened power, in bin order
    float* Pt = nullptr;   // power in pass 2's row-major-by-k1 layout (plan.ptrans)
    float* scale = nullptr;
    unsigned int* tile_ctr = nullptr;  // the harmonic sum's tile counter
    char* base = nullptr;
};

inline size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Fetch order of candidates: (template_idx, nharm, bin), deterministic whatever the order
// in which the device appended them.
inline void sort_candidates(std::vector<bps_candidate>& c)
{
    std::sort(c.begin(), c.end(), [](const bps_candidate& a, const bps_candidate& b) {
        if (a.template_idx != b.template_idx) return a.template_idx < b.template_idx;
        if (a.nharm != b.nharm) return a.nharm < b.nharm;
        return a.bin < b.bin;
    });
}

// Anchors are computed for a chunk of up to kAnchorChunk batches in one launch.
constexpr int kAnchorChunk = 8;

// Carve a workspace for batches of nt templates (anchors for anchor_templates) out of base.
inline size_t ws_carve(const Plan& p, int nt, int mode, int anchor_templates, char* base, Workspace* w)
{
    const size_t a = align256(sizeof(Anchor) * (size_t)p.nanchor *
                              (anchor_templates > 0 ? anchor_templates : nt));
    const size_t y = align256(sizeof(float2) * (size_t)(p.M + 1) * nt);
    const size_t x = mode == BPS_MODE_PLAIN ? align256(sizeof(float) * (size_t)p.n * nt) : 0;
    const size_t pp = align256(sizeof(float) * (size_t)p.M * nt);
    const size_t pt = p.ptrans ? pp : 0;
    const size_t sc = align256(sizeof(float) * (size_t)(p.M >> p.logW) * nt);
    const size_t tc = 256;
    if (w) {
        char* q = base;
        w->base = base;
        w->anc = (Anchor*)q; q += a;
        w->Y = (float2*)q; q += y;
        w->x = x ? (float*)q : nullptr; q += x;
        w->P = (float*)q; q += pp;
        w->Pt = pt ? (float*)q : nullptr; q += pt;
        w->scale = (float*)q; q += sc;
        w->tile_ctr = (unsigned int*)q;
    }
    return a + y + x + pp + pt + sc + tc;
}

// Stream-ordered allocation from the context's pool.
inline cudaError_t pool_alloc(bps_ctx* ctx, void** p, size_t bytes, cudaStream_t st)
{
    return cudaMallocFromPoolAsync(p, bytes, ctx->pool, st);
}

// A completion event from the context's free list (created when the list is empty).
inline cudaError_t event_get(bps_ctx* ctx, cudaEvent_t* e)
{
    if (!ctx->free_events.empty()) {
        *e = ctx->free_events.back();
        ctx->free_events.pop_back();
        return cudaSuccess;
    }
    return cudaEventCreateWithFlags(e, cudaEventDisableTiming);
}

inline void event_put(bps_ctx* ctx, cudaEvent_t e)
{
    if (e) ctx->free_events.push_back(e);
}

inline int ws_alloc(bps_ctx* ctx, const Plan& p, int nt, int mode, cudaStream_t st, Workspace& w,
             int anchor_templates = 0)
{
    char* base = nullptr;
    CK(pool_alloc(ctx, (void**)&base, ws_carve(p, nt, mode, anchor_templates, nullptr, nullptr), st));
    ws_carve(p, nt, mode, anchor_templates, base, &w);
    return BPS_OK;
}

inline int get_fft(bps_ctx* ctx, int64_t n, int nt, cufftHandle& h)
{
    auto it = ctx->ffts.find({n, nt});
    if (it != ctx->ffts.end()) {
        h = it->second;
        return BPS_OK;
    }
    long long nn[1] = {n};
    size_t wsz = 0;
    cufftResult r = cufftCreate(&h);
    if (r == CUFFT_SUCCESS)
        r = cufftMakePlanMany64(h, 1, nn, nullptr, 1, n, nullptr, 1, n / 2 + 1, CUFFT_R2C, nt, &wsz);
    if (r != CUFFT_SUCCESS) return fail(ctx, BPS_ERR_CUDA, "cuFFT plan failed (%d)", (int)r);
    ctx->ffts[{n, nt}] = h;
    return BPS_OK;
}

// Optional per-stage CUDA-event timing of a request.
struct StageTimer {
    Request* r = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr;
    int stage = 0;
    void begin(int s_)
    {
        stage = s_;
        if (r) r->stage_launches[s_] += 1, r->launches += 1;
        if (!r || !prof) return;
        cudaEventCreate(&a);
        cudaEventRecord(a, st);
    }
    void end()
    {
        if (!r || !prof) return;
        cudaEvent_t b;
        cudaEventCreate(&b);
        cudaEventRecord(b, st);
        r->ev.push_back({stage, {a, b}});
    }
    bool prof = false;
};

// Runs the spectrum stages for templates [t0, t0+nt): anchors -> (fused) pass1/pass2
// or (plain) resample/cuFFT/power -> block medians.  P and scale are left in w.
inline int run_spectrum(bps_ctx* ctx, const Series& s, const Bank& b, const Plan& p, int mode,
                 int64_t t0, int nt, Workspace& w, cudaStream_t st, StageTimer& tm,
                 unsigned long long* status, const Anchor* anc = nullptr)
{
    if (!anc) {
        tm.begin(BPS_STAGE_ANCHORS);
        CK(launch_anchors(b.d, t0, nt, p, w.anc, st));
        tm.end();
        anc = w.anc;
    }
    const SeriesView v = view_of(s);
    if (mode == BPS_MODE_FUSED) {
        tm.begin(BPS_STAGE_PASS1);
        CK(launch_pass1(v, anc, nt, p, ctx->tw, w.Y, status, st));
        tm.end();
        tm.begin(BPS_STAGE_PASS2);
        CK(launch_pass2(w.Y, nt, p, ctx->tw, p.ptrans ? w.Pt : w.P, status, st));
        tm.end();
    } else {
        cufftHandle h;
        int rc = get_fft(ctx, p.n, nt, h);
        if (rc) return rc;
        tm.begin(BPS_STAGE_PASS1);
        CK(launch_resample(v, anc, nt, p, w.x, st));
        tm.end();
        cufftSetStream(h, st);
        tm.begin(BPS_STAGE_PASS2);
        if (cufftExecR2C(h, w.x, (cufftComplex*)w.Y) != CUFFT_SUCCESS)
            return fail(ctx, BPS_ERR_CUDA, "cufftExecR2C failed");
        tm.end();
        tm.begin(BPS_STAGE_POWER);
        CK(launch_power_from_r2c(w.Y, nt, p, w.P, st));
        tm.end();
    }
    tm.begin(BPS_STAGE_MEDIAN);
    CK(launch_block_median(w.P, nt, p, w.scale, st, p.ptrans ? w.Pt : nullptr));
    tm.end();
    return BPS_OK;
}

// One search in progress: issues its launch groups (FP64 anchors once per chunk of
// kAnchorChunk batches, then pass 1, pass 2, median/whitening and harmonic sum of one
// batch of templates) one group at a time on its stream.
struct Job {
    bps_ctx* ctx = nullptr;
    const Series* s = nullptr;
    const Bank* b = nullptr;
    Plan p;
    int mode = BPS_MODE_FUSED;
    Thr th;
    int nt = 1;
    int64_t chunk = 1;
    Workspace w;
    cudaStream_t st = nullptr;
    Cand* cands = nullptr;
    unsigned long long* count = nullptr;
    int64_t cap = 0;
    int64_t c0 = -1, ccnt = 0, t0 = 0;
    StageTimer tm;

    bool done() const { return t0 >= b->K; }

    // plan, thresholds and workspace (stream-ordered allocation on st)
    bool owns_ws = true;

    // external: carve the workspace from this buffer (ext_bytes long) instead of allocating
    int setup(bps_ctx* c, const Series* s_, const Bank* b_, const bps_search_params& prm,
              cudaStream_t stream, Cand* cd, unsigned long long* cnt, int64_t cp,
              char* external = nullptr, size_t ext_bytes = 0)
    {
        ctx = c;
        s = s_;
        b = b_;
        st = stream;
        cands = cd;
        count = cnt;
        cap = cp;
        mode = prm.mode;
        int rc = make_plan(ctx, *s, *b, prm, p);
        if (rc) return rc;
        double thr[5];
        thresholds(&prm, s->n, b->K, thr);
        for (int L = 0; L < 5; ++L) th.v[L] = L < p.nlev ? (float)thr[L] : 0.f;
        nt = prm.batch > 0 ? (int)std::min<int64_t>(prm.batch, b->K) : default_batch(p, b->K, mode);
        if (prm.batch == 0 && ctx) {
            auto it = ctx->tuned.find(tune_key(p.logn, mode, p.lognh));
            if (it != ctx->tuned.end()) nt = (int)std::min<int64_t>(it->second[2], b->K);
        }
        chunk = std::min<int64_t>((int64_t)nt * kAnchorChunk, b->K);
        if (external) {
            if (ws_carve(p, nt, mode, (int)chunk, nullptr, nullptr) > ext_bytes)
                return fail(ctx, BPS_ERR_INVALID_ARG, "workspace too small");
            ws_carve(p, nt, mode, (int)chunk, external, &w);
            owns_ws = false;
            return BPS_OK;
        }
        return ws_alloc(ctx, p, nt, mode, st, w, (int)chunk);
    }

    // device bytes of the workspace setup() allocates (the carve's own count, so the
    // row-major power buffer of plan.ptrans is included)
    static size_t workspace_bytes(const Plan& p, int nt, int64_t chunk, int mode)
    {
        return ws_carve(p, nt, mode, (int)chunk, nullptr, nullptr);
    }

    int issue_batch()
    {
        if (c0 < 0 || t0 >= c0 + ccnt) {
            c0 = t0;
            ccnt = std::min<int64_t>(chunk, b->K - c0);
            tm.begin(BPS_STAGE_ANCHORS);
            cudaError_t e = launch_anchors(b->d, c0, (int)ccnt, p, w.anc, st);
            tm.end();
            if (e != cudaSuccess)
                return fail(ctx, BPS_ERR_CUDA, "anchor launch: %s", cudaGetErrorString(e));
        }
        const int cnt = (int)std::min<int64_t>(nt, c0 + ccnt - t0);
        int rc = run_spectrum(ctx, *s, *b, p, mode, t0, cnt, w, st, tm, count + 1,
                              w.anc + (t0 - c0) * p.nanchor);
        if (rc) return rc;
        tm.begin(BPS_STAGE_HARMSUM);
        cudaError_t e = launch_harmsum(w.P, w.scale, cnt, t0, p, th, cands, cap, count, nullptr,
                                       w.tile_ctr, st);
        tm.end();
        if (e != cudaSuccess)
            return fail(ctx, BPS_ERR_CUDA, "harmonic-sum launch: %s", cudaGetErrorString(e));
        t0 += cnt;
        return BPS_OK;
    }

    void release()
    {
        if (w.base && owns_ws) cudaFreeAsync(w.base, st);
        w.base = nullptr;
    }
};


inline int lookup(bps_ctx* ctx, int64_t sid, int64_t bid, Series*& s, Bank*& b)
{
    auto si = ctx->series.find(sid);
    if (si == ctx->series.end()) return fail(ctx, BPS_ERR_INVALID_ARG, "unknown series id %lld", (long long)sid);
    auto bi = ctx->banks.find(bid);
    if (bi == ctx->banks.end()) return fail(ctx, BPS_ERR_INVALID_ARG, "unknown bank id %lld", (long long)bid);
    s = &si->second;
    b = &bi->second;
    return BPS_OK;
}


}  // namespace rt
}  // namespace bps
