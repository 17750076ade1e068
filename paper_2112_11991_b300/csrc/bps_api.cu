// bps_api.cu -- host runtime behind the C ABI of include/bps.h: contexts,
// device-resident series and banks, the planner, stream-ordered searches,
// candidate fetch, and the stage entry points.
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

using namespace bps;

namespace {

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
    unsigned long long status = 0;  // bit 0: a bounded device wait expired
    std::vector<bps_candidate> result;
};

struct FftKey {
    int64_t n;
    int nt;
    bool operator<(const FftKey& o) const { return n < o.n || (n == o.n && nt < o.nt); }
};

}  // namespace

namespace {
struct GraphObj;
}

struct bps_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::recursive_mutex mu;
    std::string err = "";
    int64_t next_id = 1;
    std::map<int64_t, Series> series;
    std::map<int64_t, Bank> banks;
    std::map<int64_t, Request> reqs;
    std::map<FftKey, cufftHandle> ffts;
    float2* tw = nullptr;
    bool profiling = false;
    // autotuned launch shapes per (log2 n, mode, log2 nharm): tile1, tile2, batch, log C
    std::map<int, std::array<int, 4>> tuned;
    std::map<int64_t, GraphObj*> graphs;
};

namespace {

int fail(bps_ctx* c, int code, const char* fmt, ...)
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

int ilog2(int64_t v)
{
    int l = 0;
    while ((1ll << l) < v) ++l;
    return l;
}

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

// Gamma(n, 1) upper tail  Q(n, x) = e^{-x} sum_{m<n} x^m / m!  (chi^2 with 2n dof / 2).
double q_gamma(int n, double x)
{
    double term = 1.0, sum = 1.0;
    for (int m = 1; m < n; ++m) {
        term *= x / m;
        sum += term;
    }
    return std::exp(-x) * sum;
}

// Solve Q(n, x) = p (p in (0, 1)): Newton on log Q with a bisection bracket.
double solve_threshold(int n, double p)
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

int check_params(bps_ctx* ctx, const bps_search_params* pr, int64_t n)
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
        (pr->log_tile2 != 0 && pr->log_tile2 != 13 && pr->log_tile2 != 14))
        return fail(ctx, BPS_ERR_INVALID_ARG, "log_tile and log_tile2 must be 0, 13 or 14");
    if (pr->log_cols != 0 && !log_cols_ok(ilog2(n) - 1, pr->log_cols))
        return fail(ctx, BPS_ERR_INVALID_ARG, "log_cols %d is not a valid split of %lld samples",
                    pr->log_cols, (long long)n);
    return BPS_OK;
}

void thresholds(const bps_search_params* pr, int64_t n, int64_t K, double* out)
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

int tune_key(int logn, int mode, int lognh) { return (logn << 8) | (mode << 4) | lognh; }

// Geometry (plan_geometry) + anchor block length (plan_anchor_block).  Tiles not given in
// the parameters come from the context's autotuned entry for this size, else 14 / 13.
int make_plan(bps_ctx* ctx, const Series& s, const Bank& b, const bps_search_params& pr,
              Plan& p)
{
    p.n = s.n;
    p.logn = ilog2(s.n);
    p.M = s.n / 2;
    p.logM = p.logn - 1;
    int t1 = 14, t2 = 13, lc = 0;
    if (ctx) {
        auto it = ctx->tuned.find(tune_key(ilog2(s.n), pr.mode, ilog2(pr.nharm_max)));
        if (it != ctx->tuned.end()) {
            t1 = it->second[0];
            t2 = it->second[1];
            lc = it->second[3];
        }
    }
    plan_geometry(p, pr.log_tile ? pr.log_tile : t1, pr.log_tile2 ? pr.log_tile2 : t2,
                  pr.log_cols ? pr.log_cols : lc);
    p.logW = ilog2(pr.whiten_block);
    // row-major power (in groups of NP rows) when a pass-2 CTA holds at most two row pairs,
    // whose bin-order stores would be runs of one or two words, a whitening block lies
    // within one k2 (W <= R) and the warp median applies (W <= 1024).  Measured at 2^23,
    // C = 2048: NP = 2 pass 2 + median 14.5 + 7.7 us (bin order 21.1 + 5.4); NP = 4
    // 17.0 + 7.4 (bin order 18.5 + 5.4).
    p.ptrans = (pr.mode == BPS_MODE_FUSED && p.logW <= 10 && p.logW <= p.logR && p.logNP <= 1)
                   ? 1 : 0;
    p.nharm = pr.nharm_max;
    p.lognh = ilog2(pr.nharm_max);
    p.nlev = p.lognh + 1;
    p.tsamp = s.tsamp;
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

SeriesView view_of(const Series& s)
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

int default_batch(const Plan& p, int64_t K, int mode)
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
    char* base = nullptr;
};

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Fetch order of candidates: (template_idx, nharm, bin), deterministic whatever the order
// in which the device appended them.
void sort_candidates(std::vector<bps_candidate>& c)
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
size_t ws_carve(const Plan& p, int nt, int mode, int anchor_templates, char* base, Workspace* w)
{
    const size_t a = align256(sizeof(Anchor) * (size_t)p.nanchor *
                              (anchor_templates > 0 ? anchor_templates : nt));
    const size_t y = align256(sizeof(float2) * (size_t)(p.M + 1) * nt);
    const size_t x = mode == BPS_MODE_PLAIN ? align256(sizeof(float) * (size_t)p.n * nt) : 0;
    const size_t pp = align256(sizeof(float) * (size_t)p.M * nt);
    const size_t pt = p.ptrans ? pp : 0;
    const size_t sc = align256(sizeof(float) * (size_t)(p.M >> p.logW) * nt);
    if (w) {
        char* q = base;
        w->base = base;
        w->anc = (Anchor*)q; q += a;
        w->Y = (float2*)q; q += y;
        w->x = x ? (float*)q : nullptr; q += x;
        w->P = (float*)q; q += pp;
        w->Pt = pt ? (float*)q : nullptr; q += pt;
        w->scale = (float*)q;
    }
    return a + y + x + pp + pt + sc;
}

int ws_alloc(bps_ctx* ctx, const Plan& p, int nt, int mode, cudaStream_t st, Workspace& w,
             int anchor_templates = 0)
{
    char* base = nullptr;
    CK(cudaMallocAsync((void**)&base, ws_carve(p, nt, mode, anchor_templates, nullptr, nullptr), st));
    ws_carve(p, nt, mode, anchor_templates, base, &w);
    return BPS_OK;
}

int get_fft(bps_ctx* ctx, int64_t n, int nt, cufftHandle& h)
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
int run_spectrum(bps_ctx* ctx, const Series& s, const Bank& b, const Plan& p, int mode,
                 int64_t t0, int nt, Workspace& w, cudaStream_t st, StageTimer& tm,
                 const Anchor* anc = nullptr)
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
        CK(launch_pass1(v, anc, nt, p, ctx->tw, w.Y, st));
        tm.end();
        tm.begin(BPS_STAGE_PASS2);
        CK(launch_pass2(w.Y, nt, p, ctx->tw, p.ptrans ? w.Pt : w.P, st));
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
        int rc = run_spectrum(ctx, *s, *b, p, mode, t0, cnt, w, st, tm,
                              w.anc + (t0 - c0) * p.nanchor);
        if (rc) return rc;
        tm.begin(BPS_STAGE_HARMSUM);
        cudaError_t e = launch_harmsum(w.P, w.scale, cnt, t0, p, th, cands, cap, count, nullptr, st);
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

// Searches of a list of (series, bank) pairs captured into one CUDA graph: pairs are
// spread over up to kGraphBranches parallel branches (fork/join events during the
// capture); the pairs of one branch run in sequence and share its workspace.  Each pair
// has its own candidate region (cap candidates) and counter.
constexpr int kGraphBranches = 4;

struct GraphObj {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<int64_t> series, banks;
    std::vector<char*> wsbuf;
    Cand* cands = nullptr;
    unsigned long long* counts = nullptr;  // 2 per pair: count, status
    int64_t cap = 0;
    cudaEvent_t done = nullptr;
    bool launched = false, fetched = false;
    std::vector<std::vector<bps_candidate>> results;
    std::vector<unsigned long long> totals, status;
    ~GraphObj()
    {
        if (done) {
            cudaEventSynchronize(done);
            cudaEventDestroy(done);
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (char* b : wsbuf) cudaFree(b);
        if (cands) cudaFree(cands);
        if (counts) cudaFree(counts);
    }
};

int lookup(bps_ctx* ctx, int64_t sid, int64_t bid, Series*& s, Bank*& b)
{
    auto si = ctx->series.find(sid);
    if (si == ctx->series.end()) return fail(ctx, BPS_ERR_INVALID_ARG, "unknown series id %lld", (long long)sid);
    auto bi = ctx->banks.find(bid);
    if (bi == ctx->banks.end()) return fail(ctx, BPS_ERR_INVALID_ARG, "unknown bank id %lld", (long long)bid);
    s = &si->second;
    b = &bi->second;
    return BPS_OK;
}

}  // namespace

extern "C" {

void bps_default_params(bps_search_params* p)
{
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->nharm_max = 16;
    p->whiten_block = 1024;
    p->sigma_thr = 6.0;
    p->auto_thr = 0;
    p->mode = BPS_MODE_FUSED;
    p->cand_cap = 1 << 20;
    p->precision = 0;
    p->batch = 0;
    p->log_cols = 0;
}

int bps_create(bps_ctx** out, int device)
try {
    if (!out) return BPS_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return BPS_ERR_CUDA;
    bps_ctx* ctx = new bps_ctx();
    ctx->device = device;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc((void**)&ctx->tw, kTwiddleN * sizeof(float2)) != cudaSuccess ||
        launch_twiddle_init(ctx->tw, ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        delete ctx;
        return BPS_ERR_CUDA;
    }
    *out = ctx;
    return BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

static void free_series(Series& s)
{
    if (s.owned && s.f32) cudaFree(s.f32);
    if (s.f16) cudaFree(s.f16);
    if (s.scale) cudaFree(s.scale);
    if (s.d_sum) cudaFree(s.d_sum);
    if (s.d_fill) cudaFree(s.d_fill);
    s = Series();
}

static void free_request(Request& r)
{
    for (auto& e : r.ev) {
        cudaEventDestroy(e.second.first);
        cudaEventDestroy(e.second.second);
    }
    r.ev.clear();
    if (r.done) {
        cudaEventSynchronize(r.done);
        cudaEventDestroy(r.done);
    }
    if (r.d_cands) cudaFree(r.d_cands);
    if (r.d_count) cudaFree(r.d_count);
    r = Request();
}

void bps_destroy(bps_ctx* ctx)
try {
    if (!ctx) return;
    {
        std::lock_guard<std::recursive_mutex> lk(ctx->mu);
        cudaSetDevice(ctx->device);
        cudaDeviceSynchronize();
        for (auto& r : ctx->reqs) free_request(r.second);
        for (auto& s : ctx->series) free_series(s.second);
        for (auto& b : ctx->banks) cudaFree(b.second.d);
        for (auto& f : ctx->ffts) cufftDestroy(f.second);
        for (auto& gr : ctx->graphs) delete gr.second;
        if (ctx->tw) cudaFree(ctx->tw);
        if (ctx->stream) cudaStreamDestroy(ctx->stream);
    }
    delete ctx;
} catch (...) {
}

const char* bps_last_error(bps_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int bps_load_series(bps_ctx* ctx, const void* data, int64_t n, double tsamp_s, int dtype,
                    int on_device, int64_t* series_id)
try {
    if (!ctx) return BPS_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (!data || !series_id) return fail(ctx, BPS_ERR_INVALID_ARG, "null pointer");
    if (!is_pow2(n) || n < (1 << 11) || n > (1 << 25))
        return fail(ctx, BPS_ERR_INVALID_ARG, "n must be a power of two in [2^11, 2^25], got %lld", (long long)n);
    if (!(tsamp_s > 0.0) || !std::isfinite(tsamp_s))
        return fail(ctx, BPS_ERR_INVALID_ARG, "tsamp must be positive and finite");
    if (dtype != BPS_F32 && dtype != BPS_F16_SCALED)
        return fail(ctx, BPS_ERR_INVALID_ARG, "unknown dtype %d", dtype);
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    Series s;
    s.n = n;
    s.tsamp = tsamp_s;
    s.dtype = dtype;
    float* src = nullptr;
    bool tmp = false;
    if (on_device) {
        src = (float*)data;
    } else {
        CK(cudaMalloc((void**)&src, sizeof(float) * n));
        tmp = true;
        CK(cudaMemcpyAsync(src, data, sizeof(float) * n, cudaMemcpyHostToDevice, st));
    }
    CK(cudaMalloc((void**)&s.d_sum, sizeof(double)));
    CK(cudaMalloc((void**)&s.d_fill, sizeof(float)));
    CK(cudaMemsetAsync(s.d_sum, 0, sizeof(double), st));
    CK(launch_series_stats(src, n, s.d_sum, st));
    CK(launch_fill_from_sum(s.d_sum, n, s.d_fill, st));
    double sum = 0;
    CK(cudaMemcpyAsync(&sum, s.d_sum, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (dtype == BPS_F32) {
        s.f32 = src;
        s.owned = tmp;
    } else {
        CK(cudaMalloc((void**)&s.f16, sizeof(uint16_t) * n));
        CK(cudaMalloc((void**)&s.scale, sizeof(float) * (((n + 4095) >> 12) + 1)));
        CK(launch_f16_pack(src, n, s.f16, s.scale, st));
    }
    CK(cudaStreamSynchronize(st));
    if (dtype != BPS_F32 && tmp) cudaFree(src);
    s.mean = sum / (double)n;
    const int64_t id = ctx->next_id++;
    ctx->series[id] = s;
    *series_id = id;
    return BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

int bps_series_update(bps_ctx* ctx, int64_t series_id, const void* data, int on_device)
try {
    if (!ctx) return BPS_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    auto it = ctx->series.find(series_id);
    if (it == ctx->series.end() || !data)
        return fail(ctx, BPS_ERR_INVALID_ARG, "unknown series %lld or null data", (long long)series_id);
    Series& s = it->second;
    if (s.dtype == BPS_F32 && !s.owned)
        return fail(ctx, BPS_ERR_INVALID_ARG, "series %lld borrows caller memory; update that memory instead",
                    (long long)series_id);
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const size_t bytes = sizeof(float) * (size_t)s.n;
    float* src = nullptr;
    if (s.dtype == BPS_F32) {
        src = s.f32;
        CK(cudaMemcpyAsync(src, data, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    } else if (on_device) {
        src = (float*)data;
    } else {
        CK(cudaMallocAsync((void**)&src, bytes, st));
        CK(cudaMemcpyAsync(src, data, bytes, cudaMemcpyHostToDevice, st));
    }
    CK(cudaMemsetAsync(s.d_sum, 0, sizeof(double), st));
    CK(launch_series_stats(src, s.n, s.d_sum, st));
    CK(launch_fill_from_sum(s.d_sum, s.n, s.d_fill, st));
    if (s.dtype != BPS_F32) CK(launch_f16_pack(src, s.n, s.f16, s.scale, st));
    double sum = 0;
    CK(cudaMemcpyAsync(&sum, s.d_sum, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (s.dtype != BPS_F32 && !on_device) CK(cudaFreeAsync(src, st));
    CK(cudaStreamSynchronize(st));
    s.mean = sum / (double)s.n;
    return BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

int bps_load_bank(bps_ctx* ctx, const bps_template* t, int64_t count, int64_t* bank_id)
try {
    if (!ctx) return BPS_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (!t || !bank_id || count < 1 || count > (1ll << 31))
        return fail(ctx, BPS_ERR_INVALID_ARG, "bad bank pointer or count");
    for (int64_t i = 0; i < count; ++i) {
        const bps_template& q = t[i];
        if (!(q.porb_s > 0.0) || !std::isfinite(q.porb_s) || !(q.tau_lts >= 0.0) ||
            !std::isfinite(q.tau_lts) || !std::isfinite(q.phi_rad) || !std::isfinite(q.omega_rad) ||
            !(q.ecc >= 0.0 && q.ecc < 1.0))
            return fail(ctx, BPS_ERR_INVALID_ARG, "template %lld out of range", (long long)i);
    }
    CK(cudaSetDevice(ctx->device));
    Bank b;
    b.K = count;
    b.h.assign(t, t + count);
    CK(cudaMalloc((void**)&b.d, sizeof(DevTemplate) * count));
    CK(cudaMemcpy(b.d, t, sizeof(DevTemplate) * count, cudaMemcpyHostToDevice));
    const int64_t id = ctx->next_id++;
    ctx->banks[id] = std::move(b);
    *bank_id = id;
    return BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

int bps_thresholds(const bps_search_params* params, int64_t n_samples, int64_t n_templates,
                   double* thr_out)
try {
    if (!params || !thr_out || check_params(nullptr, params, n_samples)) return BPS_ERR_INVALID_ARG;
    thresholds(params, n_samples, n_templates, thr_out);
    return BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

int bps_search(bps_ctx* ctx, int64_t series_id, int64_t bank_id, const bps_search_params* params,
               void* cuda_stream, int64_t* req_id)
try {
    if (!ctx) return BPS_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (!req_id) return fail(ctx, BPS_ERR_INVALID_ARG, "req_id is NULL");
    Series* s;
    Bank* b;
    int rc = lookup(ctx, series_id, bank_id, s, b);
    if (rc) return rc;
    if ((rc = check_params(ctx, params, s->n))) return rc;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
    Request r;
    r.series = series_id;
    r.bank = bank_id;
    r.K = b->K;
    r.cap = params->cand_cap;
    CK(cudaMalloc((void**)&r.d_cands, sizeof(Cand) * (size_t)r.cap));
    CK(cudaMalloc((void**)&r.d_count, 2 * sizeof(unsigned long long)));  // count, status
    CK(cudaMemsetAsync(r.d_count, 0, 2 * sizeof(unsigned long long), st));
    CK(cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming));
    Job job;
    if ((rc = job.setup(ctx, s, b, *params, st, r.d_cands, r.d_count, r.cap))) {
        free_request(r);
        return rc;
    }
    r.batch = job.nt;
    r.logB = job.p.logB;
    job.tm.r = &r;
    job.tm.st = st;
    job.tm.prof = ctx->profiling;
    while (!job.done() && !rc) rc = job.issue_batch();
    job.release();
    if (rc) {
        cudaStreamSynchronize(st);
        free_request(r);
        return rc;
    }
    CK(cudaEventRecord(r.done, st));
    const int64_t id = ctx->next_id++;
    ctx->reqs[id] = std::move(r);
    *req_id = id;
    return BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

int bps_query(bps_ctx* ctx, int64_t req_id, int* done)
try {
    if (!ctx) return BPS_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    auto it = ctx->reqs.find(req_id);
    if (it == ctx->reqs.end() || !done) return fail(ctx, BPS_ERR_INVALID_ARG, "unknown request %lld", (long long)req_id);
    cudaError_t e = cudaEventQuery(it->second.done);
    if (e == cudaSuccess) {
        *done = 1;
        return BPS_OK;
    }
    if (e == cudaErrorNotReady) {
        *done = 0;
        return BPS_OK;
    }
    return fail(ctx, BPS_ERR_CUDA, "request %lld: %s", (long long)req_id, cudaGetErrorString(e));
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

int bps_fetch_candidates(bps_ctx* ctx, int64_t req_id, bps_candidate* out, int64_t cap,
                         int64_t* n_written, int64_t* n_total)
try {
    if (!ctx) return BPS_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    auto it = ctx->reqs.find(req_id);
    if (it == ctx->reqs.end()) return fail(ctx, BPS_ERR_INVALID_ARG, "unknown request %lld", (long long)req_id);
    Request& r = it->second;
    CK(cudaSetDevice(ctx->device));
    if (!r.synced) {
        CK(cudaEventSynchronize(r.done));
        unsigned long long cs[2];
        CK(cudaMemcpy(cs, r.d_count, sizeof cs, cudaMemcpyDeviceToHost));
        r.total = cs[0];
        r.status = cs[1];
        const int64_t kept = std::min<int64_t>((int64_t)r.total, r.cap);
        r.result.resize((size_t)kept);
        static_assert(sizeof(Cand) == sizeof(bps_candidate), "candidate layout");
        if (kept) CK(cudaMemcpy(r.result.data(), r.d_cands, sizeof(Cand) * kept, cudaMemcpyDeviceToHost));
        sort_candidates(r.result);
        r.synced = true;
        cudaFree(r.d_cands);
        r.d_cands = nullptr;
    }
    const int64_t nw = std::min<int64_t>(cap, (int64_t)r.result.size());
    if (out && nw > 0) std::memcpy(out, r.result.data(), sizeof(bps_candidate) * nw);
    if (n_written) *n_written = out ? nw : 0;
    if (n_total) *n_total = (int64_t)r.total;
    if (r.status & 1ull)
        return fail(ctx, BPS_ERR_TIMEOUT, "request %lld: a bounded device wait expired; "
                    "results incomplete", (long long)req_id);
    if ((int64_t)r.total > r.cap)
        return fail(ctx, BPS_ERR_CAND_OVERFLOW, "request %lld found %llu candidates, capacity %lld",
                    (long long)req_id, r.total, (long long)r.cap);
    return BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

int bps_unload(bps_ctx* ctx, int64_t id)
try {
    if (!ctx) return BPS_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    for (auto& gr : ctx->graphs)
        for (size_t i = 0; i < gr.second->series.size(); ++i)
            if (gr.second->series[i] == id || gr.second->banks[i] == id)
                return fail(ctx, BPS_ERR_INVALID_ARG, "id %lld is captured in graph %lld: unload the graph first",
                            (long long)id, (long long)gr.first);
    if (ctx->series.count(id)) {
        cudaDeviceSynchronize();
        free_series(ctx->series[id]);
        ctx->series.erase(id);
        return BPS_OK;
    }
    if (ctx->banks.count(id)) {
        cudaDeviceSynchronize();
        cudaFree(ctx->banks[id].d);
        ctx->banks.erase(id);
        return BPS_OK;
    }
    if (ctx->graphs.count(id)) {
        delete ctx->graphs[id];
        ctx->graphs.erase(id);
        return BPS_OK;
    }
    if (ctx->reqs.count(id)) {
        free_request(ctx->reqs[id]);
        ctx->reqs.erase(id);
        return BPS_OK;
    }
    return fail(ctx, BPS_ERR_INVALID_ARG, "unknown id %lld", (long long)id);
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

int bps_set_profiling(bps_ctx* ctx, int on)
try {
    if (!ctx) return BPS_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    ctx->profiling = on != 0;
    return BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

int bps_request_stats(bps_ctx* ctx, int64_t req_id, bps_stats* out)
try {
    if (!ctx) return BPS_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    auto it = ctx->reqs.find(req_id);
    if (it == ctx->reqs.end() || !out) return fail(ctx, BPS_ERR_INVALID_ARG, "unknown request %lld", (long long)req_id);
    Request& r = it->second;
    CK(cudaEventSynchronize(r.done));
    std::memset(out, 0, sizeof *out);
    out->templates = r.K;
    out->batch = r.batch;
    out->anchor_block = 1 << r.logB;
    out->launches = r.launches;
    out->profiled = r.ev.empty() ? 0 : 1;
    for (int i = 0; i < 8; ++i) out->stage_launches[i] = r.stage_launches[i];
    for (auto& e : r.ev) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e.second.first, e.second.second));
        out->stage_ms[e.first] += ms;
    }
    return BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

int bps_selftest_bounded_wait(bps_ctx* ctx, int32_t poll_limit, int32_t* timed_out)
try {
    if (!ctx) return BPS_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (poll_limit < 1 || !timed_out) return fail(ctx, BPS_ERR_INVALID_ARG, "bad self-test arguments");
    CK(cudaSetDevice(ctx->device));
    unsigned long long* d = nullptr;
    unsigned long long h = 0;
    CK(cudaMalloc((void**)&d, sizeof(unsigned long long)));
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned long long), ctx->stream);
    if (e == cudaSuccess) e = launch_wait_selftest(poll_limit, d, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(d);
    if (e != cudaSuccess) return fail(ctx, BPS_ERR_CUDA, "wait self-test: %s", cudaGetErrorString(e));
    *timed_out = h == 1ull ? 1 : 0;
    return BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

int bps_graph_create(bps_ctx* ctx, int64_t count, const int64_t* series_ids,
                     const int64_t* bank_ids, const bps_search_params* params, int64_t* graph_id)
try {
    if (!ctx) return BPS_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (count < 1 || !series_ids || !bank_ids || !params || !graph_id)
        return fail(ctx, BPS_ERR_INVALID_ARG, "bad graph arguments");
    if (params->mode != BPS_MODE_FUSED)
        return fail(ctx, BPS_ERR_UNSUPPORTED, "graphs capture the fused form only");
    CK(cudaSetDevice(ctx->device));
    CK(set_smem_attributes());
    CK(prepare_detect_kernels());
    const int B = (int)std::min<int64_t>(kGraphBranches, count);
    std::vector<Series*> ss((size_t)count);
    std::vector<Bank*> bb((size_t)count);
    std::vector<size_t> wsb((size_t)B, 0);
    for (int64_t i = 0; i < count; ++i) {
        int rc = lookup(ctx, series_ids[i], bank_ids[i], ss[i], bb[i]);
        if (rc) return rc;
        if ((rc = check_params(ctx, params, ss[i]->n))) return rc;
        Plan p;
        if ((rc = make_plan(ctx, *ss[i], *bb[i], *params, p))) return rc;
        int nt = params->batch > 0 ? (int)std::min<int64_t>(params->batch, bb[i]->K)
                                   : default_batch(p, bb[i]->K, params->mode);
        auto it = ctx->tuned.find(tune_key(p.logn, params->mode, p.lognh));
        if (params->batch == 0 && it != ctx->tuned.end()) nt = (int)std::min<int64_t>(it->second[2], bb[i]->K);
        const int64_t chunk = std::min<int64_t>((int64_t)nt * kAnchorChunk, bb[i]->K);
        wsb[i % B] = std::max(wsb[i % B], ws_carve(p, nt, params->mode, (int)chunk, nullptr, nullptr));
    }
    std::unique_ptr<GraphObj> g(new GraphObj());
    g->series.assign(series_ids, series_ids + count);
    g->banks.assign(bank_ids, bank_ids + count);
    g->cap = params->cand_cap;
    g->wsbuf.assign((size_t)B, nullptr);
    for (int b = 0; b < B; ++b) CK(cudaMalloc((void**)&g->wsbuf[b], wsb[b]));
    CK(cudaMalloc((void**)&g->cands, sizeof(Cand) * (size_t)g->cap * count));
    CK(cudaMalloc((void**)&g->counts, 2 * sizeof(unsigned long long) * count));
    CK(cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming));
    cudaStream_t os;
    std::vector<cudaStream_t> br((size_t)B);
    CK(cudaStreamCreateWithFlags(&os, cudaStreamNonBlocking));
    for (auto& x : br) CK(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
    cudaEvent_t fork;
    std::vector<cudaEvent_t> join((size_t)B);
    CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    for (auto& e : join) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    int rc = BPS_OK;
    cudaError_t ce = cudaStreamBeginCapture(os, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
        cudaMemsetAsync(g->counts, 0, 2 * sizeof(unsigned long long) * count, os);
        cudaEventRecord(fork, os);
        for (int b = 0; b < B; ++b) cudaStreamWaitEvent(br[b], fork, 0);
        for (int64_t i = 0; i < count && !rc; ++i) {
            Job job;
            rc = job.setup(ctx, ss[i], bb[i], *params, br[i % B], g->cands + (size_t)i * g->cap,
                           g->counts + 2 * i, g->cap, g->wsbuf[i % B], wsb[i % B]);
            while (!rc && !job.done()) rc = job.issue_batch();
        }
        for (int b = 0; b < B; ++b) {
            cudaEventRecord(join[b], br[b]);
            cudaStreamWaitEvent(os, join[b], 0);
        }
        ce = cudaStreamEndCapture(os, &g->graph);
        if (ce == cudaSuccess && !rc) ce = cudaGraphInstantiate(&g->exec, g->graph, 0);
    }
    cudaEventDestroy(fork);
    for (auto e : join) cudaEventDestroy(e);
    for (auto x : br) cudaStreamDestroy(x);
    cudaStreamDestroy(os);
    if (rc) return rc;
    if (ce != cudaSuccess) return fail(ctx, BPS_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
    const int64_t id = ctx->next_id++;
    ctx->graphs[id] = g.release();
    *graph_id = id;
    return BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

int bps_graph_launch(bps_ctx* ctx, int64_t graph_id, void* cuda_stream)
try {
    if (!ctx) return BPS_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    auto it = ctx->graphs.find(graph_id);
    if (it == ctx->graphs.end()) return fail(ctx, BPS_ERR_INVALID_ARG, "unknown graph %lld", (long long)graph_id);
    GraphObj& g = *it->second;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
    CK(cudaGraphLaunch(g.exec, st));
    CK(cudaEventRecord(g.done, st));
    g.launched = true;
    g.fetched = false;
    return BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

int bps_graph_fetch(bps_ctx* ctx, int64_t graph_id, int64_t pair, bps_candidate* out, int64_t cap,
                    int64_t* n_written, int64_t* n_total)
try {
    if (!ctx) return BPS_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    auto it = ctx->graphs.find(graph_id);
    if (it == ctx->graphs.end()) return fail(ctx, BPS_ERR_INVALID_ARG, "unknown graph %lld", (long long)graph_id);
    GraphObj& g = *it->second;
    const int64_t np = (int64_t)g.series.size();
    if (pair < 0 || pair >= np || !g.launched) return fail(ctx, BPS_ERR_INVALID_ARG, "bad pair or graph not launched");
    CK(cudaSetDevice(ctx->device));
    if (!g.fetched) {
        CK(cudaEventSynchronize(g.done));
        std::vector<unsigned long long> cs(2 * (size_t)np);
        CK(cudaMemcpy(cs.data(), g.counts, sizeof(unsigned long long) * cs.size(), cudaMemcpyDeviceToHost));
        g.results.assign((size_t)np, {});
        g.totals.assign((size_t)np, 0);
        g.status.assign((size_t)np, 0);
        for (int64_t i = 0; i < np; ++i) {
            g.totals[i] = cs[2 * i];
            g.status[i] = cs[2 * i + 1];
            const int64_t kept = std::min<int64_t>((int64_t)cs[2 * i], g.cap);
            g.results[i].resize((size_t)kept);
            if (kept)
                CK(cudaMemcpy(g.results[i].data(), g.cands + (size_t)i * g.cap, sizeof(Cand) * kept,
                              cudaMemcpyDeviceToHost));
            sort_candidates(g.results[i]);
        }
        g.fetched = true;
    }
    const auto& r = g.results[pair];
    const int64_t nw = std::min<int64_t>(cap, (int64_t)r.size());
    if (out && nw > 0) std::memcpy(out, r.data(), sizeof(bps_candidate) * nw);
    if (n_written) *n_written = out ? nw : 0;
    if (n_total) *n_total = (int64_t)g.totals[pair];
    if (g.status[pair] & 1ull) return fail(ctx, BPS_ERR_TIMEOUT, "a bounded device wait expired");
    if ((int64_t)g.totals[pair] > g.cap)
        return fail(ctx, BPS_ERR_CAND_OVERFLOW, "pair %lld: %llu candidates, capacity %lld",
                    (long long)pair, g.totals[pair], (long long)g.cap);
    return BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

int bps_autotune(bps_ctx* ctx, int64_t series_id, int64_t bank_id, const bps_search_params* base,
                 int64_t sample_templates, bps_search_params* best, double* best_ms_per_template)
try {
    if (!ctx) return BPS_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    Series* s;
    Bank* b;
    int rc = lookup(ctx, series_id, bank_id, s, b);
    if (rc) return rc;
    if ((rc = check_params(ctx, base, s->n))) return rc;
    if (!best || sample_templates < 1) return fail(ctx, BPS_ERR_INVALID_ARG, "bad autotune arguments");
    CK(cudaSetDevice(ctx->device));
    Bank sub = *b;  // the first sample_templates templates of the bank (same device array)
    sub.K = std::min<int64_t>(sample_templates, b->K);
    sub.h.resize((size_t)sub.K);
    cudaStream_t st = ctx->stream;
    Cand* cd = nullptr;
    unsigned long long* cnt = nullptr;
    CK(cudaMalloc((void**)&cd, sizeof(Cand) * (size_t)base->cand_cap));
    CK(cudaMalloc((void**)&cnt, 2 * sizeof(unsigned long long)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int tiles[2] = {13, 14};
    const int batches[4] = {8, 16, 32, 64};
    // four-step splits: the caller's, else the library's and its valid neighbours
    const int logM = ilog2(s->n) - 1;
    std::vector<int> splits;
    if (base->log_cols) splits.push_back(base->log_cols);
    else if (base->mode == BPS_MODE_PLAIN) splits.push_back(0);
    else
        for (int d : {0, -1, 1})
            if (log_cols_ok(logM, default_log_cols(logM) + d)) splits.push_back(default_log_cols(logM) + d);
    double best_ms = 1e30;
    bps_search_params bp = *base;
    for (int lc : splits)
    for (int t1 : tiles)
        for (int t2 : tiles)
            for (int nb : batches) {
                if (nb > sub.K) continue;
                bps_search_params pr = *base;
                pr.log_tile = t1;
                pr.log_tile2 = t2;
                pr.log_cols = lc;
                pr.batch = nb;
                double ms_best = 1e30;
                for (int rep = 0; rep < 2 && !rc; ++rep) {
                    cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), st);
                    Job job;
                    if ((rc = job.setup(ctx, s, &sub, pr, st, cd, cnt, pr.cand_cap))) break;
                    cudaEventRecord(e0, st);
                    while (!job.done() && !rc) rc = job.issue_batch();
                    cudaEventRecord(e1, st);
                    job.release();
                    cudaEventSynchronize(e1);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    ms_best = std::min<double>(ms_best, ms);
                }
                if (rc) break;
                if (ms_best < best_ms) {
                    best_ms = ms_best;
                    bp = pr;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(cd);
    cudaFree(cnt);
    if (rc) return rc;
    ctx->tuned[tune_key(ilog2(s->n), base->mode, ilog2(base->nharm_max))] = {bp.log_tile, bp.log_tile2,
                                                                          bp.batch, bp.log_cols};
    *best = bp;
    if (best_ms_per_template) *best_ms_per_template = best_ms / (double)sub.K;
    return BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

int bps_index_map(bps_ctx* ctx, int64_t series_id, int64_t bank_id, int64_t template_idx,
                  int32_t* idx_out, int64_t* n_precise)
try {
    if (!ctx) return BPS_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    Series* s;
    Bank* b;
    int rc = lookup(ctx, series_id, bank_id, s, b);
    if (rc) return rc;
    if (!idx_out || template_idx < 0 || template_idx >= b->K)
        return fail(ctx, BPS_ERR_INVALID_ARG, "bad template index or output");
    bps_search_params pr;
    bps_default_params(&pr);
    pr.whiten_block = 32;
    Plan p;
    if ((rc = make_plan(ctx, *s, *b, pr, p))) return rc;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    Anchor* anc = nullptr;
    int32_t* idx = nullptr;
    unsigned long long* cnt = nullptr;
    CK(cudaMallocAsync((void**)&anc, sizeof(Anchor) * p.nanchor, st));
    CK(cudaMallocAsync((void**)&idx, sizeof(int32_t) * p.n, st));
    CK(cudaMallocAsync((void**)&cnt, sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
    CK(launch_anchors(b->d, template_idx, 1, p, anc, st));
    CK(launch_index_map(anc, p, idx, cnt, st));
    unsigned long long np = 0;
    CK(cudaMemcpyAsync(idx_out, idx, sizeof(int32_t) * p.n, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&np, cnt, sizeof np, cudaMemcpyDeviceToHost, st));
    CK(cudaFreeAsync(anc, st));
    CK(cudaFreeAsync(idx, st));
    CK(cudaFreeAsync(cnt, st));
    CK(cudaStreamSynchronize(st));
    if (n_precise) *n_precise = (int64_t)np;
    return BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

int bps_whitened_spectrum(bps_ctx* ctx, int64_t series_id, int64_t bank_id, int64_t t0,
                          int64_t count, const bps_search_params* params, float* pw_out)
try {
    if (!ctx) return BPS_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    Series* s;
    Bank* b;
    int rc = lookup(ctx, series_id, bank_id, s, b);
    if (rc) return rc;
    if ((rc = check_params(ctx, params, s->n))) return rc;
    if (!pw_out || t0 < 0 || count < 1 || t0 + count > b->K)
        return fail(ctx, BPS_ERR_INVALID_ARG, "bad template range or output");
    Plan p;
    if ((rc = make_plan(ctx, *s, *b, *params, p))) return rc;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    Workspace w;
    const int nt = (int)count;
    if ((rc = ws_alloc(ctx, p, nt, params->mode, st, w))) return rc;
    float* out = nullptr;
    CK(cudaMallocAsync((void**)&out, sizeof(float) * p.M * nt, st));
    StageTimer tm;
    if ((rc = run_spectrum(ctx, *s, *b, p, params->mode, t0, nt, w, st, tm))) return rc;
    CK(launch_whitened(w.P, w.scale, nt, p, out, st));
    CK(cudaMemcpyAsync(pw_out, out, sizeof(float) * p.M * nt, cudaMemcpyDeviceToHost, st));
    CK(cudaFreeAsync(out, st));
    CK(cudaFreeAsync(w.base, st));
    CK(cudaStreamSynchronize(st));
    return BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

int bps_harmonic_sums(bps_ctx* ctx, int64_t series_id, int64_t bank_id, int64_t template_idx,
                      const bps_search_params* params, float* s_out)
try {
    if (!ctx) return BPS_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    Series* s;
    Bank* b;
    int rc = lookup(ctx, series_id, bank_id, s, b);
    if (rc) return rc;
    if ((rc = check_params(ctx, params, s->n))) return rc;
    if (!s_out || template_idx < 0 || template_idx >= b->K)
        return fail(ctx, BPS_ERR_INVALID_ARG, "bad template index or output");
    Plan p;
    if ((rc = make_plan(ctx, *s, *b, *params, p))) return rc;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    Workspace w;
    if ((rc = ws_alloc(ctx, p, 1, params->mode, st, w))) return rc;
    float* so = nullptr;
    Cand* cd = nullptr;
    unsigned long long* cnt = nullptr;
    CK(cudaMallocAsync((void**)&so, sizeof(float) * p.M * p.nlev, st));
    CK(cudaMallocAsync((void**)&cd, sizeof(Cand), st));
    CK(cudaMallocAsync((void**)&cnt, 2 * sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), st));
    StageTimer tm;
    if ((rc = run_spectrum(ctx, *s, *b, p, params->mode, template_idx, 1, w, st, tm))) return rc;
    Thr th;
    for (int L = 0; L < 5; ++L) th.v[L] = INFINITY;
    CK(launch_harmsum(w.P, w.scale, 1, template_idx, p, th, cd, 1, cnt, so, st));
    CK(cudaMemcpyAsync(s_out, so, sizeof(float) * p.M * p.nlev, cudaMemcpyDeviceToHost, st));
    CK(cudaFreeAsync(so, st));
    CK(cudaFreeAsync(cd, st));
    CK(cudaFreeAsync(cnt, st));
    CK(cudaFreeAsync(w.base, st));
    CK(cudaStreamSynchronize(st));
    return BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

int bps_whiten(bps_ctx* ctx, const float* d_power, int64_t count, int64_t nbins,
               int32_t whiten_block, float* d_pw_out, float* d_scale_out, void* cuda_stream)
try {
    if (!ctx) return BPS_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    const int logW = ilog2(whiten_block);
    const int logM = ilog2(nbins);
    if (whiten_block < 32 || whiten_block > 8192 || (1ll << logW) != whiten_block)
        return fail(ctx, BPS_ERR_INVALID_ARG, "whiten_block %d: not a power of two in [32, 8192]",
                    whiten_block);
    if (nbins < whiten_block || nbins > (1ll << 30) || (1ll << logM) != nbins)
        return fail(ctx, BPS_ERR_INVALID_ARG, "nbins %lld: not a power of two in [whiten_block, 2^30]",
                    (long long)nbins);
    if (count < 1 || count > (INT64_MAX / 4) / nbins || !d_power || !d_pw_out || !d_scale_out)
        return fail(ctx, BPS_ERR_INVALID_ARG, "bad count or null pointer");
    const int64_t nblk = nbins >> logW;
    const size_t bytes = sizeof(float) * (size_t)count * (size_t)nbins;
    const void* ptrs[3] = {d_power, d_pw_out, d_scale_out};
    for (const void* q : ptrs) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, q) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, BPS_ERR_INVALID_ARG, "not a device pointer");
        }
        if (!(a.type == cudaMemoryTypeManaged ||
              (a.type == cudaMemoryTypeDevice && a.device == ctx->device)))
            return fail(ctx, BPS_ERR_INVALID_ARG, "not device memory of the context's GPU");
    }
    const char* pin = (const char*)d_power;
    const char* pout = (const char*)d_pw_out;
    if (pin != pout && pin < pout + bytes && pout < pin + bytes)
        return fail(ctx, BPS_ERR_INVALID_ARG, "d_pw_out overlaps d_power");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (pin != pout) CK(cudaMemcpyAsync(d_pw_out, d_power, bytes, cudaMemcpyDeviceToDevice, st));
    Plan p{};
    p.M = nbins;
    p.logM = logM;
    p.logW = logW;
    p.ptrans = 0;
    for (int64_t s0 = 0; s0 < count; s0 += 65535) {
        const int nt = (int)std::min<int64_t>(65535, count - s0);
        CK(launch_block_median(d_pw_out + s0 * nbins, nt, p, d_scale_out + s0 * nblk, st));
    }
    return BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

}  // extern "C"

// =====================================================================================
// Serving: a continuously batched request loop.  A worker thread admits queued
// requests onto stream slots while the HBM budget allows, stages their series and bank
// on the device, then issues their launch groups round-robin (a few in flight per
// request), and retires finished requests (candidates to the host, device memory
// freed, slot released) so the next queued request can start.
// =====================================================================================
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <thread>

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

enum SState { S_QUEUED, S_STAGING, S_RUNNING, S_COUNTING, S_COPYING, S_DONE, S_FAILED };

constexpr int64_t kPinnedCands = 1 << 16;  // candidates copied back through pinned memory

struct SReq {
    int64_t ticket = 0;
    SState state = S_QUEUED;
    float* h_series = nullptr;  // pinned host copy of the submitted series
    int64_t n = 0;
    double tsamp = 0;
    int dtype = BPS_F32;
    std::vector<bps_template> bank;
    bps_search_params prm;
    size_t bytes = 0;
    int slot = -1;
    Series s;
    Bank b;
    float* d_stage = nullptr;
    double* d_sum = nullptr;
    double* h_sum = nullptr;
    Cand* d_cands = nullptr;
    unsigned long long* d_count = nullptr;
    unsigned long long* h_count = nullptr;
    Cand* h_cands = nullptr;
    cudaEvent_t ev = nullptr;
    std::vector<cudaEvent_t> grp;
    int gi = 0, gq = 0;  // ring position, groups queued
    std::unique_ptr<Job> job;
    double t_submit = 0, t_done = 0;
    std::vector<bps_candidate> result;
    unsigned long long total = 0, status = 0;
    int rc = BPS_OK;
    std::string err;
};

// Device bytes a request holds while resident (series + bank + workspace + candidates).
size_t request_bytes(const Plan& p, int64_t K, const bps_search_params& prm, int dtype)
{
    const int nt = prm.batch > 0 ? (int)std::min<int64_t>(prm.batch, K) : default_batch(p, K, prm.mode);
    const int64_t chunk = std::min<int64_t>((int64_t)nt * kAnchorChunk, K);
    size_t ser = dtype == BPS_F32 ? align256(4 * (size_t)p.n)
                                  : align256(2 * (size_t)p.n) + align256(4 * (size_t)((p.n + 4095) >> 12)) +
                                        align256(4 * (size_t)p.n);  // FP32 staging while packing
    return ser + align256(sizeof(DevTemplate) * (size_t)K) + Job::workspace_bytes(p, nt, chunk, prm.mode) +
           align256(sizeof(Cand) * (size_t)prm.cand_cap) + 1024;
}

}  // namespace

struct bps_server {
    bps_ctx* ctx = nullptr;
    bps_server_config cfg;
    size_t budget = 0, used = 0;
    std::vector<cudaStream_t> slots;
    std::vector<char> busy;
    std::deque<int64_t> queue;
    std::map<int64_t, std::unique_ptr<SReq>> reqs;
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    int64_t next_ticket = 1;
    size_t rr = 0;
    std::string err;
};

namespace {

int sfail(bps_server* srv, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    srv->err = buf;
    return code;
}

void release_device(SReq& q, cudaStream_t st)
{
    if (q.job) {
        q.job->release();
        q.job.reset();
    }
    if (q.s.f32) cudaFreeAsync(q.s.f32, st);
    if (q.s.f16) cudaFreeAsync(q.s.f16, st);
    if (q.s.scale) cudaFreeAsync(q.s.scale, st);
    if (q.d_stage) cudaFreeAsync(q.d_stage, st);
    if (q.d_sum) cudaFreeAsync(q.d_sum, st);
    if (q.b.d) cudaFreeAsync(q.b.d, st);
    if (q.d_cands) cudaFreeAsync(q.d_cands, st);
    if (q.d_count) cudaFreeAsync(q.d_count, st);
    q.s.f32 = nullptr;
    q.s.f16 = nullptr;
    q.s.scale = nullptr;
    q.d_stage = nullptr;
    q.d_sum = nullptr;
    q.b.d = nullptr;
    q.d_cands = nullptr;
    q.d_count = nullptr;
}

void release_host(SReq& q)
{
    if (q.h_series) cudaFreeHost(q.h_series);
    if (q.h_sum) cudaFreeHost(q.h_sum);
    if (q.h_count) cudaFreeHost(q.h_count);
    if (q.h_cands) cudaFreeHost(q.h_cands);
    q.h_series = nullptr;
    q.h_sum = nullptr;
    q.h_count = nullptr;
    q.h_cands = nullptr;
    if (q.ev) cudaEventDestroy(q.ev);
    for (auto e : q.grp) cudaEventDestroy(e);
    q.ev = nullptr;
    q.grp.clear();
}

}  // namespace

namespace {

// Stage a queued request onto a free slot: device buffers (stream-ordered), series and
// bank copies, FP16 packing, the FP64 series sum read back for the fill value.
bool admit_one(bps_server* srv, SReq& q, int slot)
{
    cudaStream_t st = srv->slots[slot];
    const size_t n = (size_t)q.n;
    bool ok = true;
    auto chk = [&](cudaError_t e) {
        if (e != cudaSuccess && ok) {
            ok = false;
            q.rc = e == cudaErrorMemoryAllocation ? BPS_ERR_OUT_OF_MEMORY : BPS_ERR_CUDA;
            q.err = cudaGetErrorString(e);
        }
    };
    q.slot = slot;
    q.s.n = q.n;
    q.s.tsamp = q.tsamp;
    q.s.dtype = q.dtype;
    q.s.owned = true;
    q.b.K = (int64_t)q.bank.size();
    q.b.h = q.bank;
    float* src = nullptr;
    if (q.dtype == BPS_F32) {
        chk(cudaMallocAsync((void**)&q.s.f32, 4 * n, st));
        src = q.s.f32;
    } else {
        chk(cudaMallocAsync((void**)&q.d_stage, 4 * n, st));
        chk(cudaMallocAsync((void**)&q.s.f16, 2 * n, st));
        chk(cudaMallocAsync((void**)&q.s.scale, 4 * (((n + 4095) >> 12) + 1), st));
        src = q.d_stage;
    }
    chk(cudaMallocAsync((void**)&q.d_sum, sizeof(double), st));
    chk(cudaMallocAsync((void**)&q.b.d, sizeof(DevTemplate) * q.bank.size(), st));
    chk(cudaMallocAsync((void**)&q.d_cands, sizeof(Cand) * (size_t)q.prm.cand_cap, st));
    chk(cudaMallocAsync((void**)&q.d_count, 2 * sizeof(unsigned long long), st));
    if (ok) {
        chk(cudaMemcpyAsync(src, q.h_series, 4 * n, cudaMemcpyHostToDevice, st));
        chk(cudaMemcpyAsync(q.b.d, q.bank.data(), sizeof(DevTemplate) * q.bank.size(),
                            cudaMemcpyHostToDevice, st));
        chk(cudaMemsetAsync(q.d_sum, 0, sizeof(double), st));
        chk(cudaMemsetAsync(q.d_count, 0, 2 * sizeof(unsigned long long), st));
        chk(launch_series_stats(src, q.n, q.d_sum, st));
        if (q.dtype != BPS_F32) chk(launch_f16_pack(src, q.n, q.s.f16, q.s.scale, st));
        chk(cudaMemcpyAsync(q.h_sum, q.d_sum, sizeof(double), cudaMemcpyDeviceToHost, st));
        chk(cudaEventRecord(q.ev, st));
    }
    srv->busy[slot] = 1;
    srv->used += q.bytes;
    q.state = ok ? S_STAGING : S_FAILED;
    return ok;
}

void finish(bps_server* srv, SReq& q, SState st_)
{
    release_device(q, srv->slots[q.slot]);
    release_host(q);
    srv->busy[q.slot] = 0;
    srv->used -= q.bytes;
    q.state = st_;
    q.t_done = now_s();
}

// Advance one resident request; returns true when something happened.
bool advance(bps_server* srv, SReq& q)
{
    cudaStream_t st = srv->slots[q.slot];
    switch (q.state) {
        case S_STAGING: {
            if (cudaEventQuery(q.ev) != cudaSuccess) return false;
            if (q.d_stage) {
                cudaFreeAsync(q.d_stage, st);
                q.d_stage = nullptr;
            }
            cudaFreeHost(q.h_series);
            q.h_series = nullptr;
            q.s.mean = *q.h_sum / (double)q.n;
            q.job.reset(new Job());
            int rc = q.job->setup(srv->ctx, &q.s, &q.b, q.prm, st, q.d_cands, q.d_count,
                                  q.prm.cand_cap);
            if (rc) {
                q.rc = rc;
                q.err = srv->ctx->err;
                finish(srv, q, S_FAILED);
                return true;
            }
            q.state = S_RUNNING;
            return true;
        }
        case S_RUNNING: {
            bool did = false;
            const int D = (int)q.grp.size();
            // keep up to D launch groups queued on the slot's stream
            while (!q.job->done()) {
                if (q.gq >= D) {
                    if (cudaEventQuery(q.grp[q.gi]) != cudaSuccess) break;
                    --q.gq;
                }
                int rc = q.job->issue_batch();
                if (rc) {
                    q.rc = rc;
                    q.err = srv->ctx->err;
                    cudaStreamSynchronize(st);
                    finish(srv, q, S_FAILED);
                    return true;
                }
                cudaEventRecord(q.grp[q.gi], st);
                q.gi = (q.gi + 1) % D;
                ++q.gq;
                did = true;
                break;  // one group per request per round: round-robin across requests
            }
            if (q.job->done()) {
                q.job->release();
                cudaMemcpyAsync(q.h_count, q.d_count, 2 * sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, st);
                cudaEventRecord(q.ev, st);
                q.state = S_COUNTING;
                did = true;
            }
            return did;
        }
        case S_COUNTING: {
            if (cudaEventQuery(q.ev) != cudaSuccess) return false;
            q.total = q.h_count[0];
            q.status = q.h_count[1];
            const int64_t kept = std::min<int64_t>((int64_t)q.total, q.prm.cand_cap);
            q.result.resize((size_t)kept);
            if (kept > 0 && kept <= kPinnedCands) {
                cudaMemcpyAsync(q.h_cands, q.d_cands, sizeof(Cand) * kept, cudaMemcpyDeviceToHost, st);
                cudaEventRecord(q.ev, st);
                q.state = S_COPYING;
                return true;
            }
            if (kept > 0) cudaMemcpy(q.result.data(), q.d_cands, sizeof(Cand) * kept, cudaMemcpyDeviceToHost);
            q.state = S_COPYING;
            cudaEventRecord(q.ev, st);
            return true;
        }
        case S_COPYING: {
            if (cudaEventQuery(q.ev) != cudaSuccess) return false;
            const int64_t kept = (int64_t)q.result.size();
            if (kept > 0 && kept <= kPinnedCands)
                std::memcpy(q.result.data(), q.h_cands, sizeof(Cand) * kept);
            sort_candidates(q.result);
            if (q.status & 1ull) {
                q.rc = BPS_ERR_TIMEOUT;
                q.err = "a bounded device wait expired; results incomplete";
            } else if ((int64_t)q.total > q.prm.cand_cap) {
                q.rc = BPS_ERR_CAND_OVERFLOW;
                q.err = "candidate capacity exceeded";
            }
            finish(srv, q, S_DONE);
            return true;
        }
        default:
            return false;
    }
}

void worker_main(bps_server* srv)
{
    cudaSetDevice(srv->ctx->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    for (;;) {
        bool progress = false;
        {
            std::lock_guard<std::recursive_mutex> cl(srv->ctx->mu);
            // admit queued requests (FIFO) while a slot is free and the budget allows
            while (!srv->queue.empty()) {
                SReq& q = *srv->reqs[srv->queue.front()];
                int slot = -1;
                for (size_t i = 0; i < srv->busy.size(); ++i)
                    if (!srv->busy[i]) {
                        slot = (int)i;
                        break;
                    }
                if (slot < 0 || srv->used + q.bytes > srv->budget) break;
                srv->queue.pop_front();
                if (!admit_one(srv, q, slot)) {
                    cudaStreamSynchronize(srv->slots[slot]);
                    finish(srv, q, S_FAILED);
                }
                progress = true;
            }
            // one round over the resident requests, starting after the last served
            std::vector<SReq*> act;
            for (auto& kv : srv->reqs)
                if (kv.second->state >= S_STAGING && kv.second->state <= S_COPYING)
                    act.push_back(kv.second.get());
            for (size_t i = 0; i < act.size(); ++i) {
                SReq& q = *act[(srv->rr + i) % act.size()];
                if (advance(srv, q)) progress = true;
            }
            if (!act.empty()) srv->rr = (srv->rr + 1) % act.size();
        }
        if (progress) srv->cv.notify_all();
        bool idle = srv->queue.empty();
        for (auto& kv : srv->reqs)
            if (kv.second->state >= S_STAGING && kv.second->state <= S_COPYING) idle = false;
        if (srv->stop && idle) break;
        if (progress) {  // let submitters and result readers in between rounds
            lk.unlock();
            std::this_thread::yield();
            lk.lock();
        } else {
            srv->cv.wait_for(lk, std::chrono::microseconds(idle ? 2000 : 30));
        }
    }
}

}  // namespace

extern "C" {

int bps_server_create(bps_ctx* ctx, const bps_server_config* cfg, bps_server** out)
try {
    if (!ctx || !cfg || !out) return BPS_ERR_INVALID_ARG;
    *out = nullptr;
    if (cfg->max_active < 1 || cfg->max_active > 64 || cfg->groups_in_flight < 1 ||
        cfg->groups_in_flight > 64 || cfg->hbm_budget < 0)
        return fail(ctx, BPS_ERR_INVALID_ARG, "server config out of range");
    std::lock_guard<std::recursive_mutex> cl(ctx->mu);
    CK(cudaSetDevice(ctx->device));
    auto* srv = new bps_server();
    srv->ctx = ctx;
    srv->cfg = *cfg;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        delete srv;
        return fail(ctx, BPS_ERR_CUDA, "cudaMemGetInfo failed");
    }
    srv->budget = cfg->hbm_budget > 0 ? (size_t)cfg->hbm_budget : (size_t)(0.9 * (double)fr);
    srv->slots.resize(cfg->max_active);
    srv->busy.assign(cfg->max_active, 0);
    for (auto& s : srv->slots) {
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            for (auto& t : srv->slots)
                if (t) cudaStreamDestroy(t);
            delete srv;
            return fail(ctx, BPS_ERR_CUDA, "stream creation failed");
        }
    }
    srv->worker = std::thread(worker_main, srv);
    *out = srv;
    return BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

void bps_server_destroy(bps_server* srv)
try {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        for (int64_t t : srv->queue) {  // never admitted: drop
            release_host(*srv->reqs[t]);
            srv->reqs[t]->state = S_FAILED;
        }
        srv->queue.clear();
        srv->stop = true;
    }
    srv->cv.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    cudaSetDevice(srv->ctx->device);
    for (auto& kv : srv->reqs) release_host(*kv.second);
    for (auto s : srv->slots) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    delete srv;
} catch (...) {
}

const char* bps_server_last_error(bps_server* srv) { return srv ? srv->err.c_str() : "null server"; }

int bps_server_submit(bps_server* srv, const float* series, int64_t n, double tsamp_s, int dtype,
                      const bps_template* bank, int64_t count, const bps_search_params* params,
                      int64_t* ticket)
try {
    if (!srv) return BPS_ERR_INVALID_ARG;
    if (!series || !bank || !params || !ticket)
        return sfail(srv, BPS_ERR_INVALID_ARG, "null pointer");
    if (!is_pow2(n) || n < (1 << 11) || n > (1 << 25))
        return sfail(srv, BPS_ERR_INVALID_ARG, "n must be a power of two in [2^11, 2^25]");
    if (!(tsamp_s > 0.0) || !std::isfinite(tsamp_s) || (dtype != BPS_F32 && dtype != BPS_F16_SCALED))
        return sfail(srv, BPS_ERR_INVALID_ARG, "bad tsamp or dtype");
    if (count < 1 || count > (1ll << 31)) return sfail(srv, BPS_ERR_INVALID_ARG, "bad bank size");
    for (int64_t i = 0; i < count; ++i) {
        const bps_template& q = bank[i];
        if (!(q.porb_s > 0.0) || !std::isfinite(q.porb_s) || !(q.tau_lts >= 0.0) ||
            !std::isfinite(q.tau_lts) || !std::isfinite(q.phi_rad) || !std::isfinite(q.omega_rad) ||
            !(q.ecc >= 0.0 && q.ecc < 1.0))
            return sfail(srv, BPS_ERR_INVALID_ARG, "template %lld out of range", (long long)i);
    }
    if (check_params(nullptr, params, n)) return sfail(srv, BPS_ERR_INVALID_ARG, "invalid search parameters");
    std::unique_ptr<SReq> q(new SReq());
    q->n = n;
    q->tsamp = tsamp_s;
    q->dtype = dtype;
    q->bank.assign(bank, bank + count);
    q->prm = *params;
    {
        Series hs;
        hs.n = n;
        hs.tsamp = tsamp_s;
        Bank hb;
        hb.K = count;
        hb.h = q->bank;
        Plan p;
        int rc = make_plan(nullptr, hs, hb, *params, p);
        if (rc) return sfail(srv, rc, "orbits outside the FP32 index-map envelope or bad size");
        q->bytes = request_bytes(p, count, *params, dtype);
    }
    if (q->bytes > srv->budget)
        return sfail(srv, BPS_ERR_OUT_OF_MEMORY, "request needs %zu bytes, server budget %zu",
                     q->bytes, srv->budget);
    cudaSetDevice(srv->ctx->device);
    if (cudaMallocHost((void**)&q->h_series, 4 * (size_t)n) != cudaSuccess ||
        cudaMallocHost((void**)&q->h_sum, sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void**)&q->h_count, 2 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost((void**)&q->h_cands, sizeof(Cand) * (size_t)std::min<int64_t>(params->cand_cap, kPinnedCands)) != cudaSuccess ||
        cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming) != cudaSuccess) {
        release_host(*q);
        return sfail(srv, BPS_ERR_OUT_OF_MEMORY, "pinned host staging failed");
    }
    q->grp.resize(srv->cfg.groups_in_flight);
    for (auto& e : q->grp) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    std::memcpy(q->h_series, series, 4 * (size_t)n);
    q->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        q->ticket = srv->next_ticket++;
        *ticket = q->ticket;
        srv->queue.push_back(q->ticket);
        srv->reqs[q->ticket] = std::move(q);
    }
    srv->cv.notify_all();
    return BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

int bps_server_result(bps_server* srv, int64_t ticket, int32_t timeout_ms, bps_candidate* out,
                      int64_t cap, int64_t* n_written, int64_t* n_total, double* latency_s)
try {
    if (!srv) return BPS_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return sfail(srv, BPS_ERR_INVALID_ARG, "unknown ticket %lld", (long long)ticket);
    auto ready = [&] { return it->second->state == S_DONE || it->second->state == S_FAILED; };
    if (timeout_ms < 0) srv->cv.wait(lk, ready);
    else srv->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
    if (!ready()) return sfail(srv, BPS_ERR_NOT_READY, "ticket %lld still running", (long long)ticket);
    SReq& q = *it->second;
    const int64_t nw = std::min<int64_t>(cap, (int64_t)q.result.size());
    if (out && nw > 0) std::memcpy(out, q.result.data(), sizeof(bps_candidate) * nw);
    if (n_written) *n_written = out ? nw : 0;
    if (n_total) *n_total = (int64_t)q.total;
    if (latency_s) *latency_s = q.t_done - q.t_submit;
    const int rc = q.rc;
    if (rc) srv->err = q.err;
    if (out || cap == 0) {  // a call with a buffer (or an explicit empty one) releases it
        if (out) srv->reqs.erase(it);
    }
    return rc;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

int bps_server_stats(bps_server* srv, int64_t* queued, int64_t* active, int64_t* finished,
                     int64_t* bytes_held)
try {
    if (!srv) return BPS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    int64_t a = 0, f = 0;
    for (auto& kv : srv->reqs) {
        if (kv.second->state >= S_STAGING && kv.second->state <= S_COPYING) ++a;
        if (kv.second->state == S_DONE || kv.second->state == S_FAILED) ++f;
    }
    if (queued) *queued = (int64_t)srv->queue.size();
    if (active) *active = a;
    if (finished) *finished = f;
    if (bytes_held) *bytes_held = (int64_t)srv->used;
    return BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

}  // extern "C"

// =====================================================================================
// Candidate distillation (host): group repeated detections of one signal -- the same
// or a harmonically related fundamental frequency, seen under several templates or
// harmonic levels -- and keep the most significant member of each group.
// =====================================================================================
namespace {

// -log Q(n, x): false-alarm exponent of a harmonic sum of n whitened bins (Gamma(n,1)
// tail), evaluated in log space so large sums do not underflow.
double neg_log_q(int n, double x)
{
    if (x <= 0.0) return 0.0;
    double lt = 0.0, lmax = 0.0;  // log of terms x^m / m!, m < n
    std::vector<double> terms((size_t)n);
    for (int m = 0; m < n; ++m) {
        lt = (m == 0) ? 0.0 : lt + std::log(x) - std::log((double)m);
        terms[(size_t)m] = lt;
        lmax = (m == 0) ? lt : std::max(lmax, lt);
    }
    double s = 0.0;
    for (double t : terms) s += std::exp(t - lmax);
    return x - (lmax + std::log(s));
}

}  // namespace

extern "C" int bps_distill(const bps_candidate* in, int64_t n_in, int64_t n_samples,
                           double tsamp_s, double tol_bins, int32_t max_ratio,
                           bps_candidate* out, int64_t cap, int64_t* n_out)
try {
    if ((!in && n_in > 0) || n_in < 0 || n_samples < 2 || !(tsamp_s > 0.0) ||
        !(tol_bins > 0.0) || max_ratio < 1 || max_ratio > 64 || !n_out || cap < 0)
        return BPS_ERR_INVALID_ARG;
    const double T = (double)n_samples * tsamp_s;
    struct Item {
        double f, sig;
        int64_t i;
    };
    std::vector<Item> it((size_t)n_in);
    for (int64_t i = 0; i < n_in; ++i) {
        const bps_candidate& c = in[i];
        if (c.nharm == 0) return BPS_ERR_INVALID_ARG;
        it[(size_t)i] = {(double)c.bin / ((double)c.nharm * T), neg_log_q(c.nharm, c.power), i};
    }
    std::sort(it.begin(), it.end(), [](const Item& a, const Item& b) {
        if (a.sig != b.sig) return a.sig > b.sig;
        return a.i < b.i;
    });
    std::vector<char> used((size_t)n_in, 0);
    const double tol = tol_bins / T;  // frequency tolerance of one fundamental bin
    int64_t k = 0;
    for (size_t a = 0; a < it.size(); ++a) {
        if (used[a]) continue;
        used[a] = 1;
        int64_t members = 1;
        const double f0 = it[a].f;
        for (size_t b = a + 1; b < it.size(); ++b) {
            if (used[b]) continue;
            const double f = it[b].f;
            bool rel = false;
            for (int p = 1; p <= max_ratio && !rel; ++p)
                for (int q = 1; q <= max_ratio && !rel; ++q)
                    // f / f0 = p / q within the tolerance scaled by the larger multiple
                    rel = std::fabs(q * f - p * f0) <= tol * (double)std::max(p, q);
            if (rel) {
                used[b] = 1;
                ++members;
            }
        }
        if (k < cap && out) {
            out[k] = in[it[a].i];
            out[k].flags = (uint16_t)std::min<int64_t>(members, 65535);
        }
        ++k;
    }
    *n_out = k;
    return k > cap ? BPS_ERR_CAND_OVERFLOW : BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}
