// bps_api.cu -- host runtime behind the C ABI of include/bps.h: contexts,
// device-resident series and banks, the planner, stream-ordered searches,
// candidate fetch, and the stage entry points.
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
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

// Geometry (plan_geometry) + anchor block length (plan_anchor_block).
int make_plan(bps_ctx* ctx, const Series& s, const Bank& b, const bps_search_params& pr,
              Plan& p)
{
    p.n = s.n;
    p.logn = ilog2(s.n);
    p.M = s.n / 2;
    p.logM = p.logn - 1;
    plan_geometry(p, pr.log_tile ? pr.log_tile : 14, pr.log_tile2 ? pr.log_tile2 : 13);
    p.logW = ilog2(pr.whiten_block);
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
    v.fill = (float)s.mean;
    return v;
}

int default_batch(const Plan& p, int64_t K, int mode)
{
    if (mode == BPS_MODE_PLAIN) return 1;
    int64_t nt = std::max<int64_t>(1, (1ll << 25) / p.M);
    nt = std::min<int64_t>(nt, 64);
    return (int)std::min<int64_t>(nt, std::max<int64_t>(K, 1));
}

struct Workspace {
    Anchor* anc = nullptr;
    float2* Y = nullptr;   // fused: M complex per template; plain: R2C output (M+1)
    float* x = nullptr;    // plain: resampled series
    float* P = nullptr;
    float* scale = nullptr;
    char* base = nullptr;
};

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Anchors are computed for a chunk of up to kAnchorChunk batches in one launch.
constexpr int kAnchorChunk = 8;

int ws_alloc(bps_ctx* ctx, const Plan& p, int nt, int mode, cudaStream_t st, Workspace& w,
             int anchor_templates = 0)
{
    const size_t a = align256(sizeof(Anchor) * (size_t)p.nanchor *
                              (anchor_templates > 0 ? anchor_templates : nt));
    const size_t y = align256(sizeof(float2) * (size_t)(p.M + 1) * nt);
    const size_t x = mode == BPS_MODE_PLAIN ? align256(sizeof(float) * (size_t)p.n * nt) : 0;
    const size_t pp = align256(sizeof(float) * (size_t)p.M * nt);
    const size_t sc = align256(sizeof(float) * (size_t)(p.M >> p.logW) * nt);
    CK(cudaMallocAsync((void**)&w.base, a + y + x + pp + sc, st));
    char* q = w.base;
    w.anc = (Anchor*)q; q += a;
    w.Y = (float2*)q; q += y;
    w.x = x ? (float*)q : nullptr; q += x;
    w.P = (float*)q; q += pp;
    w.scale = (float*)q;
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
        CK(launch_pass2(w.Y, nt, p, ctx->tw, w.P, st));
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
    CK(launch_block_median(w.P, nt, p, w.scale, st));
    tm.end();
    return BPS_OK;
}

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
}

int bps_create(bps_ctx** out, int device)
{
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
}

static void free_series(Series& s)
{
    if (s.owned && s.f32) cudaFree(s.f32);
    if (s.f16) cudaFree(s.f16);
    if (s.scale) cudaFree(s.scale);
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
{
    if (!ctx) return;
    {
        std::lock_guard<std::recursive_mutex> lk(ctx->mu);
        cudaSetDevice(ctx->device);
        cudaDeviceSynchronize();
        for (auto& r : ctx->reqs) free_request(r.second);
        for (auto& s : ctx->series) free_series(s.second);
        for (auto& b : ctx->banks) cudaFree(b.second.d);
        for (auto& f : ctx->ffts) cufftDestroy(f.second);
        if (ctx->tw) cudaFree(ctx->tw);
        if (ctx->stream) cudaStreamDestroy(ctx->stream);
    }
    delete ctx;
}

const char* bps_last_error(bps_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int bps_load_series(bps_ctx* ctx, const void* data, int64_t n, double tsamp_s, int dtype,
                    int on_device, int64_t* series_id)
{
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
    double* dsum = nullptr;
    CK(cudaMallocAsync((void**)&dsum, sizeof(double), st));
    CK(cudaMemsetAsync(dsum, 0, sizeof(double), st));
    CK(launch_series_stats(src, n, dsum, st));
    double sum = 0;
    CK(cudaMemcpyAsync(&sum, dsum, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaFreeAsync(dsum, st));
    if (dtype == BPS_F32) {
        s.f32 = src;
        s.owned = tmp;
    } else {
        CK(cudaMalloc((void**)&s.f16, sizeof(uint16_t) * n));
        CK(cudaMalloc((void**)&s.scale, sizeof(float) * ((n + 4095) >> 12)));
        CK(launch_f16_pack(src, n, s.f16, s.scale, st));
    }
    CK(cudaStreamSynchronize(st));
    if (dtype != BPS_F32 && tmp) cudaFree(src);
    s.mean = sum / (double)n;
    const int64_t id = ctx->next_id++;
    ctx->series[id] = s;
    *series_id = id;
    return BPS_OK;
}

int bps_load_bank(bps_ctx* ctx, const bps_template* t, int64_t count, int64_t* bank_id)
{
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
}

int bps_thresholds(const bps_search_params* params, int64_t n_samples, int64_t n_templates,
                   double* thr_out)
{
    if (!params || !thr_out || check_params(nullptr, params, n_samples)) return BPS_ERR_INVALID_ARG;
    thresholds(params, n_samples, n_templates, thr_out);
    return BPS_OK;
}

int bps_search(bps_ctx* ctx, int64_t series_id, int64_t bank_id, const bps_search_params* params,
               void* cuda_stream, int64_t* req_id)
{
    if (!ctx) return BPS_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (!req_id) return fail(ctx, BPS_ERR_INVALID_ARG, "req_id is NULL");
    Series* s;
    Bank* b;
    int rc = lookup(ctx, series_id, bank_id, s, b);
    if (rc) return rc;
    if ((rc = check_params(ctx, params, s->n))) return rc;
    Plan p;
    if ((rc = make_plan(ctx, *s, *b, *params, p))) return rc;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
    double thr[5];
    thresholds(params, s->n, b->K, thr);
    Thr th;
    for (int L = 0; L < 5; ++L) th.v[L] = L < p.nlev ? (float)thr[L] : 0.f;
    Request r;
    r.series = series_id;
    r.bank = bank_id;
    r.K = b->K;
    r.cap = params->cand_cap;
    CK(cudaMalloc((void**)&r.d_cands, sizeof(Cand) * (size_t)r.cap));
    CK(cudaMalloc((void**)&r.d_count, 2 * sizeof(unsigned long long)));  // count, status
    CK(cudaMemsetAsync(r.d_count, 0, 2 * sizeof(unsigned long long), st));
    CK(cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming));
    const int nt = params->batch > 0 ? (int)std::min<int64_t>(params->batch, b->K)
                                     : default_batch(p, b->K, params->mode);
    const int64_t chunk = std::min<int64_t>((int64_t)nt * kAnchorChunk, b->K);
    Workspace w;
    if ((rc = ws_alloc(ctx, p, nt, params->mode, st, w, (int)chunk))) {
        free_request(r);
        return rc;
    }
    r.batch = nt;
    r.logB = p.logB;
    StageTimer tm;
    tm.r = &r;
    tm.st = st;
    tm.prof = ctx->profiling;
    for (int64_t c0 = 0; c0 < b->K && !rc; c0 += chunk) {
        const int ccnt = (int)std::min<int64_t>(chunk, b->K - c0);
        tm.begin(BPS_STAGE_ANCHORS);
        cudaError_t e = launch_anchors(b->d, c0, ccnt, p, w.anc, st);
        tm.end();
        if (e != cudaSuccess) {
            rc = fail(ctx, BPS_ERR_CUDA, "anchor launch: %s", cudaGetErrorString(e));
            break;
        }
        for (int64_t t0 = c0; t0 < c0 + ccnt; t0 += nt) {
            const int cnt = (int)std::min<int64_t>(nt, c0 + ccnt - t0);
            if ((rc = run_spectrum(ctx, *s, *b, p, params->mode, t0, cnt, w, st, tm,
                                   w.anc + (t0 - c0) * p.nanchor)))
                break;
            tm.begin(BPS_STAGE_HARMSUM);
            e = launch_harmsum(w.P, w.scale, cnt, t0, p, th, r.d_cands, r.cap, r.d_count, nullptr,
                               st);
            tm.end();
            if (e != cudaSuccess) {
                rc = fail(ctx, BPS_ERR_CUDA, "harmonic-sum launch: %s", cudaGetErrorString(e));
                break;
            }
        }
    }
    cudaFreeAsync(w.base, st);
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
}

int bps_query(bps_ctx* ctx, int64_t req_id, int* done)
{
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
}

int bps_fetch_candidates(bps_ctx* ctx, int64_t req_id, bps_candidate* out, int64_t cap,
                         int64_t* n_written, int64_t* n_total)
{
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
        std::sort(r.result.begin(), r.result.end(), [](const bps_candidate& a, const bps_candidate& b) {
            if (a.template_idx != b.template_idx) return a.template_idx < b.template_idx;
            if (a.nharm != b.nharm) return a.nharm < b.nharm;
            return a.bin < b.bin;
        });
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
}

int bps_unload(bps_ctx* ctx, int64_t id)
{
    if (!ctx) return BPS_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
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
    if (ctx->reqs.count(id)) {
        free_request(ctx->reqs[id]);
        ctx->reqs.erase(id);
        return BPS_OK;
    }
    return fail(ctx, BPS_ERR_INVALID_ARG, "unknown id %lld", (long long)id);
}

int bps_set_profiling(bps_ctx* ctx, int on)
{
    if (!ctx) return BPS_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    ctx->profiling = on != 0;
    return BPS_OK;
}

int bps_request_stats(bps_ctx* ctx, int64_t req_id, bps_stats* out)
{
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
}

int bps_index_map(bps_ctx* ctx, int64_t series_id, int64_t bank_id, int64_t template_idx,
                  int32_t* idx_out, int64_t* n_precise)
{
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
}

int bps_whitened_spectrum(bps_ctx* ctx, int64_t series_id, int64_t bank_id, int64_t t0,
                          int64_t count, const bps_search_params* params, float* pw_out)
{
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
}

int bps_harmonic_sums(bps_ctx* ctx, int64_t series_id, int64_t bank_id, int64_t template_idx,
                      const bps_search_params* params, float* s_out)
{
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
}

}  // extern "C"
