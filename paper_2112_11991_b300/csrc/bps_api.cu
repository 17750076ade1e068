// bps_api.cu -- host runtime behind the C ABI of include/bps.h: contexts,
// device-resident series and banks, stream-ordered searches, candidate fetch, CUDA
// graphs, the launch-shape autotuner and the stage entry points.
#include "bps_runtime.h"

using namespace bps;
using namespace bps::rt;

namespace bps {
namespace rt {

// Searches of a list of (series, bank) pairs captured into one CUDA graph: series too
// large for four to share the L2 are searched one after another on one branch, then the
// other pairs are spread over up to kGraphBranches parallel branches (fork/join events
// during the capture); the pairs of one branch run in sequence and share its workspace.
// Each pair has its own candidate region (cap candidates) and counter.
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

}  // namespace rt
}  // namespace bps

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
    cudaMemPoolProps pp;
    std::memset(&pp, 0, sizeof pp);
    pp.allocType = cudaMemAllocationTypePinned;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = device;
    uint64_t keep = UINT64_MAX;
    if (cudaSetDevice(device) != cudaSuccess || cudaMemPoolCreate(&ctx->pool, &pp) != cudaSuccess ||
        cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc((void**)&ctx->tw, kTwiddleN * sizeof(float2)) != cudaSuccess ||
        launch_twiddle_init(ctx->tw, ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        if (ctx->tw) cudaFree(ctx->tw);
        if (ctx->stream) cudaStreamDestroy(ctx->stream);
        if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
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

// Return a request's device buffers to the context's pool (after its work is done) and
// its completion event to the free list.
static void free_request(bps_ctx* ctx, Request& r)
{
    for (auto& e : r.ev) {
        cudaEventDestroy(e.second.first);
        cudaEventDestroy(e.second.second);
    }
    r.ev.clear();
    if (r.done) cudaEventSynchronize(r.done);
    if (r.d_cands) cudaFreeAsync(r.d_cands, ctx->stream);
    if (r.d_count) cudaFreeAsync(r.d_count, ctx->stream);
    event_put(ctx, r.done);
    r = Request();
}

void bps_destroy(bps_ctx* ctx)
try {
    if (!ctx) return;
    {
        std::lock_guard<std::recursive_mutex> lk(ctx->mu);
        cudaSetDevice(ctx->device);
        cudaDeviceSynchronize();
        for (auto& r : ctx->reqs) free_request(ctx, r.second);
        for (auto& s : ctx->series) free_series(s.second);
        for (auto& b : ctx->banks) cudaFree(b.second.d);
        for (auto& f : ctx->ffts) cufftDestroy(f.second);
        for (auto& gr : ctx->graphs) delete gr.second;
        if (ctx->tw) cudaFree(ctx->tw);
        for (auto e : ctx->free_events) cudaEventDestroy(e);
        if (ctx->stream) {
            cudaStreamSynchronize(ctx->stream);
            cudaStreamDestroy(ctx->stream);
        }
        if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
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
        CK(pool_alloc(ctx, (void**)&src, bytes, st));
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
    const std::vector<DevTemplate> dt = dev_templates(t, count);
    CK(cudaMalloc((void**)&b.d, sizeof(DevTemplate) * count));
    CK(cudaMemcpy(b.d, dt.data(), sizeof(DevTemplate) * count, cudaMemcpyHostToDevice));
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
    // candidate buffer, counter + status word and completion event: stream-ordered from
    // the context's pool and free list (no synchronous allocation per request)
    CK(pool_alloc(ctx, (void**)&r.d_cands, sizeof(Cand) * (size_t)r.cap, st));
    CK(pool_alloc(ctx, (void**)&r.d_count, 2 * sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(r.d_count, 0, 2 * sizeof(unsigned long long), st));
    CK(event_get(ctx, &r.done));
    Job job;
    if ((rc = job.setup(ctx, s, b, *params, st, r.d_cands, r.d_count, r.cap))) {
        cudaStreamSynchronize(st);
        free_request(ctx, r);
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
        free_request(ctx, r);
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
        cudaFreeAsync(r.d_cands, ctx->stream);  // the request's work is done (synchronised)
        r.d_cands = nullptr;
    }
    const int64_t nw = std::min<int64_t>(cap, (int64_t)r.result.size());
    if (out && nw > 0) std::memcpy(out, r.result.data(), sizeof(bps_candidate) * nw);
    if (n_written) *n_written = out ? nw : 0;
    if (n_total) *n_total = (int64_t)r.total;
    if (r.status != 0)
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
        free_request(ctx, ctx->reqs[id]);
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
    // L2-aware schedule: a series that a quarter of the L2 cannot hold is searched alone
    // (phase A, one branch, in the order given), so its gathers stay in the L2 across the
    // bank's templates; the smaller ones run on B parallel branches (phase B), each pair on
    // the branch with the least work so far (templates x n log2 n)
    int l2 = 0;
    CK(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, ctx->device));
    std::vector<int> branch((size_t)count, 0);
    std::vector<char> big((size_t)count, 0);
    std::vector<double> load((size_t)B, 0.0);
    for (int64_t i = 0; i < count; ++i) {
        int rc = lookup(ctx, series_ids[i], bank_ids[i], ss[i], bb[i]);
        if (rc) return rc;
        if ((rc = check_params(ctx, params, ss[i]->n))) return rc;
        Plan p;
        if ((rc = make_plan(ctx, *ss[i], *bb[i], *params, p))) return rc;
        const size_t sbytes = (size_t)ss[i]->n * (ss[i]->dtype == BPS_F32 ? 4 : 2);
        big[i] = (B > 1 && sbytes * 4 > (size_t)l2) ? 1 : 0;
        if (!big[i]) {
            const int bmin = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            branch[i] = bmin;
            load[bmin] += (double)bb[i]->K * (double)ss[i]->n * (double)p.logn;
        }
        int nt = params->batch > 0 ? (int)std::min<int64_t>(params->batch, bb[i]->K)
                                   : default_batch(p, bb[i]->K, params->mode);
        auto it = ctx->tuned.find(tune_key(p.logn, params->mode, p.lognh));
        if (params->batch == 0 && it != ctx->tuned.end()) nt = (int)std::min<int64_t>(it->second[2], bb[i]->K);
        const int64_t chunk = std::min<int64_t>((int64_t)nt * kAnchorChunk, bb[i]->K);
        size_t& w = wsb[branch[i]];
        w = std::max(w, ws_carve(p, nt, params->mode, (int)chunk, nullptr, nullptr));
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
    cudaEvent_t fork, phase_a;
    std::vector<cudaEvent_t> join((size_t)B);
    CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&phase_a, cudaEventDisableTiming));
    for (auto& e : join) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    int rc = BPS_OK;
    cudaError_t ce = cudaStreamBeginCapture(os, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
        cudaMemsetAsync(g->counts, 0, 2 * sizeof(unsigned long long) * count, os);
        cudaEventRecord(fork, os);
        cudaStreamWaitEvent(br[0], fork, 0);
        auto capture_pair = [&](int64_t i) {
            const int b = branch[i];
            Job job;
            rc = job.setup(ctx, ss[i], bb[i], *params, br[b], g->cands + (size_t)i * g->cap,
                           g->counts + 2 * i, g->cap, g->wsbuf[b], wsb[b]);
            while (!rc && !job.done()) rc = job.issue_batch();
        };
        for (int64_t i = 0; i < count && !rc; ++i)  // phase A: large series, one at a time
            if (big[i]) capture_pair(i);
        cudaEventRecord(phase_a, br[0]);
        for (int b = 1; b < B; ++b) cudaStreamWaitEvent(br[b], phase_a, 0);
        for (int64_t i = 0; i < count && !rc; ++i)  // phase B: the rest, B branches
            if (!big[i]) capture_pair(i);
        for (int b = 0; b < B; ++b) {
            cudaEventRecord(join[b], br[b]);
            cudaStreamWaitEvent(os, join[b], 0);
        }
        ce = cudaStreamEndCapture(os, &g->graph);
        if (ce == cudaSuccess && !rc) ce = cudaGraphInstantiate(&g->exec, g->graph, 0);
    }
    cudaEventDestroy(fork);
    cudaEventDestroy(phase_a);
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
    if (g.status[pair] != 0) return fail(ctx, BPS_ERR_TIMEOUT, "a bounded device wait expired");
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
    const int tiles2[3] = {12, 13, 14};  // pass 2 (2^12: four 256-thread CTAs per SM)
    const int batches[4] = {8, 16, 32, 64};
    // four-step splits: the caller's, else the library's and its valid neighbours
    const int logM = ilog2(s->n) - 1;
    std::vector<int> splits;
    if (base->log_cols) splits.push_back(base->log_cols);
    else if (base->mode == BPS_MODE_PLAIN) splits.push_back(0);
    else
        for (int d : {0, -1, 1, 2})
            if (log_cols_ok(logM, default_log_cols(logM) + d)) splits.push_back(default_log_cols(logM) + d);
    double best_ms = 1e30;
    bps_search_params bp = *base;
    // pass 1: the one-phase kernel at both tiles, and the warp-specialised one where built
    std::vector<std::pair<int, int>> p1;  // (kind, tile)
    if (base->pass1_kind == BPS_PASS1_AUTO || base->pass1_kind == BPS_PASS1_FUSED)
        for (int t : tiles) p1.push_back({BPS_PASS1_FUSED, t});
    if (base->mode == BPS_MODE_FUSED && (base->pass1_kind == BPS_PASS1_AUTO || base->pass1_kind == BPS_PASS1_WARPSPEC))
        p1.push_back({BPS_PASS1_WARPSPEC, 13});
    if (base->mode == BPS_MODE_FUSED && (base->pass1_kind == BPS_PASS1_AUTO || base->pass1_kind == BPS_PASS1_ASYNC))
        p1.push_back({BPS_PASS1_ASYNC, 13});
    // pass 2: the one-phase kernel at both tiles, and the TMA-fed one (2^13 tiles) where built
    std::vector<std::pair<int, int>> p2;  // (kind, tile)
    if (base->pass2_kind != BPS_PASS2_TMA)
        for (int t : tiles2) p2.push_back({BPS_PASS2_FUSED, t});
    if (base->mode == BPS_MODE_FUSED && base->pass2_kind != BPS_PASS2_FUSED) p2.push_back({BPS_PASS2_TMA, 13});
    for (int lc : splits)
    for (auto k1 : p1)
        for (auto k2 : p2)
            for (int nb : batches) {
                if (nb > sub.K) continue;
                const int lcx = lc ? lc : default_log_cols(logM);
                if (k1.first != BPS_PASS1_FUSED && !ws_pass1_built(logM - lcx, lcx)) continue;
                if (k2.first == BPS_PASS2_TMA && !tma_pass2_built(logM - lcx, lcx, 13)) continue;
                bps_search_params pr = *base;
                pr.pass1_kind = k1.first;
                pr.log_tile = k1.second;
                pr.pass2_kind = k2.first;
                pr.log_tile2 = k2.second;
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
    ctx->tuned[tune_key(ilog2(s->n), base->mode, ilog2(base->nharm_max))] = {
        bp.log_tile, bp.log_tile2, bp.batch, bp.log_cols, bp.pass1_kind, bp.power_layout, bp.pass2_kind};
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
    CK(pool_alloc(ctx, (void**)&anc, sizeof(Anchor) * p.nanchor, st));
    CK(pool_alloc(ctx, (void**)&idx, sizeof(int32_t) * p.n, st));
    CK(pool_alloc(ctx, (void**)&cnt, sizeof(unsigned long long), st));
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
    unsigned long long* stw = nullptr;
    unsigned long long stv = 0;
    CK(pool_alloc(ctx, (void**)&out, sizeof(float) * p.M * nt, st));
    CK(pool_alloc(ctx, (void**)&stw, sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(stw, 0, sizeof(unsigned long long), st));
    StageTimer tm;
    if ((rc = run_spectrum(ctx, *s, *b, p, params->mode, t0, nt, w, st, tm, stw))) return rc;
    CK(launch_whitened(w.P, w.scale, nt, p, out, st));
    CK(cudaMemcpyAsync(pw_out, out, sizeof(float) * p.M * nt, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&stv, stw, sizeof stv, cudaMemcpyDeviceToHost, st));
    CK(cudaFreeAsync(out, st));
    CK(cudaFreeAsync(stw, st));
    CK(cudaFreeAsync(w.base, st));
    CK(cudaStreamSynchronize(st));
    if (stv) return fail(ctx, BPS_ERR_TIMEOUT, "a bounded device wait expired; spectrum incomplete");
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
    CK(pool_alloc(ctx, (void**)&so, sizeof(float) * p.M * p.nlev, st));
    CK(pool_alloc(ctx, (void**)&cd, sizeof(Cand), st));
    CK(pool_alloc(ctx, (void**)&cnt, 2 * sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), st));
    StageTimer tm;
    if ((rc = run_spectrum(ctx, *s, *b, p, params->mode, template_idx, 1, w, st, tm, cnt + 1))) return rc;
    Thr th;
    for (int L = 0; L < 5; ++L) th.v[L] = INFINITY;
    CK(launch_harmsum(w.P, w.scale, 1, template_idx, p, th, cd, 1, cnt, so, w.tile_ctr, st));
    unsigned long long cs[2] = {0, 0};
    CK(cudaMemcpyAsync(s_out, so, sizeof(float) * p.M * p.nlev, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(cs, cnt, sizeof cs, cudaMemcpyDeviceToHost, st));
    CK(cudaFreeAsync(so, st));
    CK(cudaFreeAsync(cd, st));
    CK(cudaFreeAsync(cnt, st));
    CK(cudaFreeAsync(w.base, st));
    CK(cudaStreamSynchronize(st));
    if (cs[1]) return fail(ctx, BPS_ERR_TIMEOUT, "a bounded device wait expired; sums incomplete");
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
