// bps_server.cu -- the serving loop behind bps_server_* (include/bps.h).
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <thread>

#include "bps_runtime.h"

// =====================================================================================
// Serving: a continuously batched request loop.  A worker thread admits queued
// requests onto stream slots while the HBM budget allows, stages their series and bank
// on the device, then issues their launch groups round-robin (a few in flight per
// request), and retires finished requests (candidates to the host, device memory
// freed, slot released) so the next queued request can start.
//
// Resident series (bps_server_load_series): a series loaded into the server stays on
// the device between requests that name it, counted against the HBM budget.  When a
// request needs room, resident series that no queued or running request names are
// evicted, least recently used first; the server keeps each series' pinned host copy,
// so an evicted series is staged again by the next request that names it.
// Device memory (series, banks, workspaces, candidates) comes from the context's
// stream-ordered pool, which keeps freed blocks mapped for the next request.
// =====================================================================================

using namespace bps;
using namespace bps::rt;

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

enum SState { S_QUEUED, S_STAGING, S_RUNNING, S_COUNTING, S_COPYING, S_DONE, S_FAILED };

constexpr int64_t kPinnedCands = 1 << 16;  // candidates copied back through pinned memory

struct SSeries;

struct SReq {
    int64_t ticket = 0;
    SState state = S_QUEUED;
    SSeries* ser = nullptr;     // resident series the request names (nullptr: its own copy)
    bool staged_here = false;   // this request's admission began staging ser
    float* h_series = nullptr;  // pinned host copy of the submitted series
    int64_t n = 0;
    double tsamp = 0;
    int dtype = BPS_F32;
    std::vector<bps_template> bank;
    std::vector<DevTemplate> dbank;  // device form of the bank (kept until its copy is done)
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

// A series loaded into the server: pinned host copy (kept for re-staging) and, while
// resident, its device storage.
struct SSeries {
    int64_t id = 0;
    int64_t n = 0;
    double tsamp = 0;
    int dtype = BPS_F32;
    float* h_series = nullptr;
    double* h_sum = nullptr;
    Series s;                  // device storage while resident (staging or staged)
    float* d_stage = nullptr;  // FP32 staging buffer of an FP16 series while it is packed
    double* d_sum = nullptr;
    cudaEvent_t ready = nullptr;
    bool resident = false, staging = false;
    size_t bytes = 0;          // device bytes while resident (after packing)
    size_t stage_bytes = 0;    // extra bytes while staging (the FP32 buffer of FP16 packing)
    int refs = 0;              // queued and running requests naming it
    int64_t times_staged = 0;
    double last_use = 0;
};

// Device bytes of a series (FP32, or FP16 + scales) and of its FP32 staging buffer.
size_t series_bytes(int64_t n, int dtype, size_t* staging)
{
    if (staging) *staging = dtype == BPS_F32 ? 0 : align256(4 * (size_t)n);
    return dtype == BPS_F32 ? align256(4 * (size_t)n)
                            : align256(2 * (size_t)n) + align256(4 * (size_t)(((n + 4095) >> 12) + 1));
}

// Device bytes a request holds while resident (bank + workspace + candidates, plus its
// own series unless it names a resident one).
size_t request_bytes(const Plan& p, int64_t K, const bps_search_params& prm, int dtype, bool own_series)
{
    const int nt = prm.batch > 0 ? (int)std::min<int64_t>(prm.batch, K) : default_batch(p, K, prm.mode);
    const int64_t chunk = std::min<int64_t>((int64_t)nt * kAnchorChunk, K);
    size_t stg = 0;
    const size_t ser = own_series ? series_bytes(p.n, dtype, &stg) + stg : 0;
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
    std::map<int64_t, std::unique_ptr<SSeries>> series;  // resident-series store
    int64_t next_series = 1;
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
    if (q.ser) {  // the storage belongs to the resident series
        q.s.f32 = nullptr;
        q.s.f16 = nullptr;
        q.s.scale = nullptr;
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

void free_series_host(SSeries& ser)
{
    if (ser.h_series) cudaFreeHost(ser.h_series);
    if (ser.h_sum) cudaFreeHost(ser.h_sum);
    if (ser.ready) cudaEventDestroy(ser.ready);
    ser.h_series = nullptr;
    ser.h_sum = nullptr;
    ser.ready = nullptr;
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

// Stage a resident series on stream st: device storage from the pool, the host copy,
// the FP64 sum (read back for the fill value) and FP16 packing; ser->ready marks the end.
cudaError_t stage_series(bps_server* srv, SSeries& ser, cudaStream_t st)
{
    const size_t n = (size_t)ser.n;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t r) {
        if (e == cudaSuccess) e = r;
    };
    ser.s = Series();
    ser.s.n = ser.n;
    ser.s.tsamp = ser.tsamp;
    ser.s.dtype = ser.dtype;
    ser.s.owned = true;
    float* src = nullptr;
    if (ser.dtype == BPS_F32) {
        chk(pool_alloc(srv->ctx, (void**)&ser.s.f32, 4 * n, st));
        src = ser.s.f32;
    } else {
        chk(pool_alloc(srv->ctx, (void**)&ser.d_stage, 4 * n, st));
        chk(pool_alloc(srv->ctx, (void**)&ser.s.f16, 2 * n, st));
        chk(pool_alloc(srv->ctx, (void**)&ser.s.scale, 4 * (((n + 4095) >> 12) + 1), st));
        src = ser.d_stage;
    }
    chk(pool_alloc(srv->ctx, (void**)&ser.d_sum, sizeof(double), st));
    if (e == cudaSuccess) {
        chk(cudaMemcpyAsync(src, ser.h_series, 4 * n, cudaMemcpyHostToDevice, st));
        chk(cudaMemsetAsync(ser.d_sum, 0, sizeof(double), st));
        chk(launch_series_stats(src, ser.n, ser.d_sum, st));
        if (ser.dtype != BPS_F32) chk(launch_f16_pack(src, ser.n, ser.s.f16, ser.s.scale, st));
        chk(cudaMemcpyAsync(ser.h_sum, ser.d_sum, sizeof(double), cudaMemcpyDeviceToHost, st));
        chk(cudaEventRecord(ser.ready, st));
    }
    ser.staging = true;
    ser.times_staged += 1;
    srv->used += ser.bytes + ser.stage_bytes;
    return e;
}

// Free a resident series' device storage (no request names it, so none of its work is
// in flight) and return its bytes to the budget.
void evict_series(bps_server* srv, SSeries& ser)
{
    cudaStream_t st = srv->ctx->stream;
    if (ser.s.f32) cudaFreeAsync(ser.s.f32, st);
    if (ser.s.f16) cudaFreeAsync(ser.s.f16, st);
    if (ser.s.scale) cudaFreeAsync(ser.s.scale, st);
    if (ser.d_stage) cudaFreeAsync(ser.d_stage, st);
    if (ser.d_sum) cudaFreeAsync(ser.d_sum, st);
    ser.s = Series();
    ser.d_stage = nullptr;
    ser.d_sum = nullptr;
    srv->used -= ser.bytes + (ser.staging ? ser.stage_bytes : 0);
    ser.resident = ser.staging = false;
}

// Evict idle resident series, least recently used first, until `need` more bytes fit the
// budget (or nothing idle is left); `keep` is never evicted.
void make_room(bps_server* srv, size_t need, const SSeries* keep)
{
    while (srv->used + need > srv->budget) {
        SSeries* lru = nullptr;
        for (auto& kv : srv->series) {
            SSeries& c = *kv.second;
            if (&c == keep || c.refs > 0 || !(c.resident || c.staging)) continue;
            if (!lru || c.last_use < lru->last_use) lru = &c;
        }
        if (!lru) return;
        evict_series(srv, *lru);
    }
}

// Stage a queued request onto a free slot: device buffers (stream-ordered), series and
// bank copies, FP16 packing, the FP64 series sum read back for the fill value.  A
// request naming a resident series stages the series if it is not on the device and
// then waits for it on its own stream.
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
    q.dbank = dev_templates(q.bank.data(), (int64_t)q.bank.size());
    if (q.ser) {
        SSeries& ser = *q.ser;
        ser.last_use = now_s();
        if (!ser.resident && !ser.staging) {
            q.staged_here = true;
            chk(stage_series(srv, ser, st));
        }
        if (ok) chk(cudaStreamWaitEvent(st, ser.ready, 0));
        chk(pool_alloc(srv->ctx, (void**)&q.b.d, sizeof(DevTemplate) * q.bank.size(), st));
        chk(pool_alloc(srv->ctx, (void**)&q.d_cands, sizeof(Cand) * (size_t)q.prm.cand_cap, st));
        chk(pool_alloc(srv->ctx, (void**)&q.d_count, 2 * sizeof(unsigned long long), st));
        if (ok) {
            chk(cudaMemcpyAsync(q.b.d, q.dbank.data(), sizeof(DevTemplate) * q.bank.size(),
                                cudaMemcpyHostToDevice, st));
            chk(cudaMemsetAsync(q.d_count, 0, 2 * sizeof(unsigned long long), st));
            chk(cudaEventRecord(q.ev, st));
        }
        srv->busy[slot] = 1;
        srv->used += q.bytes;
        q.state = ok ? S_STAGING : S_FAILED;
        return ok;
    }
    float* src = nullptr;
    if (q.dtype == BPS_F32) {
        chk(pool_alloc(srv->ctx, (void**)&q.s.f32, 4 * n, st));
        src = q.s.f32;
    } else {
        chk(pool_alloc(srv->ctx, (void**)&q.d_stage, 4 * n, st));
        chk(pool_alloc(srv->ctx, (void**)&q.s.f16, 2 * n, st));
        chk(pool_alloc(srv->ctx, (void**)&q.s.scale, 4 * (((n + 4095) >> 12) + 1), st));
        src = q.d_stage;
    }
    chk(pool_alloc(srv->ctx, (void**)&q.d_sum, sizeof(double), st));
    chk(pool_alloc(srv->ctx, (void**)&q.b.d, sizeof(DevTemplate) * q.bank.size(), st));
    chk(pool_alloc(srv->ctx, (void**)&q.d_cands, sizeof(Cand) * (size_t)q.prm.cand_cap, st));
    chk(pool_alloc(srv->ctx, (void**)&q.d_count, 2 * sizeof(unsigned long long), st));
    if (ok) {
        chk(cudaMemcpyAsync(src, q.h_series, 4 * n, cudaMemcpyHostToDevice, st));
        chk(cudaMemcpyAsync(q.b.d, q.dbank.data(), sizeof(DevTemplate) * q.bank.size(),
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
    if (q.ser) {
        // a failed request that began staging its series takes the half-staged copy down
        // (its stream is synchronised; requests waiting on the series then fail too)
        if (st_ == S_FAILED && q.staged_here && q.ser->staging) evict_series(srv, *q.ser);
        q.ser->refs -= 1;
        q.ser->last_use = now_s();
    }
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
            if (q.ser) {
                SSeries& ser = *q.ser;
                if (!ser.staging && !ser.resident) {  // its staging failed and was taken down
                    q.rc = BPS_ERR_CUDA;
                    q.err = "staging the resident series failed";
                    cudaStreamSynchronize(st);
                    finish(srv, q, S_FAILED);
                    return true;
                }
                if (ser.staging) {  // the series' staging has completed (the event waited on it)
                    if (ser.d_stage) {
                        cudaFreeAsync(ser.d_stage, st);
                        ser.d_stage = nullptr;
                    }
                    srv->used -= ser.stage_bytes;
                    ser.staging = false;
                    ser.resident = true;
                    ser.s.mean = *ser.h_sum / (double)ser.n;
                }
                q.s = ser.s;
            }
            if (q.d_stage) {
                cudaFreeAsync(q.d_stage, st);
                q.d_stage = nullptr;
            }
            if (q.h_series) {
                cudaFreeHost(q.h_series);
                q.h_series = nullptr;
            }
            if (!q.ser) q.s.mean = *q.h_sum / (double)q.n;
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
            if (q.status != 0) {
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
                if (slot < 0) break;
                size_t need = q.bytes;
                if (q.ser && !q.ser->resident && !q.ser->staging)
                    need += q.ser->bytes + q.ser->stage_bytes;
                if (srv->used + need > srv->budget) make_room(srv, need, q.ser);
                if (srv->used + need > srv->budget) break;
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
    {
        std::lock_guard<std::recursive_mutex> cl(srv->ctx->mu);
        for (auto& kv : srv->series) {
            if (kv.second->resident || kv.second->staging) evict_series(srv, *kv.second);
            free_series_host(*kv.second);
        }
        cudaStreamSynchronize(srv->ctx->stream);
    }
    delete srv;
} catch (...) {
}

const char* bps_server_last_error(bps_server* srv) { return srv ? srv->err.c_str() : "null server"; }

}  // extern "C"

namespace {

bool series_args_ok(int64_t n, double tsamp_s, int dtype)
{
    return is_pow2(n) && n >= (1 << 11) && n <= (1 << 25) && tsamp_s > 0.0 && std::isfinite(tsamp_s) &&
           (dtype == BPS_F32 || dtype == BPS_F16_SCALED);
}

// Checks a request and builds its record (pinned host buffers, events, device bytes).
// `own_series`: the request carries its own series copy (bps_server_submit), else it names
// a resident series (bps_server_submit_series).
int make_request(bps_server* srv, int64_t n, double tsamp_s, int dtype, const bps_template* bank,
                 int64_t count, const bps_search_params* params, bool own_series,
                 std::unique_ptr<SReq>& out)
{
    if (!bank || !params) return sfail(srv, BPS_ERR_INVALID_ARG, "null pointer");
    if (!series_args_ok(n, tsamp_s, dtype))
        return sfail(srv, BPS_ERR_INVALID_ARG, "n must be a power of two in [2^11, 2^25], tsamp > 0, "
                                               "dtype BPS_F32 or BPS_F16_SCALED");
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
        q->bytes = request_bytes(p, count, *params, dtype, own_series);
    }
    size_t stg = 0;
    const size_t total = q->bytes + (own_series ? 0 : series_bytes(n, dtype, &stg) + stg);
    if (total > srv->budget)
        return sfail(srv, BPS_ERR_OUT_OF_MEMORY, "request needs %zu bytes, server budget %zu",
                     total, srv->budget);
    cudaSetDevice(srv->ctx->device);
    if ((own_series && cudaMallocHost((void**)&q->h_series, 4 * (size_t)n) != cudaSuccess) ||
        cudaMallocHost((void**)&q->h_sum, sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void**)&q->h_count, 2 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost((void**)&q->h_cands, sizeof(Cand) * (size_t)std::min<int64_t>(params->cand_cap, kPinnedCands)) != cudaSuccess ||
        cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming) != cudaSuccess) {
        release_host(*q);
        return sfail(srv, BPS_ERR_OUT_OF_MEMORY, "pinned host staging failed");
    }
    q->grp.resize(srv->cfg.groups_in_flight);
    for (auto& e : q->grp) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    out = std::move(q);
    return BPS_OK;
}

void enqueue(bps_server* srv, std::unique_ptr<SReq>& q, int64_t* ticket)
{
    q->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        q->ticket = srv->next_ticket++;
        *ticket = q->ticket;
        srv->queue.push_back(q->ticket);
        srv->reqs[q->ticket] = std::move(q);
    }
    srv->cv.notify_all();
}

}  // namespace

extern "C" {

int bps_server_submit(bps_server* srv, const float* series, int64_t n, double tsamp_s, int dtype,
                      const bps_template* bank, int64_t count, const bps_search_params* params,
                      int64_t* ticket)
try {
    if (!srv) return BPS_ERR_INVALID_ARG;
    if (!series || !ticket) return sfail(srv, BPS_ERR_INVALID_ARG, "null pointer");
    std::unique_ptr<SReq> q;
    int rc = make_request(srv, n, tsamp_s, dtype, bank, count, params, true, q);
    if (rc) return rc;
    std::memcpy(q->h_series, series, 4 * (size_t)n);
    enqueue(srv, q, ticket);
    return BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

int bps_server_load_series(bps_server* srv, const float* series, int64_t n, double tsamp_s,
                           int dtype, int64_t* series_id)
try {
    if (!srv) return BPS_ERR_INVALID_ARG;
    if (!series || !series_id) return sfail(srv, BPS_ERR_INVALID_ARG, "null pointer");
    if (!series_args_ok(n, tsamp_s, dtype))
        return sfail(srv, BPS_ERR_INVALID_ARG, "n must be a power of two in [2^11, 2^25], tsamp > 0, "
                                               "dtype BPS_F32 or BPS_F16_SCALED");
    std::unique_ptr<SSeries> ser(new SSeries());
    ser->n = n;
    ser->tsamp = tsamp_s;
    ser->dtype = dtype;
    ser->bytes = series_bytes(n, dtype, &ser->stage_bytes);
    if (ser->bytes + ser->stage_bytes > srv->budget)
        return sfail(srv, BPS_ERR_OUT_OF_MEMORY, "series needs %zu bytes, server budget %zu",
                     ser->bytes + ser->stage_bytes, srv->budget);
    cudaSetDevice(srv->ctx->device);
    if (cudaMallocHost((void**)&ser->h_series, 4 * (size_t)n) != cudaSuccess ||
        cudaMallocHost((void**)&ser->h_sum, sizeof(double)) != cudaSuccess ||
        cudaEventCreateWithFlags(&ser->ready, cudaEventDisableTiming) != cudaSuccess) {
        free_series_host(*ser);
        return sfail(srv, BPS_ERR_OUT_OF_MEMORY, "pinned host copy failed");
    }
    std::memcpy(ser->h_series, series, 4 * (size_t)n);
    std::lock_guard<std::mutex> lk(srv->mu);
    ser->id = srv->next_series++;
    *series_id = ser->id;
    srv->series[ser->id] = std::move(ser);
    return BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

int bps_server_submit_series(bps_server* srv, int64_t series_id, const bps_template* bank,
                             int64_t count, const bps_search_params* params, int64_t* ticket)
try {
    if (!srv) return BPS_ERR_INVALID_ARG;
    if (!ticket) return sfail(srv, BPS_ERR_INVALID_ARG, "null pointer");
    SSeries* ser = nullptr;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        auto it = srv->series.find(series_id);
        if (it == srv->series.end())
            return sfail(srv, BPS_ERR_INVALID_ARG, "unknown server series %lld", (long long)series_id);
        ser = it->second.get();
        ser->refs += 1;  // pinned from now on: not evicted or unloaded while named
    }
    std::unique_ptr<SReq> q;
    int rc = make_request(srv, ser->n, ser->tsamp, ser->dtype, bank, count, params, false, q);
    if (rc) {
        std::lock_guard<std::mutex> lk(srv->mu);
        ser->refs -= 1;
        return rc;
    }
    q->ser = ser;
    enqueue(srv, q, ticket);
    return BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

int bps_server_unload_series(bps_server* srv, int64_t series_id)
try {
    if (!srv) return BPS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->series.find(series_id);
    if (it == srv->series.end())
        return sfail(srv, BPS_ERR_INVALID_ARG, "unknown server series %lld", (long long)series_id);
    SSeries& ser = *it->second;
    if (ser.refs > 0)
        return sfail(srv, BPS_ERR_INVALID_ARG, "server series %lld is named by %d unfinished requests",
                     (long long)series_id, ser.refs);
    {
        std::lock_guard<std::recursive_mutex> cl(srv->ctx->mu);
        cudaSetDevice(srv->ctx->device);
        if (ser.resident || ser.staging) evict_series(srv, ser);
        cudaStreamSynchronize(srv->ctx->stream);
    }
    free_series_host(ser);
    srv->series.erase(it);
    return BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

int bps_server_series_info(bps_server* srv, int64_t series_id, int32_t* resident,
                           int64_t* times_staged)
try {
    if (!srv) return BPS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->series.find(series_id);
    if (it == srv->series.end())
        return sfail(srv, BPS_ERR_INVALID_ARG, "unknown server series %lld", (long long)series_id);
    if (resident) *resident = (it->second->resident || it->second->staging) ? 1 : 0;
    if (times_staged) *times_staged = it->second->times_staged;
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
