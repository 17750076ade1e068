// bps_noalloc.cu -- allocation-free variant of the whitened-spectrum path.
//
// Some callers cannot allocate device memory while they run: real-time
// telescope back ends that reserve all of the GPU's memory at start-up and
// forbid allocation afterwards (a cudaMalloc can stall the device or fail once
// the memory is fragmented), and host frameworks whose own pool allocator owns
// every byte of device memory.  bps_whitened_spectrum_noalloc serves them: it
// runs the same kernels as bps_whitened_spectrum for one template, but its
// scratch (anchors, packed FFT intermediate, power spectrum, block scales,
// twiddle table) lives in one file-scope device array of fixed size, and it
// calls no cudaMalloc, cudaFree or allocating library routine.
//
// Limits and behaviour:
//   * series length n <= 2^20 samples (the scratch array is 8 MiB; every GPU
//     that loads the library keeps it until the process exits);
//   * the array is shared by all calls and keeps the last call's contents;
//     each call overwrites every byte it reads, so nothing needs clearing;
//   * calls whose work overlaps on the GPU (different streams, or different
//     host threads) race on the array: serialise them;
//   * every call made while its stream is not being captured looks up the array's
//     device address with cudaGetSymbolAddress (with the call's device current; the
//     lookup allocates nothing), so a context torn down and re-created in between
//     (cudaDeviceReset) is followed; a call made during a stream capture uses the
//     address of the last uncaptured call on that device, so make one call before
//     any capture;
//   * the anchor block is chosen from this one template's orbit (bps_whitened_spectrum
//     chooses it from the whole bank), so results agree with bps_whitened_spectrum
//     within the power tolerance of the parity tests, not bit for bit: near-half-
//     integer offsets can round the other way with another anchor block.
#include <cmath>
#include <mutex>

#include "../../include/bps.h"
#include "bps_internal.cuh"
#include "dev_template.h"

namespace bps {

namespace {

constexpr size_t kScratchBytes = 8u << 20;
constexpr int kMaxLogN = 20;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_dev[kMaxDevices] = {};

// Device address of g_scratch on the current device (host code may not use the
// symbol itself: on the host it names a stand-in, not device memory).  Looked up
// afresh unless the stream is being captured (then the last address looked up on
// this device is used; none yet is an error).
int scratch_address(cudaStream_t st, unsigned char** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BPS_ERR_CUDA;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return BPS_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return BPS_ERR_CUDA;
        g_scratch_dev[dev] = (unsigned char*)p;
    }
    if (!g_scratch_dev[dev]) return BPS_ERR_CUDA;
    *out = g_scratch_dev[dev];
    return BPS_OK;
}

__global__ void k_store_template(DevTemplate t, DevTemplate* dst) { *dst = t; }

// log2 of v when v is a power of two in [1, 2^62], else -1 (no shift past bit 62)
int ilog2_exact(int64_t v)
{
    if (v < 1 || v > (1ll << 62)) return -1;
    int l = 0;
    while (l < 62 && (1ll << l) < v) ++l;
    return (1ll << l) == v ? l : -1;
}

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

}  // namespace bps

using namespace bps;

extern "C" int bps_whitened_spectrum_noalloc(const float* d_series, int64_t n, double tsamp_s,
                                             double fill, const bps_template* tmpl,
                                             int32_t whiten_block, float* d_pw_out,
                                             void* cuda_stream)
try {
    if (!d_series || !tmpl || !d_pw_out) return BPS_ERR_INVALID_ARG;
    if (n > (1ll << kMaxLogN) && ilog2_exact(n) > 0) return BPS_ERR_UNSUPPORTED;
    const int logn = ilog2_exact(n);
    if (logn < 11) return BPS_ERR_INVALID_ARG;
    if (logn > kMaxLogN) return BPS_ERR_UNSUPPORTED;  // beyond the fixed scratch array
    if (!(tsamp_s > 0.0) || !std::isfinite(tsamp_s) || !std::isfinite(fill))
        return BPS_ERR_INVALID_ARG;
    const bps_template& t = *tmpl;
    if (!(t.porb_s > 0.0) || !std::isfinite(t.porb_s) || !(t.tau_lts >= 0.0) ||
        !std::isfinite(t.tau_lts) || !std::isfinite(t.phi_rad) || !std::isfinite(t.omega_rad) ||
        !(t.ecc >= 0.0 && t.ecc < 1.0))
        return BPS_ERR_INVALID_ARG;
    const int logW = ilog2_exact(whiten_block);
    if (logW < 5 || logW > 13 || whiten_block > n / 2) return BPS_ERR_INVALID_ARG;

    // geometry and anchor block, by the same rules as bps_search
    Plan p;
    p.n = n;
    p.logn = logn;
    p.M = n / 2;
    p.logM = logn - 1;
    plan_geometry(p);
    p.logW = logW;
    p.nharm = 1;
    p.lognh = 0;
    p.nlev = 1;
    p.tsamp = tsamp_s;
    p.inv_tsamp = 1.0 / tsamp_s;
    const double K = t.tau_lts / tsamp_s;
    const double g = (2.0 * M_PI / t.porb_s) * tsamp_s / (1.0 - t.ecc);
    const int logB = plan_anchor_block(K * g, K * g * g, K * g * g * g * g, logn);
    if (logB < 6) return BPS_ERR_UNSUPPORTED;
    p.logB = logB;
    p.nanchor = n >> logB;

    // carve the scratch array
    const size_t a_tw = up256(kTwiddleN * sizeof(float2));
    const size_t a_tm = up256(sizeof(DevTemplate));
    const size_t a_an = up256(sizeof(Anchor) * (size_t)p.nanchor);
    const size_t a_y = up256(sizeof(float2) * (size_t)(p.M + 1));
    const size_t a_p = up256(sizeof(float) * (size_t)p.M);
    const size_t a_sc = up256(sizeof(float) * (size_t)(p.M >> p.logW));
    if (a_tw + a_tm + a_an + a_y + a_p + a_sc > kScratchBytes) return BPS_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned char* base = nullptr;
    int rc = scratch_address(st, &base);
    if (rc) return rc;
    float2* tw = (float2*)base;
    DevTemplate* dt = (DevTemplate*)(base + a_tw);
    Anchor* anc = (Anchor*)(base + a_tw + a_tm);
    float2* Y = (float2*)(base + a_tw + a_tm + a_an);
    float* P = (float*)(base + a_tw + a_tm + a_an + a_y);
    float* scale = (float*)(base + a_tw + a_tm + a_an + a_y + a_p);

    const DevTemplate tv = rt::dev_template(t);
    SeriesView v;
    v.f32 = d_series;
    v.f16 = nullptr;
    v.scale = nullptr;
    v.fill = (float)fill;
    v.fillp = nullptr;
    v.uscalep = nullptr;
    v.uscale = 0.f;
    if (launch_twiddle_init(tw, st) != cudaSuccess) return BPS_ERR_CUDA;
    k_store_template<<<1, 1, 0, st>>>(tv, dt);
    if (cudaGetLastError() != cudaSuccess) return BPS_ERR_CUDA;
    if (launch_anchors(dt, 0, 1, p, anc, st) != cudaSuccess) return BPS_ERR_CUDA;
    if (launch_pass1(v, anc, 1, p, tw, Y, nullptr, st) != cudaSuccess) return BPS_ERR_CUDA;
    if (launch_pass2(Y, 1, p, tw, P, nullptr, st) != cudaSuccess) return BPS_ERR_CUDA;
    if (launch_block_median(P, 1, p, scale, st) != cudaSuccess) return BPS_ERR_CUDA;
    if (launch_whitened(P, scale, 1, p, d_pw_out, st) != cudaSuccess) return BPS_ERR_CUDA;
    return BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}
