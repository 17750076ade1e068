// k_detect.cu -- de-reddening, incoherent harmonic sum, threshold and compaction.
//
// De-reddening (App. A, "Fourier de-reddening"): per block of W consecutive bins
// the lower median med_b (the element of rank floor((W-1)/2)) is found by an exact
// radix select on the FP32 bit patterns (P >= 0, so bit order is value order) and
// the block is whitened in place, Pw = P ln2 / med_b (white noise -> Exp(1)).
//
// Harmonic sum (Sec. 2.1, S_L = sum_{n <= 2^L} P_n): with H = nharm_max,
// F_h = Pw[(k h + H/2) div H] for h = 1..H, and (k h' + n/2) div n equals
// (k h' (H/n) + H/2) div H, so S_1 = F_H and S_{2n} = S_n + sum over odd h of
// F_{h H / (2n)}: 16 loads per bin for all five levels.  Threshold (Sec. 2.1)
// and warp-ballot compaction: one atomic per warp and level with hits.
#include <cmath>

#include "bps_internal.cuh"

namespace bps {

namespace {

constexpr float kLn2 = 0.693147180559945309417f;

__global__ void __launch_bounds__(256) k_block_median(float* __restrict__ P, Plan p,
                                                      float* __restrict__ scale)
{
    extern __shared__ uint32_t sv[];
    __shared__ uint32_t hist[256];
    __shared__ uint32_t s_sel, s_rank;
    const int tl = blockIdx.y;
    const int64_t blk = blockIdx.x;
    const int W = 1 << p.logW;
    float* src = P + (int64_t)tl * p.M + (blk << p.logW);
    for (int i = threadIdx.x; i < W; i += blockDim.x) sv[i] = __float_as_uint(src[i]);
    uint32_t prefix = 0, pmask = 0, rank = (uint32_t)(W - 1) / 2;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < W; i += blockDim.x) {
            const uint32_t u = sv[i];
            if ((u & pmask) == prefix) atomicAdd(&hist[(u >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            uint32_t c[8], tot = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                c[q] = hist[8 * lane + q];
                tot += c[q];
            }
            uint32_t inc = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += v;
            }
            const uint32_t exc = inc - tot;
            if (exc <= rank && rank < inc) {
                uint32_t acc = exc;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (rank < acc + c[q]) {
                        s_sel = (uint32_t)(8 * lane + q);
                        s_rank = rank - acc;
                        break;
                    }
                    acc += c[q];
                }
            }
        }
        __syncthreads();
        prefix |= s_sel << shift;
        pmask |= 255u << shift;
        rank = s_rank;
        __syncthreads();
    }
    const float med = __uint_as_float(prefix);
    const float sc = (med > 0.f) ? kLn2 / med : 0.f;
    for (int i = threadIdx.x; i < W; i += blockDim.x) src[i] = __uint_as_float(sv[i]) * sc;
    if (threadIdx.x == 0) scale[(int64_t)tl * (p.M >> p.logW) + blk] = sc;
}

__global__ void k_whitened(const float* __restrict__ Pw, Plan p, float* __restrict__ out)
{
    const int tl = blockIdx.y;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= p.M) return;
    out[(int64_t)tl * p.M + k] = Pw[(int64_t)tl * p.M + k];
}

// One warp per block of W = 32*VPL bins, values in registers; exact radix select of
// the element of rank floor((W-1)/2) over four digits of the FP32 bit pattern
// (P >= 0: sign bit 0; digits = exponent [30:23], mantissa [22:15], [14:7], [6:0])
// with a per-warp shared histogram and a warp prefix scan, no block barrier.  The
// block is then whitened in place: Pw = P * ln2 / med (0 when med = 0).
template <int VPL>
__global__ void __launch_bounds__(256) k_median_warp(float* __restrict__ P, Plan p,
                                                     float* __restrict__ scale)
{
    __shared__ uint32_t hist[8][288];  // bin b at b + b/8: conflict-free scan reads
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tl = blockIdx.y;
    const int64_t nblk = p.M >> p.logW;
    const int64_t blk = (int64_t)blockIdx.x * 8 + warp;
    if (blk >= nblk) return;
    float* src = P + (int64_t)tl * p.M + (blk << p.logW);
    uint32_t u[VPL];
#pragma unroll
    for (int i = 0; i < VPL; ++i) u[i] = __float_as_uint(src[lane + 32 * i]);
    uint32_t prefix = 0, pmask = 0, rank = (uint32_t)(32 * VPL - 1) / 2;
    uint32_t* h = hist[warp];
#pragma unroll
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = pass == 0 ? 23 : pass == 1 ? 15 : pass == 2 ? 7 : 0;
        const uint32_t dm = pass == 3 ? 127u : 255u;
#pragma unroll
        for (int q = 0; q < 9; ++q) h[lane + 32 * q] = 0;
        __syncwarp();
#pragma unroll
        for (int i = 0; i < VPL; ++i) {
            if ((u[i] & pmask) == prefix) {
                const uint32_t dg = (u[i] >> shift) & dm;
                atomicAdd(&h[dg + (dg >> 3)], 1u);
            }
        }
        __syncwarp();
        uint32_t c[8], tot = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            c[q] = h[9 * lane + q];
            tot += c[q];
        }
        uint32_t inc = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        const uint32_t exc = inc - tot;
        const bool own = (exc <= rank) && (rank < inc);
        uint32_t sel = 0, nrank = 0;
        if (own) {
            uint32_t acc = exc;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (rank >= acc && rank < acc + c[q]) {
                    sel = (uint32_t)(8 * lane + q);
                    nrank = rank - acc;
                }
                acc += c[q];
            }
        }
        const int owner = __ffs(__ballot_sync(0xffffffffu, own)) - 1;
        sel = __shfl_sync(0xffffffffu, sel, owner);
        nrank = __shfl_sync(0xffffffffu, nrank, owner);
        prefix |= sel << shift;
        pmask |= dm << shift;
        rank = nrank;
        __syncwarp();
    }
    const float med = __uint_as_float(prefix);
    const float sc = (med > 0.f) ? kLn2 / med : 0.f;
#pragma unroll
    for (int i = 0; i < VPL; ++i) src[lane + 32 * i] = __uint_as_float(u[i]) * sc;
    if (lane == 0) scale[(int64_t)tl * nblk + blk] = sc;
}

// Incoherent harmonic sum of the whitened spectrum.  With H = nharm_max the h-th
// term of bin k is Pw[(k h + H/2) div H].  A warp covers 32 QN consecutive bins as
// k = k_w + lane + 32 q (q < QN), so for each h the QN terms sit at
// ((k_w + lane) h + H/2) div H + 32 q h / H: one index per h plus compile-time
// offsets, QN H independent coalesced loads per thread.
template <int NH, int QN>
__global__ void __launch_bounds__(256) k_harmsum_direct(const float* __restrict__ Pw, Plan p,
                                                        int64_t tidx0, Thr thr,
                                                        Cand* __restrict__ cands, int64_t cap,
                                                        unsigned long long* __restrict__ count,
                                                        float* __restrict__ s_out)
{
    constexpr int LOGNH = (NH == 1) ? 0 : (NH == 2) ? 1 : (NH == 4) ? 2 : (NH == 8) ? 3 : 4;
    constexpr int NLEV = LOGNH + 1;
    const int tl = blockIdx.y;
    const unsigned lane = threadIdx.x & 31u;
    const int kb = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * (32 * QN) + (int)lane;
    const float* Pt = Pw + (int64_t)tl * p.M;
    float S[QN][NLEV];
    {
        float F[QN][NH];
#pragma unroll
        for (int h = 1; h <= NH; ++h) {
            const float* ph = Pt + ((kb * h + (NH >> 1)) >> LOGNH);  // kb*h < 2^28
#pragma unroll
            for (int q = 0; q < QN; ++q) F[q][h - 1] = __ldg(ph + ((32 * q * h) >> LOGNH));
        }
#pragma unroll
        for (int q = 0; q < QN; ++q) {
            float s = F[q][NH - 1];
            S[q][0] = s;
#pragma unroll
            for (int L = 1; L < NLEV; ++L) {
                const int n = 1 << L;
                const int step = NH / n;
#pragma unroll
                for (int h = 1; h <= n; h += 2) s += F[q][h * step - 1];
                S[q][L] = s;
            }
        }
    }
    if (s_out) {
#pragma unroll
        for (int q = 0; q < QN; ++q) {
            const int k = kb + 32 * q;
#pragma unroll
            for (int L = 0; L < NLEV; ++L)
                s_out[((int64_t)tl * NLEV + L) * p.M + k] = (k >= 1) ? S[q][L] : 0.f;
        }
    }
    // threshold: one warp vote for all levels and bins first (detections are rare)
    bool any = false;
#pragma unroll
    for (int q = 0; q < QN; ++q)
#pragma unroll
        for (int L = 0; L < NLEV; ++L) any |= (S[q][L] >= thr.v[L]) && (kb + 32 * q >= 1);
    if (!__any_sync(0xffffffffu, any)) return;
#pragma unroll
    for (int q = 0; q < QN; ++q) {
        const int k = kb + 32 * q;
        const bool valid = k >= 1;
#pragma unroll
        for (int L = 0; L < NLEV; ++L) {
            const bool hit = valid && (S[q][L] >= thr.v[L]);
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (m) {
                const int leader = __ffs(m) - 1;
                unsigned long long b0 = 0;
                if ((int)lane == leader) b0 = atomicAdd(count, (unsigned long long)__popc(m));
                b0 = __shfl_sync(0xffffffffu, b0, leader);
                if (hit) {
                    const unsigned long long pos = b0 + __popc(m & ((1u << lane) - 1u));
                    if ((int64_t)pos < cap) {
                        Cand c;
                        c.tidx = (uint32_t)(tidx0 + tl);
                        c.nharm = (uint16_t)(1 << L);
                        c.flags = 0;
                        c.bin = (uint32_t)k;
                        c.power = S[q][L];
                        cands[pos] = c;
                    }
                }
            }
        }
    }
}

// ---- TMA bulk copies into shared memory, completed on an mbarrier (inline PTX) ----
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// 1D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes,
                                            uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase 0 of the barrier: false (and error flag set) after the limit.
constexpr int kWaitLimit = 1 << 22;

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned long long* status)
{
    for (int it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(bar, 0)) return true;
    if (status) atomicOr(status, 1ull);  // BPS_ERR_TIMEOUT reported by the host
    // the copies may still be in flight: give them a second bounded wait before exiting
    for (int it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(bar, 0)) break;
    return false;
}

// Incoherent harmonic sum of the whitened spectrum over a tile of 1024 bins.  With
// H = nharm_max the h-th term of bin k is Pw[(k h + H/2) div H]; over the tile these
// terms form one contiguous segment per h.  One thread issues 16-byte-aligned TMA bulk
// copies of the H segments into shared memory (about 8.6 x the tile), warp 0 waits on
// the mbarrier (bounded; on expiry the status word is flagged and the tile skipped),
// then each thread sums 4 bins k = k0 + tid + 256 q from shared memory.
constexpr int kHsTile = 1024;

template <int NH>
__global__ void __launch_bounds__(256) k_harmsum_tma(const float* __restrict__ Pw, Plan p,
                                                     int64_t tidx0, Thr thr,
                                                     Cand* __restrict__ cands, int64_t cap,
                                                     unsigned long long* __restrict__ count,
                                                     float* __restrict__ s_out)
{
    constexpr int LOGNH = (NH == 1) ? 0 : (NH == 2) ? 1 : (NH == 4) ? 2 : (NH == 8) ? 3 : 4;
    constexpr int NLEV = LOGNH + 1;
    constexpr int QN = kHsTile / 256;
    constexpr int SEG = kHsTile * (NH + 1) / 2 + 8 * NH;
    __shared__ __align__(128) float seg[SEG];
    __shared__ __align__(8) uint64_t bar;
    const int tl = blockIdx.y;
    const int k0 = blockIdx.x * kHsTile;
    const float* Pt = Pw + (int64_t)tl * p.M;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t total = 0;
#pragma unroll
        for (int h = 1; h <= NH; ++h) {
            const int a = ((k0 * h + (NH >> 1)) >> LOGNH) & ~3;
            const int b = ((((k0 + kHsTile - 1) * h + (NH >> 1)) >> LOGNH) + 4) & ~3;
            total += (uint32_t)(b - a) * 4u;
        }
        mbar_expect_tx(&bar, total);
        int off = 0;
#pragma unroll
        for (int h = 1; h <= NH; ++h) {
            const int a = ((k0 * h + (NH >> 1)) >> LOGNH) & ~3;
            const int b = ((((k0 + kHsTile - 1) * h + (NH >> 1)) >> LOGNH) + 4) & ~3;
            tma_load_1d(seg + off, Pt + a, (uint32_t)(b - a) * 4u, &bar);
            off += b - a;
        }
    }
    // per-thread base index of each segment (computed while the copies fly)
    int base[NH];
    {
        int off = 0;
#pragma unroll
        for (int h = 1; h <= NH; ++h) {
            const int a = ((k0 * h + (NH >> 1)) >> LOGNH) & ~3;
            const int b = ((((k0 + kHsTile - 1) * h + (NH >> 1)) >> LOGNH) + 4) & ~3;
            base[h - 1] = off + ((((k0 + (int)threadIdx.x) * h + (NH >> 1)) >> LOGNH) - a);
            off += b - a;
        }
    }
    // one warp waits on the barrier (the others sleep in __syncthreads, issuing nothing);
    // its acquire plus the CTA barrier make the copied segments visible to all threads
    __shared__ int s_ok;
    if (threadIdx.x < 32) {
        const bool ok = mbar_wait_bounded(&bar, threadIdx.x == 0 ? count + 1 : nullptr);
        if (threadIdx.x == 0) s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return;
    const unsigned lane = threadIdx.x & 31u;
    float S[QN][NLEV];
#pragma unroll
    for (int q = 0; q < QN; ++q) {
        float F[NH];
#pragma unroll
        for (int h = 1; h <= NH; ++h) F[h - 1] = seg[base[h - 1] + ((256 * q * h) >> LOGNH)];
        float s = F[NH - 1];
        S[q][0] = s;
#pragma unroll
        for (int L = 1; L < NLEV; ++L) {
            const int n = 1 << L;
            const int step = NH / n;
#pragma unroll
            for (int h = 1; h <= n; h += 2) s += F[h * step - 1];
            S[q][L] = s;
        }
    }
    if (s_out) {
#pragma unroll
        for (int q = 0; q < QN; ++q) {
            const int k = k0 + (int)threadIdx.x + 256 * q;
#pragma unroll
            for (int L = 0; L < NLEV; ++L)
                s_out[((int64_t)tl * NLEV + L) * p.M + k] = (k >= 1) ? S[q][L] : 0.f;
        }
    }
    bool any = false;
#pragma unroll
    for (int q = 0; q < QN; ++q)
#pragma unroll
        for (int L = 0; L < NLEV; ++L)
            any |= (S[q][L] >= thr.v[L]) && (k0 + (int)threadIdx.x + 256 * q >= 1);
    if (!__any_sync(0xffffffffu, any)) return;
#pragma unroll
    for (int q = 0; q < QN; ++q) {
        const int k = k0 + (int)threadIdx.x + 256 * q;
        const bool valid = k >= 1;
#pragma unroll
        for (int L = 0; L < NLEV; ++L) {
            const bool hit = valid && (S[q][L] >= thr.v[L]);
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (m) {
                const int leader = __ffs(m) - 1;
                unsigned long long b0 = 0;
                if ((int)lane == leader) b0 = atomicAdd(count, (unsigned long long)__popc(m));
                b0 = __shfl_sync(0xffffffffu, b0, leader);
                if (hit) {
                    const unsigned long long pos = b0 + __popc(m & ((1u << lane) - 1u));
                    if ((int64_t)pos < cap) {
                        Cand c;
                        c.tidx = (uint32_t)(tidx0 + tl);
                        c.nharm = (uint16_t)(1 << L);
                        c.flags = 0;
                        c.bin = (uint32_t)k;
                        c.power = S[q][L];
                        cands[pos] = c;
                    }
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_block_median(float* P, int nt, const Plan& p, float* scale,
                                cudaStream_t s)
{
    const int64_t nblk = p.M >> p.logW;
    dim3 wgrid((unsigned)((nblk + 7) / 8), (unsigned)nt);
    switch (p.logW) {
        case 5: k_median_warp<1><<<wgrid, 256, 0, s>>>(P, p, scale); break;
        case 6: k_median_warp<2><<<wgrid, 256, 0, s>>>(P, p, scale); break;
        case 7: k_median_warp<4><<<wgrid, 256, 0, s>>>(P, p, scale); break;
        case 8: k_median_warp<8><<<wgrid, 256, 0, s>>>(P, p, scale); break;
        case 9: k_median_warp<16><<<wgrid, 256, 0, s>>>(P, p, scale); break;
        case 10: k_median_warp<32><<<wgrid, 256, 0, s>>>(P, p, scale); break;
        default: {
            dim3 grid((unsigned)nblk, (unsigned)nt);
            k_block_median<<<grid, 256, (size_t)sizeof(uint32_t) << p.logW, s>>>(P, p, scale);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_whitened(const float* P, const float* scale, int nt, const Plan& p,
                            float* out, cudaStream_t s)
{
    dim3 grid((unsigned)((p.M + 255) / 256), (unsigned)nt);
    (void)scale;
    k_whitened<<<grid, 256, 0, s>>>(P, p, out);
    return cudaGetLastError();
}

cudaError_t launch_harmsum(const float* P, const float* scale, int nt, int64_t tidx0,
                           const Plan& p, const Thr& thr, Cand* cands, int64_t cap,
                           unsigned long long* count, float* s_out, cudaStream_t s)
{
    (void)scale;
    dim3 grid((unsigned)(p.M / kHsTile), (unsigned)nt);
    switch (p.nharm) {
        case 1: k_harmsum_tma<1><<<grid, 256, 0, s>>>(P, p, tidx0, thr, cands, cap, count, s_out); break;
        case 2: k_harmsum_tma<2><<<grid, 256, 0, s>>>(P, p, tidx0, thr, cands, cap, count, s_out); break;
        case 4: k_harmsum_tma<4><<<grid, 256, 0, s>>>(P, p, tidx0, thr, cands, cap, count, s_out); break;
        case 8: k_harmsum_tma<8><<<grid, 256, 0, s>>>(P, p, tidx0, thr, cands, cap, count, s_out); break;
        case 16: k_harmsum_tma<16><<<grid, 256, 0, s>>>(P, p, tidx0, thr, cands, cap, count, s_out); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace bps
