// k_detect.cu -- de-reddening, incoherent harmonic sum, threshold and compaction.
//
// De-reddening (App. A, "Fourier de-reddening"): per block of W consecutive bins
// the lower median med_b (the element of rank floor((W-1)/2)) is found by an exact
// 4 x 8-bit radix select on the FP32 bit patterns (P >= 0, so bit order is value
// order); the block scale ln2 / med_b makes white noise Exp(1).
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

__global__ void __launch_bounds__(256) k_block_median(const float* __restrict__ P, Plan p,
                                                      float* __restrict__ scale)
{
    extern __shared__ uint32_t sv[];
    __shared__ uint32_t hist[256];
    __shared__ uint32_t s_sel, s_rank;
    const int tl = blockIdx.y;
    const int64_t blk = blockIdx.x;
    const int W = 1 << p.logW;
    const float* src = P + (int64_t)tl * p.M + (blk << p.logW);
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
    if (threadIdx.x == 0) {
        const float med = __uint_as_float(prefix);
        scale[(int64_t)tl * (p.M >> p.logW) + blk] = (med > 0.f) ? kLn2 / med : 0.f;
    }
}

__global__ void k_whitened(const float* __restrict__ P, const float* __restrict__ scale, Plan p,
                           float* __restrict__ out)
{
    const int tl = blockIdx.y;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= p.M) return;
    out[(int64_t)tl * p.M + k] =
        P[(int64_t)tl * p.M + k] * scale[(int64_t)tl * (p.M >> p.logW) + (k >> p.logW)];
}

// One warp per block of W = 32*VPL bins, values in registers; exact radix select of
// the element of rank floor((W-1)/2) over 4 x 8-bit digits with a per-warp
// histogram (equal digits of a warp aggregated by __match_any_sync, one shared
// atomic per distinct digit) and a warp prefix scan.  No block-level barrier.
template <int VPL>
__global__ void __launch_bounds__(256) k_median_warp(const float* __restrict__ P, Plan p,
                                                     float* __restrict__ scale)
{
    __shared__ uint32_t hist[8][256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tl = blockIdx.y;
    const int64_t nblk = p.M >> p.logW;
    const int64_t blk = (int64_t)blockIdx.x * 8 + warp;
    if (blk >= nblk) return;
    const float* src = P + (int64_t)tl * p.M + (blk << p.logW);
    uint32_t u[VPL];
#pragma unroll
    for (int i = 0; i < VPL; ++i) u[i] = __float_as_uint(__ldg(src + lane + 32 * i));
    uint32_t prefix = 0, pmask = 0, rank = (uint32_t)(32 * VPL - 1) / 2;
    uint32_t* h = hist[warp];
#pragma unroll
    for (int shift = 24; shift >= 0; shift -= 8) {
#pragma unroll
        for (int q = 0; q < 8; ++q) h[lane + 32 * q] = 0;
        __syncwarp();
#pragma unroll
        for (int i = 0; i < VPL; ++i) {
            const bool in = (u[i] & pmask) == prefix;
            const uint32_t key = in ? ((u[i] >> shift) & 255u) : 256u;
            const unsigned grp = __match_any_sync(0xffffffffu, key);
            if (in && lane == __ffs(grp) - 1) atomicAdd(&h[key], (uint32_t)__popc(grp));
        }
        __syncwarp();
        uint32_t c[8], tot = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            c[q] = h[8 * lane + q];
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
        pmask |= 255u << shift;
        rank = nrank;
        __syncwarp();
    }
    if (lane == 0) {
        const float med = __uint_as_float(prefix);
        scale[(int64_t)tl * nblk + blk] = (med > 0.f) ? kLn2 / med : 0.f;
    }
}

// Harmonic sum over a tile of 1024 bins (256 threads x 4 bins, k = k0 + tid + 256 q).
// For each h = 1..H the whitened bins (k h + H/2) div H of the tile form one
// contiguous segment; all H segments are staged in shared memory (about 8.5 x
// the tile) with coalesced loads, then each bin reads its H terms from there.
constexpr int kHsTile = 1024;

template <int NH>
__global__ void __launch_bounds__(256) k_harmsum_tiled(const float* __restrict__ P,
                                                       const float* __restrict__ scale, Plan p,
                                                       int64_t tidx0, Thr thr,
                                                       Cand* __restrict__ cands, int64_t cap,
                                                       unsigned long long* __restrict__ count,
                                                       float* __restrict__ s_out)
{
    constexpr int LOGNH = (NH == 1) ? 0 : (NH == 2) ? 1 : (NH == 4) ? 2 : (NH == 8) ? 3 : 4;
    constexpr int NLEV = LOGNH + 1;
    constexpr int SEG = kHsTile * (NH + 1) / 2 + 2 * NH;
    __shared__ float seg[SEG];
    const int tl = blockIdx.y;
    const int64_t k0 = (int64_t)blockIdx.x * kHsTile;
    const float* Pt = P + (int64_t)tl * p.M;
    const float* sc = scale + (int64_t)tl * (p.M >> p.logW);
    int base[NH];
    {
        int off = 0;
#pragma unroll
        for (int h = 1; h <= NH; ++h) {
            const int64_t s0 = (k0 * h + (NH >> 1)) >> LOGNH;
            const int64_t s1 = ((k0 + kHsTile - 1) * h + (NH >> 1)) >> LOGNH;
            const int len = (int)(s1 - s0 + 1);
            for (int i = threadIdx.x; i < len; i += blockDim.x) {
                const int64_t b = s0 + i;
                seg[off + i] = __ldg(Pt + b) * __ldg(sc + (b >> p.logW));
            }
            const int64_t kb = k0 + threadIdx.x;
            base[h - 1] = off + (int)(((kb * h + (NH >> 1)) >> LOGNH) - s0);
            off += len;
        }
    }
    __syncthreads();
    const unsigned lane = threadIdx.x & 31u;
#pragma unroll
    for (int q = 0; q < kHsTile / 256; ++q) {
        const int64_t k = k0 + threadIdx.x + 256 * q;
        const bool valid = (k >= 1) && (k < p.M);
        float F[NH];
#pragma unroll
        for (int h = 1; h <= NH; ++h) F[h - 1] = seg[base[h - 1] + ((256 * q * h) >> LOGNH)];
        float S[NLEV];
        float s = F[NH - 1];
        S[0] = s;
#pragma unroll
        for (int L = 1; L < NLEV; ++L) {
            const int n = 1 << L;
            const int step = NH / n;
#pragma unroll
            for (int h = 1; h <= n; h += 2) s += F[h * step - 1];
            S[L] = s;
        }
        if (s_out && k < p.M) {
#pragma unroll
            for (int L = 0; L < NLEV; ++L)
                s_out[((int64_t)tl * NLEV + L) * p.M + k] = valid ? S[L] : 0.f;
        }
#pragma unroll
        for (int L = 0; L < NLEV; ++L) {
            const bool hit = valid && (S[L] >= thr.v[L]);
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
                        c.power = S[L];
                        cands[pos] = c;
                    }
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_block_median(const float* P, int nt, const Plan& p, float* scale,
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
    k_whitened<<<grid, 256, 0, s>>>(P, scale, p, out);
    return cudaGetLastError();
}

cudaError_t launch_harmsum(const float* P, const float* scale, int nt, int64_t tidx0,
                           const Plan& p, const Thr& thr, Cand* cands, int64_t cap,
                           unsigned long long* count, float* s_out, cudaStream_t s)
{
    dim3 grid((unsigned)(p.M / kHsTile), (unsigned)nt);
    switch (p.nharm) {
        case 1: k_harmsum_tiled<1><<<grid, 256, 0, s>>>(P, scale, p, tidx0, thr, cands, cap, count, s_out); break;
        case 2: k_harmsum_tiled<2><<<grid, 256, 0, s>>>(P, scale, p, tidx0, thr, cands, cap, count, s_out); break;
        case 4: k_harmsum_tiled<4><<<grid, 256, 0, s>>>(P, scale, p, tidx0, thr, cands, cap, count, s_out); break;
        case 8: k_harmsum_tiled<8><<<grid, 256, 0, s>>>(P, scale, p, tidx0, thr, cands, cap, count, s_out); break;
        case 16: k_harmsum_tiled<16><<<grid, 256, 0, s>>>(P, scale, p, tidx0, thr, cands, cap, count, s_out); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace bps
