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

template <int NH>
__global__ void __launch_bounds__(256) k_harmsum(const float* __restrict__ P,
                                                 const float* __restrict__ scale, Plan p,
                                                 int64_t tidx0, Thr thr, Cand* __restrict__ cands,
                                                 int64_t cap, unsigned long long* __restrict__ count,
                                                 float* __restrict__ s_out)
{
    constexpr int LOGNH = (NH == 1) ? 0 : (NH == 2) ? 1 : (NH == 4) ? 2 : (NH == 8) ? 3 : 4;
    constexpr int NLEV = LOGNH + 1;
    const int tl = blockIdx.y;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const float* Pt = P + (int64_t)tl * p.M;
    const float* sc = scale + (int64_t)tl * (p.M >> p.logW);
    const bool valid = (k >= 1) && (k < p.M);
    float F[NH];
#pragma unroll
    for (int h = 1; h <= NH; ++h) {
        float v = 0.f;
        if (valid) {
            const int64_t b = (k * h + (NH >> 1)) >> LOGNH;
            v = __ldg(Pt + b) * __ldg(sc + (b >> p.logW));
        }
        F[h - 1] = v;
    }
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
    const unsigned lane = threadIdx.x & 31u;
#pragma unroll
    for (int L = 0; L < NLEV; ++L) {
        const bool hit = valid && (S[L] >= thr.v[L]);
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (m) {
            const int leader = __ffs(m) - 1;
            unsigned long long base = 0;
            if ((int)lane == leader) base = atomicAdd(count, (unsigned long long)__popc(m));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (hit) {
                const unsigned long long pos = base + __popc(m & ((1u << lane) - 1u));
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

}  // namespace

cudaError_t launch_block_median(const float* P, int nt, const Plan& p, float* scale,
                                cudaStream_t s)
{
    dim3 grid((unsigned)(p.M >> p.logW), (unsigned)nt);
    k_block_median<<<grid, 256, (size_t)sizeof(uint32_t) << p.logW, s>>>(P, p, scale);
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
    dim3 grid((unsigned)((p.M + 255) / 256), (unsigned)nt);
    switch (p.nharm) {
        case 1: k_harmsum<1><<<grid, 256, 0, s>>>(P, scale, p, tidx0, thr, cands, cap, count, s_out); break;
        case 2: k_harmsum<2><<<grid, 256, 0, s>>>(P, scale, p, tidx0, thr, cands, cap, count, s_out); break;
        case 4: k_harmsum<4><<<grid, 256, 0, s>>>(P, scale, p, tidx0, thr, cands, cap, count, s_out); break;
        case 8: k_harmsum<8><<<grid, 256, 0, s>>>(P, scale, p, tidx0, thr, cands, cap, count, s_out); break;
        case 16: k_harmsum<16><<<grid, 256, 0, s>>>(P, scale, p, tidx0, thr, cands, cap, count, s_out); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace bps
