// k_fft.cu -- the real FFT of the resampled series as a two-pass four-step
// shared-memory Stockham FFT (Sec. 2.4: one FFT per orbital template gives the
// uniform f0 grid; App. A: "return S' to calculate FFT").
//
// The N real samples are packed as M = N/2 complex points z_j = x'_{2j} + i x'_{2j+1}
// and M = R * C is split four-step:  j = j1*C + j2,  k = k1 + R*k2,
//   pass 1 (gather fused):  Y[k1][j2] = W_M^{j2 k1} * sum_{j1} z[j1 C + j2] W_R^{j1 k1}
//   pass 2 (split + power fused):  Z[k1 + R k2] = sum_{j2} Y[k1][j2] W_C^{j2 k2}
// then X_k = E_k + W_N^k O_k with E/O the even/odd-sample spectra recovered from
// Z_k and Z_{M-k}; a pass-2 CTA owns the row pair (k1, R-k1) so both are local.
// Each pass runs radix-4 (+ radix-2) Stockham stages in shared memory, one
// sub-transform element set per thread held in registers across the barrier.
#include <cmath>

#include "bps_internal.cuh"
#include "index_map.cuh"

namespace bps {

namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <int RADIX>
__device__ __forceinline__ void dft(float2* v);

template <>
__device__ __forceinline__ void dft<2>(float2* v)
{
    const float2 a = v[0], b = v[1];
    v[0] = make_float2(a.x + b.x, a.y + b.y);
    v[1] = make_float2(a.x - b.x, a.y - b.y);
}

template <>
__device__ __forceinline__ void dft<4>(float2* v)
{
    const float2 a0 = make_float2(v[0].x + v[2].x, v[0].y + v[2].y);
    const float2 a1 = make_float2(v[0].x - v[2].x, v[0].y - v[2].y);
    const float2 a2 = make_float2(v[1].x + v[3].x, v[1].y + v[3].y);
    const float2 a3 = make_float2(v[1].x - v[3].x, v[1].y - v[3].y);
    v[0] = make_float2(a0.x + a2.x, a0.y + a2.y);
    v[2] = make_float2(a0.x - a2.x, a0.y - a2.y);
    v[1] = make_float2(a1.x + a3.y, a1.y - a3.x);  // a1 - i a3
    v[3] = make_float2(a1.x - a3.y, a1.y + a3.x);  // a1 + i a3
}

// One Stockham stage over nlines lines of length L = 2^logL held in shared memory
// (element (line, pos) at buf[line*ls + pos*es]).  Ns = 2^logNs is the length of
// the sub-transforms already done.  blockDim.x * EPT == nlines * L.
template <int LOGRADIX, int EPT, bool LINE_FAST>
__device__ __forceinline__ void fft_stage(float2* buf, int logL, int logNs, int lognl,
                                          int ls, int es, const float2* __restrict__ tw)
{
    constexpr int RADIX = 1 << LOGRADIX;
    constexpr int BPT = EPT / RADIX;
    const int logQ = logL - LOGRADIX;  // log2(L / RADIX)
    const int Q = 1 << logQ;
    const int Ns = 1 << logNs;
    const int twshift = 12 - logNs - LOGRADIX;  // 4096 / (Ns * RADIX)
    float2 v[EPT];
    int dst[BPT];
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int b = threadIdx.x + i * blockDim.x;
        int line, j;
        if (LINE_FAST) {
            line = b & ((1 << lognl) - 1);
            j = b >> lognl;
        } else {
            j = b & (Q - 1);
            line = b >> logQ;
        }
        const int k = j & (Ns - 1);
        const int base = line * ls;
#pragma unroll
        for (int s = 0; s < RADIX; ++s) {
            float2 x = buf[base + (j + s * Q) * es];
            if (s > 0) x = cmul(x, __ldg(tw + ((k * s) << twshift)));
            v[i * RADIX + s] = x;
        }
        dst[i] = base + (((j >> logNs) << (logNs + LOGRADIX)) + k) * es;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        dft<RADIX>(v + i * RADIX);
#pragma unroll
        for (int s = 0; s < RADIX; ++s) buf[dst[i] + s * Ns * es] = v[i * RADIX + s];
    }
    __syncthreads();
}

template <int EPT, bool LINE_FAST>
__device__ __forceinline__ void smem_fft(float2* buf, int logL, int lognl, int ls, int es,
                                         const float2* __restrict__ tw)
{
    int logNs = 0;
    for (; logNs + 2 <= logL; logNs += 2)
        fft_stage<2, EPT, LINE_FAST>(buf, logL, logNs, lognl, ls, es, tw);
    if (logNs < logL) fft_stage<1, EPT, LINE_FAST>(buf, logL, logNs, lognl, ls, es, tw);
}

constexpr int kEPT = 32;

__global__ void k_twiddle_init(float2* tw)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < 4096) {
        double s, c;
        sincospi((double)t / 2048.0, &s, &c);  // angle 2 pi t / 4096
        tw[t] = make_float2((float)c, (float)-s);
    }
}

// Pass 1: index map + gather of 2G consecutive samples per row, R-point column
// FFTs over j1 for G adjacent columns, four-step twiddle, coalesced store.
__global__ void __launch_bounds__(512) k_pass1(SeriesView x, const Anchor* __restrict__ anc,
                                               Plan p, const float2* __restrict__ tw,
                                               float2* __restrict__ Y)
{
    extern __shared__ float2 sm[];
    const int tl = blockIdx.y;
    const int G = 1 << p.logG;
    const int nel = 1 << (p.logR + p.logG);
    const int c0 = blockIdx.x << p.logG;
    const Anchor* at = anc + (int64_t)tl * p.nanchor;
    for (int e = threadIdx.x; e < nel; e += blockDim.x) {
        const int j1 = e >> p.logG, g = e & (G - 1);
        const int64_t m = 2 * (((int64_t)j1 << p.logC) + c0 + g);
        const int64_t b = anchor_of(m, p.logB);
        const Anchor a = at[b];
        const int d = (int)(m - anchor_centre(b, p.logB));
        bool pr;
        const int k0 = off_round(a, d, pr);
        const int k1 = off_round(a, d + 1, pr);
        const float v0 = gather_sample(x, p.n, m + a.I + k0);
        const float v1 = gather_sample(x, p.n, m + 1 + a.I + k1);
        sm[e] = make_float2(v0, v1);
    }
    __syncthreads();
    smem_fft<kEPT, true>(sm, p.logR, p.logG, 1, G, tw);
    float2* Yt = Y + (int64_t)tl * p.M;
    for (int e = threadIdx.x; e < nel; e += blockDim.x) {
        const int k1 = e >> p.logG, g = e & (G - 1);
        const int j2 = c0 + g;
        const uint32_t t = ((uint32_t)j2 * (uint32_t)k1) & (uint32_t)(p.M - 1);
        float s, c;
        sincospif(ldexpf((float)t, 1 - p.logM), &s, &c);
        Yt[((int64_t)k1 << p.logC) + j2] = cmul(sm[e], make_float2(c, -s));
    }
}

// |X_k|^2 and |X_{M-k}|^2 from Z_k, Z_{M-k}:  E = (Z_k + conj Z_{M-k})/2,
// O = -i (Z_k - conj Z_{M-k})/2,  X_k = E + W_N^k O,  X_{M-k} = conj(E - W_N^k O).
__device__ __forceinline__ void power_pair(float2 zk, float2 zm, int64_t k, int logn,
                                           float& pa, float& pb)
{
    const float2 E = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
    const float2 O = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
    float s, c;
    sincospif(ldexpf((float)k, 1 - logn), &s, &c);
    const float2 t = cmul(make_float2(c, -s), O);
    const float ar = E.x + t.x, ai = E.y + t.y;
    const float br = E.x - t.x, bi = E.y - t.y;
    pa = ar * ar + ai * ai;
    pb = br * br + bi * bi;
}

// Pass 2: C-point FFTs of the row pair (k1, R - k1) (pair 0 holds the self-
// mirrored rows 0 and R/2), real-FFT split and power, written in natural bin order.
__global__ void __launch_bounds__(512) k_pass2(const float2* __restrict__ Y, Plan p,
                                               const float2* __restrict__ tw,
                                               float* __restrict__ P)
{
    extern __shared__ float2 sm[];
    const int tl = blockIdx.y;
    const int R = 1 << p.logR, C = 1 << p.logC;
    const int pr = blockIdx.x;
    const int rowA = pr, rowB = (pr == 0) ? (R >> 1) : (R - pr);
    const float2* Yt = Y + (int64_t)tl * p.M;
    for (int e = threadIdx.x; e < 2 * C; e += blockDim.x) {
        const int line = e >> p.logC, j2 = e & (C - 1);
        const int row = line ? rowB : rowA;
        sm[e] = Yt[((int64_t)row << p.logC) + j2];
    }
    __syncthreads();
    smem_fft<kEPT, false>(sm, p.logC, 1, C, 1, tw);
    float* Pt = P + (int64_t)tl * p.M;
    if (pr != 0) {
        for (int k2 = threadIdx.x; k2 < C; k2 += blockDim.x) {
            const int64_t k = rowA + ((int64_t)k2 << p.logR);
            float pa, pb;
            power_pair(sm[k2], sm[C + (C - 1 - k2)], k, p.logn, pa, pb);
            Pt[k] = pa;
            Pt[p.M - k] = pb;
        }
    } else {
        for (int k2 = threadIdx.x; k2 <= (C >> 1); k2 += blockDim.x) {
            const int64_t k = (int64_t)k2 << p.logR;
            float pa, pb;
            power_pair(sm[k2], sm[(C - k2) & (C - 1)], k, p.logn, pa, pb);
            if (k2 == 0) {
                Pt[0] = 0.f;
            } else {
                Pt[k] = pa;
                if (k2 != (C >> 1)) Pt[p.M - k] = pb;
            }
        }
        for (int k2 = threadIdx.x; k2 < (C >> 1); k2 += blockDim.x) {
            const int64_t k = (R >> 1) + ((int64_t)k2 << p.logR);
            float pa, pb;
            power_pair(sm[C + k2], sm[C + (C - 1 - k2)], k, p.logn, pa, pb);
            Pt[k] = pa;
            Pt[p.M - k] = pb;
        }
    }
}

// Plain form: power of a cuFFT R2C output (N/2 + 1 bins per template; Nyquist dropped).
__global__ void k_power_r2c(const float2* __restrict__ X, Plan p, float* __restrict__ P)
{
    const int tl = blockIdx.y;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= p.M) return;
    const float2 z = X[(int64_t)tl * (p.M + 1) + k];
    P[(int64_t)tl * p.M + k] = (k == 0) ? 0.f : z.x * z.x + z.y * z.y;
}

}  // namespace

cudaError_t launch_twiddle_init(float2* tw4096, cudaStream_t s)
{
    k_twiddle_init<<<16, 256, 0, s>>>(tw4096);
    return cudaGetLastError();
}

cudaError_t launch_pass1(const SeriesView& x, const Anchor* anc, int nt, const Plan& p,
                         const float2* tw, float2* Y, cudaStream_t s)
{
    const int nel = 1 << (p.logR + p.logG);
    const int threads = nel / kEPT;
    const size_t smem = (size_t)nel * sizeof(float2);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_pass1, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    dim3 grid((unsigned)(1 << (p.logC - p.logG)), (unsigned)nt);
    k_pass1<<<grid, threads, smem, s>>>(x, anc, p, tw, Y);
    return cudaGetLastError();
}

cudaError_t launch_pass2(const float2* Y, int nt, const Plan& p, const float2* tw, float* P,
                         cudaStream_t s)
{
    const int nel = 2 << p.logC;
    const int threads = nel / kEPT;
    const size_t smem = (size_t)nel * sizeof(float2);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_pass2, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    dim3 grid((unsigned)(1 << (p.logR - 1)), (unsigned)nt);
    k_pass2<<<grid, threads, smem, s>>>(Y, p, tw, P);
    return cudaGetLastError();
}

cudaError_t launch_power_from_r2c(const float2* X, int nt, const Plan& p, float* P,
                                  cudaStream_t s)
{
    dim3 grid((unsigned)((p.M + 255) / 256), (unsigned)nt);
    k_power_r2c<<<grid, 256, 0, s>>>(X, p, P);
    return cudaGetLastError();
}

}  // namespace bps
