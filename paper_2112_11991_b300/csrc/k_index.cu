// k_index.cu -- FP64 anchor kernel, standalone index map, plain resampling
// gather, series statistics and FP16 packing.
//
// Anchor kernel (App. A.1, Algorithm 1; Kepler's equation, Sec. 2.1; BT Roemer
// delay, App. A): for every template and every anchor block of B samples it
// reduces the mean anomaly M = Omega t_c + alpha in FP64, solves Kepler's
// equation by FP64 Newton iteration, evaluates the BT delay against the zero
// offset Delta_R(0) (computed per template on the host, dev_template.h), and
// stores the FP32 constants the per-sample evaluation (index_map.cuh) needs.
// FP64 work is N/B Kepler solves per template (B is chosen by the planner,
// typically 4096-16384 samples).
#include <cmath>

#include "bps_internal.cuh"
#include "index_map.cuh"

namespace bps {

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

constexpr double kInvTwoPi = 0.15915494309189533576888376337251;

// x mod 2 pi in [0, 2 pi) (the quotient by a product with 1 / (2 pi): a quotient one off at
// a boundary is put right by the two corrections)
__device__ double reduce_2pi(double x)
{
    double r = x - kTwoPi * floor(x * kInvTwoPi);
    if (r < 0.0) r += kTwoPi;
    if (r >= kTwoPi) r -= kTwoPi;
    return r;
}

// One thread per anchor.  The per-template constants (Omega, sin and cos w, sqrt(1 - e^2),
// the zero offset's Delta_R(0)) come with the template from the host, so no thread waits for
// another; the kernel is bound by the FP64 pipe, so each anchor does one FP64 sincos in the
// circular case (E = M) and, for e > 0, takes sin E and cos E from the Newton iteration's last
// evaluation, advanced by its final step dE to first order (the neglected dE^2 / 2 is below
// 1e-29 once |dE| < 1e-15).
__global__ void k_anchors(const DevTemplate* __restrict__ bank, int64_t t0, Plan p,
                          Anchor* __restrict__ out)
{
    const int tl = blockIdx.y;
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= p.nanchor) return;
    const DevTemplate T = bank[t0 + tl];
    const double e = T.ecc, sw = T.sw, cw = T.cw, rt = T.rt, Om = T.om;
    const int64_t mc = (b << p.logB) + (1ll << (p.logB - 1));
    const double tc = (double)mc * p.tsamp;
    const double M = reduce_2pi(Om * tc + T.phi);
    double sE, cE;
    if (e == 0.0) {
        sincos(M, &sE, &cE);  // Kepler's equation gives E = M
    } else {
        // Kepler's equation E - e sin E = M by Newton iteration from E0 = M + e sin M,
        // keeping the last sincos
        double E = M + e * sin(M), s = 0.0, c = 1.0, dE = 0.0;
        for (int it = 0; it < 40; ++it) {
            sincos(E, &s, &c);
            dE = (E - e * s - M) / (1.0 - e * c);
            E -= dE;
            if (fabs(dE) < 1e-15) break;
        }
        sE = s - c * dE;
        cE = c + s * dE;
    }
    const double Dc = T.tau * ((cE - e) * sw + rt * sE * cw);
    const double O = (T.delta0 - Dc) * p.inv_tsamp;
    const double If = floor(O);
    const double f = O - If;
    const double K = T.tau * p.inv_tsamp;
    const double ws = Om * p.tsamp;
    const double D = 1.0 - e * cE;
    const double invD = 1.0 / D;
    const double g = ws * invD;
    const double Ac = cE * sw + rt * sE * cw;   // -(d^2 BT / dE^2) - e sin w
    const double Bc = -sE * sw + rt * cE * cw;  // d BT / dE
    const double L = K * Bc * g;
    const double u2 = -0.5 * e * sE * g * g * invD;
    const double u3 = -(e * sE * g * u2 + e * cE * g * g * g / 6.0) * invD;
    const double q2 = K * (Bc * u2 - Ac * g * g / 2.0);
    const double q3 = K * (Bc * u3 - Ac * g * u2 - Bc * g * g * g / 6.0);
    Anchor a;
    a.I = (int)If;
    a.fhi = (float)f;
    a.flo = (float)(f - (double)a.fhi);
    a.Lhi = (float)L;
    a.Llo = (float)(L - (double)a.Lhi);
    a.q2 = (float)q2;
    a.q3 = (float)q3;
    a.g = (float)g;
    a.esE = (float)(e * sE);
    a.ecE = (float)(e * cE);
    a.invD = (float)invD;
    a.KBc = (float)(K * Bc);
    a.KAc = (float)(K * Ac);
    a.pad0 = a.pad1 = a.pad2 = 0.f;
    out[(int64_t)tl * p.nanchor + b] = a;
}

__global__ void k_index_map(const Anchor* __restrict__ anc, Plan p, int32_t* __restrict__ idx,
                            unsigned long long* __restrict__ n_precise)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool precise = false;
    if (m < p.n) {
        const int64_t b = anchor_of(m, p.logB);
        const Anchor a = anc[b];
        const int d = (int)(m - anchor_centre(b, p.logB));
        const int k = off_round(a, d, precise);
        idx[m] = (int32_t)(m + a.I + k);
    }
    const unsigned mask = __ballot_sync(0xffffffffu, precise);
    if ((threadIdx.x & 31) == 0 && mask) atomicAdd(n_precise, (unsigned long long)__popc(mask));
}

__global__ void k_resample(SeriesView x, const Anchor* __restrict__ anc, Plan p,
                           float* __restrict__ out)
{
    const int tl = blockIdx.y;
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= p.n) return;
    resolve_fill(x);
    const Anchor* at = anc + (int64_t)tl * p.nanchor;
    const int64_t b = anchor_of(m, p.logB);
    const Anchor a = at[b];
    bool precise;
    const int k = off_round(a, (int)(m - anchor_centre(b, p.logB)), precise);
    out[(int64_t)tl * p.n + m] = gather_sample(x, (int)p.n, (int)(m + a.I + k));
}

__global__ void k_series_sum(const float* __restrict__ x, int64_t n, double* __restrict__ sum)
{
    __shared__ double part[32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        s += (double)x[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? part[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) atomicAdd(sum, s);
    }
}

// FP16 storage with one power-of-two scale per 4096 samples: s = 2^ceil(log2 max|x|),
// h = half(x / s) (division by s is exact, only the FP16 rounding loses bits).
__global__ void k_f16_pack(const float* __restrict__ x, int64_t n, uint16_t* __restrict__ h,
                           float* __restrict__ scale)
{
    __shared__ float wmax[32];
    __shared__ float s_scale;
    const int64_t base = (int64_t)blockIdx.x << 12;
    float mx = 0.f;
    for (int i = threadIdx.x; i < 4096; i += blockDim.x)
        if (base + i < n) mx = fmaxf(mx, fabsf(x[base + i]));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, wmax[w]);
        int ex = 0;
        if (m > 0.f) {
            const float fr = frexpf(m, &ex);  // m = fr * 2^ex, fr in [0.5, 1)
            if (fr == 0.5f) ex -= 1;           // exact power of two: 2^(ex-1) = m
        }
        // exponent rounded up to a multiple of 8: the block's largest |x| lands in
        // (2^-8, 1], well inside the FP16 normal range, and blocks of similar amplitude
        // share one scale (then the gather needs no per-sample scale load)
        ex = ((ex + 7) >> 3) << 3;
        s_scale = ldexpf(1.f, ex);
        scale[blockIdx.x] = s_scale;
    }
    __syncthreads();
    const float inv = 1.f / s_scale;  // exact: power of two
    for (int i = threadIdx.x; i < 4096; i += blockDim.x)
        if (base + i < n) h[base + i] = __half_as_ushort(__float2half_rn(x[base + i] * inv));
}

__global__ void k_fill_from_sum(const double* __restrict__ sum, int64_t n, float* __restrict__ fill)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *fill = (float)(*sum / (double)n);
}

}  // namespace

cudaError_t launch_fill_from_sum(const double* sum, int64_t n, float* fill, cudaStream_t s)
{
    k_fill_from_sum<<<1, 32, 0, s>>>(sum, n, fill);
    return cudaGetLastError();
}

cudaError_t launch_anchors(const DevTemplate* bank, int64_t t0, int nt, const Plan& p,
                           Anchor* out, cudaStream_t s)
{
    dim3 grid((unsigned)((p.nanchor + 63) / 64), (unsigned)nt);
    k_anchors<<<grid, 64, 0, s>>>(bank, t0, p, out);
    return cudaGetLastError();
}

cudaError_t launch_index_map(const Anchor* anc, const Plan& p, int32_t* idx,
                             unsigned long long* n_precise, cudaStream_t s)
{
    k_index_map<<<(unsigned)((p.n + 255) / 256), 256, 0, s>>>(anc, p, idx, n_precise);
    return cudaGetLastError();
}

cudaError_t launch_resample(const SeriesView& x, const Anchor* anc, int nt, const Plan& p,
                            float* out, cudaStream_t s)
{
    dim3 grid((unsigned)((p.n + 255) / 256), (unsigned)nt);
    k_resample<<<grid, 256, 0, s>>>(x, anc, p, out);
    return cudaGetLastError();
}

cudaError_t launch_series_stats(const float* x, int64_t n, double* sum, cudaStream_t s)
{
    int blocks = (int)((n + 1023) / 1024);
    if (blocks > 148 * 8) blocks = 148 * 8;
    k_series_sum<<<blocks, 1024, 0, s>>>(x, n, sum);
    return cudaGetLastError();
}

// scale[nb] = the common scale of blocks 0..nb-1 when they all share it, else 0
__global__ void k_scale_uniform(float* __restrict__ scale, int nb)
{
    __shared__ float smin[8], smax[8];
    float lo = 3.4e38f, hi = 0.f;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        lo = fminf(lo, scale[i]);
        hi = fmaxf(hi, scale[i]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_down_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_down_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        smin[threadIdx.x >> 5] = lo;
        smax[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) {
            lo = fminf(lo, smin[w]);
            hi = fmaxf(hi, smax[w]);
        }
        lo = fminf(lo, smin[0]);
        hi = fmaxf(hi, smax[0]);
        scale[nb] = (lo == hi) ? lo : 0.f;
    }
}

cudaError_t launch_f16_pack(const float* x, int64_t n, uint16_t* h, float* scale,
                            cudaStream_t s)
{
    const int64_t nb = (n + 4095) >> 12;
    k_f16_pack<<<(unsigned)nb, 256, 0, s>>>(x, n, h, scale);
    k_scale_uniform<<<1, 256, 0, s>>>(scale, (int)nb);
    return cudaGetLastError();
}

}  // namespace bps
