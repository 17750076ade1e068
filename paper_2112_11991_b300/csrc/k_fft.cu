// k_fft.cu -- the real FFT of the resampled series as a two-pass four-step
// shared-memory Stockham FFT (Sec. 2.4: one FFT per orbital template gives the
// uniform f0 grid; App. A: "return S' to calculate FFT").
//
// The N real samples are packed as M = N/2 complex points z_j = x'_{2j} + i x'_{2j+1}
// and M = R * C is split four-step:  j = j1*C + j2,  k = k1 + R*k2,
//   pass 1 (gather fused):  Y[k1][j2] = W_M^{j2 k1} * sum_{j1} z[j1 C + j2] W_R^{j1 k1}
//   pass 2 (split + power fused):  Z[k1 + R k2] = sum_{j2} Y[k1][j2] W_C^{j2 k2}
// then X_k = E_k + W_N^k O_k with E/O the even/odd-sample spectra recovered from
// Z_k and Z_{M-k}.  A pass-2 CTA owns NP consecutive rows k1 and their mirrors
// R - k1, so both halves of every split pair are local and the power of NP
// consecutive bins is written as one run.
//
// Both passes hold a tile of at most 2^14 complex values in shared memory (padded
// by one element per 16, which makes the strided radix-16 writes conflict-free)
// and run radix-16 Stockham stages with register butterflies, closed by one
// radix-8/4/2 stage; each thread keeps its EPT = 32 elements in registers across
// the barrier between the read and the write of a stage.
#include <algorithm>
#include <climits>
#include <cmath>
#include <mutex>

#include "bps_internal.cuh"
#include "index_map.cuh"
#include "mbar.cuh"

namespace bps {

namespace {

constexpr int kEPT = 32;   // elements per thread in pass 1 (two radix-16 butterflies)
constexpr int kEPT2 = 16;  // elements per thread in pass 2 (one radix-16 butterfly; 64 registers,
                           // twice the resident warps of 32)
constexpr int kLogTile = 14;  // largest tile (complex values per CTA) of both passes

__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }
// pad(b + s * st) for a stride st that is a multiple of 16 and b >= 0: the shift of b + 16 m
// is the shift of b plus m, so the padded address is pad(b) plus s * (st + st / 16) (a
// constant per element where st is known at compile time; one padding per butterfly)
__device__ __forceinline__ int pad_step(int st) { return st + (st >> 4); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

// Read-only load that does not allocate in L1 (data read once: the twiddle tables keep
// the L1 to themselves)
__device__ __forceinline__ float2 ld_once(const float2* p)
{
    float2 v;
    asm("ld.global.nc.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 mul_negi(float2 a) { return make_float2(a.y, -a.x); }  // a * (-i)

// In-place forward 4-point DFT, natural order in and out.
__device__ __forceinline__ void dft4(float2& a, float2& b, float2& c, float2& d)
{
    const float2 s0 = cadd(a, c), s1 = csub(a, c), s2 = cadd(b, d), s3 = csub(b, d);
    a = cadd(s0, s2);
    c = csub(s0, s2);
    b = make_float2(s1.x + s3.y, s1.y - s3.x);  // s1 - i s3
    d = make_float2(s1.x - s3.y, s1.y + s3.x);  // s1 + i s3
}

constexpr float kR2 = 0.70710678118654752440f;  // 1/sqrt(2)
constexpr float kC8 = 0.92387953251128675613f;  // cos(pi/8)
constexpr float kS8 = 0.38268343236508977173f;  // sin(pi/8)

// Radix-R butterflies in registers.  After dft<R>(v), output X[s] sits in
// v[out_pos<R>(s)] (a fixed register permutation resolved at compile time).
template <int LOGR>
struct Radix;

template <>
struct Radix<1> {
    static __device__ __forceinline__ void dft(float2* v)
    {
        const float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
    static constexpr __device__ __forceinline__ int out_pos(int s) { return s; }
};

template <>
struct Radix<2> {
    static __device__ __forceinline__ void dft(float2* v) { dft4(v[0], v[1], v[2], v[3]); }
    static constexpr __device__ __forceinline__ int out_pos(int s) { return s; }
};

// 8 = 4 x 2: n = 2 n1 + n2, k = k1 + 4 k2
template <>
struct Radix<3> {
    static __device__ __forceinline__ void dft(float2* v)
    {
        dft4(v[0], v[2], v[4], v[6]);
        dft4(v[1], v[3], v[5], v[7]);
        v[3] = make_float2(kR2 * (v[3].x + v[3].y), kR2 * (v[3].y - v[3].x));    // * W8^1
        v[5] = mul_negi(v[5]);                                                    // * W8^2
        v[7] = make_float2(kR2 * (v[7].y - v[7].x), -kR2 * (v[7].x + v[7].y));   // * W8^3
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            const float2 a = v[2 * k1], b = v[2 * k1 + 1];
            v[2 * k1] = cadd(a, b);
            v[2 * k1 + 1] = csub(a, b);
        }
    }
    static constexpr __device__ __forceinline__ int out_pos(int s) { return 2 * (s & 3) + (s >> 2); }
};

// 16 = 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2, inner twiddles W16^{n2 k1}
template <>
struct Radix<4> {
    static __device__ __forceinline__ void dft(float2* v)
    {
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) dft4(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
        v[5] = cmul(v[5], make_float2(kC8, -kS8));                                   // W16^1
        v[9] = make_float2(kR2 * (v[9].x + v[9].y), kR2 * (v[9].y - v[9].x));       // W16^2
        v[13] = cmul(v[13], make_float2(kS8, -kC8));                                 // W16^3
        v[6] = make_float2(kR2 * (v[6].x + v[6].y), kR2 * (v[6].y - v[6].x));       // W16^2
        v[10] = mul_negi(v[10]);                                                     // W16^4
        v[14] = make_float2(kR2 * (v[14].y - v[14].x), -kR2 * (v[14].x + v[14].y)); // W16^6
        v[7] = cmul(v[7], make_float2(kS8, -kC8));                                   // W16^3
        v[11] = make_float2(kR2 * (v[11].y - v[11].x), -kR2 * (v[11].x + v[11].y)); // W16^6
        v[15] = cmul(v[15], make_float2(-kC8, kS8));                                 // W16^9
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) dft4(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    }
    static constexpr __device__ __forceinline__ int out_pos(int s) { return 4 * (s & 3) + (s >> 2); }
};

// Barrier policies of the shared-memory FFT stages: the whole CTA, or the named barrier
// ID of the N threads that run the FFT (the consumer warps of a warp-specialised CTA).
struct SyncCTA {
    static __device__ __forceinline__ void sync() { __syncthreads(); }
};
template <int ID, int N>
struct SyncNamed {
    static __device__ __forceinline__ void sync() { asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(N) : "memory"); }
};

// One Stockham stage of radix 2^LOGRADIX over 2^lognl lines of length L = 2^logL in
// shared memory; element (line, pos) lives at buf[pad(line*ls + pos*es) + line*skew].
// Ns = 2^logNs is the length of the sub-transforms already done.
// (threads running the stage) * EPT == lines * L; tid is the thread's index among them.
template <int LOGRADIX, int EPT, bool LINE_FAST, class SYNC = SyncCTA>
__device__ __forceinline__ void fft_stage(float2* buf, int logL, int logNs, int lognl,
                                          int ls, int es, int skew, const float2* __restrict__ tw,
                                          int tid)
{
    constexpr int RADIX = 1 << LOGRADIX;
    constexpr int BPT = EPT / RADIX;
    const int logQ = logL - LOGRADIX;
    const int Q = 1 << logQ;
    const int Ns = 1 << logNs;
    const int twshift = 13 - logNs - LOGRADIX;  // 8192 / (Ns * RADIX)
    const int nthr = (1 << (logL + lognl)) / EPT;  // == blockDim.x
    // the butterflies of one thread (b = tid + i nthr) share k = j mod Ns, and so their
    // twiddles, when nthr steps j by a multiple of Ns
    const bool shared_k = LINE_FAST ? (((nthr >> lognl) & (Ns - 1)) == 0) : ((nthr & (Q - 1)) == 0);
    float2 v[EPT];
    float2 w[RADIX];
    int dst[BPT], lskv[BPT];
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int b = tid + i * nthr;
        int line, j;
        if (LINE_FAST) {
            line = b & ((1 << lognl) - 1);
            j = b >> lognl;
        } else {
            j = b & (Q - 1);
            line = b >> logQ;
        }
        const int k = j & (Ns - 1);
        const int base = line * ls + j * es;
        const int qs = Q * es;
        const int lsk = line * skew;
        if ((qs & 15) == 0) {
            const float2* src = buf + pad(base) + lsk;
#pragma unroll
            for (int s = 0; s < RADIX; ++s) v[i * RADIX + s] = src[s * pad_step(qs)];
        } else {
#pragma unroll
            for (int s = 0; s < RADIX; ++s) v[i * RADIX + s] = buf[pad(base + s * qs) + lsk];
        }
        if (logNs > 0) {
            // twiddles W^{k s}, s = 1..RADIX-1, from one table load: W^{2^m} by squaring,
            // the others as products of two lower powers (at most 4 products deep)
            if (i == 0 || !shared_k) {
                w[1] = __ldg(tw + (k << twshift));
#pragma unroll
                for (int s = 2; s < RADIX; ++s) {
                    const int hb = (s & (s - 1)) == 0 ? (s >> 1) : (1 << (31 - __clz(s)));
                    w[s] = cmul(w[hb], w[s - hb]);
                }
            }
#pragma unroll
            for (int s = 1; s < RADIX; ++s) v[i * RADIX + s] = cmul(v[i * RADIX + s], w[s]);
        }
        dst[i] = line * ls + (((j >> logNs) << (logNs + LOGRADIX)) + k) * es;
        lskv[i] = lsk;
    }
    SYNC::sync();
    const int nse = Ns * es;
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        Radix<LOGRADIX>::dft(v + i * RADIX);
        if ((nse & 15) == 0) {
            float2* d = buf + pad(dst[i]) + lskv[i];
#pragma unroll
            for (int s = 0; s < RADIX; ++s) d[s * pad_step(nse)] = v[i * RADIX + Radix<LOGRADIX>::out_pos(s)];
        } else {
#pragma unroll
            for (int s = 0; s < RADIX; ++s)
                buf[pad(dst[i] + s * nse) + lskv[i]] = v[i * RADIX + Radix<LOGRADIX>::out_pos(s)];
        }
    }
    SYNC::sync();
}

// Radix-16 stages, then one radix-8/4/2 stage for the remaining factor.
template <int EPT, bool LINE_FAST>
__device__ __forceinline__ void smem_fft(float2* buf, int logL, int lognl, int ls, int es,
                                         int skew, const float2* __restrict__ tw)
{
    int logNs = 0;
    for (; logNs + 4 <= logL; logNs += 4)
        fft_stage<4, EPT, LINE_FAST>(buf, logL, logNs, lognl, ls, es, skew, tw, threadIdx.x);
    const int rem = logL - logNs;
    if (rem == 3) fft_stage<3, EPT, LINE_FAST>(buf, logL, logNs, lognl, ls, es, skew, tw, threadIdx.x);
    else if (rem == 2) fft_stage<2, EPT, LINE_FAST>(buf, logL, logNs, lognl, ls, es, skew, tw, threadIdx.x);
    else if (rem == 1) fft_stage<1, EPT, LINE_FAST>(buf, logL, logNs, lognl, ls, es, skew, tw, threadIdx.x);
}

__global__ void k_twiddle_init(float2* tw)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < kTwiddleN) {
        double s, c;
        sincospi((double)t / 4096.0, &s, &c);  // angle 2 pi t / 8192
        tw[t] = make_float2((float)c, (float)-s);
    }
}

// e^{-2 pi i t / 2^logD} for an exact integer t < 2^24
__device__ __forceinline__ float2 twiddle(uint32_t t, int logD)
{
    float s, c;
    sincospif(ldexpf((float)t, 1 - logD), &s, &c);
    return make_float2(c, -s);
}

// Pass 1: index map + gather fused into the first radix-16 stage, middle radix-16
// stages in shared memory, last stage fused with the four-step twiddle and the
// coalesced store of Y.  Column FFT length R = 2^logR over G adjacent columns;
// stages: 16, 16 x k, 2^r with 4 + 4k + r = logR, r in [1, 4].
//
// First stage (Ns = 1): butterfly (g, j), j < R/16, takes rows j + s R/16 of
// column g, s = 0..15.  Each thread gathers the 32 samples of one butterfly
// (index map fast path for all of them, compensated branch for the rare
// near-boundary ones), transforms them in registers and writes the 16 outputs.
template <int LOGR_LAST>
__device__ __forceinline__ void pass1_last_stage(const float2* __restrict__ sm, int logG, int logC,
                                                 int logM, int c0, int logNs,
                                                 const float2* __restrict__ tw,
                                                 float2* __restrict__ Yt)
{
    constexpr int RL = 1 << LOGR_LAST;
    constexpr int BPT = kEPT / RL;
    const int G = 1 << logG;
    const int Ns = 1 << logNs;  // = R / RL: j < Ns, outputs at k1 = j + s Ns
    const int twshift = 13 - logNs - LOGR_LAST;
    const uint32_t Mm = (uint32_t)((1 << logM) - 1);
    const int nthr = (Ns * RL << logG) / kEPT;  // == blockDim.x
    // four-step twiddle W_M^{j2 k1}, k1 = j + s Ns: W_M^{j2 j} (W_M^{j2 Ns})^s.  The
    // column j2 = c0 + (tid mod G) is the same for all of a thread's butterflies (nthr is
    // a multiple of G), so the powers st[s] = (W_M^{j2 Ns})^s are computed once.
    const uint32_t j2 = (uint32_t)(c0 + (threadIdx.x & (G - 1)));
    float2 st[RL];
    if (RL > 1) {
        st[1] = twiddle((j2 * (uint32_t)Ns) & Mm, logM);
#pragma unroll
        for (int s = 2; s < RL; ++s) {
            const int hb = (s & (s - 1)) == 0 ? (s >> 1) : (1 << (31 - __clz(s)));
            st[s] = cmul(st[hb], st[s - hb]);
        }
    }
    // W_M^{j2 j} of the thread's butterflies: j steps by nthr / G, so with more than two
    // butterflies the later ones take one product each instead of a sincospi
    float2 u0, du;
    if (BPT > 2) {
        u0 = twiddle((j2 * (uint32_t)(threadIdx.x >> logG)) & Mm, logM);
        du = twiddle((j2 * (uint32_t)(nthr >> logG)) & Mm, logM);
    }
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int b = threadIdx.x + i * nthr;
        const int g = b & (G - 1);
        const int j = b >> logG;
        if (BPT <= 2) u0 = twiddle((j2 * (uint32_t)j) & Mm, logM);
        else if (i > 0) u0 = cmul(u0, du);
        float2 v[RL];
        {
            // G Ns is a multiple of 16 (Ns >= 16 after the first radix-16 stage)
            const float2* src = sm + pad(g + G * j);
#pragma unroll
            for (int s = 0; s < RL; ++s) v[s] = src[s * pad_step(G * Ns)];
        }
        {
            float2 w[RL];
            w[1] = __ldg(tw + (j << twshift));
#pragma unroll
            for (int s = 2; s < RL; ++s) {
                const int hb = (s & (s - 1)) == 0 ? (s >> 1) : (1 << (31 - __clz(s)));
                w[s] = cmul(w[hb], w[s - hb]);
            }
#pragma unroll
            for (int s = 1; s < RL; ++s) v[s] = cmul(v[s], w[s]);
        }
        Radix<LOGR_LAST>::dft(v);
        float2 u[RL];
        u[0] = u0;
#pragma unroll
        for (int s = 1; s < RL; ++s) u[s] = cmul(u[0], st[s]);
        // outputs k1 = j + s Ns: row k1 of Y, column j2
        float2* yb = Yt + ((int64_t)j << logC) + j2;
#pragma unroll
        for (int s = 0; s < RL; ++s)
            __stcs(yb + ((int64_t)(s * Ns) << logC), cmul(v[Radix<LOGR_LAST>::out_pos(s)], u[s]));
    }
}

// Source indices of the 32 samples of first-stage butterfly j of column col: complex
// rows j + s R/16 (s < 16), real samples 2 (row C + col) + u (u < 2).  FP32 fast path of
// the index map for all of them, the compensated branch for the rare ones whose
// fractional part lies within the guard of a rounding boundary.
__device__ __forceinline__ void pass1_indices(const Anchor* __restrict__ at, int logB, int logQ,
                                              int logC, int col, int j, int (&id)[32])
{
    const int half = 1 << (logB - 1);
    // the 16 rows of a butterfly lie N/16 samples apart, a multiple of the anchor block
    // (the planner keeps B <= N/16): all 32 samples share their offset d from their
    // anchor centre, and the anchor index steps by a constant
    const int m0 = 2 * ((j << logC) + col);
    const int d = (m0 & ((1 << logB) - 1)) - half;
    const int ab0 = m0 >> logB;
    const int dab = 1 << (logQ + logC + 1 - logB);
    const float dfs[2] = {(float)d, (float)(d + 1)};
    unsigned pm = 0;
#pragma unroll
    for (int s = 0; s < 16; ++s) {
        const int m = m0 + (s << (logQ + logC + 1));
        const int ab = ab0 + s * dab;
        const float4 a4 = __ldg(reinterpret_cast<const float4*>(at + ab));
        const float q3 = __ldg(&at[ab].q3);
        const int I = __float_as_int(a4.x) - kRoundBits;
        const float fh = a4.y, L = a4.z, q2 = a4.w;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            // xr = off - I - 1/2; outside the guard band floor(xr + 1/2) = rint(xr)
            const float df = dfs[u];
            const float xr = fh - df * fmaf(df, fmaf(df, q3, q2), L);
            const float y = __fadd_rn(xr, kRoundShift);
            const float fr = __fsub_rn(xr, __fsub_rn(y, kRoundShift));
            if (!(fabsf(fr) < 0.5f - kGuard)) pm |= 1u << (2 * s + u);
            id[2 * s + u] = m + u + I + __float_as_int(y);
        }
    }
    if (pm) {
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            if (pm & (1u << q)) {
                const int s = q >> 1, u = q & 1;
                const int m = m0 + (s << (logQ + logC + 1));
                const Anchor a = at[ab0 + s * dab];
                id[q] = m + u + a.I + off_round_precise(a, d + u);
            }
        }
    }
}

// The two first-stage butterflies (col, j) and (col + 1, j) of an even column col
// (F16: FP16 series with block scales, else FP32): rows j + s R/16 (s < 16) hold samples 2 (row C + col) + u, u < 4, four
// consecutive samples inside one anchor block (2 col is a multiple of 4), so each row's
// anchor is loaded once for all four; the index map of each sample is pass1_indices'.
// Rows go in two halves of eight (32 indices, then their 32 gathers), so all 64 gathers
// are in flight before either butterfly is transformed.  v0 gets column col + swp, v1
// column col + 1 - swp (swp = 0 or 1: the caller's store order).
template <bool F16>
__device__ __forceinline__ void pass1_gather_colpair(const SeriesView& x, int n, const Anchor* __restrict__ at,
                                                     int logB, int logQ, int logC, int col, int j, int swp,
                                                     float2 (&v0)[16], float2 (&v1)[16])
{
    const int half = 1 << (logB - 1);
    const int m0 = 2 * ((j << logC) + col);
    const int d = (m0 & ((1 << logB) - 1)) - half;
    const int ab0 = m0 >> logB;
    const int dab = 1 << (logQ + logC + 1 - logB);
    // slot u holds sample m0 + (u xor 2 swp)
    int uo[4];
    float dfs[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        uo[u] = u ^ (2 * swp);
        dfs[u] = (float)(d + uo[u]);
    }
#pragma unroll
    for (int h8 = 0; h8 < 2; ++h8) {
        int id[32];
        unsigned pm = 0;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int s = 8 * h8 + r;
            const int m = m0 + (s << (logQ + logC + 1));
            const int ab = ab0 + s * dab;
            const float4 a4 = __ldg(reinterpret_cast<const float4*>(at + ab));
            const float q3 = __ldg(&at[ab].q3);
            const int I = __float_as_int(a4.x) - kRoundBits;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float df = dfs[u];
                const float xr = a4.y - df * fmaf(df, fmaf(df, q3, a4.w), a4.z);
                const float y = __fadd_rn(xr, kRoundShift);
                const float fr = __fsub_rn(xr, __fsub_rn(y, kRoundShift));
                if (!(fabsf(fr) < 0.5f - kGuard)) pm |= 1u << (4 * r + u);
                id[4 * r + u] = m + uo[u] + I + __float_as_int(y);
            }
        }
        if (pm) {
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                if (pm & (1u << q)) {
                    const int s = 8 * h8 + (q >> 2), u = uo[q & 3];
                    const int m = m0 + (s << (logQ + logC + 1));
                    const Anchor a = at[ab0 + s * dab];
                    id[q] = m + u + a.I + off_round_precise(a, d + u);
                }
            }
        }
        if (!F16) {
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                v0[8 * h8 + r] = gather_pair_f32(x, n, id[4 * r], id[4 * r + 1]);
                v1[8 * h8 + r] = gather_pair_f32(x, n, id[4 * r + 2], id[4 * r + 3]);
            }
        } else {
            // FP16 samples: the 32 loads (and block scales) first, then the conversions
            float2 w[16];
            gather_f16_butterfly(x, n, id, w);
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                v0[8 * h8 + r] = w[2 * r];
                v1[8 * h8 + r] = w[2 * r + 1];
            }
        }
    }
}

// LR, LC, LG >= 0: log R, log C, log G fixed at compile time (index arithmetic folds
// into constants); -1: taken from the plan.  F16: the series is stored FP16 with block
// scales (a separate instantiation, so each storage form gets its own register allocation).
template <int LR, int LC, int LG, bool F16>
__global__ void __launch_bounds__(512, 1) k_pass1(SeriesView x, const Anchor* __restrict__ anc,
                                                  Plan p, const float2* __restrict__ tw,
                                                  float2* __restrict__ Y)
{
    extern __shared__ float2 sm[];
    resolve_fill(x);
    const int tl = blockIdx.y;
    const int logG = LG >= 0 ? LG : p.logG;
    const int G = 1 << logG;
    const int logR = LR >= 0 ? LR : p.logR;
    const int logC = LC >= 0 ? LC : p.logC;
    const int logM = (LR >= 0 && LC >= 0) ? LR + LC : p.logM;
    const int logQ = logR - 4;  // rows between the 16 elements of a first-stage butterfly
    const int nthr = (1 << (logR + logG)) / kEPT;  // == blockDim.x
    const int c0 = blockIdx.x << logG;
    const int n = 2 << logM;
    const Anchor* at = anc + (int64_t)tl * p.nanchor;
    constexpr int BPT1 = kEPT / 16;
    static_assert(BPT1 == 2, "two first-stage butterflies per thread");
    if (G >= 2) {
        // thread t: butterfly j = t / (G/2) of the column pair g, g + 1 (g = 2 (t mod G/2)).
        // Element (g', j) of stage row s sits at pad(g' + 16 G j) + G s + (G s) / 16 (g' < G),
        // bank pair (g' + 17 G j) mod 16: the rows j of a warp reach only 16 / G of them for
        // G < 16, so lanes whose bit log2(16 / G) of j is set write their odd column first;
        // each store instruction then hits every bank pair twice (no conflict beyond the
        // two wavefronts 32 float2 need).
        const int g = 2 * ((int)threadIdx.x & ((G >> 1) - 1));
        const int j = (int)threadIdx.x >> (logG - 1);
        const int swp = (j >> (logG < 4 ? 4 - logG : 0)) & 1;
        float2 v0[16], v1[16];
        pass1_gather_colpair<F16>(x, n, at, p.logB, logQ, logC, c0 + g, j, swp, v0, v1);
        Radix<4>::dft(v0);
        float2* d0 = sm + pad(g + swp + 16 * G * j);
#pragma unroll
        for (int s = 0; s < 16; ++s) d0[G * s + ((G * s) >> 4)] = v0[Radix<4>::out_pos(s)];
        Radix<4>::dft(v1);
        float2* d1 = sm + pad(g + 1 - swp + 16 * G * j);
#pragma unroll
        for (int s = 0; s < 16; ++s) d1[G * s + ((G * s) >> 4)] = v1[Radix<4>::out_pos(s)];
    } else {
        // one column per butterfly (G = 1: a column fills the tile)
#pragma unroll 1
        for (int i = 0; i < BPT1; ++i) {
            const int b = threadIdx.x + i * nthr;
            const int g = b & (G - 1);
            const int j = b >> logG;
            int id[32];
            pass1_indices(at, p.logB, logQ, logC, c0 + g, j, id);
            float2 v[16];
            if (!F16) {
#pragma unroll
                for (int s = 0; s < 16; ++s) v[s] = gather_pair_f32(x, n, id[2 * s], id[2 * s + 1]);
            } else {
                gather_f16_butterfly(x, n, id, v);
            }
            Radix<4>::dft(v);
            // pad(g + 16 G j + G s) = pad(g + 16 G j) + G s + (G s) / 16, as g < G
            float2* d = sm + pad(g + 16 * G * j);
#pragma unroll
            for (int s = 0; s < 16; ++s) d[G * s + ((G * s) >> 4)] = v[Radix<4>::out_pos(s)];
        }
    }
    __syncthreads();
    int logNs = 4;
    for (; logNs + 4 < logR; logNs += 4)
        fft_stage<4, kEPT, true>(sm, logR, logNs, logG, 1, G, 0, tw, threadIdx.x);
    float2* Yt = Y + ((int64_t)tl << logM);
    switch (logR - logNs) {
        case 4: pass1_last_stage<4>(sm, logG, logC, logM, c0, logNs, tw, Yt); break;
        case 3: pass1_last_stage<3>(sm, logG, logC, logM, c0, logNs, tw, Yt); break;
        case 2: pass1_last_stage<2>(sm, logG, logC, logM, c0, logNs, tw, Yt); break;
        default: pass1_last_stage<1>(sm, logG, logC, logM, c0, logNs, tw, Yt); break;
    }
}

// ---- Pass 1, warp-specialised --------------------------------------------------------
// The same column FFTs as k_pass1 (R-point FFTs over j1 of z[j1 C + j2] for G adjacent
// columns j2, four-step twiddle, Y store), with the index map and gather taken off the
// FFT warps: a persistent CTA holds kWsBufs tiles of 2^13 complex values in shared memory;
// 16 producer warps compute Algorithm 1's indices and gather the samples of tile i + 1
// (natural order, element g + G j1) while 16 consumer warps run the radix-16 Stockham
// stages of tile i in the other buffer.  Hand-off by mbarriers: full[b] (every producer
// thread arrives after its stores) and empty[b] (every consumer thread arrives after its
// last reads).  Waits are bounded; on expiry the status word gets bit 1 and the CTA
// leaves (the consumers decide together, by a barrier reduction, so none is left at a
// named barrier).
constexpr int kWsLogTile = 13;
constexpr int kWsTile = 1 << kWsLogTile;
constexpr int kWsBufStride = kWsTile + (kWsTile >> 4);  // padded float2 per buffer
constexpr int kWsConsumers = 512;                       // 16 warps x 16 elements
constexpr int kWsProducers = 512;                       // 16 warps
constexpr int kWsThreads = kWsConsumers + kWsProducers;
constexpr int kWsEPT = kWsTile / kWsConsumers;          // 16
constexpr int kWsTw = 512;                              // stage twiddles held in smem
constexpr int kWsHeader = 128;                          // bytes: mbarriers
constexpr int kWsBufs = 2;
constexpr int kWsPUnroll = 4;                           // elements per producer batch
constexpr int kWsAnchors = 2048;                        // anchors of one template held in smem
static_assert(kWsEPT == 16, "one radix-16 butterfly per consumer thread and stage");
static_assert(kWsTile % (kWsProducers * kWsPUnroll) == 0, "producer batches tile the buffer");

size_t ws_pass1_smem()
{
    return (size_t)kWsHeader + (size_t)kWsBufs * kWsBufStride * sizeof(float2) + kWsTw * sizeof(float2) +
           (size_t)kWsAnchors * (sizeof(float4) + sizeof(float));
}

// True, for every one of the 512 threads of named barrier ID (1: consumers, 2: producers),
// when any of them passes true; the threads wait in the barrier, and it orders their
// memory accesses (what one thread acquired before it is visible to all after it).
template <int ID>
__device__ __forceinline__ bool group_any(bool v)
{
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, 512, p;\n"
        " selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(ID)
        : "memory");
    return r != 0;
}

// Last column-FFT stage of the consumers: radix 2^LOGR_LAST with the stage twiddles (from
// the CTA's table stw: stw[j] = W_{Ns RL}^j, j < Ns), the four-step twiddle W_M^{j2 k1}
// and the store of Y[k1][j2].
template <int LOGR_LAST, int LG>
__device__ __forceinline__ void ws_last_stage(const float2* __restrict__ sm, int logC, int logM,
                                              int c0, int logNs, const float2* stw,
                                              float2* __restrict__ Yt, int tid)
{
    constexpr int RL = 1 << LOGR_LAST;
    constexpr int BPT = kWsEPT / RL;
    constexpr int G = 1 << LG;
    const int Ns = 1 << logNs;
    const uint32_t Mm = (uint32_t)((1 << logM) - 1);
    // all of a thread's butterflies share the column j2 (kWsConsumers is a multiple of G)
    const uint32_t j2 = (uint32_t)(c0 + (tid & (G - 1)));
    // powers of W_M^{j2 Ns}: st[s] = (W_M^{j2 Ns})^s, at most four products deep
    float2 st[RL];
    st[0] = make_float2(1.f, 0.f);
    st[1] = twiddle((j2 * (uint32_t)Ns) & Mm, logM);
#pragma unroll
    for (int s = 2; s < RL; ++s) {
        const int hb = (s & (s - 1)) == 0 ? (s >> 1) : (1 << (31 - __clz(s)));
        st[s] = cmul(st[hb], st[s - hb]);
    }
    // W_M^{j2 j} of the thread's butterflies: j steps by kWsConsumers / G
    float2 u0 = twiddle((j2 * (uint32_t)(tid >> LG)) & Mm, logM), du;
    if (BPT > 1) du = twiddle((j2 * (uint32_t)(kWsConsumers >> LG)) & Mm, logM);
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int b = tid + i * kWsConsumers;
        const int g = b & (G - 1);
        const int j = b >> LG;
        if (i > 0) u0 = cmul(u0, du);
        float2 v[RL];
#pragma unroll
        for (int s = 0; s < RL; ++s) v[s] = sm[pad(g + G * (j + s * Ns))];
        {
            float2 w[RL];
            w[1] = stw[j];
#pragma unroll
            for (int s = 2; s < RL; ++s) {
                const int hb = (s & (s - 1)) == 0 ? (s >> 1) : (1 << (31 - __clz(s)));
                w[s] = cmul(w[hb], w[s - hb]);
            }
#pragma unroll
            for (int s = 1; s < RL; ++s) v[s] = cmul(v[s], w[s]);
        }
        Radix<LOGR_LAST>::dft(v);
#pragma unroll
        for (int s = 0; s < RL; ++s) {
            const int k1 = j + s * Ns;
            __stcs(Yt + ((int64_t)k1 << logC) + j2, cmul(v[Radix<LOGR_LAST>::out_pos(s)], cmul(u0, st[s])));
        }
    }
}

// A middle radix-16 Stockham stage of the consumers (Ns = 2^logNs > 1, one butterfly per
// thread), stage twiddles from the CTA's table stw: stw[k] = W_{16 Ns}^k, k < Ns.
template <int LG, class SYNC = SyncNamed<1, kWsConsumers>>
__device__ __forceinline__ void ws_mid_stage(float2* buf, int logR, int logNs, const float2* stw, int tid)
{
    constexpr int G = 1 << LG;
    const int logQ = logR - 4;
    const int Ns = 1 << logNs;
    const int line = tid & (G - 1);
    const int j = tid >> LG;
    const int k = j & (Ns - 1);
    float2 v[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) v[s] = buf[pad(line + G * (j + (s << logQ)))];
    {
        float2 w[16];
        w[1] = stw[k];
#pragma unroll
        for (int s = 2; s < 16; ++s) {
            const int hb = (s & (s - 1)) == 0 ? (s >> 1) : (1 << (31 - __clz(s)));
            w[s] = cmul(w[hb], w[s - hb]);
        }
#pragma unroll
        for (int s = 1; s < 16; ++s) v[s] = cmul(v[s], w[s]);
    }
    const int dst = line + G * (((j >> logNs) << (logNs + 4)) + k);
    SYNC::sync();
    Radix<4>::dft(v);
#pragma unroll
    for (int s = 0; s < 16; ++s) buf[pad(dst + G * s * Ns)] = v[Radix<4>::out_pos(s)];
    SYNC::sync();
}

// Index map (FP32 fast path, compensated branch inside the guard band) and gather of the
// two samples 2m, 2m + 1 of one complex element.
__device__ __forceinline__ void ws_indices(const Anchor* __restrict__ at, const float4* a4c,
                                           const float* q3c, int logB, int m, int& i0, int& i1)
{
    const int ab = m >> logB;
    // fast-path fields from the CTA's copy of the template's anchors when it holds them
    const float4 a4 = a4c ? a4c[ab] : __ldg(reinterpret_cast<const float4*>(at + ab));
    const float q3 = a4c ? q3c[ab] : __ldg(&at[ab].q3);
    const int I = __float_as_int(a4.x) - kRoundBits;
    const int d = m - ((ab << logB) + (1 << (logB - 1)));
    unsigned bad = 0;
    int id[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const float df = (float)(d + u);
        const float xr = a4.y - df * fmaf(df, fmaf(df, q3, a4.w), a4.z);
        const float y = __fadd_rn(xr, kRoundShift);
        const float fr = __fsub_rn(xr, __fsub_rn(y, kRoundShift));
        if (!(fabsf(fr) < 0.5f - kGuard)) bad |= 1u << u;
        id[u] = m + u + I + __float_as_int(y);
    }
    if (bad) {
        const Anchor a = at[ab];
        if (bad & 1u) id[0] = m + a.I + off_round_precise(a, d);
        if (bad & 2u) id[1] = m + 1 + a.I + off_round_precise(a, d + 1);
    }
    i0 = id[0];
    i1 = id[1];
}

template <int LR, int LC>
__global__ void __launch_bounds__(kWsThreads, 1) k_pass1_ws(SeriesView x, const Anchor* __restrict__ anc,
                                                            Plan p, const float2* __restrict__ tw,
                                                            float2* __restrict__ Y, int ntiles,
                                                            unsigned long long* __restrict__ status)
{
    constexpr int LG = kWsLogTile - LR;  // columns per tile
    constexpr int G = 1 << LG;
    constexpr int LCG = LC - LG;        // log2 column groups (tiles) per template
    constexpr int LM = LR + LC;
    static_assert(LG >= 0 && LCG >= 0, "tile geometry");
    extern __shared__ __align__(128) unsigned char wsm[];
    uint64_t* full = reinterpret_cast<uint64_t*>(wsm);
    uint64_t* empty = full + kWsBufs;
    float2* bufs = reinterpret_cast<float2*>(wsm + kWsHeader);
    float2* stw = bufs + kWsBufs * kWsBufStride;  // [0, 16): W_256^k; [16, 16 + Ns_last): last stage
    float4* a4s = reinterpret_cast<float4*>(stw + kWsTw);
    float* q3s = reinterpret_cast<float*>(a4s + kWsAnchors);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int b = 0; b < kWsBufs; ++b) {
            mbar_init(&full[b], kWsProducers);
            mbar_init(&empty[b], kWsConsumers / 32);
        }
    }
    // stage twiddles from the 8192 table: W_256^k, k < 16, for the one middle radix-16
    // stage (Ns = 16), and W_{Ns RL}^j, j < Ns = 256, for the last stage (radix RL = R / 256)
    constexpr int LNS_LAST = ((LR - 1) / 4) * 4;
    constexpr int RL_LAST = LR - LNS_LAST;
    static_assert(LNS_LAST == 8 && 16 + (1 << LNS_LAST) <= kWsTw, "stages 16 x 16 x (R / 256)");
    for (int t = threadIdx.x; t < 16; t += kWsThreads) stw[t] = __ldg(tw + (t << (13 - 8)));
    for (int t = threadIdx.x; t < (1 << LNS_LAST); t += kWsThreads)
        stw[16 + t] = __ldg(tw + (t << (13 - LNS_LAST - RL_LAST)));
    __syncthreads();
    resolve_fill(x);
    const int n = 2 << LM;
    if (threadIdx.x >= kWsConsumers) {
        // ---- producers: index map + gather of tile i into buffer i mod kWsBufs ----
        const int pt = (int)threadIdx.x - kWsConsumers;
        const bool cache = p.nanchor <= kWsAnchors;
        int cached = -1;  // template whose anchors the CTA holds
        for (int i = 0;; ++i) {
            const int u = (int)blockIdx.x + i * (int)gridDim.x;
            if (u >= ntiles) break;
            const int b = i % kWsBufs, k = i / kWsBufs;
            // one producer polls for the buffer to be free, the others wait in the barrier
            bool ok = true;
            if (k > 0 && pt == 0) ok = mbar_wait_parity(&empty[b], (uint32_t)((k - 1) & 1));
            if (group_any<2>(!ok)) {
                if (pt == 0) atomicOr(status, 2ull);
                break;
            }
            const int tl = u >> LCG;
            const int c0 = (u & ((1 << LCG) - 1)) << LG;
            const Anchor* at = anc + (int64_t)tl * p.nanchor;
            if (cache && tl != cached) {  // every producer is past the previous tile here
                for (int a = pt; a < (int)p.nanchor; a += kWsProducers) {
                    a4s[a] = __ldg(reinterpret_cast<const float4*>(at + a));
                    q3s[a] = __ldg(&at[a].q3);
                }
                asm volatile("bar.sync 2, 512;" ::: "memory");
                cached = tl;
            }
            const float4* a4c = cache ? a4s : nullptr;
            float2* sb = bufs + b * kWsBufStride;
            if (x.f32 && x.fillp) {
                // FP32 series: every sample of the tile by a 4-byte asynchronous copy (the
                // series mean from its device copy outside [0, n)), so all 32 of the
                // thread's gathers are in flight at once; the mbarrier counts the thread's
                // arrival when they have landed
#pragma unroll 4
                for (int r = 0; r < kWsTile / kWsProducers; ++r) {
                    const int e = pt + r * kWsProducers;
                    const int m = 2 * (((e >> LG) << LC) + c0 + (e & (G - 1)));
                    int i0, i1;
                    ws_indices(at, a4c, q3s, p.logB, m, i0, i1);
                    const uint32_t dst = smem_u32(sb + pad(e));
                    cp_async4(dst, (unsigned)i0 < (unsigned)n ? x.f32 + i0 : x.fillp);
                    cp_async4(dst + 4u, (unsigned)i1 < (unsigned)n ? x.f32 + i1 : x.fillp);
                }
                cp_async_mbar_arrive(&full[b]);
                continue;
            }
#pragma unroll 1
            for (int e0 = 0; e0 < kWsTile; e0 += kWsProducers * kWsPUnroll) {
                int id[2 * kWsPUnroll];
#pragma unroll
                for (int r = 0; r < kWsPUnroll; ++r) {
                    const int e = e0 + pt + r * kWsProducers;
                    const int m = 2 * (((e >> LG) << LC) + c0 + (e & (G - 1)));
                    ws_indices(at, a4c, q3s, p.logB, m, id[2 * r], id[2 * r + 1]);
                }
                float2 v[kWsPUnroll];
                if (x.f32) {
#pragma unroll
                    for (int r = 0; r < kWsPUnroll; ++r) v[r] = gather_pair_f32(x, n, id[2 * r], id[2 * r + 1]);
                } else {
                    unsigned short hv[2 * kWsPUnroll];
                    float sv[2 * kWsPUnroll];
#pragma unroll
                    for (int q = 0; q < 2 * kWsPUnroll; ++q) {
                        const bool in = (unsigned)id[q] < (unsigned)n;
                        hv[q] = in ? __ldg(x.f16 + id[q]) : (unsigned short)0;
                        sv[q] = !in ? 0.f : (x.uscale > 0.f ? x.uscale : __ldg(x.scale + (id[q] >> 12)));
                    }
#pragma unroll
                    for (int r = 0; r < kWsPUnroll; ++r) {
                        const bool in0 = (unsigned)id[2 * r] < (unsigned)n;
                        const bool in1 = (unsigned)id[2 * r + 1] < (unsigned)n;
                        v[r] = make_float2(in0 ? __half2float(__ushort_as_half(hv[2 * r])) * sv[2 * r] : x.fill,
                                           in1 ? __half2float(__ushort_as_half(hv[2 * r + 1])) * sv[2 * r + 1] : x.fill);
                    }
                }
#pragma unroll
                for (int r = 0; r < kWsPUnroll; ++r) sb[pad(e0 + pt + r * kWsProducers)] = v[r];
            }
            mbar_arrive(&full[b]);
        }
        // the thread's asynchronous copies land before it leaves (the CTA's shared memory
        // outlives them also when the consumers gave up on a wait)
        asm volatile("cp.async.wait_all;" ::: "memory");
        return;
    }
    // ---- consumers: column FFTs of tile i ----
    const int ct = (int)threadIdx.x;
    for (int i = 0;; ++i) {
        const int u = (int)blockIdx.x + i * (int)gridDim.x;
        if (u >= ntiles) break;
        const int b = i % kWsBufs, k = i / kWsBufs;
        // one consumer polls for the tile, the others wait in the barrier
        bool ok = true;
        if (ct == 0) ok = mbar_wait_parity(&full[b], (uint32_t)(k & 1));
        if (group_any<1>(!ok)) {
            if (ct == 0) atomicOr(status, 2ull);
            break;
        }
        const int tl = u >> LCG;
        const int c0 = (u & ((1 << LCG) - 1)) << LG;
        float2* sb = bufs + b * kWsBufStride;
        fft_stage<4, kWsEPT, true, SyncNamed<1, kWsConsumers>>(sb, LR, 0, LG, 1, G, 0, tw, ct);
#pragma unroll
        for (int logNs = 4; logNs < LNS_LAST; logNs += 4) ws_mid_stage<LG>(sb, LR, logNs, stw, ct);
        float2* Yt = Y + ((int64_t)tl << LM);
        ws_last_stage<RL_LAST, LG>(sb, LC, LM, c0, LNS_LAST, stw + 16, Yt, ct);
        __syncwarp();
        if ((ct & 31) == 0) mbar_arrive(&empty[b]);  // the warp's reads of the buffer are done
    }
}

// |X_k|^2 and |X_{M-k}|^2 from Z_k, Z_{M-k} and w = W_N^k:
// E = (Z_k + conj Z_{M-k})/2, O = -i (Z_k - conj Z_{M-k})/2,
// X_k = E + w O,  X_{M-k} = conj(E - w O).
__device__ __forceinline__ void power_pair(float2 zk, float2 zm, float2 w, float& pa, float& pb)
{
    const float2 E = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
    const float2 O = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
    const float2 t = cmul(w, O);
    const float ar = E.x + t.x, ai = E.y + t.y;
    const float br = E.x - t.x, bi = E.y - t.y;
    pa = ar * ar + ai * ai;
    pb = br * br + bi * bi;
}

// Pass 2: C-point FFTs of NP row pairs (q, R - q), q in [q0, q0 + NP) (pair 0 holds
// the self-mirrored rows 0 and R/2), then real-FFT split and power.  Items are
// assigned q-fastest so each warp writes NP consecutive bins per k2.
// LR, LC, LNP >= 0: log R, log C, log NP fixed at compile time; -1: from the plan.
// One pass-2 tile (template tl, row pairs from q0) by the tid-th of nthr threads: the
// first radix-16 stage reads the rows from Y in global memory (STAGED = false) or from the
// unpadded copy of the tile's 2 NP rows in shared memory at src, line l at src + l C
// (STAGED = true); the tile is transformed in sm; SYNC is the barrier of the nthr threads.
template <int LR, int LC, int LNP, class SYNC, bool STAGED>
__device__ __forceinline__ void pass2_tile(const float2* __restrict__ src, int tl, int q0, const Plan& p,
                                           const float2* __restrict__ tw, float* __restrict__ P,
                                           float2* sm, float2* s_wq, int tid)
{
    const int logR = LR >= 0 ? LR : p.logR;
    const int logC = LC >= 0 ? LC : p.logC;
    const int logM = logR + logC;
    const int logn = logM + 1;
    const int64_t M = (int64_t)1 << logM;
    const int R = 1 << logR, C = 1 << logC;
    const int logNP = LNP >= 0 ? LNP : p.logNP;
    const int NP = 1 << logNP;
    const int nthr = (NP * C * 2) / kEPT2;  // threads of the tile
    const float2* Yt = src + (STAGED ? 0 : (int64_t)tl * M);
    // lines [0, NP): low rows q0 + l ; lines [NP, 2NP): their mirrors.  Line l starts
    // at pad(l*C) + l*skew (pad(l*C) is a multiple of 16 complex).  In the split phase a
    // half-warp reads NP lines at 16/NP consecutive k2 each; skew = 16/NP puts the lines
    // 16/NP complex apart modulo 16, i.e. on disjoint bank pairs (at most 64 complex of
    // slack in all).  The first radix-16 stage (Ns = 1) is fused with the load:
    // butterfly (line, j) reads elements j + s C/16 of its row straight from Y.
    const int skew = logNP <= 4 ? (16 >> logNP) : (logNP == 5 ? 1 : 0);
    // W_N^q of the NP low rows, for the row-major power layout (plan.ptrans, NP <= 2);
    // visible to all after the first-stage barrier
    if (p.ptrans && tid < NP) s_wq[tid] = twiddle((uint32_t)(q0 + tid), logn);
    const int logQ = logC - 4;
    constexpr int BPT1 = kEPT2 / 16;
#pragma unroll
    for (int i = 0; i < BPT1; ++i) {
        const int b = tid + i * nthr;
        const int j = b & ((1 << logQ) - 1);
        const int line = b >> logQ;
        const int q = q0 + (line & (NP - 1));
        const int row = (line < NP) ? q : (q == 0 ? (R >> 1) : R - q);
        float2 v[16];
        if (STAGED) {
            const float2* rs = Yt + ((int64_t)line << logC) + j;
#pragma unroll
            for (int s = 0; s < 16; ++s) v[s] = rs[s << logQ];
        } else {
            const float2* rs = Yt + ((int64_t)row << logC) + j;
#pragma unroll
            for (int s = 0; s < 16; ++s) v[s] = ld_once(rs + (s << logQ));
        }
        Radix<4>::dft(v);
        // base is a multiple of 16, so pad(base + s) = pad(base) + s for s < 16
        float2* d = sm + pad(line * C + 16 * j) + line * skew;
#pragma unroll
        for (int s = 0; s < 16; ++s) d[s] = v[Radix<4>::out_pos(s)];
    }
    SYNC::sync();
    {
        int logNs = 4;
        for (; logNs + 4 <= logC; logNs += 4)
            fft_stage<4, kEPT2, false, SYNC>(sm, logC, logNs, logNP + 1, C, 1, skew, tw, tid);
        const int rem = logC - logNs;
        if (rem == 3) fft_stage<3, kEPT2, false, SYNC>(sm, logC, logNs, logNP + 1, C, 1, skew, tw, tid);
        else if (rem == 2) fft_stage<2, kEPT2, false, SYNC>(sm, logC, logNs, logNP + 1, C, 1, skew, tw, tid);
        else if (rem == 1) fft_stage<1, kEPT2, false, SYNC>(sm, logC, logNs, logNP + 1, C, 1, skew, tw, tid);
    }
    float* Pt = P + (int64_t)tl * M;
    if (p.ptrans) {
        // row-major power, columns in blocks of 8, rows in groups of NP (kLogPowCols):
        // bin k1 + R k2 at P'[(k2 div 8) 8 R + (k1 div NP) 8 NP + (k2 mod 8) NP + k1 mod NP].
        // Items q-fastest: a warp's low-row stores are 32 NP-byte runs of whole sectors
        // (their mirrors straddle two groups), and the median kernel reads the 8 columns
        // x W rows of its blocks as one contiguous run.
        constexpr int LB = kLogPowCols;
        const int twsh = 12 - logC;
        const auto at_ = [&](int k1, int k2) -> int64_t {
            return ((int64_t)(k2 >> LB) << (logR + LB)) +
                   ((int64_t)(k1 >> logNP) << (logNP + LB)) + ((k2 & ((1 << LB) - 1)) << logNP) +
                   (k1 & (NP - 1));
        };
        static_assert(kEPT2 % 2 == 0, "items per thread");
        // a thread's items share ql and step k2 by S = nthr / NP = C / 8; when S is a multiple
        // of 16 the padded addresses of its low and mirror elements step by pad_step(S)
        const int S = nthr >> logNP;
        const bool sstep = (S & 15) == 0;
        const int ql0 = tid & (NP - 1), k20 = tid >> logNP;
        const int lo_base = pad(ql0 * C + k20) + ql0 * skew;
        const int hi_base = pad((NP + ql0) * C + (C - 1 - k20)) + (NP + ql0) * skew;
        // with S a multiple of 8 the items' output offsets step by S / 8 column blocks of
        // 8 R floats (k2 mod 8 and the row part are the same for all of a thread's items)
        const bool astep = (S & ((1 << LB) - 1)) == 0;
        const int64_t astride = (int64_t)(S >> LB) << (logR + LB);
        const int64_t a_lo = at_(q0 + ql0, k20), a_hi = at_(R - (q0 + ql0), C - 1 - k20);
#pragma unroll
        for (int r = 0; r < kEPT2 / 2; ++r) {  // items = NP C = (kEPT2 / 2) nthr
            const int it = tid + r * nthr;
            const int ql = it & (NP - 1), k2 = it >> logNP;
            const int q = q0 + ql;
            const int lowl = ql, highl = NP + ql;
            const int lo0 = lowl * skew, hi0 = highl * skew;
            float pa, pb;
            if (q != 0) {
                const float2 w = cmul(s_wq[ql], __ldg(tw + (k2 << twsh)));
                const int la = sstep ? lo_base + r * pad_step(S) : pad(lowl * C + k2) + lo0;
                const int ha = sstep ? hi_base - r * pad_step(S) : pad(highl * C + (C - 1 - k2)) + hi0;
                power_pair(sm[la], sm[ha], w, pa, pb);
                Pt[astep ? a_lo + r * astride : at_(q, k2)] = pa;
                Pt[astep ? a_hi - r * astride : at_(R - q, C - 1 - k2)] = pb;
            } else {
                if (k2 <= (C >> 1)) {  // row 0: bins R k2 and M - R k2 = R (C - k2)
                    power_pair(sm[pad(k2) + lo0], sm[pad((C - k2) & (C - 1)) + lo0],
                               __ldg(tw + (k2 << twsh)), pa, pb);
                    if (k2 == 0) {
                        Pt[0] = 0.f;
                    } else {
                        Pt[at_(0, k2)] = pa;
                        if (k2 != (C >> 1)) Pt[at_(0, C - k2)] = pb;
                    }
                }
                if (k2 < (C >> 1)) {  // row R/2: bins R/2 + R k2 and R/2 + R (C - 1 - k2)
                    const float2 w =
                        cmul(twiddle((uint32_t)(R >> 1), logn), __ldg(tw + (k2 << twsh)));
                    power_pair(sm[pad(highl * C + k2) + hi0],
                               sm[pad(highl * C + (C - 1 - k2)) + hi0], w, pa, pb);
                    Pt[at_(R >> 1, k2)] = pa;
                    Pt[at_(R >> 1, C - 1 - k2)] = pb;
                }
            }
        }
        return;
    }
    // W_N^{q + R k2} = W_N^q * W_{2C}^{k2};  W_{2C}^{k2} = tw[k2 * 8192 / (2C)]
    const int ql = tid & (NP - 1);
    const int q = q0 + ql;
    const float2 wq = twiddle((uint32_t)q, logn);
    const int twsh = 12 - logC;
    const int lowl = ql, highl = NP + ql;
    const int lo0 = lowl * skew, hi0 = highl * skew;
    const int S = nthr >> logNP;  // k2 step between a thread's items
    const bool sstep = (S & 15) == 0;
    const int lo_base = pad(lowl * C + (tid >> logNP)) + lo0;
    const int hi_base = pad(highl * C + (C - 1 - (tid >> logNP))) + hi0;
#pragma unroll
    for (int r = 0; r < kEPT2 / 2; ++r) {  // items = NP C = (kEPT2 / 2) nthr
        const int it = tid + r * nthr;
        const int k2 = it >> logNP;
        if (q != 0) {
            const int64_t k = q + ((int64_t)k2 << logR);
            const float2 w = cmul(wq, __ldg(tw + (k2 << twsh)));
            float pa, pb;
            const int la = sstep ? lo_base + r * pad_step(S) : pad(lowl * C + k2) + lo0;
            const int ha = sstep ? hi_base - r * pad_step(S) : pad(highl * C + (C - 1 - k2)) + hi0;
            power_pair(sm[la], sm[ha], w, pa, pb);
            Pt[k] = pa;
            Pt[M - k] = pb;
        } else {
            if (k2 <= (C >> 1)) {  // row 0: bins R k2 and M - R k2
                const int64_t k = (int64_t)k2 << logR;
                float pa, pb;
                power_pair(sm[pad(k2) + lo0], sm[pad((C - k2) & (C - 1)) + lo0],
                           __ldg(tw + (k2 << twsh)), pa, pb);
                if (k2 == 0) {
                    Pt[0] = 0.f;
                } else {
                    Pt[k] = pa;
                    if (k2 != (C >> 1)) Pt[M - k] = pb;
                }
            }
            if (k2 < (C >> 1)) {  // row R/2: bins R/2 + R k2 and M - (R/2 + R k2)
                const int64_t k = (R >> 1) + ((int64_t)k2 << logR);
                const float2 w =
                    cmul(twiddle((uint32_t)(R >> 1), logn), __ldg(tw + (k2 << twsh)));
                float pa, pb;
                power_pair(sm[pad(highl * C + k2) + hi0], sm[pad(highl * C + (C - 1 - k2)) + hi0],
                           w, pa, pb);
                Pt[k] = pa;
                Pt[M - k] = pb;
            }
        }
    }
}

template <int LR, int LC, int LNP>
__global__ void __launch_bounds__(1024, 1) k_pass2(const float2* __restrict__ Y, Plan p,
                                                  const float2* __restrict__ tw,
                                                  float* __restrict__ P)
{
    extern __shared__ float2 sm[];
    __shared__ float2 s_wq[64];
    const int logNP = LNP >= 0 ? LNP : p.logNP;
    pass2_tile<LR, LC, LNP, SyncCTA, false>(Y, blockIdx.y, blockIdx.x << logNP, p, tw, P, sm, s_wq,
                                           threadIdx.x);
}

// ---- Pass 1 with asynchronous gathers, two CTAs per SM ----------------------------------
// The one-phase organisation of k_pass1 (each thread gathers the 32 samples of its first
// radix-16 butterfly, then all run the column FFTs of the tile), with the gather issued as
// 4-byte cp.async copies straight into the tile: no register holds a sample while the L2
// answers, so 16 elements per thread fit 64 registers and two 512-thread CTAs (2^13 tiles)
// share an SM, one gathering while the other transforms.  Index map as k_pass1's (one
// anchor offset per butterfly); FP32 series with a device copy of the fill value only.
template <int LR, int LC>
__global__ void __launch_bounds__(512, 2) k_pass1_async(SeriesView x, const Anchor* __restrict__ anc,
                                                        Plan p, const float2* __restrict__ tw,
                                                        float2* __restrict__ Y)
{
    constexpr int LG = 13 - LR;
    constexpr int G = 1 << LG;
    constexpr int LM = LR + LC;
    constexpr int LQ = LR - 4;
    constexpr int LNS_LAST = ((LR - 1) / 4) * 4;
    constexpr int RL_LAST = LR - LNS_LAST;
    static_assert(LNS_LAST == 8, "stages 16 x 16 x (R / 256)");
    extern __shared__ __align__(16) float2 asm_[];
    float2* sm = asm_;
    float2* stw = asm_ + kWsBufStride;  // [0, 16): W_256^k; [16, 272): last stage
    const int tid = (int)threadIdx.x;
    const int tl = blockIdx.y;
    const int c0 = blockIdx.x << LG;
    const int n = 2 << LM;
    resolve_fill(x);
    if (tid < 16) stw[tid] = __ldg(tw + (tid << (13 - 8)));
    if (tid < 256) stw[16 + tid] = __ldg(tw + (tid << (13 - LNS_LAST - RL_LAST)));
    // ---- gather: butterfly (g, j) takes rows j + s R/16 of column g ----
    {
        const Anchor* at = anc + (int64_t)tl * p.nanchor;
        const int g = tid & (G - 1), j = tid >> LG;
        const int logB = p.logB;
        const int half = 1 << (logB - 1);
        const int m0 = 2 * ((j << LC) + c0 + g);
        const int d = (m0 & ((1 << logB) - 1)) - half;
        const int ab0 = m0 >> logB;
        const int dab = 1 << (LQ + LC + 1 - logB);
        const float dfs[2] = {(float)d, (float)(d + 1)};
#pragma unroll
        for (int s2 = 0; s2 < 16; ++s2) {
            const int m = m0 + (s2 << (LQ + LC + 1));
            const int ab = ab0 + s2 * dab;
            const float4 a4 = __ldg(reinterpret_cast<const float4*>(at + ab));
            const float q3 = __ldg(&at[ab].q3);
            const int I = __float_as_int(a4.x) - kRoundBits;
            const uint32_t dst = smem_u32(sm + pad(g + G * (j + (s2 << LQ))));
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const float df = dfs[u];
                const float xr = a4.y - df * fmaf(df, fmaf(df, q3, a4.w), a4.z);
                const float y = __fadd_rn(xr, kRoundShift);
                const float fr = __fsub_rn(xr, __fsub_rn(y, kRoundShift));
                int id = m + u + I + __float_as_int(y);
                if (!(fabsf(fr) < 0.5f - kGuard)) {
                    const Anchor a = at[ab];
                    id = m + u + a.I + off_round_precise(a, d + u);
                }
                cp_async4(dst + 4u * u, (unsigned)id < (unsigned)n ? x.f32 + id : x.fillp);
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    }
    __syncthreads();
    fft_stage<4, 16, true>(sm, LR, 0, LG, 1, G, 0, tw, tid);
    ws_mid_stage<LG, SyncCTA>(sm, LR, 4, stw, tid);
    ws_last_stage<RL_LAST, LG>(sm, LC, LM, c0, LNS_LAST, stw + 16, Y + ((int64_t)tl << LM), tid);
}

// ---- Pass 2 fed by TMA bulk copies ------------------------------------------------------
// A persistent CTA per SM walks the pass-2 tiles (2 NP rows of C complex = 2^13 values):
// one producer thread copies the 2 NP rows of tile i + 1 from Y into an unpadded staging
// buffer with 1D bulk copies (each row is one contiguous run of 8 C bytes, completed on
// the buffer's "full" mbarrier), while 16 consumer warps transform tile i: the first
// radix-16 stage reads the staging buffer (lanes read consecutive elements: no bank
// conflicts without padding) into the padded work tile, the rest is pass2_tile's.  The
// buffer returns to the producer ("empty", one arrival per consumer warp) when its tile is
// done.  Waits are bounded; on expiry the status word gets bit 2.
constexpr int kP2Consumers = 512;
constexpr int kP2Threads = kP2Consumers + 32;
constexpr int kP2Stages = 2;
constexpr int kP2Tile = 1 << 13;
constexpr int kP2Work = kP2Tile + (kP2Tile >> 4) + 64;  // padded work tile + line skew (float2)

size_t p2tma_smem()
{
    return 128 + (size_t)(kP2Stages * kP2Tile + kP2Work + 64) * sizeof(float2);
}

template <int LR, int LC, int LNP>
__global__ void __launch_bounds__(kP2Threads, 1) k_pass2_tma(const float2* __restrict__ Y, Plan p,
                                                             const float2* __restrict__ tw,
                                                             float* __restrict__ P, int ntiles,
                                                             unsigned long long* __restrict__ status)
{
    constexpr int NP = 1 << LNP;
    constexpr int C = 1 << LC;
    constexpr int R = 1 << LR;
    constexpr int LTPT = LR - 1 - LNP;  // log2 of the tiles per template
    static_assert(2 * NP * C == kP2Tile && LTPT >= 0, "tiles of 2^13 complex values");
    extern __shared__ __align__(128) unsigned char psm[];
    uint64_t* full = reinterpret_cast<uint64_t*>(psm);
    uint64_t* empty = full + kP2Stages;
    float2* stg = reinterpret_cast<float2*>(psm + 128);
    float2* sm = stg + kP2Stages * kP2Tile;
    float2* s_wq = sm + kP2Work;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int b = 0; b < kP2Stages; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], kP2Consumers / 32);
        }
    }
    __syncthreads();
    const int64_t M = (int64_t)1 << (LR + LC);
    if (threadIdx.x >= kP2Consumers) {
        // ---- producer: lane 0 of the last warp ----
        if (threadIdx.x != kP2Consumers) return;
        int i = 0;
        for (;; ++i) {
            const int u = (int)blockIdx.x + i * (int)gridDim.x;
            if (u >= ntiles) break;
            const int b = i % kP2Stages, k = i / kP2Stages;
            if (k > 0 && !mbar_wait_parity(&empty[b], (uint32_t)((k - 1) & 1))) {
                atomicOr(status, 4ull);
                break;
            }
            const int tl = u >> LTPT;
            const int q0 = (u & ((1 << LTPT) - 1)) << LNP;
            mbar_expect_tx(&full[b], (uint32_t)(kP2Tile * sizeof(float2)));
#pragma unroll
            for (int l = 0; l < 2 * NP; ++l) {
                const int q = q0 + (l & (NP - 1));
                const int row = (l < NP) ? q : (q == 0 ? (R >> 1) : R - q);
                tma_load_1d(stg + b * kP2Tile + l * C, Y + (int64_t)tl * M + ((int64_t)row << LC),
                            (uint32_t)(C * sizeof(float2)), &full[b]);
            }
        }
        // let the copies issued last land before the CTA's shared memory can go away
        for (int m = (i > kP2Stages ? i - kP2Stages : 0); m < i; ++m)
            (void)mbar_wait_parity(&full[m % kP2Stages], (uint32_t)((m / kP2Stages) & 1));
        return;
    }
    // ---- consumers ----
    const int ct = (int)threadIdx.x;
    for (int i = 0;; ++i) {
        const int u = (int)blockIdx.x + i * (int)gridDim.x;
        if (u >= ntiles) break;
        const int b = i % kP2Stages, k = i / kP2Stages;
        bool ok = true;
        if (ct == 0) ok = mbar_wait_parity(&full[b], (uint32_t)(k & 1));
        if (group_any<1>(!ok)) {
            if (ct == 0) atomicOr(status, 4ull);
            break;
        }
        const int tl = u >> LTPT;
        const int q0 = (u & ((1 << LTPT) - 1)) << LNP;
        pass2_tile<LR, LC, LNP, SyncNamed<1, kP2Consumers>, true>(stg + b * kP2Tile, tl, q0, p, tw, P, sm,
                                                                  s_wq, ct);
        SyncNamed<1, kP2Consumers>::sync();  // the work tile and s_wq are free for the next tile
        __syncwarp();
        if ((ct & 31) == 0) mbar_arrive(&empty[b]);
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

// padded tile plus the pass-2 line skew (at most 32 complex in total)
size_t tile_smem(int logt) { return (size_t)(((1 << logt) + ((1 << logt) >> 4) + 64) * sizeof(float2)); }

// Compile-time geometries of the two passes for 2^20..2^25 samples at pass-1 tiles 2^13 /
// 2^14 and pass-2 tiles 2^12 / 2^13 / 2^14, with the library's four-step split and, for
// 2^23 and 2^24, the split with twice the row length (other plans use the <-1, -1, -1>
// kernels).
using Pass1Fn = void (*)(SeriesView, const Anchor*, Plan, const float2*, float2*);
using Pass2Fn = void (*)(const float2*, Plan, const float2*, float*);

#define BPS_PASS1_GEOMETRIES(X) \
    X(9, 10, 5) X(9, 10, 4) \
    X(10, 10, 4) X(10, 10, 3) X(11, 10, 3) X(11, 10, 2) X(12, 10, 2) X(12, 10, 1) X(12, 11, 2) \
    X(12, 11, 1) X(12, 12, 2) X(12, 12, 1) X(11, 11, 3) X(11, 11, 2) X(11, 12, 3) X(11, 12, 2) \
    X(-1, -1, -1)
#define BPS_PASS2_GEOMETRIES(X) \
    X(9, 10, 2) X(9, 10, 3) X(9, 10, 1) X(10, 10, 1) X(11, 10, 1) X(12, 10, 1) X(12, 11, 0) X(11, 11, 0) \
    X(10, 10, 2) X(10, 10, 3) X(11, 10, 2) X(11, 10, 3) X(12, 10, 2) X(12, 10, 3) X(12, 11, 1) \
    X(12, 11, 2) X(12, 12, 0) X(12, 12, 1) X(11, 11, 1) X(11, 11, 2) X(11, 12, 0) X(11, 12, 1) \
    X(-1, -1, -1)

Pass1Fn pick_pass1(const Plan& p, bool f16)
{
#define BPS_PICK(a, b, c)                                                  \
    if ((a < 0) || (p.logR == a && p.logC == b && p.logG == c))            \
        return f16 ? k_pass1<a, b, c, true> : k_pass1<a, b, c, false>;
    BPS_PASS1_GEOMETRIES(BPS_PICK)
#undef BPS_PICK
    return f16 ? k_pass1<-1, -1, -1, true> : k_pass1<-1, -1, -1, false>;
}

Pass2Fn pick_pass2(const Plan& p)
{
#define BPS_PICK(a, b, c) \
    if ((a < 0) || (p.logR == a && p.logC == b && p.logNP == c)) return k_pass2<a, b, c>;
    BPS_PASS2_GEOMETRIES(BPS_PICK)
#undef BPS_PICK
    return k_pass2<-1, -1, -1>;
}

}  // namespace

namespace {
cudaError_t ws_attributes(int* nsm);
cudaError_t p2tma_attributes(int* nsm);
cudaError_t async_attributes();
}

// Large dynamic shared memory for the FFT passes, set once per device (a host-side
// function attribute, so it is also safe to call while a stream is being captured).
cudaError_t set_smem_attributes()
{
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) return e != cudaSuccess ? e : cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return cudaSuccess;
    const int bytes = (int)tile_smem(kLogTile);
#define BPS_ATTR(a, b, c)                                                                               \
    if (e == cudaSuccess)                                                                                \
        e = cudaFuncSetAttribute(k_pass1<a, b, c, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes); \
    if (e == cudaSuccess)                                                                                \
        e = cudaFuncSetAttribute(k_pass1<a, b, c, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    BPS_PASS1_GEOMETRIES(BPS_ATTR)
#undef BPS_ATTR
#define BPS_ATTR(a, b, c) \
    if (e == cudaSuccess)  \
        e = cudaFuncSetAttribute(k_pass2<a, b, c>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    BPS_PASS2_GEOMETRIES(BPS_ATTR)
#undef BPS_ATTR
    int nsm = 0;
    if (e == cudaSuccess) e = ws_attributes(&nsm);
    if (e == cudaSuccess) e = p2tma_attributes(&nsm);
    if (e == cudaSuccess) e = async_attributes();
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

cudaError_t launch_twiddle_init(float2* tw, cudaStream_t s)
{
    k_twiddle_init<<<kTwiddleN / 256, 256, 0, s>>>(tw);
    return cudaGetLastError();
}

namespace {

using WsFn = void (*)(SeriesView, const Anchor*, Plan, const float2*, float2*, int, unsigned long long*);

// (log R, log C) of the warp-specialised pass 1: 2^20..2^24 complex points, R = 2^10..2^12
#define BPS_WS_GEOMETRIES(X)                                                                          X(10, 10) X(11, 9) X(12, 8) X(10, 11) X(11, 10) X(12, 9) X(10, 12) X(11, 11) X(12, 10)            X(11, 12) X(12, 11) X(12, 12)

WsFn pick_ws(const Plan& p)
{
#define BPS_PICK(a, b) \
    if (p.logR == a && p.logC == b) return k_pass1_ws<a, b>;
    BPS_WS_GEOMETRIES(BPS_PICK)
#undef BPS_PICK
    return nullptr;
}

cudaError_t ws_attributes(int* nsm)
{
    static std::mutex mu;
    static int done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!done[dev]) {
        const int bytes = (int)ws_pass1_smem();
#define BPS_ATTR(a, b) \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pass1_ws<a, b>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        BPS_WS_GEOMETRIES(BPS_ATTR)
#undef BPS_ATTR
        int n = 0;
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        done[dev] = n;
    }
    *nsm = done[dev];
    return cudaSuccess;
}

}  // namespace

namespace {

using AsyncFn = void (*)(SeriesView, const Anchor*, Plan, const float2*, float2*);

AsyncFn pick_async(const Plan& p)
{
#define BPS_PICK(a, b) \
    if (p.logR == a && p.logC == b) return k_pass1_async<a, b>;
    BPS_WS_GEOMETRIES(BPS_PICK)
#undef BPS_PICK
    return nullptr;
}

size_t async_smem() { return (size_t)(kWsBufStride + 272) * sizeof(float2); }

cudaError_t async_attributes()
{
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!done[dev]) {
        const int bytes = (int)async_smem();
#define BPS_ATTR(a, b) \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pass1_async<a, b>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        BPS_WS_GEOMETRIES(BPS_ATTR)
#undef BPS_ATTR
        if (e != cudaSuccess) return e;
        done[dev] = true;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_pass1(const SeriesView& x, const Anchor* anc, int nt, const Plan& p,
                         const float2* tw, float2* Y, unsigned long long* status, cudaStream_t s)
{
    if (p.p1async && x.f32 && x.fillp) {
        const AsyncFn f = pick_async(p);
        if (!f) return cudaErrorInvalidValue;
        cudaError_t e = async_attributes();
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)(1 << (p.logC - (13 - p.logR))), (unsigned)nt);
        f<<<grid, 512, async_smem(), s>>>(x, anc, p, tw, Y);
        return cudaGetLastError();
    }
    if (p.p1ws) {
        const WsFn f = pick_ws(p);
        if (!f || !status) return cudaErrorInvalidValue;
        int nsm = 0;
        cudaError_t e = ws_attributes(&nsm);
        if (e != cudaSuccess) return e;
        const int64_t ntiles = (int64_t)nt << (p.logC - (kWsLogTile - p.logR));
        if (ntiles < 1 || ntiles > INT32_MAX) return cudaErrorInvalidValue;
        const int grid = (int)std::min<int64_t>(ntiles, nsm);
        f<<<grid, kWsThreads, ws_pass1_smem(), s>>>(x, anc, p, tw, Y, (int)ntiles, status);
        return cudaGetLastError();
    }
    const int logt = p.logR + p.logG;
    cudaError_t e = set_smem_attributes();
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(1 << (p.logC - p.logG)), (unsigned)nt);
    pick_pass1(p, x.f16 != nullptr)<<<grid, (1 << logt) / kEPT, tile_smem(logt), s>>>(x, anc, p, tw, Y);
    return cudaGetLastError();
}

namespace {

using P2TmaFn = void (*)(const float2*, Plan, const float2*, float*, int, unsigned long long*);

// (log R, log C) of the TMA-fed pass 2 (2^13-complex tiles: NP = 2^12 / C row pairs)
#define BPS_P2TMA_GEOMETRIES(X) \
    X(10, 10) X(11, 10) X(12, 10) X(10, 11) X(11, 11) X(12, 11) X(10, 12) X(11, 12) X(12, 12)

P2TmaFn pick_p2tma(const Plan& p)
{
#define BPS_PICK(a, b) \
    if (p.logR == a && p.logC == b) return k_pass2_tma<a, b, 12 - b>;
    BPS_P2TMA_GEOMETRIES(BPS_PICK)
#undef BPS_PICK
    return nullptr;
}

cudaError_t p2tma_attributes(int* nsm)
{
    static std::mutex mu;
    static int done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!done[dev]) {
        const int bytes = (int)p2tma_smem();
#define BPS_ATTR(a, b) \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pass2_tma<a, b, 12 - b>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        BPS_P2TMA_GEOMETRIES(BPS_ATTR)
#undef BPS_ATTR
        int n = 0;
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        done[dev] = n;
    }
    *nsm = done[dev];
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_pass2(const float2* Y, int nt, const Plan& p, const float2* tw, float* P,
                         unsigned long long* status, cudaStream_t s)
{
    if (p.p2tma) {
        const P2TmaFn f = pick_p2tma(p);
        if (!f || !status || p.logTile2 != 13) return cudaErrorInvalidValue;
        int nsm = 0;
        cudaError_t e = p2tma_attributes(&nsm);
        if (e != cudaSuccess) return e;
        const int64_t ntiles = (int64_t)nt << (p.logR - 1 - p.logNP);
        if (ntiles < 1 || ntiles > INT32_MAX) return cudaErrorInvalidValue;
        const int grid = (int)std::min<int64_t>(ntiles, nsm);
        f<<<grid, kP2Threads, p2tma_smem(), s>>>(Y, p, tw, P, (int)ntiles, status);
        return cudaGetLastError();
    }
    const int logt = p.logNP + 1 + p.logC;
    cudaError_t e = set_smem_attributes();
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(1 << (p.logR - 1 - p.logNP)), (unsigned)nt);
    pick_pass2(p)<<<grid, (1 << logt) / kEPT2, tile_smem(logt), s>>>(Y, p, tw, P);
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
