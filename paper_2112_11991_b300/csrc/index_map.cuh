// index_map.cuh -- per-sample evaluation of the nearest-neighbour demodulation
// index map of Algorithm 1 (App. A.1) from FP64-derived anchor constants.
//
//   off(m) = (Delta_R(0) - Delta_R(m t_s)) / t_s ,   idx(m) = m + floor(off(m) + 1/2)
//
// Around an anchor centre c the offset is off(c + d) = I + f - inc(d).  The fast
// path evaluates inc(d) ~ L d + q2 d^2 + q3 d^3 in FP32; when the fractional part
// of off + 1/2 lies within GUARD of an integer it falls back to the precise
// path, which keeps the linear term exact (FMA product error, TwoSum) and solves
// Kepler's equation for the eccentric-anomaly increment
//   u - e sinE_c (cos u - 1) - e cosE_c sin u = Omega t_s d
// in FP32 (the increment is small, so FP32 gives ~1e-7 sample absolute error).
#pragma once

#include <cuda_fp16.h>

#include "bps_internal.cuh"

namespace bps {

constexpr float kGuard = 1e-4f;

// Round-to-nearest by the 1.5 * 2^23 shift: for |x| < 2^22, y = x + kRoundShift holds
// rint(x) in its low mantissa bits, so rint(x) = y - kRoundShift (exact) and, as an
// integer, __float_as_int(y) - kRoundBits.
constexpr float kRoundShift = 12582912.0f;
constexpr int kRoundBits = 0x4B400000;

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Exact-rounding evaluation of floor(off + 1/2) - I for anchor a at offset d.
static __device__ __noinline__ int off_round_precise(const Anchor& a, int d)
{
    const float df = (float)d;
    const float p = __fmul_rn(a.Lhi, df);
    const float perr = __fmaf_rn(a.Lhi, df, -p);  // Lhi*df = p + perr exactly
    const float u1 = __fmul_rn(a.g, df);            // linear eccentric-anomaly step
    float eps = 0.f, cm1 = 0.f, smu = 0.f;
#pragma unroll
    for (int it = 0; it < 3; ++it) {
        const float u = u1 + eps;
        const float u2 = u * u;
        cm1 = u2 * (-0.5f + u2 * (1.f / 24.f - u2 * (1.f / 720.f)));  // cos u - 1
        smu = u * u2 * (-1.f / 6.f + u2 * (1.f / 120.f));              // sin u - u
        eps = (a.esE * cm1 + a.ecE * smu) * a.invD;
    }
    {
        const float u = u1 + eps;
        const float u2 = u * u;
        cm1 = u2 * (-0.5f + u2 * (1.f / 24.f - u2 * (1.f / 720.f)));
        smu = u * u2 * (-1.f / 6.f + u2 * (1.f / 120.f));
    }
    // R = inc - L d = K[Bc (sin u - u1) + Ac (cos u - 1)],  sin u - u1 = eps + (sin u - u)
    const float R = a.KBc * (eps + smu) + a.KAc * cm1;
    float s, e1, s2, e2;
    two_sum(a.fhi, -p, s, e1);
    two_sum(s, 0.5f, s2, e2);
    const float c = __fsub_rn(__fadd_rn(__fadd_rn(e1, e2), a.flo),
                              __fadd_rn(__fmaf_rn(a.Llo, df, perr), R));
    const float fl = floorf(s2);
    const float v = __fadd_rn(__fsub_rn(s2, fl), c);
    return (int)fl + (int)floorf(v);
}

// floor(off + 1/2) - I; *precise set when the compensated branch was taken.  Fast
// path: xr = off - I - 1/2 in FP32; outside the guard band floor(xr + 1/2) = rint(xr)
// (ties lie inside the band), taken by the shift of kRoundShift.
__device__ __forceinline__ int off_round(const Anchor& a, int d, bool& precise)
{
    const float df = (float)d;
    const float xr = a.fhi - df * fmaf(df, fmaf(df, a.q3, a.q2), a.Lhi);
    const float y = __fadd_rn(xr, kRoundShift);
    const float fr = __fsub_rn(xr, __fsub_rn(y, kRoundShift));
    if (fabsf(fr) < 0.5f - kGuard) {
        precise = false;
        return __float_as_int(y) - kRoundBits;
    }
    precise = true;
    return off_round_precise(a, d);
}

// Anchor index and centre of sample m.
__device__ __forceinline__ int64_t anchor_of(int64_t m, int logB) { return m >> logB; }
__device__ __forceinline__ int64_t anchor_centre(int64_t b, int logB)
{
    return (b << logB) + (1ll << (logB - 1));
}

// Fast-path fields only (first 16 bytes + q3/flo/Llo/g in the second 16).
__device__ __forceinline__ Anchor load_anchor(const Anchor* __restrict__ anc, int64_t b)
{
    return anc[b];
}

// Kernels that gather call this once at entry: the fill value comes from the device copy
// when there is one (series updated in place, graphs), so the gathers below read a register.
__device__ __forceinline__ void resolve_fill(SeriesView& x)
{
    if (x.fillp) x.fill = __ldg(x.fillp);
    x.uscale = x.uscalep ? __ldg(x.uscalep) : 0.f;
}

// Gathered sample x[idx] (the series mean outside [0, n)), FP32 or FP16+scale.
__device__ __forceinline__ float gather_sample(const SeriesView& x, int n, int idx)
{
    if ((unsigned)idx >= (unsigned)n) return x.fill;
    if (x.f32) return __ldg(x.f32 + idx);
    const __half h = __ushort_as_half(__ldg(x.f16 + idx));
    return __half2float(h) * __ldg(x.scale + (idx >> 12));
}

// Two gathered FP32 samples x[i0], x[i1] (the series mean outside [0, n)).
__device__ __forceinline__ float2 gather_pair_f32(const SeriesView& x, int n, int i0, int i1)
{
    return make_float2((unsigned)i0 < (unsigned)n ? __ldg(x.f32 + i0) : x.fill,
                       (unsigned)i1 < (unsigned)n ? __ldg(x.f32 + i1) : x.fill);
}

// The 32 FP16 samples of a first-stage butterfly (pairs id[2s], id[2s+1] -> v[s]): every
// load first (the halves and their block scales), then the conversions, so all the
// loads are in flight together (converting each value as it arrives serialised them).
__device__ __forceinline__ void gather_f16_butterfly(const SeriesView& x, int n, const int (&id)[32],
                                                     float2 (&v)[16])
{
    unsigned short hv[32];
    float sv[32];
    if (x.uscale > 0.f) {  // all blocks share one scale: no per-sample scale loads
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            const int i = id[q];
            hv[q] = (unsigned)i < (unsigned)n ? __ldg(x.f16 + i) : (unsigned short)0;
            sv[q] = x.uscale;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            const int i = id[q];
            const bool in = (unsigned)i < (unsigned)n;
            hv[q] = in ? __ldg(x.f16 + i) : (unsigned short)0;
            sv[q] = in ? __ldg(x.scale + (i >> 12)) : 0.f;
        }
    }
#pragma unroll
    for (int s = 0; s < 16; ++s) {
        const bool in0 = (unsigned)id[2 * s] < (unsigned)n, in1 = (unsigned)id[2 * s + 1] < (unsigned)n;
        v[s] = make_float2(in0 ? __half2float(__ushort_as_half(hv[2 * s])) * sv[2 * s] : x.fill,
                           in1 ? __half2float(__ushort_as_half(hv[2 * s + 1])) * sv[2 * s + 1] : x.fill);
    }
}

}  // namespace bps
