// bps_internal.cuh -- device data layouts and launcher declarations shared by the
// CUDA translation units of libbps (never by the FP64 oracle).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bps {

// One orbital template on the device (App. A, BT model): the public bps_template's five
// parameters followed by per-template constants of the anchor kernel, computed once on the
// host in FP64 (dev_template in bps_runtime.h): Omega = 2 pi / P_orb, sin and cos of the
// periastron longitude, sqrt(1 - e^2), and the zero offset's delay Delta_R(0) (Kepler's
// equation at M = alpha; Algorithm 1 subtracts it so that idx_0 = 0).
struct DevTemplate {
    double porb, tau, phi, omega, ecc;
    double om, sw, cw, rt, delta0;
};

// Per-anchor constants of the index map (Algorithm 1), evaluated in FP64 at the
// anchor centre c = b*B + B/2 and rounded to FP32.  For d = m - c the offset is
//   off(m) = I + f - inc(d),  inc(d) = (Delta_R(t_c + d t_s) - Delta_R(t_c)) / t_s
// with inc(d) = L d + R(d) and, for the fast path, R(d) ~ q2 d^2 + q3 d^3.
// Field order: the fast path reads only the first 16 + 4 bytes.
struct __align__(16) Anchor {
    int   I;     // floor(O_c), O_c = (Delta_R(0) - Delta_R(t_c)) / t_s
    float fhi;   // O_c - I, high part
    float Lhi;   // d inc / d d at d = 0, high part  [samples / sample]
    float q2;    // (1/2) d^2 inc / dd^2
    float q3;    // (1/6) d^3 inc / dd^3
    float flo;   // low part of O_c - I
    float Llo;   // low part of L
    float g;     // dE/dd = Omega t_s / (1 - e cos E_c)
    float esE;   // e sin E_c
    float ecE;   // e cos E_c
    float invD;  // 1 / (1 - e cos E_c)
    float KBc;   // (tau/t_s) * dBT/dE at E_c
    float KAc;   // (tau/t_s) * (cos E_c sin w + sqrt(1-e^2) sin E_c cos w)
    float pad0, pad1, pad2;
};
static_assert(sizeof(Anchor) == 64, "Anchor must be 64 bytes");

// Problem geometry of one search (host-built, passed by value to kernels).
// Row-major power layout of pass 2 (plan.ptrans): columns k2 in blocks of 2^kLogPowCols,
// rows k1 in groups of NP; bin k1 + R k2 at
//   P'[(k2 div 8) 8 R + (k1 div NP) 8 NP + (k2 mod 8) NP + k1 mod NP]
// so the 8 columns x W rows of whitening blocks the median kernel takes are contiguous.
constexpr int kLogPowCols = 3;

struct Plan {
    int64_t n;      // real samples N (power of two)
    int64_t M;      // N/2 complex points of the packed FFT
    int logn, logM;
    int logR, logC; // M = R * C (four-step: R-point column FFTs, C-point row FFTs)
    int logG;       // columns per CTA in pass 1
    int logNP;      // row pairs per CTA in pass 2
    int logTile;    // complex values per CTA tile of pass 1 (13 or 14)
    int logTile2;   // complex values per CTA tile of pass 2 (12, 13 or 14)
    int logB;       // anchor block length B (samples)
    int64_t nanchor;// N / B
    int logW;       // whitening block W (bins)
    int nharm;      // nharm_max (power of two <= 16)
    int lognh;
    int nlev;       // log2(nharm) + 1
    int ptrans;     // 1: pass 2 writes the power row-major by k1, P'[k1 C + k2] for bin
                    // k1 + R k2, and the median kernel transposes it into bin order
    int p1ws;       // 1: warp-specialised pass 1 (producer warps gather, consumer warps FFT)
    int p1async;    // 1: pass 1 with cp.async gathers, 2^13 tiles, two CTAs per SM (FP32
                    // series with a device fill value; the one-phase kernel otherwise)
    int p2tma;      // 1: pass 2 fed by TMA bulk copies of its rows (persistent, 2^13 tiles)
    double tsamp;
    double inv_tsamp;  // 1 / tsamp
};

// Four-step splits (log R, log C) the warp-specialised pass 1 is built for (2^13-complex
// tiles of 2^(13 - log R) columns).
inline bool ws_pass1_built(int logR, int logC)
{
    const int lm = logR + logC;
    return (logR == 10 || logR == 11 || logR == 12) && logC >= 13 - logR && lm >= 20 && lm <= 24 &&
           logC <= 12;
}

// Four-step split of the packed FFT, M = R * C, with CTA tiles of 2^logTile (pass 1)
// and 2^logTile2 (pass 2) complex values in shared memory (pass 1 at 32 elements per
// thread: 2^13 = 256 threads, two CTAs per SM, 2^14 = 512, one; pass 2 at 16: 2^12 = 256
// threads, four CTAs per SM, 2^13 two, 2^14 one): C = 2^min(10, logM - 5) row length (pass 2), raised
// to M / 2^12 where R would exceed 2^12 column length (pass 1), unless logCols (checked
// by log_cols_ok) chooses another split; G = tile1 / R adjacent columns per pass-1 CTA,
// NP = tile2 / (2C) row pairs per pass-2 CTA.
inline int default_log_cols(int logM)
{
    int lc = logM - 5 < 10 ? logM - 5 : 10;
    if (logM - lc > 12) lc = logM - 12;
    return lc;
}

// Valid four-step splits: C >= 32, R >= 32, R <= 2^12, C <= 2^12 (pass 2's split
// twiddles W_{2C}^k come from the 8192-entry table).
inline bool log_cols_ok(int logM, int lc)
{
    return lc >= 5 && lc >= logM - 12 && lc <= logM - 5 && lc <= 12;
}

inline void plan_geometry(Plan& p, int logTile = 14, int logTile2 = 13, int logCols = 0)
{
    p.logTile = logTile;
    p.logTile2 = logTile2;
    p.logC = logCols ? logCols : default_log_cols(p.logM);
    p.logR = p.logM - p.logC;
    const int lt = logTile > p.logR ? logTile : p.logR;  // a column must fit one tile
    p.logG = p.logC < lt - p.logR ? p.logC : lt - p.logR;
    p.logNP = (logTile2 - 1 - p.logC) < (p.logR - 1) ? (logTile2 - 1 - p.logC) : (p.logR - 1);
    if (p.logNP < 0) p.logNP = 0;
    p.ptrans = 0;
    p.p1ws = 0;
    p.p1async = 0;
    p.p2tma = 0;
}

// Four-step splits the TMA-fed pass 2 is built for (2^13-complex tiles).
inline bool tma_pass2_built(int logR, int logC, int logTile2)
{
    return logTile2 == 13 && logR >= 10 && logR <= 12 && logC >= 10 && logC <= 12;
}

// Anchor block length B = 2^logB: the largest (<= 2^14, <= n/16) for which every
// template keeps the FP32 fast path of the index map far inside its 1e-4 guard:
// |linear increment| <= 128 samples, quadratic term <= 0.25 sample, quartic
// remainder <= 1e-5 sample, with h = B/2 the largest distance to the anchor centre.
// kg1, kg2, kg4 are the bank maxima of K g, K g^2, K g^4 (K = tau / t_s,
// g = Omega t_s / (1 - e)).  Returns -1 when even B = 64 does not qualify.
inline int plan_anchor_block(double kg1, double kg2, double kg4, int logn)
{
    // B <= N/16 as well: the 16 rows of a pass-1 butterfly (N/16 samples apart) then sit at
    // the same offset from their anchor centres
    int logB = logn - 4 < 14 ? logn - 4 : 14;
    for (; logB >= 6; --logB) {
        const double h = (double)(1 << (logB - 1));
        if (kg1 * h <= 128.0 && kg2 * h * h <= 0.25 && kg4 * h * h * h * h <= 1e-5) return logB;
    }
    return -1;
}

// Thresholds of the harmonic levels, by value.
struct Thr {
    float v[5];
};

// Candidate record: same layout as the public bps_candidate.
struct Cand {
    uint32_t tidx;
    uint16_t nharm;
    uint16_t flags;
    uint32_t bin;
    float power;
};

// Series storage descriptor.
struct SeriesView {
    const float* f32;          // FP32 samples (or nullptr)
    const uint16_t* f16;       // FP16 samples (or nullptr)
    const float* scale;        // per-4096-sample scale for FP16; scale[n_blocks] holds the
                               // common scale when all blocks share one, else 0
    float fill;                // mean of the series (value for out-of-range samples)
    const float* fillp;        // device copy of the fill value (used when non-null)
    const float* uscalep;      // &scale[n_blocks] (FP16; nullptr otherwise)
    float uscale;              // *uscalep, read at kernel entry (0: per-block scales)
};

// Launchers (stream-ordered, return cudaGetLastError()).
// tw[t] = exp(-2 pi i t / kTwiddleN), t in [0, kTwiddleN): covers every FFT length <= 8192
constexpr int kTwiddleN = 8192;
cudaError_t launch_twiddle_init(float2* tw, cudaStream_t s);
cudaError_t launch_anchors(const DevTemplate* bank, int64_t t0, int nt, const Plan& p,
                           Anchor* out, cudaStream_t s);
cudaError_t launch_index_map(const Anchor* anc, const Plan& p, int32_t* idx,
                             unsigned long long* n_precise, cudaStream_t s);
cudaError_t launch_resample(const SeriesView& x, const Anchor* anc, int nt, const Plan& p,
                            float* out, cudaStream_t s);
cudaError_t set_smem_attributes();
// Function attributes and occupancy of the median and harmonic-sum kernels, once per
// device (host-side only; called before a graph capture so none happens during one).
cudaError_t prepare_detect_kernels();
// One CTA polls an mbarrier that never completes at most `limit` times; status[0] = 1
// when the wait expired (the bounded-wait path of the harmonic sum, exercised safely).
cudaError_t launch_wait_selftest(int limit, unsigned long long* status, cudaStream_t s);
// status: a device word of the request; the warp-specialised form sets bit 1 when one of
// its bounded mbarrier waits expired (unused by the one-phase form)
cudaError_t launch_pass1(const SeriesView& x, const Anchor* anc, int nt, const Plan& p,
                         const float2* tw, float2* Y, unsigned long long* status, cudaStream_t s);
// status: as launch_pass1 (the TMA-fed form sets bit 2 when a bounded wait expired)
cudaError_t launch_pass2(const float2* Y, int nt, const Plan& p, const float2* tw,
                         float* P, unsigned long long* status, cudaStream_t s);
cudaError_t launch_power_from_r2c(const float2* X, int nt, const Plan& p, float* P,
                                  cudaStream_t s);
// Lower median of each block of W bins and whitening into P (bin order; scale receives
// ln2/med per block).  With p.ptrans the power is read from Pt (pass 2's
// row-major-by-k1 layout) and the kernel transposes it; otherwise P is whitened in
// place (Pt unused).
cudaError_t launch_block_median(float* P, int nt, const Plan& p, float* scale,
                                cudaStream_t s, const float* Pt = nullptr);
// copies the whitened spectrum left by launch_block_median (scale unused)
cudaError_t launch_whitened(const float* P, const float* scale, int nt, const Plan& p,
                            float* out, cudaStream_t s);
// P holds the whitened spectrum (after launch_block_median); scale unused.  count[0]
// is the candidate counter, count[1] a status word (bit 0: a bounded wait of the harmonic sum
// expired; bits 1 and 2 are set by the producer/consumer forms of passes 1 and 2).
// tile_ctr: a device word the launch zeroes and the CTAs take tiles from.
cudaError_t launch_harmsum(const float* P, const float* scale, int nt, int64_t tidx0,
                           const Plan& p, const Thr& thr, Cand* cands, int64_t cap,
                           unsigned long long* count, float* s_out, unsigned int* tile_ctr,
                           cudaStream_t s);
cudaError_t launch_series_stats(const float* x, int64_t n, double* sum, cudaStream_t s);
// fill = (float)(sum / n) on the device
cudaError_t launch_fill_from_sum(const double* sum, int64_t n, float* fill, cudaStream_t s);
// FP16 packing with a power-of-two scale per 4096 samples; scale needs n_blocks + 1
// floats (the last receives the common scale, or 0)
cudaError_t launch_f16_pack(const float* x, int64_t n, uint16_t* h, float* scale,
                            cudaStream_t s);

}  // namespace bps
