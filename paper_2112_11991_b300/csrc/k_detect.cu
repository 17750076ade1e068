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
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "bps_internal.cuh"
#include "mbar.cuh"

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

// Exact lower median (element of rank floor((W-1)/2), W = 32*VPL) of the FP32 values
// held by one warp, VPL per lane: radix select on the bit pattern (values >= 0: sign bit
// 0) with the warp's padded 288-word shared histogram h (bin b at b + b/8: conflict-free
// scan reads) and a warp prefix scan, no block barrier.  Digits: exponent [30:23],
// mantissa [22:15], [14:7], [6:0].  The values left after the first two share the
// median's top 16 bits (a relative width of 2^-8: one or two of 1024 for noise power);
// when at most 32 are left they are gathered into h by ballot and each lane ranks its
// own against them (ties counted, so the element of the remaining rank is found
// exactly) instead of the last two digits.  Returns the median's bits.
template <int VPL>
__device__ __forceinline__ uint32_t warp_lower_median(const uint32_t (&u)[VPL], uint32_t* h, int lane)
{
    uint32_t prefix = 0, pmask = 0, rank = (uint32_t)(32 * VPL - 1) / 2;
#pragma unroll
    for (int pass = 0; pass < 4; ++pass) {
        if (pass == 2) {
            const uint32_t lt = (1u << lane) - 1u;
            uint32_t m = 0;
#pragma unroll
            for (int i = 0; i < VPL; ++i) {
                const bool c = (u[i] & pmask) == prefix;
                const uint32_t b = __ballot_sync(0xffffffffu, c);
                if (b) {
                    const uint32_t pos = m + __popc(b & lt);
                    if (c && pos < 32u) h[pos] = u[i];
                    m += __popc(b);
                }
            }
            __syncwarp();
            if (m <= 32u) {
                const uint32_t mine = (uint32_t)lane < m ? h[lane] : 0xffffffffu;
                uint32_t less = 0, eq = 0;
                for (uint32_t j = 0; j < m; ++j) {
                    const uint32_t o = h[j];
                    less += (o < mine) ? 1u : 0u;
                    eq += (o == mine) ? 1u : 0u;
                }
                const bool own = (uint32_t)lane < m && less <= rank && rank < less + eq;
                const int owner = __ffs(__ballot_sync(0xffffffffu, own)) - 1;
                const uint32_t med = __shfl_sync(0xffffffffu, mine, owner);
                __syncwarp();
                return med;
            }
        }
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
    return prefix;
}

// One warp per block of W = 32*VPL bins (bin order), values in registers; the block is
// whitened in place: Pw = P * ln2 / med (0 when med = 0).
template <int VPL>
__global__ void __launch_bounds__(256, 4) k_median_warp(float* __restrict__ P, Plan p,
                                                     float* __restrict__ scale)
{
    __shared__ uint32_t hist[8][288];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tl = blockIdx.y;
    const int64_t nblk = p.M >> p.logW;
    const int64_t blk = (int64_t)blockIdx.x * 8 + warp;
    if (blk >= nblk) return;
    float* src = P + (int64_t)tl * p.M + (blk << p.logW);
    uint32_t u[VPL];
#pragma unroll
    for (int i = 0; i < VPL; ++i) u[i] = __float_as_uint(src[lane + 32 * i]);
    const float med = __uint_as_float(warp_lower_median<VPL>(u, hist[warp], lane));
    const float sc = (med > 0.f) ? kLn2 / med : 0.f;
#pragma unroll
    for (int i = 0; i < VPL; ++i) src[lane + 32 * i] = __uint_as_float(u[i]) * sc;
    if (lane == 0) scale[(int64_t)tl * nblk + blk] = sc;
}

// The same from pass 2's row-major power (kLogPowCols: columns in blocks of 8, rows in
// groups of T = NP = 2^LOGT, T <= 2, W <= R): a CTA of kMedCols = 8 warps takes the 8
// blocks at k2 in [k20, k20 + 8), k1 in [q0, q0 + W) -- one contiguous run of 32 W bytes
// -- into a column-major shared tile (column c = block k20 + c, stride W + 4 words); warp
// w takes the median of column w (consecutive words: conflict-free) and writes its
// whitened block to P in bin order.  A float4 of the run holds T rows of 4 / T columns;
// with T = 2 its elements are two pairs of rows adjacent in the tile, written as two 8-byte
// stores.  The stride's 4 words of padding spread the stores over all banks (two
// wavefronts per 8-byte store instruction, one per 4-byte one; a row-major tile padded to
// 9 words a row had two-way conflicts on every 4-byte store).  (Measured at C = 2048 and
// 4096: 8 columns with four CTAs per SM beat 16 with two, whose 16 warps need more than 64
// registers with the candidate gather of the median.)
constexpr int kMedCols = 8;
constexpr int kLogMedCols = 3;
constexpr int kMedPad = 4;
static_assert(kLogMedCols == kLogPowCols, "the median CTA takes one column block");

template <int VPL, int LOGT>
__global__ void __launch_bounds__(32 * kMedCols) k_median_warp_t(const float* __restrict__ Pt, Plan p,
                                                                   float* __restrict__ P,
                                                                   float* __restrict__ scale)
{
    static_assert(LOGT == 0 || LOGT == 1, "rows in groups of one or two");
    constexpr int W = 32 * VPL;
    constexpr int CS = W + kMedPad;  // tile column stride (words)
    extern __shared__ __align__(16) uint32_t tsm[];
    uint32_t* tile = tsm;                   // kMedCols columns of W words
    uint32_t* hist = tsm + kMedCols * CS;   // kMedCols x 288
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tl = blockIdx.y;
    const int lg = p.logC - kLogMedCols;  // groups of kMedCols k2 per row
    const int k20 = (int)(blockIdx.x & ((1u << lg) - 1)) * kMedCols;
    const int qb = (int)(blockIdx.x >> lg);
    const int q0 = qb * W;
    const float* src = Pt + (int64_t)tl * p.M;
    constexpr int LCH = kLogMedCols + LOGT;  // log2 of the floats of one group's kMedCols columns
    const float* g0 = src + ((int64_t)(k20 >> kLogMedCols) << (p.logR + kLogMedCols)) +
                      ((int64_t)(q0 >> LOGT) << LCH);
    // thread t loads float4 t + 256 i: floats f = 4 t + 1024 i, group f / 2^LCH (rows
    // T (f / 2^LCH) + 0..T-1), place o = f mod 2^LCH in it (element o + u: column (o + u) / T,
    // row offset (o + u) mod T).  1024 is a whole number of groups, so o is the same for all
    // of a thread's loads.
    constexpr int FSTEP = 4 * 32 * kMedCols;
    static_assert(FSTEP % (1 << LCH) == 0, "load step is a whole number of groups");
    const int nf4 = (W * kMedCols) / 4;
    const int f0 = 4 * (int)threadIdx.x;
    const int o = f0 & ((1 << LCH) - 1);
#pragma unroll 4
    for (int i = 0; i < (W * kMedCols + FSTEP - 1) / FSTEP; ++i) {
        if ((int)threadIdx.x + i * 32 * kMedCols >= nf4) break;  // W < 128: fewer float4s than threads
        const float4 v = __ldg(reinterpret_cast<const float4*>(g0 + f0 + i * FSTEP));
        const int r0 = ((f0 + i * FSTEP) >> LCH) << LOGT;
        if (LOGT == 1) {
            *reinterpret_cast<uint2*>(tile + (o >> 1) * CS + r0) =
                make_uint2(__float_as_uint(v.x), __float_as_uint(v.y));
            *reinterpret_cast<uint2*>(tile + ((o >> 1) + 1) * CS + r0) =
                make_uint2(__float_as_uint(v.z), __float_as_uint(v.w));
        } else {
            tile[o * CS + r0] = __float_as_uint(v.x);
            tile[(o + 1) * CS + r0] = __float_as_uint(v.y);
            tile[(o + 2) * CS + r0] = __float_as_uint(v.z);
            tile[(o + 3) * CS + r0] = __float_as_uint(v.w);
        }
    }
    __syncthreads();
    uint32_t u[VPL];
#pragma unroll
    for (int i = 0; i < VPL; ++i) u[i] = tile[warp * CS + lane + 32 * i];
    const float med = __uint_as_float(warp_lower_median<VPL>(u, hist + 288 * warp, lane));
    const float sc = (med > 0.f) ? kLn2 / med : 0.f;
    const int64_t nblk = p.M >> p.logW;
    const int64_t blk = ((int64_t)(k20 + warp) << (p.logR - p.logW)) + qb;
    float* dst = P + (int64_t)tl * p.M + (blk << p.logW);
#pragma unroll
    for (int i = 0; i < VPL; ++i) dst[lane + 32 * i] = __uint_as_float(u[i]) * sc;
    if (lane == 0) scale[(int64_t)tl * nblk + blk] = sc;
}

template <int VPL>
constexpr size_t med_t_smem() { return sizeof(uint32_t) * ((size_t)kMedCols * (32 * VPL + kMedPad) + 288 * kMedCols); }


// Self-test of the bounded waits: an mbarrier expecting one arrival that nothing makes,
// so its phase never completes; thread 0 polls it at most `limit` times with the same
// helper the harmonic sum uses and records the outcome (1 = the wait expired).  No copy
// is in flight and nothing faults: the kernel simply returns.
__global__ void k_wait_selftest(int limit, unsigned long long* status)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        status[0] = mbar_wait_parity(&bar, 0u, limit) ? 0ull : 1ull;
    }
}


// Incoherent harmonic sum of the whitened spectrum over tiles of kHsTile = 1024 bins.
// With H = nharm_max the h-th term of bin k is Pw[(k h + H/2) div H].  For a tile
// starting at k0 (a multiple of 1024) and k = k0 + t + 256 q (thread t < 256, q < 4):
//   (k h + H/2) div H = k0 h / H + 256 q h / H + (t h + H/2) div H,
// since k0 h / H and 256 q h / H are whole.  So the terms of h form the segment
// Pw[k0 h / H, k0 h / H + len_h) with len_h independent of k0, the segment's place in
// shared memory is the same for every tile, and a thread's h-th address is a per-thread
// register plus a compile-time offset: 16 shared loads and no index arithmetic per bin.
// Warp-specialised pipeline: one producer warp copies the H segments of a tile into a
// ring of kHsStages stages (16-byte-aligned TMA bulk copies, one per lane, completed on
// the stage's "full" mbarrier); 8 consumer warps sum, threshold and compact, then release
// the stage on its "empty" mbarrier.  CTAs are persistent; the producer takes its tiles
// from a global counter, kHsChunk consecutive ones per claim, claiming the next chunk while
// the current one is copied, and passes each index to the consumers with the stage, so all
// CTAs work on one frontier: a template's whitened spectrum (the segments of a tile reach
// back to bin k h / 16) stays in the L2 while its tiles are summed.  (With a fixed stride
// j = blockIdx.x + i gridDim.x the CTAs drifted apart over a 32-template launch, the
// spectra of several templates were live at once, and 1.7x 2N came from DRAM.)  Two
// stages (70 KB) let three CTAs share an SM: measured at 2^23, 9.9 us per
// template against 10.4 with three stages and two CTAs, 18.2 with four stages and one.
// Every wait is bounded: on expiry the status word is flagged (reported as
// BPS_ERR_TIMEOUT) and the warp leaves after a bounded drain of its copies in flight.
constexpr int kHsTile = 1024;
constexpr int kHsConsumerWarps = 8;
constexpr int kHsThreads = 32 * (kHsConsumerWarps + 1);
constexpr int kHsQN = kHsTile / (32 * kHsConsumerWarps);
constexpr int kHsStages = 2;
constexpr int kHsHeader = 128;  // bytes: full and empty barriers, the stages' tile indices
constexpr int kHsChunk = 4;     // consecutive tiles per claim on the tile counter

template <int NH>
struct HsGeom {
    static constexpr int LOGNH = (NH == 1) ? 0 : (NH == 2) ? 1 : (NH == 4) ? 2 : (NH == 8) ? 3 : 4;
    // segment length (floats, multiple of 4) and offset of harmonic h within a stage
    __host__ __device__ static constexpr int len(int h) { return ((((kHsTile - 1) * h + (NH >> 1)) >> LOGNH) + 4) & ~3; }
    __host__ __device__ static constexpr int off(int h) { return h <= 1 ? 0 : off(h - 1) + len(h - 1); }
    static constexpr int SEG = off(NH + 1);  // floats per stage
    static constexpr uint32_t BYTES = (uint32_t)SEG * 4u;
    static constexpr size_t SMEM = kHsHeader + (size_t)kHsStages * SEG * sizeof(float);
};

template <int NH>
__global__ void __launch_bounds__(kHsThreads, 3) k_harmsum(const float* __restrict__ Pw, Plan p,
                                                        int64_t tidx0, Thr thr,
                                                        Cand* __restrict__ cands, int64_t cap,
                                                        unsigned long long* __restrict__ count,
                                                        float* __restrict__ s_out, int ntiles,
                                                        unsigned int* __restrict__ tile_ctr)
{
    using Gm = HsGeom<NH>;
    constexpr int LOGNH = Gm::LOGNH;
    constexpr int NLEV = LOGNH + 1;
    constexpr int QN = kHsQN;
    constexpr int CT = 32 * kHsConsumerWarps;  // consumer threads
    constexpr int SEG = Gm::SEG;
    extern __shared__ __align__(128) unsigned char hsm[];
    uint64_t* full = reinterpret_cast<uint64_t*>(hsm);
    uint64_t* empty = full + kHsStages;
    volatile int* s_tile = reinterpret_cast<volatile int*>(empty + kHsStages);  // -1: no more tiles
    float* seg = reinterpret_cast<float*>(hsm + kHsHeader);
    const int logtpt = p.logM - 10;  // tiles per template = M / 1024
    const int warp = threadIdx.x >> 5;
    const unsigned lane = threadIdx.x & 31u;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int s = 0; s < kHsStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kHsConsumerWarps);
        }
    }
    __syncthreads();

    if (warp == kHsConsumerWarps) {
        // ---- producer warp: lane h - 1 copies segment h ----
        const int h = (int)lane + 1;
        const bool copier = h <= NH;
        int soff = 0, slen = 0;
#pragma unroll
        for (int hh = 1; hh <= NH; ++hh)
            if (hh == h) soff = Gm::off(hh), slen = Gm::len(hh);
        // tiles come in chunks of kHsChunk consecutive ones; the next chunk is claimed as soon
        // as the current one is, so the atomic's round trip overlaps the chunk's copies
        int jc = 0, jn = 0, sub = 0;
        if (lane == 0) {
            jc = (int)atomicAdd(tile_ctr, (unsigned)kHsChunk);
            jn = (int)atomicAdd(tile_ctr, (unsigned)kHsChunk);
        }
        jc = __shfl_sync(0xffffffffu, jc, 0);
        int i = 0;
        for (;; ++i) {
            const int s = i % kHsStages;
            if (i >= kHsStages &&
                !mbar_wait_parity(&empty[s], (uint32_t)(((i / kHsStages) - 1) & 1))) {
                if (lane == 0) atomicOr(count + 1, 1ull);
                break;
            }
            const int j = jc + sub;
            if (++sub == kHsChunk) {  // move to the claimed chunk, claim the one after it
                sub = 0;
                jc = __shfl_sync(0xffffffffu, jn, 0);
                if (lane == 0 && jc < ntiles) jn = (int)atomicAdd(tile_ctr, (unsigned)kHsChunk);
            }
            if (j >= ntiles) {  // no more tiles: the stage carries the end mark
                if (lane == 0) {
                    s_tile[s] = -1;
                    mbar_arrive(&full[s]);
                }
                ++i;
                break;
            }
            if (lane == 0) s_tile[s] = j;
            const int tl = j >> logtpt;
            const int k0 = (j & ((1 << logtpt) - 1)) << 10;
            if (lane == 0) mbar_expect_tx(&full[s], Gm::BYTES);
            __syncwarp();
            if (copier)
                tma_load_1d(seg + s * SEG + soff, Pw + ((int64_t)tl << p.logM) + ((k0 * h) >> LOGNH),
                            (uint32_t)slen * 4u, &full[s]);
        }
        // let the copies issued last land before the CTA's shared memory can go away
        for (int m = (i > kHsStages ? i - kHsStages : 0); m < i; ++m)
            (void)mbar_wait_parity(&full[m % kHsStages], (uint32_t)((m / kHsStages) & 1));
        return;
    }

    // ---- consumer warps: thread t sums bins k0 + t + 256 q ----
    const int t = (int)threadIdx.x;
    uint32_t addr[NH];  // shared address of term h of bin k0 + t in stage 0
#pragma unroll
    for (int h = 1; h <= NH; ++h)
        addr[h - 1] = smem_u32(seg) + 4u * (uint32_t)(Gm::off(h) + ((t * h + (NH >> 1)) >> LOGNH));
    for (int i0 = 0;; i0 += kHsStages) {
#pragma unroll
        for (int s = 0; s < kHsStages; ++s) {
            const int i = i0 + s;
            if (!mbar_wait_parity(&full[s], (uint32_t)((i / kHsStages) & 1))) {
                if (lane == 0) atomicOr(count + 1, 1ull);
                return;
            }
            const int j = s_tile[s];  // written before the producer's arrival on full[s]
            if (j < 0) return;
            float acc[QN];
            float S[QN][NLEV];
#pragma unroll
            for (int L = 0; L < NLEV; ++L) {
                const int step = NH >> L;
#pragma unroll
                for (int h = step; h <= NH; h += 2 * step) {
#pragma unroll
                    for (int q = 0; q < QN; ++q) {
                        float f;
                        asm volatile("ld.shared.f32 %0, [%1];"
                                     : "=f"(f)
                                     : "r"(addr[h - 1] + 4u * (uint32_t)(s * SEG + ((CT * q * h) >> LOGNH))));
                        acc[q] = (L == 0) ? f : acc[q] + f;
                    }
                }
#pragma unroll
                for (int q = 0; q < QN; ++q) S[q][L] = acc[q];
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);  // stage s may be refilled
            const int tl = j >> logtpt;
            const int kk = ((j & ((1 << logtpt) - 1)) << 10) + t;
            if (s_out) {
#pragma unroll
                for (int q = 0; q < QN; ++q) {
                    const int k = kk + CT * q;
#pragma unroll
                    for (int L = 0; L < NLEV; ++L)
                        s_out[((int64_t)tl * NLEV + L) * p.M + k] = (k >= 1) ? S[q][L] : 0.f;
                }
            }
            bool any = false;
#pragma unroll
            for (int L = 0; L < NLEV; ++L) {
                float m = S[0][L];
#pragma unroll
                for (int q = 1; q < QN; ++q) m = fmaxf(m, S[q][L]);
                any |= m >= thr.v[L];
            }
            if (!__any_sync(0xffffffffu, any)) continue;
#pragma unroll
            for (int q = 0; q < QN; ++q) {
                const int k = kk + CT * q;
                const bool valid = k >= 1;
#pragma unroll
                for (int L = 0; L < NLEV; ++L) {
                    const bool hit = valid && (S[q][L] >= thr.v[L]);
                    const unsigned mk = __ballot_sync(0xffffffffu, hit);
                    if (mk) {
                        const int leader = __ffs(mk) - 1;
                        unsigned long long b0 = 0;
                        if ((int)lane == leader) b0 = atomicAdd(count, (unsigned long long)__popc(mk));
                        b0 = __shfl_sync(0xffffffffu, b0, leader);
                        if (hit) {
                            const unsigned long long pos = b0 + __popc(mk & ((1u << lane) - 1u));
                            if ((int64_t)pos < cap) {
                                Cand cd;
                                cd.tidx = (uint32_t)(tidx0 + tl);
                                cd.nharm = (uint16_t)(1 << L);
                                cd.flags = 0;
                                cd.bin = (uint32_t)k;
                                cd.power = S[q][L];
                                cands[pos] = cd;
                            }
                        }
                    }
                }
            }
        }
    }
}

}  // namespace

namespace {
// Dynamic shared memory of the transposing median kernels, set once per device.
cudaError_t med_t_attributes()
{
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return cudaSuccess;
#define BPS_MED_ATTR(v)                                                                             \
    if (e == cudaSuccess)                                                                           \
        e = cudaFuncSetAttribute(k_median_warp_t<v, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)med_t_smem<v>());                                             \
    if (e == cudaSuccess)                                                                           \
        e = cudaFuncSetAttribute(k_median_warp_t<v, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)med_t_smem<v>());
    BPS_MED_ATTR(1) BPS_MED_ATTR(2) BPS_MED_ATTR(4) BPS_MED_ATTR(8) BPS_MED_ATTR(16) BPS_MED_ATTR(32)
#undef BPS_MED_ATTR
    if (e == cudaSuccess) done[dev] = true;
    return e;
}
}  // namespace

cudaError_t launch_block_median(float* P, int nt, const Plan& p, float* scale,
                                cudaStream_t s, const float* Pt)
{
    const int64_t nblk = p.M >> p.logW;
    if (p.ptrans) {
        if (!Pt || p.logW > 10 || p.logW > p.logR || p.logC < kLogMedCols || p.logNP > 1)
            return cudaErrorInvalidValue;
        cudaError_t e = med_t_attributes();
        if (e != cudaSuccess) return e;
        dim3 tgrid((unsigned)(nblk / kMedCols), (unsigned)nt);
        const int th = 32 * kMedCols;
#define BPS_MED_T(v, lt) k_median_warp_t<v, lt><<<tgrid, th, med_t_smem<v>(), s>>>(Pt, p, P, scale)
#define BPS_MED_T_W(lt)                    \
    switch (p.logW) {                      \
        case 5: BPS_MED_T(1, lt); break;   \
        case 6: BPS_MED_T(2, lt); break;   \
        case 7: BPS_MED_T(4, lt); break;   \
        case 8: BPS_MED_T(8, lt); break;   \
        case 9: BPS_MED_T(16, lt); break;  \
        default: BPS_MED_T(32, lt); break; \
    }
        if (p.logNP == 0) {
            BPS_MED_T_W(0)
        } else {
            BPS_MED_T_W(1)
        }
#undef BPS_MED_T_W
#undef BPS_MED_T
        return cudaGetLastError();
    }
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

namespace {

// Once per device and H: the stage ring's dynamic shared memory and the resident CTAs per
// SM it allows (host-side attributes and queries only, so this is safe during capture).
template <int NH>
cudaError_t hs_shape(int& ctas)
{
    static std::mutex mu;
    static int cached[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!cached[dev]) {
        const int smem = (int)HsGeom<NH>::SMEM;
        e = cudaFuncSetAttribute(k_harmsum<NH>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0, nsm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_harmsum<NH>, kHsThreads, smem);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        cached[dev] = std::max(1, per_sm) * std::max(1, nsm);
    }
    ctas = cached[dev];
    return cudaSuccess;
}

template <int NH>
cudaError_t launch_hs(const float* P, int nt, int64_t tidx0, const Plan& p, const Thr& thr,
                      Cand* cands, int64_t cap, unsigned long long* count, float* s_out,
                      unsigned int* tile_ctr, cudaStream_t s)
{
    int ctas = 0;
    cudaError_t e = hs_shape<NH>(ctas);
    if (e != cudaSuccess) return e;
    const int64_t ntiles = (p.M / kHsTile) * (int64_t)nt;
    if (ntiles < 1 || ntiles > INT32_MAX) return cudaErrorInvalidValue;
    const int grid = (int)std::min<int64_t>(ntiles, ctas);
    e = cudaMemsetAsync(tile_ctr, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    k_harmsum<NH><<<grid, kHsThreads, HsGeom<NH>::SMEM, s>>>(P, p, tidx0, thr, cands, cap, count,
                                                                  s_out, (int)ntiles, tile_ctr);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_harmsum(const float* P, const float* scale, int nt, int64_t tidx0,
                           const Plan& p, const Thr& thr, Cand* cands, int64_t cap,
                           unsigned long long* count, float* s_out, unsigned int* tile_ctr,
                           cudaStream_t s)
{
    (void)scale;
    if (!tile_ctr) return cudaErrorInvalidValue;
    switch (p.nharm) {
        case 1: return launch_hs<1>(P, nt, tidx0, p, thr, cands, cap, count, s_out, tile_ctr, s);
        case 2: return launch_hs<2>(P, nt, tidx0, p, thr, cands, cap, count, s_out, tile_ctr, s);
        case 4: return launch_hs<4>(P, nt, tidx0, p, thr, cands, cap, count, s_out, tile_ctr, s);
        case 8: return launch_hs<8>(P, nt, tidx0, p, thr, cands, cap, count, s_out, tile_ctr, s);
        case 16: return launch_hs<16>(P, nt, tidx0, p, thr, cands, cap, count, s_out, tile_ctr, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_wait_selftest(int limit, unsigned long long* status, cudaStream_t s)
{
    if (limit < 1) return cudaErrorInvalidValue;
    k_wait_selftest<<<1, 32, 0, s>>>(limit, status);
    return cudaGetLastError();
}

cudaError_t prepare_detect_kernels()
{
    int c = 0;
    cudaError_t e = med_t_attributes();
    if (e == cudaSuccess) e = hs_shape<1>(c);
    if (e == cudaSuccess) e = hs_shape<2>(c);
    if (e == cudaSuccess) e = hs_shape<4>(c);
    if (e == cudaSuccess) e = hs_shape<8>(c);
    if (e == cudaSuccess) e = hs_shape<16>(c);
    return e;
}

}  // namespace bps
