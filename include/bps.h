/*
 * bps.h -- C ABI of the B300-native coherent template-bank binary-pulsar search
 * (Balakrishnan et al., arXiv:2112.11991).
 *
 * The library runs, for every orbital template of a bank, the per-template hot
 * path of the paper on one CUDA device (sm_103a):
 *
 *   index map (BT Roemer delay + Kepler, App. A, Algorithm 1)
 *   -> nearest-neighbour resampling gather (Algorithm 1)
 *   -> real FFT of the resampled series (Sec. 2.4: uniform f0 grid)
 *   -> power |X_k|^2 (Sec. 2.1, detection statistic)
 *   -> block-median de-reddening (App. A, "Fourier de-reddening")
 *   -> incoherent 1/2/4/8/16-harmonic sums (Sec. 2.1, S_L)
 *   -> threshold (Sec. 2.1, false-alarm statistics) and compaction.
 *
 * Conventions (readings of the paper, identical in the FP64 oracle):
 *   off_j = (Delta_R(0) - Delta_R(j t_s)) / t_s,  idx_j = j + floor(off_j + 1/2),
 *   resampled x'_j = x[idx_j] (series mean when idx_j is outside [0, n));
 *   X_k = sum_j x'_j exp(-2 pi i j k / n), k in [0, n/2), P_0 := 0;
 *   Pw_k = P_k ln2 / med_b, med_b the lower median of block b of W bins;
 *   S_n[k] = sum_{h=1}^{n} Pw[(k h + n/2) div n], k in [1, n/2);
 *   candidate (template, n, k) when S_n[k] >= thr_n, where thr_n solves
 *   Q(n, thr_n) = erfc(sigma / sqrt 2) / 2 and Q is the Gamma(n, 1) tail.
 *
 * Errors: every int-returning call returns BPS_OK (0) or a negative BPS_ERR_*
 * code; bps_last_error() then holds a message.  Calls on one context are
 * serialised by an internal mutex (thread-safe per context).
 * Ownership: the library copies series and banks into device memory it owns
 * (or borrows a caller device pointer, see bps_load_series); output buffers
 * passed to the library belong to the caller.  Host pointers must stay valid
 * for the duration of the call only.
 */
#ifndef BPS_H
#define BPS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---------------------------------------------------------- */
#define BPS_OK                  0
#define BPS_ERR_INVALID_ARG    -1  /* bad size, parameter or id                   */
#define BPS_ERR_OUT_OF_MEMORY  -2  /* device allocation refused (admission)       */
#define BPS_ERR_NOT_READY      -3  /* request still running                       */
#define BPS_ERR_CAND_OVERFLOW  -4  /* candidates truncated; n_total is the truth   */
#define BPS_ERR_TIMEOUT        -5  /* a bounded wait expired                      */
#define BPS_ERR_CUDA           -6  /* CUDA runtime / launch failure               */
#define BPS_ERR_UNSUPPORTED    -7  /* size or mode outside what is built          */

/* ---- series dtypes --------------------------------------------------------- */
#define BPS_F32          0  /* float32 samples                                    */
#define BPS_F16_SCALED   1  /* float32 input, stored on device as FP16 with one   */
                            /* power-of-two FP32 scale per 4096 samples            */

/* ---- search modes (bps_search_params.mode) ------------------------------- */
#define BPS_MODE_FUSED   0  /* hand-written kernels: gather fused into FFT pass 1, */
                            /* split + power fused into pass 2                     */
#define BPS_MODE_PLAIN   1  /* plain FP32 per-template form: index map -> gather   */
                            /* -> cuFFT R2C -> power; same whitening/harmonic sum  */

/* One orbital template (App. A, BT model).  Circular templates: omega = ecc = 0,
 * for which Delta_R = tau sin(Omega t + phi) (Sec. 2.1, circular phase model). */
typedef struct {
    double porb_s;    /* orbital period P_orb [s], > 0 ; Omega = 2 pi / P_orb    */
    double tau_lts;   /* projected semi-major axis a sin(eps)/c [lt-s], >= 0     */
    double phi_rad;   /* initial orbital phase alpha [rad] (M(0) = alpha)         */
    double omega_rad; /* longitude of periastron psi [rad]                         */
    double ecc;       /* eccentricity e in [0, 1)                                  */
} bps_template;

/* One detection: harmonic sum S_n[bin] >= thr_n.  The fundamental frequency is
 * bin / (nharm * T), T = n_samples * t_samp.  16 bytes. */
typedef struct {
    uint32_t template_idx; /* index into the bank                                  */
    uint16_t nharm;        /* n in {1, 2, 4, 8, 16}                                 */
    uint16_t flags;        /* reserved, 0                                           */
    uint32_t bin;          /* k, the bin of the n-th harmonic                       */
    float    power;        /* S_n[k] in units of the whitened noise mean            */
} bps_candidate;

typedef struct {
    int32_t nharm_max;     /* 1, 2, 4, 8 or 16 (Sec. 2.1: up to 16 harmonics)       */
    int32_t whiten_block;  /* W: power of two in [32, n/2]; 1024 in the paper's runs */
    double  sigma_thr;     /* Gaussian-equivalent significance of the threshold     */
    int32_t auto_thr;      /* 1: sigma = S/N_min(n_trials), n_trials =              */
                           /*    (n/2) * levels * templates (Sec. 2.1)               */
    int32_t mode;          /* BPS_MODE_FUSED or BPS_MODE_PLAIN                      */
    int64_t cand_cap;      /* device candidate capacity of the request (>= 1)       */
    int32_t precision;     /* reserved, 0 (the storage precision is the series')    */
    int32_t batch;         /* templates per launch batch; 0 = library's choice       */
    int32_t log_tile;      /* FFT pass-1 tile: 2^log_tile complex values per CTA,    */
                           /* 13 or 14; 0 = library's choice (14)                     */
    int32_t log_tile2;     /* FFT pass-2 tile, 12, 13 or 14 (at least one row pair); */
                           /* 0 = library's choice (13)                               */
    int32_t log_cols;      /* log2 C of the four-step split N/2 = R x C (pass-1 column  */
                           /* length R, pass-2 row length C: the radix structure of   */
                           /* both passes), in [max(5, log2(N/2) - 12),               */
                           /* min(log2(N/2) - 5, 12)]; 0 = library's choice           */
    int32_t pass1_kind;    /* BPS_PASS1_*: how pass 1 (index map + gather + column FFTs) */
                           /* is organised; 0 = library's choice                        */
    int32_t power_layout;  /* BPS_POWER_*: how pass 2 stores the power spectrum;        */
                           /* 0 = library's choice                                      */
    int32_t pass2_kind;    /* BPS_PASS2_*: how pass 2 (row FFTs + split + power) gets    */
                           /* its rows; 0 = library's choice                            */
} bps_search_params;

/* bps_search_params.pass2_kind */
#define BPS_PASS2_AUTO      0  /* the autotuned choice, else the one-phase kernel            */
#define BPS_PASS2_FUSED     1  /* each CTA loads its rows into registers for the first stage */
#define BPS_PASS2_TMA       2  /* persistent CTAs: one thread copies the next tile's rows    */
                               /* into a staging buffer with TMA bulk copies while 16 warps  */
                               /* transform the current one (2^13-complex tiles, R and C in  */
                               /* 2^10..2^12, else INVALID_ARG)                               */

/* bps_search_params.pass1_kind */
#define BPS_PASS1_AUTO      0  /* the autotuned choice, else the one-phase kernel            */
#define BPS_PASS1_FUSED     1  /* one phase per tile: every warp gathers, then all run the   */
                               /* FFT stages (tiles of 2^log_tile complex values)            */
#define BPS_PASS1_WARPSPEC  2  /* warp-specialised: producer warps gather tile i+1 while     */
                               /* consumer warps FFT tile i (2^13-complex tiles; built for   */
                               /* R = 2^10..2^12 and 2^21..2^25 samples, else INVALID_ARG)   */
#define BPS_PASS1_ASYNC     3  /* one phase per tile with the gather as asynchronous copies  */
                               /* into shared memory: 2^13 tiles, two CTAs per SM (same     */
                               /* splits as WARPSPEC; FP16 series use the one-phase kernel)  */

/* bps_search_params.power_layout (results are identical; only the memory traffic differs) */
#define BPS_POWER_AUTO      0  /* row-major when a pass-2 CTA holds at most two row pairs,   */
                               /* W <= R and W <= 1024, else bin order                       */
#define BPS_POWER_BINS      1  /* pass 2 writes bins in order; whitening in place            */
#define BPS_POWER_ROWS      2  /* pass 2 writes row-major blocks of 8 columns; the whitening */
                               /* kernel transposes (needs <= 2 row pairs per pass-2 CTA,    */
                               /* W <= R, W <= 1024, else INVALID_ARG)                       */

typedef struct bps_ctx bps_ctx;

/* Fill *p with the defaults: nharm_max 16, W 1024, sigma 6, fused mode,
 * cand_cap 1<<20, batch 0. */
void bps_default_params(bps_search_params* p);

/* Create a context bound to CUDA device `device`.  *out receives the handle.
 * Returns BPS_ERR_CUDA if the device cannot be used. */
int bps_create(bps_ctx** out, int device);

/* Destroy a context: waits for its work, frees every series, bank and request. */
void bps_destroy(bps_ctx* ctx);

/* Load a dedispersed time series S sampled at t_samp (App. A.1: "dedispersed
 * timeseries S ... sampled at t_samp").
 *   data      n float32 samples (host pointer, or device pointer if on_device)
 *   n         power of two in [2^11, 2^25]
 *   tsamp_s   sampling time [s], > 0
 *   dtype     BPS_F32 or BPS_F16_SCALED (storage on the device)
 *   on_device 0: data is host memory, copied; 1: data is device memory of this
 *             context's device -- copied for BPS_F16_SCALED, borrowed (not
 *             copied, caller keeps it alive until bps_unload) for BPS_F32
 * The series mean (the fill value for samples mapped outside the series) is
 * computed on the device in FP64.  *series_id receives an id (> 0). */
int bps_load_series(bps_ctx* ctx, const void* data, int64_t n, double tsamp_s,
                    int dtype, int on_device, int64_t* series_id);

/* Replace the samples of a loaded series (same n, tsamp and storage) and recompute
 * its mean on the device; ordered on the context's stream and synchronous on return.
 * Searches and graphs that read the series see the new data from then on.  Not for
 * series that borrow caller device memory (update that memory instead). */
int bps_series_update(bps_ctx* ctx, int64_t series_id, const void* data, int on_device);

/* Load a template bank (Algorithm 1: "K orbital templates in template bank").
 * t: host array of count templates (copied).  Checks porb > 0, tau >= 0,
 * 0 <= ecc < 1, finite values.  *bank_id receives an id (> 0). */
int bps_load_bank(bps_ctx* ctx, const bps_template* t, int64_t count, int64_t* bank_id);

/* Enqueue the search of every template of a bank over a series on
 * `cuda_stream` (a cudaStream_t; NULL = the context's own stream): Algorithm 1's
 * outer loop over the K templates, each template resampled, FFT'd (Sec. 2.4),
 * whitened ("Fourier de-reddening", App. A), harmonic-summed (Sec. 2.1, S_L) and
 * thresholded (Sec. 2.1, false-alarm statistics) as described at the top of
 * this file.  Returns at once; *req_id receives a request id.
 *   params      search parameters (see bps_search_params); checked before any
 *               work is enqueued (BPS_ERR_INVALID_ARG, BPS_ERR_UNSUPPORTED when
 *               an orbit is too fast for the FP32 index map)
 * Workspace is allocated stream-ordered and freed when the request completes;
 * the candidate buffer (params->cand_cap records) and its counters come from a
 * pool owned by the context and return to it when the request is unloaded. */
int bps_search(bps_ctx* ctx, int64_t series_id, int64_t bank_id,
               const bps_search_params* params, void* cuda_stream, int64_t* req_id);

/* Non-blocking completion test: *done = 1 when the request has finished. */
int bps_query(bps_ctx* ctx, int64_t req_id, int* done);

/* Wait for a request and copy its candidates -- the peak-detection output of
 * App. A: every (template, harmonic level n, bin k) with S_n[k] >= thr_n
 * (Sec. 2.1) -- sorted by (template_idx, nharm, bin), into out[0 .. cap)
 * (host memory of the caller; out may be NULL with cap = 0 to query the count).
 * *n_written = candidates copied, *n_total = all candidates found.  Returns
 * BPS_ERR_CAND_OVERFLOW when the device capacity (cand_cap) was exceeded: then
 * the kept subset is arbitrary; BPS_ERR_TIMEOUT when a bounded device wait
 * expired (results incomplete). */
int bps_fetch_candidates(bps_ctx* ctx, int64_t req_id, bps_candidate* out,
                         int64_t cap, int64_t* n_written, int64_t* n_total);

/* Free a series, bank or request id. */
int bps_unload(bps_ctx* ctx, int64_t id);

/* Message of the last error on this context (never NULL). */
const char* bps_last_error(bps_ctx* ctx);

/* ---- stage entry points (inspection and parity; same kernels as bps_search) */

/* Algorithm 1 index map of one template: idx_out[j] = idx_j for j in [0, n)
 * (int32, host buffer of n entries).  *n_precise receives how many samples
 * took the compensated-precision branch (offset within 1e-4 of a rounding
 * boundary in the fast evaluation). */
int bps_index_map(bps_ctx* ctx, int64_t series_id, int64_t bank_id,
                  int64_t template_idx, int32_t* idx_out, int64_t* n_precise);

/* Whitened power spectrum Pw_k, k in [0, n/2), of templates [t0, t0 + count)
 * into pw_out (host, count * n/2 floats, template-major). */
int bps_whitened_spectrum(bps_ctx* ctx, int64_t series_id, int64_t bank_id,
                          int64_t t0, int64_t count, const bps_search_params* params,
                          float* pw_out);

/* Harmonic sums S_{2^L}[k] of one template, L in [0, levels), k in [0, n/2),
 * into s_out (host, levels * n/2 floats, level-major; S[.][0] = 0). */
int bps_harmonic_sums(bps_ctx* ctx, int64_t series_id, int64_t bank_id,
                      int64_t template_idx, const bps_search_params* params,
                      float* s_out);

/* Whitening of caller-provided power spectra with the search's own block-median
 * kernels (App. A, "Fourier de-reddening"): for spectrum s in [0, count) and block b
 * of W = whiten_block consecutive bins, med_b is the block's lower median (its
 * element of rank floor((W-1)/2), counted from 0 in ascending order) and
 *   d_scale_out[s * nbins/W + b] = ln2 / med_b      (FP32 division; 0 when med_b = 0)
 *   d_pw_out[s * nbins + k]      = d_power[s * nbins + k] * scale of k's block
 *                                                     (one FP32 product)
 *   d_power      device memory of the context's GPU, count * nbins floats, read
 *                only; values >= 0 and not NaN (other values give an unspecified
 *                result, never a fault)
 *   count        number of spectra, >= 1
 *   nbins        bins per spectrum, a power of two in [whiten_block, 2^30]
 *   whiten_block power of two in [32, 8192]
 *   d_pw_out     device, count * nbins floats; equal to d_power (in place) or not
 *                overlapping it
 *   d_scale_out  device, count * nbins / whiten_block floats
 *   cuda_stream  cudaStream_t to run on (NULL = legacy default stream)
 * Returns BPS_OK, BPS_ERR_INVALID_ARG or BPS_ERR_CUDA; the work is enqueued on the
 * stream and the call does not wait for it.  No device memory is allocated. */
int bps_whiten(bps_ctx* ctx, const float* d_power, int64_t count, int64_t nbins,
               int32_t whiten_block, float* d_pw_out, float* d_scale_out, void* cuda_stream);

/* ---- measurement ------------------------------------------------------------ */

/* Stage indices of bps_stats.stage_ms / stage_launches. */
#define BPS_STAGE_ANCHORS   0  /* FP64 anchor kernel                               */
#define BPS_STAGE_PASS1     1  /* fused: index map + gather + column FFTs          */
                               /* plain: index map + gather into a series          */
#define BPS_STAGE_PASS2     2  /* fused: row FFTs + real split + power; plain: cuFFT */
#define BPS_STAGE_POWER     3  /* plain only: |X_k|^2                               */
#define BPS_STAGE_MEDIAN    4  /* block lower medians                              */
#define BPS_STAGE_HARMSUM   5  /* harmonic sums + threshold + compaction           */
#define BPS_NSTAGES         6

typedef struct {
    int64_t templates;       /* templates searched                                 */
    int32_t batch;           /* templates per launch                               */
    int32_t anchor_block;    /* B, samples per FP64 anchor                          */
    int32_t launches;        /* kernel launches of this library (cuFFT counted 1)   */
    int32_t profiled;        /* 1 when stage_ms holds CUDA-event timings            */
    int32_t stage_launches[8];
    float   stage_ms[8];     /* summed device time per stage (profiled requests)    */
} bps_stats;

/* Enable (1) or disable (0) per-stage CUDA-event timing of later bps_search calls
 * on this context.  Events are recorded on the request's stream around each
 * stage launch. */
int bps_set_profiling(bps_ctx* ctx, int on);

/* Statistics of a finished request (waits for it).  Stage times are filled only
 * when profiling was on when the request was enqueued. */
int bps_request_stats(bps_ctx* ctx, int64_t req_id, bps_stats* out);

/* Failure-path self-test: launches one CTA that polls, with the harmonic sum's bounded
 * mbarrier wait, a barrier whose phase nothing completes, at most poll_limit times.  The
 * wait expires, the kernel records it and returns (no fault, nothing in flight), and the
 * context stays usable.  *timed_out = 1 when the wait expired as designed.  Returns
 * BPS_OK, or BPS_ERR_INVALID_ARG / BPS_ERR_CUDA. */
int bps_selftest_bounded_wait(bps_ctx* ctx, int32_t poll_limit, int32_t* timed_out);

/* ---- CUDA graphs: many searches, one launch --------------------------------- */

/* Capture the searches of `count` (series, bank) pairs (series of any supported
 * lengths, each with its own bank) into one CUDA graph: pairs run on up to 4 parallel
 * branches, each branch with one reusable workspace; each pair has its own candidate
 * region of params->cand_cap candidates.  Fused mode only (BPS_ERR_UNSUPPORTED
 * otherwise).  Series and banks must stay loaded while the graph exists; use
 * bps_series_update to search new data with the same graph.  *graph_id is freed by
 * bps_unload. */
int bps_graph_create(bps_ctx* ctx, int64_t count, const int64_t* series_ids,
                     const int64_t* bank_ids, const bps_search_params* params, int64_t* graph_id);

/* Replay the graph on cuda_stream (NULL = the context's stream).  A replay overwrites
 * the previous one's candidates: fetch them first. */
int bps_graph_launch(bps_ctx* ctx, int64_t graph_id, void* cuda_stream);

/* Wait for the last replay and copy pair `pair`'s candidates, sorted by (template_idx,
 * nharm, bin); return codes as bps_fetch_candidates. */
int bps_graph_fetch(bps_ctx* ctx, int64_t graph_id, int64_t pair, bps_candidate* out, int64_t cap,
                    int64_t* n_written, int64_t* n_total);

/* ---- random template banks from the parameter-space metric (host routines) ------ */

/* Search region and bank requirements (Sec. 2.3-2.4; defaults = Table 1).  Circular
 * orbits (3 orbital coordinates tau, Omega, alpha) when ecc_max = 0, elliptical (adds
 * omega, e) otherwise. */
typedef struct {
    double tobs_s;            /* observation length T                                      */
    double f_max_hz;          /* spin frequency the metric is projected at (f_max)         */
    double mismatch;          /* nominal mismatch m* (0, 1)                                */
    double coverage;          /* coverage eta (0, 1)                                       */
    double porb_min_s, porb_max_s;  /* P_orb uniform prior                                */
    double tau_max_lts;       /* > 0: tau uniform in [0, tau_max_lts]; 0: tau in
                                 [0, tau_max(P_orb)] from Kepler's third law and the masses */
    double m_pulsar_min_msun; /* lightest pulsar (Kepler bound)                            */
    double m_comp_max_msun;   /* heaviest companion (Kepler bound)                         */
    double ecc_max;           /* e uniform in [0, ecc_max]; 0 = circular                   */
    int32_t n_time;           /* midpoint-rule points for the time averages (>= 16)        */
    int32_t n_volume;         /* Monte Carlo points for the proper volume (>= 100)         */
} bps_bank_spec;

/* Table 1 values: T = 1.2 h, f_max = 66.67 Hz, m* = 0.2, eta = 0.9, P_orb U(6, 12) h,
 * m_p,min = 1.4, m_c,max = 8 Msun, e U(0, 0.1), n_time 256, n_volume 20000. */
void bps_default_bank_spec(bps_bank_spec* spec);

/* sqrt(det gamma) of the frequency-projected metric (Sec. 2.4: gamma_ab = g_ab -
 * g_fa g_fb / g_ff, g_ab = <d_a Phi d_b Phi> - <d_a Phi><d_b Phi> over [0, T], Phi =
 * 2 pi f_max (t - Delta_R)) at each of `count` templates, in the orbital coordinates
 * (tau [lt-s], Omega [rad/s], alpha[, omega, e]).  BPS_ERR_INVALID_ARG on a bad spec
 * or template. */
int bps_metric_density(const bps_bank_spec* spec, const bps_template* t, int64_t count,
                       double* sqrt_det_out);

/* The projected metric itself at one template: n x n row-major into gamma_out (n = 3
 * circular, 5 elliptical). */
int bps_metric_projected(const bps_bank_spec* spec, const bps_template* t, double* gamma_out);

/* Random template bank (Sec. 2.4, "Random Template Banks"): proper volume V of the prior
 * region by Monte Carlo, N_R = ln(1 - eta) / ln(1 - m*^(n/2) C_n / V) templates drawn
 * with density proportional to sqrt(det gamma) (rejection sampling, seeded).  Writes
 * ceil(N_R) templates to out (*n_out = that count; BPS_ERR_CAND_OVERFLOW and nothing
 * written if it exceeds cap; out = NULL with cap = 0 computes the count only),
 * *proper_volume = V, *n_expected = N_R (either may be NULL).  Host threads evaluate
 * the densities; the result is deterministic for a given seed and spec.
 * BPS_ERR_OUT_OF_MEMORY if host memory or threads cannot be had. */
int bps_metric_bank(const bps_bank_spec* spec, uint64_t seed, bps_template* out, int64_t cap,
                    int64_t* n_out, double* proper_volume, double* n_expected);

/* Candidate distillation (App. A: repeated detections of one candidate are grouped).
 * Host routine, no device work.  Each candidate's fundamental frequency is
 * f = bin / (nharm T), T = n_samples t_samp, and its significance the false-alarm
 * exponent -ln Q(nharm, power) of the Gamma(nharm, 1) tail.  In order of decreasing
 * significance, each candidate not yet grouped starts a group and takes every other
 * ungrouped candidate whose f satisfies |q f - p f_0| <= tol_bins/T * max(p, q) for
 * some 1 <= p, q <= max_ratio (same signal under another template, or a harmonic /
 * subharmonic of it).  Writes the group leaders (most significant first) to out with
 * flags = group size, *n_out = number of groups; BPS_ERR_CAND_OVERFLOW if > cap. */
int bps_distill(const bps_candidate* in, int64_t n_in, int64_t n_samples, double tsamp_s,
                double tol_bins, int32_t max_ratio, bps_candidate* out, int64_t cap,
                int64_t* n_out);

/* Autotuner: times every combination of pass-1 tile (2^13, 2^14), pass-2 tile (2^13,
 * 2^14) and templates per launch (4, 8, 16, 32) on the first sample_templates
 * templates of the bank over the series (CUDA events, best of two runs), writes the
 * fastest parameters to *best (other fields copied from *base) and its device time per
 * template to *best_ms_per_template, and remembers the choice in the context: later
 * searches of the same series length, mode and harmonic count that leave log_tile,
 * log_tile2, log_cols or batch at 0 use it.  Candidates: pass-1 and pass-2 tiles 13/14,
 * the library's four-step split and its neighbours log_cols +- 1, batches 8..64. */
int bps_autotune(bps_ctx* ctx, int64_t series_id, int64_t bank_id, const bps_search_params* base,
                 int64_t sample_templates, bps_search_params* best, double* best_ms_per_template);

/* ---- serving: a continuously batched request loop (native scheduler) ---------- */

/* A server owns a worker thread that admits submitted search requests onto the
 * device as stream slots and HBM free up, and interleaves their launch groups (one
 * batch of templates each) round-robin, a few groups in flight per request, so a
 * request that arrives while others run starts within a launch group instead of
 * waiting for them to finish.  A request submitted with its own series
 * (bps_server_submit) has its series and bank copied to the device at admission
 * and freed when its candidates are on the host; a request on a resident series
 * (bps_server_load_series + bps_server_submit_series) finds the series already on
 * the device.  Device memory comes from the context's stream-ordered pool, which
 * keeps freed blocks for later requests.  Results of a
 * request do not depend on what else runs (the per-template computation is the same
 * as bps_search's with the same parameters). */
typedef struct bps_server bps_server;

typedef struct {
    int32_t max_active;        /* requests resident on the device at once, >= 1     */
    int32_t groups_in_flight;  /* launch groups queued per active request, >= 1     */
    int64_t hbm_budget;        /* device bytes the server may hold; 0 = 90 % of the */
                               /* free memory when the server is created             */
} bps_server_config;

/* Create a server on ctx's device (the context must outlive the server). */
int bps_server_create(bps_ctx* ctx, const bps_server_config* cfg, bps_server** out);

/* Stop the worker (after finishing admitted requests) and free everything. */
void bps_server_destroy(bps_server* srv);

/* Submit a search of `count` templates over a host series of n samples (copied
 * before the call returns; dtype BPS_F32 or BPS_F16_SCALED storage).  Returns at
 * once with *ticket; BPS_ERR_OUT_OF_MEMORY when the request alone exceeds the HBM
 * budget, BPS_ERR_INVALID_ARG for bad sizes/parameters (as bps_load_series,
 * bps_load_bank, bps_search). */
int bps_server_submit(bps_server* srv, const float* series, int64_t n, double tsamp_s,
                      int dtype, const bps_template* bank, int64_t count,
                      const bps_search_params* params, int64_t* ticket);

/* Load a series into the server's resident store (Algorithm 1's "dedispersed
 * timeseries S sampled at t_samp", kept for many searches): the host data (n
 * float32 samples, copied into pinned host memory before the call returns) is
 * staged on the device by the first request that names it and stays there,
 * counted against the HBM budget, for later requests.  When a request needs room,
 * resident series that no queued or running request names are evicted, least
 * recently used first; an evicted series is staged again from the host copy by
 * the next request that names it.  Same sizes and dtypes as bps_load_series.
 * *series_id receives the id (> 0) used by bps_server_submit_series.
 * BPS_ERR_OUT_OF_MEMORY when the series alone exceeds the budget. */
int bps_server_load_series(bps_server* srv, const float* series, int64_t n, double tsamp_s,
                           int dtype, int64_t* series_id);

/* Submit a search of `count` templates (host array, copied) over a resident series;
 * the request pins the series (it is neither evicted nor unloadable) until its
 * result is on the host.  Otherwise as bps_server_submit. */
int bps_server_submit_series(bps_server* srv, int64_t series_id, const bps_template* bank,
                             int64_t count, const bps_search_params* params, int64_t* ticket);

/* Remove a series from the resident store (device copy and host copy).
 * BPS_ERR_INVALID_ARG while unfinished requests name it, or for an unknown id. */
int bps_server_unload_series(bps_server* srv, int64_t series_id);

/* *resident = 1 while the series is on the device; *times_staged counts how often it
 * was staged (1 + the times it was evicted and staged again).  Either may be NULL. */
int bps_server_series_info(bps_server* srv, int64_t series_id, int32_t* resident,
                           int64_t* times_staged);

/* Wait up to timeout_ms (< 0: no limit) for a ticket; BPS_ERR_NOT_READY when it is
 * still running.  Then copies its sorted candidates like bps_fetch_candidates and
 * reports *latency_s, from submission to candidates on the host.  The ticket is
 * released by the first call that returns its result. */
int bps_server_result(bps_server* srv, int64_t ticket, int32_t timeout_ms, bps_candidate* out,
                      int64_t cap, int64_t* n_written, int64_t* n_total, double* latency_s);

/* Snapshot: requests queued, resident, finished and not yet fetched; bytes held. */
int bps_server_stats(bps_server* srv, int64_t* queued, int64_t* active, int64_t* finished,
                     int64_t* bytes_held);

/* Message of the last error of the server (never NULL). */
const char* bps_server_last_error(bps_server* srv);

/* ---- allocation-free entry point -------------------------------------------- */

/* The paper has no counterpart to this call: it serves callers that must not
 * allocate device memory while they run -- e.g. real-time back ends that
 * reserve all GPU memory at start-up, or host frameworks whose own pool
 * allocator owns the device memory.  It computes the same whitened spectrum as
 * bps_whitened_spectrum for ONE template, with the same kernels, but needs no
 * context and calls no cudaMalloc, cudaFree or allocating library routine: its
 * scratch is one fixed 8 MiB device array inside the library (held on every
 * GPU that loads the library until the process exits).
 *   d_series     n float32 samples in device memory of the current device
 *   n            power of two in [2^11, 2^20]; larger n -> BPS_ERR_UNSUPPORTED
 *   tsamp_s      sampling time [s], > 0
 *   fill         value of samples mapped outside the series (the series mean)
 *   tmpl         host pointer to one template (read during the call)
 *   whiten_block power of two in [32, min(8192, n/2)]
 *   d_pw_out     device buffer of n/2 floats receiving Pw_k, k in [0, n/2)
 *   cuda_stream  cudaStream_t to run on (NULL = legacy default stream)
 * Returns BPS_OK, BPS_ERR_INVALID_ARG, BPS_ERR_UNSUPPORTED or BPS_ERR_CUDA;
 * the work is enqueued on the stream and the call does not wait for it.
 * Results agree with bps_whitened_spectrum within the power tolerance, not bit
 * for bit: the FP64 anchor block is chosen from this template alone
 * (bps_whitened_spectrum chooses it from the whole bank), and an offset within
 * rounding distance of a half-integer can round the other way with another block.
 * The scratch array is shared by every call and keeps the last call's
 * contents; calls that overlap on the GPU race on it and must be serialised.
 * Each call whose stream is not being captured looks up the array's address
 * (cudaGetSymbolAddress, with the current device; it allocates nothing); a call
 * during a stream capture reuses the last address looked up on that device, so
 * make one call on the device before any stream capture. */
int bps_whitened_spectrum_noalloc(const float* d_series, int64_t n, double tsamp_s,
                                  double fill, const bps_template* tmpl,
                                  int32_t whiten_block, float* d_pw_out,
                                  void* cuda_stream);

/* Per-level thresholds thr_n (n = 1, 2, ..., nharm_max) the search will use for
 * these parameters and problem size (host FP64). */
int bps_thresholds(const bps_search_params* params, int64_t n_samples,
                   int64_t n_templates, double* thr_out);

#ifdef __cplusplus
}
#endif

#endif /* BPS_H */
