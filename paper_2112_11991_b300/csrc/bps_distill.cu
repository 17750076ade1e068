// bps_distill.cu -- candidate distillation behind bps_distill (include/bps.h; host code).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "../../include/bps.h"

// =====================================================================================
// Candidate distillation (host): group repeated detections of one signal -- the same
// or a harmonically related fundamental frequency, seen under several templates or
// harmonic levels -- and keep the most significant member of each group.
// =====================================================================================
namespace {

// -log Q(n, x): false-alarm exponent of a harmonic sum of n whitened bins (Gamma(n,1)
// tail), evaluated in log space so large sums do not underflow.
double neg_log_q(int n, double x)
{
    if (x <= 0.0) return 0.0;
    double lt = 0.0, lmax = 0.0;  // log of terms x^m / m!, m < n
    std::vector<double> terms((size_t)n);
    for (int m = 0; m < n; ++m) {
        lt = (m == 0) ? 0.0 : lt + std::log(x) - std::log((double)m);
        terms[(size_t)m] = lt;
        lmax = (m == 0) ? lt : std::max(lmax, lt);
    }
    double s = 0.0;
    for (double t : terms) s += std::exp(t - lmax);
    return x - (lmax + std::log(s));
}

}  // namespace

extern "C" int bps_distill(const bps_candidate* in, int64_t n_in, int64_t n_samples,
                           double tsamp_s, double tol_bins, int32_t max_ratio,
                           bps_candidate* out, int64_t cap, int64_t* n_out)
try {
    if ((!in && n_in > 0) || n_in < 0 || n_samples < 2 || !(tsamp_s > 0.0) ||
        !(tol_bins > 0.0) || max_ratio < 1 || max_ratio > 64 || !n_out || cap < 0)
        return BPS_ERR_INVALID_ARG;
    const double T = (double)n_samples * tsamp_s;
    struct Item {
        double f, sig;
        int64_t i;
    };
    std::vector<Item> it((size_t)n_in);
    for (int64_t i = 0; i < n_in; ++i) {
        const bps_candidate& c = in[i];
        if (c.nharm == 0) return BPS_ERR_INVALID_ARG;
        it[(size_t)i] = {(double)c.bin / ((double)c.nharm * T), neg_log_q(c.nharm, c.power), i};
    }
    std::sort(it.begin(), it.end(), [](const Item& a, const Item& b) {
        if (a.sig != b.sig) return a.sig > b.sig;
        return a.i < b.i;
    });
    std::vector<char> used((size_t)n_in, 0);
    const double tol = tol_bins / T;  // frequency tolerance of one fundamental bin
    int64_t k = 0;
    for (size_t a = 0; a < it.size(); ++a) {
        if (used[a]) continue;
        used[a] = 1;
        int64_t members = 1;
        const double f0 = it[a].f;
        for (size_t b = a + 1; b < it.size(); ++b) {
            if (used[b]) continue;
            const double f = it[b].f;
            bool rel = false;
            for (int p = 1; p <= max_ratio && !rel; ++p)
                for (int q = 1; q <= max_ratio && !rel; ++q)
                    // f / f0 = p / q within the tolerance scaled by the larger multiple
                    rel = std::fabs(q * f - p * f0) <= tol * (double)std::max(p, q);
            if (rel) {
                used[b] = 1;
                ++members;
            }
        }
        if (k < cap && out) {
            out[k] = in[it[a].i];
            out[k].flags = (uint16_t)std::min<int64_t>(members, 65535);
        }
        ++k;
    }
    *n_out = k;
    return k > cap ? BPS_ERR_CAND_OVERFLOW : BPS_OK;
} catch (...) {
    return BPS_ERR_OUT_OF_MEMORY;  // host allocation failed
}

