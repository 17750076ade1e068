// bps_bank.cu -- random template banks from the frequency-projected parameter-space
// metric (host code, no device work).
//
// Phase model of a pulsar in a binary (Sec. 2.2): Phi(t) = 2 pi f0 (t - Delta_R(t)),
// Delta_R the BT Roemer delay (App. A) of the orbit (tau, Omega, alpha, omega, e).
// Metric (Sec. 2.3, "Definition of Metric and Mismatch"):
//   g_ab = <d_a Phi d_b Phi>_T - <d_a Phi>_T <d_b Phi>_T
// over lambda = (f0, tau, Omega, alpha[, omega, e]); the frequency-projected metric
// (Sec. 2.4) gamma_ab = g_ab - g_fa g_fb / g_ff on the orbital coordinates at f0 = f_max.
// Random template bank (Sec. 2.4, "Random Template Banks"): templates are drawn with
// probability density proportional to sqrt(det gamma) over the prior region; with proper
// volume V = int sqrt(det gamma) d^n lambda, unit-ball volume C_n = pi^(n/2)/Gamma(n/2+1)
// and nominal mismatch m*, coverage eta needs
//   N_R = ln(1 - eta) / ln(1 - m*^(n/2) C_n / V)
// templates (Eq. for the total number of random templates).
//
// Time averages: midpoint rule over n_time points of [0, T].  Volume: Monte Carlo over
// the prior box in (P_orb, tau, alpha[, omega, e]) with the Jacobian |dOmega/dP_orb| =
// 2 pi / P_orb^2.  Prior (Table 1): P_orb uniform, tau in [0, tau_max(P_orb)] with
// tau_max from Kepler's third law for the lightest pulsar and heaviest companion (or a
// fixed bound), alpha and omega in [0, 2 pi), e in [0, e_max].
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <thread>
#include <vector>

#include "../../include/bps.h"

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi = 2.0 * kPi;
constexpr double kGNewton = 6.67430e-11;   // m^3 kg^-1 s^-2
constexpr double kMsun = 1.98847e30;       // kg
constexpr double kLight = 299792458.0;     // m/s

// xoshiro256** seeded by splitmix64: uniform doubles in [0, 1)
struct Rng {
    uint64_t s[4];
    explicit Rng(uint64_t seed)
    {
        for (auto& v : s) {
            seed += 0x9E3779B97F4A7C15ull;
            uint64_t z = seed;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            v = z ^ (z >> 31);
        }
    }
    static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
    uint64_t next()
    {
        const uint64_t r = rotl(s[1] * 5, 7) * 9;
        const uint64_t t = s[1] << 17;
        s[2] ^= s[0];
        s[3] ^= s[1];
        s[1] ^= s[2];
        s[0] ^= s[3];
        s[2] ^= t;
        s[3] = rotl(s[3], 45);
        return r;
    }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

int orbital_dims(const bps_bank_spec& sp) { return sp.ecc_max > 0.0 ? 5 : 3; }

double tau_bound(const bps_bank_spec& sp, double porb)
{
    if (sp.tau_max_lts > 0.0) return sp.tau_max_lts;
    // tau_max = G^(1/3) Omega^(-2/3) m_c / (c (m_p + m_c)^(2/3))  (Table 1)
    const double om = kTwoPi / porb;
    const double mc = sp.m_comp_max_msun * kMsun, mp = sp.m_pulsar_min_msun * kMsun;
    return std::cbrt(kGNewton) * std::pow(om, -2.0 / 3.0) * mc / (kLight * std::pow(mp + mc, 2.0 / 3.0));
}

// Eccentric anomaly: Newton from E0 = M + e sin M (|dE| < 1e-15, at most 50 steps).
double kepler(double M, double e)
{
    double E = M + e * std::sin(M);
    for (int i = 0; i < 50; ++i) {
        const double d = (E - e * std::sin(E) - M) / (1.0 - e * std::cos(E));
        E -= d;
        if (std::fabs(d) < 1e-15) break;
    }
    return E;
}

// Phase derivatives d Phi / d lambda, lambda = (f0, tau, Omega, alpha[, omega, e]), at the
// n_time midpoint sample times of [0, T], into A column-major (A[c * n_time + i]).
void phase_derivatives(const bps_bank_spec& sp, const bps_template& t, std::vector<double>& A)
{
    const int n = orbital_dims(sp);
    const int nt = sp.n_time;
    const double f0 = sp.f_max_hz, T = sp.tobs_s;
    const double om = kTwoPi / t.porb_s, e = sp.ecc_max > 0.0 ? t.ecc : 0.0;
    const double w = sp.ecc_max > 0.0 ? t.omega_rad : 0.0;
    const double sq = std::sqrt(1.0 - e * e), sw = std::sin(w), cw = std::cos(w);
    A.assign((size_t)nt * (n + 1), 0.0);
    for (int i = 0; i < nt; ++i) {
        const double tt = (i + 0.5) * T / nt;
        const double E = kepler(om * tt + t.phi_rad, e);  // M = Omega t + alpha
        const double cE = std::cos(E), sE = std::sin(E);
        const double shape = (cE - e) * sw + sq * sE * cw;  // Delta / tau
        const double dD_dE = t.tau_lts * (-sE * sw + sq * cE * cw);
        const double dE_dM = 1.0 / (1.0 - e * cE);
        // Phi = 2 pi f0 (t - Delta)
        A[0 * (size_t)nt + i] = kTwoPi * (tt - t.tau_lts * shape);
        A[1 * (size_t)nt + i] = -kTwoPi * f0 * shape;
        A[2 * (size_t)nt + i] = -kTwoPi * f0 * dD_dE * dE_dM * tt;  // Omega
        A[3 * (size_t)nt + i] = -kTwoPi * f0 * dD_dE * dE_dM;       // alpha
        if (n == 5) {
            const double dD_dw = t.tau_lts * ((cE - e) * cw - sq * sE * sw);
            const double dD_de = t.tau_lts * (-sw - (e / sq) * sE * cw) + dD_dE * sE * dE_dM;
            A[4 * (size_t)nt + i] = -kTwoPi * f0 * dD_dw;
            A[5 * (size_t)nt + i] = -kTwoPi * f0 * dD_de;
        }
    }
}

// Frequency-projected metric gamma (n x n, orbital coordinates tau, Omega, alpha[, omega,
// e]) of the template (porb, tau, alpha, omega, e) at f0 = f_max.
void projected_metric(const bps_bank_spec& sp, const bps_template& t, std::vector<double>& gam)
{
    const int n = orbital_dims(sp);
    const int d = n + 1;  // with f0 first
    const int nt = sp.n_time;
    std::vector<double> A;
    phase_derivatives(sp, t, A);
    std::vector<double> mean((size_t)d, 0.0), g((size_t)d * d, 0.0);
    for (int a = 0; a < d; ++a)
        for (int i = 0; i < nt; ++i) mean[a] += A[(size_t)a * nt + i] / nt;
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
            double acc = 0.0;
            for (int i = 0; i < nt; ++i)
                acc += (A[(size_t)a * nt + i] - mean[a]) * (A[(size_t)b * nt + i] - mean[b]);
            g[a * d + b] = acc / nt;
        }
    gam.assign((size_t)n * n, 0.0);
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b)
            gam[a * n + b] = g[(a + 1) * d + (b + 1)] - g[(a + 1) * d] * g[(b + 1) * d] / g[0];
}

// sqrt(det gamma) without forming the metric: with D the n_time x (n+1) matrix of the
// phase derivatives at the sample times, columns centred (f0 first), g = D^T D / n_time
// and det gamma = det g / g_ff (gamma is the Schur complement of g_ff).  det g comes
// from a Householder QR of D with unit-norm columns (|det R| times the column norms),
// which keeps the accuracy of the small directions: for observations much shorter than
// the orbit g spans 15+ orders of magnitude and its determinant is lost in rounding.
double density(const bps_bank_spec& sp, const bps_template& t)
{
    const int n = orbital_dims(sp);
    const int d = n + 1;
    const int nt = sp.n_time;
    std::vector<double> A((size_t)nt * d);  // column-major: A[c * nt + i]
    phase_derivatives(sp, t, A);
    double logdet = 0.0;  // log det(D^T D)
    std::vector<double> norm((size_t)d);
    for (int c = 0; c < d; ++c) {
        double* col = &A[(size_t)c * nt];
        double m = 0.0;
        for (int i = 0; i < nt; ++i) m += col[i];
        m /= nt;
        double s2 = 0.0;
        for (int i = 0; i < nt; ++i) {
            col[i] -= m;
            s2 += col[i] * col[i];
        }
        if (!(s2 > 0.0)) return 0.0;
        norm[c] = std::sqrt(s2);
        for (int i = 0; i < nt; ++i) col[i] /= norm[c];
        logdet += 2.0 * std::log(norm[c]);
    }
    const double gff = norm[0] * norm[0] / nt;
    // Householder QR of the normalised columns: |det R| = prod |R_cc|
    for (int c = 0; c < d; ++c) {
        double* col = &A[(size_t)c * nt];
        double s2 = 0.0;
        for (int i = c; i < nt; ++i) s2 += col[i] * col[i];
        const double alpha = col[c] > 0.0 ? -std::sqrt(s2) : std::sqrt(s2);
        if (alpha == 0.0) return 0.0;
        logdet += 2.0 * std::log(std::fabs(alpha));
        // v = x - alpha e_c, stored in col[c..]; H = I - 2 v v^T / (v^T v)
        col[c] -= alpha;
        double vv = 0.0;
        for (int i = c; i < nt; ++i) vv += col[i] * col[i];
        if (vv == 0.0) continue;
        for (int k = c + 1; k < d; ++k) {
            double* ck = &A[(size_t)k * nt];
            double dot = 0.0;
            for (int i = c; i < nt; ++i) dot += col[i] * ck[i];
            const double f = 2.0 * dot / vv;
            for (int i = c; i < nt; ++i) ck[i] -= f * col[i];
        }
    }
    // det g = det(D^T D) / nt^d; det gamma = det g / g_ff
    const double lg = logdet - d * std::log((double)nt) - std::log(gff);
    return std::exp(0.5 * lg);
}

// dens[i] = density(ts[i]) * jac[i] for all i, on the host's cores (fixed split, so the
// result does not depend on scheduling)
void densities(const bps_bank_spec& sp, const std::vector<bps_template>& ts,
               const std::vector<double>& jac, std::vector<double>& dens)
{
    const size_t n = ts.size();
    dens.assign(n, 0.0);
    const unsigned hw = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
    const size_t nth = std::min<size_t>(hw, std::max<size_t>(1, n / 64));
    std::vector<std::thread> pool;
    for (size_t w = 0; w < nth; ++w)
        pool.emplace_back([&, w]() {
            for (size_t i = w; i < n; i += nth) dens[i] = density(sp, ts[i]) * jac[i];
        });
    for (auto& th : pool) th.join();
}

bool spec_ok(const bps_bank_spec* sp)
{
    return sp && sp->tobs_s > 0.0 && sp->f_max_hz > 0.0 && sp->mismatch > 0.0 && sp->mismatch < 1.0 &&
           sp->coverage > 0.0 && sp->coverage < 1.0 && sp->porb_min_s > 0.0 &&
           sp->porb_max_s >= sp->porb_min_s && sp->tau_max_lts >= 0.0 &&
           (sp->tau_max_lts > 0.0 || (sp->m_pulsar_min_msun > 0.0 && sp->m_comp_max_msun > 0.0)) &&
           sp->ecc_max >= 0.0 && sp->ecc_max < 1.0 && sp->n_time >= 16 && sp->n_volume >= 100;
}

// A uniform point of the bounding box; false when it falls outside the prior region
// (tau above tau_max(P_orb)).  *jac = |dOmega/dP_orb|.
bool draw_box(const bps_bank_spec& sp, double tau_top, Rng& rng, bps_template& t, double* jac)
{
    t.porb_s = sp.porb_min_s + (sp.porb_max_s - sp.porb_min_s) * rng.uniform();
    t.tau_lts = tau_top * rng.uniform();
    t.phi_rad = kTwoPi * rng.uniform();
    t.omega_rad = sp.ecc_max > 0.0 ? kTwoPi * rng.uniform() : 0.0;
    t.ecc = sp.ecc_max > 0.0 ? sp.ecc_max * rng.uniform() : 0.0;
    *jac = kTwoPi / (t.porb_s * t.porb_s);
    return t.tau_lts <= tau_bound(sp, t.porb_s);
}

// Upper end of the bounding box in tau (tau_max grows with P_orb as Omega^(-2/3)).
double tau_top(const bps_bank_spec& sp)
{
    return std::fmax(tau_bound(sp, sp.porb_min_s), tau_bound(sp, sp.porb_max_s));
}

double box_volume(const bps_bank_spec& sp, double top)
{
    double v = (sp.porb_max_s - sp.porb_min_s) * top * kTwoPi;
    if (sp.ecc_max > 0.0) v *= kTwoPi * sp.ecc_max;
    return v;
}

}  // namespace

extern "C" {

void bps_default_bank_spec(bps_bank_spec* sp)
{
    if (!sp) return;
    sp->tobs_s = 1.2 * 3600.0;  // Table 1
    sp->f_max_hz = 66.67;
    sp->mismatch = 0.2;
    sp->coverage = 0.9;
    sp->porb_min_s = 6.0 * 3600.0;
    sp->porb_max_s = 12.0 * 3600.0;
    sp->tau_max_lts = 0.0;
    sp->m_pulsar_min_msun = 1.4;
    sp->m_comp_max_msun = 8.0;
    sp->ecc_max = 0.1;
    sp->n_time = 256;
    sp->n_volume = 20000;
}

int bps_metric_density(const bps_bank_spec* spec, const bps_template* t, int64_t count,
                       double* sqrt_det_out)
{
    if (!spec_ok(spec) || (count > 0 && (!t || !sqrt_det_out)) || count < 0) return BPS_ERR_INVALID_ARG;
    try {
        for (int64_t i = 0; i < count; ++i) {
            if (!(t[i].porb_s > 0.0) || !(t[i].tau_lts >= 0.0) || !(t[i].ecc >= 0.0 && t[i].ecc < 1.0))
                return BPS_ERR_INVALID_ARG;
            sqrt_det_out[i] = density(*spec, t[i]);
        }
    } catch (...) {
        return BPS_ERR_OUT_OF_MEMORY;
    }
    return BPS_OK;
}

int bps_metric_projected(const bps_bank_spec* spec, const bps_template* t, double* gamma_out)
{
    if (!spec_ok(spec) || !t || !gamma_out || !(t->porb_s > 0.0)) return BPS_ERR_INVALID_ARG;
    try {
        std::vector<double> gam;
        projected_metric(*spec, *t, gam);
        for (size_t i = 0; i < gam.size(); ++i) gamma_out[i] = gam[i];
    } catch (...) {
        return BPS_ERR_OUT_OF_MEMORY;
    }
    return BPS_OK;
}

namespace {
int metric_bank_impl(const bps_bank_spec* spec, uint64_t seed, bps_template* out, int64_t cap,
                     int64_t* n_out, double* proper_volume, double* n_expected)
{
    const bps_bank_spec& sp = *spec;
    const int n = orbital_dims(sp);
    Rng rng(seed);
    const double top = tau_top(sp);
    // proper volume by Monte Carlo over the bounding box (points outside the prior region
    // count zero), and the largest sampled density
    std::vector<bps_template> ts((size_t)sp.n_volume);
    std::vector<double> jac((size_t)sp.n_volume), dens;
    for (int i = 0; i < sp.n_volume; ++i)
        if (!draw_box(sp, top, rng, ts[i], &jac[i])) jac[i] = 0.0;
    densities(sp, ts, jac, dens);
    double acc = 0.0, dmax = 0.0;
    for (double v : dens) {
        acc += v;
        dmax = std::fmax(dmax, v);
    }
    const double V = box_volume(sp, top) * acc / sp.n_volume;
    const double Cn = std::pow(kPi, 0.5 * n) / std::tgamma(0.5 * n + 1.0);
    const double x = std::pow(sp.mismatch, 0.5 * n) * Cn / V;
    const double NR = (x > 0.0 && x < 1.0) ? std::log(1.0 - sp.coverage) / std::log1p(-x) : 1.0;
    if (proper_volume) *proper_volume = V;
    if (n_expected) *n_expected = NR;
    const int64_t N = (int64_t)std::ceil(NR);
    *n_out = N;
    if (cap == 0 && !out) return BPS_OK;  // count only
    if (N > cap) return BPS_ERR_CAND_OVERFLOW;
    // rejection sampling with density sqrt(det gamma) |dOmega/dP_orb| over the prior
    // region, in batches evaluated in parallel and accepted in draw order; the bound is
    // twice the sampled maximum (a denser draw raises it)
    double bound = 2.0 * dmax;
    const size_t B = 4096;
    std::vector<double> uacc(B);
    ts.resize(B);
    jac.resize(B);
    for (int64_t k = 0; k < N;) {
        for (size_t i = 0; i < B; ++i) {
            if (!draw_box(sp, top, rng, ts[i], &jac[i])) jac[i] = 0.0;
            uacc[i] = rng.uniform();
        }
        densities(sp, ts, jac, dens);
        for (size_t i = 0; i < B && k < N; ++i) {
            if (dens[i] > bound) bound = dens[i];
            if (uacc[i] * bound < dens[i]) out[k++] = ts[i];
        }
    }
    return BPS_OK;
}
}  // namespace

int bps_metric_bank(const bps_bank_spec* spec, uint64_t seed, bps_template* out, int64_t cap,
                    int64_t* n_out, double* proper_volume, double* n_expected)
{
    if (!spec_ok(spec) || !n_out || cap < 0 || (cap > 0 && !out)) return BPS_ERR_INVALID_ARG;
    try {
        return metric_bank_impl(spec, seed, out, cap, n_out, proper_volume, n_expected);
    } catch (...) {  // allocation or thread creation failed
        return BPS_ERR_OUT_OF_MEMORY;
    }
}

}  // extern "C"
