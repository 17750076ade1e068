// dev_template.h -- host construction of the device form of orbital templates:
// the parameters of bps_template plus the per-template FP64 constants the anchor kernel
// reads (shared by the runtime and the allocation-free entry point).
#pragma once

#include <cmath>
#include <vector>

#include "../../include/bps.h"
#include "bps_internal.cuh"

namespace bps {
namespace rt {

// Kepler's equation E - e sin E = M by FP64 Newton iteration from E0 = M + e sin M (the
// anchor kernel's iteration, here for the zero offset of dev_template).
inline double kepler_host(double M, double e)
{
    double E = M + e * std::sin(M);
    for (int it = 0; it < 40; ++it) {
        const double dE = (E - e * std::sin(E) - M) / (1.0 - e * std::cos(E));
        E -= dE;
        if (std::fabs(dE) < 1e-15) break;
    }
    return E;
}

// The device form of a template: its parameters and the per-template constants of the
// anchor kernel in FP64 (the BT delay at t = 0, M = alpha reduced to [0, 2 pi)).
inline DevTemplate dev_template(const bps_template& t)
{
    constexpr double kTwoPiH = 6.283185307179586476925286766559;
    DevTemplate d;
    d.porb = t.porb_s;
    d.tau = t.tau_lts;
    d.phi = t.phi_rad;
    d.omega = t.omega_rad;
    d.ecc = t.ecc;
    d.om = kTwoPiH / t.porb_s;
    d.sw = std::sin(t.omega_rad);
    d.cw = std::cos(t.omega_rad);
    d.rt = std::sqrt(1.0 - t.ecc * t.ecc);
    double M0 = t.phi_rad - kTwoPiH * std::floor(t.phi_rad / kTwoPiH);
    if (M0 < 0.0) M0 += kTwoPiH;
    if (M0 >= kTwoPiH) M0 -= kTwoPiH;
    const double E0 = kepler_host(M0, t.ecc);
    d.delta0 = t.tau_lts * ((std::cos(E0) - t.ecc) * d.sw + d.rt * std::sin(E0) * d.cw);
    return d;
}

inline std::vector<DevTemplate> dev_templates(const bps_template* t, int64_t count)
{
    std::vector<DevTemplate> v((size_t)count);
    for (int64_t i = 0; i < count; ++i) v[(size_t)i] = dev_template(t[i]);
    return v;
}

}  // namespace rt
}  // namespace bps
