// Closed-form phase functions (Scenario 1 of Table 1) evaluated in FP64.
//
// FIO2D is Example 1 of Sec. 4: Phi = x.xi + sqrt(c1(x)^2 xi1^2 + c2(x)^2 xi2^2)
// with c1 = (2 + sin 2pi x1 sin 2pi x2)/16 and c2 = (2 + cos 2pi x1 cos 2pi x2)/16.
// FIO3D uses c_k = (2 + sin 2pi x_k cos 2pi x_{k+1})/16 (cyclic); FIO2D_JUMP adds
// 0.5 |xi| sign(x1 - 0.5) with sign(0) = +1 (one discontinuity, allowed by the
// piecewise-smooth setting of eq. (1)); DOT is the Fourier phase of Example 2;
// DISTANCE is |x - xi|, the Helmholtz phase h |x - xi| of Example 3 once the
// points are scaled by h.
#include "internal.hpp"

namespace midbf {

double Phase::eval_xy(const double* x, const double* w) const {
    const double twopi = 2.0 * M_PI;
    double dot = 0.0;
    for (int k = 0; k < d; ++k) dot += x[k] * w[k];
    switch (family) {
        case MIDBF_PHASE_DOT:
            return dot;
        case MIDBF_PHASE_ZERO:
            return 0.0;
        case MIDBF_PHASE_DISTANCE: {
            double s = 0.0;
            for (int k = 0; k < d; ++k) s += (x[k] - w[k]) * (x[k] - w[k]);
            return std::sqrt(s);
        }
        case MIDBF_PHASE_SEPARABLE: {
            double a = 0.0, b = 0.0;
            for (int k = 0; k < d; ++k) {
                a += std::sin(twopi * x[k]);
                b += w[k] * w[k];
            }
            return a + 0.05 * b;
        }
        case MIDBF_PHASE_FIO2D:
        case MIDBF_PHASE_FIO2D_JUMP: {
            double s1 = std::sin(twopi * x[0]), s2 = std::sin(twopi * x[1]);
            double c1x = std::cos(twopi * x[0]), c2x = std::cos(twopi * x[1]);
            double c1 = (2.0 + s1 * s2) / 16.0;
            double c2 = (2.0 + c1x * c2x) / 16.0;
            double v = dot + std::sqrt(c1 * c1 * w[0] * w[0] + c2 * c2 * w[1] * w[1]);
            if (family == MIDBF_PHASE_FIO2D_JUMP) {
                double sg = (x[0] - 0.5 >= 0.0) ? 1.0 : -1.0;
                v += 0.5 * std::sqrt(w[0] * w[0] + w[1] * w[1]) * sg;
            }
            return v;
        }
        case MIDBF_PHASE_FIO3D: {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) {
                double ck = (2.0 + std::sin(twopi * x[k]) * std::cos(twopi * x[(k + 1) % 3])) / 16.0;
                acc += ck * ck * w[k] * w[k];
            }
            return dot + std::sqrt(acc);
        }
        default:
            fail(MIDBF_EINVAL, "unknown phase family " + std::to_string(family));
    }
}

namespace {

inline cplx unit(double p) {
    p -= std::nearbyint(p);
    double s, c;
    sincos(2.0 * M_PI * p, &s, &c);
    return cplx(c, s);
}

}  // namespace

void Phase::kernel_block(const int64_t* xi, size_t na, const int64_t* wj, size_t nb, cplx* out, size_t sx,
                         size_t sw) const {
    const double twopi = 2.0 * M_PI;
    auto xp = [&](size_t a) { return &X[(size_t)xi[a] * d]; };
    auto wp = [&](size_t b) { return &W[(size_t)wj[b] * d]; };
    auto dot = [&](const double* x, const double* w) {
        double s = 0.0;
        for (int k = 0; k < d; ++k) s += x[k] * w[k];
        return s;
    };
    switch (family) {
        case MIDBF_PHASE_FIO2D:
        case MIDBF_PHASE_FIO2D_JUMP: {
            // per row: c1^2, c2^2 (and the sign of x1 - 1/2); per column: |xi| / 2
            const bool jump = family == MIDBF_PHASE_FIO2D_JUMP;
            std::vector<double> c1s(na), c2s(na), sg(na), hn(jump ? nb : 0);
            for (size_t a = 0; a < na; ++a) {
                const double* x = xp(a);
                const double c1 = (2.0 + std::sin(twopi * x[0]) * std::sin(twopi * x[1])) / 16.0;
                const double c2 = (2.0 + std::cos(twopi * x[0]) * std::cos(twopi * x[1])) / 16.0;
                c1s[a] = c1 * c1;
                c2s[a] = c2 * c2;
                sg[a] = (x[0] - 0.5 >= 0.0) ? 1.0 : -1.0;
            }
            for (size_t b = 0; b < (jump ? nb : 0); ++b) {
                const double* w = wp(b);
                hn[b] = 0.5 * std::sqrt(w[0] * w[0] + w[1] * w[1]);
            }
            for (size_t b = 0; b < nb; ++b) {
                const double* w = wp(b);
                for (size_t a = 0; a < na; ++a) {
                    double v = dot(xp(a), w) + std::sqrt(c1s[a] * w[0] * w[0] + c2s[a] * w[1] * w[1]);
                    if (jump) v += hn[b] * sg[a];
                    out[a * sx + b * sw] = unit(v);
                }
            }
            return;
        }
        case MIDBF_PHASE_FIO3D: {
            std::vector<double> cs(na * 3);
            for (size_t a = 0; a < na; ++a) {
                const double* x = xp(a);
                for (int k = 0; k < 3; ++k) {
                    const double ck = (2.0 + std::sin(twopi * x[k]) * std::cos(twopi * x[(k + 1) % 3])) / 16.0;
                    cs[a * 3 + k] = ck * ck;
                }
            }
            for (size_t b = 0; b < nb; ++b) {
                const double* w = wp(b);
                for (size_t a = 0; a < na; ++a) {
                    double acc = 0.0;
                    for (int k = 0; k < 3; ++k) acc += cs[a * 3 + k] * w[k] * w[k];
                    out[a * sx + b * sw] = unit(dot(xp(a), w) + std::sqrt(acc));
                }
            }
            return;
        }
        case MIDBF_PHASE_SEPARABLE: {
            std::vector<double> ra(na), cb(nb);
            for (size_t a = 0; a < na; ++a) {
                double s = 0.0;
                for (int k = 0; k < d; ++k) s += std::sin(twopi * xp(a)[k]);
                ra[a] = s;
            }
            for (size_t b = 0; b < nb; ++b) {
                double s = 0.0;
                for (int k = 0; k < d; ++k) s += wp(b)[k] * wp(b)[k];
                cb[b] = s;
            }
            for (size_t b = 0; b < nb; ++b)
                for (size_t a = 0; a < na; ++a) out[a * sx + b * sw] = unit(ra[a] + 0.05 * cb[b]);
            return;
        }
        default:
            for (size_t b = 0; b < nb; ++b)
                for (size_t a = 0; a < na; ++a) out[a * sx + b * sw] = kernel(xi[a], wj[b]);
    }
}

void phase_check(const Phase& ph) {
    if (ph.d != 2 && ph.d != 3) fail(MIDBF_EINVAL, "d must be 2 or 3");
    if (ph.nx <= 0 || ph.nw <= 0) fail(MIDBF_EINVAL, "empty point set");
    if ((int64_t)ph.X.size() != ph.nx * ph.d || (int64_t)ph.W.size() != ph.nw * ph.d)
        fail(MIDBF_EINVAL, "coordinate arrays have the wrong size");
    switch (ph.family) {
        case MIDBF_PHASE_FIO2D:
        case MIDBF_PHASE_FIO2D_JUMP:
            if (ph.d != 2) fail(MIDBF_EINVAL, "FIO2D phases need d = 2");
            break;
        case MIDBF_PHASE_FIO3D:
            if (ph.d != 3) fail(MIDBF_EINVAL, "FIO3D phase needs d = 3");
            break;
        case MIDBF_PHASE_DOT:
        case MIDBF_PHASE_ZERO:
        case MIDBF_PHASE_SEPARABLE:
        case MIDBF_PHASE_DISTANCE:
            break;
        case MIDBF_PHASE_LOWRANK:
            if (ph.r <= 0 || (int64_t)ph.U.size() != ph.nx * ph.r || (int64_t)ph.V.size() != ph.nw * ph.r)
                fail(MIDBF_EINVAL, "low-rank phase factors have the wrong size");
            break;
        default:
            fail(MIDBF_EINVAL, "unknown phase family " + std::to_string(ph.family));
    }
    for (double v : ph.U)
        if (!std::isfinite(v)) fail(MIDBF_EINVAL, "non-finite low-rank factor U");
    for (double v : ph.V)
        if (!std::isfinite(v)) fail(MIDBF_EINVAL, "non-finite low-rank factor V");
    for (double v : ph.X)
        if (!std::isfinite(v)) fail(MIDBF_EINVAL, "non-finite coordinate in X");
    for (double v : ph.W)
        if (!std::isfinite(v)) fail(MIDBF_EINVAL, "non-finite coordinate in W");
}

}  // namespace midbf
