// Ohmic bath rates and Lamb shift (arXiv:1710.03431, Sec. V and Sec. II/App. E).
//
// gamma(w) = 2 pi eta_g2 w e^{-|w|/w_c} / (1 - e^{-beta w}), gamma(0) = 2 pi eta_g2 / beta;
// it satisfies the KMS condition gamma(-w) = e^{-beta w} gamma(w) (Sec. II, Eq. KMS).
// S(w) = (1/2pi) P int gamma(x) / (w - x) dx, the principal-value partner of
// gamma in the one-sided bath correlation integral; the paper names H_LS but
// does not write S out.
//
// S is tabulated once per bath on three uniform zones (finer near w = 0, where
// the kink of gamma at 0 gives S logarithmic curvature) and read back with
// four-point Lagrange interpolation. Each node is an adaptive Gauss-Legendre
// quadrature of the pole-subtracted integrand
//   P int_{-L}^{L} g(x)/(w-x) dx = int (g(x)-g(w))/(w-x) dx + g(w) ln((L+w)/(L-w)).
#include "aqt_internal.h"

#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

namespace aqt {

double Bath::gamma(double w) const {
    if (w == 0.0) return 2.0 * M_PI * eta_g2 / beta;
    // w / (1 - e^{-beta w}) = w / (-expm1(-beta w)); for large negative w the
    // denominator overflows to -inf and gamma underflows to 0 as it should.
    const double den = -std::expm1(-beta * w);
    return 2.0 * M_PI * eta_g2 * w * std::exp(-std::fabs(w) / omega_c) / den;
}

// d gamma / dw for w != 0: gamma = 2 pi eta_g2 q(w) e^{-|w|/w_c} with
// q(w) = w / (1 - e^{-beta w}); q'(w) = (1 - e^{-x} (1 + x)) / (1 - e^{-x})^2,
// x = beta w, written for x < 0 as e^x (e^x - 1 - x) / (e^x - 1)^2 so that
// neither form overflows, and as its Taylor series 1/2 + x/6 - x^3/180 for
// |x| < 1e-4 (where the closed form cancels).
double Bath::gamma_deriv(double w) const {
    const double x = beta * w;
    double dq;
    if (std::fabs(x) < 1e-4) {
        dq = 0.5 + x / 6.0 - x * x * x / 180.0;  // series of d/dx [x / (1 - e^{-x})]
    } else if (x >= 0.0) {
        const double em = -std::expm1(-x);  // 1 - e^{-x}
        dq = (em - x * std::exp(-x)) / (em * em);
    } else {
        const double ep = std::expm1(x);  // e^x - 1
        dq = std::exp(x) * (ep - x) / (ep * ep);
    }
    const double q = w / (-std::expm1(-x));
    const double e = std::exp(-std::fabs(w) / omega_c);
    const double sgn = w > 0.0 ? 1.0 : -1.0;
    return 2.0 * M_PI * eta_g2 * e * (dq - sgn * q / omega_c);
}

double Bath::lamb_deriv(double w) const {
    if (!lamb_shift) return 0.0;
    const double h = 1e-5 * std::max(1.0, std::fabs(w));
    return (lamb(w + h) - lamb(w - h)) / (2.0 * h);
}

namespace {

// 15-point Gauss-Legendre nodes/weights on [-1, 1], computed by Newton
// iteration on P_15 at start-up (no stored constants).
struct GL {
    static constexpr int n = 15;
    double x[n], w[n];
    GL() {
        for (int i = 0; i < n; ++i) {
            double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
            double dp = 0.0;
            for (int it = 0; it < 100; ++it) {
                double p0 = 1.0, p1 = z;
                for (int k = 2; k <= n; ++k) {
                    const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                    p0 = p1;
                    p1 = p2;
                }
                dp = n * (z * p1 - p0) / (z * z - 1.0);
                const double dz = p1 / dp;
                z -= dz;
                if (std::fabs(dz) < 1e-16) break;
            }
            x[i] = z;
            w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
        }
    }
};

const GL &gl() {
    static const GL g;
    return g;
}

template <class F>
double gl_panel(const F &f, double a, double b) {
    const GL &g = gl();
    const double c = 0.5 * (a + b), h = 0.5 * (b - a);
    double acc = 0.0;
    for (int i = 0; i < GL::n; ++i) acc += g.w[i] * f(c + h * g.x[i]);
    return acc * h;
}

// Bisect a panel until the 15-point rule agrees with its two halves to a
// relative 1e-13 (or an absolute floor); at most `depth` levels, so the cost
// is bounded even where rounding noise (next to the removed pole) never settles.
template <class F>
double adaptive(const F &f, double a, double b, double whole, double abs_tol, int depth) {
    const double m = 0.5 * (a + b);
    const double left = gl_panel(f, a, m), right = gl_panel(f, m, b);
    const double sum = left + right;
    if (depth <= 0 || std::fabs(sum - whole) <= std::max(abs_tol, 1e-13 * std::fabs(sum))) return sum;
    return adaptive(f, a, m, left, 0.5 * abs_tol, depth - 1) + adaptive(f, m, b, right, 0.5 * abs_tol, depth - 1);
}

}  // namespace

double Bath::lamb_direct(double w) const {
    const double L = 60.0 * omega_c;  // tail beyond: below 1e-22 of the peak
    const double gw = gamma(w);
    auto f = [&](double x) {
        const double d = w - x;
        if (d == 0.0) return 0.0;
        return (gamma(x) - gw) / d;
    };
    // panel edges: the (removed) pole, the kink at 0, and a geometric ladder
    std::vector<double> edges = {-L, L, 0.0};
    for (double r : {0.05, 0.5, 2.0, 8.0, 1.0 * omega_c, 4.0 * omega_c, 15.0 * omega_c}) {
        edges.push_back(r);
        edges.push_back(-r);
    }
    if (w > -L && w < L) edges.push_back(w);
    std::sort(edges.begin(), edges.end());
    double total = 0.0;
    for (size_t i = 0; i + 1 < edges.size(); ++i) {
        const double a = edges[i], b = edges[i + 1];
        if (b - a <= 0.0) continue;
        total += adaptive(f, a, b, gl_panel(f, a, b), 1e-16, 12);
    }
    total += gw * std::log((L + w) / (L - w));
    return total / (2.0 * M_PI);
}

void Bath::build_lamb(double wmax) {
    zones.clear();
    if (!lamb_shift) return;
    // (half-width, spacing) of each zone
    const double spec[3][2] = {{0.05, 2.5e-4}, {10.0, 0.01}, {std::max(wmax, 10.0), 0.1}};
    for (auto &zs : spec) {
        Zone z;
        z.h = zs[1];
        z.half = zs[0];
        z.n0 = (int)std::ceil(z.half / z.h) + 3;  // nodes k = -n0..n0, node k at k*h
        z.val.assign(2 * z.n0 + 1, 0.0);
        zones.push_back(std::move(z));
    }
    // evaluate all nodes in parallel
    std::vector<std::pair<int, int>> jobs;
    for (int zi = 0; zi < (int)zones.size(); ++zi)
        for (int k = 0; k < (int)zones[zi].val.size(); ++k) jobs.push_back({zi, k});
    unsigned nt = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t) {
        th.emplace_back([&, t] {
            for (size_t j = t; j < jobs.size(); j += nt) {
                Zone &z = zones[jobs[j].first];
                const double w = (jobs[j].second - z.n0) * z.h;
                z.val[jobs[j].second] = lamb_direct(w);
            }
        });
    }
    for (auto &x : th) x.join();
}

void Bath::rates(double w, double *g, double *dg, double *s, double *ds) const {
    *g = gamma(w);
    *dg = w == 0.0 ? 0.0 : gamma_deriv(w);
    *s = 0.0;
    *ds = 0.0;
    if (!lamb_shift) return;
    for (const Zone &z : zones) {
        if (std::fabs(w) > z.half) continue;
        const double u = w / z.h;
        const int k = (int)std::floor(u);
        const double t = u - k;
        const double *v = &z.val[k + z.n0 - 1];
        // the Lagrange interpolant of lamb() and its derivative in t (nodes -1, 0, 1, 2)
        const double l0 = -t * (t - 1.0) * (t - 2.0) / 6.0;
        const double l1 = (t + 1.0) * (t - 1.0) * (t - 2.0) / 2.0;
        const double l2 = -(t + 1.0) * t * (t - 2.0) / 2.0;
        const double l3 = (t + 1.0) * t * (t - 1.0) / 6.0;
        const double d0 = -(3.0 * t * t - 6.0 * t + 2.0) / 6.0;
        const double d1 = (3.0 * t * t - 4.0 * t - 1.0) / 2.0;
        const double d2 = -(3.0 * t * t - 2.0 * t - 2.0) / 2.0;
        const double d3 = (3.0 * t * t - 1.0) / 6.0;
        *s = l0 * v[0] + l1 * v[1] + l2 * v[2] + l3 * v[3];
        *ds = (d0 * v[0] + d1 * v[1] + d2 * v[2] + d3 * v[3]) / z.h;
        return;
    }
    *s = lamb_direct(w);
    *ds = lamb_deriv(w);
}

double Bath::lamb(double w) const {
    if (!lamb_shift) return 0.0;
    for (const Zone &z : zones) {
        if (std::fabs(w) > z.half) continue;
        const double u = w / z.h;
        int k = (int)std::floor(u);  // stencil k-1..k+2
        const double t = u - k;
        const double *v = &z.val[k + z.n0 - 1];
        // Lagrange weights for nodes at -1, 0, 1, 2
        const double l0 = -t * (t - 1.0) * (t - 2.0) / 6.0;
        const double l1 = (t + 1.0) * (t - 1.0) * (t - 2.0) / 2.0;
        const double l2 = -(t + 1.0) * t * (t - 2.0) / 2.0;
        const double l3 = (t + 1.0) * t * (t - 1.0) / 6.0;
        return l0 * v[0] + l1 * v[1] + l2 * v[2] + l3 * v[3];
    }
    return lamb_direct(w);  // outside the table: direct quadrature
}

}  // namespace aqt
