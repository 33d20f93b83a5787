// Lowest eigenpairs of the transverse-field Ising Hamiltonian without forming
// it, in FP64, for the truncated model that keeps the lowest levels of a
// system too large to diagonalise densely (the paper's 16-qubit example,
// Sec. V.C, is the use).
//
// H = A (-sum_i sx_i) + B diag(E_z), acting on a vector of 2^n amplitudes
// (basis index x, bit i = qubit i): (H v)[x] = B E_z[x] v[x] - A sum_i v[x ^ 2^i].
//
// Method: Chebyshev-filtered subspace iteration with Rayleigh-Ritz (the
// published scheme of Zhou and Saad): a block of p vectors is multiplied by
// the Chebyshev polynomial of degree d of H that is bounded by 1 on the
// unwanted interval [a, b] (a: the largest Ritz value of the block, b: an
// upper bound of the spectrum) and grows fast below a, so each pass damps
// the unwanted part of the block by the polynomial's growth ratio; the
// filtered block is orthonormalised (two Gram-Schmidt passes) and the Ritz
// pairs of H on it replace it. Converged when the residuals |H x - theta x|
// of the wanted pairs are below tol. A warm start (the previous grid point's
// vectors) converges in a pass or two; a cold start uses fixed pseudo-random
// vectors.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "aqt_internal.h"

namespace aqt {

namespace {

// y = H v for one vector of D = 2^n amplitudes
void apply_h(int n, double A, double B, const double *Ez, const double *v, double *y) {
    const size_t D = (size_t)1 << n;
    for (size_t x = 0; x < D; ++x) {
        double acc = B * Ez[x] * v[x];
        for (int i = 0; i < n; ++i) acc -= A * v[x ^ ((size_t)1 << i)];
        y[x] = acc;
    }
}

double dot(const double *a, const double *b, size_t D) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    size_t i = 0;
    for (; i + 4 <= D; i += 4) {
        s0 += a[i] * b[i];
        s1 += a[i + 1] * b[i + 1];
        s2 += a[i + 2] * b[i + 2];
        s3 += a[i + 3] * b[i + 3];
    }
    for (; i < D; ++i) s0 += a[i] * b[i];
    return (s0 + s1) + (s2 + s3);
}

void axpy(double a, const double *x, double *y, size_t D) {
    for (size_t i = 0; i < D; ++i) y[i] += a * x[i];
}

// Orthogonalise v against the first k vectors of Z (vector-major, D each) with
// two classical Gram-Schmidt passes, then normalise; false if v lies in their
// span (relative norm below 1e-10).
bool orth_against(const std::vector<double> &Z, int k, double *v, size_t D) {
    const double n0 = std::sqrt(dot(v, v, D));
    if (!(n0 > 0.0)) return false;
    std::vector<double> c(k);
    for (int pass = 0; pass < 2; ++pass) {
        for (int j = 0; j < k; ++j) c[j] = dot(&Z[(size_t)j * D], v, D);
        for (int j = 0; j < k; ++j) axpy(-c[j], &Z[(size_t)j * D], v, D);
    }
    const double n1 = std::sqrt(dot(v, v, D));
    if (!(n1 > 1e-10 * n0)) return false;
    const double inv = 1.0 / n1;
    for (size_t i = 0; i < D; ++i) v[i] *= inv;
    return true;
}

// Fixed pseudo-random start vector j (splitmix64 of (x, j)), entries in [-1, 1).
double start_entry(size_t x, int j) {
    uint64_t z = (uint64_t)x * 0x9E3779B97F4A7C15ull + (uint64_t)(j + 1) * 0xD1B54A32D192ED03ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

}  // namespace

bool lowest_eigen(int n, double A, double B, const double *Ez, int p, int want, const double *X0, double *evals,
                  double *X, int *restarts, double *next_lower) {
    const size_t D = (size_t)1 << n;
    constexpr int kDegree = 16;
    constexpr int kMaxPasses = 300;
    if (p < want || (size_t)p > D || want < 1) return false;
    // upper bound of the spectrum (|H| <= |A| n + |B| max |E_z|), scale for the residual test
    double ez = 0.0;
    for (size_t x = 0; x < D; ++x) ez = std::max(ez, std::fabs(Ez[x]));
    const double hb = std::fabs(A) * n + std::fabs(B) * ez;
    const double tol = 1e-12 * std::max(1.0, hb);

    std::vector<double> Q((size_t)p * D), HQ((size_t)p * D), Y0((size_t)p * D), Y1((size_t)p * D), T, Yv, theta(p);
    auto fill = [&](const double *src) {
        for (int j = 0; j < p; ++j)
            for (size_t x = 0; x < D; ++x) Q[(size_t)j * D + x] = src ? src[(size_t)j * D + x] : start_entry(x, j);
    };
    // orthonormalise the block in place; dependent vectors are replaced by
    // pseudo-random ones (made orthogonal to the rest)
    auto orthonormalise = [&]() {
        for (int j = 0, salt = 0; j < p; ++j) {
            double *v = &Q[(size_t)j * D];
            int tries = 0;
            while (!orth_against(Q, j, v, D)) {
                if (++tries > 4) return false;
                for (size_t x = 0; x < D; ++x) v[x] = start_entry(x, p + 17 * (++salt) + j);
            }
        }
        return true;
    };
    // Rayleigh-Ritz on the orthonormal block: Q <- Q Y, HQ <- HQ Y, theta ascending;
    // returns the largest residual of the wanted pairs (the residual of the
    // pair after them goes to r_next)
    double r_next = INFINITY;
    auto rayleigh_ritz = [&]() -> double {
        for (int j = 0; j < p; ++j) apply_h(n, A, B, Ez, &Q[(size_t)j * D], &HQ[(size_t)j * D]);
        T.assign((size_t)p * p, 0.0);
        for (int i = 0; i < p; ++i)
            for (int j = i; j < p; ++j) {
                const double t = 0.5 * (dot(&Q[(size_t)i * D], &HQ[(size_t)j * D], D) +
                                        dot(&Q[(size_t)j * D], &HQ[(size_t)i * D], D));
                T[(size_t)i * p + j] = T[(size_t)j * p + i] = t;
            }
        Yv.assign((size_t)p * p, 0.0);
        if (!sym_eigen(p, T.data(), theta.data(), Yv.data())) return INFINITY;  // Yv[i][k]: vector k
        for (int k = 0; k < p; ++k) {
            double *y = &Y0[(size_t)k * D], *hy = &Y1[(size_t)k * D];
            std::fill(y, y + D, 0.0);
            std::fill(hy, hy + D, 0.0);
            for (int i = 0; i < p; ++i) {
                const double c = Yv[(size_t)i * p + k];
                axpy(c, &Q[(size_t)i * D], y, D);
                axpy(c, &HQ[(size_t)i * D], hy, D);
            }
        }
        Q.swap(Y0);
        HQ.swap(Y1);
        double worst = 0.0;
        for (int k = 0; k < std::min(p, want + 1); ++k) {
            const double *x = &Q[(size_t)k * D], *hx = &HQ[(size_t)k * D];
            double r = 0.0;
            for (size_t i = 0; i < D; ++i) {
                const double d = hx[i] - theta[k] * x[i];
                r += d * d;
            }
            if (k < want) worst = std::max(worst, std::sqrt(r));
            else r_next = std::sqrt(r);
        }
        return worst;
    };

    fill(X0);
    if (!orthonormalise()) return false;
    double worst = rayleigh_ritz();
    int extra = 0;
    for (int pass = 0; pass <= kMaxPasses; ++pass) {
        if (restarts) *restarts = pass;
        if (worst <= tol) {
            // the pair after the wanted ones bounds the next eigenvalue from
            // below (Ritz value minus its residual); a few more passes try to
            // separate it from the last wanted one
            const double lower = p > want ? theta[want] - r_next : INFINITY;
            const double gap = 1e-12 * std::max(1.0, std::fabs(theta[want - 1]));
            if (p == want || lower > theta[want - 1] + gap || extra >= 20) {
                std::copy_n(theta.data(), p, evals);
                std::copy_n(Q.data(), (size_t)p * D, X);
                if (next_lower) *next_lower = lower;
                return true;
            }
            ++extra;
        }
        if (pass == kMaxPasses || !std::isfinite(worst)) break;
        // Chebyshev filter of degree kDegree, bounded by 1 on [a, b]
        const double a = theta[p - 1], b = std::max(hb, a + 1e-9 * std::max(1.0, hb));
        const double c = 0.5 * (a + b), e = 0.5 * (b - a);
        // Y0 = Q, Y1 = (H - c) Q / e, Y_{k+1} = 2 (H - c) Y_k / e - Y_{k-1}
        Y0 = Q;
        for (size_t i = 0; i < (size_t)p * D; ++i) Y1[i] = (HQ[i] - c * Q[i]) / e;
        std::vector<double> hy(D);
        for (int k = 2; k <= kDegree; ++k) {
            for (int j = 0; j < p; ++j) {
                double *y1 = &Y1[(size_t)j * D], *y0 = &Y0[(size_t)j * D];
                apply_h(n, A, B, Ez, y1, hy.data());
                for (size_t i = 0; i < D; ++i) {
                    const double nx = 2.0 * (hy[i] - c * y1[i]) / e - y0[i];
                    y0[i] = y1[i];
                    y1[i] = nx;
                }
            }
        }
        Q.swap(Y1);
        if (!orthonormalise()) return false;
        worst = rayleigh_ritz();
    }
    return false;
}

}  // namespace aqt
