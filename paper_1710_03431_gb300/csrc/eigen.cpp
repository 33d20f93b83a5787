// Dense real-symmetric eigensolver (FP64): Householder reduction to
// tridiagonal form, then the implicit QL iteration with Wilkinson-type shifts
// (Golub & Van Loan, Matrix Computations, Secs. 8.3.1-8.3.3; Wilkinson &
// Reinsch, Handbook for Automatic Computation II). Used once per grid point
// to obtain the instantaneous eigenstates |eps_a(t)> of H_S(t) that define the
// Lindblad operators (arXiv:1710.03431, Sec. II, Eq. Lindblad2).
#include "aqt_internal.h"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

namespace aqt {

namespace {
// Two-lane FP64 vector (GCC vector extension: NEON on aarch64, SSE2 on x86-64,
// no target flags); aligned(8) makes accesses through it unaligned-safe.
typedef double v2d __attribute__((vector_size(16), aligned(8)));
// Apply the Givens rotations of one QL sweep to the rows of ZT (n x n,
// row-major): rotation r mixes rows i = m-1-r and i+1 of every column x as
//   (z_{i+1}, z_i) <- (s z_i + c z_{i+1}, c z_i - s z_{i+1}),
// in the order r = 0, 1, ... Columns are independent, so the whole sequence
// is applied to one block of columns at a time, the row shared by
// consecutive rotations carried in registers (16 independent two-lane chains
// per block of 32 columns).
template <int NV>
static inline void sweep_block(double *ZT, int n, int m, int nrot, const double *rc, const double *rs, int x0) {
    v2d t[NV];
    for (int u = 0; u < NV; ++u) t[u] = *(const v2d *)(ZT + (size_t)m * n + x0 + 2 * u);
    for (int r = 0; r < nrot; ++r) {
        const int i = m - 1 - r;
        const v2d sv = {rs[r], rs[r]}, cv = {rc[r], rc[r]};
        const v2d *zi = (const v2d *)(ZT + (size_t)i * n + x0);
        v2d *zi1 = (v2d *)(ZT + (size_t)(i + 1) * n + x0);
        for (int u = 0; u < NV; ++u) {
            const v2d z = zi[u];
            zi1[u] = sv * z + cv * t[u];
            t[u] = cv * z - sv * t[u];
        }
    }
    v2d *zl = (v2d *)(ZT + (size_t)(m - nrot) * n + x0);
    for (int u = 0; u < NV; ++u) zl[u] = t[u];
}

void apply_sweep(double *ZT, int n, int m, int nrot, const double *rc, const double *rs) {
    if (nrot == 0) return;
    int x0 = 0;
    for (; x0 + 32 <= n; x0 += 32) sweep_block<16>(ZT, n, m, nrot, rc, rs, x0);
    for (; x0 + 8 <= n; x0 += 8) sweep_block<4>(ZT, n, m, nrot, rc, rs, x0);
    for (; x0 < n; ++x0) {
        double t = ZT[(size_t)m * n + x0];
        for (int r = 0; r < nrot; ++r) {
            const int i = m - 1 - r;
            const double z = ZT[(size_t)i * n + x0];
            ZT[(size_t)(i + 1) * n + x0] = rs[r] * z + rc[r] * t;
            t = rc[r] * z - rs[r] * t;
        }
        ZT[(size_t)(m - nrot) * n + x0] = t;
    }
}
}  // namespace

// A: n x n row-major symmetric (destroyed; only its lower triangle is read).
// evals ascending; V row-major with column a the eigenvector of evals[a].
// Returns false if QL does not converge.
bool sym_eigen(int n, double *A, double *evals, double *V) {
    std::vector<double> d(n), e(n, 0.0), v(n), p(n), w(n), beta(n, 0.0);
    // --- Householder tridiagonalisation: A = Q T Q^T --------------------------
    // Step k zeroes A[k+2:, k]; its reflector v_k is kept in A[k+1:, k]. Only
    // the lower triangle of the trailing block is updated and read.
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        double *col = &v[0];
        double alpha2 = 0.0;
        for (int i = 0; i < m; ++i) {
            col[i] = A[(size_t)(k + 1 + i) * n + k];
            alpha2 += col[i] * col[i];
        }
        const double alpha = std::sqrt(alpha2);
        if (alpha == 0.0) {
            e[k] = 0.0;
            beta[k] = 0.0;
            continue;
        }
        const double sgn = col[0] >= 0.0 ? 1.0 : -1.0;
        col[0] += sgn * alpha;
        // |v|^2 = 2 alpha (alpha + |x_0|) for v = x + sign(x_0) alpha e_1
        const double b = 2.0 / (2.0 * alpha * (alpha + std::fabs(col[0] - sgn * alpha)));
        // p = b * S v over the trailing block S = A[k+1:, k+1:], read from its
        // lower triangle only (S is symmetric; the upper triangle is not kept
        // up to date): row i gives sum_{j<i} S[i][j] v[j] to p[i] and
        // S[i][j] v[i] to every p[j], j < i, in one pass over the row
        for (int i = 0; i < m; ++i) p[i] = 0.0;
        for (int i = 0; i < m; ++i) {
            const double *row = &A[(size_t)(k + 1 + i) * n + (k + 1)];
            const double vi = col[i];
            const v2d viv = {vi, vi};
            v2d dacc = {0.0, 0.0};
            int j = 0;
            for (; j + 2 <= i; j += 2) {
                const v2d r = *(const v2d *)(row + j);
                dacc += r * *(const v2d *)(col + j);
                *(v2d *)(&p[j]) += r * viv;
            }
            double dot = dacc[0] + dacc[1];
            for (; j < i; ++j) {
                dot += row[j] * col[j];
                p[j] += row[j] * vi;
            }
            p[i] += row[i] * vi + dot;
        }
        for (int i = 0; i < m; ++i) p[i] *= b;
        double pv = 0.0;
        for (int i = 0; i < m; ++i) pv += p[i] * col[i];
        const double K = 0.5 * b * pv;
        for (int i = 0; i < m; ++i) w[i] = p[i] - K * col[i];
        // S -= v w^T + w v^T on the lower triangle
        for (int i = 0; i < m; ++i) {
            double *row = &A[(size_t)(k + 1 + i) * n + (k + 1)];
            const double vi = col[i], wi = w[i];
            for (int j = 0; j <= i; ++j) row[j] -= vi * w[j] + wi * col[j];
        }
        e[k] = -sgn * alpha;
        beta[k] = b;
        for (int i = 0; i < m; ++i) A[(size_t)(k + 1 + i) * n + k] = col[i];
    }
    for (int i = 0; i < n; ++i) d[i] = A[(size_t)i * n + i];
    if (n >= 2) e[n - 2] = A[(size_t)(n - 1) * n + (n - 2)];
    // e[k] for k <= n-3 was recorded with its reflector; e[n-2] is A[n-1][n-2].
    // --- Backward accumulation of Q = H_0 H_1 ... H_{n-3}, stored as ZT = Q^T ---
    std::vector<double> Q((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
    for (int k = n - 3; k >= 0; --k) {
        const double b = beta[k];
        if (b == 0.0) continue;
        const int m = n - k - 1;
        // rows k+1.. of Q, columns k+1..: Q_sub -= b v (v^T Q_sub)
        for (int j = k + 1; j < n; ++j) w[j] = 0.0;
        for (int i = 0; i < m; ++i) {
            const double vi = A[(size_t)(k + 1 + i) * n + k];
            const double *row = &Q[(size_t)(k + 1 + i) * n];
            for (int j = k + 1; j < n; ++j) w[j] += vi * row[j];
        }
        for (int i = 0; i < m; ++i) {
            const double vi = b * A[(size_t)(k + 1 + i) * n + k];
            double *row = &Q[(size_t)(k + 1 + i) * n];
            for (int j = k + 1; j < n; ++j) row[j] -= vi * w[j];
        }
    }
    // ZT[i][x] = Q[x][i]
    std::vector<double> ZT((size_t)n * n);
    for (int x = 0; x < n; ++x)
        for (int i = 0; i < n; ++i) ZT[(size_t)i * n + x] = Q[(size_t)x * n + i];
    // --- Implicit QL on the tridiagonal (d, e), e[i] couples i and i+1 ---------
    e[n - 1] = 0.0;
    const double eps = 2.220446049250313e-16;
    // Deflation test against the norm of T (robust when diagonal entries vanish,
    // as for the equally spaced, highly degenerate spectrum of H_S(0)).
    double tnorm = 0.0;
    for (int i = 0; i < n; ++i) tnorm = std::max(tnorm, std::fabs(d[i]) + std::fabs(e[i]) + (i ? std::fabs(e[i - 1]) : 0.0));
    const double small = eps * tnorm;
    std::vector<double> rc(n), rs(n);
    for (int l = 0; l < n; ++l) {
        int iter = 0;
        for (;;) {
            int m = l;
            for (; m < n - 1; ++m) {
                if (std::fabs(e[m]) <= small) break;
            }
            if (m == l) break;
            if (++iter > 100) return false;
            // shift from the leading 2x2 of the unreduced block
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = std::hypot(g, 1.0);
            g = d[m] - d[l] + e[l] / (g + (g >= 0.0 ? r : -r));
            double s = 1.0, c = 1.0, pp = 0.0;
            int i = m - 1;
            int nrot = 0;  // rotations of this sweep, on rows (m-1-r, m-r), r = 0..nrot-1
            bool underflow = false;
            for (; i >= l; --i) {
                const double f = s * e[i];
                const double bb = c * e[i];
                r = std::hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) {
                    d[i + 1] -= pp;
                    e[m] = 0.0;
                    underflow = true;
                    break;
                }
                s = f / r;
                c = g / r;
                g = d[i + 1] - pp;
                r = (d[i] - g) * s + 2.0 * c * bb;
                pp = s * r;
                d[i + 1] = g + pp;
                g = c * r - bb;
                rs[nrot] = s;
                rc[nrot] = c;
                ++nrot;
            }
            apply_sweep(ZT.data(), n, m, nrot, rc.data(), rs.data());
            if (underflow) continue;
            d[l] -= pp;
            e[l] = g;
            e[m] = 0.0;
        }
    }
    // --- sort ascending ---------------------------------------------------------
    std::vector<int> ord(n);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return d[a] < d[b]; });
    for (int a = 0; a < n; ++a) {
        evals[a] = d[ord[a]];
        const double *z = &ZT[(size_t)ord[a] * n];
        // sign convention: the largest-magnitude component is positive
        int xm = 0;
        for (int x = 1; x < n; ++x)
            if (std::fabs(z[x]) > std::fabs(z[xm]) + 1e-12) xm = x;
        const double sg = z[xm] < 0.0 ? -1.0 : 1.0;
        for (int x = 0; x < n; ++x) V[(size_t)x * n + a] = sg * z[x];
    }
    return true;
}

}  // namespace aqt
