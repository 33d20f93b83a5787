// FP64 host tables for the AME trajectory path, one set per grid point s_g.
//
// arXiv:1710.03431: H_S(s) of Sec. V (Eq. H_S); Lindblad operators of Sec. II
// (Eq. Lindblad2) with independent sz baths (Sec. V; App. F), rates absorbed
// (Sec. III, Eq. Aired); effective Hamiltonian of Sec. III (Eq. Heff) with the
// Lamb shift of App. E. In the instantaneous eigenframe (columns of V_g) the
// state is a coefficient vector c (psi = V_g c), and with
//   M_alpha = V^T sz_alpha V,   w_ab = E(m(b)) - E(m(a)),   f = S - (i/2) gamma,
// the eigenframe H_eff is block diagonal over degenerate manifolds:
//   K[b,b'] = eps_b delta_bb' + sum_alpha sum_a f(w_ab) M_alpha[a,b] M_alpha[a,b'].
// The library requires K to be diagonal (true whenever every manifold is a
// single level, and at s = 0 of the transverse-field Ising model where each
// block is a multiple of the identity); otherwise it reports AQT_EDEGEN.
//
// Readings shared with the test oracle (which implements them separately):
// manifolds chain consecutive eigenvalues within tol = 1e-12 max(1, max|eps|)
// and take the mean energy; Bohr frequencies use manifold energies; classes of
// equal Bohr frequency chain within tol and must be tight (spread <= tol).
#include "aqt_internal.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <thread>

namespace aqt {

namespace {

unsigned n_threads() {
    unsigned h = std::thread::hardware_concurrency();
    return std::max(1u, std::min(64u, h));
}

template <class F>
void parallel_for(int count, F f) {
    std::atomic<int> next{0};
    std::vector<std::thread> th;
    const unsigned nt = std::min<unsigned>(n_threads(), (unsigned)std::max(count, 1));
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back([&] {
            for (int i = next++; i < count; i = next++) f(i);
        });
    for (auto &x : th) x.join();
}

// out[i*ld + j] = sum_k X[i][k] Y[j][k] for i < ni, j < nj (rows of length len,
// row-major), in 4x4 register blocks. With sym set, X == Y and only j >= i
// blocks are computed (the caller mirrors them).
void gram(const double *X, const double *Y, int ni, int nj, int len, double *out, int ld, bool sym) {
    for (int i0 = 0; i0 < ni; i0 += 4)
        for (int j0 = sym ? (i0 / 4) * 4 : 0; j0 < nj; j0 += 4) {
            double acc[4][4] = {};
            const int ib = std::min(4, ni - i0), jb = std::min(4, nj - j0);
            if (ib == 4 && jb == 4) {
                const double *x0 = X + (size_t)i0 * len, *y0 = Y + (size_t)j0 * len;
                for (int k = 0; k < len; ++k) {
                    const double xa = x0[k], xb = x0[len + k], xc = x0[2 * len + k], xd = x0[3 * len + k];
                    const double ya = y0[k], yb = y0[len + k], yc = y0[2 * len + k], yd = y0[3 * len + k];
                    acc[0][0] += xa * ya; acc[0][1] += xa * yb; acc[0][2] += xa * yc; acc[0][3] += xa * yd;
                    acc[1][0] += xb * ya; acc[1][1] += xb * yb; acc[1][2] += xb * yc; acc[1][3] += xb * yd;
                    acc[2][0] += xc * ya; acc[2][1] += xc * yb; acc[2][2] += xc * yc; acc[2][3] += xc * yd;
                    acc[3][0] += xd * ya; acc[3][1] += xd * yb; acc[3][2] += xd * yc; acc[3][3] += xd * yd;
                }
            } else {
                for (int i = 0; i < ib; ++i)
                    for (int j = 0; j < jb; ++j) {
                        double a = 0.0;
                        for (int k = 0; k < len; ++k) a += X[(size_t)(i0 + i) * len + k] * Y[(size_t)(j0 + j) * len + k];
                        acc[i][j] = a;
                    }
            }
            for (int i = 0; i < ib; ++i)
                for (int j = 0; j < jb; ++j) out[(size_t)(i0 + i) * ld + j0 + j] = acc[i][j];
        }
}

// Two-lane FP64 vector (GCC vector extension: NEON on aarch64, SSE2 on x86-64,
// no target flags); aligned(8) makes loads through it unaligned-safe.
typedef double v2d __attribute__((vector_size(16), aligned(8)));

// M_alpha = V^T sz_alpha V for every qubit alpha, written in full into
// M[alpha][a][b] (V row-major [x][a], N = 2^n). With P_alpha the projector on
// basis states whose bit alpha is set, sz_alpha = 1 - 2 P_alpha and
// M_alpha = I - 2 W_alpha, W_alpha[a][b] = sum over x with bit alpha set of
// V[x][a] V[x][b]. Split x into high bits u and low bits l (x = u 2^nl + l):
// the partial Gram matrices of the rows sharing u (resp. l) are formed once,
// and W_alpha for a high (low) bit is the sum of the partials whose u (l) has
// that bit, which halves the multiply-adds of forming each W_alpha from its
// own N/2 rows. Register blocks of 4 (a) x 8 (b); only b >= a is formed, the
// rest mirrored.
void sz_frames(const double *V, int n, double *M) {
    const int N = 1 << n, nl = n / 2, nh = n - nl, NU = 1 << nh, NL = 1 << nl;
    const size_t NN = (size_t)N * N;
    std::vector<double> Wt((size_t)n * 32);
    for (int i0 = 0; i0 < N; i0 += 4)
        for (int j0 = (i0 / 8) * 8; j0 < N; j0 += 8) {
            const int ib = std::min(4, N - i0), jb = std::min(8, N - j0);
            std::fill(Wt.begin(), Wt.end(), 0.0);
            // one partial over the rows of a group: over u (group l) or over l (group u)
            auto partial = [&](int grp, bool by_u, double *out) {
                const int cnt = by_u ? NL : NU;
                if (ib == 4 && jb == 8) {
                    v2d acc[4][4];
                    for (int ii = 0; ii < 4; ++ii)
                        for (int jj = 0; jj < 4; ++jj) acc[ii][jj] = v2d{0.0, 0.0};
                    for (int k = 0; k < cnt; ++k) {
                        const int x = by_u ? (grp << nl) | k : (k << nl) | grp;
                        const double *r = V + (size_t)x * N;
                        const v2d *rb = (const v2d *)(r + j0);
                        const v2d b0 = rb[0], b1 = rb[1], b2 = rb[2], b3 = rb[3];
                        for (int ii = 0; ii < 4; ++ii) {
                            const v2d a = {r[i0 + ii], r[i0 + ii]};
                            acc[ii][0] += a * b0;
                            acc[ii][1] += a * b1;
                            acc[ii][2] += a * b2;
                            acc[ii][3] += a * b3;
                        }
                    }
                    for (int ii = 0; ii < 4; ++ii)
                        for (int jj = 0; jj < 4; ++jj) {
                            out[ii * 8 + 2 * jj] = acc[ii][jj][0];
                            out[ii * 8 + 2 * jj + 1] = acc[ii][jj][1];
                        }
                } else {
                    for (int ii = 0; ii < ib; ++ii)
                        for (int jj = 0; jj < jb; ++jj) {
                            double a = 0.0;
                            for (int k = 0; k < cnt; ++k) {
                                const int x = by_u ? (grp << nl) | k : (k << nl) | grp;
                                a += V[(size_t)x * N + i0 + ii] * V[(size_t)x * N + j0 + jj];
                            }
                            out[ii * 8 + jj] = a;
                        }
                }
            };
            double part[32] = {};
            for (int u = 0; u < NU; ++u) {  // high bits alpha = nl .. n-1
                partial(u, true, part);
                for (int al = nl; al < n; ++al)
                    if ((u >> (al - nl)) & 1)
                        for (int e = 0; e < 32; ++e) Wt[(size_t)al * 32 + e] += part[e];
            }
            for (int l = 0; l < NL && nl > 0; ++l) {  // low bits alpha = 0 .. nl-1
                partial(l, false, part);
                for (int al = 0; al < nl; ++al)
                    if ((l >> al) & 1)
                        for (int e = 0; e < 32; ++e) Wt[(size_t)al * 32 + e] += part[e];
            }
            for (int al = 0; al < n; ++al) {
                double *Ma = M + (size_t)al * NN;
                for (int ii = 0; ii < ib; ++ii)
                    for (int jj = 0; jj < jb; ++jj) {
                        const int a = i0 + ii, b = j0 + jj;
                        if (b < a) continue;
                        const double v = (a == b ? 1.0 : 0.0) - 2.0 * Wt[(size_t)al * 32 + ii * 8 + jj];
                        Ma[(size_t)a * N + b] = v;
                        Ma[(size_t)b * N + a] = v;
                    }
            }
        }
}

// The same for a truncated eigenvector table: V row-major [x][a] with D = 2^n
// rows and L columns, M[alpha][a][b] for a, b < L. W_alpha = sum over rows
// with bit alpha set of V[x][a] V[x][b], formed as a Gram matrix of those rows.
void sz_frames_rect(const double *V, int n, int L, double *M) {
    const size_t D = (size_t)1 << n, LL = (size_t)L * L;
    std::vector<double> Xa((size_t)L * (D / 2)), W(LL);
    for (int al = 0; al < n; ++al) {
        // columns of V over the rows with bit alpha set, vector-major
        size_t k = 0;
        for (size_t x = 0; x < D; ++x) {
            if (!((x >> al) & 1)) continue;
            for (int a = 0; a < L; ++a) Xa[(size_t)a * (D / 2) + k] = V[x * L + a];
            ++k;
        }
        gram(Xa.data(), Xa.data(), L, L, (int)(D / 2), W.data(), L, true);
        double *Ma = M + (size_t)al * LL;
        for (int a = 0; a < L; ++a)
            for (int b = a; b < L; ++b) {
                const double v = (a == b ? 1.0 : 0.0) - 2.0 * W[(size_t)a * L + b];
                Ma[(size_t)a * L + b] = v;
                Ma[(size_t)b * L + a] = v;
            }
    }
}

// M_alpha for every qubit from the eigenvector table of one grid point.
void frames_of(const Tables &tab, const double *V, double *M) {
    if (tab.truncated) sz_frames_rect(V, tab.n, tab.N, M);
    else sz_frames(V, tab.n, M);
}

// Ascending sort of non-negative doubles (their bit patterns order like the
// values): least-significant-digit radix sort, 11-bit digits.
void sort_nonnegative(std::vector<double> &w) {
    const size_t n = w.size();
    std::vector<uint64_t> a(n), b(n);
    std::memcpy(a.data(), w.data(), n * 8);
    for (int shift = 0; shift < 64; shift += 11) {
        std::vector<size_t> cnt(2049, 0);
        for (size_t i = 0; i < n; ++i) ++cnt[((a[i] >> shift) & 2047) + 1];
        for (int d = 0; d < 2048; ++d) cnt[d + 1] += cnt[d];
        for (size_t i = 0; i < n; ++i) b[cnt[(a[i] >> shift) & 2047]++] = a[i];
        a.swap(b);
    }
    std::memcpy(w.data(), a.data(), n * 8);
}

void schedule_at(const Inputs &in, double s, double *A, double *B) {
    const auto &ks = in.ks;
    size_t j = 0;
    while (j + 2 < ks.size() && s > ks[j + 1]) ++j;
    const double u = (s - ks[j]) / (ks[j + 1] - ks[j]);
    *A = in.kA[j] + u * (in.kA[j + 1] - in.kA[j]);
    *B = in.kB[j] + u * (in.kB[j + 1] - in.kB[j]);
}

}  // namespace

aqt_status build_tables(const Inputs &in, Tables &tab, std::string *err) {
    const int n = in.n, D = 1 << n, N = in.levels(), K = in.K;
    const bool trunc = N < D;
    if (!trunc && n > 10) {
        *err = "more than 10 qubits need a truncation to the lowest levels (aqt_set_levels)";
        return AQT_EINVAL;
    }
    tab.n = n;
    tab.N = N;
    tab.D = D;
    tab.truncated = trunc;
    tab.K = K;
    tab.dt = in.t_f / (K - 1);
    tab.tau = 0.5 * tab.dt;
    const size_t NN = (size_t)N * N, DN = (size_t)D * N;
    tab.evals.resize((size_t)K * N);  // written in full below
    tab.V.resize((size_t)K * DN);
    tab.ev_next.assign(trunc ? K : 0, 0.0);
    tab.lanczos_restarts = 0;
    tab.kdiag.assign((size_t)K * N * 2, 0.0);
    tab.ehalf.assign((size_t)K * N * 2, 0.0);
    tab.d2.assign((size_t)K * N, 0.0);
    tab.G.assign((size_t)K * n * N, 0.0);
    tab.Mdiag.assign((size_t)K * n * N, 0.0);
    // truncated: every source level's jump amplitudes are tabled (the device
    // then needs no eigenvectors: they have 2^n rows)
    tab.n_low = trunc ? N : std::min(N, kLowSources);
    tab.Rlow.resize((size_t)K * n * tab.n_low * N);
    tab.gslot.assign(K, -1);
    tab.n_general = 0;
    tab.Rgen.clear();
    tab.lvlE.assign((size_t)K * N, 0.0);
    tab.mfirst.assign((size_t)K * N, 0);
    tab.msize.assign((size_t)K * N, 0);
    tab.meta.assign(K, GridMeta{0, 1, 1, 0, 0.0});
    tab.OT.resize((size_t)(K - 1) * NN);

    // classical energies sum_i hz_i z_i + sum_{i<j} J_ij z_i z_j, z = 1 - 2 bit
    std::vector<double> Ez(D, 0.0);
    for (int x = 0; x < D; ++x) {
        double e = 0.0;
        for (int i = 0; i < n; ++i) {
            const int zi = 1 - 2 * ((x >> i) & 1);
            e += in.hz[i] * zi;
        }
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j)
                e += in.J[(size_t)i * n + j] * (1 - 2 * ((x >> i) & 1)) * (1 - 2 * ((x >> j) & 1));
        Ez[x] = e;
    }

    std::mutex mu;
    aqt_status st = AQT_OK;
    auto fail = [&](aqt_status s, const std::string &m) {
        std::lock_guard<std::mutex> lk(mu);
        if (st == AQT_OK) {
            st = s;
            *err = m;
        }
    };

    // ---- pass 1: eigensystems ----------------------------------------------
    if (!trunc) {
        parallel_for(K, [&](int g) {
            const double s = (double)g / (K - 1);
            double A, B;
            schedule_at(in, s, &A, &B);
            std::vector<double> H(NN, 0.0);
            for (int x = 0; x < N; ++x) {
                H[(size_t)x * N + x] = B * Ez[x];
                for (int i = 0; i < n; ++i) H[(size_t)x * N + (x ^ (1 << i))] = -A;
            }
            if (!sym_eigen(N, H.data(), &tab.evals[(size_t)g * N], &tab.V[(size_t)g * NN]))
                fail(AQT_ENOCONV, "eigensolver did not converge at grid point " + std::to_string(g));
        });
    } else {
        // the lowest N eigenpairs (the block carries guard vectors; the next
        // eigenvalue is bounded from below to check the cut) by the
        // Chebyshev-filtered block solver; the grid splits into one contiguous
        // chunk per thread, each point warm-started from the previous one's vectors
        const int p = std::min(D, N + std::max(8, N / 4)), want = N;
        const int nchunk = std::max(1, std::min<int>(K, (int)n_threads()));
        std::atomic<int> worst_restarts{0};
        parallel_for(nchunk, [&](int c) {
            const int g0 = (int)((int64_t)K * c / nchunk), g1 = (int)((int64_t)K * (c + 1) / nchunk);
            std::vector<double> X((size_t)p * D), Xprev((size_t)p * D), ev(p);
            for (int g = g0; g < g1; ++g) {
                double A, B;
                schedule_at(in, (double)g / (K - 1), &A, &B);
                int it = 0;
                double lower = INFINITY;
                if (!lowest_eigen(n, A, B, Ez.data(), p, want, g == g0 ? nullptr : Xprev.data(), ev.data(), X.data(),
                                  &it, &lower)) {
                    fail(AQT_ENOCONV, "the block eigensolver did not converge at grid point " + std::to_string(g));
                    return;
                }
                int w = worst_restarts.load();
                while (it > w && !worst_restarts.compare_exchange_weak(w, it)) {
                }
                std::copy_n(ev.data(), N, &tab.evals[(size_t)g * N]);
                tab.ev_next[g] = lower;
                double *Vg = &tab.V[(size_t)g * DN];
                for (int x = 0; x < D; ++x)
                    for (int a = 0; a < N; ++a) Vg[(size_t)x * N + a] = X[(size_t)a * D + x];
                Xprev.swap(X);
            }
        });
        tab.lanczos_restarts = worst_restarts.load();
    }
    if (st != AQT_OK) return st;

    double wmax = 10.0;
    for (int g = 0; g < K; ++g)
        wmax = std::max(wmax, tab.evals[(size_t)g * N + N - 1] - tab.evals[(size_t)g * N]);
    tab.bath = in.bath;
    tab.bath.build_lamb(wmax * 1.05 + 1.0);
    const Bath &bath = tab.bath;

    // ---- pass 2: manifolds, M_alpha, rates, H_eff ----------------------------
    parallel_for(K, [&](int g) {
        const double *ev = &tab.evals[(size_t)g * N];
        const double *V = &tab.V[(size_t)g * DN];
        double emax = 1.0;
        for (int a = 0; a < N; ++a) emax = std::max(emax, std::fabs(ev[a]));
        const double tol = 1e-12 * emax;
        if (trunc && !(tab.ev_next[g] - ev[N - 1] > tol)) {
            fail(AQT_EDEGEN, "keeping " + std::to_string(N) + " levels splits a degenerate manifold (or the next " +
                                 "level could not be separated from the kept ones) at grid point " + std::to_string(g));
            return;
        }
        GridMeta &meta = tab.meta[g];
        meta.tol = tol;
        double *lvlE = &tab.lvlE[(size_t)g * N];
        int32_t *mf = &tab.mfirst[(size_t)g * N];
        int32_t *ms = &tab.msize[(size_t)g * N];
        std::vector<int> first;  // first level of each manifold
        for (int a = 0; a < N; ++a)
            if (a == 0 || ev[a] - ev[a - 1] > tol) first.push_back(a);
        first.push_back(N);
        std::vector<double> E(first.size() - 1);
        meta.degenerate = 0;
        for (size_t m = 0; m + 1 < first.size(); ++m) {
            double acc = 0.0;
            for (int a = first[m]; a < first[m + 1]; ++a) acc += ev[a];
            const int sz = first[m + 1] - first[m];
            E[m] = acc / sz;
            if (sz > 1) meta.degenerate = 1;
            for (int a = first[m]; a < first[m + 1]; ++a) {
                lvlE[a] = E[m];
                mf[a] = first[m];
                ms[a] = sz;
            }
        }
        meta.gs_size = first[1] - first[0];
        if (g == 0 && meta.gs_size != 1) {
            fail(AQT_EDEGEN, "ground state of H_S(0) is degenerate: the initial state is ambiguous");
            return;
        }
        // Bohr classes over manifold pairs must be tight chains; a grid point is
        // "simple" when every class of nonzero frequency holds one manifold pair.
        // The negative frequencies mirror the positive ones, and no chain crosses
        // zero (distinct manifolds are more than tol apart), so the positive half
        // decides both.
        meta.simple = 1;
        {
            const size_t nm = E.size();
            std::vector<double> w;
            w.reserve(nm * (nm - 1) / 2);
            for (size_t ma = 0; ma < nm; ++ma)
                for (size_t mb = ma + 1; mb < nm; ++mb) w.push_back(E[mb] - E[ma]);
            sort_nonnegative(w);
            size_t st0 = 0;
            for (size_t i = 1; i <= w.size(); ++i) {
                if (i == w.size() || w[i] - w[i - 1] > tol) {
                    if (i - st0 > 1) meta.simple = 0;
                    if (i > 0 && w[i - 1] - w[st0] > tol) {
                        fail(AQT_EDEGEN, "ambiguous Bohr-frequency grouping at grid point " + std::to_string(g));
                        return;
                    }
                    st0 = i;
                }
            }
        }
        std::vector<double> Mbuf((size_t)n * NN);
        double *Mg = Mbuf.data();
        frames_of(tab, V, Mg);
        // rates: gamma and S per level pair (a <- b), reused over alpha
        std::vector<double> gam(NN), lam(NN);
        for (int a = 0; a < N; ++a)
            for (int b = 0; b < N; ++b) {
                const double w = lvlE[b] - lvlE[a];
                gam[(size_t)a * N + b] = bath.gamma(w);
                lam[(size_t)a * N + b] = bath.lamb(w);
            }
        double *Gg = &tab.G[(size_t)g * n * N];
        double *kd = &tab.kdiag[(size_t)g * N * 2];
        for (int b = 0; b < N; ++b) {
            kd[2 * b] = ev[b];
            kd[2 * b + 1] = 0.0;
        }
        for (int al = 0; al < n; ++al) {
            const double *Ma = Mg + (size_t)al * NN;
            for (int a = 0; a < N; ++a) {
                const double *row = Ma + (size_t)a * N;  // M[a][b] over b
                for (int b = 0; b < N; ++b) {
                    const double m2 = row[b] * row[b];
                    const double gm = gam[(size_t)a * N + b];
                    Gg[(size_t)al * N + b] += gm * m2;
                    kd[2 * b] += lam[(size_t)a * N + b] * m2;
                    kd[2 * b + 1] -= 0.5 * gm * m2;
                }
            }
        }
        // degenerate manifolds: the off-diagonal block of K must vanish
        if (meta.degenerate) {
            const double ktol = 1e-12 * emax;
            for (size_t m = 0; m + 1 < first.size(); ++m) {
                for (int b = first[m]; b < first[m + 1]; ++b)
                    for (int bp = b + 1; bp < first[m + 1]; ++bp) {
                        double re = 0.0, im = 0.0;
                        for (int al = 0; al < n; ++al) {
                            const double *Ma = Mg + (size_t)al * NN;
                            for (int a = 0; a < N; ++a) {
                                const double mm = Ma[(size_t)a * N + b] * Ma[(size_t)a * N + bp];
                                re += lam[(size_t)a * N + b] * mm;
                                im -= 0.5 * gam[(size_t)a * N + b] * mm;
                            }
                        }
                        if (std::hypot(re, im) > ktol) {
                            fail(AQT_EDEGEN, "effective Hamiltonian is not diagonal inside a degenerate "
                                             "manifold at grid point " + std::to_string(g));
                            return;
                        }
                    }
            }
        }
        // diagonals of M_alpha (the zero-frequency jump operators, up to sqrt(gamma(0)))
        for (int al = 0; al < n; ++al)
            for (int b = 0; b < N; ++b)
                tab.Mdiag[((size_t)g * n + al) * N + b] = Mg[(size_t)al * NN + (size_t)b * N + b];
        // jump amplitudes of the lowest sources (Eq. Aired: R = sqrt(gamma) M), source-major;
        // M_alpha is symmetric, so row b of M gives column b
        for (int al = 0; al < n; ++al)
            for (int b = 0; b < tab.n_low; ++b) {
                double *dst = &tab.Rlow[(((size_t)g * n + al) * tab.n_low + b) * N];
                const double *Mb = Mg + (size_t)al * NN + (size_t)b * N;
                for (int a = 0; a < N; ++a) dst[a] = std::sqrt(gam[(size_t)a * N + b]) * Mb[a];
            }
        // half-step factors exp(-i K tau) and |.|^2
        double *eh = &tab.ehalf[(size_t)g * N * 2];
        double *dd = &tab.d2[(size_t)g * N];
        for (int b = 0; b < N; ++b) {
            const double re = kd[2 * b], im = kd[2 * b + 1];
            const double amp = std::exp(im * tab.tau);
            eh[2 * b] = amp * std::cos(re * tab.tau);
            eh[2 * b + 1] = -amp * std::sin(re * tab.tau);
            dd[b] = std::exp(2.0 * im * tab.tau);
        }
    });
    if (st != AQT_OK) return st;

    // ---- pass 2b: full jump amplitudes at the grid points that need the general
    // jump routine (Eq. Aired: R = sqrt(gamma) M, stored source-major) ----------
    std::vector<int> general;
    for (int g = 0; g < K; ++g)
        if (tab.meta[g].degenerate || !tab.meta[g].simple) {
            tab.gslot[g] = (int32_t)general.size();
            general.push_back(g);
        }
    tab.n_general = (int)general.size();
    tab.Rgen.resize((size_t)tab.n_general * n * NN);
    parallel_for(tab.n_general, [&](int i) {
        const int g = general[i];
        std::vector<double> R((size_t)n * NN);
        jump_amplitudes(in, tab, g, R.data());
        double *dst = &tab.Rgen[(size_t)i * n * NN];
        for (int al = 0; al < n; ++al)
            for (int a = 0; a < N; ++a)
                for (int b = 0; b < N; ++b) dst[(size_t)al * NN + (size_t)b * N + a] = R[(size_t)al * NN + (size_t)a * N + b];
    });

    // ---- time-step conditions of Eq. newcond (Sec. IV; App. A, App. B.1) --------
    // |H_eff| is the largest |K_bb| (H_eff = V K V^T with V orthogonal, K
    // diagonal). |dH_eff/dt| is estimated from above: the schedule derivative
    // of H_S by the triangle inequality (|H^X| = n, |H^Z| = max |E_z|), plus the
    // rate of change of the dissipative and Lamb-shift part of the diagonal
    // (forward differences). lambda is taken per eigenstate, lambda_b =
    // -2 Im K_bb (the jump rate of a trajectory in level b), over the levels
    // with a jump probability above 1e-6 over the whole run.
    {
        double hz_max = 0.0;
        for (int x = 0; x < D; ++x) hz_max = std::max(hz_max, std::fabs(Ez[x]));
        for (int i = 0; i < 3; ++i) {
            tab.dt_bound[i] = INFINITY;
            tab.dt_bound_at[i] = 0;
        }
        const double t_f = in.t_f;
        for (int g = 0; g < K; ++g) {
            const int g1 = g + 1 < K ? g + 1 : g - 1;  // neighbour for the difference
            const double s0 = (double)g / (K - 1), s1 = (double)g1 / (K - 1);
            double A0, B0, A1, B1;
            schedule_at(in, std::min(s0, s1), &A0, &B0);
            schedule_at(in, std::max(s0, s1), &A1, &B1);
            const double dsdt = 1.0 / t_f, ds = std::fabs(s1 - s0);
            const double hs_dot = (std::fabs(A1 - A0) * n + std::fabs(B1 - B0) * hz_max) / ds * dsdt;
            const double *k0 = &tab.kdiag[(size_t)g * N * 2], *k1 = &tab.kdiag[(size_t)g1 * N * 2];
            const double *e0 = &tab.evals[(size_t)g * N], *e1 = &tab.evals[(size_t)g1 * N];
            const double dtg = ds * t_f;
            double hnorm = 0.0, diss_dot = 0.0, lam_term = INFINITY;
            for (int b = 0; b < N; ++b) {
                hnorm = std::max(hnorm, std::hypot(k0[2 * b], k0[2 * b + 1]));
                const double dre = (k1[2 * b] - e1[b]) - (k0[2 * b] - e0[b]);
                const double dim = k1[2 * b + 1] - k0[2 * b + 1];
                diss_dot = std::max(diss_dot, std::hypot(dre, dim) / dtg);
                const double lam = -2.0 * k0[2 * b + 1], lam1 = -2.0 * k1[2 * b + 1];
                if (!(lam * t_f > 1e-6)) continue;
                const double lam_dot = (g1 > g ? lam1 - lam : lam - lam1) / dtg;
                const double den = std::fabs(lam * lam - lam_dot);
                if (den > 0.0) lam_term = std::min(lam_term, lam / den);
            }
            const double hdot = hs_dot + diss_dot;
            const double terms[3] = {hdot > 0.0 ? 2.0 * hnorm / hdot : INFINITY,
                                     hnorm > 0.0 ? 1.0 / hnorm : INFINITY, lam_term};
            for (int i = 0; i < 3; ++i)
                if (terms[i] < tab.dt_bound[i]) {
                    tab.dt_bound[i] = terms[i];
                    tab.dt_bound_at[i] = g;
                }
        }
    }

    // ---- pass 3: frame rotations OT_g[b][a] = (V_g^T V_{g+1})[b][a] ------------
    // (truncated: N x N blocks of the rotation between the kept spans, not
    // orthogonal; the weight they lose is the leakage the kernels renormalise away)
    parallel_for(K - 1, [&](int g) {
        const double *V0 = &tab.V[(size_t)g * DN];
        const double *V1 = &tab.V[(size_t)(g + 1) * DN];
        std::vector<double> T0(DN), T1(DN);
        for (int x = 0; x < D; ++x)
            for (int a = 0; a < N; ++a) {
                T0[(size_t)a * D + x] = V0[(size_t)x * N + a];
                T1[(size_t)a * D + x] = V1[(size_t)x * N + a];
            }
        gram(T0.data(), T1.data(), N, N, D, &tab.OT[(size_t)g * NN], N, false);
    });
    return AQT_OK;
}

void jump_amplitudes(const Inputs &in, const Tables &tab, int g, double *out) {
    const int n = tab.n, N = tab.N;
    const size_t NN = (size_t)N * N;
    frames_of(tab, &tab.V[(size_t)g * tab.D * N], out);  // M_alpha[a][b]
    const double *lvlE = &tab.lvlE[(size_t)g * N];
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
            const double sg = std::sqrt(in.bath.gamma(lvlE[b] - lvlE[a]));
            for (int al = 0; al < n; ++al) out[(size_t)al * NN + (size_t)a * N + b] *= sg;
        }
}

// Exported helpers of the gradient contraction (grad.cpp).
void gram_rows(const double *X, const double *Y, int ni, int nj, int len, double *out, int ld) {
    gram(X, Y, ni, nj, len, out, ld, false);
}

void sz_frames_at(const Tables &tab, int g, double *M) {
    frames_of(tab, &tab.V[(size_t)g * tab.D * tab.N], M);
}

void schedule_value(const Inputs &in, double s, double *A, double *B) { schedule_at(in, s, A, B); }

}  // namespace aqt
