// Gradient runs: d<P>/dtheta of the trajectory average of the ground-manifold
// population at s = 1, for the schedule knots, the fields and the couplings
// (C ABI aqt_grad_*). The paper has no derivatives; the estimator is stated in
// adjoint.cuh.
//
// Device (the context's stream): a forward run that checkpoints every
// trajectory every `every` grid points; then, segment by segment from the
// last, a recompute of the segment from its checkpoint (the forward kernel in
// segment mode: the same arithmetic, so the same jumps), the backward sweep of
// the adjoint through it (adjoint.cuh), and the per-grid-point outer products
// X_g. Host (FP64, threads over grid points): the contraction of those sums
// with the derivatives of the tables.
//
// Host contraction at grid point g. With H' = V^T (dH_S/dtheta) V, first-order
// perturbation theory of the instantaneous eigensystem (nondegenerate levels)
// gives d eps_a = H'_aa and dV = V F, F_ab = H'_ab / (eps_b - eps_a) (a != b),
// F antisymmetric; so dO_{g-1} = -F_g O_{g-1} + O_{g-1} F_{g-1} and
// dM_alpha = M_alpha F - F M_alpha for M_alpha = V^T sz_alpha V. Every table the
// trajectories use at g depends on theta through eps and M_alpha:
//   K_bb = eps_b + sum_alpha sum_a f(E_b - E_a) M_alpha[a][b]^2,  f = S - (i/2) gamma
//   (Sec. III Eq. Heff; App. E), and the jump operators
//   A[a][b] = sqrt(gamma(E_b - E_a)) M_alpha[a][b] on the pairs of a Bohr class
//   (Eq. Aired, Eq. Lindblad2).
// Collecting dF = sum_a y_a d eps_a + sum_ab Xt_ab F_ab, with
//   Xt = X_g + sum_alpha (M_alpha Y_alpha - Y_alpha M_alpha),
// Y_alpha the derivative in the entries of M_alpha, the antisymmetric part of Xt
// is what F sees, and dF = <V W V^T, dH_S/dtheta> with W symmetric,
// W_aa = y_a, W_ab = (Xt_ab - Xt_ba) / (2 (eps_b - eps_a)) (zero inside a
// degenerate manifold). dH_S/dtheta is -sum sx times the schedule's hat
// function (A knots), diag(E_z) times it (B knots), B(s) sz_i (h_i) or
// B(s) sz_i sz_j (J_ij); only diag(V W V^T) and its sum over sx-neighbours
// are needed.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstring>
#include <limits>
#include <string>
#include <thread>
#include <vector>

#include "aqt_internal.h"

namespace aqt {

struct GradState {
    unsigned char *ws = nullptr;
    size_t bytes = 0;
    int every = 64, slots = 16, n_seg = 0, n_ckpt = 0;
    int64_t jcap = 0;
    size_t ckpt = 0, ckpt_clock = 0, ckpt_nj = 0, seg_c = 0, seg_nrot = 0, seg_mu = 0, carry = 0, lev = 0, jrec = 0,
           jvec = 0, jn = 0, jout = 0, jout_vec = 0, jout_n = 0, wscr = 0, xout = 0, dummy = 0, total = 0;
    size_t back_smem = 0;
    bool forward_done = false, ran = false;
    cudaStream_t stream = nullptr;
    uint64_t version = 0;
    double baseline = 0.0;
};

void grad_free(GradState *g) { delete g; }

namespace {

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

int n_params_of(const Inputs &in) { return 2 * (int)in.ks.size() + in.n + in.n * (in.n - 1) / 2; }

aqt_status layout(aqt_ctx *c, GradState &G, const GradAccess &A, int every, int64_t jcap) {
    const Inputs &in = *A.in;
    const size_t N = (size_t)in.levels(), K = in.K, M = in.M;
    const size_t rs = in.precision == AQT_PREC_FP64 ? 8 : 4;
    G.every = every;
    G.n_seg = (int)((K + every - 1) / every);
    G.n_ckpt = G.n_seg - 1;
    G.jcap = jcap;
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t o = off;
        off = al256(off + std::max<size_t>(b, 1));
        return o;
    };
    G.ckpt = take((size_t)G.n_ckpt * M * N * 2 * rs);
    G.ckpt_clock = take((size_t)G.n_ckpt * M * 2 * 8);
    G.ckpt_nj = take((size_t)G.n_ckpt * M * 4);
    G.seg_c = take((size_t)every * 2 * M * N * 2 * rs);
    G.seg_mu = take((size_t)every * 2 * M * N * 2 * rs);
    G.seg_nrot = take((size_t)every * M * 8);
    G.carry = take(M * N * 2 * rs);
    G.lev = take(K * N * 2 * 8);
    G.jrec = take(M * G.slots * sizeof(AdjJump));
    G.jvec = take(M * G.slots * 4 * N * 8);
    G.jn = take(M * 4);
    G.jout = take((size_t)jcap * sizeof(AdjJumpOut));
    G.jout_vec = take((size_t)jcap * 4 * N * 8);
    G.jout_n = take(8);
    G.wscr = take((size_t)A.n_cta * 8 * 10 * N * 8);
    G.xout = take(K * N * N * 8);
    G.dummy = take(8);
    G.total = off;
    G.back_smem = in.precision == AQT_PREC_FP64 ? adjoint_smem_bytes_f64((int)N, A.TT)
                                                : adjoint_smem_bytes_f32((int)N, A.TT);
    if (G.back_smem > 227 * 1024)
        return set_error(c, AQT_EINVAL, "the backward tile needs more shared memory than a CTA has");
    return AQT_OK;
}

aqt_status check_inputs(aqt_ctx *c, const GradAccess &A) {
    const Inputs &in = *A.in;
    if (in.precision != AQT_PREC_FP64 && in.precision != AQT_PREC_FP32)
        return set_error(c, AQT_EINVAL, "gradient runs take AQT_PREC_FP64 or AQT_PREC_FP32");
    if (in.timing != AQT_JUMP_REFINED) return set_error(c, AQT_EINVAL, "gradient runs take AQT_JUMP_REFINED timing");
    if (in.levels() != (1 << in.n)) return set_error(c, AQT_EINVAL, "gradient runs keep every level (no aqt_set_levels)");
    if (in.levels() > 256) return set_error(c, AQT_EINVAL, "gradient runs take at most 8 qubits");
    return AQT_OK;
}

// ---------------------------------------------------------------- contraction --
struct Contract {
    const Inputs &in;
    const Tables &tab;
    const std::vector<double> &xout;      // [K][N][N]
    const std::vector<double> &lev;       // [K][N][2]
    const std::vector<AdjJumpOut> &jumps;
    const std::vector<double> &jvec;      // [j][2][N][2]
    std::vector<std::vector<size_t>> by_g;
};

// Two-lane FP64 vector (GCC vector extension: NEON on aarch64, SSE2 on x86-64).
typedef double v2d __attribute__((vector_size(16), aligned(8)));

// out[i*ld + j] = sum_k X[i][k] Y[j][k] (rows of length len, row-major): 4 x 4
// register blocks, k in pairs on two-lane vectors (len even).
void rows_dot(const double *X, const double *Y, int ni, int nj, int len, double *out, int ld) {
    if (len % 2 || ni % 4 || nj % 4) {
        gram_rows(X, Y, ni, nj, len, out, ld);
        return;
    }
    for (int i0 = 0; i0 < ni; i0 += 4)
        for (int j0 = 0; j0 < nj; j0 += 4) {
            v2d acc[4][4];
            for (int a = 0; a < 4; ++a)
                for (int b = 0; b < 4; ++b) acc[a][b] = v2d{0.0, 0.0};
            const double *x = X + (size_t)i0 * len, *y = Y + (size_t)j0 * len;
            for (int k = 0; k < len; k += 2) {
                const v2d xa = *(const v2d *)(x + k), xb = *(const v2d *)(x + len + k);
                const v2d xc = *(const v2d *)(x + 2 * len + k), xd = *(const v2d *)(x + 3 * len + k);
                const v2d ya = *(const v2d *)(y + k), yb = *(const v2d *)(y + len + k);
                const v2d yc = *(const v2d *)(y + 2 * len + k), yd = *(const v2d *)(y + 3 * len + k);
                acc[0][0] += xa * ya; acc[0][1] += xa * yb; acc[0][2] += xa * yc; acc[0][3] += xa * yd;
                acc[1][0] += xb * ya; acc[1][1] += xb * yb; acc[1][2] += xb * yc; acc[1][3] += xb * yd;
                acc[2][0] += xc * ya; acc[2][1] += xc * yb; acc[2][2] += xc * yc; acc[2][3] += xc * yd;
                acc[3][0] += xd * ya; acc[3][1] += xd * yb; acc[3][2] += xd * yc; acc[3][3] += xd * yd;
            }
            for (int a = 0; a < 4; ++a)
                for (int b = 0; b < 4; ++b) out[(size_t)(i0 + a) * ld + j0 + b] = acc[a][b][0] + acc[a][b][1];
        }
}

// d/dw sqrt(gamma(w)) = gamma'(w) / (2 sqrt(gamma(w)))
double dsqrt_gamma(const Bath &b, double w) { return b.gamma_deriv(w) / (2.0 * std::sqrt(b.gamma(w))); }

// Adds the contribution of grid point g to grad[P]; marks undefined parameters in und.
void contract_point(const Contract &C, int g, std::vector<double> &grad, std::vector<char> &und) {
    const Inputs &in = C.in;
    const Tables &tab = C.tab;
    const Bath &bath = tab.bath;  // with its Lamb-shift table (in.bath has none: S would be integrated per call)
    const int n = in.n, N = tab.N, D = tab.D, K = tab.K;
    const size_t NN = (size_t)N * N;
    const double *ev = &tab.evals[(size_t)g * N];
    const double *E = &tab.lvlE[(size_t)g * N];
    const double *V = &tab.V[(size_t)g * D * N];
    const int32_t *mfirst = &tab.mfirst[(size_t)g * N];
    const int32_t *msize = &tab.msize[(size_t)g * N];
    const GridMeta meta = tab.meta[g];
    std::vector<double> Mall((size_t)n * NN);
    sz_frames_at(tab, g, Mall.data());
    // y: d/d eps; Y[alpha]: d/d M_alpha entries
    std::vector<double> y(N, 0.0), Y((size_t)n * NN, 0.0);
    // manifold energy derivative: dE_m = mean of d eps over the manifold
    auto add_dE = [&](int a, double v) {
        const int f = mfirst[a], m = msize[a];
        for (int q = f; q < f + m; ++q) y[q] += v / m;
    };
    // ---- effective Hamiltonian diagonal K_bb -------------------------------------------
    // coefficients per level pair (a <- b): cf = Re(kappa_b^* f(w)), cd = Re(kappa_b^* f'(w)),
    // kappa^* = rho - i sig (rho, sig: the sums for d Re K_bb, d Im K_bb), f = S - (i/2) gamma
    const double *lv = &C.lev[(size_t)g * N * 2];
    std::vector<double> cf(NN), cd(NN, 0.0), m2(NN, 0.0);
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
            const double rho = lv[2 * b], sig = lv[2 * b + 1];
            double gam, dgam, lam, dlam;
            bath.rates(E[b] - E[a], &gam, &dgam, &lam, &dlam);
            cf[(size_t)a * N + b] = rho * lam - 0.5 * sig * gam;
            if (mfirst[a] != mfirst[b]) cd[(size_t)a * N + b] = rho * dlam - 0.5 * sig * dgam;  // w = 0 identically otherwise
        }
    for (int b = 0; b < N; ++b) y[b] += lv[2 * b];
    for (int al = 0; al < n; ++al) {
        const double *Ma = &Mall[(size_t)al * NN];
        double *Ya = &Y[(size_t)al * NN];
        for (size_t i = 0; i < NN; ++i) {
            Ya[i] += 2.0 * cf[i] * Ma[i];
            m2[i] += Ma[i] * Ma[i];
        }
    }
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
            const double v = cd[(size_t)a * N + b] * m2[(size_t)a * N + b];
            if (v != 0.0) {
                add_dE(b, v);
                add_dE(a, -v);
            }
        }
    // ---- jumps at this grid point ---------------------------------------------------------
    for (size_t idx : C.by_g[g]) {
        const AdjJumpOut &J = C.jumps[idx];
        const double *cb = &C.jvec[idx * 4 * N];
        const double *mu = cb + 2 * N;
        const int al = J.r.alpha, bs = J.r.bsrc, ad = J.r.adst;
        const double *Ma = &Mall[(size_t)al * NN];
        double *Ya = &Y[(size_t)al * NN];
        // class pairs (a <- b) with their amplitude sqrt(gamma) M
        std::vector<std::pair<int, int>> pairs;
        const double wstar = E[bs] - E[ad];
        if (!J.r.general && ad != bs) {
            pairs.push_back({ad, bs});
        } else if (!J.r.general) {
            for (int q = 0; q < N; ++q) pairs.push_back({q, q});
        } else {
            for (int a = 0; a < N; ++a)
                for (int q = 0; q < N; ++q)
                    if (std::fabs(E[q] - E[a] - wstar) <= meta.tol) pairs.push_back({a, q});
        }
        // nu = |A c|
        std::vector<double> yr(N, 0.0), yi(N, 0.0);
        for (auto &pq : pairs) {
            const double amp = std::sqrt(bath.gamma(E[pq.second] - E[pq.first])) * Ma[(size_t)pq.first * N + pq.second];
            yr[pq.first] += amp * cb[2 * pq.second];
            yi[pq.first] += amp * cb[2 * pq.second + 1];
        }
        double nu2 = 0.0;
        for (int a = 0; a < N; ++a) nu2 += yr[a] * yr[a] + yi[a] * yi[a];
        const double inv = 1.0 / std::sqrt(nu2);
        for (auto &pq : pairs) {
            const int a = pq.first, q = pq.second;
            const double Jab = 2.0 * (mu[2 * a] * cb[2 * q] + mu[2 * a + 1] * cb[2 * q + 1]) * inv;  // 2 Re(mu_a^* c_q) / nu
            const double w = E[q] - E[a];
            const double sg = std::sqrt(bath.gamma(w));
            Ya[(size_t)a * N + q] += Jab * sg;
            if (mfirst[a] != mfirst[q]) {
                const double d = Jab * dsqrt_gamma(bath, w) * Ma[(size_t)a * N + q];
                add_dE(q, d);
                add_dE(a, -d);
            }
        }
    }
    // ---- antisymmetric part of Xt --------------------------------------------------------
    std::vector<double> Xa(NN), S(NN), MS(NN);
    const double *Xg = &C.xout[(size_t)g * NN];
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) Xa[(size_t)a * N + b] = Xg[(size_t)a * N + b] - Xg[(size_t)b * N + a];
    for (int al = 0; al < n; ++al) {
        const double *Ya = &Y[(size_t)al * NN];
        bool any = false;
        for (size_t i = 0; i < NN && !any; ++i) any = Ya[i] != 0.0;
        if (!any) continue;
        for (int a = 0; a < N; ++a)
            for (int b = 0; b < N; ++b) S[(size_t)a * N + b] = Ya[(size_t)a * N + b] + Ya[(size_t)b * N + a];
        // (M S)[a][b] = sum_e M[a][e] S[e][b] = sum_e M[a][e] S[b][e]
        rows_dot(&Mall[(size_t)al * NN], S.data(), N, N, N, MS.data(), N);
        for (int a = 0; a < N; ++a)
            for (int b = 0; b < N; ++b) Xa[(size_t)a * N + b] += MS[(size_t)a * N + b] - MS[(size_t)b * N + a];
    }
    // ---- W and P = V W V^T -----------------------------------------------------------
    std::vector<double> W(NN, 0.0), U((size_t)D * N);
    for (int a = 0; a < N; ++a) {
        W[(size_t)a * N + a] = y[a];
        for (int b = 0; b < N; ++b) {
            if (a == b || mfirst[a] == mfirst[b]) continue;
            W[(size_t)a * N + b] = Xa[(size_t)a * N + b] / (2.0 * (ev[b] - ev[a]));
        }
    }
    // U[x][a] = sum_b V[x][b] W[a][b]
    rows_dot(V, W.data(), D, N, N, U.data(), N);
    std::vector<double> diagP(D, 0.0);
    double xsum = 0.0;  // sum_x sum_i P[x][x ^ 2^i]
    for (int x = 0; x < D; ++x) {
        const double *u = &U[(size_t)x * N];
        double d = 0.0;
        for (int a = 0; a < N; ++a) d += u[a] * V[(size_t)x * N + a];
        diagP[x] = d;
        for (int i = 0; i < n; ++i) {
            const double *v2 = &V[(size_t)(x ^ (1 << i)) * N];
            double o = 0.0;
            for (int a = 0; a < N; ++a) o += u[a] * v2[a];
            xsum += o;
        }
    }
    // ---- parameters -----------------------------------------------------------------------
    const double s = K > 1 ? (double)g / (K - 1) : 0.0;
    double As, Bs;
    schedule_value(in, s, &As, &Bs);
    (void)As;
    const int nk = (int)in.ks.size();
    std::vector<double> hat(nk, 0.0);
    {
        size_t j = 0;
        while (j + 2 < in.ks.size() && s > in.ks[j + 1]) ++j;
        const double u = (s - in.ks[j]) / (in.ks[j + 1] - in.ks[j]);
        hat[j] = 1.0 - u;
        hat[j + 1] = u;
    }
    std::vector<double> zsum(n, 0.0), zzsum((size_t)n * n, 0.0);
    double ezsum = 0.0;
    for (int x = 0; x < D; ++x) {
        double ez = 0.0;
        for (int i = 0; i < n; ++i) {
            const double zi = (x >> i) & 1 ? -1.0 : 1.0;
            ez += in.hz[i] * zi;
            zsum[i] += zi * diagP[x];
            for (int j = i + 1; j < n; ++j) {
                const double zj = (x >> j) & 1 ? -1.0 : 1.0;
                ez += in.J[(size_t)i * n + j] * zi * zj;
                zzsum[(size_t)i * n + j] += zi * zj * diagP[x];
            }
        }
        ezsum += ez * diagP[x];
    }
    int pi = 0;
    for (int k = 0; k < nk; ++k) grad[pi++] += hat[k] * (-xsum);
    for (int k = 0; k < nk; ++k) grad[pi++] += hat[k] * ezsum;
    for (int i = 0; i < n; ++i) grad[pi++] += Bs * zsum[i];
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) grad[pi++] += Bs * zzsum[(size_t)i * n + j];
    // ---- parameters whose dH mixes a degenerate manifold here: no derivative -------------
    if (meta.degenerate) {
        std::vector<double> dHd(D);
        auto mixes = [&](const std::vector<double> &dd, bool sx) -> bool {
            // off-diagonal entries of V^T dH V inside each manifold
            for (int a = 0; a < N; ++a) {
                if (msize[a] < 2) continue;
                for (int b = a + 1; b < mfirst[a] + msize[a]; ++b) {
                    double h = 0.0;
                    for (int x = 0; x < D; ++x) {
                        if (sx) {
                            double t = 0.0;
                            for (int i = 0; i < n; ++i) t -= V[(size_t)(x ^ (1 << i)) * N + b];
                            h += V[(size_t)x * N + a] * t;
                        } else {
                            h += V[(size_t)x * N + a] * dd[x] * V[(size_t)x * N + b];
                        }
                    }
                    if (std::fabs(h) > 1e-9) return true;
                }
            }
            return false;
        };
        std::vector<double> ez(D, 0.0);
        for (int x = 0; x < D; ++x)
            for (int i = 0; i < n; ++i) {
                const double zi = (x >> i) & 1 ? -1.0 : 1.0;
                ez[x] += in.hz[i] * zi;
                for (int j = i + 1; j < n; ++j) ez[x] += in.J[(size_t)i * n + j] * zi * ((x >> j) & 1 ? -1.0 : 1.0);
            }
        const bool mx = mixes(dHd, true), mz = mixes(ez, false);
        int q = 0;
        for (int k = 0; k < nk; ++k, ++q)
            if (hat[k] != 0.0 && mx) und[q] = 1;
        for (int k = 0; k < nk; ++k, ++q)
            if (hat[k] != 0.0 && mz) und[q] = 1;
        if (Bs != 0.0) {
            for (int i = 0; i < n; ++i, ++q) {
                for (int x = 0; x < D; ++x) dHd[x] = (x >> i) & 1 ? -1.0 : 1.0;
                if (mixes(dHd, false)) und[q] = 1;
            }
            for (int i = 0; i < n; ++i)
                for (int j = i + 1; j < n; ++j, ++q) {
                    for (int x = 0; x < D; ++x) dHd[x] = (((x >> i) ^ (x >> j)) & 1) ? -1.0 : 1.0;
                    if (mixes(dHd, false)) und[q] = 1;
                }
        }
    }
}

aqt_status grad_ready(aqt_ctx *c, GradAccess &A, GradState *&G) {
    aqt_status s = grad_access(c, &A, true);
    if (s != AQT_OK) return s;
    if ((s = check_inputs(c, A)) != AQT_OK) return s;
    G = grad_state_get(c);
    if (!G) return set_error(c, AQT_EINVAL, "bind a gradient workspace first");
    if (G->version != A.version) return set_error(c, AQT_EINVAL, "inputs changed since the gradient workspace was bound");
    return AQT_OK;
}

}  // namespace

}  // namespace aqt

using namespace aqt;

extern "C" {

aqt_status aqt_grad_n_params(aqt_ctx *c, int *n_params) {
    if (!c || !n_params) return AQT_EINVAL;
    const Inputs *in = ctx_inputs(c);
    if (!in) return set_error(c, AQT_EINVAL, "set all inputs first");
    *n_params = n_params_of(*in);
    return AQT_OK;
}

aqt_status aqt_grad_workspace_size(aqt_ctx *c, int checkpoint_every, int64_t jump_capacity, size_t *bytes) {
    if (!c || !bytes) return AQT_EINVAL;
    if (checkpoint_every < 1) return set_error(c, AQT_EINVAL, "checkpoint_every must be >= 1");
    if (jump_capacity < 1) return set_error(c, AQT_EINVAL, "jump_capacity must be >= 1");
    GradAccess A;
    aqt_status s = grad_access(c, &A, false);
    if (s != AQT_OK) return s;
    if ((s = check_inputs(c, A)) != AQT_OK) return s;
    GradState G;
    if ((s = layout(c, G, A, checkpoint_every, jump_capacity)) != AQT_OK) return s;
    *bytes = G.total;
    return AQT_OK;
}

aqt_status aqt_grad_bind_workspace(aqt_ctx *c, int checkpoint_every, int64_t jump_capacity, void *dptr,
                                   size_t bytes) {
    if (!c || !dptr) return AQT_EINVAL;
    if ((reinterpret_cast<uintptr_t>(dptr) & 255) != 0) return set_error(c, AQT_EINVAL, "workspace must be 256-byte aligned");
    if (checkpoint_every < 1 || jump_capacity < 1) return set_error(c, AQT_EINVAL, "bad checkpoint_every or jump_capacity");
    GradAccess A;
    aqt_status s = grad_access(c, &A, false);
    if (s != AQT_OK) return s;
    if ((s = check_inputs(c, A)) != AQT_OK) return s;
    GradState *G = new GradState();
    if ((s = layout(c, *G, A, checkpoint_every, jump_capacity)) != AQT_OK) {
        delete G;
        return s;
    }
    if (bytes < G->total) {
        delete G;
        return set_error(c, AQT_ENOMEM, "gradient workspace smaller than aqt_grad_workspace_size");
    }
    G->ws = (unsigned char *)dptr;
    G->bytes = bytes;
    G->version = A.version;
    grad_state_set(c, G);
    return AQT_OK;
}

aqt_status aqt_grad_forward(aqt_ctx *c, void *stream) {
    if (!c) return AQT_EINVAL;
    GradAccess A;
    GradState *G = nullptr;
    aqt_status s = grad_ready(c, A, G);
    if (s != AQT_OK) return s;
    const Inputs &in = *A.in;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *w = G->ws;
    RunParams p = A.p;
    cudaError_t e = cudaMemsetAsync(p.jcount, 0, 8, st);
    if (!e) e = cudaMemsetAsync(p.status, 0, 4, st);
    if (!e) e = cudaMemsetAsync(p.norm_err, 0, 4, st);
    if (e) return set_error(c, AQT_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    p.adj.ckpt = w + G->ckpt;
    p.adj.ckpt_clock = (double *)(w + G->ckpt_clock);
    p.adj.ckpt_nj = (int32_t *)(w + G->ckpt_nj);
    p.adj.ckpt_every = G->every;
    int ce = launch_run(p, in.precision, stream, A.smem);
    if (ce) return set_error(c, AQT_ECUDA, std::string("forward launch: ") + cudaGetErrorString((cudaError_t)ce));
    grad_mark_ran(c, stream);
    G->forward_done = true;
    G->ran = false;
    return AQT_OK;
}

aqt_status aqt_grad_backward(aqt_ctx *c, double baseline, void *stream) {
    if (!c) return AQT_EINVAL;
    GradAccess A;
    GradState *G = nullptr;
    aqt_status s = grad_ready(c, A, G);
    if (s != AQT_OK) return s;
    if (!G->forward_done) return set_error(c, AQT_EINVAL, "run aqt_grad_forward first");
    const Inputs &in = *A.in;
    const bool f64 = in.precision == AQT_PREC_FP64;
    const int K = in.K, N = in.levels();
    const int64_t M = in.M;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *w = G->ws;
    const RunParams &p = A.p;
    int ce = 0;
    cudaError_t e = cudaMemsetAsync(w + G->lev, 0, (size_t)K * N * 2 * 8, st);
    if (!e) e = cudaMemsetAsync(w + G->jout_n, 0, 8, st);
    if (!e) e = cudaMemsetAsync(w + G->xout, 0, (size_t)K * N * N * 8, st);  // the outer products add into it
    if (e) return set_error(c, AQT_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    // ---- segments, last first -----------------------------------------------------------
    for (int sgi = G->n_seg - 1; sgi >= 0; --sgi) {
        const int g0 = sgi * G->every, g1 = std::min(K - 1, g0 + G->every - 1);
        // the recompute's jump counter must start at zero: its records are
        // dropped by the capacity test (idx < 0 = capacity), which a stale count
        // would pass
        e = cudaMemsetAsync(w + G->jn, 0, (size_t)M * 4, st);
        if (!e) e = cudaMemsetAsync(w + G->dummy, 0, 8, st);
        if (e) return set_error(c, AQT_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
        RunParams q = A.p;
        q.jcap = 0;
        q.jcount = (unsigned long long *)(w + G->dummy);
        q.adj.ckpt = w + G->ckpt;
        q.adj.ckpt_clock = (double *)(w + G->ckpt_clock);
        q.adj.ckpt_nj = (int32_t *)(w + G->ckpt_nj);
        q.adj.ckpt_every = G->every;
        q.adj.g_begin = g0;
        q.adj.g_end = g1;
        q.adj.seg_c = w + G->seg_c;
        q.adj.seg_nrot = (double *)(w + G->seg_nrot);
        q.adj.jrec = (AdjJump *)(w + G->jrec);
        q.adj.jvec = (double *)(w + G->jvec);
        q.adj.jn = (int32_t *)(w + G->jn);
        q.adj.slots = G->slots;
        ce = f64 ? launch_simt_f64(q, stream, A.smem) : launch_simt_f32(q, stream, A.smem);
        if (ce) return set_error(c, AQT_ECUDA, std::string("recompute launch: ") + cudaGetErrorString((cudaError_t)ce));
        AdjBack b{};
        b.seg_c = w + G->seg_c;
        b.seg_nrot = (const double *)(w + G->seg_nrot);
        b.seg_mu = w + G->seg_mu;
        b.carry = w + G->carry;
        b.lev = (double *)(w + G->lev);
        b.jrec = (const AdjJump *)(w + G->jrec);
        b.jvec = (const double *)(w + G->jvec);
        b.jn = (const int32_t *)(w + G->jn);
        b.jout = (AdjJumpOut *)(w + G->jout);
        b.jout_vec = (double *)(w + G->jout_vec);
        b.jout_n = (unsigned long long *)(w + G->jout_n);
        b.jout_cap = G->jcap;
        b.wscr = (double *)(w + G->wscr);
        b.baseline = baseline;
        b.g_begin = g0;
        b.g_end = g1;
        b.slots = G->slots;
        b.status = p.status;
        ce = f64 ? launch_adjoint_f64(q, b, stream, G->back_smem) : launch_adjoint_f32(q, b, stream, G->back_smem);
        if (ce) return set_error(c, AQT_ECUDA, std::string("backward launch: ") + cudaGetErrorString((cudaError_t)ce));
        ce = f64 ? launch_xgemm_f64(w + G->seg_c, w + G->seg_mu, M, N, K, g0, g1 - g0 + 1, (double *)(w + G->xout), stream)
                 : launch_xgemm_f32(w + G->seg_c, w + G->seg_mu, M, N, K, g0, g1 - g0 + 1, (double *)(w + G->xout), stream);
        if (ce) return set_error(c, AQT_ECUDA, std::string("outer-product launch: ") + cudaGetErrorString((cudaError_t)ce));
    }
    G->ran = true;
    G->stream = st;
    G->baseline = baseline;
    return AQT_OK;
}

aqt_status aqt_grad_get(aqt_ctx *c, double *grad, int n_params, double *value) {
    if (!c || !grad) return AQT_EINVAL;
    GradAccess A;
    aqt_status s = grad_access(c, &A, true);
    if (s != AQT_OK) return s;
    GradState *G = grad_state_get(c);
    if (!G || !G->ran) return set_error(c, AQT_EINVAL, "no gradient run to read");
    const Inputs &in = *A.in;
    const Tables &tab = *A.tab;
    const int P = n_params_of(in);
    if (n_params != P) return set_error(c, AQT_EINVAL, "n_params is " + std::to_string(P));
    cudaError_t e = cudaStreamSynchronize(G->stream);
    if (e) return set_error(c, AQT_ECUDA, std::string("gradient run: ") + cudaGetErrorString(e));
    int32_t status = 0;
    unsigned long long nj = 0;
    e = cudaMemcpy(&status, A.p.status, 4, cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(&nj, G->ws + G->jout_n, 8, cudaMemcpyDeviceToHost);
    if (e) return set_error(c, AQT_ECUDA, std::string("status readback: ") + cudaGetErrorString(e));
    if (status & 2) return set_error(c, AQT_ENUMERIC, "non-finite norm or too many jumps in one half-step");
    if (status & 8)
        return set_error(c, AQT_EOVERFLOW, "more than " + std::to_string(G->slots) + " jumps of one trajectory in one "
                                           "checkpoint segment: use a smaller checkpoint_every");
    if ((status & 16) || (int64_t)nj > G->jcap)
        return set_error(c, AQT_EOVERFLOW, "gradient jump list full: " + std::to_string(nj) + " jumps for a capacity of " +
                                               std::to_string(G->jcap));
    const int K = in.K, N = tab.N;
    std::vector<double> xout((size_t)K * N * N), lev((size_t)K * N * 2), obs((size_t)K * 2);
    std::vector<AdjJumpOut> jumps(nj);
    std::vector<double> jvec(nj * 4 * N);
    e = cudaMemcpy(xout.data(), G->ws + G->xout, xout.size() * 8, cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(lev.data(), G->ws + G->lev, lev.size() * 8, cudaMemcpyDeviceToHost);
    if (!e && nj) e = cudaMemcpy(jumps.data(), G->ws + G->jout, nj * sizeof(AdjJumpOut), cudaMemcpyDeviceToHost);
    if (!e && nj) e = cudaMemcpy(jvec.data(), G->ws + G->jout_vec, jvec.size() * 8, cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(obs.data(), A.p.obs_sum, obs.size() * 8, cudaMemcpyDeviceToHost);
    if (e) return set_error(c, AQT_ECUDA, std::string("gradient readback: ") + cudaGetErrorString(e));
    Contract C{in, tab, xout, lev, jumps, jvec, {}};
    C.by_g.assign(K, {});
    for (size_t i = 0; i < jumps.size(); ++i) C.by_g[jumps[i].r.g].push_back(i);
    // grid points on the host's cores, each into its own row; rows summed in grid
    // order (the same bits for any thread count)
    const unsigned nt = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
    std::vector<std::vector<double>> part(K, std::vector<double>(P, 0.0));
    std::vector<std::vector<char>> und(K, std::vector<char>(P, 0));
    std::atomic<int> next{0};
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back([&] {
            for (int g = next++; g < K; g = next++) contract_point(C, g, part[g], und[g]);
        });
    for (auto &x : th) x.join();
    const double inv_m = 1.0 / (double)in.M;
    for (int i = 0; i < P; ++i) {
        double acc = 0.0;
        bool u = false;
        for (int g = 0; g < K; ++g) {
            acc += part[g][i];
            u = u || und[g][i];
        }
        grad[i] = u ? std::numeric_limits<double>::quiet_NaN() : acc * inv_m;
    }
    if (value) *value = obs[2 * (K - 1)] * inv_m;
    return AQT_OK;
}

}  // extern "C"
