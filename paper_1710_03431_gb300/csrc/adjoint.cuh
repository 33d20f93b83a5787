// Backward sweep of a gradient run: the adjoint of the trajectories'
// propagation through one segment of grid points, and the per-grid-point
// trajectory sums that the parameter derivatives need.
//
// The paper has no derivatives. What is differentiated: the trajectory
// average of the ground-manifold population at s = 1, <P> = E[p_T]. A
// trajectory's record (its jump times and channels) has probability density
// |psi~_T|^2, the squared norm of the unnormalised state built from it (the
// waiting-time density of Sec. IV / App. C times the channel probability of
// App. B.1, Eq. Pi(t), is |A_i psi~(t)|^2). So <P> is the integral over records
// of <psi~_T|P|psi~_T>, and with the record held fixed the derivative is
//   d<P>/dtheta = E[ 2 Re <(P - b) psi_T, dpsi~_T/dtheta> / |psi~_T| ]
// (b any constant: it multiplies the score of the record, whose mean is zero):
// a pathwise adjoint through the no-jump propagators, the frame rotations and
// the jump operators at fixed jump times, which carries the score of the
// waiting times and of the channel choice through the unnormalised norm.
//
// In the eigenframe a trajectory is a product of linear maps T_k (half-step
// diagonals D = exp(-i K l), rotations O_g = V_{g+1}^T V_g, jump operators A)
// applied to c_0 = e_0, each followed by a renormalisation by
// nu_k = |T_k c_{k-1}|. With mu_L = (P - b) c_L and mu_{k-1} = T_k^dag mu_k / nu_k,
//   d<P>/dtheta = E[ sum_k 2 Re <mu_k, dT_k c_{k-1}> / nu_k ].
// Per grid point g this needs, summed over trajectories:
//   * for the eigenvectors V_g (through O_{g-1}, O_g): the outer products
//     X_g = 2 [Re(mu_e^* c_e^T) - Re(mu_s^* c_s^T)] at the end (e) and start (s)
//     of g's frozen span (formed by adj_xgemm from the stored vectors);
//   * for the diagonal K_g: per level, 2 l Im(mu_a^* c_a) and 2 l Re(mu_a^* c_a)
//     at the end of each stretch of length l without a jump (dK_re, dK_im);
//   * at every jump: the state before it and the adjoint after it (the host
//     differentiates the jump operator in FP64).
// The host contracts these with the derivatives of the FP64 tables.
//
// Layout: one CTA owns TT trajectories; the adjoint tile stays in shared
// memory as planar [level][trajectory] (as the forward's state); the frame
// rotation's adjoint O^T streams O in chunks, transposed into shared memory.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "aqt_internal.h"
#include "device_jump.cuh"

namespace aqt {
namespace adj {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kChunkBytes = 32768;

using namespace dev;

enum : int32_t { kStatusJumpList = 16 };

// conj(exp(-i K_aa l)) of level a at grid point g, and exp(2 Im K_aa l), FP64
static __device__ __forceinline__ void cdecay(const RunParams &p, int g, int a, double l, double *re, double *im,
                                       double *e2) {
    const double kr = p.tab.kdiag[((size_t)g * p.N + a) * 2], ki = p.tab.kdiag[((size_t)g * p.N + a) * 2 + 1];
    double sn, cs;
    sincos(kr * l, &sn, &cs);
    const double amp = exp(ki * l);
    *re = amp * cs;
    *im = amp * sn;
    *e2 = amp * amp;
}

// The general Bohr-class operator of a jump at grid point g (qubit al, source
// level bsrc, target adst), A[a][b'] = R_alpha[a][b'] for pairs of frequency
// E(bsrc) - E(adst) within the grid point's tolerance (Eq. Lindblad2), applied
// to x (transposed when tr): out_a = sum_b' A[a][b'] x_b' (or out_b' = sum_a
// A[a][b'] x_a). x, out: per-warp FP64 scratch of N complex.
static __device__ void general_apply(const RunParams &p, int g, int al, int bsrc, int adst, bool tr, const double *x,
                              double *out, int lane) {
    const int N = p.N, n = p.n;
    const double *lvlE = p.tab.lvlE + (size_t)g * N;
    const double wstar = lvlE[bsrc] - lvlE[adst];
    const double tol = p.tab.meta[g].tol;
    const double *Ra = p.tab.Rgen + ((size_t)p.tab.gslot[g] * n + al) * N * N;  // [b'][a]
    for (int i = lane; i < N; i += 32) {
        // pairs (a, b') with E(b') - E(a) = wstar: for out_a, b' has energy E(a) + wstar; for
        // out_b', a has energy E(b') - wstar
        const double centre = tr ? lvlE[i] - wstar : lvlE[i] + wstar;
        int lo = 0, hi = N;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (lvlE[mid] < centre - tol) lo = mid + 1; else hi = mid;
        }
        double yr = 0.0, yi = 0.0;
        for (int j = lo; j < N && lvlE[j] <= centre + tol; ++j) {
            const double amp = tr ? Ra[(size_t)i * N + j] : Ra[(size_t)j * N + i];
            yr += amp * x[2 * j];
            yi += amp * x[2 * j + 1];
        }
        out[2 * i] = yr;
        out[2 * i + 1] = yi;
    }
    __syncwarp();
}

// Backward through the frozen span of grid point g for one trajectory that
// jumped in it, by one warp in FP64. On entry mu (level a = 32 j + lane) is the
// adjoint at the span's end; on return, at its start. Adds the per-level sums
// of every stretch to lsum (shared memory) and appends each jump to the
// compact list for the host.
template <int NPL>
__device__ __noinline__ void span_with_jumps(const RunParams &p, const AdjBack &b, int g, int64_t traj,
                                             const double *c_s, const double *c_e, double *mu, double *lsum,
                                             int k_lo, int k_hi, double *scr, int lane) {
    double mr[NPL], mi[NPL];
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
        const int a = 32 * j + lane;
        mr[j] = a < p.N ? mu[2 * a] : 0.0;
        mi[j] = a < p.N ? mu[2 * a + 1] : 0.0;
    }
    const int N = p.N, K = p.K;
    const double tau = p.tau;
    const double L = (g == 0 || g == K - 1) ? tau : 2.0 * tau;
    // time of a jump from the span's start: half 1 of an inner grid point starts tau in
    auto t_span = [&](const AdjJump &r) { return r.t_rel + ((r.half == 1 && g > 0) ? tau : 0.0); };
    double cr[NPL], ci[NPL];  // state at the end of the current stretch
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
        const int a = 32 * j + lane;
        cr[j] = a < N ? c_e[2 * a] : 0.0;
        ci[j] = a < N ? c_e[2 * a + 1] : 0.0;
    }
    double t_end = L;
    for (int k = k_hi - 1; k >= k_lo - 1; --k) {
        const bool first = k < k_lo;  // the stretch from the span's start to the first jump
        const AdjJump r = first ? AdjJump{} : b.jrec[(size_t)traj * b.slots + k];
        const double ts = first ? 0.0 : t_span(r);
        const double l = t_end - ts;
        // per-level sums at the end of this stretch
#pragma unroll
        for (int j = 0; j < NPL; ++j) {
            const int a = 32 * j + lane;
            if (a < N) {
                const double zr = mr[j] * cr[j] + mi[j] * ci[j];  // Re(mu^* c)
                const double zi = mr[j] * ci[j] - mi[j] * cr[j];  // Im(mu^* c)
                atomicAdd(&lsum[2 * a], 2.0 * l * zi);
                atomicAdd(&lsum[2 * a + 1], 2.0 * l * zr);
            }
        }
        // the stretch's start state: after the jump, or the span's start
        const double *cv = first ? c_s : b.jvec + (((size_t)traj * b.slots + k) * 2 + 1) * 2 * N;
        double s = 0.0;
        double dre[NPL], dim_[NPL];
#pragma unroll
        for (int j = 0; j < NPL; ++j) {
            const int a = 32 * j + lane;
            double e2 = 0.0;
            dre[j] = dim_[j] = 0.0;
            if (a < N) {
                cdecay(p, g, a, l, &dre[j], &dim_[j], &e2);
                s += (cv[2 * a] * cv[2 * a] + cv[2 * a + 1] * cv[2 * a + 1]) * e2;
            }
        }
        s = warp_sum(s);
        const double inv = 1.0 / sqrt(s);
#pragma unroll
        for (int j = 0; j < NPL; ++j) {
            const double r_ = (dre[j] * mr[j] - dim_[j] * mi[j]) * inv;
            const double i_ = (dre[j] * mi[j] + dim_[j] * mr[j]) * inv;
            mr[j] = r_;
            mi[j] = i_;
        }
        if (first) break;
        // mu is now the adjoint right after jump k: hand it to the host with the state before it
        const double *cb = b.jvec + (((size_t)traj * b.slots + k) * 2) * 2 * N;
        unsigned long long idx = 0;
        if (lane == 0) idx = atomicAdd(b.jout_n, 1ull);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if ((int64_t)idx < b.jout_cap) {
            double *o = b.jout_vec + idx * 4 * N;
#pragma unroll
            for (int j = 0; j < NPL; ++j) {
                const int a = 32 * j + lane;
                if (a < N) {
                    o[2 * a] = cb[2 * a];
                    o[2 * a + 1] = cb[2 * a + 1];
                    o[2 * N + 2 * a] = mr[j];
                    o[2 * N + 2 * a + 1] = mi[j];
                }
            }
            if (lane == 0) {
                AdjJumpOut jo;
                jo.r = r;
                jo.traj = traj;
                b.jout[idx] = jo;
            }
        } else if (lane == 0) {
            atomicOr(b.status, kStatusJumpList);
        }
        // through the jump: mu <- A^T mu / |A c_before|
        const int al = r.alpha, bs = r.bsrc, ad = r.adst;
        if (!r.general && ad != bs) {
            // single pair (ad <- bs): A c / |A c| = sign(M) c_bs / |c_bs| on ad, so
            // A^T mu / |A c| = e_bs sign(M) mu_ad / |c_bs|; the sign is read off the states
            const double *ca = cv;  // state after the jump: nonzero on ad only
            const double br = cb[2 * bs], bi = cb[2 * bs + 1];
            const double m2 = br * br + bi * bi;
            const double ratio = (ca[2 * ad] * br + ca[2 * ad + 1] * bi) / m2;  // real: sign(M) / |c_bs|
            const double mar = __shfl_sync(0xffffffffu, reg_at(mr, ad >> 5), ad & 31);
            const double mai = __shfl_sync(0xffffffffu, reg_at(mi, ad >> 5), ad & 31);
#pragma unroll
            for (int j = 0; j < NPL; ++j) {
                const bool hit = 32 * j + lane == bs;
                mr[j] = hit ? ratio * mar : 0.0;
                mi[j] = hit ? ratio * mai : 0.0;
            }
        } else if (!r.general) {
            // zero frequency: A = sqrt(gamma(0)) diag(M_alpha); A^T mu / |A c| = d mu / |d c|
            const double *Md = p.tab.Mdiag + ((size_t)g * p.n + al) * N;
            double s2 = 0.0;
#pragma unroll
            for (int j = 0; j < NPL; ++j) {
                const int a = 32 * j + lane;
                if (a < N) s2 += Md[a] * Md[a] * (cb[2 * a] * cb[2 * a] + cb[2 * a + 1] * cb[2 * a + 1]);
            }
            s2 = warp_sum(s2);
            const double iv = 1.0 / sqrt(s2);
#pragma unroll
            for (int j = 0; j < NPL; ++j) {
                const int a = 32 * j + lane;
                const double d = a < N ? Md[a] * iv : 0.0;
                mr[j] *= d;
                mi[j] *= d;
            }
        } else {
            double *x = scr, *y = scr + 2 * N;
            // |A c_before|
            general_apply(p, g, al, bs, ad, false, cb, y, lane);
            double s2 = 0.0;
            for (int a = lane; a < N; a += 32) s2 += y[2 * a] * y[2 * a] + y[2 * a + 1] * y[2 * a + 1];
            s2 = warp_sum(s2);
            __syncwarp();
#pragma unroll
            for (int j = 0; j < NPL; ++j) {
                const int a = 32 * j + lane;
                if (a < N) {
                    x[2 * a] = mr[j];
                    x[2 * a + 1] = mi[j];
                }
            }
            __syncwarp();
            general_apply(p, g, al, bs, ad, true, x, y, lane);
            const double iv = 1.0 / sqrt(s2);
#pragma unroll
            for (int j = 0; j < NPL; ++j) {
                const int a = 32 * j + lane;
                mr[j] = a < N ? y[2 * a] * iv : 0.0;
                mi[j] = a < N ? y[2 * a + 1] * iv : 0.0;
            }
            __syncwarp();
        }
        // the next (earlier) stretch ends at the state before this jump
#pragma unroll
        for (int j = 0; j < NPL; ++j) {
            const int a = 32 * j + lane;
            cr[j] = a < N ? cb[2 * a] : 0.0;
            ci[j] = a < N ? cb[2 * a + 1] : 0.0;
        }
        t_end = ts;
    }
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
        const int a = 32 * j + lane;
        if (a < N) {
            mu[2 * a] = mr[j];
            mu[2 * a + 1] = mi[j];
        }
    }
    __syncwarp();
}

// span_with_jumps for the register tile that holds N levels
static __device__ __forceinline__ void span_with_jumps_any(const RunParams &p, const AdjBack &b, int g, int64_t traj,
                                                    const double *c_s, const double *c_e, double *mu, double *lsum,
                                                    int k_lo, int k_hi, double *scr, int lane) {
    if (p.N <= 32) span_with_jumps<1>(p, b, g, traj, c_s, c_e, mu, lsum, k_lo, k_hi, scr, lane);
    else if (p.N <= 64) span_with_jumps<2>(p, b, g, traj, c_s, c_e, mu, lsum, k_lo, k_hi, scr, lane);
    else if (p.N <= 128) span_with_jumps<4>(p, b, g, traj, c_s, c_e, mu, lsum, k_lo, k_hi, scr, lane);
    else if (p.N <= 256) span_with_jumps<8>(p, b, g, traj, c_s, c_e, mu, lsum, k_lo, k_hi, scr, lane);
    else span_with_jumps<16>(p, b, g, traj, c_s, c_e, mu, lsum, k_lo, k_hi, scr, lane);
}

// Four consecutive entries of a 16-byte aligned tile row.
static __device__ __forceinline__ void load4(const float *p, float v[4]) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
static __device__ __forceinline__ void load4(const double *p, double v[4]) {
    const double2 q0 = *reinterpret_cast<const double2 *>(p);
    const double2 q1 = *reinterpret_cast<const double2 *>(p + 2);
    v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}

// Shared memory of the backward tile (bytes).
inline size_t back_smem_bytes(int N, int TT, size_t rs) {
    const int LD = TT + 4;
    const int KB = std::min(N, std::max(1, kChunkBytes / (int)(N * rs)));
    return 2 * (size_t)N * 8               // level sums of jumped spans (im, re), FP64
           + 6 * (size_t)N * rs            // level sums of the other spans, the span's conj decay, exp(2 Im K L)
           + 2 * (size_t)N * LD * rs       // adjoint tile
           + (size_t)KB * (N + 1) * rs     // transposed O chunk
           + 64;
}

// One segment of the backward sweep for the trajectories of tile `cta`.
template <typename R, int RA>
__device__ __forceinline__ void back_tile(const RunParams &p, const AdjBack &b, int cta, unsigned char *smem) {
    const int N = p.N, K = p.K, TT = p.TT;
    const int LD = TT + 4;
    const int TXN = TT / 4, TYN = kThreads / TXN;
    const int KB = min(N, max(1, kChunkBytes / (int)(N * sizeof(R))));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double *lsum = reinterpret_cast<double *>(smem);  // [N][2]: im, re sums of the jumped spans (with 2 l)
    R *lsumR = reinterpret_cast<R *>(lsum + 2 * N);   // [N][2]: im, re sums of mu^* c of the other spans
    R *cdr = lsumR + 2 * N;                           // [N][2]: conj decay of the whole span, then [N] exp(2 Im K L)
    R *mre = cdr + 4 * N;
    R *mim = mre + (size_t)N * LD;
    R *osm = mim + (size_t)N * LD;  // [KB][N + 1]
    const int64_t t0 = (int64_t)cta * TT;
    const size_t MN2 = (size_t)p.M * N * 2;
    const R *segc = reinterpret_cast<const R *>(b.seg_c);
    R *segm = reinterpret_cast<R *>(b.seg_mu);
    R *carry = reinterpret_cast<R *>(b.carry);
    double *scr = b.wscr + ((size_t)cta * kWarps + warp) * 10 * N;
    const double bl = isnan(b.baseline) ? p.obs_sum[2 * (K - 1)] / (double)p.M : b.baseline;

    // adjoint at the end of g_end: the terminal condition (P - b) c_e at the last grid
    // point, else the carry of the later segment
    const int gsK = p.tab.meta[K - 1].gs_size;
    for (int i = tid; i < N * TT; i += kThreads) {
        const int t = i / N, a = i % N;
        R vr = 0, vi = 0;
        if (t0 + t < p.M) {
            if (b.g_end == K - 1) {
                const R *ce = segc + ((size_t)(b.g_end - b.g_begin) * 2 + 1) * MN2 + (size_t)(t0 + t) * N * 2;
                const R w = (R)((a < gsK ? 1.0 : 0.0) - bl);
                vr = w * ce[2 * a];
                vi = w * ce[2 * a + 1];
            } else {
                vr = carry[((size_t)(t0 + t) * N + a) * 2];
                vi = carry[((size_t)(t0 + t) * N + a) * 2 + 1];
            }
        }
        mre[a * LD + t] = vr;
        mim[a * LD + t] = vi;
    }
    const int tx = tid % TXN, ty = tid / TXN;
    for (int g = b.g_end; g >= b.g_begin; --g) {
        const int gl = g - b.g_begin;
        const double L = (g == 0 || g == K - 1) ? p.tau : 2.0 * p.tau;
        for (int a = tid; a < N; a += kThreads) {
            double re, im, e2;
            cdecay(p, g, a, L, &re, &im, &e2);
            cdr[2 * a] = (R)re;
            cdr[2 * a + 1] = (R)im;
            cdr[2 * N + a] = (R)e2;
            lsum[2 * a] = lsum[2 * a + 1] = 0.0;
            lsumR[2 * a] = lsumR[2 * a + 1] = (R)0;
        }
        __syncthreads();
        // ---- the span of g, one warp per trajectory ----------------------------------
        for (int t = warp; t < TT; t += kWarps) {
            const int64_t traj = t0 + t;
            if (traj >= p.M) continue;
            const R *ce = segc + ((size_t)gl * 2 + 1) * MN2 + (size_t)traj * N * 2;
            const R *cs = segc + ((size_t)gl * 2) * MN2 + (size_t)traj * N * 2;
            R *me = segm + ((size_t)gl * 2 + 1) * MN2 + (size_t)traj * N * 2;
            R *ms = segm + ((size_t)gl * 2) * MN2 + (size_t)traj * N * 2;
            for (int a = lane; a < N; a += 32) {
                me[2 * a] = mre[a * LD + t];
                me[2 * a + 1] = mim[a * LD + t];
            }
            // jumps of this trajectory inside g's span
            int k_lo = 0, k_hi = 0;
            const int nj = b.jn[traj];
            if (nj > 0) {
                int lo = nj, hi = 0;
                for (int k = 0; k < nj && k < b.slots; ++k)
                    if (b.jrec[(size_t)traj * b.slots + k].g == g) {
                        lo = min(lo, k);
                        hi = k + 1;
                    }
                if (hi > 0) {
                    k_lo = lo;
                    k_hi = hi;
                }
            }
            if (k_hi > k_lo) {
                // c_s, c_e and the adjoint in FP64 per-warp scratch; the general
                // jump operator uses a second block
                double *c_s = scr, *c_e = scr + 2 * N, *mu = scr + 4 * N;
                double *wk = scr + 6 * N;
                for (int a = lane; a < N; a += 32) {
                    c_s[2 * a] = g == 0 ? (a == 0 ? 1.0 : 0.0) : (double)cs[2 * a];
                    c_s[2 * a + 1] = g == 0 ? 0.0 : (double)cs[2 * a + 1];
                    c_e[2 * a] = (double)ce[2 * a];
                    c_e[2 * a + 1] = (double)ce[2 * a + 1];
                    mu[2 * a] = (double)mre[a * LD + t];
                    mu[2 * a + 1] = (double)mim[a * LD + t];
                }
                __syncwarp();
                span_with_jumps_any(p, b, g, traj, c_s, c_e, mu, lsum, k_lo, k_hi, wk, lane);
                for (int a = lane; a < N; a += 32) {
                    mre[a * LD + t] = (R)mu[2 * a];
                    mim[a * LD + t] = (R)mu[2 * a + 1];
                }
            } else {
                // no jump: mu_s = conj(D_L) mu_e / |D_L c_s|; mu^* c is the same at both
                // ends. In the state precision (the FP32 path's sums over a CTA's
                // trajectories are FP32; across CTAs and steps FP64).
                R s = (R)0;
                if (g == 0) {
                    s = cdr[2 * N];
                } else {
                    for (int a = lane; a < N; a += 32) {
                        const R re = cs[2 * a], im = cs[2 * a + 1];
                        s += (re * re + im * im) * cdr[2 * N + a];
                    }
                    s = warp_sum(s);
                }
                const R inv = (R)1 / sqrt(s);
                for (int a = lane; a < N; a += 32) {
                    const R mr_ = mre[a * LD + t], mi_ = mim[a * LD + t];
                    const R er = ce[2 * a], ei = ce[2 * a + 1];
                    atomicAdd(&lsumR[2 * a], mr_ * ei - mi_ * er);
                    atomicAdd(&lsumR[2 * a + 1], mr_ * er + mi_ * ei);
                    const R dr = cdr[2 * a], di = cdr[2 * a + 1];
                    mre[a * LD + t] = (dr * mr_ - di * mi_) * inv;
                    mim[a * LD + t] = (dr * mi_ + di * mr_) * inv;
                }
            }
            __syncwarp();
            for (int a = lane; a < N; a += 32) {
                ms[2 * a] = mre[a * LD + t];
                ms[2 * a + 1] = mim[a * LD + t];
            }
        }
        __syncthreads();
        for (int a = tid; a < N; a += kThreads) {
            atomicAdd(&b.lev[((size_t)g * N + a) * 2], lsum[2 * a] + 2.0 * L * (double)lsumR[2 * a]);
            atomicAdd(&b.lev[((size_t)g * N + a) * 2 + 1], lsum[2 * a + 1] + 2.0 * L * (double)lsumR[2 * a + 1]);
        }
        if (g == 0) break;
        // ---- frame rotation's adjoint: mu_e(g-1) = O_{g-1}^T mu_s(g) / |O c_e(g-1)| ------
        R accr[RA][4], acci[RA][4];
#pragma unroll
        for (int i = 0; i < RA; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) accr[i][j] = acci[i][j] = (R)0;
        const R *OT = reinterpret_cast<const R *>(p.tab.OT) + (size_t)(g - 1) * N * N;  // OT[b][a] = O[a][b]
        for (int a0 = 0; a0 < N; a0 += KB) {
            __syncthreads();
            // rows a0 .. a0 + KB - 1 of O, i.e. columns of OT, into osm[aa][b] (stride N + 1)
            for (int i = tid; i < KB * N; i += kThreads) {
                const int aa = i % KB, bb = i / KB;
                osm[aa * (N + 1) + bb] = OT[(size_t)bb * N + a0 + aa];
            }
            __syncthreads();
            for (int aa = 0; aa < KB; ++aa) {
                R vr[4], vi[4];
                load4(&mre[(a0 + aa) * LD + 4 * tx], vr);
                load4(&mim[(a0 + aa) * LD + 4 * tx], vi);
#pragma unroll
                for (int i = 0; i < RA; ++i) {
                    const int bo = ty + i * TYN;
                    const R o = bo < N ? osm[aa * (N + 1) + bo] : (R)0;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        accr[i][j] = fma(o, vr[j], accr[i][j]);
                        acci[i][j] = fma(o, vi[j], acci[i][j]);
                    }
                }
            }
        }
        __syncthreads();
        const double *nrot = b.seg_nrot + (size_t)gl * p.M;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int t = 4 * tx + j;
            const R sc = (t0 + t < p.M) ? (R)(1.0 / nrot[t0 + t]) : (R)0;
#pragma unroll
            for (int i = 0; i < RA; ++i) {
                const int bo = ty + i * TYN;
                if (bo < N) {
                    mre[bo * LD + t] = accr[i][j] * sc;
                    mim[bo * LD + t] = acci[i][j] * sc;
                }
            }
        }
        __syncthreads();
    }
    if (b.g_begin > 0) {
        // adjoint at the end of g_begin - 1 for the earlier segment
        for (int i = tid; i < N * TT; i += kThreads) {
            const int t = i / N, a = i % N;
            if (t0 + t < p.M) {
                carry[((size_t)(t0 + t) * N + a) * 2] = mre[a * LD + t];
                carry[((size_t)(t0 + t) * N + a) * 2 + 1] = mim[a * LD + t];
            }
        }
    }
}

template <typename R, int RA>
__global__ void __launch_bounds__(kThreads, 2)
    adjoint_segment(const __grid_constant__ RunParams p, const __grid_constant__ AdjBack b) {
    extern __shared__ __align__(16) unsigned char smem[];
    back_tile<R, RA>(p, b, blockIdx.x, smem);
}

// X_g = 2 sum over trajectories [Re(mu_e^* c_e^T) - Re(mu_s^* c_s^T)] for the grid
// points of a segment (start term for g >= 1, end term for g <= K - 2), added
// into FP64 xout [g][a][b] (zeroed before the first segment). One CTA per
// 128 x 128 output tile, grid point and block of kXM trajectories; 256
// threads, each 8 x 8 outputs: levels a0 + 4 ty + i and a0 + 64 + 4 ty + i (and
// the same for b with tx), so that a quarter-warp's operand loads fall on
// distinct banks but pairs; trajectories in chunks staged in shared memory,
// summed in the state precision over the block, then added in FP64 (atomics
// across the blocks).
constexpr int kXT = 128, kXM = 2048;

template <typename R>
__global__ void __launch_bounds__(256) adj_xgemm(const R *seg_c, const R *seg_mu, int64_t M, int N, int K,
                                                 int g_begin, double *xout) {
    constexpr int kXC = 16 / sizeof(R) * 2;  // trajectories per staged chunk: 8 (FP32), 4 (FP64)
    constexpr int V = 16 / sizeof(R);        // values per 16-byte vector
    typedef typename std::conditional<sizeof(R) == 4, float4, double2>::type vec;
    __shared__ __align__(16) R sa[2][kXC][2 * kXT];  // mu_e, mu_s
    __shared__ __align__(16) R sb[2][kXC][2 * kXT];  // c_e, c_s
    const int tiles = N / kXT;
    const int gl = blockIdx.y;
    const int g = g_begin + gl;
    const int a0 = (blockIdx.x / tiles) * kXT, b0 = (blockIdx.x % tiles) * kXT;
    const int64_t m0 = (int64_t)blockIdx.z * kXM, m1 = min(M, m0 + kXM);
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const bool has_e = g <= K - 2, has_s = g >= 1;
    const size_t MN2 = (size_t)M * N * 2;
    const R *ce = seg_c + ((size_t)gl * 2 + 1) * MN2, *cs = seg_c + ((size_t)gl * 2) * MN2;
    const R *me = seg_mu + ((size_t)gl * 2 + 1) * MN2, *ms = seg_mu + ((size_t)gl * 2) * MN2;
    R acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = (R)0;
    for (int64_t t0 = m0; t0 < m1; t0 += kXC) {
        __syncthreads();
        // 4 arrays x kXC trajectories x 2 kXT values, as 16-byte vectors
        constexpr int per = 2 * kXT / V;  // vectors per trajectory row
        for (int i = tid; i < 4 * kXC * per; i += 256) {
            const int w = i / (kXC * per), r = i % (kXC * per);
            const int t = r / per, v = r % per;
            const int64_t tr = t0 + t;
            const int lev0 = (w < 2 ? a0 : b0);
            const R *src = w == 0 ? me : w == 1 ? ms : w == 2 ? ce : cs;
            const bool on = tr < m1 && ((w % 2 == 0) ? has_e : has_s);
            vec val;
            if (on) val = *reinterpret_cast<const vec *>(src + (size_t)tr * N * 2 + 2 * lev0 + V * v);
            else val = vec{};
            R *dst = w < 2 ? &sa[w][t][V * v] : &sb[w - 2][t][V * v];
            *reinterpret_cast<vec *>(dst) = val;
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < kXC; ++t) {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const R sg = e == 0 ? (R)1 : (R)-1;
                R ar[8], ai[8], br[8], bi[8];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const R *pa = &sa[e][t][2 * (64 * h + 4 * ty)];
                    const R *pb = &sb[e][t][2 * (64 * h + 4 * tx)];
                    R va[8], vb[8];
#pragma unroll
                    for (int q = 0; q < 8 / V; ++q) {
                        *reinterpret_cast<vec *>(&va[V * q]) = *reinterpret_cast<const vec *>(pa + V * q);
                        *reinterpret_cast<vec *>(&vb[V * q]) = *reinterpret_cast<const vec *>(pb + V * q);
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        ar[4 * h + i] = sg * va[2 * i];
                        ai[4 * h + i] = sg * va[2 * i + 1];
                        br[4 * h + i] = vb[2 * i];
                        bi[4 * h + i] = vb[2 * i + 1];
                    }
                }
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fma(ar[i], br[j], fma(ai[i], bi[j], acc[i][j]));
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int a = a0 + 64 * (i >> 2) + 4 * ty + (i & 3);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int b = b0 + 64 * (j >> 2) + 4 * tx + (j & 3);
            atomicAdd(&xout[((size_t)g * N + a) * N + b], 2.0 * (double)acc[i][j]);
        }
    }
}

// The same for other N (not a multiple of 128): one thread per output entry,
// FP64 accumulation, written (not added).
template <typename R>
__global__ void __launch_bounds__(256) adj_xgemm_small(const R *seg_c, const R *seg_mu, int64_t M, int N, int K,
                                                       int g_begin, double *xout) {
    const int gl = blockIdx.y, g = g_begin + gl;
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= N * N) return;
    const int a = i / N, bb = i % N;
    const bool has_e = g <= K - 2, has_s = g >= 1;
    const size_t MN2 = (size_t)M * N * 2;
    const R *ce = seg_c + ((size_t)gl * 2 + 1) * MN2, *cs = seg_c + ((size_t)gl * 2) * MN2;
    const R *me = seg_mu + ((size_t)gl * 2 + 1) * MN2, *ms = seg_mu + ((size_t)gl * 2) * MN2;
    double acc = 0.0;
    for (int64_t t = 0; t < M; ++t) {
        const size_t o = (size_t)t * N * 2;
        if (has_e)
            acc += (double)me[o + 2 * a] * (double)ce[o + 2 * bb] + (double)me[o + 2 * a + 1] * (double)ce[o + 2 * bb + 1];
        if (has_s)
            acc -= (double)ms[o + 2 * a] * (double)cs[o + 2 * bb] + (double)ms[o + 2 * a + 1] * (double)cs[o + 2 * bb + 1];
    }
    xout[((size_t)g * N + a) * N + bb] = 2.0 * acc;
}

template <typename R, int RA>
int launch_back(const RunParams &p, const AdjBack &b, cudaStream_t st, size_t smem) {
    auto kern = adjoint_segment<R, RA>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    kern<<<p.n_cta, kThreads, smem, st>>>(p, b);
    return (int)cudaGetLastError();
}

template <typename R>
int launch_back_ra(const RunParams &p, const AdjBack &b, cudaStream_t st, size_t smem) {
    switch (p.RA) {
        case 1: return launch_back<R, 1>(p, b, st, smem);
        case 2: return launch_back<R, 2>(p, b, st, smem);
        case 4: return launch_back<R, 4>(p, b, st, smem);
        case 8: return launch_back<R, 8>(p, b, st, smem);
        default: return (int)cudaErrorInvalidValue;
    }
}

template <typename R>
int launch_xgemm(const void *seg_c, const void *seg_mu, int64_t M, int N, int K, int g_begin, int n_g, double *xout,
                 cudaStream_t st) {
    if (N % kXT == 0) {
        dim3 grid((N / kXT) * (N / kXT), n_g, (unsigned)((M + kXM - 1) / kXM));
        adj_xgemm<R><<<grid, 256, 0, st>>>(reinterpret_cast<const R *>(seg_c), reinterpret_cast<const R *>(seg_mu), M,
                                           N, K, g_begin, xout);
    } else {
        dim3 grid((N * N + 255) / 256, n_g);
        adj_xgemm_small<R><<<grid, 256, 0, st>>>(reinterpret_cast<const R *>(seg_c),
                                                 reinterpret_cast<const R *>(seg_mu), M, N, K, g_begin, xout);
    }
    return (int)cudaGetLastError();
}

}  // namespace adj
}  // namespace aqt
