// Jump resolution shared by the propagation kernels.
//
// arXiv:1710.03431, Sec. IV and App. C: inside one frozen half-step the
// squared norm of the normalised state evolves as
//   |c(t)|^2 = 1 + delta(t),   delta(t) = sum_a |c_a|^2 expm1(2 Im K_aa t)
// (K diagonal), and a jump happens when the clock ell + log1p(delta(t)) falls
// to the threshold log r. The warp that owns the trajectory holds its state in
// registers (level a = 32 j + lane in slot j), finds the crossing time by
// Newton's method (the function is convex and decreasing), draws the channel
// with the probabilities of App. B.1 (Eq. Pi(t)), applies the Bohr-class
// operator (Eq. jump), renormalises, draws a new threshold and finishes the
// half-step, possibly jumping again.
//
// Precision: the state and its no-jump propagation are in the state's
// precision T (double on the FP64 path; float on the FP32 and tensor-core
// paths). Everything that decides a jump is FP64 on every path: the clock,
// the decay sums delta(t) formed from the populations |c_a|^2 (exact products
// of the state's entries), the crossing time (for float states a cheap FP32
// Newton start, then Newton on the FP64 function), and the cumulative sums of
// both channel draws. Writing the decay as expm1 terms keeps its relative
// accuracy however small it is.
//
// Fast path (every manifold a single level and every Bohr class of nonzero
// frequency a single level pair, the generic case once s > 0): stage one
// picks (alpha, source b) from the FP64 rates G; stage two needs column b of
// R_alpha = sqrt(gamma) M_alpha, M_alpha = V^T sz_alpha V: a table row for the
// lowest sources (where the population is), otherwise a column of M_alpha
// that the warp forms from the eigenvector table (O(N^2) per jump), weighted
// by gamma(E_b - E_a). The class operator then maps the source level to the
// target level alone, or, at zero frequency, scales each level by the
// diagonal of M_alpha. Other grid points
// go through a general FP64 routine over degenerate manifolds and
// multi-pair classes, with the full jump amplitudes of those grid points.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "aqt_internal.h"
#include "philox.cuh"

namespace aqt {
namespace dev {

constexpr int kMaxJumpsPerHalf = 64;
constexpr int kMaxAlpha = 16;
enum : int32_t { kStatusNumeric = 2, kStatusTimeout = 4, kStatusAdjSlots = 8 };

template <typename T>
static __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Two sums in one pass of butterfly shuffles (the xor butterfly leaves the
// same value on every lane: each addition meets the same operand pair).
template <typename T>
static __device__ __forceinline__ void warp_sum2(T &a, T &b) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
}

static __device__ __forceinline__ float m_exp(float x) { return expf(x); }
static __device__ __forceinline__ double m_exp(double x) { return exp(x); }
static __device__ __forceinline__ float m_expm1(float x) { return expm1f(x); }
static __device__ __forceinline__ double m_expm1(double x) { return expm1(x); }
static __device__ __forceinline__ float m_log1p(float x) { return log1pf(x); }
static __device__ __forceinline__ double m_log1p(double x) { return log1p(x); }
static __device__ __forceinline__ float m_rsqrt(float x) { return rsqrtf(x); }
static __device__ __forceinline__ double m_rsqrt(double x) { return 1.0 / sqrt(x); }
static __device__ __forceinline__ void m_sincos(float x, float *s, float *c) { sincosf(x, s, c); }
static __device__ __forceinline__ void m_sincos(double x, double *s, double *c) { sincos(x, s, c); }

// v[j] for a warp-uniform runtime j, without indexing the register array.
template <typename T, int NPL>
static __device__ __forceinline__ T reg_at(const T (&v)[NPL], int j) {
    T r = v[0];
#pragma unroll
    for (int i = 1; i < NPL; ++i)
        if (i == j) r = v[i];
    return r;
}

// Inverse-CDF pick over items i = 32 j + lane with weights w[j] (zero past the
// end): the first item whose inclusive prefix sum exceeds target; if rounding
// leaves none, the last item of positive weight; -1 if all weights are zero.
// Same result on every lane.
template <typename T, int NPL>
static __device__ __forceinline__ int reg_pick(const T (&w)[NPL], T target, int lane) {
    T tot[NPL];
#pragma unroll
    for (int j = 0; j < NPL; ++j) tot[j] = w[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int j = 0; j < NPL; ++j) tot[j] += __shfl_xor_sync(0xffffffffu, tot[j], o);
    T cum = T(0);
    int jsel = -1;
#pragma unroll
    for (int j = 0; j < NPL; ++j)
        if (jsel < 0) {
            if (tot[j] > T(0) && cum + tot[j] > target) jsel = j;
            else cum += tot[j];
        }
    if (jsel >= 0) {
        const T wj = reg_at(w, jsel);
        T pre = wj;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T u = __shfl_up_sync(0xffffffffu, pre, o);
            if (lane >= o) pre += u;
        }
        const unsigned hit = __ballot_sync(0xffffffffu, wj > T(0) && cum + pre > target);
        if (hit) return 32 * jsel + __ffs(hit) - 1;
    }
    int last = -1;
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
        const unsigned pos = __ballot_sync(0xffffffffu, w[j] > T(0));
        if (pos) last = 32 * j + 31 - __clz(pos);
    }
    return last;
}

// General jump (any grid point): draw (alpha, source manifold) and the target
// level with the two-stage probabilities of App. B.1, then apply the Bohr-class
// operator A_{alpha, omega*} (Eq. jump) in FP64. c64 holds the normalised
// state (N entries) and receives the normalised post-jump state; y64 is
// scratch. Returns alpha (or -1 on a numeric failure), source and target.
using RT = double;
static __device__ int general_draw_apply(const RunParams &p, int g, double u1, double u2, double2 *c64, double2 *y64,
                                         int lane, int *bsrc_out, int *adst_out) {
    const int N = p.N, n = p.n;
    const double *lvlE = p.tab.lvlE + (size_t)g * N;
    const int32_t *mfirst = p.tab.mfirst + (size_t)g * N;
    const int32_t *msize = p.tab.msize + (size_t)g * N;
    const GridMeta meta = p.tab.meta[g];
    const int slot = p.tab.gslot[g];
    if (slot < 0) return -1;  // tables missing for this grid point
    const RT *Rg = p.tab.Rgen + (size_t)slot * n * N * N;  // [alpha][b][a]
    const double *Gg = p.tab.G + (size_t)g * n * N;
    // stage-one weight of unit (alpha, manifold starting at b); -1 marks a
    // degenerate manifold, whose weight the warp computes with manifold_w
    auto unit_w = [&](int al, int b) -> double {
        if (mfirst[b] != b) return 0.0;
        if (msize[b] == 1) {
            const double2 v = c64[b];
            return (v.x * v.x + v.y * v.y) * Gg[(size_t)al * N + b];
        }
        return -1.0;
    };
    // |R_alpha P_B c|^2 for the degenerate manifold B starting at b (the rate
    // depends on manifold energies only, so it sits inside R)
    auto manifold_w = [&](int al, int b) -> double {
        const int ms = msize[b];
        const RT *Ra = Rg + (size_t)al * N * N;
        double acc = 0.0;
        for (int a = lane; a < N; a += 32) {
            double yr = 0.0, yi = 0.0;
            for (int bp = b; bp < b + ms; ++bp) {
                const double m = (double)Ra[(size_t)bp * N + a];
                yr += m * c64[bp].x;
                yi += m * c64[bp].y;
            }
            acc += yr * yr + yi * yi;
        }
        return warp_sum(acc);
    };
    double S[kMaxAlpha];
    double total = 0.0;
    for (int al = 0; al < n; ++al) {
        double acc = 0.0;
        for (int b = lane; b < N; b += 32) {
            const double w = unit_w(al, b);
            if (w > 0.0) acc += w;
        }
        acc = warp_sum(acc);
        if (meta.degenerate) {
            for (int b = 0; b < N; ++b)
                if (mfirst[b] == b && msize[b] > 1) acc += manifold_w(al, b);
        }
        S[al] = acc;
        total += acc;
    }
    int al_s = -1;
    double cum = 0.0;
    const double target = u1 * total;
    for (int al = 0; al < n; ++al) {
        if (S[al] > 0.0 && cum + S[al] > target) {
            al_s = al;
            break;
        }
        cum += S[al];
    }
    if (al_s < 0)
        for (int al = n - 1; al >= 0; --al)
            if (S[al] > 0.0) {
                al_s = al;
                cum = 0.0;
                for (int q = 0; q < al; ++q) cum += S[q];
                break;
            }
    if (al_s < 0) return -1;  // no channel has weight: cannot happen for a decaying norm
    // source unit: walk the manifolds of alpha in level order
    int bsrc = -1, lastb = -1;
    {
        double c2 = cum;
        for (int b0 = 0; b0 < N && bsrc < 0; b0 += 32) {
            const int b = b0 + lane;
            double w = 0.0;
            if (b < N) {
                w = unit_w(al_s, b);
                if (w < 0.0) w = 0.0;
            }
            const bool has_deg = __any_sync(0xffffffffu, b < N && mfirst[b] == b && msize[b] > 1);
            if (!has_deg) {
                double pre = w;
                for (int o = 1; o < 32; o <<= 1) {
                    const double u = __shfl_up_sync(0xffffffffu, pre, o);
                    if (lane >= o) pre += u;
                }
                const unsigned pos = __ballot_sync(0xffffffffu, w > 0.0);
                if (pos) lastb = b0 + 31 - __clz(pos);
                const unsigned hit = __ballot_sync(0xffffffffu, w > 0.0 && c2 + pre > target);
                if (hit) bsrc = b0 + __ffs(hit) - 1;
                c2 += __shfl_sync(0xffffffffu, pre, 31);
            } else {
                for (int i = 0; i < 32 && b0 + i < N && bsrc < 0; ++i) {
                    const int bb = b0 + i;
                    if (mfirst[bb] != bb) continue;
                    const double wb = msize[bb] == 1 ? __shfl_sync(0xffffffffu, w, i) : manifold_w(al_s, bb);
                    if (wb > 0.0) lastb = bb;
                    if (wb > 0.0 && c2 + wb > target) bsrc = bb;
                    c2 += wb;
                }
            }
        }
        if (bsrc < 0) bsrc = lastb;
    }
    if (bsrc < 0) return -1;
    // stage two: target level a, weight |(R_alpha P_B c)_a|^2
    const int ms = msize[bsrc];
    const RT *Ra = Rg + (size_t)al_s * N * N;
    auto target_w = [&](int a) -> double {
        if (ms == 1) {
            const double m = (double)Ra[(size_t)bsrc * N + a];
            return m * m;
        }
        double yr = 0.0, yi = 0.0;
        for (int bp = bsrc; bp < bsrc + ms; ++bp) {
            const double m = (double)Ra[(size_t)bp * N + a];
            yr += m * c64[bp].x;
            yi += m * c64[bp].y;
        }
        return yr * yr + yi * yi;
    };
    double tot2 = 0.0;
    for (int a = lane; a < N; a += 32) tot2 += target_w(a);
    tot2 = warp_sum(tot2);
    int adst = -1, lasta = -1;
    {
        double c2 = 0.0;
        const double tg = u2 * tot2;
        for (int a0 = 0; a0 < N && adst < 0; a0 += 32) {
            const int a = a0 + lane;
            const double w = a < N ? target_w(a) : 0.0;
            double pre = w;
            for (int o = 1; o < 32; o <<= 1) {
                const double u = __shfl_up_sync(0xffffffffu, pre, o);
                if (lane >= o) pre += u;
            }
            const unsigned pos = __ballot_sync(0xffffffffu, w > 0.0);
            if (pos) lasta = a0 + 31 - __clz(pos);
            const unsigned hit = __ballot_sync(0xffffffffu, w > 0.0 && c2 + pre > tg);
            if (hit) adst = a0 + __ffs(hit) - 1;
            c2 += __shfl_sync(0xffffffffu, pre, 31);
        }
        if (adst < 0) adst = lasta;
    }
    if (adst < 0) return -1;
    // class operator: y_a = sum over b with E_b - E_a = omega* (within tol) of R_alpha[a][b] c_b
    const double wstar = lvlE[bsrc] - lvlE[adst];
    const double tol = meta.tol;
    double s = 0.0;
    for (int a = lane; a < N; a += 32) {
        const double lo_e = lvlE[a] + wstar - tol, hi_e = lvlE[a] + wstar + tol;
        int lo = 0, hi = N;  // first level with lvlE >= lo_e
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (lvlE[mid] < lo_e) lo = mid + 1; else hi = mid;
        }
        double yr = 0.0, yi = 0.0;
        for (int bp = lo; bp < N && lvlE[bp] <= hi_e; ++bp) {
            const double amp = (double)Ra[(size_t)bp * N + a];
            yr += amp * c64[bp].x;
            yi += amp * c64[bp].y;
        }
        y64[a] = make_double2(yr, yi);
        s += yr * yr + yi * yi;
    }
    s = warp_sum(s);
    __syncwarp();
    if (!(s > 0.0)) return -1;
    const double inv = 1.0 / sqrt(s);
    for (int a = lane; a < N; a += 32) c64[a] = make_double2(y64[a].x * inv, y64[a].y * inv);
    __syncwarp();
    *bsrc_out = bsrc;
    *adst_out = adst;
    return al_s;
}

// Gamma of the Ohmic bath (Sec. V): 2 pi eta g^2 w e^{-|w|/w_c} / (1 - e^{-beta w}),
// with its limit 2 pi eta g^2 / beta at w = 0, in the state's precision (the
// stage-two weights need no more accuracy than the state's column of M).
static __device__ __forceinline__ double bath_gamma(const RunParams &p, double w) {
    if (w == 0.0) return 2.0 * 3.14159265358979323846 * p.eta_g2 / p.beta;
    return 2.0 * 3.14159265358979323846 * p.eta_g2 * w * exp(-fabs(w) / p.omega_c) / (-expm1(-p.beta * w));
}
static __device__ __forceinline__ float bath_gamma(const RunParams &p, float w) {
    const float c = 6.2831853071795864769f * (float)p.eta_g2;
    if (w == 0.0f) return c / (float)p.beta;
    return c * w * expf(-fabsf(w) / (float)p.omega_c) / (-expm1f(-(float)p.beta * w));
}

// e^y - 1 in FP64. For |y| <= 2^-6 (every decay exponent 2 Im K_aa t of a
// frozen half-step at the grid sizes used here) the Taylor polynomial of
// degree 7 in Horner form: its truncation error is below y^8 / 8! < 1e-17 |y|.
// Otherwise the library function.
static __device__ __forceinline__ double expm1_small(double y) {
    if (fabs(y) > 0.015625) return expm1(y);
    return y * (1.0 + y * (1.0 / 2 + y * (1.0 / 6 + y * (1.0 / 24 + y * (1.0 / 120 + y * (1.0 / 720 + y * (1.0 / 5040)))))));
}

// Column b of M_alpha = V^T sz_alpha V at grid point g for the levels a = 32 j
// + lane of this lane: M[a][b] = delta_ab - 2 sum over basis states x with bit
// alpha set of V[x][a] V[x][b] (sz_alpha = 1 - 2 P_alpha). V in the state's
// precision, accumulated in it.
template <typename T, int NPL>
static __device__ __forceinline__ void m_column(const RunParams &p, int g, int al, int b, int lane, T (&m)[NPL]) {
    const int N = p.N;
    const T *Vg = static_cast<const T *>(p.tab.V) + (size_t)g * N * N;
#pragma unroll
    for (int j = 0; j < NPL; ++j) m[j] = T(0);
    const int lo_mask = (1 << al) - 1;
#pragma unroll 8
    for (int i = 0; i < N / 2; ++i) {
        const int x = ((i >> al) << (al + 1)) | (1 << al) | (i & lo_mask);
        const T *row = Vg + (size_t)x * N;
        const T vb = row[b];
#pragma unroll
        for (int j = 0; j < NPL; ++j) {
            const int a = 32 * j + lane;
            if (a < N) m[j] = fma(row[a], vb, m[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < NPL; ++j) m[j] = (32 * j + lane == b ? T(1) : T(0)) - T(2) * m[j];
}

// Draw the jump channel with (u1, u2) (two stages, App. B.1 Eq. Pi(t)) and
// apply its Bohr-class operator (Eq. jump) to the normalised state held in
// registers (level a = 32 j + lane), which is replaced by the normalised
// post-jump state. Returns alpha, or -1 on a numeric failure; *bsrc_out and
// *adst_out get the source and target levels.
template <typename T, int NPL>
static __device__ __forceinline__ int draw_apply(const RunParams &p, int g, T (&cr)[NPL], T (&ci)[NPL], double u1,
                                                 double u2, int lane, double2 *slow, int *bsrc_out, int *adst_out) {
    const int N = p.N, n = p.n;
    const GridMeta meta = p.tab.meta[g];
    const double *kd = p.tab.kdiag + (size_t)g * N * 2;
    const double *Gg = p.tab.G + (size_t)g * n * N;
    const bool fast = meta.simple && !meta.degenerate;
    auto kim2d = [&](int j) -> double {
        const int a = 32 * j + lane;
        return a < N ? 2.0 * kd[2 * a + 1] : 0.0;
    };
    auto pop = [&](int j) -> double { return (double)cr[j] * (double)cr[j] + (double)ci[j] * (double)ci[j]; };
    int al = -1, bsrc = -1, adst = -1;
    if (fast) {
        double qv[NPL];
#pragma unroll
        for (int j = 0; j < NPL; ++j) qv[j] = pop(j);
        // stage one over units (alpha, b) in that order. The total rate is
        // sum_b |c_b|^2 sum_alpha G_alpha[b] = -sum_b |c_b|^2 2 Im K_bb, so the
        // walk over alpha stops at the first alpha whose cumulative sum passes
        // the target, one warp sum per alpha visited.
        double total = 0.0, cum = 0.0, cum_last = 0.0;
        int last = -1;
#pragma unroll
        for (int j = 0; j < NPL; ++j) total -= qv[j] * kim2d(j);
        total = warp_sum(total);
        const double target = u1 * total;
        for (int a_ = 0; a_ < n && al < 0; ++a_) {
            double acc = 0.0;
#pragma unroll
            for (int j = 0; j < NPL; ++j) {
                const int b = 32 * j + lane;
                if (b < N) acc += qv[j] * Gg[(size_t)a_ * N + b];
            }
            acc = warp_sum(acc);
            if (acc > 0.0) {
                last = a_;
                cum_last = cum;
            }
            if (acc > 0.0 && cum + acc > target) al = a_;
            else cum += acc;
        }
        if (al < 0) {  // rounding at the top of the distribution
            al = last;
            cum = cum_last;
        }
        if (al >= 0) {
            double w[NPL];
#pragma unroll
            for (int j = 0; j < NPL; ++j) {
                const int b = 32 * j + lane;
                w[j] = b < N ? qv[j] * Gg[(size_t)al * N + b] : 0.0;
            }
            bsrc = reg_pick(w, target - cum, lane);
        }
        if (bsrc >= 0) {
            // stage two: target a with weight R_alpha[a][b]^2 = gamma(E_b - E_a) M_alpha[a][b]^2,
            // from the table for the lowest sources, else from a column of M formed here
            T m[NPL];
            double w[NPL], tot2 = 0.0;
            if (bsrc < p.n_low) {
                const T *row = static_cast<const T *>(p.tab.Rlow) + (((size_t)g * n + al) * p.n_low + bsrc) * N;
#pragma unroll
                for (int j = 0; j < NPL; ++j) {
                    const int a = 32 * j + lane;
                    m[j] = a < N ? row[a] : T(0);
                    w[j] = (double)m[j] * (double)m[j];
                    tot2 += w[j];
                }
            } else {
                m_column<T, NPL>(p, g, al, bsrc, lane, m);
                const double *lvlE = p.tab.lvlE + (size_t)g * N;
                const double eb = lvlE[bsrc];
#pragma unroll
                for (int j = 0; j < NPL; ++j) {
                    const int a = 32 * j + lane;
                    w[j] = a < N ? (double)bath_gamma(p, (T)(eb - lvlE[a])) * ((double)m[j] * (double)m[j]) : 0.0;
                    tot2 += w[j];
                }
            }
            tot2 = warp_sum(tot2);
            adst = reg_pick(w, u2 * tot2, lane);
            if (adst >= 0 && adst != bsrc) {
                // nonzero frequency: the class is the single pair (adst <- bsrc), so
                // the normalised result is sign(M[adst][bsrc]) c_bsrc / |c_bsrc| on adst
                const T br = __shfl_sync(0xffffffffu, reg_at(cr, bsrc >> 5), bsrc & 31);
                const T bi = __shfl_sync(0xffffffffu, reg_at(ci, bsrc >> 5), bsrc & 31);
                const T ra = __shfl_sync(0xffffffffu, reg_at(m, adst >> 5), adst & 31);
                const T m2 = br * br + bi * bi;
                if (m2 > T(0)) {
                    const T f = (ra < T(0) ? T(-1) : T(1)) * m_rsqrt(m2);
#pragma unroll
                    for (int j = 0; j < NPL; ++j) {
                        const bool hit = 32 * j + lane == adst;
                        cr[j] = hit ? br * f : T(0);
                        ci[j] = hit ? bi * f : T(0);
                    }
                } else {
                    al = -1;
                }
            } else if (adst >= 0) {
                // zero frequency: every level pairs with itself, y_a = sqrt(gamma(0)) M_alpha[a][a] c_a
                const double *Md = p.tab.Mdiag + ((size_t)g * n + al) * N;
                T s = T(0);
#pragma unroll
                for (int j = 0; j < NPL; ++j) {
                    const int a = 32 * j + lane;
                    const T d = a < N ? (T)Md[a] : T(0);
                    cr[j] *= d;
                    ci[j] *= d;
                    s += cr[j] * cr[j] + ci[j] * ci[j];
                }
                s = warp_sum(s);
                if (s > T(0)) {
                    const T inv = m_rsqrt(s);
#pragma unroll
                    for (int j = 0; j < NPL; ++j) {
                        cr[j] *= inv;
                        ci[j] *= inv;
                    }
                } else {
                    al = -1;
                }
            }
        }
        if (bsrc < 0 || adst < 0) al = -1;
    } else {
#pragma unroll
        for (int j = 0; j < NPL; ++j) {
            const int a = 32 * j + lane;
            if (a < N) slow[a] = make_double2((double)cr[j], (double)ci[j]);
        }
        __syncwarp();
        al = general_draw_apply(p, g, u1, u2, slow, slow + N, lane, &bsrc, &adst);
#pragma unroll
        for (int j = 0; j < NPL; ++j) {
            const int a = 32 * j + lane;
            if (a < N) {
                cr[j] = (T)slow[a].x;
                ci[j] = (T)slow[a].y;
            }
        }
        __syncwarp();
    }
    *bsrc_out = bsrc;
    *adst_out = adst;
    return al;
}

// Append one jump record (lane 0; records past the capacity are counted, not kept).
static __device__ __forceinline__ void record_jump(const RunParams &p, int64_t traj, int g, int half, int al, int bsrc,
                                                   int adst, double t, int lane) {
    const int N = p.N;
    if (lane == 0) {
        const unsigned long long idx = atomicAdd(p.jcount, 1ull);
        if ((int64_t)idx < p.jcap) {
            const double *lvlE = p.tab.lvlE + (size_t)g * N;
            aqt_jump rec;
            rec.traj = (int32_t)traj;
            rec.grid = g;
            rec.half = half;
            rec.alpha = al;
            rec.src = bsrc;
            rec.dst = p.tab.mfirst[(size_t)g * N + adst];
            rec.t = t;
            rec.omega = lvlE[bsrc] - lvlE[adst];
            p.jumps[idx] = rec;
        }
    }
}

// One frozen half-step of one trajectory that may cross its threshold,
// resolved by one warp with the state in registers (NPL levels per lane,
// 32 NPL >= N). sre/sim: the state, level a at [a * stride] (normalised or
// not); on return, the normalised state at the end of the half-step. ell,
// logr, nj: the trajectory's clock, log threshold and jump count (the same on
// every lane). slow: 2N double2 of per-warp scratch for the general jump.
// klev (FP32 paths, optional): (Re K_aa, 2 Im K_aa) of grid point g staged in
// shared memory for the FP32 propagation; otherwise the FP64 table is read.
template <typename T, int NPL>
static __device__ __forceinline__ void jump_half_step(const RunParams &p, int g, int half, int64_t traj, T *sre,
                                                      T *sim, int stride, double &ell, double &logr, int &nj,
                                                      int lane, double2 *slow, const float2 *klev = nullptr) {
    constexpr bool f32 = std::is_same<T, float>::value;
    const int N = p.N;
    const double *kd = p.tab.kdiag + (size_t)g * N * 2;
    T cr[NPL], ci[NPL];
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
        const int a = 32 * j + lane;
        const bool v = a < N;
        cr[j] = v ? sre[(size_t)a * stride] : T(0);
        ci[j] = v ? sim[(size_t)a * stride] : T(0);
    }
    // diagonal of K per level (re, 2 im) in the state's precision, re-read from
    // the cache where used to keep registers free
    auto kre = [&](int j) -> T {
        const int a = 32 * j + lane;
        if constexpr (f32)
            if (klev) return a < N ? klev[a].x : 0.0f;
        return a < N ? (T)kd[2 * a] : T(0);
    };
    auto kim2 = [&](int j) -> T {
        const int a = 32 * j + lane;
        if constexpr (f32)
            if (klev) return a < N ? klev[a].y : 0.0f;
        return a < N ? (T)(2.0 * kd[2 * a + 1]) : T(0);
    };
    // 2 Im K_aa in FP64 (decay sums of the clock)
    auto kim2d = [&](int j) -> double {
        const int a = 32 * j + lane;
        return a < N ? 2.0 * kd[2 * a + 1] : 0.0;
    };
    // |c_a|^2 in FP64 (exact for float entries)
    auto pop = [&](int j) -> double { return (double)cr[j] * (double)cr[j] + (double)ci[j] * (double)ci[j]; };
    // c <- c exp(-i K t) / |.|; false if the norm is not positive and finite
    auto advance = [&](T t) -> bool {
        T s = T(0);
#pragma unroll
        for (int j = 0; j < NPL; ++j) {
            T sn, cs;
            m_sincos(kre(j) * t, &sn, &cs);
            const T amp = m_exp(T(0.5) * kim2(j) * t);
            const T r = amp * (cr[j] * cs + ci[j] * sn), i = amp * (ci[j] * cs - cr[j] * sn);
            cr[j] = r;
            ci[j] = i;
            s += r * r + i * i;
        }
        s = warp_sum(s);
        if (!(s > T(0)) || !isfinite(s)) return false;
        const T inv = m_rsqrt(s);
#pragma unroll
        for (int j = 0; j < NPL; ++j) {
            cr[j] *= inv;
            ci[j] *= inv;
        }
        return true;
    };
    // delta(t) of the normalised state and its derivative, FP64
    auto decay64 = [&](double t, double *d1) -> double {
        double d = 0.0, e1 = 0.0;
#pragma unroll
        for (int j = 0; j < NPL; ++j) {
            const double q = pop(j), x = kim2d(j);
            const double e = expm1_small(x * t);
            d += q * e;
            e1 += q * x * (e + 1.0);
        }
        warp_sum2(d, e1);
        *d1 = e1;
        return d;
    };
    // the same in single precision (a cheap start for the root of float states)
    auto decay32 = [&](float t, float *d1) -> float {
        float d = 0.0f, e1 = 0.0f;
#pragma unroll
        for (int j = 0; j < NPL; ++j) {
            const float q = (float)(cr[j] * cr[j] + ci[j] * ci[j]);
            const float x = (float)kim2(j);
            const float e = expm1f(x * t);
            d += q * e;
            e1 += q * x * (e + 1.0f);
        }
        warp_sum2(d, e1);
        *d1 = e1;
        return d;
    };
    bool ok = advance(T(0));
    double ell0 = ell;
    double tau_rem = p.tau;
    const double t_half0 = half == 0 ? g * p.dt - p.tau : g * p.dt;
    double dend = 0.0;
    for (int it = 0; ok; ++it) {
        double dd;
        const double C = ell0 - logr;  // > 0 until the threshold is reached
        if constexpr (f32) {
            // float states: a single-precision decay sum first. It differs from
            // the FP64 sum by at most ~1e-6 of |delta| (FP32 products and sums of
            // at most N terms), so a margin of 1e-5 |delta| shows that the
            // threshold is not reached without the FP64 sum; then the clock takes
            // the single-precision decay, as the tensor-core epilogue's does.
            float d1f;
            const float d32 = decay32((float)tau_rem, &d1f);
            if (C + log1p((double)d32) > 1e-5 * fabs((double)d32) + 1e-12) {
                dend = (double)d32;
                break;
            }
        }
        dend = decay64(tau_rem, &dd);
        if (C + log1p(dend) > 0.0) break;
        if (it >= kMaxJumpsPerHalf) {
            ok = false;
            break;
        }
        // --- crossing time --------------------------------------------------------------
        double t = tau_rem;  // GRID timing: the end of the half-step
        if (p.timing == kTimingRefined) {
            t = 0.0;
            if constexpr (f32) {
                // FP32 Newton from the left to ~1e-3 relative
                const float Cf = (float)C;
                float tf = 0.0f;
                for (int k = 0; k < 40; ++k) {
                    float d1;
                    const float d = decay32(tf, &d1);
                    const float phi = Cf + log1pf(d);
                    if (!(phi > 0.0f) || !(d1 < 0.0f)) break;
                    const float step = -phi * (1.0f + d) / d1;
                    float tn = tf + step;
                    if (tn > (float)tau_rem) tn = (float)tau_rem;
                    if (!(tn > tf)) break;
                    tf = tn;
                    if (step <= 1e-6f * tf) break;
                }
                t = (double)tf;
            }
            // Newton on the FP64 function (from either side: convexity brings an
            // iterate right of the root back to its left in one step). The
            // function is nearly linear over a half-step (its curvature relative to
            // its slope is the decay rate, and rate x tau << 1), so a step of s
            // leaves an error ~ rate s^2: from the FP32 start (~1e-6 t) one step
            // lands within ~1e-12 t, and a step below 1e-5 t ends the iteration.
            const double stop_rel = f32 ? 1e-5 : 1e-7;
            for (int k = 0; k < 60; ++k) {
                double d1;
                const double d = decay64(t, &d1);
                const double phi = C + log1p(d);
                if (phi == 0.0 || !(d1 < 0.0)) break;
                if (!f32 && !(phi > 0.0)) break;
                const double step = -phi * (1.0 + d) / d1;
                double tn = t + step;
                if (tn > tau_rem) tn = tau_rem;
                if (tn < 0.0) tn = 0.0;
                if (tn == t) break;
                t = tn;
                if (fabs(step) <= stop_rel * t) break;
            }
        }
        if (!advance((T)t)) {
            ok = false;
            break;
        }
        // --- draw and apply the jump --------------------------------------------------
        ++nj;
        const Philox4 rnd = traj_event(p.seed, traj, nj);
        const double u1 = uniform01(rnd.x[0]), u2 = uniform01(rnd.x[1]), u3 = uniform01(rnd.x[2]);
        // segment recompute of a gradient run: keep the states around the jump
        int aslot = -1;
        if (p.adj.jrec) {
            aslot = __shfl_sync(0xffffffffu, lane == 0 ? p.adj.jn[traj] : 0, 0);
            if (aslot < p.adj.slots) {
                double *v = p.adj.jvec + ((size_t)traj * p.adj.slots + aslot) * 4 * N;
#pragma unroll
                for (int j = 0; j < NPL; ++j) {
                    const int a = 32 * j + lane;
                    if (a < N) {
                        v[2 * a] = (double)cr[j];
                        v[2 * a + 1] = (double)ci[j];
                    }
                }
            } else if (lane == 0) {
                atomicOr(p.status, kStatusAdjSlots);
            }
        }
        int bsrc = -1, adst = -1;
        const int al = draw_apply<T, NPL>(p, g, cr, ci, u1, u2, lane, slow, &bsrc, &adst);
        if (al < 0) {
            ok = false;
            break;
        }
        if (aslot >= 0 && aslot < p.adj.slots) {
            double *v = p.adj.jvec + (((size_t)traj * p.adj.slots + aslot) * 2 + 1) * 2 * N;
#pragma unroll
            for (int j = 0; j < NPL; ++j) {
                const int a = 32 * j + lane;
                if (a < N) {
                    v[2 * a] = (double)cr[j];
                    v[2 * a + 1] = (double)ci[j];
                }
            }
            if (lane == 0) {
                const GridMeta meta = p.tab.meta[g];
                AdjJump r;
                r.g = g;
                r.half = half;
                r.alpha = al;
                r.bsrc = bsrc;
                r.adst = adst;
                r.general = !(meta.simple && !meta.degenerate);
                r.t_rel = (p.tau - tau_rem) + t;
                p.adj.jrec[(size_t)traj * p.adj.slots + aslot] = r;
                p.adj.jn[traj] = aslot + 1;
            }
        }
        record_jump(p, traj, g, half, al, bsrc, adst, t_half0 + (p.tau - tau_rem) + t, lane);
        __syncwarp();
        logr = log(u3);
        ell0 = 0.0;
        tau_rem -= t;
    }
    if (!ok && lane == 0) atomicOr(p.status, kStatusNumeric);
    // finish the half-step without further jumps
    advance((T)tau_rem);
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
        const int a = 32 * j + lane;
        if (a < N) {
            sre[(size_t)a * stride] = cr[j];
            sim[(size_t)a * stride] = ci[j];
        }
    }
    ell = ell0 + log1p(dend);
    __syncwarp();
}

// The jump of the fixed-step sampler (App. B.1): at the start of a frozen
// half-step whose jump test fired, draw the channel with (u1, u2) and apply it
// to the state (no deterministic evolution in this half-step); the state at
// sre/sim (level a at [a * stride], any norm) is replaced by the normalised
// post-jump state. Jump time: the start of the half-step.
template <typename T, int NPL>
static __device__ __forceinline__ void fixed_step_jump(const RunParams &p, int g, int half, int64_t traj, T *sre, T *sim,
                                                       int stride, double u1, double u2, int lane, double2 *slow) {
    const int N = p.N;
    T cr[NPL], ci[NPL];
    T s = T(0);
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
        const int a = 32 * j + lane;
        const bool v = a < N;
        cr[j] = v ? sre[(size_t)a * stride] : T(0);
        ci[j] = v ? sim[(size_t)a * stride] : T(0);
        s += cr[j] * cr[j] + ci[j] * ci[j];
    }
    s = warp_sum(s);
    int al = -1, bsrc = -1, adst = -1;
    if (s > T(0) && isfinite(s)) {
        const T inv = m_rsqrt(s);
#pragma unroll
        for (int j = 0; j < NPL; ++j) {
            cr[j] *= inv;
            ci[j] *= inv;
        }
        al = draw_apply<T, NPL>(p, g, cr, ci, u1, u2, lane, slow, &bsrc, &adst);
    }
    if (al < 0) {
        if (lane == 0) atomicOr(p.status, kStatusNumeric);
    } else {
        record_jump(p, traj, g, half, al, bsrc, adst, half == 0 ? g * p.dt - p.tau : g * p.dt, lane);
#pragma unroll
        for (int j = 0; j < NPL; ++j) {
            const int a = 32 * j + lane;
            if (a < N) {
                sre[(size_t)a * stride] = cr[j];
                sim[(size_t)a * stride] = ci[j];
            }
        }
    }
    __syncwarp();
}

}  // namespace dev
}  // namespace aqt

namespace aqt {
namespace dev {

// Out-of-line entry for the SIMT kernels (one copy per state type and tile,
// shared by all their instantiations). The clock, threshold and jump count
// live in shared memory; lane 0 writes them back.
template <typename T, int NPL>
static __device__ __noinline__ void jump_half_step_ool(const RunParams &p, int g, int half, int64_t traj, T *sre,
                                                       T *sim, int stride, double *ell, double *logr, int *nj,
                                                       int lane, double2 *slow) {
    double e = *ell, lr = *logr;
    int k = *nj;
    __syncwarp();
    jump_half_step<T, NPL>(p, g, half, traj, sre, sim, stride, e, lr, k, lane, slow);
    if (lane == 0) {
        *ell = e;
        *logr = lr;
        *nj = k;
    }
    __syncwarp();
}

template <typename T, int NPL>
static __device__ __noinline__ void fixed_step_jump_ool(const RunParams &p, int g, int half, int64_t traj, T *sre,
                                                        T *sim, int stride, double u1, double u2, int lane,
                                                        double2 *slow) {
    __syncwarp();
    fixed_step_jump<T, NPL>(p, g, half, traj, sre, sim, stride, u1, u2, lane, slow);
}

template <typename T>
static __device__ __forceinline__ void fixed_step_jump_any(const RunParams &p, int g, int half, int64_t traj, T *sre,
                                                           T *sim, int stride, double u1, double u2, int lane,
                                                           double2 *slow) {
    const int N = p.N;
    if (N <= 32) fixed_step_jump_ool<T, 1>(p, g, half, traj, sre, sim, stride, u1, u2, lane, slow);
    else if (N <= 64) fixed_step_jump_ool<T, 2>(p, g, half, traj, sre, sim, stride, u1, u2, lane, slow);
    else if (N <= 128) fixed_step_jump_ool<T, 4>(p, g, half, traj, sre, sim, stride, u1, u2, lane, slow);
    else if (N <= 256) fixed_step_jump_ool<T, 8>(p, g, half, traj, sre, sim, stride, u1, u2, lane, slow);
    else fixed_step_jump_ool<T, 16>(p, g, half, traj, sre, sim, stride, u1, u2, lane, slow);
}

// Register tile from N for the SIMT kernels (N <= 512).
template <typename T>
static __device__ __forceinline__ void jump_half_step_any(const RunParams &p, int g, int half, int64_t traj, T *sre,
                                                          T *sim, int stride, double *ell, double *logr, int *nj,
                                                          int lane, double2 *slow) {
    const int N = p.N;
    if (N <= 32) jump_half_step_ool<T, 1>(p, g, half, traj, sre, sim, stride, ell, logr, nj, lane, slow);
    else if (N <= 64) jump_half_step_ool<T, 2>(p, g, half, traj, sre, sim, stride, ell, logr, nj, lane, slow);
    else if (N <= 128) jump_half_step_ool<T, 4>(p, g, half, traj, sre, sim, stride, ell, logr, nj, lane, slow);
    else if (N <= 256) jump_half_step_ool<T, 8>(p, g, half, traj, sre, sim, stride, ell, logr, nj, lane, slow);
    else jump_half_step_ool<T, 16>(p, g, half, traj, sre, sim, stride, ell, logr, nj, lane, slow);
}

}  // namespace dev
}  // namespace aqt
