// Jump resolution shared by the propagation kernels.
//
// arXiv:1710.03431, Sec. IV and App. C: inside one frozen half-step the
// squared norm of the normalised state evolves as
//   |c(t)|^2 = 1 + delta(t),   delta(t) = sum_a |c_a|^2 expm1(2 Im K_aa t)
// (K diagonal), and a jump happens when the clock ell + log1p(delta(t)) falls
// to the threshold log r. The warp that owns the trajectory holds its state in
// registers (level a = 32 j + lane in slot j), finds the crossing time by
// Newton's method from the left (the function is convex and decreasing, so
// the iterates never overshoot), draws the channel with the probabilities of
// App. B.1 (Eq. Pi(t)), applies the Bohr-class operator (Eq. jump),
// renormalises, draws a new threshold and finishes the half-step, possibly
// jumping again.
//
// The clock is FP64. The per-level arithmetic runs in the state's precision T
// (double for the FP64 path; float for the FP32 and tensor-core paths, whose
// states are FP32); writing the norm decay as expm1 terms keeps its relative
// accuracy however small it is.
//
// Fast path (every manifold a single level and every Bohr class of nonzero
// frequency a single level pair, the generic case once s > 0): the class
// operator maps the source level to the target level alone, or, at zero
// frequency, scales each level by its diagonal amplitude. Otherwise the state
// goes to per-warp scratch and a general FP64 routine draws and applies the
// jump over degenerate manifolds and multi-pair classes.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "aqt_internal.h"
#include "philox.cuh"

namespace aqt {
namespace dev {

constexpr int kMaxJumpsPerHalf = 64;
constexpr int kMaxAlpha = 10;
enum : int32_t { kStatusNumeric = 2, kStatusTimeout = 4 };

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

// Newton stops once a step is this small relative to t: the error left after
// it is of the order of its square.
template <typename T>
static __device__ __forceinline__ T newton_rel();
template <>
__device__ __forceinline__ float newton_rel<float>() { return 1e-3f; }
template <>
__device__ __forceinline__ double newton_rel<double>() { return 1e-7; }

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
template <typename RT>
static __device__ int general_draw_apply(const RunParams &p, int g, double u1, double u2, double2 *c64, double2 *y64,
                                         int lane, int *bsrc_out, int *adst_out) {
    const int N = p.N, n = p.n;
    const double *lvlE = p.tab.lvlE + (size_t)g * N;
    const int32_t *mfirst = p.tab.mfirst + (size_t)g * N;
    const int32_t *msize = p.tab.msize + (size_t)g * N;
    const GridMeta meta = p.tab.meta[g];
    const RT *Rg = static_cast<const RT *>(p.tab.Rt) + (size_t)g * n * N * N;  // [alpha][b][a]
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

// One frozen half-step of one trajectory that may cross its threshold,
// resolved by one warp with the state in registers (NPL levels per lane,
// 32 NPL >= N). sre/sim: the state, level a at [a * stride] (normalised or
// not); on return, the normalised state at the end of the half-step. ell,
// logr, nj: the trajectory's clock, log threshold and jump count (the same on
// every lane). slow: 2N double2 of per-warp scratch for the general jump.
// klev (FP32 paths, optional): (Re K_aa, 2 Im K_aa) of grid point g staged in
// shared memory; otherwise the FP64 table is read.
template <typename T, int NPL>
static __device__ __forceinline__ void jump_half_step(const RunParams &p, int g, int half, int64_t traj, T *sre,
                                                      T *sim, int stride, double &ell, double &logr, int &nj,
                                                      int lane, double2 *slow, const float2 *klev = nullptr) {
    const int N = p.N, n = p.n;
    const GridMeta meta = p.tab.meta[g];
    const double *kd = p.tab.kdiag + (size_t)g * N * 2;
    const double *Gg = p.tab.G + (size_t)g * n * N;
    const T *Rg = static_cast<const T *>(p.tab.Rt) + (size_t)g * n * N * N;  // [alpha][b][a]
    const bool fast = meta.simple && !meta.degenerate;
    T cr[NPL], ci[NPL];
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
        const int a = 32 * j + lane;
        const bool v = a < N;
        cr[j] = v ? sre[(size_t)a * stride] : T(0);
        ci[j] = v ? sim[(size_t)a * stride] : T(0);
    }
    // diagonal of K per level (re, 2 im), re-read from the cache where used to
    // keep registers free
    auto kre = [&](int j) -> T {
        const int a = 32 * j + lane;
        if constexpr (std::is_same<T, float>::value)
            if (klev) return a < N ? klev[a].x : 0.0f;
        return a < N ? (T)kd[2 * a] : T(0);
    };
    auto kim2 = [&](int j) -> T {
        const int a = 32 * j + lane;
        if constexpr (std::is_same<T, float>::value)
            if (klev) return a < N ? klev[a].y : 0.0f;
        return a < N ? (T)(2.0 * kd[2 * a + 1]) : T(0);
    };
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
    // delta(t) of the normalised state and its derivative
    auto decay = [&](T t, T *d1) -> T {
        T d = T(0), e1 = T(0);
#pragma unroll
        for (int j = 0; j < NPL; ++j) {
            const T q = cr[j] * cr[j] + ci[j] * ci[j];
            const T x = kim2(j);
            const T e = m_expm1(x * t);
            d += q * e;
            e1 += q * x * (e + T(1));
        }
        warp_sum2(d, e1);
        *d1 = e1;
        return d;
    };
    bool ok = advance(T(0));
    double ell0 = ell;
    double tau_rem = p.tau;
    const double t_half0 = half == 0 ? g * p.dt - p.tau : g * p.dt;
    T dend = T(0);
    for (int it = 0; ok; ++it) {
        T dd;
        dend = decay((T)tau_rem, &dd);
        const double C = ell0 - logr;  // > 0 until the threshold is reached
        if (C + (double)m_log1p(dend) > 0.0) break;
        if (it >= kMaxJumpsPerHalf) {
            ok = false;
            break;
        }
        // --- crossing time: Newton from the left on C + log1p(delta(t)) ------------
        const T Ct = (T)C;
        T t = T(0);
        for (int k = 0; k < 40; ++k) {
            T d1;
            const T d = decay(t, &d1);
            const T phi = Ct + m_log1p(d);
            if (!(phi > T(0)) || !(d1 < T(0))) break;
            const T step = -phi * (T(1) + d) / d1;
            T tn = t + step;
            if (tn > (T)tau_rem) tn = (T)tau_rem;
            if (!(tn > t)) break;
            t = tn;
            if (step <= newton_rel<T>() * t) break;
        }
        if (!advance(t)) {
            ok = false;
            break;
        }
        // --- draw and apply the jump --------------------------------------------------
        ++nj;
        const Philox4 rnd = traj_event(p.seed, traj, nj);
        const double u1 = uniform01(rnd.x[0]), u2 = uniform01(rnd.x[1]), u3 = uniform01(rnd.x[2]);
        int al = -1, bsrc = -1, adst = -1;
        if (fast) {
            T qv[NPL];
#pragma unroll
            for (int j = 0; j < NPL; ++j) qv[j] = cr[j] * cr[j] + ci[j] * ci[j];
            // stage one over units (alpha, b) in that order
            T total = T(0);
            T cum = T(0), cum_last = T(0);
            int last = -1;
            if constexpr (std::is_same<T, float>::value) {
                // all per-alpha totals in one pass over the level-major FP32 rates
                // (8 alphas per level, two float4)
                const float4 *gt = reinterpret_cast<const float4 *>(p.tab.Gt32) + (size_t)g * N * 2;
                float S8[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) S8[k] = 0.0f;
#pragma unroll
                for (int j = 0; j < NPL; ++j) {
                    const int b = 32 * j + lane;
                    if (b < N) {
                        const float4 x = gt[2 * b], y = gt[2 * b + 1];
                        S8[0] = fmaf(qv[j], x.x, S8[0]);
                        S8[1] = fmaf(qv[j], x.y, S8[1]);
                        S8[2] = fmaf(qv[j], x.z, S8[2]);
                        S8[3] = fmaf(qv[j], x.w, S8[3]);
                        S8[4] = fmaf(qv[j], y.x, S8[4]);
                        S8[5] = fmaf(qv[j], y.y, S8[5]);
                        S8[6] = fmaf(qv[j], y.z, S8[6]);
                        S8[7] = fmaf(qv[j], y.w, S8[7]);
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                    for (int k = 0; k < 8; ++k) S8[k] += __shfl_xor_sync(0xffffffffu, S8[k], o);
#pragma unroll
                for (int k = 0; k < 8; ++k) total += S8[k];
                const T target = (T)u1 * total;
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    if (al < 0 && k < n) {
                        if (S8[k] > 0.0f) {
                            last = k;
                            cum_last = cum;
                        }
                        if (S8[k] > 0.0f && cum + S8[k] > target) al = k;
                        else cum += S8[k];
                    }
            } else {
                // The total rate is sum_b |c_b|^2 sum_alpha G_alpha[b] = -sum_b |c_b|^2
                // 2 Im K_bb, so the walk over alpha stops at the first alpha whose
                // cumulative sum passes the target, one warp sum per alpha visited.
#pragma unroll
                for (int j = 0; j < NPL; ++j) total -= qv[j] * kim2(j);
                total = warp_sum(total);
                const T target = (T)u1 * total;
                for (int a_ = 0; a_ < n && al < 0; ++a_) {
                    T acc = T(0);
#pragma unroll
                    for (int j = 0; j < NPL; ++j) {
                        const int b = 32 * j + lane;
                        if (b < N) acc += qv[j] * (T)Gg[(size_t)a_ * N + b];
                    }
                    acc = warp_sum(acc);
                    if (acc > T(0)) {
                        last = a_;
                        cum_last = cum;
                    }
                    if (acc > T(0) && cum + acc > target) al = a_;
                    else cum += acc;
                }
            }
            const T target = (T)u1 * total;
            if (al < 0) {  // rounding at the top of the distribution
                al = last;
                cum = cum_last;
            }
            if (al >= 0) {
                T w[NPL];
#pragma unroll
                for (int j = 0; j < NPL; ++j) {
                    const int b = 32 * j + lane;
                    if constexpr (std::is_same<T, float>::value)
                        w[j] = b < N ? qv[j] * p.tab.Gt32[((size_t)g * N + b) * 8 + al] : 0.0f;  // cached by stage one
                    else
                        w[j] = b < N ? qv[j] * (T)Gg[(size_t)al * N + b] : T(0);
                }
                bsrc = reg_pick(w, target - cum, lane);
            }
            if (bsrc >= 0) {
                // stage two: target a with weight R_alpha[a][bsrc]^2 (source row of Rt)
                const T *row = Rg + ((size_t)al * N + bsrc) * N;
                T r[NPL], w[NPL], tot2 = T(0);
#pragma unroll
                for (int j = 0; j < NPL; ++j) {
                    const int a = 32 * j + lane;
                    r[j] = a < N ? row[a] : T(0);
                    w[j] = r[j] * r[j];
                    tot2 += w[j];
                }
                tot2 = warp_sum(tot2);
                adst = reg_pick(w, (T)u2 * tot2, lane);
                if (adst >= 0 && adst != bsrc) {
                    // nonzero frequency: the class is the single pair (adst <- bsrc), so
                    // the normalised result is sign(R[adst][bsrc]) c_bsrc / |c_bsrc| on adst
                    const T br = __shfl_sync(0xffffffffu, reg_at(cr, bsrc >> 5), bsrc & 31);
                    const T bi = __shfl_sync(0xffffffffu, reg_at(ci, bsrc >> 5), bsrc & 31);
                    const T ra = __shfl_sync(0xffffffffu, reg_at(r, adst >> 5), adst & 31);
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
                    // zero frequency: every level pairs with itself, y_a = R_alpha[a][a] c_a
                    const T *Ra = Rg + (size_t)al * N * N;
                    T s = T(0);
#pragma unroll
                    for (int j = 0; j < NPL; ++j) {
                        const int a = 32 * j + lane;
                        const T d = a < N ? Ra[(size_t)a * N + a] : T(0);
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
            al = general_draw_apply<T>(p, g, u1, u2, slow, slow + N, lane, &bsrc, &adst);
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
        if (al < 0) {
            ok = false;
            break;
        }
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
                rec.t = t_half0 + (p.tau - tau_rem) + (double)t;
                rec.omega = lvlE[bsrc] - lvlE[adst];
                p.jumps[idx] = rec;
            }
        }
        __syncwarp();
        logr = log(u3);
        ell0 = 0.0;
        tau_rem -= (double)t;
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
    ell = ell0 + (double)m_log1p(dend);
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

// Register tile from N for the SIMT kernels (N <= 256).
template <typename T>
static __device__ __forceinline__ void jump_half_step_any(const RunParams &p, int g, int half, int64_t traj, T *sre,
                                                          T *sim, int stride, double *ell, double *logr, int *nj,
                                                          int lane, double2 *slow) {
    const int N = p.N;
    if (N <= 32) jump_half_step_ool<T, 1>(p, g, half, traj, sre, sim, stride, ell, logr, nj, lane, slow);
    else if (N <= 64) jump_half_step_ool<T, 2>(p, g, half, traj, sre, sim, stride, ell, logr, nj, lane, slow);
    else if (N <= 128) jump_half_step_ool<T, 4>(p, g, half, traj, sre, sim, stride, ell, logr, nj, lane, slow);
    else jump_half_step_ool<T, 8>(p, g, half, traj, sre, sim, stride, ell, logr, nj, lane, slow);
}

}  // namespace dev
}  // namespace aqt
