// FP64 jump resolution shared by the propagation kernels.
//
// arXiv:1710.03431, Sec. IV and App. C: inside one frozen half-step the
// unnormalised squared norm is sum_a |c_a|^2 exp(2 Im K_aa t) (K diagonal);
// a jump happens when it falls to the threshold r. The warp that owns the
// trajectory finds that time in FP64 (Newton from the left on a convex,
// decreasing function: no overshoot), draws the channel with the
// probabilities of App. B.1 (Eq. Pi(t)), applies the Bohr-class operator
// (Eq. jump), renormalises, draws a new threshold and finishes the half-step,
// possibly jumping again.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "aqt_internal.h"
#include "philox.cuh"

namespace aqt {
namespace dev {

constexpr int kMaxJumpsPerHalf = 64;
enum : int32_t { kStatusNumeric = 2, kStatusTimeout = 4 };

static __device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

static __device__ __forceinline__ double warp_incl_scan(double v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Per-level factors exp(x) and (sin, cos)(x) in the precision TR: double for
// the FP64 path; float for the FP32 and tensor-core paths, whose states are
// FP32 (the sums, the clock and the crossing time stay FP64 either way).
static __device__ __forceinline__ double lvl_exp(double x, double) { return exp(x); }
static __device__ __forceinline__ double lvl_exp(double x, float) { return (double)expf((float)x); }
static __device__ __forceinline__ void lvl_sincos(double x, double *s, double *c, double) { sincos(x, s, c); }
static __device__ __forceinline__ void lvl_sincos(double x, double *s, double *c, float) {
    float sf, cf;
    sincosf((float)x, &sf, &cf);
    *s = sf;
    *c = cf;
}


// Find the first index in [0, N) chosen by inverse CDF over weights wfun(i):
// the first i with prefix_sum(i) > target. Returns -1 if none (rounding).
template <class WF>
static __device__ int warp_pick(int N, double target, int lane, WF wfun) {
    double cum = 0.0;
    int last_pos = -1;
    for (int base = 0; base < N; base += 32) {
        const int i = base + lane;
        const double w = i < N ? wfun(i) : 0.0;
        const double pre = warp_incl_scan(w, lane);
        const double tot = __shfl_sync(0xffffffffu, pre, 31);
        const unsigned pos = __ballot_sync(0xffffffffu, w > 0.0);
        if (pos) last_pos = base + 31 - __clz(pos);
        if (cum + tot > target) {
            const unsigned hit = __ballot_sync(0xffffffffu, i < N && cum + pre > target);
            if (hit) return base + __ffs(hit) - 1;
        }
        cum += tot;
    }
    return last_pos;
}

// Resolve every jump of one trajectory inside one frozen half-step, in FP64.
// c64 holds the normalised state at the start of the half-step; on return it
// holds the normalised state at its end, and ell/logr/nj are updated.
template <typename TR>
static __device__ void resolve_half(const RunParams &p, int g, int half, int64_t traj, double2 *c64, double2 *y64,
                                   double &ell, double &logr, int &nj, int lane) {
    const TR tr{};
    const int N = p.N, n = p.n;
    const double *kd = p.tab.kdiag + (size_t)g * N * 2;
    const double *lvlE = p.tab.lvlE + (size_t)g * N;
    const int32_t *mfirst = p.tab.mfirst + (size_t)g * N;
    const int32_t *msize = p.tab.msize + (size_t)g * N;
    const GridMeta meta = p.tab.meta[g];
    const double *Rg = p.tab.R + (size_t)g * n * N * N;
    const double *Gg = p.tab.G + (size_t)g * n * N;
    const double t_half0 = half == 0 ? g * p.dt - p.tau : g * p.dt;
    double ell0 = ell, tau_rem = p.tau;

    for (int it = 0;; ++it) {
        if (it >= kMaxJumpsPerHalf) {
            if (lane == 0) atomicOr(p.status, kStatusNumeric);
            break;
        }
        // --- crossing time: root of ell0 + log sum |c|^2 e^{2 Im K t} = log r ---
        double t = 0.0;
        for (int k = 0; k < 200; ++k) {
            double s0 = 0.0, s1 = 0.0;
            for (int a = lane; a < N; a += 32) {
                const double im = kd[2 * a + 1];
                const double q = (c64[a].x * c64[a].x + c64[a].y * c64[a].y) * lvl_exp(2.0 * im * t, tr);
                s0 += q;
                s1 += 2.0 * im * q;
            }
            s0 = warp_sum(s0);
            s1 = warp_sum(s1);
            const double F = ell0 + log(s0) - logr;
            if (F <= 0.0 || s1 >= 0.0) break;
            double tn = t - F * s0 / s1;
            if (tn >= tau_rem) tn = tau_rem;
            const bool done = tn - t <= 1e-16 * p.tau;
            t = tn;
            if (done) break;
        }
        // --- propagate to the crossing and renormalise -----------------------
        {
            double s = 0.0;
            for (int a = lane; a < N; a += 32) {
                const double re = kd[2 * a], im = kd[2 * a + 1];
                double sn, cs;
                lvl_sincos(re * t, &sn, &cs, tr);
                const double amp = lvl_exp(im * t, tr);
                const double2 v = c64[a];
                const double2 r = make_double2(amp * (v.x * cs + v.y * sn), amp * (v.y * cs - v.x * sn));
                c64[a] = r;
                s += r.x * r.x + r.y * r.y;
            }
            s = warp_sum(s);
            const double inv = 1.0 / sqrt(s);
            for (int a = lane; a < N; a += 32) {
                c64[a].x *= inv;
                c64[a].y *= inv;
            }
            __syncwarp();
        }
        // --- draw the jump ----------------------------------------------------
        ++nj;
        const Philox4 rnd = traj_event(p.seed, traj, nj);
        const double u1 = uniform01(rnd.x[0]), u2 = uniform01(rnd.x[1]), u3 = uniform01(rnd.x[2]);
        // stage-one weight of unit (alpha, manifold starting at b)
        auto unit_w = [&](int al, int b) -> double {
            if (mfirst[b] != b) return 0.0;
            const int ms = msize[b];
            if (ms == 1) {
                const double2 v = c64[b];
                return (v.x * v.x + v.y * v.y) * Gg[(size_t)al * N + b];
            }
            return -1.0;  // computed by the warp below
        };
        // manifold weight for non-singleton source manifolds (degenerate grids)
        // (the rate depends on manifold energies only, so it sits inside R)
        auto manifold_w = [&](int al, int b) -> double {
            const int ms = msize[b];
            const double *Ra = Rg + (size_t)al * N * N;
            double acc = 0.0;
            for (int a = lane; a < N; a += 32) {
                double yr = 0.0, yi = 0.0;
                for (int bp = b; bp < b + ms; ++bp) {
                    const double m = Ra[(size_t)a * N + bp];
                    yr += m * c64[bp].x;
                    yi += m * c64[bp].y;
                }
                acc += yr * yr + yi * yi;
            }
            return warp_sum(acc);
        };
        // per-alpha totals (identical on all lanes)
        double S[16];
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
        if (al_s < 0) {  // no channel has weight: cannot happen for a decaying norm
            if (lane == 0) atomicOr(p.status, kStatusNumeric);
            break;
        }
        int bsrc;
        if (!meta.degenerate) {
            bsrc = warp_pick(N, target - cum, lane, [&](int b) { return unit_w(al_s, b); });
        } else {
            // sequential walk over manifolds (rare path)
            double c2 = cum;
            bsrc = -1;
            int lastb = -1;
            for (int b = 0; b < N; ++b) {
                if (mfirst[b] != b) continue;
                const double w = msize[b] == 1 ? unit_w(al_s, b) : manifold_w(al_s, b);
                if (w > 0.0) lastb = b;
                if (w > 0.0 && c2 + w > target) {
                    bsrc = b;
                    break;
                }
                c2 += w;
            }
            if (bsrc < 0) bsrc = lastb;
        }
        if (bsrc < 0) {
            if (lane == 0) atomicOr(p.status, kStatusNumeric);
            break;
        }
        // stage two: target level a
        const int ms = msize[bsrc];
        const double *Ra = Rg + (size_t)al_s * N * N;
        auto target_w = [&](int a) -> double {
            if (ms == 1) {
                const double m = Ra[(size_t)a * N + bsrc];
                return m * m;
            }
            double yr = 0.0, yi = 0.0;
            for (int bp = bsrc; bp < bsrc + ms; ++bp) {
                const double m = Ra[(size_t)a * N + bp];
                yr += m * c64[bp].x;
                yi += m * c64[bp].y;
            }
            return yr * yr + yi * yi;
        };
        double tot2 = 0.0;
        for (int a = lane; a < N; a += 32) tot2 += target_w(a);
        tot2 = warp_sum(tot2);
        const int adst = warp_pick(N, u2 * tot2, lane, target_w);
        if (adst < 0) {
            if (lane == 0) atomicOr(p.status, kStatusNumeric);
            break;
        }
        // --- apply the class operator A_{alpha, omega*} (Eq. jump) ---------------
        const double wstar = lvlE[bsrc] - lvlE[adst];
        const double tol = meta.tol;
        double s = 0.0;
        for (int a = lane; a < N; a += 32) {
            const double lo_e = lvlE[a] + wstar - tol, hi_e = lvlE[a] + wstar + tol;
            int lo = 0, hi = N;  // first index with lvlE >= lo_e
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (lvlE[mid] < lo_e) lo = mid + 1; else hi = mid;
            }
            double yr = 0.0, yi = 0.0;
            for (int bp = lo; bp < N && lvlE[bp] <= hi_e; ++bp) {
                const double amp = Ra[(size_t)a * N + bp];
                yr += amp * c64[bp].x;
                yi += amp * c64[bp].y;
            }
            y64[a] = make_double2(yr, yi);
            s += yr * yr + yi * yi;
        }
        s = warp_sum(s);
        __syncwarp();
        const double inv = 1.0 / sqrt(s);
        for (int a = lane; a < N; a += 32) c64[a] = make_double2(y64[a].x * inv, y64[a].y * inv);
        __syncwarp();
        const double t_jump = t_half0 + (p.tau - tau_rem) + t;
        if (lane == 0) {
            const unsigned long long idx = atomicAdd(p.jcount, 1ull);
            if ((int64_t)idx < p.jcap) {
                aqt_jump rec;
                rec.traj = (int32_t)traj;
                rec.grid = g;
                rec.half = half;
                rec.alpha = al_s;
                rec.src = bsrc;
                rec.dst = mfirst[adst];
                rec.t = t_jump;
                rec.omega = wstar;
                p.jumps[idx] = rec;
            }
        }
        logr = log(u3);
        ell0 = 0.0;
        tau_rem -= t;
        // --- rest of the half-step: another crossing? ------------------------------
        double s0 = 0.0;
        for (int a = lane; a < N; a += 32)
            s0 += (c64[a].x * c64[a].x + c64[a].y * c64[a].y) * lvl_exp(2.0 * kd[2 * a + 1] * tau_rem, tr);
        s0 = warp_sum(s0);
        if (tau_rem > 0.0 && log(s0) - logr <= 0.0) continue;
        break;
    }
    // finish the half-step without further jumps
    double s0 = 0.0;
    for (int a = lane; a < N; a += 32) {
        const double re = kd[2 * a], im = kd[2 * a + 1];
        double sn, cs;
        lvl_sincos(re * tau_rem, &sn, &cs, tr);
        const double amp = lvl_exp(im * tau_rem, tr);
        const double2 v = c64[a];
        const double2 r = make_double2(amp * (v.x * cs + v.y * sn), amp * (v.y * cs - v.x * sn));
        c64[a] = r;
        s0 += r.x * r.x + r.y * r.y;
    }
    s0 = warp_sum(s0);
    ell = ell0 + log(s0);
    const double inv = 1.0 / sqrt(s0);
    for (int a = lane; a < N; a += 32) {
        c64[a].x *= inv;
        c64[a].y *= inv;
    }
    __syncwarp();
}

// One frozen half-step in FP64 for a trajectory held in c64 (normalised):
// propagate exactly when the threshold is not reached, resolve jumps when it is.
template <typename TR>
static __device__ void half_step64(const RunParams &p, int g, int half, int64_t traj, double2 *c64, double2 *y64,
                                   double &ell, double &logr, int &nj, int lane) {
    const int N = p.N;
    const double *d2 = p.tab.d2 + (size_t)g * N;
    double f = 0.0;
    for (int a = lane; a < N; a += 32) f += (c64[a].x * c64[a].x + c64[a].y * c64[a].y) * d2[a];
    f = warp_sum(f);
    if (ell + log(f) > logr) {
        const double *eh = p.tab.ehalf + (size_t)g * N * 2;
        const double inv = 1.0 / sqrt(f);
        for (int a = lane; a < N; a += 32) {
            const double2 v = c64[a];
            const double er = eh[2 * a], ei = eh[2 * a + 1];
            c64[a] = make_double2((v.x * er - v.y * ei) * inv, (v.x * ei + v.y * er) * inv);
        }
        ell += log(f);
        __syncwarp();
        return;
    }
    resolve_half<TR>(p, g, half, traj, c64, y64, ell, logr, nj, lane);
}

}  // namespace dev
}  // namespace aqt
