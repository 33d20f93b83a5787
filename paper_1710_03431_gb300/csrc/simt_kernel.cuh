// SIMT propagation of AME quantum-jump trajectories (FP64 or FP32 state).
//
// arXiv:1710.03431, Sec. IV: each trajectory carries its normalised
// eigenframe coefficients c (psi = V_g c), the log of the unnormalised
// squared norm accumulated since its last jump (ell) and the log of its
// threshold r. Per grid step g-1 -> g:
//   c <- O_{g-1} c                      frame change, O = V_g^T V_{g-1} (rotation GEMM)
//   half-step frozen at s_g:            c_a <- c_a exp(-i K_aa tau), ell += log ||c||^2
//   observe the ground-manifold population at s_g
//   half-step frozen at s_g (first half of the next interval)
// with K the diagonal eigenframe H_eff (Sec. III, Eq. Heff). When ell falls to
// log r inside a half-step (Sec. IV; App. C), the warp that owns the
// trajectory finds the crossing time, draws the jump (App. B.1, Eq. Pi(t)),
// applies it (Eq. jump), draws a new threshold and finishes the half-step,
// possibly jumping again (device_jump.cuh).
//
// Layout: one CTA owns a tile of TT trajectories of one instance for the
// whole run; their states stay in shared memory as planar real/imaginary
// [level][trajectory] tiles. The frame rotation streams O^T from the tables in
// chunks of KB rows. Each warp owns whole trajectories in the per-step
// epilogue (norms by warp shuffles).
//
// Two kernels run the same tile body (simt_tile): propagate_simt, one CTA per
// tile of one instance, and propagate_simt_batch, a persistent kernel whose
// CTAs take (instance, tile) work items of many instances from a queue.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "aqt_internal.h"
#include "device_jump.cuh"
#include "philox.cuh"

namespace aqt {
namespace simt {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kChunkBytes = 32768;

using namespace dev;

struct Scalars {
    double *logr, *ell;
    int *nj;
};

template <typename R>
struct Vec4;
template <>
struct Vec4<float> {
    static __device__ __forceinline__ void load(const float *p, float v[4]) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
};
template <>
struct Vec4<double> {
    static __device__ __forceinline__ void load(const double *p, double v[4]) {
        const double2 q0 = *reinterpret_cast<const double2 *>(p);
        const double2 q1 = *reinterpret_cast<const double2 *>(p + 2);
        v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
    }
};

template <typename R>
__device__ __forceinline__ const R *ehalf_table(const RunParams &p);
template <>
__device__ __forceinline__ const float *ehalf_table<float>(const RunParams &p) { return p.tab.ehalf32; }
template <>
__device__ __forceinline__ const double *ehalf_table<double>(const RunParams &p) { return p.tab.ehalf; }

// One trajectory's renormalisation, frozen half-step and crossing check. The
// state is normalised before each rotation, so after it (half = 0) nu - 1 is
// the rotation's own relative norm error, kept in *nerr.
template <typename R>
__device__ void half_step(const RunParams &p, int g, int half, int t, int64_t traj, R *cre, R *cim, int LD,
                          const R *eh, const double *d2s, const double *gam, Scalars sc, double2 *c64, int lane,
                          float *nerr, double *leak) {
    const int N = p.N;
    double nu = 0.0, f = 0.0;
    for (int a = lane; a < N; a += 32) {
        const double re = cre[a * LD + t], im = cim[a * LD + t];
        const double q = re * re + im * im;
        nu += q;
        f += q * d2s[a];
    }
    nu = warp_sum(nu);
    f = warp_sum(f);
    if (!(nu > 0.0) || !isfinite(nu)) {
        if (lane == 0) atomicOr(p.status, kStatusNumeric);
        return;
    }
    if (half == 0 && g > 0) {
        *nerr = fmaxf(*nerr, (float)fabs(nu - 1.0));
        if (lane == 0) leak[t] = 1.0 - nu;  // the rotation's norm loss (leakage when truncated)
    }
    if (p.timing == kTimingFixed) {
        // App. B.1: jump with probability tau lambda, lambda = sum_b |c_b|^2 Gamma_b / nu
        double lam = 0.0;
        for (int a = lane; a < N; a += 32) {
            const double re = cre[a * LD + t], im = cim[a * LD + t];
            lam += (re * re + im * im) * gam[a];
        }
        lam = warp_sum(lam) / nu;
        const Philox4 rnd = piece_draws(p.seed, traj, 2 * (int64_t)g + half - 1);
        if (p.tau * lam > uniform01(rnd.x[0])) {
            fixed_step_jump_any<R>(p, g, half, traj, cre + t, cim + t, LD, uniform01(rnd.x[1]), uniform01(rnd.x[2]),
                                   lane, c64);
            return;
        }
        const R scale = (R)(1.0 / sqrt(f));
        for (int a = lane; a < N; a += 32) {
            const R re = cre[a * LD + t], im = cim[a * LD + t];
            const R er = eh[2 * a], ei = eh[2 * a + 1];
            cre[a * LD + t] = (re * er - im * ei) * scale;
            cim[a * LD + t] = (re * ei + im * er) * scale;
        }
        __syncwarp();
        return;
    }
    f /= nu;
    const double ell = sc.ell[t], logr = sc.logr[t];
    const double ell_new = ell + log(f);
    if (ell_new > logr) {
        const R scale = (R)(1.0 / sqrt(f * nu));
        for (int a = lane; a < N; a += 32) {
            const R re = cre[a * LD + t], im = cim[a * LD + t];
            const R er = eh[2 * a], ei = eh[2 * a + 1];
            cre[a * LD + t] = (re * er - im * ei) * scale;
            cim[a * LD + t] = (re * ei + im * er) * scale;
        }
        if (lane == 0) sc.ell[t] = ell_new;
        __syncwarp();
        return;
    }
    // crossing inside this half-step: the warp resolves it with the state in registers
    jump_half_step_any<R>(p, g, half, traj, cre + t, cim + t, LD, &sc.ell[t], &sc.logr[t], &sc.nj[t], lane, c64);
}

// The whole run of tile `cta` of one instance (trajectories cta*TT ..
// cta*TT + TT - 1): states in shared memory (smem, simt_smem_bytes(N, TT)),
// jump scratch at scr (kScratchSlots x kSlotDouble2 x N double2, one slot per
// warp), observable partials at p.obs_part[cta][g][3]. RA: rows of the rotation
// per thread; RA x (kThreads / (TT/4)) >= N.
template <typename R, int RA>
__device__ __forceinline__ void simt_tile(const RunParams &p, int cta, double2 *scr, unsigned char *smem) {
    const int N = p.N, K = p.K, TT = p.TT;
    const int LD = TT + 4;
    const int TXN = TT / 4, TYN = kThreads / TXN;
    const int KB = min(N, max(1, kChunkBytes / (int)(N * sizeof(R))));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // shared-memory carve (all offsets multiples of 16 bytes)
    double *d2s = reinterpret_cast<double *>(smem);
    double *gam = d2s + N;  // -2 Im K_aa: the level's total jump rate
    double *logr = gam + N;
    double *ell = logr + TT;
    double *obs = ell + TT;                         // [kWarps][3]
    double *leak = obs + 3 * kWarps;                // [TT] this step's norm loss of the rotation
    int *nj = reinterpret_cast<int *>(leak + TT);
    R *cre = reinterpret_cast<R *>(nj + ((TT + 3) & ~3));
    R *cim = cre + (size_t)N * LD;
    R *osm = cim + (size_t)N * LD;
    R *eh = osm + (size_t)KB * N;
    Scalars sc{logr, ell, nj};

    const int64_t t0 = (int64_t)cta * TT;
    static_assert(kWarps <= kScratchSlots, "one jump scratch slot per warp");
    double2 *c64 = scr + (size_t)warp * kSlotDouble2 * N;

    // Gradient runs: a segment recompute (seg) restarts from a checkpoint and
    // runs grid points g_begin .. g_end only; a checkpointed forward run (ckpt)
    // writes the checkpoints on the way.
    const AdjParams &adj = p.adj;
    const bool seg = adj.seg_c != nullptr;
    const bool ckpt = !seg && adj.ckpt != nullptr;
    const int g_begin = seg ? adj.g_begin : 0, g_end = seg ? adj.g_end : K - 1;
    if (seg && g_begin > 0) {
        // restart from checkpoint g_begin / ckpt_every: the state at the end of grid point g_begin - 1
        const size_t j = (size_t)(g_begin / adj.ckpt_every - 1);
        const R *cs = reinterpret_cast<const R *>(adj.ckpt);
        for (int i = tid; i < N * LD; i += kThreads) {
            const int t = i / N, a = i % N;
            if (t >= LD) continue;
            const bool v = t < TT && t0 + t < p.M;
            const size_t o = ((j * p.M + t0 + t) * N + a) * 2;
            cre[a * LD + t] = v ? cs[o] : (R)0;
            cim[a * LD + t] = v ? cs[o + 1] : (R)0;
        }
        for (int t = tid; t < TT; t += kThreads) {
            const bool v = t0 + t < p.M;
            const size_t o = j * p.M + t0 + t;
            ell[t] = v ? adj.ckpt_clock[2 * o] : 0.0;
            logr[t] = v ? adj.ckpt_clock[2 * o + 1] : 0.0;
            nj[t] = v ? adj.ckpt_nj[o] : 0;
            leak[t] = 0.0;
        }
    } else {
        // initial state: ground state of H_S(0) (level 0), threshold from event 0
        for (int i = tid; i < N * LD; i += kThreads) {
            const int a = i / LD, t = i % LD;
            cre[i] = (a == 0 && t < TT && t0 + t < p.M) ? (R)1 : (R)0;
            cim[i] = (R)0;
        }
        for (int t = tid; t < TT; t += kThreads) {
            ell[t] = 0.0;
            leak[t] = 0.0;
            nj[t] = 0;
            logr[t] = (t0 + t < p.M) ? log(uniform01(traj_event(p.seed, t0 + t, 0).x[0])) : 0.0;
        }
    }
    // segment recompute: normalised state of every trajectory at the start (e = 0)
    // or end (e = 1) of grid point g's frozen span, and the rotated state's norm
    auto seg_store = [&](int g, int e, bool normalise) {
        R *dst = reinterpret_cast<R *>(adj.seg_c) + (size_t)((g - g_begin) * 2 + e) * p.M * N * 2;
        for (int t = warp; t < TT; t += kWarps) {
            if (t0 + t >= p.M) continue;
            R sc = (R)1;
            if (normalise) {
                R nu = (R)0;
                for (int a = lane; a < N; a += 32) {
                    const R re = cre[a * LD + t], im = cim[a * LD + t];
                    nu += re * re + im * im;
                }
                nu = warp_sum(nu);
                sc = (R)1 / sqrt(nu);
                if (lane == 0) adj.seg_nrot[(size_t)(g - g_begin) * p.M + t0 + t] = (double)sqrt(nu);
            }
            R *q = dst + (size_t)(t0 + t) * N * 2;
            for (int a = lane; a < N; a += 32) {
                q[2 * a] = cre[a * LD + t] * sc;
                q[2 * a + 1] = cim[a * LD + t] * sc;
            }
        }
    };
    auto ckpt_store = [&](int g) {
        const size_t j = (size_t)((g + 1) / adj.ckpt_every - 1);
        R *cs = reinterpret_cast<R *>(adj.ckpt);
        for (int t = warp; t < TT; t += kWarps) {
            if (t0 + t >= p.M) continue;
            R *q = cs + ((j * p.M + t0 + t) * N) * 2;
            for (int a = lane; a < N; a += 32) {
                q[2 * a] = cre[a * LD + t];
                q[2 * a + 1] = cim[a * LD + t];
            }
            if (lane == 0) {
                const size_t o = j * p.M + t0 + t;
                adj.ckpt_clock[2 * o] = ell[t];
                adj.ckpt_clock[2 * o + 1] = logr[t];
                adj.ckpt_nj[o] = nj[t];
            }
        }
    };
    const R *eh_tab = ehalf_table<R>(p);
    auto load_grid = [&](int g) {
        for (int a = tid; a < N; a += kThreads) {
            d2s[a] = p.tab.d2[(size_t)g * N + a];
            gam[a] = -2.0 * p.tab.kdiag[((size_t)g * N + a) * 2 + 1];
            eh[2 * a] = eh_tab[((size_t)g * N + a) * 2];
            eh[2 * a + 1] = eh_tab[((size_t)g * N + a) * 2 + 1];
        }
    };
    const int gs0 = p.tab.meta[0].gs_size;
    auto observe = [&](int g, int gs) {
        double wx = 0.0, wx2 = 0.0, wl = 0.0;
        for (int t = warp; t < TT; t += kWarps) {
            if (t0 + t >= p.M) continue;
            double x = 0.0;
            for (int a = lane; a < gs; a += 32) {
                const double re = cre[a * LD + t], im = cim[a * LD + t];
                x += re * re + im * im;
            }
            x = warp_sum(x);
            wx += x;
            wx2 += x * x;
            wl += leak[t];
        }
        if (lane == 0) {
            obs[3 * warp] = wx;
            obs[3 * warp + 1] = wx2;
            obs[3 * warp + 2] = wl;
        }
        __syncthreads();
        if (tid == 0) {
            double s = 0.0, s2 = 0.0, sl = 0.0;
            for (int w = 0; w < kWarps; ++w) {
                s += obs[3 * w];
                s2 += obs[3 * w + 1];
                sl += obs[3 * w + 2];
            }
            double *q = p.obs_part + ((size_t)cta * K + g) * 3;
            q[0] = s;
            q[1] = s2;
            q[2] = sl;
        }
    };
    float nerr = 0.0f;
    auto half_all = [&](int g, int half) {
        for (int t = warp; t < TT; t += kWarps) {
            if (t0 + t >= p.M) continue;
            half_step<R>(p, g, half, t, t0 + t, cre, cim, LD, eh, d2s, gam, sc, c64, lane, &nerr, leak);
        }
    };

    if (g_begin == 0) {
        load_grid(0);
        __syncthreads();
        if (!seg) observe(0, gs0);
        half_all(0, 1);
        if (seg) {
            __syncthreads();
            seg_store(0, 1, false);
        }
        if (ckpt && adj.ckpt_every == 1 && K > 1) {
            __syncthreads();
            ckpt_store(0);
        }
    }

    const int tx = tid % TXN, ty = tid / TXN;
    for (int g = max(g_begin, 1); g <= g_end; ++g) {
        // ---- rotation c <- O_{g-1} c ---------------------------------------------
        R accr[RA][4], acci[RA][4];
#pragma unroll
        for (int i = 0; i < RA; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) accr[i][j] = acci[i][j] = (R)0;
        const R *OT = reinterpret_cast<const R *>(p.tab.OT) + (size_t)(g - 1) * N * N;
        for (int b0 = 0; b0 < N; b0 += KB) {
            __syncthreads();
            for (int i = tid; i < KB * N; i += kThreads) osm[i] = OT[(size_t)b0 * N + i];
            __syncthreads();
            for (int bb = 0; bb < KB; ++bb) {
                R vr[4], vi[4];
                Vec4<R>::load(&cre[(b0 + bb) * LD + 4 * tx], vr);
                Vec4<R>::load(&cim[(b0 + bb) * LD + 4 * tx], vi);
#pragma unroll
                for (int i = 0; i < RA; ++i) {
                    const int a = ty + i * TYN;
                    const R o = a < N ? osm[bb * N + a] : (R)0;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        accr[i][j] = fma(o, vr[j], accr[i][j]);
                        acci[i][j] = fma(o, vi[j], acci[i][j]);
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < RA; ++i) {
            const int a = ty + i * TYN;
            if (a < N) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    cre[a * LD + 4 * tx + j] = accr[i][j];
                    cim[a * LD + 4 * tx + j] = acci[i][j];
                }
            }
        }
        load_grid(g);
        __syncthreads();
        if (seg) {
            seg_store(g, 0, true);
            __syncthreads();
        }
        // ---- epilogue: half-step into s_g, observe, half-step out of s_g ------------
        half_all(g, 0);
        __syncthreads();
        if (!seg) observe(g, p.tab.meta[g].gs_size);
        if (g < K - 1) half_all(g, 1);
        if (seg) {
            __syncthreads();
            seg_store(g, 1, false);
        } else if (ckpt && g < K - 1 && (g + 1) % adj.ckpt_every == 0) {
            __syncthreads();
            ckpt_store(g);
        }
    }
    if (seg) return;
    if (p.norm_err && lane == 0) atomicMax(p.norm_err, __float_as_uint(nerr));
    __syncthreads();
    for (int i = tid; i < N * TT; i += kThreads) {
        const int t = i / N, a = i % N;
        if (t0 + t < p.M) {
            p.final_state[((size_t)(t0 + t) * N + a) * 2] = (double)cre[a * LD + t];
            p.final_state[((size_t)(t0 + t) * N + a) * 2 + 1] = (double)cim[a * LD + t];
        }
    }
}

// One CTA per tile of one instance.
template <typename R, int RA>
__global__ void __launch_bounds__(kThreads, 2) propagate_simt(const __grid_constant__ RunParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    double2 *scr = reinterpret_cast<double2 *>(p.scratch) + (size_t)blockIdx.x * kScratchSlots * kSlotDouble2 * p.N;
    simt_tile<R, RA>(p, blockIdx.x, scr, smem);
}

// Persistent kernel over the work items of many instances: each CTA takes the
// next item from the queue (items are ordered by decreasing cost, so the
// longest tiles start first) until none is left. ps[i]: run parameters of
// instance i (TT per instance, RA common); scratch: one jump-scratch block of
// scr_stride double2 per CTA of this launch. The queue counter starts at 0.
template <typename R, int RA>
__global__ void __launch_bounds__(kThreads, 2)
    propagate_simt_batch(const RunParams *ps, const BatchItem *items, int n_items, int *queue, double2 *scratch,
                         size_t scr_stride) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ RunParams sp;
    __shared__ int s_item;
    double2 *scr = scratch + (size_t)blockIdx.x * scr_stride;
    for (;;) {
        __syncthreads();  // the previous item is done with the shared memory
        if (threadIdx.x == 0) {
            s_item = atomicAdd(queue, 1);
            if (s_item < n_items) sp = ps[items[s_item].inst];
        }
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        simt_tile<R, RA>(sp, items[it].cta, scr, smem);
    }
}

template <typename R, int RA>
int launch_simt(const RunParams &p, cudaStream_t st, size_t smem) {
    auto kern = propagate_simt<R, RA>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    kern<<<p.n_cta, kThreads, smem, st>>>(p);
    return (int)cudaGetLastError();
}

template <typename R>
int launch_simt_ra(const RunParams &p, cudaStream_t st, size_t smem) {
    switch (p.RA) {
        case 1: return launch_simt<R, 1>(p, st, smem);
        case 2: return launch_simt<R, 2>(p, st, smem);
        case 4: return launch_simt<R, 4>(p, st, smem);
        case 8: return launch_simt<R, 8>(p, st, smem);
        default: return (int)cudaErrorInvalidValue;
    }
}

template <typename R, int RA>
int launch_batch(const BatchLaunch &b, cudaStream_t st) {
    auto kern = propagate_simt_batch<R, RA>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b.smem);
    if (e != cudaSuccess) return (int)e;
    if (b.prepare_only) return 0;
    kern<<<b.n_cta, kThreads, b.smem, st>>>(b.params, b.items, b.n_items, b.queue,
                                                reinterpret_cast<double2 *>(b.scratch), b.scr_stride);
    return (int)cudaGetLastError();
}

template <typename R>
int launch_batch_ra(const BatchLaunch &b, cudaStream_t st) {
    switch (b.RA) {
        case 2: return launch_batch<R, 2>(b, st);
        case 4: return launch_batch<R, 4>(b, st);
        case 8: return launch_batch<R, 8>(b, st);
        default: return (int)cudaErrorInvalidValue;
    }
}

// Resident CTAs per SM of the persistent kernel with `smem` bytes of dynamic
// shared memory (0 if it cannot run).
template <typename R, int RA>
int batch_occupancy(size_t smem) {
    auto kern = propagate_simt_batch<R, RA>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kThreads, smem) != cudaSuccess) return 0;
    return nb;
}

template <typename R>
int batch_occupancy_ra(int RA, size_t smem) {
    switch (RA) {
        case 2: return batch_occupancy<R, 2>(smem);
        case 4: return batch_occupancy<R, 4>(smem);
        case 8: return batch_occupancy<R, 8>(smem);
        default: return 0;
    }
}

}  // namespace simt
}  // namespace aqt
