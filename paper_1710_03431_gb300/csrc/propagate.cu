// Launch glue of the propagation kernels: tile shapes of the SIMT kernels,
// the observable reductions, and the dispatch by precision. The SIMT kernels
// themselves are in simt_kernel.cuh (instantiated in propagate_f32.cu and
// propagate_f64.cu), the tensor-core kernel in propagate_tc.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "aqt_internal.h"

namespace aqt {

namespace {

constexpr int kThreads = 256;  // threads of a SIMT CTA (simt_kernel.cuh)
constexpr int kWarps = kThreads / 32;
constexpr int kChunkBytes = 32768;

// Sum of the per-tile observable partials ([tile][g][3]) of one instance, in
// tile order (fixed order: the same bits for any launch shape of the same
// tiles).
__device__ __forceinline__ void reduce_one(const RunParams &p, int g) {
    double s = 0.0, s2 = 0.0, sl = 0.0;
    for (int c = 0; c < p.n_cta; ++c) {
        const double *q = p.obs_part + ((size_t)c * p.K + g) * 3;
        s += q[0];
        s2 += q[1];
        sl += q[2];
    }
    p.obs_sum[2 * g] = s;
    p.obs_sum[2 * g + 1] = s2;
    if (p.leak_sum) p.leak_sum[g] = sl;
}

__global__ void reduce_obs(const __grid_constant__ RunParams p) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < p.K) reduce_one(p, g);
}

// The same for every instance of a batch: block y = instance.
__global__ void reduce_obs_batch(const RunParams *ps) {
    const RunParams &p = ps[blockIdx.y];
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < p.K) reduce_one(p, g);
}

}  // namespace

size_t simt_smem_bytes(int N, int TT, int precision) {
    const size_t rs = precision == AQT_PREC_FP64 ? 8 : 4;
    const int LD = TT + 4;
    const int KB = std::min(N, std::max(1, kChunkBytes / (int)(N * rs)));
    size_t b = 0;
    b += 2 * (size_t)N * 8 + 3 * (size_t)TT * 8 + 3 * kWarps * 8;  // d2s, gam, logr, ell, leak, obs
    b += (size_t)((TT + 3) & ~3) * 4;                           // nj
    b += 2 * (size_t)N * LD * rs;                               // cre, cim
    b += (size_t)KB * N * rs;                                   // O chunk
    b += 2 * (size_t)N * rs;                                    // eh
    return b;
}

// Rows of the rotation per thread for a tile of TT trajectories: (TT/4)
// threads share each row group, kThreads / (TT/4) row groups cover N.
int simt_rows_per_thread(int N, int TT) {
    const int tyn = kThreads / (TT / 4);
    return (N + tyn - 1) / tyn;
}

// Pick trajectories per CTA (TT) and GEMM rows per thread (RA) so that
// TT/4 * (256 / (TT/4)) threads cover N rows with RA <= 8 and the grid has
// at least two CTAs per SM when M allows.
void simt_shape(int N, int64_t M, int precision, int num_sms, int *TT, int *RA) {
    const int cands[] = {64, 32, 16, 8, 4};
    int best_tt = 4, best_ra = 8;
    for (int tt : cands) {
        int ra = 1;
        while (ra < simt_rows_per_thread(N, tt)) ra *= 2;
        if (ra > 8) continue;
        if (simt_smem_bytes(N, tt, precision) > kSimtSmemLimit) continue;
        best_tt = tt;
        best_ra = ra;
        if ((M + tt - 1) / tt >= 2LL * num_sms) break;
    }
    *TT = best_tt;
    *RA = best_ra;
}

int launch_run(const RunParams &p, int precision, void *stream, size_t smem) {
    cudaStream_t st = (cudaStream_t)stream;
    int e = precision == AQT_PREC_F16SPLIT ? launch_tc(p, stream, smem)
            : precision == AQT_PREC_FP64   ? launch_simt_f64(p, stream, smem)
                                           : launch_simt_f32(p, stream, smem);
    if (e) return e;
    reduce_obs<<<(p.K + 127) / 128, 128, 0, st>>>(p);
    return (int)cudaGetLastError();
}

int launch_reduce_batch(const RunParams *dev_params, int n_inst, int max_K, void *stream) {
    if (n_inst <= 0) return 0;
    dim3 grid((max_K + 127) / 128, n_inst);
    reduce_obs_batch<<<grid, 128, 0, (cudaStream_t)stream>>>(dev_params);
    return (int)cudaGetLastError();
}

}  // namespace aqt
