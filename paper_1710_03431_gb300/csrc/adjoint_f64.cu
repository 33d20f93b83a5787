// FP64 instantiation of the backward sweep of gradient runs (adjoint.cuh).
#include "adjoint.cuh"

namespace aqt {

int launch_adjoint_f64(const RunParams &p, const AdjBack &b, void *stream, size_t smem) {
    return adj::launch_back_ra<double>(p, b, (cudaStream_t)stream, smem);
}

int launch_xgemm_f64(const void *seg_c, const void *seg_mu, int64_t M, int N, int K, int g_begin, int n_g,
                     double *xout, void *stream) {
    return adj::launch_xgemm<double>(seg_c, seg_mu, M, N, K, g_begin, n_g, xout, (cudaStream_t)stream);
}

size_t adjoint_smem_bytes_f64(int N, int TT) { return adj::back_smem_bytes(N, TT, sizeof(double)); }

}  // namespace aqt
