// SIMT propagation kernel with a float state, one CTA per tile of one
// instance; the tile body is in simt_kernel.cuh.
#include "simt_kernel.cuh"

namespace aqt {

int launch_simt_f32(const RunParams &p, void *stream, size_t smem) {
    return simt::launch_simt_ra<float>(p, (cudaStream_t)stream, smem);
}

}  // namespace aqt
