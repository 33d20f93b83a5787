// Persistent multi-instance SIMT propagation kernel with a float state (work
// items of a batch from a queue); the tile body is in simt_kernel.cuh.
#include "simt_kernel.cuh"

namespace aqt {

int launch_simt_batch_f32(const BatchLaunch &b, void *stream) {
    return simt::launch_batch_ra<float>(b, (cudaStream_t)stream);
}

int simt_batch_occupancy_f32(int RA, size_t smem) { return simt::batch_occupancy_ra<float>(RA, smem); }

}  // namespace aqt
