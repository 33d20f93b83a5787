// A run entry point that allocates no device memory for its scratch.
//
// Who needs it: callers that cannot allocate device memory when they run the
// propagation -- for example code that lives inside another framework's
// memory pool with a budget fixed at start-up, or host threads on which
// device allocation is not allowed. They still own and pass the tables
// (built into their workspace by aqt_build_tables) and the output buffers;
// the scratch the kernel needs (FP64 jump-resolution vectors and per-CTA
// partial sums of the observable) comes from one fixed array compiled into
// this library instead of from the caller.
//
// The array lives for as long as the library is loaded, on every GPU that
// loads it. All calls on a device share it: it keeps whatever the last call
// left there, and two calls whose kernels overlap on the GPU (different
// streams, or no ordering between them) race on it.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "aqt_internal.h"

namespace {

constexpr size_t kStaticScratchBytes = 32ull << 20;  // 32 MiB per device
constexpr int kMaxDevices = 64;

// File-scope device scratch. In host code this name is only a host-side
// handle: its device address must be obtained with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_mu;
struct SavedAddress {
    unsigned long long ctx_id = 0;  // driver id of the context the address belongs to
    void *ptr = nullptr;
};
SavedAddress g_saved[kMaxDevices];

// Unique id of the calling thread's current CUDA context (cuCtxGetId, through
// the runtime's driver entry points: the library does not link the driver).
// A context created after cudaDeviceReset gets a new id even if the driver
// reuses the old handle.
cudaError_t current_context_id(unsigned long long *id) {
    typedef int (*GetCurrentFn)(void **);
    typedef int (*GetIdFn)(void *, unsigned long long *);
    static GetCurrentFn get_current = nullptr;
    static GetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void *f0 = nullptr, *f1 = nullptr;
        cudaDriverEntryPointQueryResult q0, q1;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0);
        if (e == cudaSuccess) e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1);
        if (e != cudaSuccess) return e;
        if (q0 != cudaDriverEntryPointSuccess || q1 != cudaDriverEntryPointSuccess || !f0 || !f1)
            return cudaErrorSymbolNotFound;
        get_current = reinterpret_cast<GetCurrentFn>(f0);
        get_id = reinterpret_cast<GetIdFn>(f1);
    }
    void *ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx) return cudaErrorDeviceUninitialized;
    if (get_id(ctx, id) != 0) return cudaErrorDeviceUninitialized;
    return cudaSuccess;
}

// Device address of g_static_scratch in the current context of `device` (the
// device current on this thread). Looked up once per device and context, with
// that device current, and kept; a new context on the device (after
// cudaDeviceReset, say) makes the saved address stale, so it is looked up
// again.
cudaError_t scratch_address(int device, void **out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    unsigned long long id = 0;
    cudaError_t e = current_context_id(&id);
    if (e != cudaSuccess) return e;
    SavedAddress &s = g_saved[device];
    if (!s.ptr || s.ctx_id != id) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        s.ptr = p;
        s.ctx_id = id;
    }
    *out = s.ptr;
    return cudaSuccess;
}

}  // namespace

extern "C" aqt_status aqt_run_static_scratch(aqt_ctx *ctx, void *stream, double *obs_sums,
                                             double *final_states, aqt_jump *jumps, int64_t jump_capacity,
                                             unsigned long long *jump_count, int32_t *status) {
    if (!ctx || !obs_sums || !final_states || !jump_count || !status || jump_capacity < 0 ||
        (jump_capacity > 0 && !jumps))
        return AQT_EINVAL;
    size_t need = 0;
    aqt_status st = aqt::static_scratch_need(ctx, &need);
    if (st != AQT_OK) return st;
    if (need > kStaticScratchBytes)
        return aqt::set_error(ctx, AQT_EINVAL,
                              "this run needs " + std::to_string(need) + " bytes of scratch, more than the " +
                                  std::to_string(kStaticScratchBytes) + "-byte static array");
    aqt::RunParams p{};
    st = aqt::static_run_params(ctx, &p);
    if (st != AQT_OK) return st;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    void *base = nullptr;
    if (e == cudaSuccess) e = scratch_address(dev, &base);
    if (e != cudaSuccess)
        return aqt::set_error(ctx, AQT_ECUDA, std::string("static scratch address: ") + cudaGetErrorString(e));
    // Scratch carve: per-CTA observable partials, then per-warp FP64 jump
    // vectors. Every element the kernel reads is written earlier in the same
    // call, so nothing here has to start at zero.
    unsigned char *b = static_cast<unsigned char *>(base);
    const size_t part_bytes = (size_t)p.n_cta * p.K * 3 * sizeof(double);
    p.obs_part = reinterpret_cast<double *>(b);
    p.scratch = reinterpret_cast<double *>(b + ((part_bytes + 255) & ~(size_t)255));
    // Outputs belong to the caller; the two counters must start at zero.
    p.obs_sum = obs_sums;
    p.leak_sum = nullptr;  // the leakage sums are not recorded here
    p.final_state = final_states;
    p.jumps = jumps;
    p.jcap = jump_capacity;
    p.jcount = jump_count;
    p.status = status;
    p.norm_err = nullptr;  // the rotation-error diagnostic is not recorded here
    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMemsetAsync(jump_count, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return aqt::set_error(ctx, AQT_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    const int ce = aqt::launch_run(p, aqt::run_precision(ctx), stream, aqt::run_smem(ctx));
    if (ce) return aqt::set_error(ctx, AQT_ECUDA, std::string("kernel launch: ") + cudaGetErrorString((cudaError_t)ce));
    return AQT_OK;
}
