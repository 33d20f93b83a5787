// C ABI of the AME trajectory library (declarations and contracts in include/aqt.h).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "aqt_internal.h"

using namespace aqt;

struct Layout {
    size_t kdiag, ehalf, ehalf32, d2, G, Mdiag, V, Rlow, gslot, Rgen, lvlE, mfirst, msize, meta, OT, tclvl;
    size_t final_state, jumps, jcount, obs_part, obs_sum, leak_sum, scratch, status, norm_err, total;
};

struct aqt_ctx {
    int device = -1;
    int num_sms = 152;
    std::string err;
    Inputs in;
    Tables tab;
    bool tables_built = false;
    bool tables_on_device = false;
    // launch shape
    int TT = 0, RA = 0, n_cta = 0;
    size_t smem = 0;
    Layout lay{};
    unsigned char *ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t stream = nullptr;
    bool ran = false;
    long long wait_polls = kDefaultWaitPolls;
    size_t uploaded = 0;  // bytes copied to the device by the last aqt_build_tables
    uint64_t version = 0;  // changes whenever the device tables or the workspace stop being valid
    GradState *grad = nullptr;  // gradient-run workspace and state (grad.cpp)
    ~aqt_ctx() { grad_free(grad); }
};

namespace {

aqt_status fail(aqt_ctx *c, aqt_status s, const std::string &m) {
    if (c) c->err = m;
    return s;
}

aqt_status cuda_fail(aqt_ctx *c, cudaError_t e, const char *what) {
    return fail(c, AQT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool inputs_complete(const aqt_ctx *c) {
    const Inputs &in = c->in;
    return in.have_ising && in.have_sched && in.have_bath && in.have_grid && in.have_traj;
}

void invalidate(aqt_ctx *c) {
    ++c->version;
    c->tables_built = false;
    c->tables_on_device = false;
    c->ran = false;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// f(i) for i < count on the host's cores.
template <class F>
void parallel_rows(size_t count, F f) {
    const unsigned nt = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
    std::atomic<size_t> next{0};
    std::vector<std::thread> th;
    for (unsigned t = 0; t < std::min<size_t>(nt, std::max<size_t>(count, 1)); ++t)
        th.emplace_back([&] {
            for (size_t i = next++; i < count; i = next++) f(i);
        });
    for (auto &x : th) x.join();
}

void compute_layout(aqt_ctx *c) {
    const Inputs &in = c->in;
    const size_t n = in.n, N = (size_t)in.levels(), K = in.K;
    const bool tc = in.precision == AQT_PREC_F16SPLIT;
    const size_t rs = in.precision == AQT_PREC_FP64 ? 8 : tc ? 4 : 4;
    if (tc) {
        c->TT = tc_shape((int)N, in.M, c->num_sms);
        c->RA = 0;
        c->smem = tc_smem_bytes((int)N, c->TT);
    } else {
        simt_shape((int)N, in.M, in.precision, c->num_sms, &c->TT, &c->RA);
        c->smem = simt_smem_bytes((int)N, c->TT, in.precision);
    }
    c->n_cta = (int)((in.M + c->TT - 1) / c->TT);
    Layout &L = c->lay;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    L.kdiag = take(K * N * 2 * 8);
    L.ehalf = take(K * N * 2 * 8);
    L.ehalf32 = take(K * N * 2 * 4);
    L.d2 = take(K * N * 8);
    L.G = take(K * n * N * 8);
    L.Mdiag = take(K * n * N * 8);
    // eigenvectors for the jump columns of sources above the tabled ones (none
    // when truncated: every source is tabled)
    L.V = take(c->tab.truncated ? 0 : K * N * N * (in.precision == AQT_PREC_FP64 ? 8 : 4));
    L.Rlow = take(K * n * (size_t)c->tab.n_low * N * (in.precision == AQT_PREC_FP64 ? 8 : 4));
    L.gslot = take(K * 4);
    L.Rgen = take((size_t)c->tab.n_general * n * N * N * 8);
    L.lvlE = take(K * N * 8);
    L.mfirst = take(K * N * 4);
    L.msize = take(K * N * 4);
    L.meta = take(K * sizeof(GridMeta));
    L.OT = take((K - 1) * N * N * rs);  // FP16 hi + lo for the tensor-core path: also 4 bytes per entry
    L.tclvl = take(tc ? K * N * 16 : 0);
    L.final_state = take((size_t)in.M * N * 2 * 8);
    L.jumps = take((size_t)std::max<int64_t>(in.jcap, 1) * sizeof(aqt_jump));
    L.jcount = take(8);
    L.obs_part = take((size_t)c->n_cta * K * 3 * 8);
    L.obs_sum = take(K * 2 * 8);
    L.leak_sum = take(K * 8);
    L.scratch = take(scratch_bytes(c->n_cta, (int)N, c->TT, tc));
    L.status = take(4);
    L.norm_err = take(4);
    L.total = off;
}

// Sizes the device paths take: the SIMT kernels take N <= 512 (the jump
// warp holds N/32 levels per lane in registers, at most 16); the tensor-core
// tiles take N = 128 or 256.
aqt_status device_shape_check(aqt_ctx *c) {
    const int N = c->in.levels();
    if (N > 512) return fail(c, AQT_EINVAL, "device runs take at most 512 levels (n_qubits <= 9, or aqt_set_levels)");
    if (c->in.precision == AQT_PREC_F16SPLIT && N != 128 && N != 256)
        return fail(c, AQT_EINVAL, "the tensor-core path takes N = 128 or 256 (n_qubits 7 or 8)");
    if (c->in.precision == AQT_PREC_F16SPLIT && c->in.timing == AQT_JUMP_FIXED_STEP)
        return fail(c, AQT_EINVAL, "the fixed-step sampler runs on the SIMT paths (AQT_PREC_FP64, AQT_PREC_FP32)");
    return AQT_OK;
}

aqt_status use_device(aqt_ctx *c) {
    if (c->device < 0) return fail(c, AQT_ENODEV, "context was created without a device");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    return AQT_OK;
}

// Run parameters over the context's device tables; outputs and scratch point
// into the workspace (the static-scratch entry point replaces them).
void fill_params(const aqt_ctx *c, RunParams *p) {
    const Layout &L = c->lay;
    const Inputs &in = c->in;
    *p = RunParams{};
    p->n = in.n;
    p->N = in.levels();
    p->K = in.K;
    p->TT = c->TT;
    p->RA = c->RA;
    p->n_cta = c->n_cta;
    p->timing = in.timing;
    p->M = in.M;
    p->seed = in.seed;
    p->tau = c->tab.tau;
    p->dt = c->tab.dt;
    p->eta_g2 = in.bath.eta_g2;
    p->omega_c = in.bath.omega_c;
    p->beta = in.bath.beta;
    p->tab.kdiag = (const double *)(c->ws + L.kdiag);
    p->tab.ehalf = (const double *)(c->ws + L.ehalf);
    p->tab.ehalf32 = (const float *)(c->ws + L.ehalf32);
    p->tab.d2 = (const double *)(c->ws + L.d2);
    p->tab.G = (const double *)(c->ws + L.G);
    p->tab.Mdiag = (const double *)(c->ws + L.Mdiag);
    p->tab.V = c->ws + L.V;
    p->tab.Rlow = c->ws + L.Rlow;
    p->n_low = c->tab.n_low;
    p->tab.gslot = (const int32_t *)(c->ws + L.gslot);
    p->tab.Rgen = (const double *)(c->ws + L.Rgen);
    p->tab.lvlE = (const double *)(c->ws + L.lvlE);
    p->tab.mfirst = (const int32_t *)(c->ws + L.mfirst);
    p->tab.msize = (const int32_t *)(c->ws + L.msize);
    p->tab.meta = (const GridMeta *)(c->ws + L.meta);
    p->tab.OT = c->ws + L.OT;
    p->tab.tclvl = c->ws + L.tclvl;
    p->final_state = (double *)(c->ws + L.final_state);
    p->jumps = (aqt_jump *)(c->ws + L.jumps);
    p->jcap = in.jcap;
    p->jcount = (unsigned long long *)(c->ws + L.jcount);
    p->obs_part = (double *)(c->ws + L.obs_part);
    p->obs_sum = (double *)(c->ws + L.obs_sum);
    p->leak_sum = (double *)(c->ws + L.leak_sum);
    p->scratch = (double *)(c->ws + L.scratch);
    p->status = (int32_t *)(c->ws + L.status);
    p->norm_err = (unsigned int *)(c->ws + L.norm_err);
    p->wait_polls = c->wait_polls;
}

// The host tables (built once per set of inputs): the workspace layout depends
// on them (the jump amplitudes are kept only at grid points that need them).
aqt_status ensure_host_tables(aqt_ctx *c) {
    if (c->tables_built) return AQT_OK;
    std::string err;
    aqt_status s = build_tables(c->in, c->tab, &err);
    if (s != AQT_OK) return fail(c, s, err);
    c->tables_built = true;
    return AQT_OK;
}

// AQT_WDT when the grid step is not well below a term of Eq. newcond (Sec. IV)
// that applies to the chosen jump timing, AQT_OK otherwise. "Well below":
// dt <= 0.1 x the term. The 1/|H_eff| term bounds the error of a first-order
// no-jump step; here the frozen-generator phases are exact, so it is reported
// (aqt_get_dt_bounds) but not checked. The lambda term bounds the error of a
// fixed-step jump probability, which GRID timing and the fixed-step sampler make.
aqt_status dt_warning(aqt_ctx *c) {
    const Tables &t = c->tab;
    static const char *what[3] = {"2|H_eff|/|dH_eff/dt|", "1/|H_eff|", "|lambda/(lambda^2 - dlambda/dt)|"};
    std::string msg;
    for (int i = 0; i < 3; ++i) {
        if (i == 1 || (i == 2 && c->in.timing == AQT_JUMP_REFINED)) continue;
        if (t.dt > 0.1 * t.dt_bound[i])
            msg += std::string(msg.empty() ? "" : "; ") + "dt = " + std::to_string(t.dt) + " ns is not << " + what[i] +
                   " = " + std::to_string(t.dt_bound[i]) + " ns (grid point " + std::to_string(t.dt_bound_at[i]) + ")";
    }
    if (msg.empty()) return AQT_OK;
    return fail(c, AQT_WDT, "time-step condition of Eq. newcond: " + msg);
}

}  // namespace

// ---- accessors for the static-scratch entry point (static_scratch.cu) ------
namespace aqt {

aqt_status set_error(aqt_ctx *c, aqt_status st, const std::string &msg) { return fail(c, st, msg); }

int run_precision(const aqt_ctx *c) { return c->in.precision; }

size_t run_smem(const aqt_ctx *c) { return c->smem; }

aqt_status static_scratch_need(aqt_ctx *c, size_t *bytes) {
    if (!inputs_complete(c)) return fail(c, AQT_EINVAL, "set all inputs first");
    aqt_status s = device_shape_check(c);
    if (s == AQT_OK) s = use_device(c);
    if (s != AQT_OK) return s;
    compute_layout(c);
    const size_t N = (size_t)c->in.levels(), K = c->in.K;
    const size_t part = ((size_t)c->n_cta * K * 3 * 8 + 255) & ~(size_t)255;
    *bytes = part + scratch_bytes(c->n_cta, (int)N, c->TT, c->in.precision == AQT_PREC_F16SPLIT);
    return AQT_OK;
}

aqt_status batch_member(aqt_ctx *c, BatchMember *m) {
    if (!c->tables_on_device) return fail(c, AQT_EINVAL, "build tables on the device before batching");
    aqt_status s = device_shape_check(c);
    if (s == AQT_OK) s = use_device(c);
    if (s != AQT_OK) return s;
    fill_params(c, &m->p);
    m->device = c->device;
    m->num_sms = c->num_sms;
    m->precision = c->in.precision;
    m->version = c->version;
    return AQT_OK;
}

uint64_t ctx_version(const aqt_ctx *c) { return c->version; }

void batch_member_ran(aqt_ctx *c, void *stream) {
    c->stream = (cudaStream_t)stream;
    c->ran = true;
}

aqt_status grad_access(aqt_ctx *c, GradAccess *a, bool need_device_tables) {
    if (!inputs_complete(c)) return fail(c, AQT_EINVAL, "set all inputs first");
    aqt_status s = device_shape_check(c);
    if (s == AQT_OK) s = use_device(c);
    if (s != AQT_OK) return s;
    if (need_device_tables) {
        if (!c->tables_on_device) return fail(c, AQT_EINVAL, "build tables on the device before running");
        fill_params(c, &a->p);
    } else {
        if ((s = ensure_host_tables(c)) != AQT_OK) return s;
        compute_layout(c);
        a->p = RunParams{};
    }
    a->in = &c->in;
    a->tab = &c->tab;
    a->TT = c->TT;
    a->RA = c->RA;
    a->n_cta = c->n_cta;
    a->smem = c->smem;
    a->version = c->version;
    return AQT_OK;
}

GradState *grad_state_get(aqt_ctx *c) { return c->grad; }

const Inputs *ctx_inputs(const aqt_ctx *c) { return inputs_complete(c) ? &c->in : nullptr; }

void grad_state_set(aqt_ctx *c, GradState *g) {
    grad_free(c->grad);
    c->grad = g;
}

void grad_mark_ran(aqt_ctx *c, void *stream) {
    c->stream = (cudaStream_t)stream;
    c->ran = true;
}

aqt_status static_run_params(aqt_ctx *c, RunParams *p) {
    aqt_status s = use_device(c);
    if (s != AQT_OK) return s;
    if (!c->tables_on_device) return fail(c, AQT_EINVAL, "build tables on the device before running");
    fill_params(c, p);
    return AQT_OK;
}

}  // namespace aqt

extern "C" {

aqt_status aqt_create(aqt_ctx **out, int device) {
    if (!out) return AQT_EINVAL;
    *out = nullptr;
    aqt_ctx *c = new (std::nothrow) aqt_ctx();
    if (!c) return AQT_EINVAL;
    c->device = device;
    if (device >= 0) {
        int nd = 0;
        cudaError_t e = cudaGetDeviceCount(&nd);
        if (e != cudaSuccess || device >= nd) {
            delete c;
            return AQT_ECUDA;
        }
        e = cudaSetDevice(device);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
        if (e != cudaSuccess) {
            delete c;
            return AQT_ECUDA;
        }
    } else if (device != -1) {
        delete c;
        return AQT_EINVAL;
    }
    *out = c;
    return AQT_OK;
}

void aqt_destroy(aqt_ctx *c) { delete c; }

const char *aqt_last_error(const aqt_ctx *c) { return c ? c->err.c_str() : "null context"; }

aqt_status aqt_set_ising(aqt_ctx *c, int n_qubits, const double *hz, const double *Jzz) {
    if (!c) return AQT_EINVAL;
    if (n_qubits < 1 || n_qubits > 16) return fail(c, AQT_EINVAL, "n_qubits must be in [1, 16]");
    if (!hz || !Jzz) return fail(c, AQT_EINVAL, "hz and Jzz must be non-null");
    for (int i = 0; i < n_qubits; ++i)
        if (!std::isfinite(hz[i])) return fail(c, AQT_EINVAL, "hz has a non-finite entry");
    for (int i = 0; i < n_qubits * n_qubits; ++i)
        if (!std::isfinite(Jzz[i])) return fail(c, AQT_EINVAL, "Jzz has a non-finite entry");
    c->in.n = n_qubits;
    c->in.hz.assign(hz, hz + n_qubits);
    c->in.J.assign(Jzz, Jzz + n_qubits * n_qubits);
    c->in.have_ising = true;
    invalidate(c);
    return AQT_OK;
}

aqt_status aqt_set_schedule(aqt_ctx *c, int n_knots, const double *s, const double *A, const double *B) {
    if (!c) return AQT_EINVAL;
    if (n_knots < 2 || !s || !A || !B) return fail(c, AQT_EINVAL, "schedule needs >= 2 knots");
    if (s[0] != 0.0 || s[n_knots - 1] != 1.0) return fail(c, AQT_EINVAL, "schedule knots must span [0, 1]");
    for (int i = 0; i < n_knots; ++i) {
        if (!std::isfinite(A[i]) || !std::isfinite(B[i])) return fail(c, AQT_EINVAL, "schedule has a non-finite value");
        if (i && !(s[i] > s[i - 1])) return fail(c, AQT_EINVAL, "schedule knots must increase strictly");
    }
    c->in.ks.assign(s, s + n_knots);
    c->in.kA.assign(A, A + n_knots);
    c->in.kB.assign(B, B + n_knots);
    c->in.have_sched = true;
    invalidate(c);
    return AQT_OK;
}

aqt_status aqt_set_bath(aqt_ctx *c, double eta_g2, double omega_c, double beta, int lamb_shift) {
    if (!c) return AQT_EINVAL;
    if (!(eta_g2 >= 0.0) || !(omega_c > 0.0) || !(beta > 0.0) || !std::isfinite(eta_g2) ||
        !std::isfinite(omega_c) || !std::isfinite(beta))
        return fail(c, AQT_EINVAL, "bath needs eta_g2 >= 0, omega_c > 0, beta > 0");
    c->in.bath = Bath();
    c->in.bath.eta_g2 = eta_g2;
    c->in.bath.omega_c = omega_c;
    c->in.bath.beta = beta;
    c->in.bath.lamb_shift = lamb_shift != 0;
    c->in.have_bath = true;
    invalidate(c);
    return AQT_OK;
}

aqt_status aqt_set_levels(aqt_ctx *c, int n_levels) {
    if (!c) return AQT_EINVAL;
    if (n_levels < 0 || n_levels > 65536) return fail(c, AQT_EINVAL, "n_levels must be in [0, 65536]");
    c->in.n_levels = n_levels;
    invalidate(c);
    return AQT_OK;
}

aqt_status aqt_set_grid(aqt_ctx *c, double t_f, int n_grid) {
    if (!c) return AQT_EINVAL;
    if (!(t_f > 0.0) || !std::isfinite(t_f) || n_grid < 2 || n_grid > 1000000)
        return fail(c, AQT_EINVAL, "grid needs t_f > 0 and 2 <= n_grid <= 1e6");
    c->in.t_f = t_f;
    c->in.K = n_grid;
    c->in.have_grid = true;
    invalidate(c);
    return AQT_OK;
}

aqt_status aqt_set_trajectories(aqt_ctx *c, int64_t M, uint64_t seed, int precision, int jump_timing,
                                int64_t jump_capacity) {
    if (!c) return AQT_EINVAL;
    if (M < 1 || M > (int64_t)1 << 31) return fail(c, AQT_EINVAL, "M must be in [1, 2^31]");
    if (precision != AQT_PREC_FP64 && precision != AQT_PREC_FP32 && precision != AQT_PREC_F16SPLIT)
        return fail(c, AQT_EINVAL, "unknown precision");
    if (jump_timing != AQT_JUMP_REFINED && jump_timing != AQT_JUMP_GRID && jump_timing != AQT_JUMP_FIXED_STEP)
        return fail(c, AQT_EINVAL, "unknown jump timing");
    if (jump_capacity < 0) return fail(c, AQT_EINVAL, "jump_capacity must be >= 0");
    c->in.M = M;
    c->in.seed = seed;
    c->in.precision = precision;
    c->in.timing = jump_timing;
    c->in.jcap = jump_capacity;
    c->in.have_traj = true;
    invalidate(c);
    return AQT_OK;
}

aqt_status aqt_workspace_size(aqt_ctx *c, size_t *bytes) {
    if (!c || !bytes) return AQT_EINVAL;
    if (!inputs_complete(c)) return fail(c, AQT_EINVAL, "set ising, schedule, bath, grid and trajectories first");
    aqt_status s = device_shape_check(c);
    if (s == AQT_OK) s = ensure_host_tables(c);
    if (s != AQT_OK) return s;
    compute_layout(c);
    *bytes = c->lay.total;
    return AQT_OK;
}

aqt_status aqt_bind_workspace(aqt_ctx *c, void *dptr, size_t bytes) {
    if (!c) return AQT_EINVAL;
    if (!inputs_complete(c)) return fail(c, AQT_EINVAL, "set all inputs before binding a workspace");
    aqt_status s = device_shape_check(c);
    if (s == AQT_OK) s = ensure_host_tables(c);
    if (s != AQT_OK) return s;
    compute_layout(c);
    if (!dptr || ((uintptr_t)dptr & 255)) return fail(c, AQT_EINVAL, "workspace must be 256-byte aligned");
    if (bytes < c->lay.total) return fail(c, AQT_ENOMEM, "workspace smaller than aqt_workspace_size");
    c->ws = (unsigned char *)dptr;
    c->ws_bytes = bytes;
    ++c->version;
    c->tables_on_device = false;
    c->ran = false;
    return AQT_OK;
}

aqt_status aqt_build_tables(aqt_ctx *c, void *stream) {
    if (!c) return AQT_EINVAL;
    if (!inputs_complete(c)) return fail(c, AQT_EINVAL, "set all inputs before building tables");
    aqt_status s = ensure_host_tables(c);
    if (s != AQT_OK) return s;
    if (c->device < 0) return dt_warning(c);
    s = device_shape_check(c);
    if (s == AQT_OK) s = use_device(c);
    if (s != AQT_OK) return s;
    if (!c->ws) return fail(c, AQT_EINVAL, "bind a workspace before building tables on a device");
    compute_layout(c);
    if (c->ws_bytes < c->lay.total) return fail(c, AQT_ENOMEM, "workspace smaller than aqt_workspace_size");
    cudaStream_t st = (cudaStream_t)stream;
    const Tables &t = c->tab;
    const Layout &L = c->lay;
    const size_t N = t.N, K = t.K, NN = N * N;
    c->uploaded = 0;
    auto put = [&](size_t off, const void *src, size_t bytes) -> cudaError_t {
        if (!bytes) return cudaSuccess;
        c->uploaded += bytes;
        return cudaMemcpyAsync(c->ws + off, src, bytes, cudaMemcpyHostToDevice, st);
    };
    std::vector<float> e32(t.ehalf.begin(), t.ehalf.end());
    cudaError_t e = cudaSuccess;
    if (!e) e = put(L.kdiag, t.kdiag.data(), t.kdiag.size() * 8);
    if (!e) e = put(L.ehalf, t.ehalf.data(), t.ehalf.size() * 8);
    if (!e) e = put(L.ehalf32, e32.data(), e32.size() * 4);
    if (!e) e = put(L.d2, t.d2.data(), t.d2.size() * 8);
    if (!e) e = put(L.G, t.G.data(), t.G.size() * 8);
    if (!e) e = put(L.Mdiag, t.Mdiag.data(), t.Mdiag.size() * 8);
    if (!e) e = put(L.gslot, t.gslot.data(), t.gslot.size() * 4);
    if (!e) e = put(L.Rgen, t.Rgen.data(), t.Rgen.size() * 8);
    if (!e) e = put(L.lvlE, t.lvlE.data(), t.lvlE.size() * 8);
    if (!e) e = put(L.mfirst, t.mfirst.data(), t.mfirst.size() * 4);
    if (!e) e = put(L.msize, t.msize.data(), t.msize.size() * 4);
    if (!e) e = put(L.meta, t.meta.data(), t.meta.size() * sizeof(GridMeta));
    // eigenvectors (jump columns) and frame rotations in the state precision
    hvec<float> v32, o32;
    hvec<__half> o16;
    std::vector<float> lv;
    hvec<float> rl32;
    if (c->in.precision == AQT_PREC_FP64) {
        if (!e && !t.truncated) e = put(L.V, t.V.data(), t.V.size() * 8);
        if (!e) e = put(L.Rlow, t.Rlow.data(), t.Rlow.size() * 8);
        if (!e) e = put(L.OT, t.OT.data(), t.OT.size() * 8);
    } else {
        if (!t.truncated) {
            v32.resize(K * NN);
            parallel_rows(K, [&](size_t g) {
                for (size_t i = 0; i < NN; ++i) v32[g * NN + i] = (float)t.V[g * NN + i];
            });
            if (!e) e = put(L.V, v32.data(), v32.size() * 4);
        }
        rl32.assign(t.Rlow.begin(), t.Rlow.end());
        if (!e) e = put(L.Rlow, rl32.data(), rl32.size() * 4);
    }
    if (c->in.precision == AQT_PREC_F16SPLIT) {
        // A-operand tiles in the order the tensor-core kernel streams them: per grid
        // step, 128-level block h of rows a, and pair of K-blocks (16 levels b
        // each), a 16 KB stage: the hi halves of O[a][b] for the two K-blocks
        // (4 KB each), then the lo halves. Each 4 KB block holds 8x16-byte core
        // matrices: core (a/8, k/8) at ((a/8)*2 + k/8)*128 bytes, row a%8 at 16
        // bytes, column k%8 at 2 bytes (a, k local to the block).
        const size_t NK = N / 16, MH = N / 128;
        o16.resize((K - 1) * NN * 2);
        parallel_rows(K - 1, [&](size_t g) {
            for (size_t h = 0; h < MH; ++h)
                for (size_t kb = 0; kb < NK; ++kb) {
                    __half *hi = &o16[((g * MH + h) * (NK / 2) + kb / 2) * 8192 + (kb & 1) * 2048];
                    __half *lo = hi + 4096;
                    for (size_t al = 0; al < 128; ++al)
                        for (size_t k = 0; k < 16; ++k) {
                            const double o = t.OT[g * NN + (kb * 16 + k) * N + 128 * h + al];
                            const __half hh = __float2half_rn((float)o);
                            const __half ll = __float2half_rn((float)(o - (double)__half2float(hh)));
                            const size_t off = ((al >> 3) * 2 + (k >> 3)) * 64 + (al & 7) * 8 + (k & 7);
                            hi[off] = hh;
                            lo[off] = ll;
                        }
                }
        });
        lv.resize(K * N * 4);
        for (size_t g = 0; g < K; ++g)
            for (size_t a = 0; a < N; ++a) {
                const double im = t.kdiag[(g * N + a) * 2 + 1];
                lv[(g * N + a) * 4 + 0] = (float)t.ehalf[(g * N + a) * 2];
                lv[(g * N + a) * 4 + 1] = (float)t.ehalf[(g * N + a) * 2 + 1];
                lv[(g * N + a) * 4 + 2] = (float)(-std::expm1(2.0 * im * t.tau));
                lv[(g * N + a) * 4 + 3] = (float)t.d2[g * N + a];
            }
        if (!e) e = put(L.OT, o16.data(), o16.size() * sizeof(__half));
        if (!e) e = put(L.tclvl, lv.data(), lv.size() * 4);
    } else if (c->in.precision == AQT_PREC_FP32) {
        o32.resize((K - 1) * NN);
        parallel_rows(K - 1, [&](size_t g) {
            for (size_t i = 0; i < NN; ++i) o32[g * NN + i] = (float)t.OT[g * NN + i];
        });
        if (!e) e = put(L.OT, o32.data(), o32.size() * 4);
    }
    if (!e) e = cudaStreamSynchronize(st);  // host staging buffers go out of scope
    if (e) return cuda_fail(c, e, "table upload");
    c->tables_on_device = true;
    return dt_warning(c);
}

aqt_status aqt_run(aqt_ctx *c, void *stream) {
    if (!c) return AQT_EINVAL;
    aqt_status s = use_device(c);
    if (s != AQT_OK) return s;
    if (!c->tables_on_device) return fail(c, AQT_EINVAL, "build tables on the device before running");
    const Layout &L = c->lay;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(c->ws + L.jcount, 0, 8, st);
    if (!e) e = cudaMemsetAsync(c->ws + L.status, 0, 4, st);
    if (!e) e = cudaMemsetAsync(c->ws + L.norm_err, 0, 4, st);
    if (e) return cuda_fail(c, e, "cudaMemsetAsync");
    RunParams p;
    fill_params(c, &p);
    int ce = launch_run(p, c->in.precision, stream, c->smem);
    if (ce) return cuda_fail(c, (cudaError_t)ce, "kernel launch");
    c->stream = st;
    c->ran = true;
    return AQT_OK;
}

aqt_status aqt_sync(aqt_ctx *c) {
    if (!c) return AQT_EINVAL;
    aqt_status s = use_device(c);
    if (s != AQT_OK) return s;
    if (!c->ran) return fail(c, AQT_EINVAL, "no run to wait for");
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e) return cuda_fail(c, e, "run");
    int32_t status = 0;
    unsigned long long cnt = 0;
    e = cudaMemcpy(&status, c->ws + c->lay.status, 4, cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(&cnt, c->ws + c->lay.jcount, 8, cudaMemcpyDeviceToHost);
    if (e) return cuda_fail(c, e, "status readback");
    if (status & 4) {
        std::string where;
        static const char *site[] = {"producer ring slot", "producer drain", "B operand ready", "ring stage full",
                                     "product done", "abort drain"};
        for (int i = 0; i < 6; ++i)
            if (status & (1 << (8 + i))) where += std::string(where.empty() ? "" : ", ") + site[i];
        return fail(c, AQT_ETIMEOUT, "a bounded wait expired in the tensor-core kernel (" + where + ")");
    }
    if (status & 2) return fail(c, AQT_ENUMERIC, "non-finite norm or too many jumps in one half-step");
    if ((int64_t)cnt > c->in.jcap)
        return fail(c, AQT_EOVERFLOW, "jump log full: " + std::to_string((int64_t)cnt - c->in.jcap) + " dropped");
    return AQT_OK;
}

aqt_status aqt_get_observable_sums(aqt_ctx *c, double *sum_x, double *sum_x2) {
    if (!c || !sum_x || !sum_x2) return AQT_EINVAL;
    aqt_status s = use_device(c);
    if (s != AQT_OK) return s;
    if (!c->ran) return fail(c, AQT_EINVAL, "run first");
    const int K = c->in.K;
    std::vector<double> buf((size_t)K * 2);
    cudaError_t e = cudaMemcpy(buf.data(), c->ws + c->lay.obs_sum, buf.size() * 8, cudaMemcpyDeviceToHost);
    if (e) return cuda_fail(c, e, "observable readback");
    for (int g = 0; g < K; ++g) {
        sum_x[g] = buf[2 * g];
        sum_x2[g] = buf[2 * g + 1];
    }
    return AQT_OK;
}

aqt_status aqt_get_leakage(aqt_ctx *c, double *sum_leak) {
    if (!c || !sum_leak) return AQT_EINVAL;
    aqt_status s = use_device(c);
    if (s != AQT_OK) return s;
    if (!c->ran) return fail(c, AQT_EINVAL, "run first");
    cudaError_t e = cudaMemcpy(sum_leak, c->ws + c->lay.leak_sum, (size_t)c->in.K * 8, cudaMemcpyDeviceToHost);
    if (e) return cuda_fail(c, e, "leakage readback");
    return AQT_OK;
}

aqt_status aqt_set_wait_limit(aqt_ctx *c, int64_t polls) {
    if (!c) return AQT_EINVAL;
    if (polls < 0 || polls > kDefaultWaitPolls) return fail(c, AQT_EINVAL, "poll limit must be in [0, 2^22]");
    c->wait_polls = polls;
    return AQT_OK;
}

aqt_status aqt_get_dt_bounds(aqt_ctx *c, double *bounds, int32_t *at) {
    if (!c || !bounds) return AQT_EINVAL;
    if (!c->tables_built) return fail(c, AQT_EINVAL, "build tables first");
    for (int i = 0; i < 3; ++i) {
        bounds[i] = c->tab.dt_bound[i];
        if (at) at[i] = c->tab.dt_bound_at[i];
    }
    return AQT_OK;
}

aqt_status aqt_get_rotation_error(aqt_ctx *c, double *max_rel) {
    if (!c || !max_rel) return AQT_EINVAL;
    aqt_status s = use_device(c);
    if (s != AQT_OK) return s;
    if (!c->ran) return fail(c, AQT_EINVAL, "run first");
    unsigned int bits = 0;
    cudaError_t e = cudaMemcpy(&bits, c->ws + c->lay.norm_err, 4, cudaMemcpyDeviceToHost);
    if (e) return cuda_fail(c, e, "norm error readback");
    float v;
    std::memcpy(&v, &bits, 4);
    *max_rel = v;
    return AQT_OK;
}

aqt_status aqt_observables_from_sums(int n_grid, int64_t M, const double *sum_x, const double *sum_x2,
                                     double *mean, double *stderr_) {
    if (n_grid < 1 || M < 1 || !sum_x || !sum_x2 || !mean || !stderr_) return AQT_EINVAL;
    const double R = (double)M;
    for (int g = 0; g < n_grid; ++g) {
        mean[g] = sum_x[g] / R;
        // Eq. stderror: sigma^2 = sum (x - mean)^2 / (R (R - 1))
        const double ss = std::max(0.0, sum_x2[g] - R * mean[g] * mean[g]);
        stderr_[g] = R > 1 ? std::sqrt(ss / (R * (R - 1.0))) : 0.0;
    }
    return AQT_OK;
}

aqt_status aqt_get_observables(aqt_ctx *c, double *mean, double *stderr_) {
    if (!c || !mean || !stderr_) return AQT_EINVAL;
    const int K = c->in.K;
    std::vector<double> s1(K), s2(K);
    aqt_status s = aqt_get_observable_sums(c, s1.data(), s2.data());
    if (s != AQT_OK) return s;
    return aqt_observables_from_sums(K, c->in.M, s1.data(), s2.data(), mean, stderr_);
}

aqt_status aqt_get_jumps(aqt_ctx *c, aqt_jump *host_buf, int64_t cap, int64_t *n_out, int64_t *n_dropped) {
    if (!c || !n_out || !n_dropped || cap < 0 || (cap > 0 && !host_buf)) return AQT_EINVAL;
    aqt_status s = use_device(c);
    if (s != AQT_OK) return s;
    if (!c->ran) return fail(c, AQT_EINVAL, "run first");
    unsigned long long cnt = 0;
    cudaError_t e = cudaMemcpy(&cnt, c->ws + c->lay.jcount, 8, cudaMemcpyDeviceToHost);
    if (e) return cuda_fail(c, e, "jump count readback");
    const int64_t kept = std::min<int64_t>((int64_t)cnt, c->in.jcap);
    std::vector<aqt_jump> all((size_t)kept);
    if (kept) {
        e = cudaMemcpy(all.data(), c->ws + c->lay.jumps, (size_t)kept * sizeof(aqt_jump), cudaMemcpyDeviceToHost);
        if (e) return cuda_fail(c, e, "jump readback");
    }
    std::sort(all.begin(), all.end(), [](const aqt_jump &a, const aqt_jump &b) {
        if (a.traj != b.traj) return a.traj < b.traj;
        return a.t < b.t;
    });
    const int64_t nout = std::min<int64_t>(kept, cap);
    if (nout) std::memcpy(host_buf, all.data(), (size_t)nout * sizeof(aqt_jump));
    *n_out = nout;
    *n_dropped = (int64_t)cnt - kept;
    return AQT_OK;
}

aqt_status aqt_get_final_state(aqt_ctx *c, int basis, double *host_buf) {
    if (!c || !host_buf || (basis != 0 && basis != 1)) return AQT_EINVAL;
    aqt_status s = use_device(c);
    if (s != AQT_OK) return s;
    if (!c->ran) return fail(c, AQT_EINVAL, "run first");
    const size_t N = (size_t)c->in.levels(), D = (size_t)1 << c->in.n, M = (size_t)c->in.M;
    if (basis == 0) {
        cudaError_t e = cudaMemcpy(host_buf, c->ws + c->lay.final_state, M * N * 2 * 8, cudaMemcpyDeviceToHost);
        if (e) return cuda_fail(c, e, "final state readback");
        return AQT_OK;
    }
    // computational basis: psi = V c with the eigenvectors of s = 1 (D x N)
    std::vector<double> eig(M * N * 2);
    cudaError_t e = cudaMemcpy(eig.data(), c->ws + c->lay.final_state, M * N * 2 * 8, cudaMemcpyDeviceToHost);
    if (e) return cuda_fail(c, e, "final state readback");
    const double *V = &c->tab.V[(size_t)(c->in.K - 1) * D * N];
    for (size_t m = 0; m < M; ++m) {
        const double *cm = &eig[m * N * 2];
        double *out = host_buf + m * D * 2;
        for (size_t x = 0; x < D; ++x) {
            double re = 0.0, im = 0.0;
            for (size_t a = 0; a < N; ++a) {
                re += V[x * N + a] * cm[2 * a];
                im += V[x * N + a] * cm[2 * a + 1];
            }
            out[2 * x] = re;
            out[2 * x + 1] = im;
        }
    }
    return AQT_OK;
}

aqt_status aqt_debug_table(aqt_ctx *c, int which, int grid, double *out) {
    if (!c || !out) return AQT_EINVAL;
    if (!c->tables_built) return fail(c, AQT_EINVAL, "build tables first");
    const Tables &t = c->tab;
    const size_t N = t.N, n = t.n, NN = N * N;
    if (grid < 0 || grid >= t.K || (which == 4 && grid >= t.K - 1)) return fail(c, AQT_EINVAL, "grid out of range");
    const size_t g = grid;
    switch (which) {
        case 0: std::copy_n(&t.evals[g * N], N, out); break;
        case 1: std::copy_n(&t.kdiag[g * N * 2], N * 2, out); break;
        case 2: std::copy_n(&t.G[g * n * N], n * N, out); break;
        case 3: jump_amplitudes(c->in, t, (int)g, out); break;
        case 4:
            for (size_t a = 0; a < N; ++a)
                for (size_t b = 0; b < N; ++b) out[a * N + b] = t.OT[g * NN + b * N + a];
            break;
        case 5: std::copy_n(&t.V[g * (size_t)t.D * N], (size_t)t.D * N, out); break;
        case 6: std::copy_n(&t.lvlE[g * N], N, out); break;
        case 7:
            out[0] = t.meta[g].degenerate;
            out[1] = t.meta[g].gs_size;
            out[2] = t.meta[g].simple;
            out[3] = t.meta[g].tol;
            break;
        case 8:
            out[0] = t.n_general;
            out[1] = (double)c->uploaded;
            break;
        case 9:  // truncated: the first eigenvalue above the kept levels, and the most Lanczos restarts of a point
            out[0] = t.truncated ? t.ev_next[g] : 0.0;
            out[1] = t.lanczos_restarts;
            break;
        default: return fail(c, AQT_EINVAL, "unknown table");
    }
    return AQT_OK;
}

}  // extern "C"
