// Internal declarations shared by the host table builder, the C ABI and the
// CUDA kernels of the AME trajectory library.
#pragma once

#include <cstddef>
#include <cstdint>
#include <memory>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "../../include/aqt.h"

namespace aqt {

// ---------------------------------------------------------------- bath -----
struct Bath {
    double eta_g2 = 0.0, omega_c = 1.0, beta = 1.0;
    bool lamb_shift = false;
    struct Zone {
        double h = 0.0, half = 0.0;
        int n0 = 0;
        std::vector<double> val;
    };
    std::vector<Zone> zones;
    double gamma(double w) const;
    double lamb_direct(double w) const;
    double lamb(double w) const;
    void build_lamb(double wmax);
    // derivatives in w: of gamma in closed form (w != 0), of the tabulated S by
    // a central difference of the interpolant
    double gamma_deriv(double w) const;
    double lamb_deriv(double w) const;
    // gamma, gamma' (0 at w = 0), S and the derivative of its interpolant, in one call
    void rates(double w, double *g, double *dg, double *s, double *ds) const;
};

bool sym_eigen(int n, double *A, double *evals, double *V);

// The lowest eigenpairs of H = A (-sum_i sx_i) + B diag(Ez) on n qubits
// (matrix-free Chebyshev-filtered subspace iteration, FP64, block of p
// vectors), the lowest `want` converged to a residual of 1e-12 of the scale of
// H. X0: p start vectors ([p][2^n], any norm) or null for fixed pseudo-random
// ones. Out: evals[p] ascending (Ritz values), X [p][2^n] orthonormal,
// *restarts: filter passes used, *next_lower: a lower estimate of the next
// eigenvalue after the wanted ones (its Ritz value minus its residual). false
// if not converged.
bool lowest_eigen(int n, double A, double B, const double *Ez, int p, int want, const double *X0, double *evals,
                  double *X, int *restarts, double *next_lower);

// Allocator whose value-initialisation leaves trivial elements uninitialised:
// the large tables are written in full by the (threaded) builder, so zero
// filling them first only costs time.
template <typename T, typename A = std::allocator<T>>
class default_init_allocator : public A {
    using traits = std::allocator_traits<A>;

   public:
    template <typename U>
    struct rebind {
        using other = default_init_allocator<U, typename traits::template rebind_alloc<U>>;
    };
    using A::A;
    template <typename U>
    void construct(U *ptr) noexcept(std::is_nothrow_default_constructible<U>::value) {
        ::new (static_cast<void *>(ptr)) U;
    }
    template <typename U, typename... Args>
    void construct(U *ptr, Args &&...args) {
        traits::construct(static_cast<A &>(*this), ptr, std::forward<Args>(args)...);
    }
};
template <typename T>
using hvec = std::vector<T, default_init_allocator<T>>;

// --------------------------------------------------------------- tables -----
// Per-grid-point metadata (device-visible POD).
struct GridMeta {
    int32_t degenerate;  // some degenerate manifold has more than one level
    int32_t gs_size;     // size of the lowest manifold (observable support)
    int32_t simple;      // every Bohr class of nonzero frequency holds one manifold pair
    int32_t pad;
    double tol;          // energy tolerance for manifolds and Bohr classes
};

struct Tables {
    int n = 0, N = 0, K = 0;
    // basis dimension 2^n; N = D unless the lowest levels only are kept (N < D)
    int D = 0;
    bool truncated = false;
    std::vector<double> ev_next;  // [K] truncated: the first eigenvalue above the kept levels
    int lanczos_restarts = 0;     // truncated: largest number of restarts of one grid point
    double dt = 0.0, tau = 0.0;
    hvec<double> evals;          // [K][N]
    hvec<double> V;              // [K][D][N]  row x, column a
    std::vector<double> kdiag;   // [K][N][2]  diag of the eigenframe H_eff
    std::vector<double> ehalf;   // [K][N][2]  exp(-i K_aa tau)
    std::vector<double> d2;      // [K][N]     exp(2 Im K_aa tau)
    std::vector<double> G;       // [K][n][N]  sum_a gamma(w_ab) M_alpha[a,b]^2
    std::vector<double> Mdiag;   // [K][n][N]  M_alpha[b,b], M_alpha = V^T sz_alpha V
    // Jump amplitudes R_alpha[a][b] = sqrt(gamma(w_ab)) M_alpha[a][b], kept only
    // for the grid points that need the general jump routine (a degenerate
    // manifold, or a Bohr class of nonzero frequency with several level
    // pairs); source-major: Rgen[slot][alpha][b][a]. Elsewhere the device forms
    // the one column of M_alpha a jump needs from V.
    // Jump amplitudes of the lowest n_low source levels at every grid point
    // (where the population, hence nearly every jump, is), source-major:
    // Rlow[g][alpha][b][a] = R_alpha[a][b], b < n_low.
    int n_low = 0;
    hvec<double> Rlow;           // [K][n][n_low][N]
    std::vector<int32_t> gslot;  // [K] slot in Rgen, or -1
    int n_general = 0;
    hvec<double> Rgen;           // [n_general][n][N][N]
    std::vector<double> lvlE;    // [K][N]     energy of each level's manifold
    std::vector<int32_t> mfirst; // [K][N]     first level of each level's manifold
    std::vector<int32_t> msize;  // [K][N]     size of each level's manifold
    std::vector<GridMeta> meta;  // [K]
    hvec<double> OT;             // [K-1][N][N] transpose of O_g = V_{g+1}^T V_g: OT[b][a] = O[a][b]
    // Time-step conditions of Eq. newcond (Sec. IV), each term's minimum over the
    // grid (ns) and the grid point where it is reached: 2 |H_eff| / |dH_eff/dt|,
    // 1 / |H_eff|, |lambda / (lambda^2 - dlambda/dt)|.
    double dt_bound[3] = {0.0, 0.0, 0.0};
    int dt_bound_at[3] = {0, 0, 0};
    Bath bath;  // the bath with the Lamb-shift table the tables were built with
};

struct Inputs {
    int n = 0;
    std::vector<double> hz, J;
    std::vector<double> ks, kA, kB;
    Bath bath;
    bool have_ising = false, have_sched = false, have_bath = false, have_grid = false, have_traj = false;
    double t_f = 0.0;
    int K = 0;
    int64_t M = 0;
    uint64_t seed = 0;
    int precision = 0;
    int timing = 0;
    int64_t jcap = 0;
    int n_levels = 0;  // keep the lowest n_levels instantaneous levels (0: all)
    // levels the trajectories carry: n_levels when it truncates, else 2^n
    int levels() const { return (n_levels > 0 && n_levels < (1 << n)) ? n_levels : (1 << n); }
};

// Returns AQT_OK or an error with a message in *err.
aqt_status build_tables(const Inputs &in, Tables &tab, std::string *err);

// out[i*ld + j] = sum_k X[i][k] Y[j][k] (rows of length len, row-major).
void gram_rows(const double *X, const double *Y, int ni, int nj, int len, double *out, int ld);
// M_alpha = V_g^T sz_alpha V_g for every qubit, out[alpha][a][b], from the tables' eigenvectors.
void sz_frames_at(const Tables &tab, int g, double *M);
// A(s), B(s) of the piecewise-linear schedule.
void schedule_value(const Inputs &in, double s, double *A, double *B);

// Jump amplitudes R_alpha[a][b] = sqrt(gamma(w_ab)) M_alpha[a][b] of grid point
// g, out[alpha][a][b], recomputed from the tables' eigenvectors (inspection).
void jump_amplitudes(const Inputs &in, const Tables &tab, int g, double *out);

// ------------------------------------------------------------- kernels ------
struct DevTables {
    const double *kdiag, *ehalf, *d2, *G, *lvlE;
    const double *Mdiag;  // [g][alpha][N] diagonal of M_alpha
    const void *V;        // [g][x][a] eigenvectors in the state precision (double or float)
    const void *Rlow;     // [g][alpha][b][a], b < n_low: jump amplitudes in the state precision
    const int32_t *gslot; // [g] slot of the general jump tables, -1 at simple grid points
    const double *Rgen;   // [slot][alpha][b][a] jump amplitudes at general grid points
    const float *ehalf32;
    const int32_t *mfirst, *msize;
    const GridMeta *meta;
    const void *OT;     // FP64 or FP32 [g][b][a]; FP16 hi/lo K-block tiles for the tensor-core path
    const void *tclvl;  // tensor-core path: float4 [g][N] = (Re, Im of exp(-i K tau), 1 - d2, d2)
};

// When a jump happens inside a frozen half-step (Sec. IV): at the root of the
// norm-crossing condition (REFINED), or at the end of the half-step in which
// the norm fell to the threshold (GRID); or the fixed-step sampler of App. B.1
// (FIXED: a jump test with probability tau lambda at the start of each
// half-step).
enum JumpTiming : int { kTimingRefined = 0, kTimingGrid = 1, kTimingFixed = 2 };

// One jump of a segment recompute of a gradient run, kept for the backward
// sweep: where it happened (grid point, half-step, time after the half-step's
// start), its channel (qubit, source and target levels as draw_apply returns
// them) and whether the grid point used the general routine.
struct AdjJump {
    int32_t g, half, alpha, bsrc, adst, general;
    double t_rel;
};

// Gradient runs only (all pointers null otherwise). The forward run writes a
// checkpoint of every trajectory at the end of grid point ckpt_every*j - 1
// (j = 1, 2, ...): its state, clock, log threshold and jump count. A segment
// recompute restarts from checkpoint g_begin / ckpt_every (or the initial
// state), runs grid points g_begin .. g_end and writes, per grid point and
// trajectory, the normalised state at the start of the grid point's frozen
// span (after the frame rotation into it) and at its end, the norm of the
// rotated state, and its jumps.
struct AdjParams {
    void *ckpt;          // [n_ckpt][M][N][2] state precision
    double *ckpt_clock;  // [n_ckpt][M][2]: ell, log r
    int32_t *ckpt_nj;    // [n_ckpt][M]
    int ckpt_every;
    int g_begin, g_end;
    void *seg_c;         // [g - g_begin][2: start, end][M][N][2] state precision
    double *seg_nrot;    // [g - g_begin][M]
    AdjJump *jrec;       // [M][slots]
    double *jvec;        // [M][slots][2][N][2]: normalised state before and after the jump (FP64)
    int32_t *jn;         // [M] jumps of the segment so far
    int slots;
};

// One compact record of a jump for the host: where and which channel, then
// (in jump_vec) the normalised state before the jump and the adjoint after it.
struct AdjJumpOut {
    AdjJump r;
    int64_t traj;
};

struct AdjBack {
    const void *seg_c;       // [g - g_begin][2][M][N][2] state precision: c_s, c_e
    const double *seg_nrot;  // [g - g_begin][M]
    void *seg_mu;            // [g - g_begin][2][M][N][2]: mu_s, mu_e (written)
    void *carry;             // [M][N][2]: adjoint at the end of g_end (read), of g_begin - 1 (written)
    double *lev;             // [K][N][2] trajectory sums of 2 l (Im, Re)(mu_a^* c_a) (atomics)
    const AdjJump *jrec;     // [M][slots]
    const double *jvec;      // [M][slots][2][N][2]
    const int32_t *jn;       // [M]
    AdjJumpOut *jout;           // [jcap] compact jump list for the host
    double *jout_vec;        // [jcap][2][N][2]: state before, adjoint after (FP64)
    unsigned long long *jout_n;
    int64_t jout_cap;
    double *wscr;            // [n_cta][8 warps][10 N] FP64 per-warp scratch (jumped spans)
    double baseline;         // b; NaN: the run's mean of P at s = 1
    int g_begin, g_end, slots;
    int32_t *status;
};

struct RunParams {
    int n, N, K, TT, RA, n_cta;
    int timing;
    int n_low;  // source levels with a jump-amplitude table
    int64_t M;
    uint64_t seed;
    double tau, dt;
    double eta_g2, omega_c, beta;
    DevTables tab;
    double *final_state;           // [M][N][2]
    aqt_jump *jumps;
    int64_t jcap;
    unsigned long long *jcount;
    // per-tile partials [n_cta][K][3]: sum of x, sum of x^2, sum of the frame
    // rotation's norm loss 1 - |O c|^2 (the leakage of a truncated model; the
    // rounding of the rotation otherwise)
    double *obs_part;
    double *obs_sum;               // [K][2]
    double *leak_sum;              // [K] sum of 1 - |O c|^2 over trajectories, or null
    double *scratch;               // [n_cta][kScratchSlots][kSlotDouble2 * N][2] jump scratch
    int32_t *status;
    // Poll limit of the tensor-core kernel's bounded waits between its roles
    // (the waits also end after about 2 s).
    long long wait_polls;
    // Largest |(squared norm after a frame rotation) / (before) - 1| over all
    // trajectories and steps, as the bits of a non-negative float (atomicMax on
    // the bits orders like the values); not recorded when null.
    unsigned int *norm_err;
    AdjParams adj;
};

// Jump scratch per warp (SIMT) or jump slot (tensor-core path), in double2
// units per level: two FP64 vectors for the general jump operator, then one
// FP32 state (real, imaginary planes) handed between the epilogue warps.
constexpr int kSlotDouble2 = 3;
constexpr long long kDefaultWaitPolls = 1ll << 22;
constexpr int kLowSources = 16;  // source levels whose jump amplitudes are tabled at every grid point
constexpr int kScratchSlots = 8;

// Scratch bytes of a run: the jump slots of every CTA, then, for the
// tensor-core path, one next-step product per trajectory ([cta][TT][N] FP32
// complex) for trajectories that jump after the rotation has read their state.
inline size_t scratch_bytes(int n_cta, int N, int TT, bool tensor_core) {
    return (size_t)n_cta * kScratchSlots * kSlotDouble2 * N * 16 + (tensor_core ? (size_t)n_cta * TT * N * 8 : 0);
}

// Launch the propagation (precision per aqt_precision) and the observable
// reduction on `stream`. Returns a CUDA error code (0 on success).
int launch_run(const RunParams &p, int precision, void *stream, size_t smem_bytes);
int launch_simt_f32(const RunParams &p, void *stream, size_t smem);
// Gradient runs: one segment of the backward sweep (adjoint.cuh), the
// per-grid-point outer products X_g of a segment, and the backward tile's
// shared memory.
int launch_adjoint_f32(const RunParams &p, const AdjBack &b, void *stream, size_t smem);
int launch_adjoint_f64(const RunParams &p, const AdjBack &b, void *stream, size_t smem);
int launch_xgemm_f32(const void *seg_c, const void *seg_mu, int64_t M, int N, int K, int g_begin, int n_g,
                     double *xout, void *stream);
int launch_xgemm_f64(const void *seg_c, const void *seg_mu, int64_t M, int N, int K, int g_begin, int n_g,
                     double *xout, void *stream);
size_t adjoint_smem_bytes_f32(int N, int TT);
size_t adjoint_smem_bytes_f64(int N, int TT);
int launch_simt_f64(const RunParams &p, void *stream, size_t smem);

// ---------------------------------------------------------- batches ---------
// One work item of a batched launch: tile `cta` (trajectories cta*TT ..) of
// instance `inst`.
struct BatchItem {
    int32_t inst, cta;
};

// A persistent launch over the work items of many instances (device
// pointers): params[inst] are the instances' run parameters, items the work
// items in the order CTAs take them (queue: a counter that starts at 0),
// scratch one jump-scratch block of scr_stride double2 per CTA of the launch.
struct BatchLaunch {
    const RunParams *params = nullptr;
    const BatchItem *items = nullptr;
    int n_items = 0;
    int *queue = nullptr;
    void *scratch = nullptr;
    size_t scr_stride = 0;
    int n_cta = 0;   // CTAs of the launch
    int RA = 0;      // SIMT: rotation rows per thread (all instances of the launch)
    int MH = 0;      // tensor cores: 128-level blocks (all instances of the launch)
    size_t smem = 0; // dynamic shared memory per CTA
    uint32_t tc_tail = 0;  // tensor cores: shared-memory offset of the per-CTA words
    bool prepare_only = false;  // set the kernel's attributes only (before a stream capture)
};
int launch_simt_batch_f32(const BatchLaunch &b, void *stream);
int launch_simt_batch_f64(const BatchLaunch &b, void *stream);
int simt_batch_occupancy_f32(int RA, size_t smem);
int simt_batch_occupancy_f64(int RA, size_t smem);
int launch_tc_batch(const BatchLaunch &b, void *stream);
size_t tc_batch_scratch_double2(int N, int TT_max);
size_t tc_batch_smem_bytes(int N, int TT_max, uint32_t *tail);
// Sum the observable partials of every instance of a batch (params on the device).
int launch_reduce_batch(const RunParams *dev_params, int n_inst, int max_K, void *stream);
int simt_rows_per_thread(int N, int TT);
constexpr size_t kSimtSmemLimit = 200 * 1024;

// Context accessors for the static-scratch run entry point (static_scratch.cu):
// the scratch bytes a run of the current inputs needs, the run parameters
// pointing at the context's device tables (outputs and scratch left unset),
// the precision and the kernel's dynamic shared memory.
aqt_status static_scratch_need(aqt_ctx *ctx, size_t *bytes);

// Gradient runs (grad.cpp): the context's inputs, host tables and launch
// shape, and (need_device_tables) its run parameters over the device tables;
// the gradient state the context owns; marking the context's run as done on
// `stream` (for aqt_sync and the getters).
struct GradState;
void grad_free(GradState *g);
struct GradAccess {
    RunParams p;
    const Inputs *in = nullptr;
    const Tables *tab = nullptr;
    int TT = 0, RA = 0, n_cta = 0;
    size_t smem = 0;
    uint64_t version = 0;
};
aqt_status grad_access(aqt_ctx *ctx, GradAccess *a, bool need_device_tables);
GradState *grad_state_get(aqt_ctx *ctx);
// The context's inputs once every set_* call has been made, else null (no device needed).
const Inputs *ctx_inputs(const aqt_ctx *ctx);
void grad_state_set(aqt_ctx *ctx, GradState *g);
void grad_mark_ran(aqt_ctx *ctx, void *stream);
aqt_status static_run_params(aqt_ctx *ctx, RunParams *p);

// A context as a member of a batch: its run parameters over its device tables
// and workspace outputs (obs_part and scratch are replaced by the batch's),
// device, SM count, precision, and the version of its tables and workspace
// (a batch refuses to run once a member's version has changed).
struct BatchMember {
    RunParams p;
    int device = -1, num_sms = 0, precision = 0;
    uint64_t version = 0;
};
aqt_status batch_member(aqt_ctx *ctx, BatchMember *m);
uint64_t ctx_version(const aqt_ctx *ctx);
// Let aqt_sync and the getters of the context read the batch's run on `stream`.
void batch_member_ran(aqt_ctx *ctx, void *stream);
aqt_status set_error(aqt_ctx *ctx, aqt_status st, const std::string &msg);
int run_precision(const aqt_ctx *ctx);
size_t run_smem(const aqt_ctx *ctx);
size_t simt_smem_bytes(int N, int TT, int precision);
size_t tc_smem_bytes(int N, int TT);
int tc_shape(int N, int64_t M, int num_sms);
int launch_tc(const RunParams &p, void *stream, size_t smem);
void simt_shape(int N, int64_t M, int precision, int num_sms, int *TT, int *RA);

}  // namespace aqt
