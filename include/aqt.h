/*
 * aqt — quantum-jump trajectories of the time-dependent adiabatic master
 * equation (AME) on one GB300 GPU (sm_103a).
 *
 * Method: Yip, Albash, Lidar, "Quantum trajectories for time-dependent
 * adiabatic master equations" (arXiv:1710.03431). The library propagates M
 * independent N-level trajectories of a transverse-field Ising annealing
 * Hamiltonian under the non-Hermitian effective Hamiltonian of Sec. III
 * (Eq. Heff), detects each trajectory's jump when its squared norm falls to
 * a uniform random threshold (Sec. IV; App. C), draws the jump channel with
 * the probabilities of App. B.1 (Eq. Pi(t)), applies it (Eq. jump),
 * renormalises, and accumulates the ground-state population (Sec. V) with
 * its standard error (Sec. VI.A, Eq. stderror).
 *
 * Conventions (all calls):
 *  - Units: hbar = 1; energies and rates in rad/ns, times in ns, beta in ns.
 *  - Basis index x = sum_i bit_i 2^i; qubit i <-> bit i; bit 0 <-> sz = +1.
 *  - Every call returns an aqt_status; errors are returned, never thrown.
 *    After a non-OK status, aqt_last_error() gives a one-line reason.
 *  - Host arrays passed in are copied before the call returns; the library
 *    keeps no host pointer of the caller.
 *  - Device memory is owned by the caller: one workspace buffer, sized by
 *    aqt_workspace_size() and bound with aqt_bind_workspace(). The library
 *    allocates no device memory of its own.
 *  - Streams are the caller's (a cudaStream_t passed as void*; NULL is the
 *    legacy default stream).
 *  - A context is not thread-safe; use one per host thread.
 *
 * Call order: create -> set_ising, set_schedule, set_bath, set_grid,
 * set_trajectories -> workspace_size -> bind_workspace -> build_tables ->
 * run -> sync -> get_observables / get_jumps / get_final_state. Changing any
 * set_* input invalidates the tables and the workspace size.
 */
#ifndef AQT_H
#define AQT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct aqt_ctx aqt_ctx;

typedef enum {
    AQT_OK = 0,
    AQT_EINVAL = 1,     /* bad argument, bad call order, or size out of range */
    AQT_ECUDA = 2,      /* a CUDA runtime call failed (message names it) */
    AQT_ENOMEM = 3,     /* bound workspace smaller than aqt_workspace_size() */
    AQT_EOVERFLOW = 4,  /* jump log full: records were dropped (run completed) */
    AQT_ENUMERIC = 5,   /* non-finite or non-positive norm, or too many jumps in one half-step */
    AQT_ENOCONV = 6,    /* eigensolver did not converge */
    AQT_EDEGEN = 7,     /* degenerate structure outside what the GPU path supports */
    AQT_ENODEV = 8,     /* context has no device (created with device -1) */
    AQT_ETIMEOUT = 9,   /* a bounded wait inside the tensor-core kernel expired (about 2 s);
                           the kernel stopped early and freed its resources; outputs are invalid */
    AQT_WDT = 10        /* warning from aqt_build_tables: the tables are built and usable, but the
                           grid step is not well below (dt > 0.1 x) a term of the time-step
                           condition of Sec. IV, Eq. newcond, that applies to the jump timing
                           (aqt_get_dt_bounds gives the terms) */
} aqt_status;

/* Propagation precision. The host tables, the jump clock, the crossing time
 * (root of the norm condition of Sec. IV, Newton's method on the FP64 decay
 * sums formed from the state's populations) and the cumulative sums of both
 * channel draws (App. B.1, Eq. Pi(t)) are FP64 on every path; the state, its
 * no-jump propagation and the jump operator's application run in the state's
 * precision. The eigenvectors, from which a jump forms the column of
 * V^T sz_alpha V it needs, are held on the device in the state precision. */
typedef enum {
    AQT_PREC_FP64 = 0,      /* SIMT FP64 state and rotation */
    AQT_PREC_FP32 = 1,      /* SIMT FP32 state and rotation, FP64 norm sums */
    AQT_PREC_F16SPLIT = 2   /* tensor cores (tcgen05): rotation as O_hi C_hi + O_hi C_lo + O_lo C_hi
                               in FP16 with FP32 accumulation (22-bit mantissa), FP32 state;
                               N = 128 or 256 (n_qubits 7 or 8) */
} aqt_precision;

/* When a jump happens inside a frozen half-step (Sec. IV: the norm of the
 * unnormalised state falls to the threshold r at t + tau). The paper gives the
 * condition, not how finely tau is resolved. */
typedef enum {
    AQT_JUMP_REFINED = 0,   /* at the root of |psi(t)|^2 = r inside the half-step (FP64 Newton) */
    AQT_JUMP_GRID = 1,      /* at the end of the half-step in which |psi|^2 fell to r: the
                               time-step-resolution variant, with an O(dt) bias in the jump times */
    AQT_JUMP_FIXED_STEP = 2 /* the fixed-step unravelling of App. B.1: at the start of each half-step
                               (length tau) a jump happens with probability tau lambda, lambda =
                               sum_i <A_i^dag A_i> (Eq. lambda), its channel drawn by Eq. Pi(t), in
                               place of that half-step's no-jump evolution; O(dt) bias. Draws:
                               counter (trajectory, half-step index, 1, 0) -> (jump test, u1, u2).
                               SIMT paths only (AQT_PREC_FP64, AQT_PREC_FP32) */
} aqt_jump_timing;

/* One jump. t is the jump time in ns; the jump happened while the generator
 * was frozen at grid point `grid`, in the half-step before s_grid (half = 0)
 * or after it (half = 1). alpha is the qubit whose sz caused it; src and dst
 * are the lowest levels of the source and target degenerate manifolds
 * (instantaneous eigenbasis, ascending energy; a level inside a degenerate
 * manifold depends on the arbitrary eigenbasis, the manifold does not);
 * omega = E(src) - E(dst) is its Bohr frequency (rad/ns). */
typedef struct {
    int32_t traj, grid, half, alpha, src, dst;
    double t, omega;
} aqt_jump;

/* Create a context on CUDA device `device` (>= 0), or a host-only context
 * (device = -1) that can build and inspect tables but not run. *out is NULL
 * on failure. */
aqt_status aqt_create(aqt_ctx **out, int device);
void aqt_destroy(aqt_ctx *ctx);
const char *aqt_last_error(const aqt_ctx *ctx);

/* Ising terms of H_S (Sec. V, Eq. H_S, with the field sign written out):
 *   H(s) = A(s) (-sum_i sx_i) + B(s) (sum_i hz_i sz_i + sum_{i<j} Jzz_ij sz_i sz_j).
 * The paper's H^Z = -sum h sz + sum J sz sz maps to hz = -h.
 * n_qubits in [1, 16] (above 10 only with aqt_set_levels); hz[n]; Jzz[n*n]
 * row-major, entries with i < j used. */
aqt_status aqt_set_ising(aqt_ctx *ctx, int n_qubits, const double *hz, const double *Jzz);

/* Piecewise-linear annealing schedule through n_knots (s, A, B) points,
 * s strictly increasing from 0 to 1 (Sec. V, Eq. H_S; App. D). */
aqt_status aqt_set_schedule(aqt_ctx *ctx, int n_knots, const double *s, const double *A,
                            const double *B);

/* Ohmic bath of Sec. V: gamma(w) = 2 pi eta_g2 w e^{-|w|/omega_c} / (1 - e^{-beta w}),
 * independent sz coupling per qubit. lamb_shift = 1 adds
 * H_LS = sum S(w) L^dag L with S(w) = (1/2pi) P int gamma(x)/(w - x) dx (Sec. II; App. E). */
aqt_status aqt_set_bath(aqt_ctx *ctx, double eta_g2, double omega_c, double beta, int lamb_shift);

/* Truncated model: keep only the n_levels lowest instantaneous eigenstates of
 * H_S(s) at every grid point (0, the default, or 2^n keeps all). The paper
 * does not discuss truncation; its 16-qubit example (Sec. V.C) is where the
 * full space is too large. Reading: the system's Hilbert space at s is the
 * span of the kept eigenstates; the jump operators and the Lamb shift act
 * within it (P A P); the frame change between grid points is the n_levels x
 * n_levels block O = V_k^T V_{k-1}, which is not orthogonal: the weight it
 * moves out of the kept levels (the leakage) is renormalised away with the
 * rest of the rotation's norm change and never counted as jump probability
 * (aqt_get_rotation_error reports the largest one of a run). The eigenpairs
 * come from FP64 block Lanczos without forming H (2^n amplitudes per vector),
 * warm-started along the grid; the cut must fall between degenerate
 * manifolds at every grid point (at s = 0 of the transverse-field model the
 * multiplicities are C(n, k), so allowed cuts are 1, 1 + n, 1 + n + C(n,2),
 * ...), else aqt_build_tables returns AQT_EDEGEN. Device runs take
 * n_levels <= 512; every source level's jump amplitudes are tabled, so the
 * device needs no eigenvectors. */
aqt_status aqt_set_levels(aqt_ctx *ctx, int n_levels);

/* Shared time grid s_k = k/(n_grid-1), t_k = s_k t_f, n_grid >= 2. The generator
 * is frozen at s_{k-1} for the first half of [t_{k-1}, t_k] and at s_k for the
 * second (symmetric split; the paper leaves the integrator open, Sec. IV). */
aqt_status aqt_set_grid(aqt_ctx *ctx, double t_f, int n_grid);

/* M trajectories, all starting in the ground state of H_S(0) (Sec. V.A).
 * Random streams: Philox4x64-10, key (seed, 0x171003431), counter
 * (trajectory, event, 0, 0); event 0 gives the first threshold, event j the
 * draws of the j-th jump. jump_timing: aqt_jump_timing. jump_capacity =
 * records kept on the device. */
aqt_status aqt_set_trajectories(aqt_ctx *ctx, int64_t M, uint64_t seed, int precision, int jump_timing,
                                int64_t jump_capacity);

/* Device bytes the caller must provide for the current inputs. Device runs
 * take n_qubits <= 9 (N <= 512; the jump warp keeps N/32 levels per lane in
 * registers) and, for AQT_PREC_F16SPLIT, n_qubits 7 or 8; otherwise
 * AQT_EINVAL (host-only contexts build tables up to n_qubits = 10). The size depends on
 * the spectrum (full jump amplitudes are kept for the grid points with
 * degenerate levels or coinciding Bohr frequencies), so this call builds the
 * host tables of aqt_build_tables if they are not built yet, and can return
 * its errors (AQT_ENOCONV, AQT_EDEGEN). */
aqt_status aqt_workspace_size(aqt_ctx *ctx, size_t *bytes);

/* Bind caller-owned device memory (256-byte aligned, at least
 * aqt_workspace_size bytes). It must stay allocated until the context is
 * destroyed or rebound; the library never frees it. */
aqt_status aqt_bind_workspace(aqt_ctx *ctx, void *dptr, size_t bytes);

/* Build the FP64 per-grid-point tables (instantaneous eigensystems,
 * degenerate manifolds and Bohr classes per Eq. Lindblad2, the eigenframe
 * H_eff of Eq. Heff, rate tables, frame rotations) on the host, then copy
 * them into the workspace on `stream`. Blocks until the copies are done and
 * the host buffers may be reused. Errors: AQT_ENOCONV, AQT_EDEGEN, AQT_ECUDA;
 * warning (tables built and usable): AQT_WDT. On a host-only context the
 * tables are built and kept for aqt_debug_table. */
aqt_status aqt_build_tables(aqt_ctx *ctx, void *stream);

/* The three terms of the time-step condition of Sec. IV, Eq. newcond,
 *   dt << min_t { 2 |H_eff| / |dH_eff/dt|,  1 / |H_eff|,  |lambda / (lambda^2 - dlambda/dt)| },
 * each minimised over the grid: bounds[3] in ns, at[3] the grid points (at may
 * be NULL). |.| is the operator norm: |H_eff| = max |K_bb| exactly;
 * |dH_eff/dt| is an upper estimate (schedule derivative of H_S by the
 * triangle inequality plus the rate of change of the dissipative and
 * Lamb-shift diagonal), so the first term is a lower estimate; lambda is taken
 * per instantaneous eigenstate (lambda_b = -2 Im K_bb, levels whose jump
 * probability over the run exceeds 1e-6). aqt_build_tables returns AQT_WDT
 * when dt > 0.1 x the first term, or, with AQT_JUMP_GRID or
 * AQT_JUMP_FIXED_STEP, the third; the second bounds a first-order no-jump step
 * and does not apply to the exact frozen-generator phases used here. Needs the host tables (aqt_build_tables
 * or aqt_workspace_size). */
aqt_status aqt_get_dt_bounds(aqt_ctx *ctx, double *bounds, int32_t *at);

/* Propagate all trajectories over the whole grid (Sec. IV). Asynchronous on
 * `stream`; results are valid after aqt_sync. Each call restarts from the
 * initial state with the same random streams. */
aqt_status aqt_run(aqt_ctx *ctx, void *stream);

/* Failure injection for tests (the default needs no call): the poll limit of
 * the tensor-core kernel's bounded waits between its roles, 0 .. 2^22
 * (default 2^22; the waits also end after about 2 s). With 0 every such wait
 * expires at once: the kernel records AQT_ETIMEOUT with the waits' names,
 * issues no products, waits (with the default limits) for the copies it has
 * in flight, frees its tensor memory and ends; the context stays usable. */
aqt_status aqt_set_wait_limit(aqt_ctx *ctx, int64_t polls);

/* Wait for the last run and return its device status: AQT_OK, AQT_EOVERFLOW
 * (jump records dropped), AQT_ENUMERIC or AQT_ETIMEOUT. */
aqt_status aqt_sync(aqt_ctx *ctx);

/* Ground-manifold population at each grid point: mean[n_grid] and the
 * standard error of the mean stderr_[n_grid] (Eq. stderror). */
aqt_status aqt_get_observables(aqt_ctx *ctx, double *mean, double *stderr_);

/* Raw FP64 sums over trajectories, sum_x[n_grid] and sum_x2[n_grid]. */
aqt_status aqt_get_observable_sums(aqt_ctx *ctx, double *sum_x, double *sum_x2);

/* Mean and standard error of the mean (Sec. VI.A, Eq. stderror,
 * sigma^2 = sum (x - mean)^2 / (M (M - 1))) from raw sums over M trajectories:
 * the statistics of aqt_get_observables for sums merged across contexts or
 * ranks (trajectories sharded over several GPUs add their sums; the merge is
 * one sum of 2 n_grid doubles per rank). Host only; no context. */
aqt_status aqt_observables_from_sums(int n_grid, int64_t M, const double *sum_x, const double *sum_x2,
                                     double *mean, double *stderr_);

/* Per grid point g >= 1, the sum over trajectories of the frame rotation's
 * norm loss 1 - |O c|^2 into s_g (c normalised): with aqt_set_levels, the
 * leakage out of the kept levels at each step (divide by M for the mean);
 * otherwise the rotation's rounding (O is orthogonal). sum_leak[n_grid],
 * entry 0 is 0. */
aqt_status aqt_get_leakage(aqt_ctx *ctx, double *sum_leak);

/* Precision check of the frame rotation (its own arithmetic, as run): the
 * largest |(squared norm after a rotation c <- O c) / (before) - 1| over all
 * trajectories and grid steps of the last run. O is orthogonal, so this is
 * the rounding of the rotation (split products and FP32 sums on the
 * tensor-core path); the state is renormalised after every step. */
aqt_status aqt_get_rotation_error(aqt_ctx *ctx, double *max_rel);

/* Copy up to cap jump records, sorted by (traj, t), to host_buf.
 * *n_out = records copied, *n_dropped = records lost to a full device log. */
aqt_status aqt_get_jumps(aqt_ctx *ctx, aqt_jump *host_buf, int64_t cap, int64_t *n_out,
                         int64_t *n_dropped);

/* Final normalised states at s = 1 (re, im) FP64. basis 0: instantaneous
 * eigenbasis of H_S(1) (the library's eigenvector signs), host_buf[M][N][2]
 * with N the levels carried; basis 1: computational basis,
 * host_buf[M][2^n][2]. */
aqt_status aqt_get_final_state(aqt_ctx *ctx, int basis, double *host_buf);

/* Run without caller-provided scratch (the paper has no counterpart: this is
 * a deployment convenience). For callers that cannot allocate device memory
 * when they run -- code inside another framework's memory pool with a budget
 * fixed at start-up, or host threads where device allocation is not allowed.
 * It runs the same propagation as aqt_run on the context's device tables
 * (aqt_build_tables must have run on a bound workspace) and writes to the
 * caller's device outputs: obs_sums[n_grid][2] (sum of x, sum of x^2),
 * final_states[M][N][2] (eigenbasis, FP64), jumps[jump_capacity] (unsorted),
 * *jump_count (records produced, kept or not) and *status (0; bit 1 for a
 * numeric problem; bit 2 when a bounded wait of the tensor-core kernel
 * expired, with bits 8-13 naming the wait). The kernel's scratch -- per-CTA observable partials and
 * FP64 jump vectors -- comes from one 32 MiB array compiled into the library,
 * held on every GPU that loads the library until the process exits. No
 * device memory is allocated by this call.
 *  - The first call on each device looks up that array's device address
 *    (cudaGetSymbolAddress with the device current) and keeps it for that
 *    device's current context; a new context on the device (after
 *    cudaDeviceReset) is detected and the address looked up again. Make the
 *    first call on a device (and the first after a reset) before any stream
 *    capture.
 *  - A run that needs more than 32 MiB of scratch (it grows with
 *    M x n_grid and with M x N) returns AQT_EINVAL with the size in the message.
 *  - All calls on one device share the array and it keeps the last call's
 *    contents; calls whose kernels can overlap on the GPU race on it, so
 *    order them (one stream, or events).
 * Asynchronous on `stream`; *jump_count and *status are zeroed on the stream
 * before the kernel starts. */
aqt_status aqt_run_static_scratch(aqt_ctx *ctx, void *stream, double *obs_sums, double *final_states,
                                  aqt_jump *jumps, int64_t jump_capacity, unsigned long long *jump_count,
                                  int32_t *status);

/* ---- Batches: many instances in one launch ------------------------------------
 * Many independent annealing instances -- each its own context with its own
 * Hamiltonian, grid, trajectories and precision, sizes N = 2 .. 512 mixed --
 * propagated together: the trajectories of different instances are as
 * independent as those of one instance (Sec. VI.C), so a batch is a list of
 * work items (instance, tile of trajectories) that one persistent kernel per
 * kernel form takes from a queue, longest first. Forms: SIMT FP64, SIMT FP32
 * (any N) and tensor cores (AQT_PREC_F16SPLIT, N = 128 or 256; one launch per
 * N). One run is one CUDA graph launch (counters zeroed, the persistent
 * kernels, the observable reductions). Results are those of aqt_run on each
 * member: each member's outputs (observables, jumps, final states, status)
 * are read with that member's getters after aqt_batch_sync.
 *
 * Tile shapes come from an autotuner: per kernel form it times the candidate
 * shapes (SIMT: rotation rows per thread 2, 4, 8 with the trajectories per
 * tile that follow; tensor cores: the largest tile and half of it) on the
 * batch itself over its first 33 grid points, and keeps the fastest. The
 * choice is cached for the process per (device, form, instance sizes), so a
 * second batch of the same sizes is not timed again.
 *
 * Members: contexts on one device, each with its tables built on a bound
 * workspace (aqt_build_tables); a context belongs to at most one batch at a
 * time, and must not run on its own while the batch runs. Changing a member's
 * inputs or workspace makes aqt_batch_run return AQT_EINVAL (create a new
 * batch). The batch's own device memory (run parameters, work items,
 * per-tile observable partials, jump scratch of the persistent CTAs) is one
 * caller-owned workspace, as for a context. Not thread-safe. */
typedef struct aqt_batch aqt_batch;

/* members[n_members]: distinct contexts with device tables. Errors: AQT_EINVAL
 * (no member, repeated member, members on different devices, tables not on
 * the device), AQT_ECUDA. */
aqt_status aqt_batch_create(aqt_batch **out, aqt_ctx *const *members, int n_members);
void aqt_batch_destroy(aqt_batch *batch);
const char *aqt_batch_last_error(const aqt_batch *batch);
/* Device bytes of the batch's workspace (sized for every tuning candidate). */
aqt_status aqt_batch_workspace_size(aqt_batch *batch, size_t *bytes);
/* 256-byte-aligned caller-owned device memory of at least that size; it must
 * outlive the batch or be rebound. */
aqt_status aqt_batch_bind_workspace(aqt_batch *batch, void *dptr, size_t bytes);
/* Run the autotuner now (otherwise the first aqt_batch_run does). Blocking:
 * waits for `stream`, then times the candidates on an internal stream. The
 * tuning runs write into the members' outputs, which the next run replaces. */
aqt_status aqt_batch_tune(aqt_batch *batch, void *stream);
/* One run of every member (asynchronous on `stream` after the first call,
 * which tunes and builds the graph). Each call restarts every member from its
 * initial state with the same random streams. */
aqt_status aqt_batch_run(aqt_batch *batch, void *stream);
/* Wait for the run; member_status[n_members] (may be NULL) gets each member's
 * aqt_sync status. Returns AQT_OK, or the first member error (message names
 * the member). */
aqt_status aqt_batch_sync(aqt_batch *batch, int32_t *member_status);
/* Shape the last run used for member i: shape[4] = (form: 0 SIMT FP64, 1 SIMT
 * FP32, 2 tensor cores; trajectories per tile; rotation rows per thread
 * (SIMT) or 128-level blocks (tensor cores); tiles). */
aqt_status aqt_batch_get_shape(aqt_batch *batch, int member, int32_t *shape);

/* ---- Gradients (the paper has no derivatives; this extends its method) ----
 *
 * d<P>/dtheta of the trajectory average of the ground-manifold population of
 * H_S(1), <P>, for the parameters theta, in this order: A(s) at the schedule
 * knots, B(s) at the knots, hz_i (i = 0..n-1), Jzz_ij (i < j, row by row); there
 * are 2 n_knots + n + n (n - 1) / 2 of them (aqt_grad_n_params).
 *
 * Estimator: a trajectory's record (jump times and channels) has probability
 * density |psi~_T|^2, the squared norm of its unnormalised final state (the
 * waiting-time density of Sec. IV / App. C times the channel probability
 * Pi_i of App. B.1, Eq. Pi(t), is |A_i psi~|^2), so <P> is the integral over
 * records of <psi~_T|P|psi~_T> and, with the record held fixed,
 *   d<P>/dtheta = E[ dp/dtheta + (p - b) d log|psi~_T|^2 / dtheta ],
 * p the final population of the normalised state, b any constant (the
 * score d log|psi~_T|^2 has mean zero; b near <P> lowers the variance). The
 * first term is the pathwise derivative through the no-jump propagation
 * between jumps, the frame rotations and the jump operators at fixed jump
 * times; the second is the score of the waiting times and of the channel
 * choice. The device computes it by an adjoint sweep (backward through every
 * trajectory, recomputed segment by segment from checkpoints written by a
 * forward run every checkpoint_every grid points); the host (FP64) contracts
 * the adjoint's per-grid-point sums with the derivatives of the instantaneous
 * eigensystem (first-order perturbation theory), of gamma and S, and of the
 * jump operators.
 *
 * Scope: AQT_PREC_FP64 or AQT_PREC_FP32, AQT_JUMP_REFINED, every level kept
 * (no aqt_set_levels), at most 8 qubits; otherwise AQT_EINVAL. A parameter
 * whose dH_S/dtheta couples two levels of one degenerate manifold at some
 * grid point (at s = 0 of the transverse-field model: B at the first knot)
 * has no derivative in the secular AME (the Bohr classes of Eq. Lindblad2
 * regroup as the degeneracy lifts): its entry is NaN. */
aqt_status aqt_grad_n_params(aqt_ctx *ctx, int *n_params);  /* needs the inputs only (any context) */

/* Device bytes of a gradient run for the current inputs (a second workspace,
 * beside aqt_workspace_size's): checkpoints every checkpoint_every grid points
 * ([n_grid / checkpoint_every] x M x N states), one segment's states and
 * adjoints (4 x checkpoint_every x M x N), the per-grid-point sums
 * (n_grid x N x N FP64), 16 jump slots per trajectory for one segment and
 * room for jump_capacity jumps of the whole run (2 x N FP64 vectors each).
 * Builds the host tables if needed. */
aqt_status aqt_grad_workspace_size(aqt_ctx *ctx, int checkpoint_every, int64_t jump_capacity, size_t *bytes);

/* Bind caller-owned device memory (256-byte aligned, at least
 * aqt_grad_workspace_size bytes for the same checkpoint_every and
 * jump_capacity) for gradient runs. It must stay allocated while the context
 * uses it; the library never frees it. Changing any set_* input invalidates
 * it (aqt_grad_forward and aqt_grad_backward then return AQT_EINVAL). */
aqt_status aqt_grad_bind_workspace(aqt_ctx *ctx, int checkpoint_every, int64_t jump_capacity, void *dptr,
                                   size_t bytes);

/* Forward run with checkpoints: the same propagation as aqt_run (the
 * observables, jumps and final states are readable afterwards, and aqt_sync
 * waits for it), plus every trajectory's state every checkpoint_every grid
 * points. Asynchronous on `stream`. Tables must be built on the device
 * (aqt_build_tables). */
aqt_status aqt_grad_forward(aqt_ctx *ctx, void *stream);

/* Backward sweep after aqt_grad_forward, asynchronous on `stream` (the same
 * stream, or one ordered after it). baseline: the constant b of the
 * estimator; NaN takes the forward run's own mean of P at s = 1 (a bias of
 * order 1/M). */
aqt_status aqt_grad_backward(aqt_ctx *ctx, double baseline, void *stream);

/* Wait for the gradient run, then contract on the host: grad[n_params] gets
 * d<P>/dtheta (NaN where undefined, see above), *value (may be NULL) the run's
 * mean of P at s = 1. Errors: AQT_ENUMERIC; AQT_EOVERFLOW when a trajectory
 * jumped more than 16 times inside one checkpoint segment (use a smaller
 * checkpoint_every) or the run had more jumps than jump_capacity. */
aqt_status aqt_grad_get(aqt_ctx *ctx, double *grad, int n_params, double *value);

/* Table inspection (tests). N: the levels carried (aqt_set_levels), D = 2^n.
 * which: 0 eigenvalues [N]; 1 diag of H_eff,
 * [N][2] (re, im); 2 stage-one rates G[n][N]; 3 jump amplitudes
 * R_alpha[a][b] = sqrt(gamma(E_b - E_a)) <a|sz_alpha|b>, [n][N][N] (FP64,
 * formed from the eigenvectors on request); 4 frame rotation
 * O_g = V_{g+1}^T V_g [N][N] (g < n_grid-1); 5 eigenvectors V [D][N]
 * (column a = level a); 6 manifold energy per level [N]; 7 grid metadata [4]:
 * (some manifold degenerate, ground-manifold size, every Bohr class of
 * nonzero frequency is a single manifold pair, energy tolerance); 8 [2]:
 * (number of grid points that keep full jump amplitudes, bytes copied to the
 * device by the last aqt_build_tables; grid is ignored); 9 [2]: (truncated
 * model: the first eigenvalue above the kept levels at `grid`, the most
 * block-Lanczos restarts any grid point needed). */
aqt_status aqt_debug_table(aqt_ctx *ctx, int which, int grid, double *out);

#ifdef __cplusplus
}
#endif
#endif /* AQT_H */
