// Tensor-core propagation of AME quantum-jump trajectories (sm_103a, tcgen05).
//
// Same path as the SIMT kernel (arXiv:1710.03431, Sec. IV; eigenframe split of
// H_eff, Eq. Heff), for N a multiple of 128 levels. Per grid step g-1 -> g the
// frame rotation c <- O_{g-1} c of all TT trajectories of a CTA is one
// tensor-core product D[level][column] = O[level][b] C[b][column], columns =
// (trajectory, re/im) pairs, in split-FP16 form with FP32 accumulation:
//   O C ~ O_hi C_hi + O_hi C_lo + O_lo C_hi   (hi = fp16(x), lo = fp16(x - hi)),
// a 22-bit-mantissa product. Roles (one CTA per SM, persistent over the grid):
//   warp 0  streams O_hi/O_lo K-blocks (16 levels) into a 4-stage shared-memory
//           ring with bulk copies (cp.async.bulk, mbarrier transaction counts)
//           and warms L2 with its slice of the next step's rotation tile;
//   warp 1  owns the tensor memory and issues tcgen05.mma from one lane;
//   warps 2-13 are the epilogue (3 column groups x 4 TMEM lane quarters).
// Per step the epilogue (1) waits for the products D, (2) in one pass turns D
// into the next operand C = D E^2 / kappa_{g-1} (both frozen half-steps around
// s_g with their exact diagonal factors, normalisation deferred by one step)
// and releases it to the next rotation at once, then, while that rotation
// runs, (3) recomputes the per-trajectory norms and decay sums from the
// operand it wrote (cross-lane reductions), advances the FP64 jump clocks,
// finds crossings and records the observable. A trajectory whose clock
// crosses its threshold is resolved by one epilogue warp with the same
// register routine as the SIMT kernel (App. C; App. B.1, Eq. Pi(t);
// Eq. jump); since the rotation already ran on its old state, the epilogue
// computes the product of its new state (FP32 over the same FP16 hi/lo
// tiles) and writes it into tensor memory before the next pass (2). At the
// last grid point there is no next rotation and the sums come from D.
//
// Operand layouts (no swizzle, 8x16-byte core matrices):
//   A = O block [N rows][16 cols], K-major: core (r/8, k/8) at ((r/8)*2 + k/8)*128 B
//       (K-core stride 128 B, M-core stride 256 B); hi then lo (N*32 B each).
//   B = C [N levels][NC cols], MN-major: core (b/8, n/8) at ((b/8)*(NC/8) + n/8)*128 B
//       (N-core stride 128 B, K-core stride NC*16 B).
// Every wait on an mbarrier is bounded; on expiry the kernel records
// kStatusTimeout, stops issuing work, and still frees its tensor memory.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "aqt_internal.h"
#include "device_jump.cuh"
#include "philox.cuh"

namespace aqt {

namespace {

using namespace dev;

constexpr int kEpiWarps = 12;                       // 3 column groups x 4 TMEM lane quarters
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kTcThreads = 64 + kEpiThreads;
constexpr int kStages = 4;
// One ring stage: 128 rows (block h of the product) x 2 K-blocks of 16 levels
// of O, FP16 hi (two 4 KB blocks) then lo (two 4 KB blocks).
constexpr uint32_t kStageBytes = 16384;
constexpr int kSlots = kScratchSlots;
constexpr int kPassBatch = 1;  // pass 1: chunks of 8 product columns whose TMEM loads are in flight together
constexpr int kSumBatch = 3;   // partial-sum reductions interleaved
constexpr long long kWaitLimit = 1ll << 22;           // polls, and
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s: far above any legitimate wait (~1 ms)
// wait sites, reported as status bits 8.. next to kStatusTimeout
enum : int { kSiteSlot = 0, kSiteDrain, kSiteBReady, kSiteFull, kSiteDFull, kSiteAbort };

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait (poll count and wall time, since one try_wait may suspend the
// thread for a while): false, with the abort flag set and the site recorded,
// when the limit expires; false at once when another role has aborted. polls:
// the poll limit (the run's setting; 0 makes the wait expire without polling).
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag, int32_t *status, int site,
                          long long polls) {
    const unsigned long long t0 = global_ns();
    for (long long i = 0; i < polls; ++i) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if ((i & 255) == 255 && global_ns() - t0 > kWaitNs) break;
    }
    *abort_flag = 1;
    atomicOr(status, kStatusTimeout | (1 << (8 + site)));
    return false;
}

// Wait for work this thread itself put in flight (its bulk copies), also after
// an abort, with the fixed limits: false, with the site recorded, if it expires.
__device__ bool mbar_drain(uint32_t bar, uint32_t parity, int32_t *status, int site) {
    const unsigned long long t0 = global_ns();
    for (long long i = 0; i < kWaitLimit; ++i) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 255) == 255 && global_ns() - t0 > kWaitNs) break;
    }
    atomicOr(status, kStatusTimeout | (1 << (8 + site)));
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Fetch [src, src + bytes) into L2 (16-byte aligned, size a multiple of 16).
__device__ __forceinline__ void l2_prefetch(const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// The same product, A kept in the tensor core's collector buffer for the next
// product (fill) or taken from it and then released (lastuse): the next
// product with the same A does not read A from shared memory again.
__device__ __forceinline__ void umma_f16_afill(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_f16_alastuse(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                                  uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}


// Issue a 32-lane x 8-column TMEM load without waiting (tcgen05.wait::ld and
// reg_fence must follow before the values are used).
__device__ __forceinline__ void tmem_ld8_issue(uint32_t addr, uint32_t r[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(addr));
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// Keep uses of loaded registers after the wait (a data dependency on an asm
// that is ordered after tcgen05.wait::ld).
__device__ __forceinline__ void reg_fence(uint32_t r[8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i) asm volatile("" : "+r"(r[i]));
}

__device__ __forceinline__ void tmem_ld8(uint32_t addr, float v[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    reg_fence(r);
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Store two consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_st2(uint32_t addr, float x, float y) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(__float_as_uint(x)),
                 "r"(__float_as_uint(y))
                 : "memory");
}
// Store / load four consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_st4(uint32_t addr, const float v[4]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(__float_as_uint(v[0])),
                 "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3]))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld4_issue(uint32_t addr, uint32_t r[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory"); }

// Split x into (hi, lo) halves.
__device__ __forceinline__ void split_half(float x, __half &hi, __half &lo) {
    hi = __float2half_rn(x);
    lo = __float2half_rn(x - __half2float(hi));
}

struct TcShared {
    // per-trajectory state (TT entries each), carved from dynamic smem
    double *ell, *logr;
    float *x, *kinv, *P, *fscale;  // observable, 1/kappa of the stored operand, raw |D|^2, final-state scale
    int *nj, *flag, *list;
    int *plist, *pcount;  // trajectories whose product this step comes from the patch buffer
    float2 *cst;          // [N] one jumped state staged for its next-step product
    float *d2gs;          // [N] |exp(-i K_aa tau)|^2 at the current grid point for the ground-manifold levels
    float *red;  // [4][NC/8][16] partial sums per TMEM lane quarter
    int *count;
    volatile int *abort_flag;
    int *epi_ok;  // the epilogue's go/stop decision for the current wait, one writer
    uint32_t *tmem_base;
    uint64_t *bars;  // full[kStages], empty[kStages], dfull, rowsA, rowsB, b1lo
};

// Epilogue threads write the rows of B (levels a of this thread) for one
// chunk of 8 columns: (re, im) of 4 trajectories as FP16 hi/lo.
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo) {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

// The same split from a packed pair, with packed FP32x2 arithmetic (same
// roundings as split2).
__device__ __forceinline__ void split2p(float2 x, uint32_t &hi, uint32_t &lo) {
    const __half2 h = __float22half2_rn(x);
    const float2 hf = __half22float2(h);
    const __half2 l = __float22half2_rn(__ffma2_rn(hf, make_float2(-1.0f, -1.0f), x));
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

__device__ __forceinline__ void store_chunk(unsigned char *sB_hi, unsigned char *sB_lo, int NC, int a, int c,
                                            const float v[8]) {
    uint4 ph, pl;
    split2(v[0], v[1], ph.x, pl.x);
    split2(v[2], v[3], ph.y, pl.y);
    split2(v[4], v[5], ph.z, pl.z);
    split2(v[6], v[7], ph.w, pl.w);
    const size_t off = ((size_t)(a >> 3) * (NC >> 3) + c) * 128 + (a & 7) * 16;
    *reinterpret_cast<uint4 *>(sB_hi + off) = ph;
    *reinterpret_cast<uint4 *>(sB_lo + off) = pl;
}

// Write one trajectory's (re, im) at level a into B (2 of the 8 halves of a row chunk).
__device__ __forceinline__ void store_one(unsigned char *sB_hi, unsigned char *sB_lo, int NC, int a, int t,
                                          double re, double im) {
    const int n = 2 * t;
    const size_t off = ((size_t)(a >> 3) * (NC >> 3) + (n >> 3)) * 128 + (a & 7) * 16 + (n & 7) * 2;
    __half h0, l0, h1, l1;
    split_half((float)re, h0, l0);
    split_half((float)im, h1, l1);
    *reinterpret_cast<uint32_t *>(sB_hi + off) =
        (uint32_t)__half_as_ushort(h0) | ((uint32_t)__half_as_ushort(h1) << 16);
    *reinterpret_cast<uint32_t *>(sB_lo + off) =
        (uint32_t)__half_as_ushort(l0) | ((uint32_t)__half_as_ushort(l1) << 16);
}

// Reduce 16 per-lane values over the warp; afterwards the even lane 2*i
// (and its odd partner) holds the warp total of value index
// ((lane>>4)&1)*8 + ((lane>>3)&1)*4 + ((lane>>2)&1)*2 + ((lane>>1)&1).
__device__ __forceinline__ float reduce_scatter16(float v[16], int lane) {
#pragma unroll
    for (int o = 16, n = 16; o >= 2; o >>= 1, n >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < n / 2; ++i) {
            const float send = upper ? v[i] : v[i + n / 2];
            const float keep = upper ? v[i + n / 2] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// The same for B independent sets of 16 values, stage by stage (the shuffles
// of the B chains are independent and overlap).
template <int B>
__device__ __forceinline__ void reduce_scatter16_multi(float (&v)[B][16], int lane, float (&out)[B]) {
#pragma unroll
    for (int o = 16, n = 16; o >= 2; o >>= 1, n >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < n / 2; ++i)
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const float send = upper ? v[b][i] : v[b][i + n / 2];
                const float keep = upper ? v[b][i + n / 2] : v[b][i];
                v[b][i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
    }
#pragma unroll
    for (int b = 0; b < B; ++b) out[b] = v[b][0] + __shfl_xor_sync(0xffffffffu, v[b][0], 1);
}

__device__ __forceinline__ int scatter_index(int lane) {
    return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}

// Next-step product y = O c of one state staged in shared memory (cs[b] =
// (re, im), N levels), thread = level a of the product, with O from the FP16
// hi/lo tiles that the tensor cores use: the product the next rotation would
// have given, had it seen this state.
template <int MH>
__device__ __forceinline__ float2 rotate_row(const unsigned char *tile, const float2 *cs, int a) {
    constexpr int N = 128 * MH, NK = N / 16;
    float yr = 0.0f, yi = 0.0f;
    const int al = a & 127;
    const unsigned char *row = tile + (size_t)(a >> 7) * (NK / 2) * kStageBytes + (al >> 3) * 256 + (al & 7) * 16;
#pragma unroll 8
    for (int kh = 0; kh < 2 * NK; ++kh) {  // 8 levels b at a time: K-block kb = kh/2, core column kh%2
        const int kb = kh >> 1;
        const unsigned char *blk = row + (size_t)(kb >> 1) * kStageBytes + (kb & 1) * 4096 + (kh & 1) * 128;
        uint4 w[2];
        w[0] = *reinterpret_cast<const uint4 *>(blk);         // hi
        w[1] = *reinterpret_cast<const uint4 *>(blk + 8192);  // lo
        const __half2 *hh = reinterpret_cast<const __half2 *>(w);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 hi = __half22float2(hh[i]), lo = __half22float2(hh[4 + i]);
            const float2 c0 = cs[8 * kh + 2 * i], c1 = cs[8 * kh + 2 * i + 1];
            yr = fmaf(hi.x + lo.x, c0.x, yr);
            yi = fmaf(hi.x + lo.x, c0.y, yi);
            yr = fmaf(hi.y + lo.y, c1.x, yr);
            yi = fmaf(hi.y + lo.y, c1.y, yi);
        }
    }
    return make_float2(yr, yi);
}

// The whole run of tile `cta` of one instance (trajectories cta*TT .. cta*TT +
// TT - 1). kBatch = false: the CTA owns its tensor memory here (one tile per
// CTA). kBatch = true: the caller (a persistent CTA that runs tiles one after
// another) holds 512 tensor-memory columns at tmem_batch; each tile
// initialises its barriers and, at the end, makes sure every arrival on them
// has landed and invalidates them, so that the next tile can initialise them
// again. scr: this CTA's jump slots; patch: its next-step products of jumped
// trajectories ([TT][N] float2).
template <int MH, bool kBatch>  // 128-level blocks of the state (N = 128 MH)
__device__ __forceinline__ bool tc_tile(const RunParams &p, int cta, unsigned char *smem, uint32_t tmem_batch,
                                        double2 *scr, float2 *patch) {
    const int N = p.N, K = p.K, TT = p.TT, NC = 2 * TT, NK = N / 16, nchunk = NC / 8;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const size_t b_bytes = (size_t)N * NC * 2;
    unsigned char *sB_hi = smem;
    unsigned char *sB_lo = smem + b_bytes;
    unsigned char *sA = smem + 2 * b_bytes;
    const uint32_t stage_bytes = kStageBytes;
    unsigned char *misc = sA + (size_t)kStages * stage_bytes;
    TcShared S;
    S.bars = reinterpret_cast<uint64_t *>(misc);  // 2 kStages + 2 barriers (4 reserved)
    S.tmem_base = reinterpret_cast<uint32_t *>(misc + 8 * (2 * kStages + 4));
    S.abort_flag = reinterpret_cast<volatile int *>(misc + 8 * (2 * kStages + 4) + 4);
    S.count = reinterpret_cast<int *>(misc + 8 * (2 * kStages + 4) + 8);
    S.epi_ok = reinterpret_cast<int *>(misc + 8 * (2 * kStages + 4) + 12);
    S.ell = reinterpret_cast<double *>(misc + 8 * (2 * kStages + 4) + 16);
    S.logr = S.ell + TT;
    S.x = reinterpret_cast<float *>(S.logr + TT);
    S.kinv = S.x + TT;
    S.P = S.kinv + TT;
    S.fscale = S.P + TT;
    S.nj = reinterpret_cast<int *>(S.fscale + TT);
    S.flag = S.nj + TT;
    S.list = S.flag + TT;
    S.plist = S.list + TT;
    S.pcount = S.plist + TT;
    S.cst = reinterpret_cast<float2 *>(S.pcount + 4);
    S.d2gs = reinterpret_cast<float *>(S.cst + N);
    S.red = S.d2gs + N;

    const uint32_t bar_full = smem_u32(S.bars), bar_empty = bar_full + 8 * kStages;
    // rowsA / rowsB: the next operand's levels [0, N/2) / [N/2, N) are written and
    // the products of block h = 0 / h = 1 read
    const uint32_t bar_dfull = bar_full + 16 * kStages, bar_rowsA = bar_dfull + 8, bar_rowsB = bar_rowsA + 8;
    // b1lo: the products of block h = 1 no longer read the operand's first half
    // of levels (all products of block 0 are done too)
    const uint32_t bar_b1lo = bar_rowsB + 8;
    const int64_t t0 = (int64_t)cta * TT;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(bar_full + 8 * s, 1);
            mbar_init(bar_empty + 8 * s, 1);
        }
        mbar_init(bar_dfull, 1);
        mbar_init(bar_rowsA, kEpiThreads);
        mbar_init(bar_rowsB, kEpiThreads);
        mbar_init(bar_b1lo, 1);
        *S.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // products (MH * NC columns), then 12 columns of parked partial sums per chunk
    const uint32_t park = (uint32_t)(MH * NC);
    uint32_t ncols = 32;
    while (ncols < (uint32_t)(MH * NC + 12 * nchunk)) ncols <<= 1;
    if (!kBatch && warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(S.tmem_base)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = kBatch ? tmem_batch : *S.tmem_base;
    const unsigned char *otab = reinterpret_cast<const unsigned char *>(p.tab.OT);
    const size_t tile = (size_t)N * N * 4;  // one step's rotation: FP16 hi + lo

    if (warp == 0) {
        // ---------------- bulk-copy producer ----------------
        if (lane == 0) {
            // every CTA reads the same rotation tile in each step; each warms L2 with
            // its slice of the tile one step ahead, so the ring's copies hit L2
            const size_t piece = ((tile + p.n_cta - 1) / p.n_cta + 15) & ~(size_t)15;
            const size_t poff = (size_t)cta * piece;
            auto warm = [&](int tg) {
                if (tg < K - 1 && poff < tile)
                    l2_prefetch(otab + (size_t)tg * tile + poff, (uint32_t)(piece < tile - poff ? piece : tile - poff));
            };
            warm(0);
            long long it = 0;
            bool run = true;
            for (int g = 1; g < K && run && !*S.abort_flag; ++g) {
                warm(g);
                for (int s = 0; s < MH * NK / 2; ++s, ++it) {
                    const int slot = (int)(it % kStages);
                    if (it >= kStages && !mbar_wait(bar_empty + 8 * slot, (uint32_t)(((it / kStages) - 1) & 1),
                                                    S.abort_flag, p.status, kSiteSlot, p.wait_polls)) {
                        run = false;
                        break;
                    }
                    mbar_expect_tx(bar_full + 8 * slot, stage_bytes);
                    bulk_g2s(smem_u32(sA + (size_t)slot * stage_bytes), otab + (size_t)(g - 1) * tile + (size_t)s * stage_bytes,
                             stage_bytes, bar_full + 8 * slot);
                }
            }
            // drain: wait (bounded) for the copies still in flight, also after an
            // abort (the shared memory they write must outlive them)
            for (long long j = (it > kStages ? it - kStages : 0); j < it; ++j)
                if (!mbar_drain(bar_full + 8 * (int)(j % kStages), (uint32_t)((j / kStages) & 1), p.status, kSiteDrain))
                    break;
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        // Per step: block h = 0 of the products over K-blocks 0..NK-1, then h = 1,
        // two K-blocks per ring stage. K-blocks below NK/2 read the operand's
        // levels [0, N/2), written by the epilogue before rowsA; the rest need
        // rowsB. dfull tells the epilogue that all products are done.
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | (0u << 7) | (0u << 10) | (0u << 15) | (1u << 16) |
                                   ((uint32_t)(NC >> 3) << 17) | ((128u >> 4) << 24);
            const uint32_t a_lbo = 128, a_sbo = 256;
            const uint32_t b_lbo = (uint32_t)NC * 16, b_sbo = 128;
            const uint32_t bhi = smem_u32(sB_hi), blo = smem_u32(sB_lo);
            // ring slot 0 and K-block 0 of the operand: every other descriptor is
            // these plus (byte offset >> 4) in the address field (shared-memory
            // addresses < 256 KB keep the 14-bit field from overflowing)
            const uint64_t dA = umma_desc(smem_u32(sA), a_lbo, a_sbo);
            const uint64_t dBh = umma_desc(bhi, b_lbo, b_sbo), dBl = umma_desc(blo, b_lbo, b_sbo);
            long long it = 0;
            uint32_t last_bar = 0, last_par = 0;
            long long b1lo_commits = 0;
            bool run = true;
            for (int g = 1; g < K && run; ++g) {
                for (int h = 0; h < MH && run; ++h)
                    for (int kp = 0; kp < NK / 2; ++kp, ++it) {
                        if (h == 0 && (kp == 0 || kp == NK / 4)) {
                            if (!mbar_wait(kp == 0 ? bar_rowsA : bar_rowsB, (uint32_t)((g - 1) & 1), S.abort_flag,
                                           p.status, kSiteBReady, p.wait_polls)) {
                                run = false;
                                break;
                            }
                            fence_after();
                        }
                        const int slot = (int)(it % kStages);
                        if (!mbar_wait(bar_full + 8 * slot, (uint32_t)((it / kStages) & 1), S.abort_flag, p.status,
                                       kSiteFull, p.wait_polls)) {
                            run = false;
                            break;
                        }
                        fence_after();
                        const uint64_t a0 = dA + ((uint64_t)slot * stage_bytes >> 4);
                        const uint32_t d = tmem + (uint32_t)(h * NC);
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const int kb = 2 * kp + u;
                            const uint64_t ahi = a0 + (uint64_t)u * 256, alo = ahi + 512;  // +4096 B, +8192 B
                            const uint64_t bk = (uint64_t)kb * NC * 2;                    // kb * NC * 32 B
                            umma_f16_afill(d, ahi, dBh + bk, idesc, kb > 0 ? 1u : 0u);
                            umma_f16_alastuse(d, ahi, dBl + bk, idesc, 1u);
                            umma_f16(d, alo, dBh + bk, idesc, 1u);
                        }
                        umma_commit(bar_empty + 8 * slot);
                        last_bar = bar_empty + 8 * slot;
                        last_par = (uint32_t)((it / kStages) & 1);
                        if (MH == 2 && h == 1 && kp == NK / 4 - 1) {
                            umma_commit(bar_b1lo);
                            ++b1lo_commits;
                        }
                    }
                if (run) umma_commit(bar_dfull);
            }
            // between the tiles of a persistent CTA: every commit of the last ring
            // round and of b1lo has arrived before the barriers are invalidated
            if (kBatch) {
                for (long long j = (it > kStages ? it - kStages : 0); j < it; ++j)
                    if (!mbar_drain(bar_empty + 8 * (int)(j % kStages), (uint32_t)((j / kStages) & 1), p.status,
                                    kSiteAbort))
                        break;
                if (MH == 2 && b1lo_commits > 0)
                    mbar_drain(bar_b1lo, (uint32_t)((b1lo_commits - 1) & 1), p.status, kSiteAbort);
            }
            // on an abort, let the products already issued finish (bounded)
            // before the tensor memory is released
            if (!kBatch && *S.abort_flag && last_bar) {
                const unsigned long long ta = global_ns();
                for (long long i = 0; i < kWaitLimit; ++i) {
                    if (mbar_try(last_bar, last_par)) break;
                    if ((i & 255) == 255 && global_ns() - ta > kWaitNs) {
                        atomicOr(p.status, kStatusTimeout | (1 << (8 + kSiteAbort)));
                        break;
                    }
                }
            }
        }
    } else {
        // ---------------- epilogue (warps 2..13) ----------------
        const int etid = tid - 64, e = etid >> 5, q = warp & 3, ch = e >> 2;  // ch: column group 0..2
        const int c_begin = (ch * nchunk) / 3, c_end = ((ch + 1) * nchunk) / 3;
        // jump slots (scr): general-jump scratch (2N double2), then the FP32 state planes
        auto slot_re = [&](int sidx) { return reinterpret_cast<float *>(scr + ((size_t)sidx * kSlotDouble2 + 2) * N); };
        // next-step products of trajectories that jumped: patch[TT][N]
        const float4 *lvl = reinterpret_cast<const float4 *>(p.tab.tclvl);

        // ---- initial state e_0 and the half-step after s_0 ------------------------
        if (etid < TT) {
            const int t = etid;
            const bool active = t0 + t < p.M;
            S.nj[t] = 0;
            S.kinv[t] = 1.0f;
            S.x[t] = active ? 1.0f : 0.0f;
            if (active) {
                S.logr[t] = log(uniform01(traj_event(p.seed, t0 + t, 0).x[0]));
                const double l = log(p.tab.d2[0]);
                S.ell[t] = l;
                S.flag[t] = (l <= S.logr[t]) ? 1 : 0;
            } else {
                S.logr[t] = 0.0;
                S.ell[t] = 0.0;
                S.flag[t] = 2;
            }
        }
        if (etid == 0) {
            *S.count = 0;
            *S.pcount = 0;
        }
        epi_sync();
        if (etid < TT && S.flag[etid] == 1) S.list[atomicAdd(S.count, 1)] = etid;
        // B rows for all levels: level 0 holds exp(-i K_00 tau)/|.| for non-crossed
        {
            const double er = p.tab.ehalf[0], ei = p.tab.ehalf[1];
            const double nrm = sqrt(er * er + ei * ei);
            for (int h = 0; h < MH; ++h) {
                const int a = 128 * h + 32 * q + lane;
                for (int c = c_begin; c < c_end; ++c) {
                    float v[8];
                    for (int j = 0; j < 4; ++j) {
                        const int t = 4 * c + j;
                        const bool keep = a == 0 && S.flag[t] == 0;
                        v[2 * j] = keep ? (float)(er / nrm) : 0.0f;
                        v[2 * j + 1] = keep ? (float)(ei / nrm) : 0.0f;
                    }
                    store_chunk(sB_hi, sB_lo, NC, a, c, v);
                }
            }
        }
        epi_sync();
        // crossed at the first half-step: warp resolution from e_0
        for (int base = 0; base < *S.count; base += kSlots) {
            const int nr = min(kSlots, *S.count - base);
            for (int sidx = 0; sidx < nr; ++sidx)
                for (int h = 0; h < MH; ++h) {
                    const int a = 128 * h + 32 * q + lane;
                    if (ch == 0) {
                        slot_re(sidx)[a] = a == 0 ? 1.0f : 0.0f;
                        slot_re(sidx)[N + a] = 0.0f;
                    }
                }
            epi_sync();
            if (e < nr) {
                const int t = S.list[base + e];
                double el = 0.0, lr = S.logr[t];
                int nj = S.nj[t];
                float *sre = slot_re(e);
                jump_half_step<float, 4 * MH>(p, 0, 1, t0 + t, sre, sre + N, 1, el, lr, nj, lane,
                                              scr + (size_t)e * kSlotDouble2 * N);
                if (lane == 0) {
                    S.ell[t] = el;
                    S.logr[t] = lr;
                    S.nj[t] = nj;
                }
            }
            epi_sync();
            for (int sidx = 0; sidx < nr; ++sidx) {
                const int t = S.list[base + sidx];
                for (int h = 0; h < MH; ++h) {
                    const int a = 128 * h + 32 * q + lane;
                    if (ch == 0) {
                        const float *sre = slot_re(sidx);
                        store_one(sB_hi, sB_lo, NC, a, t, sre[a], sre[N + a]);
                    }
                }
            }
            epi_sync();
        }
        // observable at s_0 (every active trajectory is in the ground state)
        if (e == 0) {
            double sx = 0.0, sx2 = 0.0;
            for (int t = lane; t < TT; t += 32) {
                const double x = S.x[t];
                sx += x;
                sx2 += x * x;
            }
            warp_sum2(sx, sx2);
            if (lane == 0) {
                p.obs_part[((size_t)cta * K) * 3] = sx;
                p.obs_part[((size_t)cta * K) * 3 + 1] = sx2;
                p.obs_part[((size_t)cta * K) * 3 + 2] = 0.0;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        fence_before();
        mbar_arrive(bar_rowsA);
        mbar_arrive(bar_rowsB);

        // per-level factors of the next grid point, loaded one step ahead
        float4 Lnext[MH];
        int gs_next = 1;
        if (K > 1) {
#pragma unroll
            for (int h = 0; h < MH; ++h) Lnext[h] = lvl[(size_t)1 * N + 128 * h + 32 * q + lane];
            gs_next = p.tab.meta[1].gs_size;
        }
        float nerr = 0.0f;  // this thread's trajectory: largest relative norm change of a rotation
        for (int g = 1; g < K; ++g) {
            const bool last = g == K - 1;
            const int gs = gs_next;
            float4 L[MH];
#pragma unroll
            for (int h = 0; h < MH; ++h) L[h] = Lnext[h];
            if (g + 1 < K) {
#pragma unroll
                for (int h = 0; h < MH; ++h) Lnext[h] = lvl[(size_t)(g + 1) * N + 128 * h + 32 * q + lane];
                gs_next = p.tab.meta[g + 1].gs_size;
            }
            // exp(-i K tau) squared: both half-steps at s_g (one at the last grid point)
            float e2r[MH], e2i[MH];
#pragma unroll
            for (int h = 0; h < MH; ++h) {
                e2r[h] = last ? L[h].x : L[h].x * L[h].x - L[h].y * L[h].y;
                e2i[h] = last ? L[h].y : 2.f * L[h].x * L[h].y;
                // the ground-manifold levels' decay factors for the observable below
                // (read after the barriers of pass 1; the previous step's reads are done)
                const int a = 128 * h + 32 * q + lane;
                if (ch == 0 && a < gs) S.d2gs[a] = L[h].w;
            }
            // ---- single pass: per-trajectory sums over levels, and the next operand ----
            // D = kappa_{g-1} O c_{g-1}; the operand written now is D E^2 / kappa_{g-1}
            // = (O c) E^2, whose norm is restored to 1 through kappa_g next step. The
            // operand is released to the next step's products before this step's jump
            // decisions are known; a trajectory that jumps gets its next product from
            // the patch buffer.
            // Phases: with two blocks of levels, block 0 of the products is complete and
            // the running rotation has stopped reading the operand's first half at b1lo,
            // so pass 1 of block 0 overlaps the rest of the rotation; block 1 follows
            // dfull. One phase at the last grid point and for a single block.
            bool stop = false;
            const int nph = (last || MH == 1) ? 1 : MH;
            for (int ph = 0; ph < nph && !stop; ++ph) {
                // one thread waits; all epilogue threads then take the same decision
                // (a bounded wait can expire for one thread only)
                if (etid == 0)
                    *S.epi_ok = mbar_wait(nph == 2 && ph == 0 ? bar_b1lo : bar_dfull, (uint32_t)((g - 1) & 1),
                                          S.abort_flag, p.status, kSiteDFull, p.wait_polls) ? 1 : 0;
                epi_sync();
                if (!*S.epi_ok) {
                    stop = true;
                    break;
                }
                fence_after();
                const int hlo = nph == 2 ? ph : 0, hhi = nph == 2 ? ph + 1 : MH;
                // trajectories that jumped last step: their products come from the patch buffer
                if (*S.pcount > 0) {
                    if (ch == 0) {
                        for (int i = 0; i < *S.pcount; ++i) {
                            const int t = S.plist[i];
                            for (int h = hlo; h < hhi; ++h) {
                                const float2 y = patch[(size_t)t * N + 128 * h + 32 * q + lane];
                                tmem_st2(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(h * NC + 2 * t), y.x, y.y);
                            }
                        }
                        tmem_st_wait();
                    }
                    fence_before();
                    epi_sync();
                    fence_after();
                    if (ph == nph - 1 && etid == 0) *S.pcount = 0;
                }
                if (last) {
                    auto process = [&](int c, uint32_t (&r)[MH][8]) {
                        float ki[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) ki[j] = S.kinv[4 * c + j];
                        float v16[16];
#pragma unroll
                        for (int i = 0; i < 16; ++i) v16[i] = 0.0f;
#pragma unroll
                        for (int h = 0; h < MH; ++h) {
                            const int a = 128 * h + 32 * q + lane;
                            const float w = L[h].z, d2 = L[h].w;
                            const bool in_gs = a < gs;
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const float re = __uint_as_float(r[h][2 * j]), im = __uint_as_float(r[h][2 * j + 1]);
                                // |D|^2 kinv^2: the scale the sums have at the other grid points
                                const float qv = fmaf(re, re, im * im) * ki[j] * ki[j];
                                v16[j] += qv;
                                v16[4 + j] = fmaf(qv, w, v16[4 + j]);
                                if (in_gs) v16[12 + j] = fmaf(qv, d2, v16[12 + j]);
                            }
                        }
                        const float tot = reduce_scatter16(v16, lane);
                        if ((lane & 1) == 0) S.red[((size_t)q * nchunk + c) * 16 + scatter_index(lane)] = tot;
                    };
                    for (int c = c_begin; c < c_end; ++c) {
                        uint32_t r[MH][8];
#pragma unroll
                        for (int h = 0; h < MH; ++h)
                            tmem_ld8_issue(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(h * NC + 8 * c), r[h]);
                        tmem_wait();
#pragma unroll
                        for (int h = 0; h < MH; ++h) reg_fence(r[h]);
                        process(c, r);
                    }
                } else {
                    // pass 1 of this phase's blocks of 128 levels: the operand rows of this
                    // thread's level. The TMEM loads of kPassBatch chunks (products, and for
                    // block 1 the partial sums parked by block 0) are in flight together and
                    // waited for once.
#pragma unroll
                    for (int h = 0; h < MH; ++h) {
                        if (h < hlo || h >= hhi) continue;
                        const float2 e2 = make_float2(e2r[h], e2i[h]);
                        const float w = L[h].z, d2w = L[h].w * L[h].z;
                        const int a = 128 * h + 32 * q + lane;
                        const uint32_t lbase = tmem + ((uint32_t)(32 * q) << 16);
                        for (int c0 = c_begin; c0 < c_end; c0 += kPassBatch) {
                            const int nb = min(kPassBatch, c_end - c0);  // warp-uniform
                            uint32_t r[kPassBatch][8], o[kPassBatch][12];
#pragma unroll
                            for (int cc = 0; cc < kPassBatch; ++cc)
                                if (cc < nb) {
                                    tmem_ld8_issue(lbase + (uint32_t)(h * NC + 8 * (c0 + cc)), r[cc]);
                                    if (h > 0) {
                                        const uint32_t pa = lbase + park + 12u * (uint32_t)(c0 + cc);
                                        tmem_ld4_issue(pa, o[cc]);
                                        tmem_ld4_issue(pa + 4, o[cc] + 4);
                                        tmem_ld4_issue(pa + 8, o[cc] + 8);
                                    }
                                }
                            tmem_wait();
#pragma unroll
                            for (int cc = 0; cc < kPassBatch; ++cc) {
                                if (cc >= nb) continue;
                                reg_fence(r[cc]);
                                const int c = c0 + cc;
                                // v = D E^2 kinv per trajectory in packed FP32x2 arithmetic (the
                                // same roundings as the scalar form), split into FP16 hi / lo
                                const float4 k4 = *reinterpret_cast<const float4 *>(S.kinv + 4 * c);
                                const float kj[4] = {k4.x, k4.y, k4.z, k4.w};
                                uint32_t ph[4], pl[4];
                                float ps[12];  // this level's share of sum |D|^2 kinv^2 (1, w, d2 w)
#pragma unroll
                                for (int j = 0; j < 4; ++j) {
                                    const float re = __uint_as_float(r[cc][2 * j]), im = __uint_as_float(r[cc][2 * j + 1]);
                                    const float2 f = __fmul2_rn(e2, make_float2(kj[j], kj[j]));  // (fr, fi)
                                    const float2 v = __ffma2_rn(make_float2(re, re), f,
                                                                __fmul2_rn(make_float2(im, im), make_float2(-f.y, f.x)));
                                    split2p(v, ph[j], pl[j]);
                                    const float qv = fmaf(re, re, im * im) * (kj[j] * kj[j]);
                                    ps[j] = qv;
                                    ps[4 + j] = qv * w;
                                    ps[8 + j] = qv * d2w;
                                }
                                // park the partial sums in spare TMEM columns (the block-1 pass adds
                                // its share to block 0's); the warp reductions run beside the next
                                // rotation
                                if (h > 0) {
#pragma unroll
                                    for (int i = 0; i < 12; ++i) {
                                        asm volatile("" : "+r"(o[cc][i]));
                                        ps[i] += __uint_as_float(o[cc][i]);
                                    }
                                }
                                const uint32_t pa = lbase + park + 12u * (uint32_t)c;
                                tmem_st4(pa, ps);
                                tmem_st4(pa + 4, ps + 4);
                                tmem_st4(pa + 8, ps + 8);
                                const size_t off = ((size_t)(a >> 3) * (NC >> 3) + c) * 128 + (a & 7) * 16;
                                *reinterpret_cast<uint4 *>(sB_hi + off) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
                                *reinterpret_cast<uint4 *>(sB_lo + off) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
                            }
                        }
                    }
                }
                // this phase's operand rows are written and its products read
                if (!last) tmem_st_wait();
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                fence_before();
                if (nph == 1) {
                    mbar_arrive(bar_rowsA);
                    mbar_arrive(bar_rowsB);
                } else {
                    mbar_arrive(ph == 0 ? bar_rowsA : bar_rowsB);
                }
            }
            if (stop) break;
            // ---- warp reductions of the partial sums parked by pass 1, while the next
            // rotation runs (its products use other TMEM columns) ------------------------
            if (!last) {
                // kSumBatch chunks at a time: their TMEM loads in flight together, then
                // their reductions interleaved (independent shuffle chains)
                for (int c0 = c_begin; c0 < c_end; c0 += kSumBatch) {
                    const int nb = min(kSumBatch, c_end - c0);  // warp-uniform
                    uint32_t o[kSumBatch][12];
#pragma unroll
                    for (int cc = 0; cc < kSumBatch; ++cc) {
                        if (cc < nb) {
                            const uint32_t pa = tmem + ((uint32_t)(32 * q) << 16) + park + 12u * (uint32_t)(c0 + cc);
                            tmem_ld4_issue(pa, o[cc]);
                            tmem_ld4_issue(pa + 4, o[cc] + 4);
                            tmem_ld4_issue(pa + 8, o[cc] + 8);
                        } else {
#pragma unroll
                            for (int i = 0; i < 12; ++i) o[cc][i] = 0u;
                        }
                    }
                    tmem_wait();
                    float v[kSumBatch][16];
#pragma unroll
                    for (int cc = 0; cc < kSumBatch; ++cc) {
#pragma unroll
                        for (int i = 0; i < 12; ++i) {
                            asm volatile("" : "+r"(o[cc][i]));
                            v[cc][i] = __uint_as_float(o[cc][i]);
                        }
#pragma unroll
                        for (int i = 12; i < 16; ++i) v[cc][i] = 0.0f;
                    }
                    float tot[kSumBatch];
                    reduce_scatter16_multi<kSumBatch>(v, lane, tot);
#pragma unroll
                    for (int cc = 0; cc < kSumBatch; ++cc)
                        if (cc < nb && (lane & 1) == 0)
                            S.red[((size_t)q * nchunk + c0 + cc) * 16 + scatter_index(lane)] = tot[cc];
                }
            }
            if (etid == 0) *S.count = 0;
            epi_sync();
            // ---- per trajectory: clock, crossings, next kappa, observable -------------------
            if (etid < TT) {
                const int t = etid, c = t >> 2, j = t & 3;
                if (S.flag[t] != 2) {
                    float Pt = 0.f, Db = 0.f, Da = 0.f, X = 0.f;
                    for (int qq = 0; qq < 4; ++qq) {
                        const float *rr = S.red + ((size_t)qq * nchunk + c) * 16;
                        Pt += rr[j];
                        Db += rr[4 + j];
                        Da += rr[8 + j];
                        X += rr[12 + j];
                    }
                    if (!last) {
                        // ground-manifold weight sum_{a < gs} |D_a|^2 kinv^2 d2_a = sum |B_a|^2 / d2_a,
                        // from the few operand rows it needs
                        X = 0.f;
                        for (int a = 0; a < gs; ++a) {
                            const size_t off = ((size_t)(a >> 3) * (NC >> 3) + c) * 128 + (a & 7) * 16 + j * 4;
                            const __half2 bh = *reinterpret_cast<const __half2 *>(sB_hi + off);
                            const __half2 bl = *reinterpret_cast<const __half2 *>(sB_lo + off);
                            const float br = __low2float(bh) + __low2float(bl), bi = __high2float(bh) + __high2float(bl);
                            X += fmaf(br, br, bi * bi) / S.d2gs[a];
                        }
                    }
                    S.P[t] = Pt;
                    // Pt = |O c|^2 for the normalised c the rotation read (kinv carries
                    // the deferred normalisation), so Pt - 1 is the rotation's own
                    // relative norm error (split products, FP32 sums)
                    nerr = fmaxf(nerr, fabsf(Pt - 1.0f));
                    const float nB = Pt - Db;
                    const float dB = Db / Pt;
                    const double lB = S.ell[t] + (double)log1pf(-dB);
                    bool cross = lB <= S.logr[t];
                    float dA = 0.f;
                    double lA = lB;
                    if (!cross && !last) {
                        dA = Da / nB;
                        lA = lB + (double)log1pf(-dA);
                        cross = lA <= S.logr[t];
                    }
                    if (!(Pt > 0.f) || !isfinite(Pt)) {
                        atomicOr(p.status, kStatusNumeric);
                        cross = false;
                    }
                    if (!cross) {
                        S.flag[t] = 0;
                        S.ell[t] = last ? lB : lA;
                        S.x[t] = X / nB;
                        // kappa_g^2 = |O c|^2 (1 - dB)(1 - dA) with |O c|^2 = P (the sums are of
                        // |D|^2 kinv_{g-1}^2)
                        const float ko = S.kinv[t];
                        S.kinv[t] = rsqrtf(Pt * (1.0f - dB) * (1.0f - dA));
                        // final-state scale at the last grid point: 1/|D E| = kinv_{g-1} / sqrt(nB)
                        S.fscale[t] = ko * rsqrtf(nB);
                    } else {
                        S.flag[t] = 1;
                        S.list[atomicAdd(S.count, 1)] = t;
                    }
                }
            }
            epi_sync();
            // ---- last grid point: normalised final states ----------------------------------------
            if (last) {
                for (int c = c_begin; c < c_end; ++c)
                    for (int h = 0; h < MH; ++h) {
                        float d[8];
                        tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(h * NC + 8 * c), d);
                        const int a = 128 * h + 32 * q + lane;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int t = 4 * c + j;
                            if (S.flag[t] != 0) continue;
                            const float re = d[2 * j], im = d[2 * j + 1];
                            const float sc = S.fscale[t];
                            double *fs = p.final_state + ((size_t)(t0 + t) * N + a) * 2;
                            fs[0] = (re * e2r[h] - im * e2i[h]) * sc;
                            fs[1] = (re * e2i[h] + im * e2r[h]) * sc;
                        }
                    }
            }
            // ---- crossed trajectories: warp resolution of both half-steps ---------------------
            const int ncross = *S.count;
            for (int base = 0; base < ncross; base += kSlots) {
                const int nr = min(kSlots, ncross - base);
                // the diagonal of K at s_g for the resolving warps (both half-steps)
                if (etid < N) {
                    const double *kd = p.tab.kdiag + (size_t)g * N * 2;
                    S.cst[etid] = make_float2((float)kd[2 * etid], (float)(2.0 * kd[2 * etid + 1]));
                }
                if (ch == 0) {
                    // the state after the rotation of this step, normalised later: from the
                    // products (last step) or from the operand written above, D = B / E^2
                    for (int sidx = 0; sidx < nr; ++sidx) {
                        const int t = S.list[base + sidx];
                        const int c = t >> 2, j = t & 3;
                        for (int h = 0; h < MH; ++h) {
                            const int a = 128 * h + 32 * q + lane;
                            float re, im;
                            if (last) {
                                float d[8];
                                tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(h * NC + 8 * c), d);
                                re = d[2 * j];
                                im = d[2 * j + 1];
                            } else {
                                const size_t off = ((size_t)(a >> 3) * (NC >> 3) + c) * 128 + (a & 7) * 16 + j * 4;
                                const __half2 bh = *reinterpret_cast<const __half2 *>(sB_hi + off);
                                const __half2 bl = *reinterpret_cast<const __half2 *>(sB_lo + off);
                                const float br = __low2float(bh) + __low2float(bl);
                                const float bi = __high2float(bh) + __high2float(bl);
                                const float m = 1.0f / (e2r[h] * e2r[h] + e2i[h] * e2i[h]);
                                re = (br * e2r[h] + bi * e2i[h]) * m;
                                im = (bi * e2r[h] - br * e2i[h]) * m;
                            }
                            slot_re(sidx)[a] = re;
                            slot_re(sidx)[N + a] = im;
                        }
                    }
                }
                epi_sync();
                if (e < nr) {
                    const int t = S.list[base + e];
                    double el = S.ell[t], lr = S.logr[t];
                    int nj = S.nj[t];
                    float *sre = slot_re(e);
                    double2 *slow = scr + (size_t)e * kSlotDouble2 * N;
                    double xs = 0.0;
                    // both half-steps through one copy of the jump routine: the routine
                    // runs rarely, so its instructions are usually not in the
                    // instruction cache; a second inlined copy for the second half-step
                    // would miss again (a probe measured ~30 us per call either way)
#pragma unroll 1
                    for (int hf = 0; hf < (last ? 1 : 2); ++hf) {
                        jump_half_step<float, 4 * MH>(p, g, hf, t0 + t, sre, sre + N, 1, el, lr, nj, lane, slow,
                                                      S.cst);
                        if (hf == 0) {
                            for (int a = lane; a < gs; a += 32)
                                xs += (double)sre[a] * sre[a] + (double)sre[N + a] * sre[N + a];
                            xs = warp_sum(xs);
                        }
                    }
                    if (lane == 0) {
                        S.ell[t] = el;
                        S.logr[t] = lr;
                        S.nj[t] = nj;
                        S.x[t] = (float)xs;
                        S.kinv[t] = 1.0f;
                        if (!last) S.plist[atomicAdd(S.pcount, 1)] = t;
                    }
                }
                epi_sync();
                // next step's products of the new states (the rotation already ran on the old ones)
                for (int sidx = 0; sidx < nr && !last; ++sidx) {
                    if (etid < N) S.cst[etid] = make_float2(slot_re(sidx)[etid], slot_re(sidx)[N + etid]);
                    epi_sync();
                    if (etid < N)
                        patch[(size_t)S.list[base + sidx] * N + etid] = rotate_row<MH>(otab + (size_t)g * tile, S.cst, etid);
                    epi_sync();
                }
                for (int sidx = 0; sidx < nr && ch == 0 && last; ++sidx) {
                    const int t = S.list[base + sidx];
                    for (int h = 0; h < MH; ++h) {
                        const int a = 128 * h + 32 * q + lane;
                        double *fs = p.final_state + ((size_t)(t0 + t) * N + a) * 2;
                        fs[0] = slot_re(sidx)[a];
                        fs[1] = slot_re(sidx)[N + a];
                    }
                }
                epi_sync();
            }
            // ---- observable partials (fixed order) -----------------------------------------
            if (e == 0) {
                // per-CTA partials in FP64 (the per-trajectory values are FP32),
                // with the rotation's norm loss 1 - P
                double sx = 0.0, sx2 = 0.0, sl = 0.0;
                for (int t = lane; t < TT; t += 32) {
                    if (S.flag[t] == 2) continue;
                    const double x = S.x[t];
                    sx += x;
                    sx2 += x * x;
                    sl += 1.0 - (double)S.P[t];
                }
                warp_sum2(sx, sx2);
                sl = warp_sum(sl);
                if (lane == 0) {
                    p.obs_part[((size_t)cta * K + g) * 3] = sx;
                    p.obs_part[((size_t)cta * K + g) * 3 + 1] = sx2;
                    p.obs_part[((size_t)cta * K + g) * 3 + 2] = sl;
                }
            }
        }
        if (p.norm_err && etid < TT && t0 + etid < p.M) atomicMax(p.norm_err, __float_as_uint(nerr));
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (!kBatch && warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
    const bool completed = *S.abort_flag == 0;
    if (kBatch && tid == 0 && completed) {
        // every arrival has landed (the roles waited for their last phases above)
        for (int i = 0; i < 2 * kStages + 4; ++i)
            asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar_full + 8 * i) : "memory");
    }
    return completed;
}

// One CTA per tile of one instance.
template <int MH>
__global__ void __launch_bounds__(kTcThreads, 1) propagate_tc(const __grid_constant__ RunParams p) {
    extern __shared__ __align__(1024) unsigned char smem[];
    double2 *scr = reinterpret_cast<double2 *>(p.scratch) + (size_t)blockIdx.x * kSlots * kSlotDouble2 * p.N;
    float2 *patch = reinterpret_cast<float2 *>(reinterpret_cast<double2 *>(p.scratch) +
                                               (size_t)p.n_cta * kSlots * kSlotDouble2 * p.N) +
                    (size_t)blockIdx.x * p.TT * p.N;
    tc_tile<MH, false>(p, blockIdx.x, smem, 0u, scr, patch);
}

// Persistent kernel over the work items of many instances with the same N
// (one CTA per SM): the CTA holds 512 tensor-memory columns for its whole
// life and runs the tiles it takes from the queue one after another. Its own
// scratch block (scr_stride double2): the jump slots, then the patch buffer
// of the largest tile. tail: byte offset of three words past the largest
// tile's shared memory (item index, tensor-memory base, and the run
// parameters after them).
template <int MH>
__global__ void __launch_bounds__(kTcThreads, 1)
    propagate_tc_batch(const RunParams *ps, const BatchItem *items, int n_items, int *queue, double2 *scratch,
                       size_t scr_stride, uint32_t tail) {
    extern __shared__ __align__(1024) unsigned char smem[];
    int *s_item = reinterpret_cast<int *>(smem + tail);
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + tail + 16);
    RunParams *sp = reinterpret_cast<RunParams *>(smem + tail + 64);
    const int warp = threadIdx.x >> 5;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *s_tmem;
    double2 *scr = scratch + (size_t)blockIdx.x * scr_stride;
    for (;;) {
        __syncthreads();  // the previous tile is done with the shared memory
        if (threadIdx.x == 0) {
            *s_item = atomicAdd(queue, 1);
            if (*s_item < n_items) *sp = ps[items[*s_item].inst];
        }
        __syncthreads();
        const int it = *s_item;
        if (it >= n_items) break;
        float2 *patch = reinterpret_cast<float2 *>(scr + (size_t)kSlots * kSlotDouble2 * sp->N);
        // after an abort (a bounded wait expired; the instance reports
        // AQT_ETIMEOUT) commits may still be landing on this tile's barriers, so
        // the CTA takes no further tile
        if (!tc_tile<MH, true>(*sp, items[it].cta, smem, tmem, scr, patch)) break;
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

}  // namespace

size_t tc_smem_bytes(int N, int TT) {
    const int NC = 2 * TT, nchunk = NC / 8;
    size_t b = 2 * (size_t)N * NC * 2 + (size_t)kStages * kStageBytes;
    b += 8 * (2 * kStages + 4) + 16 + (size_t)TT * (8 * 2 + 4 * 4 + 4 * 4) + 16 +
         (size_t)4 * nchunk * 16 * 4 + (size_t)N * 8 + (size_t)N * 4;
    b = (b + 1023) & ~(size_t)1023;
    // one CTA per SM: the kernel allocates tensor-memory columns without sharing
    return b < 120 * 1024 ? 120 * 1024 : b;
}

// Trajectories per CTA: a multiple of 8 (columns in chunks of 16) so that the
// grid fills the SMs once, within shared memory and 256 tensor-core columns.
int tc_shape(int N, int64_t M, int num_sms) {
    int tt = (int)((M + num_sms - 1) / num_sms);
    tt = (tt + 7) & ~7;
    if (tt < 8) tt = 8;
    // shared memory, and tensor-memory columns: products plus parked sums (12 per 8 columns)
    while (tt > 8 && (tc_smem_bytes(N, tt) > 227 * 1024 || 2 * tt * (N / 128) + 3 * tt > 512 || 2 * tt > 256)) tt -= 8;
    return tt;
}

// Scratch of one persistent CTA of a batch (double2): jump slots and the
// patch buffer of the largest tile.
size_t tc_batch_scratch_double2(int N, int TT_max) {
    return (size_t)kSlots * kSlotDouble2 * N + ((size_t)TT_max * N + 1) / 2;
}

// Shared memory of a persistent batch CTA: the largest tile's, then the tail
// (item index, tensor-memory base, run parameters).
size_t tc_batch_smem_bytes(int N, int TT_max, uint32_t *tail) {
    const size_t base = tc_smem_bytes(N, TT_max);
    *tail = (uint32_t)base;
    return base + 64 + ((sizeof(RunParams) + 15) & ~(size_t)15);
}

int launch_tc_batch(const BatchLaunch &b, void *stream) {
    auto kern = b.MH == 1 ? propagate_tc_batch<1> : b.MH == 2 ? propagate_tc_batch<2> : nullptr;
    if (!kern) return (int)cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b.smem);
    if (e != cudaSuccess) return (int)e;
    if (b.prepare_only) return 0;
    kern<<<b.n_cta, kTcThreads, b.smem, (cudaStream_t)stream>>>(b.params, b.items, b.n_items, b.queue,
                                                                 reinterpret_cast<double2 *>(b.scratch), b.scr_stride,
                                                                 b.tc_tail);
    return (int)cudaGetLastError();
}

int launch_tc(const RunParams &p, void *stream, size_t smem) {
    cudaStream_t st = (cudaStream_t)stream;
    auto kern = p.N == 128 ? propagate_tc<1> : p.N == 256 ? propagate_tc<2> : nullptr;
    if (!kern) return (int)cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    kern<<<p.n_cta, kTcThreads, smem, st>>>(p);
    return (int)cudaGetLastError();
}

}  // namespace aqt
