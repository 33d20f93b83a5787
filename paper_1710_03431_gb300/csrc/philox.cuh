// Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11), device side.
// Stream layout of one trajectory (the paper only says "draw a random
// number", arXiv:1710.03431 Sec. IV):
//   key = (seed, 0x0000000171003431), counter = (trajectory, event, 0, 0);
//   event 0 -> x0: first threshold r;  event j >= 1 -> x0: u1, x1: u2, x2: next r;
//   uniform(x) = ((x >> 12) + 0.5) * 2^-52, strictly inside (0, 1).
// Fixed-step sampler (App. B.1): counter (trajectory, piece, 1, 0) for frozen
// half-step `piece` (0, 1, ... in time order) -> x0: jump test, x1: u1, x2: u2.
#pragma once
#include <cstdint>

namespace aqt {

struct Philox4 {
    uint64_t x[4];
};

__device__ __forceinline__ Philox4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                                uint64_t k0, uint64_t k1) {
    // round multipliers and Weyl increments from SC'11 (Table 2)
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    Philox4 o;
    o.x[0] = c0;
    o.x[1] = c1;
    o.x[2] = c2;
    o.x[3] = c3;
    return o;
}

__device__ __forceinline__ double uniform01(uint64_t x) {
    return ((double)(x >> 12) + 0.5) * 2.220446049250313080847263336181640625e-16;  // 2^-52
}

__device__ __forceinline__ Philox4 traj_event(uint64_t seed, int64_t traj, int64_t event) {
    return philox4x64_10((uint64_t)traj, (uint64_t)event, 0ull, 0ull, seed, 0x0000000171003431ull);
}

__device__ __forceinline__ Philox4 piece_draws(uint64_t seed, int64_t traj, int64_t piece) {
    return philox4x64_10((uint64_t)traj, (uint64_t)piece, 1ull, 0ull, seed, 0x0000000171003431ull);
}

}  // namespace aqt
