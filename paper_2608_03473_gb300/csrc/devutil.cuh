// devutil.cuh -- device helpers shared by the lexing kernels (lex.cu,
// lexwarp.cu): shared-memory access through 32-bit shared addresses, the
// global timer, and the decoupled look-back over per-tile status words.
// Not part of the C ABI.
#pragma once

#include <cstdint>

namespace lx {

// ---- shared memory ----
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t lds_u8(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared.u8 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t lds_u16(uint32_t a)
{
    unsigned short v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts_u8(uint32_t a, uint32_t v)
{
    asm volatile("st.shared.u8 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void sts_u32(uint32_t a, uint32_t v)
{
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---- decoupled look-back ----
// A status word carries a flag and a count in one 64-bit store; nothing else
// a predecessor wrote is read, so relaxed gpu-scope accesses suffice.
constexpr unsigned long long ST_AGG = 1ull << 62;    // the tile's own kept count
constexpr unsigned long long ST_INCL = 2ull << 62;   // kept count of the tile and all before it
constexpr unsigned long long ST_VAL = (1ull << 62) - 1;

__device__ __forceinline__ unsigned long long ld_status(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_status(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

constexpr int LB_PER_LANE = 8;   // predecessor words per lane and round: 256 tiles per round

// One warp resolves the exclusive prefix of `tile` (whose aggregate `agg`
// is already published): each round its 32 lanes read 8 predecessor status
// words each, the round ends at the nearest inclusive prefix (summing the
// aggregates before it) or, with none, adds all 256 aggregates and moves
// back.  A word not yet published before the nearest inclusive prefix makes
// the round repeat, bounded by `timeout_ns` and by another CTA having given
// up (*error != 0); then *timed_out is set.  Lane 0 publishes the tile's
// inclusive prefix unless tile == withhold.
__device__ __forceinline__ uint64_t lookback(unsigned long long *status, uint32_t tile, uint64_t agg,
                                             uint64_t timeout_ns, const unsigned int *error, uint32_t withhold,
                                             bool &timed_out)
{
    const int lane = threadIdx.x & 31;
    if (tile == 0) return 0;
    uint64_t G = 0;
    int64_t base = (int64_t)tile - 1;
    const uint64_t t0 = globaltimer();
    uint32_t spins = 0;
    for (;;) {
        unsigned long long v[LB_PER_LANE];
#pragma unroll
        for (int j = 0; j < LB_PER_LANE; j++) {
            const int64_t k = base - (int64_t)LB_PER_LANE * lane - j;
            v[j] = k >= 0 ? ld_status(&status[k]) : ST_INCL;
        }
        int jstar = LB_PER_LANE;   // first inclusive word of this lane
        bool zero_before = false;
        unsigned long long lsum = 0;
#pragma unroll
        for (int j = 0; j < LB_PER_LANE; j++) {
            if (jstar == LB_PER_LANE) {
                const unsigned long long f = v[j] & ~ST_VAL;
                if (f == 0) zero_before = true;
                lsum += v[j] & ST_VAL;
                if (f == ST_INCL) jstar = j;
            }
        }
        const unsigned incl = __ballot_sync(0xffffffffu, jstar < LB_PER_LANE);
        const unsigned zero = __ballot_sync(0xffffffffu, zero_before);
        const unsigned upto = incl ? (incl & (0u - incl)) : 0u;            // lowest lane holding one
        const unsigned lanes = incl ? ((upto - 1u) | upto) : 0xffffffffu;  // lanes to sum
        if (zero & lanes) {
            if ((++spins & 15) == 0 &&
                (globaltimer() - t0 > timeout_ns || *(volatile const unsigned int *)error != 0)) {
                timed_out = true;
                break;
            }
            __nanosleep(32);
            continue;
        }
        unsigned long long x = ((lanes >> lane) & 1u) ? lsum : 0ull;
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        G += x;
        if (incl) break;
        base -= 32 * LB_PER_LANE;
    }
    if (lane == 0 && tile != withhold) st_status(&status[tile], ST_INCL | (G + agg));
    return G;
}

}  // namespace lx
