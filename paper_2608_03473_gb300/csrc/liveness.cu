// liveness.cu -- the prepass of the failed-lookahead guard: the liveness
// automaton of the token set (internal.h) run from right to left over the
// input, writing its state at every offset 0..n.
//
// Longest-match scanning can repeat failed lookahead at successive token
// starts (Section 9: over the tokens a, a+b and ; the input a^n costs
// Theta(n^2) steps, and certified cuts do not help where the cut byte never
// occurs).  With the set live_k of the states that still have an accepting
// position ahead of offset k, a scan ends its token as soon as its state
// leaves live_k, so each token costs its length plus one step.  live_k
// depends on the whole suffix, so the pass is a right-to-left DFA run over
// the input, parallel in three steps:
//   (1) lv_piece: per piece of LV_PIECE bytes and per automaton state r, the
//       state at the piece's start when the piece is entered at its end in r
//       (runs from different r that meet a reset class -- one whose
//       transition ignores the state -- agree from there on; all but r = 0
//       stop at the first one and take r = 0's result);
//   (2) lv_group / lv_link / lv_ends: the pieces' maps composed per group of
//       LV_GROUP pieces, the groups linked from the empty set at offset n
//       (one thread), then every piece's end state;
//   (3) lv_fill: per piece, the run from its end state, writing the state of
//       every offset.

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "runtime.h"

namespace lx {
namespace {

constexpr uint32_t LV_PIECE = 4096;   // input bytes per piece
constexpr uint32_t LV_GROUP = 64;     // pieces per group of the link step
constexpr int LV_NT = 256;
constexpr uint8_t LV_MERGED = 0xFF;   // a run that met a reset class: take the r = 0 run's result

struct LvParams {
    const uint8_t *in;
    uint64_t n;
    const uint8_t *blob;          // byte_class | next | reset (member not needed here)
    uint32_t blob_bytes;          // bytes of the blob staged in shared memory
    uint32_t R, C, next_off, reset_off;
    uint32_t M, NG;               // pieces, groups
    uint8_t *f;                   // [M * R] start state of a piece entered at its end in r
    uint8_t *g;                   // [NG * R] the same per group
    uint8_t *gend;                // [NG] state at each group's end
    uint8_t *pend;                // [M] state at each piece's end
    uint8_t *live;                // [n + 1] state at every offset
};

__device__ __forceinline__ const uint8_t *stage(const LvParams &P, uint8_t *smem)
{
    for (uint32_t i = threadIdx.x; i < P.blob_bytes / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(smem)[i] = reinterpret_cast<const uint4 *>(P.blob)[i];
    __syncthreads();
    return smem;
}

__device__ __forceinline__ uint64_t piece_end(const LvParams &P, uint32_t p)
{
    const uint64_t e = (uint64_t)(p + 1) * LV_PIECE;
    return e < P.n ? e : P.n;
}

// f of piece p entered in r, MERGED resolved
__device__ __forceinline__ uint32_t fval(const LvParams &P, uint32_t p, uint32_t r)
{
    const uint32_t v = P.f[(size_t)p * P.R + r];
    return v == LV_MERGED ? P.f[(size_t)p * P.R] : v;
}

__global__ void __launch_bounds__(LV_NT) lv_piece(LvParams P)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const uint8_t *T = stage(P, smem);
    const uint8_t *cls = T, *nx = T + P.next_off, *rst = T + P.reset_off;
    const uint64_t total = (uint64_t)P.M * P.R;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t p = (uint32_t)(i / P.R), r = (uint32_t)(i % P.R);
        const uint64_t b0 = (uint64_t)p * LV_PIECE;
        uint32_t x = r;
        bool merged = false;
        for (uint64_t k = piece_end(P, p); k-- > b0;) {
            const uint32_t c = cls[__ldg(P.in + k)];
            if (r != 0 && rst[c]) {
                merged = true;
                break;
            }
            x = nx[c * P.R + x];
        }
        P.f[i] = merged ? LV_MERGED : (uint8_t)x;
    }
}

__global__ void __launch_bounds__(LV_NT) lv_group(LvParams P)
{
    const uint64_t total = (uint64_t)P.NG * P.R;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t G = (uint32_t)(i / P.R), r = (uint32_t)(i % P.R);
        const uint32_t p0 = G * LV_GROUP, p1 = min(P.M, p0 + LV_GROUP);
        uint32_t x = r;
        for (uint32_t p = p1; p-- > p0;) x = fval(P, p, x);
        P.g[i] = (uint8_t)x;
    }
}

// one thread: the groups from the empty set (state 0) at offset n
__global__ void lv_link(LvParams P)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    uint32_t x = 0;
    for (uint32_t G = P.NG; G-- > 0;) {
        P.gend[G] = (uint8_t)x;
        x = P.g[(size_t)G * P.R + x];
    }
}

__global__ void __launch_bounds__(LV_NT) lv_ends(LvParams P)
{
    const uint32_t G = blockIdx.x * blockDim.x + threadIdx.x;
    if (G >= P.NG) return;
    const uint32_t p0 = G * LV_GROUP, p1 = min(P.M, p0 + LV_GROUP);
    uint32_t x = P.gend[G];
    for (uint32_t p = p1; p-- > p0;) {
        P.pend[p] = (uint8_t)x;
        x = fval(P, p, x);
    }
}

__global__ void __launch_bounds__(LV_NT) lv_fill(LvParams P)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const uint8_t *T = stage(P, smem);
    const uint8_t *cls = T, *nx = T + P.next_off;
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0) P.live[P.n] = 0;   // nothing is live past the end
    if (p >= P.M) return;
    const uint64_t b0 = (uint64_t)p * LV_PIECE;
    uint32_t x = P.pend[p];
    for (uint64_t k = piece_end(P, p); k-- > b0;) {
        x = nx[cls[__ldg(P.in + k)] * P.R + x];
        P.live[k] = (uint8_t)x;
    }
}

}  // namespace

int liveness_device(lx_ctx *c, const lx_tokenset *ts, const uint8_t *d_in, uint64_t n, uint8_t *d_out,
                    cudaStream_t s, const uint8_t **live, const uint32_t **member)
{
    const LiveTable &lt = ts->liveness;
    if (lt.status != LX_OK) return lt.status;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != c->device) return LX_E_INVAL;
    DeviceTables dt;
    int rc = ensure_device_tables(ts, dev, &dt);
    if (rc != LX_OK) return rc;
    const uint64_t M64 = (n + LV_PIECE - 1) / LV_PIECE;
    if (M64 > 0xFFFFFFF0ull / 256) return LX_E_INVAL;
    const uint32_t M = (uint32_t)M64, NG = (M + LV_GROUP - 1) / LV_GROUP;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_live = 0, o_f = al(d_out ? 0 : n + 1), o_g = al(o_f + (size_t)M * lt.R);
    const size_t o_gend = al(o_g + (size_t)NG * lt.R), o_pend = al(o_gend + NG), total = al(o_pend + M);
    rc = grow(&c->lv_dev, &c->lv_dev_bytes, total);
    if (rc != LX_OK) return rc;
    uint8_t *d = static_cast<uint8_t *>(c->lv_dev);
    LvParams P;
    P.in = d_in;
    P.n = n;
    P.blob = static_cast<const uint8_t *>(dt.d_live);
    P.blob_bytes = lt.member_off;   // byte_class, next and reset; 16-byte multiple
    P.R = lt.R;
    P.C = lt.C;
    P.next_off = lt.next_off;
    P.reset_off = lt.reset_off;
    P.M = M;
    P.NG = NG;
    P.f = d + o_f;
    P.g = d + o_g;
    P.gend = d + o_gend;
    P.pend = d + o_pend;
    P.live = d_out ? d_out : d + o_live;
    if (P.blob_bytes > 64u * 1024u) return LX_E_TOOBIG;
    static bool attr_done[64] = {false};
    if (dev < 64 && !attr_done[dev]) {
        if (cudaFuncSetAttribute(lv_piece, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024) != cudaSuccess ||
            cudaFuncSetAttribute(lv_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024) != cudaSuccess)
            return LX_E_CUDA;
        attr_done[dev] = true;
    }
    if (M) {
        const uint64_t pr = (uint64_t)M * lt.R;
        const uint32_t grid = (uint32_t)std::min<uint64_t>((pr + LV_NT - 1) / LV_NT, 64ull * c->num_sms);
        lv_piece<<<grid, LV_NT, P.blob_bytes, s>>>(P);
        const uint64_t gr = (uint64_t)NG * lt.R;
        lv_group<<<(uint32_t)std::min<uint64_t>((gr + LV_NT - 1) / LV_NT, 64ull * c->num_sms), LV_NT, 0, s>>>(P);
        lv_link<<<1, 32, 0, s>>>(P);
        lv_ends<<<(NG + LV_NT - 1) / LV_NT, LV_NT, 0, s>>>(P);
    }
    lv_fill<<<std::max<uint32_t>(1u, (M + LV_NT - 1) / LV_NT), LV_NT, P.blob_bytes, s>>>(P);
    rc = cuda_err(cudaGetLastError());
    if (rc != LX_OK) return rc;
    if (live) *live = P.live;
    if (member) *member = reinterpret_cast<const uint32_t *>(static_cast<const uint8_t *>(dt.d_live) + lt.member_off);
    return LX_OK;
}

}  // namespace lx

using namespace lx;

extern "C" int lx_liveness(lx_ctx *c, const lx_tokenset *ts, const uint8_t *d_in, uint64_t n, uint8_t *d_live,
                           void *stream)
{
    if (!c || !ts || !d_live || (n && !d_in)) return LX_E_INVAL;
    return liveness_device(c, ts, d_in, n, d_live, static_cast<cudaStream_t>(stream), nullptr, nullptr);
}
