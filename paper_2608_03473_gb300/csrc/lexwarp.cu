// lexwarp.cu -- GB300 (sm_103a) certified-split lexing with warp-owned tiles:
// the default kernel of lx_lex for token sets with an event-code walk table
// (internal.h) and 16-byte aligned inputs.
//
// Every warp claims tiles of WT (6144) input bytes from a global counter and owns
// them end to end; nothing but the one-time table staging synchronises the
// CTA.  Per tile:
//   (a) halo scan: the 32 lanes find the first certified byte at or past the
//       tile end (the end of the tile's last chunk), 128 bytes per round;
//   (b) walk, phase 1: lane i starts its SLICE-byte slice in the PRE row,
//       which absorbs bytes until the first certified byte of the slice
//       (the planner of Section 6 with one target per lane: the chunk start)
//       and from there runs the longest-match scanner of Section 3 with every
//       certified byte ending the token in progress.  Lanes step 16-byte
//       blocks read from global memory (four bytes per shared-memory lookup
//       chain); each table entry carries the event code of its transition,
//       so four codes per word are packed with PRMT and stored at their
//       positions in the warp's event buffer;
//   (c) walk, phase 2: a warp suffix minimum gives each lane its chunk end
//       (the next lane's chunk start, or the halo's certified byte); lanes
//       run on to it, storing nothing past it, so each position has exactly
//       one writer.  SLOW (no transition and no accept) replays the token
//       from q0 to its last accepting position (longest match with
//       backtracking) and re-walks from there;
//   (d) count: each lane counts the kept codes of a contiguous slice of the
//       event buffer; the warp publishes the tile's count for a two-level
//       decoupled look-back (tiles within groups of GS, groups);
//   (e) emit: each lane turns its events into (kind, length) pairs in a
//       shared stage; the warp resolves the tile's output offset after its
//       next tile's walk (its predecessors have published by then) and copies
//       the stage to the output with coalesced stores.  The first lexing
//       failure (Corollary 1) truncates the count.
// A chunk whose end is not in the halo is walked byte by byte by lane 0 from
// global memory (counted, then emitted after the look-back).

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "devutil.cuh"
#include "internal.h"
#include "runtime.h"

namespace lx {
namespace {

constexpr uint32_t WT = 6144;                 // input bytes per warp tile (6 KiB: measured best of 2-8 KiB)
// The kernels' FORM template argument: bit 0 the table's lookup form
// (FORM_BYTE / FORM_CLASS), bit 1 (WIN) split-window rows (exact modes),
// bit 2 (DENSE) the geometry for many kept tokens per tile or far-apart cuts.
constexpr int WIN = 2;
constexpr int DENSE = 4;
constexpr uint32_t SLICE = WT / 32;           // bytes per lane slice (phase 1)
constexpr uint32_t BLK = 16;                  // bytes per lockstep step of a lane
constexpr uint32_t NB1 = SLICE / BLK;         // phase-1 steps
// A warp's geometry.  Sparse (the default): a chunk may end up to 512
// positions past its tile and 1 536 kept tokens are staged in shared memory.
// Dense: 2 048 positions (certified bytes far apart) and 768 staged tokens, a
// tile's further tokens going to the warp's spill slot in global memory (many
// kept tokens per tile), so that as many warps fit.
// Event code of position p at ev + p + 4 (p >> 7): a 4-byte pad after every
// 128 positions, so the 32 lanes' phase-1 stores (slices 128 positions
// apart) fall in 32 different banks.
template <int FORM>
struct Geo {
    static constexpr bool dense = (FORM & DENSE) != 0;
    static constexpr uint32_t HALO = dense ? 2048 : 512;   // positions past the tile a chunk may end at
    static constexpr uint32_t EVB = WT + HALO;             // event buffer positions
    static constexpr uint32_t LIMIT = EVB - BLK;           // chunk ends must lie below (room for the last block)
    static constexpr uint32_t EV_BYTES = ((EVB + 16 + 4 * ((EVB + 16) / 128 + 1)) + 15) / 16 * 16;
    static constexpr uint32_t STAGE_CAP = dense ? 768 : 1536;   // kept tokens per tile staged for coalesced writes
    static constexpr uint32_t WAREA = EV_BYTES + 4 * STAGE_CAP;  // shared bytes per warp
};
constexpr uint32_t SPARSE_LIMIT = Geo<0>::LIMIT;
constexpr uint32_t SPILL_CAP = Geo<DENSE>::LIMIT;   // spill slot entries per warp: a tile's kept tokens, at most
constexpr uint32_t GS = 64;                   // tiles per look-back group
constexpr uint32_t NONE = 0xFFFFFFFFu;
constexpr uint32_t BIG = 0x7FFFFFFFu;
constexpr int MAX_WARPS = 20;                 // warps per CTA at most (as many as shared memory allows)
constexpr unsigned ERR_TIMEOUT = 1u;
constexpr unsigned ERR_SMEM = 2u;
constexpr unsigned ERR_SPARSE = 4u;   // a chunk ran past the sparse limit: certified bytes too far apart
constexpr unsigned ERR_LOOKAHEAD = 8u;   // backtracking past its step budget (failed lookahead)

static_assert(SLICE % BLK == 0 && Geo<0>::WAREA % 16 == 0 && Geo<DENSE>::WAREA % 16 == 0, "geometry");
static_assert(Geo<0>::LIMIT - Geo<0>::STAGE_CAP <= SPILL_CAP, "spill slot");

struct WResult {
    unsigned long long total;          // kept tokens over all tiles
    unsigned long long inv_fail_pos;   // ~min failure offset (atomicMax), 0 = none
    unsigned long long inv_fail_tok;   // ~output index at that failure
    unsigned int error;
    unsigned int pad;
    unsigned int long_tiles;           // tiles whose last chunk ends past the sparse geometry's halo
    unsigned int pad2[3];
};

// Batches: a document's tiles are consecutive in the launch's tile sequence
// from first_tile; `set` indexes the WSet array staged with the tables.
struct WDoc {
    const uint8_t *in;
    uint64_t n;
    uint32_t first_tile;
    uint32_t set;
};

// One token set's rows and maps in a batch's combined table (offsets from
// the table's start; the rows of all sets lie in one 16-bit address window).
struct WSet {
    uint32_t p_start, p_pre, p_slow, kmap_off, cmap_off, cut_off, ctx_off, pad;
};

struct WDocRes {
    unsigned long long total;          // kept tokens of the document's tiles (any after a failure included)
    unsigned long long inv_fail_pos;   // ~min failure offset within the document, 0 = none
    unsigned long long inv_fail_tok;   // ~output index at that failure
    unsigned long long out_off1;       // output index of its first token + 1 (0: not yet resolved)
};

struct WParams {
    const uint8_t *in;
    uint64_t n;
    const uint8_t *blob;
    uint32_t blob_bytes, rows_bytes, row_shift;
    uint32_t p_start, p_pre, acc_off, kmap_off, cmap_off, cut_off, ctx_off;
    uint16_t *out_kinds;
    uint32_t *out_lens;
    uint64_t cap;
    uint32_t *spill;               // SPILL_CAP stage entries per warp of the grid
    unsigned long long *status;    // per tile: ST_AGG | kept count
    unsigned long long *gstatus;   // per group of GS tiles: ST_AGG | group count, or ST_INCL | inclusive prefix
    unsigned int *gdone;           // per group: tiles that have published
    unsigned int *tile_counter;
    WResult *res;
    uint32_t n_tiles;
    uint64_t timeout_ns;
    uint32_t withhold;
    uint64_t sparse_limit;   // longest chunk walked byte by byte before giving up (0: no limit)
    // batches
    const WDoc *docs;
    const uint32_t *tile_doc;   // document of every tile
    WDocRes *dres;
    uint32_t sets_off;          // WSet array in the table blob
    uint32_t n_ctx;             // split-window context classes of the table (0: none)
};

// Shared addresses of the tables and of this warp's buffers, and the tile.
struct WEnv {
    uint32_t P_start, P_pre, P_slow;
    uint32_t tb_s, acc_s, kmap_s, cmap_s, cut_s, ctx_s, shift;   // P_pre: the first PRE row (PRE_k follow)
    uint32_t ev;                 // event buffer: code of position p at ev + p
    unsigned int *err;           // the result record's error word
    uint32_t guard;              // 1: backtracking past its step budget stops the call (ERR_LOOKAHEAD)
    const uint8_t *in;           // the tile's first byte
    uint32_t nrel;               // input bytes from the tile start (clamped)
    uint64_t nrel64;
};

__device__ __forceinline__ uint32_t eva(const WEnv &E, uint32_t p) { return E.ev + p + ((p >> 7) << 2); }

__device__ __forceinline__ uint4 ldg16(const uint8_t *p)
{
    return __ldg(reinterpret_cast<const uint4 *>(p));
}

// One byte step: the next entry (row address | code << 1).
template <int FORM>
__device__ __forceinline__ uint32_t wstep(const WEnv &E, uint32_t e, uint32_t b)
{
    const uint32_t a = (FORM & 1) == FORM_BYTE ? ((e & ~0x1FEu) | (b << 1)) : ((e & ~0xFFu) | lds_u8(E.cmap_s + b));
    return lds_u16(a);
}

__device__ __forceinline__ uint32_t acc_code(const WEnv &E, uint32_t e)
{
    return lds_u8(E.acc_s + ((e - E.tb_s) >> E.shift));
}

// Whether a chunk may start at byte b after byte a: a certified byte, or a
// certified two-byte window (the cut table's row of a's context class).
__device__ __forceinline__ bool is_cut(const WEnv &E, uint32_t a, uint32_t b)
{
    return lds_u8(E.cut_s + (lds_u8(E.ctx_s + a) << 8) + b) != 0;
}

// Four byte steps over the little-endian word w as branch-free PTX; the
// dependent chain per byte is one LOP3 and the table load (the class form
// adds an independent PRMT and class-map load per byte).  The four event
// codes (the low byte of each entry) are packed into one word and stored at
// `ev` when the predicate holds: phase 1 (PH 1) stores a word that did not
// begin in a PRE row (x = P_pre, the first of them); phase 2 (PH 2) a word whose last byte y lies at
// or before the chunk end x.  cm: the class map's shared address.
#define LXW_PRED1 "setp.lo.u32 ps, %0, %3;\n\t"
#define LXW_PRED2 "setp.le.u32 ps, %4, %3;\n\t"
#define LXW_B(XOP, VIN, VOUT)                                                  \
    XOP "lop3.b32 a, " VIN ", t, %7, 0xD8;\n\t"                                \
        "ld.shared.u16 " VOUT ", [a];\n\t"
#define LXW_C(SEL, VIN, VOUT)                                                  \
    "prmt.b32 t, %2, %6, " SEL ";\n\t"                                         \
    "ld.shared.u8 c, [t];\n\t"                                                 \
    "lop3.b32 a, " VIN ", c, %7, 0xD8;\n\t"                                    \
    "ld.shared.u16 " VOUT ", [a];\n\t"
#define LXW_PACK                                                               \
    "prmt.b32 t0, v0, v1, 0x0040;\n\t"                                         \
    "prmt.b32 t1, v2, %0, 0x0040;\n\t"                                         \
    "prmt.b32 %1, t0, t1, 0x5410;\n\t"                                         \
    "@ps st.shared.u32 [%5], %1;\n\t}"
#define LXW_BYTE_BODY                                                          \
    LXW_B("shl.b32 t, %2, 1;\n\t", "%0", "v0")                                 \
    LXW_B("shr.b32 t, %2, 7;\n\t", "v0", "v1")                                 \
    LXW_B("shr.b32 t, %2, 15;\n\t", "v1", "v2")                                \
    LXW_B("shr.b32 t, %2, 23;\n\t", "v2", "%0")
#define LXW_CLASS_BODY                                                         \
    LXW_C("0x7650", "%0", "v0")                                                \
    LXW_C("0x7651", "v0", "v1")                                                \
    LXW_C("0x7652", "v1", "v2")                                                \
    LXW_C("0x7653", "v2", "%0")
#define LXW_HEAD "{\n\t.reg .pred ps;\n\t.reg .b32 t, a, c, v0, v1, v2, v3, t0, t1;\n\t"

template <int FORM, int PH>
__device__ __forceinline__ uint32_t wword(uint32_t &e, uint32_t w, uint32_t ev, uint32_t x, uint32_t y, uint32_t cm)
{
    uint32_t pk;
    const uint32_t mask = (FORM & 1) == FORM_BYTE ? 0x1FEu : 0xFFu;   // the address bits an entry's byte or class replaces
    if ((FORM & 1) == FORM_BYTE && PH == 1)
        asm volatile(LXW_HEAD LXW_PRED1 LXW_BYTE_BODY LXW_PACK
                     : "+r"(e), "=r"(pk) : "r"(w), "r"(x), "r"(y), "r"(ev), "r"(cm), "r"(mask) : "memory");
    else if ((FORM & 1) == FORM_BYTE)
        asm volatile(LXW_HEAD LXW_PRED2 LXW_BYTE_BODY LXW_PACK
                     : "+r"(e), "=r"(pk) : "r"(w), "r"(x), "r"(y), "r"(ev), "r"(cm), "r"(mask) : "memory");
    else if (PH == 1)
        asm volatile(LXW_HEAD LXW_PRED1 LXW_CLASS_BODY LXW_PACK
                     : "+r"(e), "=r"(pk) : "r"(w), "r"(x), "r"(y), "r"(ev), "r"(cm), "r"(mask) : "memory");
    else
        asm volatile(LXW_HEAD LXW_PRED2 LXW_CLASS_BODY LXW_PACK
                     : "+r"(e), "=r"(pk) : "r"(w), "r"(x), "r"(y), "r"(ev), "r"(cm), "r"(mask) : "memory");
    return pk;
}

__device__ __forceinline__ uint32_t byte_of(uint32_t w, uint32_t k) { return (w >> (8 * k)) & 0xFFu; }

__device__ __forceinline__ uint32_t pick4(uint32_t i, uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    return i == 0 ? a : i == 1 ? b : i == 2 ? c : d;
}

// A lane's walk state.
struct Lane {
    uint32_t e;       // row entry after the last stepped byte
    uint32_t p;       // next position to step
    uint32_t s;       // chunk start (first certified byte of the slice), NONE while in PRE
    uint32_t fail;    // failure offset (a token start with no accepting prefix), NONE
    uint32_t own;     // positions below this may record a failure (the chunk end)
    bool act;
    bool coarse;      // s is the start of the block in which PRE was left, not yet the byte
    uint4 blk;        // that block's bytes
    uint32_t pe;      // the PRE row at that block's start
};

// The block walk only notes the 16-byte block in which a lane left PRE (and
// keeps its bytes and its PRE row at the block start in registers); this
// finds the byte (the first certified byte or window of the block, where the
// PRE rows are left) and stores the event codes after it in its word, which
// the block step did not store (the word began in PRE): the state after the
// chunk's first byte is q0's step on it.
template <int FORM>
__device__ void refine_start(const WEnv &E, Lane &L)
{
    if (!L.coarse) return;
    L.coarse = false;
    const uint32_t pb = L.s;
    const uint4 c = L.blk;
    uint32_t j = 0, e = L.pe;
    if (FORM & WIN) {   // replay the PRE rows over the block: the byte where they are left
        for (; j < BLK; j++) {
            const uint32_t v = wstep<FORM>(E, e, byte_of(pick4(j >> 2, c.x, c.y, c.z, c.w), j & 3u));
            e = v;
            if (v < E.P_pre) break;
        }
    } else {            // the first certified byte: PRE's step on it as q0's
        uint32_t b = 0;
        for (; j < BLK; j++) {
            b = byte_of(pick4(j >> 2, c.x, c.y, c.z, c.w), j & 3u);
            if (lds_u8(E.cut_s + b)) break;
        }
        e = wstep<FORM>(E, E.P_start, b);
    }
    if (j == BLK) j = BLK - 1;   // unreachable: the block leaves PRE
    L.s = pb + j;
    for (uint32_t k = j + 1; k < ((j + 4) & ~3u); k++) {
        e = wstep<FORM>(E, e, byte_of(pick4(k >> 2, c.x, c.y, c.z, c.w), k & 3u));
        sts_u8(eva(E, pb + k), e & 0xFFu);
    }
}

// SLOW was reached before position `upto`: replay the token in progress from
// q0 (its start is the last event at or before hi, or the chunk start) to
// its last accepting position r, record the token end at r and re-walk from
// r to `upto`, storing codes only at positions <= hi.  Repeats while the
// re-walk falls into SLOW again at or before hi; a SLOW past hi belongs to
// the next chunk and stops the lane.  No accepting prefix: a failure at the
// token start (Corollary 1), recorded when it lies inside this chunk.
// Failed lookahead that repeats at successive token starts makes the repeats
// quadratic in the chunk length (Section 9); past a budget of steps linear in
// it the lane stops and flags ERR_LOOKAHEAD (with E.guard), and the caller
// lexes the input with the failed-lookahead guard instead.
template <int FORM>
__device__ void slow_fix(const WEnv &E, Lane &L, uint32_t upto, uint32_t hi)
{
    refine_start<FORM>(E, L);
    const uint32_t budget = 16u * (upto - L.s) + 65536u;
    uint32_t steps = 0;
    for (;;) {
        uint32_t tok = L.s;
        for (uint32_t j = min(upto - 1, hi); j > L.s; j--)
            if (lds_u8(eva(E, j))) {
                tok = j;
                break;
            }
        uint32_t q = E.P_start, r = NONE, rc = 0;
        for (uint32_t k = tok; k < upto; k++) {
            const uint32_t v = wstep<FORM>(E, q, __ldg(E.in + k));
            if ((v & 0xFFu) || v == E.P_slow) break;
            q = v;
            const uint32_t ac = acc_code(E, q);
            if (ac) {
                r = k + 1;
                rc = ac;
            }
        }
        if (r == NONE) {
            if (tok < L.own) L.fail = tok;
            L.act = false;
            return;
        }
        if (r <= hi) sts_u8(eva(E, r), rc);
        uint32_t e = E.P_start, kslow = NONE;
        for (uint32_t k = r; k < upto; k++) {
            const uint32_t v = wstep<FORM>(E, e, __ldg(E.in + k));
            if (k > r && k <= hi) sts_u8(eva(E, k), v & 0xFFu);   // the step at r (from START) ends nothing
            if (v == E.P_slow && e != E.P_slow) kslow = k;
            e = v;
        }
        L.e = e;
        if (e != E.P_slow) return;
        if (kslow > hi || r > hi) {
            L.act = false;
            return;
        }
        steps += upto - tok;
        if (E.guard && steps > budget) {
            atomicOr(E.err, ERR_LOOKAHEAD);
            L.act = false;
            return;
        }
    }
}

// Byte steps from L.p up to `upto` with the storing rule of the block steps.
template <int FORM>
__device__ void scalar_steps(const WEnv &E, Lane &L, uint32_t upto, uint32_t hi)
{
    while (L.p < upto && L.act) {
        const uint32_t k = L.p, e0 = L.e;
        const uint32_t v = wstep<FORM>(E, e0, __ldg(E.in + k));
        if (e0 >= E.P_pre && v < E.P_pre && L.s == NONE) L.s = k;
        if (e0 < E.P_pre && k <= hi) sts_u8(eva(E, k), v & 0xFFu);
        L.e = v;
        L.p = k + 1;
        if (v == E.P_slow) {
            if (k > hi) {
                L.act = false;
                return;
            }
            slow_fix<FORM>(E, L, k + 1, hi);
        }
    }
}

// At the end of the input: an accepting row ends its token there; a row
// that does not accept backtracks like SLOW.
template <int FORM>
__device__ void finalize(const WEnv &E, Lane &L, uint32_t hi)
{
    if (E.nrel > hi) {
        L.act = false;
        return;
    }
    while (L.act) {
        const uint32_t e = L.e;
        if (e == E.P_start || e >= E.P_pre) return;
        if (e != E.P_slow) {
            const uint32_t ac = acc_code(E, e);
            if (ac) {
                sts_u8(eva(E, E.nrel), ac);
                return;
            }
            L.e = E.P_slow;
        }
        slow_fix<FORM>(E, L, E.nrel, hi);
    }
}

// The chunk that starts at the certified byte `start` and leaves the halo,
// walked byte by byte from global memory up to the first certified byte at
// or past the tile end (or the end of the input).  Counts its kept tokens
// and, with out != nullptr, writes them from output index `o`.  Returns the
// kept count; *fail = the failure offset or NONE64.  With limit != 0 a
// chunk longer than `limit` bytes stops there and sets *over.
constexpr uint64_t NONE64 = ~0ull;

// Bytes of the input read through one 16-byte block held in registers (the
// byte-by-byte walk of a long chunk would otherwise wait on a load per byte).
struct ByteReader {
    const uint8_t *in;
    uint64_t n, pos = ~0ull;
    uint4 b;
    __device__ __forceinline__ uint32_t at(uint64_t q)
    {
        const uint64_t base = q & ~15ull;
        if (base != pos) {
            pos = base;
            if (base + 16 <= n) {
                b = __ldg(reinterpret_cast<const uint4 *>(in + base));
            } else {
                uint32_t w[4] = {0, 0, 0, 0};
                for (uint32_t k = 0; base + k < n; k++) w[k >> 2] |= (uint32_t)__ldg(in + base + k) << (8 * (k & 3));
                b = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        const uint32_t r = (uint32_t)(q & 15);
        return byte_of(pick4(r >> 2, b.x, b.y, b.z, b.w), r & 3);
    }
};

template <int FORM>
__device__ uint64_t generic_chunk(const WEnv &E, uint64_t start, uint64_t *fail, uint16_t *kinds, uint32_t *lens,
                                  uint64_t cap, uint64_t o, uint64_t limit = 0, unsigned *over = nullptr)
{
    const uint64_t n = E.nrel64;
    ByteReader rd{E.in, n};
    uint64_t p = start, tok = start, cnt = 0, steps = 0;
    uint32_t e = E.P_start;
    *fail = NONE64;
    const uint64_t stop = limit ? start + limit : ~0ull;
    auto emit = [&](uint32_t code, uint64_t len) {
        if (code < 4) return;
        if (kinds && o + cnt < cap) {
            kinds[o + cnt] = (uint16_t)lds_u16(E.kmap_s + 2 * (code >> 1));
            lens[o + cnt] = (uint32_t)len;
        }
        cnt++;
    };
    for (;;) {
        if (p == n) {
            if (e == E.P_start) return cnt;
            const uint32_t ac = e != E.P_slow ? acc_code(E, e) : 0u;
            if (ac) {
                emit(ac, p - tok);
                return cnt;
            }
        } else {
            if (p >= stop) {
                *over = ERR_SPARSE;
                return cnt;
            }
            const uint32_t b = rd.at(p);
            const uint32_t v = wstep<FORM>(E, e, b);
            if (v != E.P_slow) {
                if (v & 0xFFu) {
                    emit(v & 0xFFu, p - tok);
                    tok = p;
                    if (p >= WT && ((FORM & WIN) ? is_cut(E, rd.at(p - 1), b) : lds_u8(E.cut_s + b) != 0))
                        return cnt;
                }
                e = v;
                p++;
                continue;
            }
        }
        // longest match with backtracking: replay [tok, p) from q0; repeated
        // failed lookahead past a budget linear in the chunk stops the call
        steps += p - tok;
        if (limit && steps > 4 * limit) {
            *over = ERR_LOOKAHEAD;
            return cnt;
        }
        uint32_t q = E.P_start, rc = 0;
        uint64_t r = NONE64;
        for (uint64_t k = tok; k < p; k++) {
            const uint32_t v = wstep<FORM>(E, q, rd.at(k));
            if ((v & 0xFFu) || v == E.P_slow) break;
            q = v;
            const uint32_t ac = acc_code(E, q);
            if (ac) {
                r = k + 1;
                rc = ac;
            }
        }
        if (r == NONE64) {
            *fail = tok;
            return cnt;
        }
        emit(rc, r - tok);
        tok = p = r;
        e = E.P_start;
        if (r == n) return cnt;
        if (r >= WT && ((FORM & WIN) ? is_cut(E, rd.at(r - 1), rd.at(r)) : lds_u8(E.cut_s + rd.at(r)) != 0))
            return cnt;
    }
}

// One byte of a word in the emission: byte K of w is an event code; d is
// the distance from the previous event to this byte.  A kept code (>= 4)
// stores (code << 16 | d) at s and advances s; any event sets d to 0; d
// then steps to the next byte.  The PRMT takes d's low half and the code
// byte (d < 65536, so d's byte 3 is zero).
#define LXE_BYTE(K, SEL)                                                       \
    "bfe.u32 c, %2, " #K "*8, 8;\n\t"                                         \
    "setp.gt.u32 pk, c, 3;\n\t"                                                \
    "setp.ne.u32 pe, c, 0;\n\t"                                                \
    "prmt.b32 v, %1, %2, " SEL ";\n\t"                                         \
    "@pk st.shared.u32 [%0], v;\n\t"                                           \
    "@pk add.u32 %0, %0, 4;\n\t"                                               \
    "@pe mov.u32 %1, 0;\n\t"                                                   \
    "add.u32 %1, %1, 1;\n\t"

// The kept codes of one word of the event buffer, in position order, into
// the stage (s: next stage address, d: distance from the previous event to
// the word's first byte); both are updated.
__device__ __forceinline__ void emit_word(uint32_t &s, uint32_t &d, uint32_t w)
{
    asm volatile("{\n\t.reg .pred pk, pe;\n\t.reg .b32 c, v;\n\t"
                 LXE_BYTE(0, "0x3410") LXE_BYTE(1, "0x3510") LXE_BYTE(2, "0x3610") LXE_BYTE(3, "0x3710")
                 "}"
                 : "+r"(s), "+r"(d) : "r"(w) : "memory");
}

__device__ __forceinline__ uint32_t kept_mask(uint32_t w)   // bit 7 of every byte >= 4 (a kept code)
{
    return (((w | 0x80808080u) - 0x04040404u) | w) & 0x80808080u;
}
__device__ __forceinline__ uint32_t event_mask(uint32_t w)  // bit 7 of every nonzero byte
{
    return (((w | 0x80808080u) - 0x01010101u) | w) & 0x80808080u;
}

// ---- two-level decoupled look-back ----
// Tiles form groups of GS.  A tile publishes its kept count (ST_AGG) and
// counts itself into its group; the warp that completes a group sums the
// group's counts and publishes the group aggregate (group 0: its inclusive
// prefix).  A tile's output offset is the exclusive prefix of its group
// (a look-back over group words, a few dozen deep) plus the counts of the
// tiles before it in the group.  Every wait is bounded by the time budget
// and ends early once another warp has given up.
// Polls back off exponentially (64 ns doubling to 4 us): while one slow tile
// (say, a chunk walked byte by byte) holds up its group, thousands of waiting
// warps must not flood L2 with status reads and starve that tile's own loads.
struct Waiter {
    uint64_t t0;
    uint32_t spins;
    // false (and the error flag raised) once the budget is spent
    __device__ bool again(const WParams &P)
    {
        if ((++spins & 3) == 0 &&
            (globaltimer() - t0 > P.timeout_ns || *(volatile const unsigned int *)&P.res->error != 0)) {
            if ((threadIdx.x & 31) == 0) atomicOr(&P.res->error, ERR_TIMEOUT);
            return false;
        }
        __nanosleep(64u << min(spins, 6u));
        return true;
    }
};

__device__ void publish_tile(const WParams &P, uint32_t tile, uint64_t agg)
{
    const int lane = threadIdx.x & 31;
    const uint32_t g = tile / GS, f = g * GS;
    const uint32_t gsize = min(GS, P.n_tiles - f);
    uint32_t last = 0;
    if (lane == 0 && agg) atomicAdd(&P.res->total, agg);
    if (lane == 0 && tile != P.withhold) {
        st_status(&P.status[tile], ST_AGG | agg);
        // release: the status store before the count; acquire: the group's
        // other status stores visible to the warp that completes it
        uint32_t old;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(&P.gdone[g]) : "memory");
        last = old + 1 == gsize ? 1u : 0u;
    }
    if (!__shfl_sync(0xffffffffu, last, 0)) return;
    __threadfence();   // every lane reads the statuses lane 0's acquire made visible
    // every tile of the group has published: its aggregate
    unsigned long long x = 0;
    for (uint32_t j = lane; j < gsize; j += 32) x += ld_status(&P.status[f + j]) & ST_VAL;
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) st_status(&P.gstatus[g], (g == 0 ? ST_INCL : ST_AGG) | x);
}

// Lane 0 waits until status word *p is published; the warp learns whether
// the wait ended in time.  Only one word is polled: thousands of waiting warps
// re-reading whole rounds of status words would crowd the L2 lines that
// every warp reads and slow the very tile they wait for.
__device__ bool wait_word(const WParams &P, Waiter &W, const unsigned long long *p)
{
    uint32_t ok = 1;
    if ((threadIdx.x & 31) == 0)
        while (ld_status(p) == 0)
            if (!W.again(P)) {
                ok = 0;
                break;
            }
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// The output offset of `tile`; false when a wait ran out of time.
__device__ bool resolve_tile(const WParams &P, uint32_t tile, uint64_t &G)
{
    const int lane = threadIdx.x & 31;
    const uint32_t g = tile / GS, f = g * GS;
    Waiter W{globaltimer(), 0};
    // the tiles before this one in its group (at most GS - 1 < 64 words)
    unsigned long long w = 0;
    for (;;) {
        uint32_t miss = NONE;
        w = 0;
        for (uint32_t j = f + lane; j < tile; j += 32) {
            const unsigned long long v = ld_status(&P.status[j]);
            if (v == 0) miss = min(miss, j);
            w += v & ST_VAL;
        }
        miss = __reduce_min_sync(0xffffffffu, miss);
        if (miss == NONE) break;
        if (!wait_word(P, W, &P.status[miss])) return false;
    }
    for (int o = 16; o; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    // the groups before: sum aggregates back to the nearest inclusive prefix
    uint64_t GE = 0;
    int64_t base = (int64_t)g - 1;
    while (base >= 0) {
        unsigned long long v[LB_PER_LANE];
#pragma unroll
        for (int j = 0; j < LB_PER_LANE; j++) {
            const int64_t k = base - (int64_t)LB_PER_LANE * lane - j;
            v[j] = k >= 0 ? ld_status(&P.gstatus[k]) : ST_INCL;
        }
        int jstar = LB_PER_LANE;
        uint32_t zk = NONE;   // an unpublished group word of this lane before its first inclusive one
        unsigned long long lsum = 0;
#pragma unroll
        for (int j = 0; j < LB_PER_LANE; j++) {
            if (jstar == LB_PER_LANE) {
                const unsigned long long fl = v[j] & ~ST_VAL;
                if (fl == 0 && zk == NONE) zk = (uint32_t)(base - (int64_t)LB_PER_LANE * lane - j);
                lsum += v[j] & ST_VAL;
                if (fl == ST_INCL) jstar = j;
            }
        }
        const unsigned incl = __ballot_sync(0xffffffffu, jstar < LB_PER_LANE);
        const unsigned upto = incl ? (incl & (0u - incl)) : 0u;
        const unsigned lanes = incl ? ((upto - 1u) | upto) : 0xffffffffu;
        const uint32_t wait_k = __reduce_min_sync(0xffffffffu, ((lanes >> lane) & 1u) ? zk : NONE);
        if (wait_k != NONE) {
            if (!wait_word(P, W, &P.gstatus[wait_k])) return false;
            continue;
        }
        unsigned long long x = ((lanes >> lane) & 1u) ? lsum : 0ull;
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        GE += x;
        if (incl) break;
        base -= 32 * LB_PER_LANE;
    }
    // once the group is complete, its inclusive prefix shortens later look-backs
    if (lane == 0 && g > 0) {
        const unsigned long long gv = ld_status(&P.gstatus[g]);
        if ((gv & ~ST_VAL) == ST_AGG) st_status(&P.gstatus[g], ST_INCL | (GE + (gv & ST_VAL)));
    }
    G = GE + w;
    return true;
}

// A tile whose tokens wait in the warp's stage for their output offset.
struct Pending {
    uint32_t tile;      // NONE: nothing pending
    uint32_t staged;    // the tile's kept tokens (dense: | how many of them are in the stage << 16)
    uint64_t fail;      // failure offset within the tile, or NONE64
    uint64_t agg;
    uint32_t doc, dtile;   // batches: its document and its index there
    uint32_t kmap_s;       // the kind map of its token set
};

// After a tile's output offset G is known: its failure (the first of the
// input, or of its document in a batch) and, for a document's first tile,
// the document's output offset.
template <bool BATCH>
__device__ void report_failure(const WParams &P, uint32_t tile, uint64_t fail, uint64_t G, uint64_t agg,
                               uint32_t doc, uint32_t dtile)
{
    if ((threadIdx.x & 31) != 0) return;
    if (BATCH) {
        if (dtile == 0) P.dres[doc].out_off1 = G + 1;
        if (fail != NONE64) {
            atomicMax(&P.dres[doc].inv_fail_pos, ~(unsigned long long)((uint64_t)dtile * WT + fail));
            atomicMax(&P.dres[doc].inv_fail_tok, ~(unsigned long long)(G + agg));
        }
    } else if (fail != NONE64) {
        atomicMax(&P.res->inv_fail_pos, ~(unsigned long long)((uint64_t)tile * WT + fail));
        atomicMax(&P.res->inv_fail_tok, ~(unsigned long long)(G + agg));
    }
}

// The staged tokens of a tile to the output from index G, coalesced: the
// first `split` from the shared stage, the rest from the warp's spill slot;
// kmap_s: the kind map of the tile's token set.  Each lane writes V
// consecutive tokens at a time (kinds as one 2V-byte store, lengths as one
// 4V-byte store) from the first index where G + i is a multiple of V, when
// the output arrays are aligned for it and the capacity does not cut the
// tile; the tokens before and after those groups, and every token otherwise,
// one by one.  V = 2 for the sparse geometry, 4 for the dense one (measured).
template <uint32_t V>
__device__ void copy_stage(const WParams &P, uint32_t kmap_s, uint32_t stage, const uint32_t *spill, uint32_t split,
                           uint32_t staged, uint64_t G)
{
    static_assert(V == 2 || V == 4, "group size");
    const uint32_t lane = threadIdx.x & 31;
    auto val = [&](uint32_t i) { return i < split ? lds_u32(stage + 4 * i) : spill[i - split]; };
    auto one = [&](uint32_t i) {
        const uint64_t o = G + i;
        if (o < P.cap) {
            const uint32_t v = val(i);
            P.out_kinds[o] = (uint16_t)lds_u16(kmap_s + (v >> 16));
            P.out_lens[o] = v & 0xFFFFu;
        }
    };
    const bool aligned = ((reinterpret_cast<uintptr_t>(P.out_kinds) & (2 * V - 1)) |
                          (reinterpret_cast<uintptr_t>(P.out_lens) & (4 * V - 1))) == 0;
    if (!aligned || G + staged > P.cap) {
        for (uint32_t i = lane; i < staged; i += 32) one(i);
        return;
    }
    const uint32_t h = min((uint32_t)((V - (G & (V - 1))) & (V - 1)), staged);   // tokens before the first group
    if (lane < h) one(lane);
    const uint32_t ng = (staged - h) / V;
    for (uint32_t q = lane; q < ng; q += 32) {
        const uint32_t i = h + V * q;
        const uint64_t o = G + i;
        if (V == 2) {
            const uint32_t v0 = val(i), v1 = val(i + 1);
            const uint32_t k0 = lds_u16(kmap_s + (v0 >> 16)), k1 = lds_u16(kmap_s + (v1 >> 16));
            *reinterpret_cast<uint32_t *>(P.out_kinds + o) = k0 | (k1 << 16);
            *reinterpret_cast<uint2 *>(P.out_lens + o) = make_uint2(v0 & 0xFFFFu, v1 & 0xFFFFu);
        } else {
            uint32_t v0, v1, v2, v3;
            if (i + 4 <= split && ((stage + 4 * i) & 15u) == 0) {
                asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                             : "=r"(v0), "=r"(v1), "=r"(v2), "=r"(v3) : "r"(stage + 4 * i));
            } else {
                v0 = val(i);
                v1 = val(i + 1);
                v2 = val(i + 2);
                v3 = val(i + 3);
            }
            const uint32_t k0 = lds_u16(kmap_s + (v0 >> 16)), k1 = lds_u16(kmap_s + (v1 >> 16));
            const uint32_t k2 = lds_u16(kmap_s + (v2 >> 16)), k3 = lds_u16(kmap_s + (v3 >> 16));
            *reinterpret_cast<uint2 *>(P.out_kinds + o) = make_uint2(k0 | (k1 << 16), k2 | (k3 << 16));
            *reinterpret_cast<uint4 *>(P.out_lens + o) =
                make_uint4(v0 & 0xFFFFu, v1 & 0xFFFFu, v2 & 0xFFFFu, v3 & 0xFFFFu);
        }
    }
    const uint32_t t = h + V * ng;   // the last tokens, fewer than V
    if (lane < staged - t) one(t + lane);
}

__device__ __forceinline__ uint4 blk_at(const WEnv &E, uint32_t q)
{
    return q + BLK <= E.nrel ? ldg16(E.in + q) : make_uint4(0, 0, 0, 0);
}

__device__ __forceinline__ void zero16(uint32_t a)
{
    asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};" ::"r"(a), "r"(0u) : "memory");
}

// Phase 1, one lockstep step of a lane: the block at L.p (words in `cur`),
// or, where fewer than 16 bytes remain, the rest of the input byte by byte.
template <int FORM>
__device__ __forceinline__ void phase1_step(const WEnv &E, Lane &L, const uint4 &cur)
{
    if (!L.act) return;
    if (L.p + BLK <= E.nrel) {
        const uint32_t pb = L.p, ev = eva(E, pb), e_in = L.e;
        wword<FORM, 1>(L.e, cur.x, ev, E.P_pre, 0, E.cmap_s);
        wword<FORM, 1>(L.e, cur.y, ev + 4, E.P_pre, 0, E.cmap_s);
        wword<FORM, 1>(L.e, cur.z, ev + 8, E.P_pre, 0, E.cmap_s);
        wword<FORM, 1>(L.e, cur.w, ev + 12, E.P_pre, 0, E.cmap_s);
        if (L.s == NONE && L.e < E.P_pre) {   // PRE was left in this block (the byte: refine_start)
            L.s = pb;
            L.coarse = true;
            L.blk = cur;
            if (FORM & WIN) L.pe = e_in;
        }
        L.p = pb + BLK;
        if (L.e == E.P_slow) slow_fix<FORM>(E, L, L.p, BIG);
    } else {
        scalar_steps<FORM>(E, L, E.nrel, BIG);
        finalize<FORM>(E, L, BIG);
        L.act = false;
    }
}

// Phase 2, one lockstep step of a lane: the block at L.p, storing the codes of
// positions up to the chunk end `end`; the lane stops after the block that
// holds the end.  `act` is the lane's phase-2 activity.
template <int FORM>
__device__ __forceinline__ void phase2_step(const WEnv &E, Lane &L, const uint4 &cur, uint32_t end, bool &act)
{
    if (!act) return;
    if (L.p + BLK <= E.nrel) {
        const uint32_t pb = L.p, ev = eva(E, pb);
        const uint32_t pk0 = wword<FORM, 2>(L.e, cur.x, ev, end, pb + 3, E.cmap_s);
        const uint32_t pk1 = wword<FORM, 2>(L.e, cur.y, ev + 4, end, pb + 7, E.cmap_s);
        const uint32_t pk2 = wword<FORM, 2>(L.e, cur.z, ev + 8, end, pb + 11, E.cmap_s);
        const uint32_t pk3 = wword<FORM, 2>(L.e, cur.w, ev + 12, end, pb + 15, E.cmap_s);
        L.p = pb + BLK;
        if (L.p > end) {
            // the block holds the chunk end: the codes of its word up to the end
            const uint32_t wk = (end - pb) >> 2, pk = pick4(wk, pk0, pk1, pk2, pk3);
            for (uint32_t k = 0; k <= ((end - pb) & 3u); k++) sts_u8(ev + 4 * wk + k, byte_of(pk, k));
            if (L.e == E.P_slow && byte_of(pk, (end - pb) & 3u) == 0) slow_fix<FORM>(E, L, L.p, end);
            act = false;
        } else if (L.e == E.P_slow) {
            slow_fix<FORM>(E, L, L.p, end);
            act = L.act;
        }
    } else {
        scalar_steps<FORM>(E, L, E.nrel, end);
        finalize<FORM>(E, L, end);
        act = false;
    }
}

template <int FORM, bool BATCH>
__global__ void __launch_bounds__(32 * MAX_WARPS, 1) lex_warps(WParams P)
{
    extern __shared__ __align__(16) uint8_t smem[];
    constexpr bool dense = Geo<FORM>::dense;
    constexpr uint32_t EVB = Geo<FORM>::EVB, LIMIT = Geo<FORM>::LIMIT, EV_BYTES = Geo<FORM>::EV_BYTES;
    constexpr uint32_t STAGE_CAP = Geo<FORM>::STAGE_CAP, WAREA = Geo<FORM>::WAREA;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t sbase = smem_u32(smem);
    const uint32_t tb_s = (sbase + 511u) & ~511u;
    if (tb_s + P.rows_bytes > 65536u) {   // 16-bit row addresses must reach every row
        if (threadIdx.x == 0) atomicOr(&P.res->error, ERR_SMEM);
        return;
    }
    {   // stage the tables; row offsets become shared addresses
        uint16_t *dst = reinterpret_cast<uint16_t *>(smem + (tb_s - sbase));
        const uint16_t *src = reinterpret_cast<const uint16_t *>(P.blob);
        const uint32_t n16 = P.blob_bytes / 2, r16 = P.rows_bytes / 2;
        for (uint32_t i = threadIdx.x; i < n16; i += blockDim.x) {
            const uint32_t v = src[i];
            dst[i] = (uint16_t)(i < r16 ? v + tb_s : v);
        }
    }
    WEnv E;
    E.P_slow = tb_s;
    E.P_start = tb_s + P.p_start;
    E.P_pre = tb_s + P.p_pre;
    E.tb_s = tb_s;
    E.acc_s = tb_s + P.acc_off;
    E.kmap_s = tb_s + P.kmap_off;
    E.cmap_s = tb_s + P.cmap_off;
    E.cut_s = tb_s + P.cut_off;
    E.ctx_s = tb_s + P.ctx_off;
    E.shift = P.row_shift;
    E.err = &P.res->error;
    E.guard = P.sparse_limit != 0 ? 1u : 0u;
    const uint32_t warea = ((tb_s + P.blob_bytes + 15u) & ~15u) + (uint32_t)wid * WAREA;
    E.ev = warea;
    const uint32_t stage = warea + EV_BYTES;
    uint32_t *const spill = P.spill + ((size_t)blockIdx.x * (blockDim.x >> 5) + wid) * SPILL_CAP;
    for (uint32_t i = lane; i < EV_BYTES / 16; i += 32) zero16(E.ev + 16 * i);
    __syncthreads();
    const uint32_t ahead = gridDim.x * (blockDim.x / 32);   // tiles the other warps take meanwhile

    Pending pend{NONE, 0, NONE64, 0, 0, 0, 0};
    for (;;) {
        uint32_t tile = 0;
        if (lane == 0) {
            tile = atomicAdd(P.tile_counter, 1u);
            if (*(volatile unsigned int *)&P.res->error != 0) tile = P.n_tiles;   // a wait gave up: stop
        }
        tile = __shfl_sync(0xffffffffu, tile, 0);
        if (tile >= P.n_tiles) break;
        uint32_t doc = 0, dtile = tile;
        if (BATCH) {   // the tile's document and its token set's rows and maps
            doc = __ldg(P.tile_doc + tile);
            const WDoc D = P.docs[doc];
            dtile = tile - D.first_tile;
            E.in = D.in + (uint64_t)dtile * WT;
            E.nrel64 = D.n - (uint64_t)dtile * WT;
            const uint32_t ws = tb_s + P.sets_off + D.set * (uint32_t)sizeof(WSet);
            E.P_start = tb_s + lds_u32(ws);
            E.P_pre = tb_s + lds_u32(ws + 4);
            E.P_slow = tb_s + lds_u32(ws + 8);
            E.kmap_s = tb_s + lds_u32(ws + 12);
            E.cmap_s = tb_s + lds_u32(ws + 16);
            E.cut_s = tb_s + lds_u32(ws + 20);
            E.ctx_s = tb_s + lds_u32(ws + 24);
        } else {
            E.in = P.in + (uint64_t)tile * WT;
            E.nrel64 = P.n - (uint64_t)tile * WT;
        }
        E.nrel = E.nrel64 < BIG ? (uint32_t)E.nrel64 : BIG;
        const uint32_t nrel = E.nrel;
        if (!BATCH && lane == 0 && tile + ahead < P.n_tiles) {   // a tile some warp takes about one tile from now, into L2
            const uint64_t fb = (uint64_t)(tile + ahead) * WT;
            const uint64_t left = P.n - fb;
            const uint32_t bytes = (uint32_t)(left < EVB ? left : EVB) & ~15u;
            if (bytes)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(P.in + fb), "r"(bytes) : "memory");
        }

        // (a) the first certified byte at or past the tile end, below LIMIT
        uint32_t c1;
        if (nrel <= WT) {
            c1 = nrel;
        } else {
            const uint32_t lim = nrel < LIMIT ? nrel : LIMIT;
            c1 = NONE;
            uint32_t carry = (FORM & WIN) ? __ldg(E.in + WT - 1) : 0u;   // the byte before the round (windows)
            for (uint32_t b0 = WT; b0 < lim; b0 += 128) {
                const uint32_t pos = b0 + 4 * lane;
                uint32_t m = 0, w = 0;
                if (pos + 4 <= lim) {
                    w = __ldg(reinterpret_cast<const uint32_t *>(E.in + pos));
                } else {
                    for (uint32_t k = 0; pos + k < lim; k++) w |= (uint32_t)__ldg(E.in + pos + k) << (8 * k);
                }
                if (FORM & WIN) {   // each byte with the byte before it
                    const uint32_t up = __shfl_up_sync(0xffffffffu, w, 1);
                    uint32_t prev = lane == 0 ? carry : up >> 24;
                    for (uint32_t k = 0; k < 4 && pos + k < lim; k++) {
                        const uint32_t b = byte_of(w, k);
                        if (is_cut(E, prev, b)) m |= 1u << k;
                        prev = b;
                    }
                    carry = __shfl_sync(0xffffffffu, w, 31) >> 24;
                } else {           // single certified bytes: the cut table's first row
                    for (uint32_t k = 0; k < 4 && pos + k < lim; k++)
                        if (lds_u8(E.cut_s + byte_of(w, k))) m |= 1u << k;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, m != 0);
                if (bal) {
                    const int src = __ffs(bal) - 1;
                    const uint32_t mm = __shfl_sync(0xffffffffu, m, src);
                    c1 = b0 + 4 * src + __ffs(mm) - 1;
                    break;
                }
            }
            if (c1 == NONE && lim == nrel) c1 = nrel;   // no certified byte before the end of the input
        }

        // (b) phase 1: every lane walks its slice from the PRE row
        const uint32_t t0 = (uint32_t)lane * SLICE;
        const bool first = dtile == 0 && lane == 0;   // the input's (document's) first chunk starts at 0
        Lane L;
        // a lane starts in the PRE row of the context of the byte before its slice
        uint32_t pre0 = E.P_pre;
        if ((FORM & WIN) && !first && t0 < nrel) pre0 += lds_u8(E.ctx_s + __ldg(E.in + (int64_t)t0 - 1)) << E.shift;
        L.e = first ? E.P_start : pre0;
        L.s = first ? 0u : NONE;
        L.p = t0;
        L.fail = NONE;
        L.own = NONE;
        L.act = t0 < nrel;
        L.coarse = false;
        // two register blocks in turn: a block is loaded two steps before it is walked
        uint4 A = blk_at(E, t0), B = blk_at(E, t0 + BLK);
#pragma unroll 1
        for (uint32_t it = 0; it < NB1; it += 2) {
            phase1_step<FORM>(E, L, A);
            A = blk_at(E, L.p + BLK);
            phase1_step<FORM>(E, L, B);
            B = blk_at(E, L.p + BLK);
        }

        refine_start<FORM>(E, L);

        // (c) chunk ends: the next lane's chunk start, else the halo's
        uint32_t smin = L.s;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_down_sync(0xffffffffu, smin, o);
            if (lane + o < 32) smin = min(smin, y);
        }
        uint32_t end = __shfl_down_sync(0xffffffffu, smin, 1);
        if (lane == 31) end = NONE;
        if (end == NONE) end = c1;
        const uint32_t c0 = __shfl_sync(0xffffffffu, smin, 0);
        const bool long_lane = L.s != NONE && end == NONE;   // its chunk leaves the halo
        bool act2 = L.act && L.s != NONE && end != NONE;
        L.own = end;
        while (__any_sync(0xffffffffu, act2)) {
            phase2_step<FORM>(E, L, A, end, act2);
            if (act2) A = blk_at(E, L.p + BLK);
            if (!__any_sync(0xffffffffu, act2)) break;
            phase2_step<FORM>(E, L, B, end, act2);
            if (act2) B = blk_at(E, L.p + BLK);
        }
        __syncwarp();

        // (d) count the kept codes of (c0, hi]
        const uint32_t fail = __reduce_min_sync(0xffffffffu, L.fail);
        const uint32_t long_s1 = __reduce_max_sync(0xffffffffu, long_lane ? L.s + 1 : 0u);
        uint32_t hi = c1 != NONE ? c1 : long_s1 - 1;
        if (fail < hi) hi = fail;
        uint32_t wa = 0, wb = 0, last = 0, cnt = 0;
        uint32_t lastw = NONE;   // the last word of this lane's range holding a code
        if (c0 != NONE) {
            if (hi != c1) {   // a failure or a chunk past the halo: clear every code after hi
                const uint32_t z0 = eva(E, hi) + 1, z1 = (z0 + 15u) & ~15u;
                for (uint32_t a = z0 + lane; a < z1; a += 32) sts_u8(a, 0);
                for (uint32_t a = z1 + 16 * lane; a < E.ev + EV_BYTES; a += 16 * 32) zero16(a);
                __syncwarp();
            }
            const uint32_t w0 = (c0 + 1) >> 2, w1 = max((hi >> 2) + 1, w0);
            const uint32_t per = (w1 - w0 + 31) / 32;
            wa = min(w0 + lane * per, w1);
            wb = min(wa + per, w1);
            for (uint32_t i = wa; i < wb; i++) {
                const uint32_t w = lds_u32(eva(E, 4 * i));
                cnt += __popc(kept_mask(w));
                if (w) lastw = i;
            }
            if (lastw != NONE)   // the lane's last code
                last = 4 * lastw + (31 - __clz(lds_u32(eva(E, 4 * lastw)))) / 8;
        }
        uint32_t excl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, excl, o);
            if (lane >= o) excl += y;
        }
        const uint32_t fast_total = __shfl_sync(0xffffffffu, excl, 31);
        excl -= cnt;
        // the chunk past the halo, counted by lane 0
        uint64_t gen_cnt = 0, gen_fail = NONE64;
        const bool do_long = c0 != NONE && long_s1 != 0 && fail > long_s1 - 1;
        unsigned over = 0;
        if (do_long && lane == 0) {
            gen_cnt = generic_chunk<FORM>(E, long_s1 - 1, &gen_fail, nullptr, nullptr, 0, 0, P.sparse_limit, &over);
            if (over) atomicOr(&P.res->error, over);   // the caller lexes the input another way
            if (!dense) atomicAdd(&P.res->long_tiles, 1u);
        }
        if (dense && lane == 0 && c0 != NONE && (c1 == NONE || (c1 >= SPARSE_LIMIT && c1 < nrel)))
            atomicAdd(&P.res->long_tiles, 1u);   // long for the sparse geometry
        if (__shfl_sync(0xffffffffu, over ? 1u : 0u, 0)) {
            publish_tile(P, tile, 0);
            break;
        }
        gen_cnt = __shfl_sync(0xffffffffu, gen_cnt, 0);
        gen_fail = __shfl_sync(0xffffffffu, gen_fail, 0);
        const uint64_t agg = fast_total + gen_cnt;
        const uint64_t fpos = fail != NONE ? (uint64_t)fail : gen_fail;
        if (BATCH && lane == 0 && agg) atomicAdd(&P.dres[doc].total, agg);
        publish_tile(P, tile, agg);

        // the previous tile's output: its predecessors have had a whole tile to publish
        if (pend.tile != NONE) {
            uint64_t G = 0;
            if (!resolve_tile(P, pend.tile, G)) break;
            report_failure<BATCH>(P, pend.tile, pend.fail, G, pend.agg, pend.doc, pend.dtile);
            copy_stage<dense ? 4 : 2>(P, pend.kmap_s, stage, spill, dense ? pend.staged >> 16 : STAGE_CAP,
                       dense ? pend.staged & 0xFFFFu : pend.staged, G);
            pend.tile = NONE;
            __syncwarp();
        }

        // (e) emit: (kind, length) of every kept code, in order, into the stage
        // (past STAGE_CAP into the warp's spill slot)
        const bool defer = !do_long;
        uint64_t G = 0;
        uint32_t split = STAGE_CAP;   // dense: how many kept tokens are in the stage (the rest: spill slot)
        if (!defer) {   // rare: a chunk past the halo is written at once
            if (!resolve_tile(P, tile, G)) break;
            report_failure<BATCH>(P, tile, fpos, G, agg, doc, dtile);
        }
        if (c0 != NONE) {
            uint32_t prev = last;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, prev, o);
                if (lane >= o) prev = max(prev, y);
            }
            prev = __shfl_up_sync(0xffffffffu, prev, 1);
            if (lane == 0 || prev < c0) prev = c0;
            // every lane its words, four codes per word without branches;
            // the words read are cleared for the next tile
            if (!dense) {
                uint32_t d = 4 * wa - prev;
                if (excl + cnt <= STAGE_CAP) {
                    uint32_t sa = stage + 4 * excl;
                    for (uint32_t i = wa; i < wb; i++) {
                        const uint32_t a = eva(E, 4 * i);
                        emit_word(sa, d, lds_u32(a));
                        sts_u32(a, 0);
                    }
                } else {   // this lane's codes reach past the stage
                    uint32_t idx = excl;
                    for (uint32_t i = wa; i < wb; i++) {
                        const uint32_t a = eva(E, 4 * i), w = lds_u32(a);
    #pragma unroll
                        for (uint32_t k = 0; k < 4; k++) {
                            const uint32_t code = (w >> (8 * k)) & 0xFFu;
                            if (code > 3) {
                                const uint32_t v = (code << 16) | d;
                                if (idx < STAGE_CAP) sts_u32(stage + 4 * idx, v);
                                else spill[idx - STAGE_CAP] = v;
                                idx++;
                            }
                            d = code ? 1u : d + 1;
                        }
                        sts_u32(a, 0);
                    }
                }
            } else if (fast_total <= STAGE_CAP) {
                split = fast_total;
                uint32_t d = 4 * wa - prev, sa = stage + 4 * excl;
                for (uint32_t i = wa; i < wb; i++) {
                    const uint32_t a = eva(E, 4 * i);
                    emit_word(sa, d, lds_u32(a));
                    sts_u32(a, 0);
                }
            } else {
                // all lanes one loop through generic pointers: excl + cnt ascends
                // with the lane, so the lanes that fit the stage are a prefix; the
                // others write the spill slot from the first misfit lane's index on
                uint32_t d = 4 * wa - prev;
                const uint32_t fit = __popc(__ballot_sync(0xffffffffu, excl + cnt <= STAGE_CAP));
                split = fit == 32 ? fast_total : __shfl_sync(0xffffffffu, excl, fit & 31u);
                uint32_t *gp = (uint32_t)lane < fit ? reinterpret_cast<uint32_t *>(smem + (stage - sbase)) + excl
                                                    : spill + (excl - split);
                for (uint32_t i = wa; i < wb; i++) {
                    const uint32_t a = eva(E, 4 * i), w = lds_u32(a);
#pragma unroll
                    for (uint32_t k = 0; k < 4; k++) {
                        const uint32_t c = (w >> (8 * k)) & 0xFFu;
                        if (c > 3) *gp++ = (c << 16) | d;
                        d = c ? 1u : d + 1u;
                    }
                    sts_u32(a, 0);
                }
            }
        }
        __syncwarp();
        if (defer) {
            pend.tile = tile;
            pend.staged = dense ? fast_total | (split << 16) : fast_total;
            pend.fail = fpos;
            pend.agg = agg;
            pend.doc = doc;
            pend.dtile = dtile;
            pend.kmap_s = E.kmap_s;
        } else {
            copy_stage<dense ? 4 : 2>(P, E.kmap_s, stage, spill, split, fast_total, G);
            if (do_long && lane == 0) {
                uint64_t f2;
                generic_chunk<FORM>(E, long_s1 - 1, &f2, P.out_kinds, P.out_lens, P.cap, G + fast_total);
            }
            __syncwarp();
        }
    }
    if (pend.tile != NONE) {
        uint64_t G = 0;
        if (resolve_tile(P, pend.tile, G)) {
            report_failure<BATCH>(P, pend.tile, pend.fail, G, pend.agg, pend.doc, pend.dtile);
            copy_stage<dense ? 4 : 2>(P, pend.kmap_s, stage, spill, dense ? pend.staged >> 16 : STAGE_CAP,
                       dense ? pend.staged & 0xFFFFu : pend.staged, G);
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
constexpr uint32_t SMEM_BUDGET = 227 * 1024;   // dynamic shared memory one CTA may use

template <int FORM, bool BATCH>
int occupancy_of(uint32_t threads, uint32_t smem, int *o)
{
    cudaError_t e = cudaFuncSetAttribute(lex_warps<FORM, BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         SMEM_BUDGET);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(o, lex_warps<FORM, BATCH>, threads, smem);
    return e == cudaSuccess ? LX_OK : LX_E_CUDA;
}

int warp_occupancy(lx_ctx *c, int form, bool batch, uint32_t threads, uint32_t smem, int *occ)
{
    const uint64_t key = (3ull << 62) | ((uint64_t)threads << 40) | ((uint64_t)batch << 36) | ((uint64_t)form << 32) |
                         smem;
    for (auto &kv : c->occupancy)
        if (kv.first == key) {
            *occ = kv.second;
            return LX_OK;
        }
    int o = 0, rc;
    if (batch) {
        rc = occupancy_of<FORM_CLASS, true>(threads, smem, &o);
    } else {
        switch (form) {
        case FORM_BYTE: rc = occupancy_of<FORM_BYTE, false>(threads, smem, &o); break;
        case FORM_CLASS: rc = occupancy_of<FORM_CLASS, false>(threads, smem, &o); break;
        case FORM_BYTE | WIN: rc = occupancy_of<FORM_BYTE | WIN, false>(threads, smem, &o); break;
        case FORM_CLASS | WIN: rc = occupancy_of<FORM_CLASS | WIN, false>(threads, smem, &o); break;
        case FORM_BYTE | DENSE: rc = occupancy_of<FORM_BYTE | DENSE, false>(threads, smem, &o); break;
        case FORM_CLASS | DENSE: rc = occupancy_of<FORM_CLASS | DENSE, false>(threads, smem, &o); break;
        case FORM_BYTE | WIN | DENSE: rc = occupancy_of<FORM_BYTE | WIN | DENSE, false>(threads, smem, &o); break;
        case FORM_CLASS | WIN | DENSE: rc = occupancy_of<FORM_CLASS | WIN | DENSE, false>(threads, smem, &o); break;
        default: return LX_E_INVAL;
        }
    }
    if (rc != LX_OK) return rc;
    if (o < 1) return LX_E_TOOBIG;
    c->occupancy.emplace_back(key, o);
    *occ = o;
    return LX_OK;
}

// Warps per CTA next to a table blob of `blob_bytes`: as many as the shared
// memory budget holds, at most MAX_WARPS (or the context's setting).
uint32_t warps_for(uint32_t want, uint32_t blob_bytes, uint32_t *smem, bool dense = false)
{
    const uint32_t WAREA = dense ? Geo<DENSE>::WAREA : Geo<0>::WAREA;
    const uint32_t fixed = 512 + blob_bytes + 16;
    if (fixed + WAREA > SMEM_BUDGET) return 0;
    uint32_t nw = std::min<uint32_t>(MAX_WARPS, (SMEM_BUDGET - fixed) / WAREA);
    if (want) nw = std::min<uint32_t>(nw, want);
    *smem = fixed + nw * WAREA;
    return nw;
}

// One warp per document writes the document's index over its tiles.
__global__ void bt_tile_docs(const WDoc *docs, uint32_t n_docs, uint32_t *tile_doc)
{
    const uint32_t lane = threadIdx.x & 31u, nw = gridDim.x * (blockDim.x / 32u);
    for (uint32_t d = (blockIdx.x * blockDim.x + threadIdx.x) / 32u; d < n_docs; d += nw) {
        const WDoc D = docs[d];
        const uint32_t nt = (uint32_t)((D.n + WT - 1) / WT);
        for (uint32_t k = lane; k < nt; k += 32) tile_doc[D.first_tile + k] = d;
    }
}

// The async variant's status from the launch record.
__global__ void as_finish(const WResult *r, uint64_t n, uint64_t cap, lx_async_result *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    lx_async_result o{LX_OK, 0, r->total, n};
    if (r->inv_fail_pos) {
        o.consumed = ~r->inv_fail_pos;
        o.n_tokens = ~r->inv_fail_tok;
    }
    if (r->error & ERR_TIMEOUT) o.status = LX_E_TIMEOUT;
    else if (r->error & ERR_SMEM) o.status = LX_E_TOOBIG;
    else if (r->error) o.status = LX_E_CUDA;
    else if (o.n_tokens > cap) o.status = LX_E_CAPACITY;
    *out = o;
}

}  // namespace

// True when lx_lex can take the warp-tile kernel for this call.
bool warp_path_ok(const lx_tokenset *ts, int mode, const uint8_t *d_in)
{
    return ts->walk[mode].status == LX_OK && (reinterpret_cast<uintptr_t>(d_in) & 15u) == 0;
}

namespace {

// One input's launch: parameters, zeroed scratch size and shape.
struct WarpLaunch {
    WParams P;
    uint32_t grid = 0, nwarps = 0, smem = 0;
    size_t need = 0;
    int form = FORM_BYTE;
    bool dense = false;
};

// The geometry of the next call on (ts, mode): the context's setting, else
// what the last call on them showed (sparse until one has run).
bool warp_dense(const lx_ctx *c, const lx_tokenset *ts, int mode)
{
    if (c->warp_geometry != LX_WARP_GEOMETRY_AUTO) return c->warp_geometry == LX_WARP_GEOMETRY_DENSE;
    const uint64_t key = ts->serial * 8 + (uint64_t)mode;
    for (const auto &kv : c->warp_dense)
        if (kv.first == key) return kv.second;
    return false;
}

// After a call of n_tiles tiles: the dense geometry pays where the tiles
// hold more kept tokens on average than the sparse stage, or where more than
// one tile in 20 000 has its last chunk end past the sparse halo (every such
// tile walks that chunk byte by byte while every later tile waits for its count).
void note_geometry(lx_ctx *c, const lx_tokenset *ts, int mode, uint64_t tokens, uint64_t n_tiles, uint32_t long_tiles)
{
    const bool dense = tokens > (uint64_t)Geo<0>::STAGE_CAP * n_tiles || (uint64_t)long_tiles * 20000 > n_tiles;
    const uint64_t key = ts->serial * 8 + (uint64_t)mode;
    for (auto &kv : c->warp_dense)
        if (kv.first == key) {
            kv.second = dense;
            return;
        }
    c->warp_dense.emplace_back(key, dense);
}

// The spill slots of a launch of `grid` CTAs of `nwarps` warps (uninitialised).
int warp_spill(lx_ctx *c, uint32_t grid, uint32_t nwarps, uint32_t **out)
{
    const int rc = grow(&c->w_spill, &c->w_spill_bytes, sizeof(uint32_t) * SPILL_CAP * (size_t)grid * nwarps);
    *out = static_cast<uint32_t *>(c->w_spill);
    return rc;
}

int warp_prepare(lx_ctx *c, const lx_tokenset *ts, const uint8_t *d_in, uint64_t n, int mode, uint16_t *d_kinds,
                 uint32_t *d_lens, uint64_t capacity, uint64_t sparse_limit, WarpLaunch &L)
{
    const WalkTable &w = ts->walk[mode];
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != c->device) return LX_E_INVAL;
    DeviceTables dt;
    int rc = ensure_device_tables(ts, dev, &dt);
    if (rc != LX_OK) return rc;
    const uint64_t n_tiles64 = (n + WT - 1) / WT;
    if (n_tiles64 > 0xFFFFFFF0ull) return LX_E_INVAL;
    const uint32_t n_tiles = (uint32_t)n_tiles64;
    L.dense = warp_dense(c, ts, mode);
    L.nwarps = warps_for(warps_setting(c, ts, mode), (uint32_t)w.blob.size(), &L.smem, L.dense);
    if (L.nwarps < 1) return LX_E_TOOBIG;
    L.form = w.form | (w.n_ctx ? WIN : 0) | (L.dense ? DENSE : 0);
    int occ = 0;
    rc = warp_occupancy(c, L.form, false, 32 * L.nwarps, L.smem, &occ);
    if (rc != LX_OK) return rc;
    L.grid = (uint32_t)std::min<uint64_t>((uint64_t)occ * c->num_sms, (n_tiles + L.nwarps - 1) / L.nwarps);

    const uint32_t n_groups = (n_tiles + GS - 1) / GS;
    const size_t o_gstatus = 64 + 8 * (size_t)n_tiles, o_gdone = o_gstatus + 8 * (size_t)n_groups;
    L.need = o_gdone + 4 * (size_t)n_groups;   // zeroed per call
    rc = grow(&c->scratch, &c->scratch_bytes, L.need);
    if (rc != LX_OK) return rc;
    uint8_t *scr = static_cast<uint8_t *>(c->scratch);
    WParams &P = L.P;
    P = WParams{};
    rc = warp_spill(c, L.grid, L.nwarps, &P.spill);
    if (rc != LX_OK) return rc;
    P.in = d_in;
    P.n = n;
    P.blob = static_cast<const uint8_t *>(dt.d_walk[mode]);
    P.blob_bytes = (uint32_t)w.blob.size();
    P.rows_bytes = w.rows_bytes;
    P.row_shift = w.row_shift;
    P.p_start = w.p_start;
    P.p_pre = w.p_pre;
    P.acc_off = w.acc_off;
    P.kmap_off = w.kmap_off;
    P.cmap_off = w.cmap_off;
    P.cut_off = w.cut_off;
    P.ctx_off = w.ctx_off;
    P.n_ctx = w.n_ctx;
    P.out_kinds = d_kinds;
    P.out_lens = d_lens;
    P.cap = capacity;
    P.res = reinterpret_cast<WResult *>(scr);
    P.tile_counter = reinterpret_cast<unsigned int *>(scr + sizeof(WResult));
    P.status = reinterpret_cast<unsigned long long *>(scr + 64);
    P.gstatus = reinterpret_cast<unsigned long long *>(scr + o_gstatus);
    P.gdone = reinterpret_cast<unsigned int *>(scr + o_gdone);
    P.n_tiles = n_tiles;
    P.timeout_ns = c->timeout_ns;
    P.withhold = c->withhold;
    P.sparse_limit = sparse_limit;
    static_assert(sizeof(WResult) == 48 && sizeof(WResult) + 4 <= 64 && sizeof(WResult) <= LAUNCH_RECORD_BYTES,
                  "record layout");
    return LX_OK;
}

void warp_launch(const WarpLaunch &L, cudaStream_t st)
{
#define LXW_LAUNCH(F) \
    case F: lex_warps<F, false><<<L.grid, 32 * L.nwarps, L.smem, st>>>(L.P); break;
    switch (L.form) {
        LXW_LAUNCH(FORM_BYTE)
        LXW_LAUNCH(FORM_CLASS)
        LXW_LAUNCH(FORM_BYTE | WIN)
        LXW_LAUNCH(FORM_CLASS | WIN)
        LXW_LAUNCH(FORM_BYTE | DENSE)
        LXW_LAUNCH(FORM_CLASS | DENSE)
        LXW_LAUNCH(FORM_BYTE | WIN | DENSE)
        LXW_LAUNCH(FORM_CLASS | WIN | DENSE)
    default: break;
    }
#undef LXW_LAUNCH
}

}  // namespace

int lex_warp_device(lx_ctx *c, const lx_tokenset *ts, const uint8_t *d_in, uint64_t n, int mode, uint16_t *d_kinds,
                    uint32_t *d_lens, uint64_t capacity, uint64_t *n_tokens, uint64_t *consumed, cudaStream_t st,
                    uint64_t sparse_limit)
{
    if (n == 0) {
        *n_tokens = 0;
        *consumed = 0;
        return LX_OK;
    }
    WarpLaunch L;
    int rc = warp_prepare(c, ts, d_in, n, mode, d_kinds, d_lens, capacity, sparse_limit, L);
    if (rc != LX_OK) return rc;
    rc = cuda_err(cudaMemsetAsync(c->scratch, 0, L.need, st));
    if (rc != LX_OK) return rc;
    if (c->timing) cudaEventRecord(c->ev[0], st);
    warp_launch(L, st);
    rc = cuda_err(cudaGetLastError());
    if (c->timing) cudaEventRecord(c->ev[1], st);
    if (rc != LX_OK) return rc;
    rc = cuda_err(cudaMemcpyAsync(c->h_res, L.P.res, sizeof(WResult), cudaMemcpyDeviceToHost, st));
    if (rc == LX_OK) rc = cuda_err(cudaStreamSynchronize(st));
    if (rc != LX_OK) return rc;
    const WResult r = *static_cast<const WResult *>(c->h_res);
    if (r.error & ERR_LOOKAHEAD) return LX_LOOKAHEAD;
    if (r.error == 0 && c->warp_geometry == LX_WARP_GEOMETRY_AUTO)
        note_geometry(c, ts, mode, r.total, L.P.n_tiles, r.long_tiles);
    if (r.error & ERR_SPARSE) return LX_SPARSE;
    if (r.error & ERR_TIMEOUT) return LX_E_TIMEOUT;
    if (r.error & ERR_SMEM) return LX_E_TOOBIG;
    uint64_t tokens = r.total, con = n;
    if (r.inv_fail_pos) {
        con = ~r.inv_fail_pos;
        tokens = ~r.inv_fail_tok;
    }
    *n_tokens = tokens;
    *consumed = con;
    return tokens > capacity ? LX_E_CAPACITY : LX_OK;
}

int lex_warp_async(lx_ctx *c, const lx_tokenset *ts, const uint8_t *d_in, uint64_t n, int mode, uint16_t *d_kinds,
                   uint32_t *d_lens, uint64_t capacity, lx_async_result *d_result, cudaStream_t st)
{
    if (n == 0) {
        const lx_async_result z{LX_OK, 0, 0, 0};
        return cuda_err(cudaMemcpyAsync(d_result, &z, sizeof z, cudaMemcpyHostToDevice, st));
    }
    WarpLaunch L;
    int rc = warp_prepare(c, ts, d_in, n, mode, d_kinds, d_lens, capacity, 0, L);
    if (rc != LX_OK) return rc;
    rc = cuda_err(cudaMemsetAsync(c->scratch, 0, L.need, st));
    if (rc != LX_OK) return rc;
    warp_launch(L, st);
    as_finish<<<1, 32, 0, st>>>(L.P.res, n, capacity, d_result);
    return cuda_err(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// host buffers: pieces copied in, lexed and copied out in a pipeline
// ---------------------------------------------------------------------------
namespace {

// A launch record into pinned host memory by a one-warp kernel rather than a
// device-to-host copy, which would queue on the copy engine behind the
// previous piece's tokens.
__global__ void copy_wrecord(const WResult *src, WResult *dst)
{
    if (threadIdx.x < sizeof(WResult) / 8)
        reinterpret_cast<volatile unsigned long long *>(dst)[threadIdx.x] =
            reinterpret_cast<const volatile unsigned long long *>(src)[threadIdx.x];
}

}  // namespace

int lex_warp_host(lx_ctx *c, const lx_tokenset *ts, const uint8_t *h_in, uint64_t n, int mode, uint16_t *h_kinds,
                  uint32_t *h_lens, uint64_t capacity, const uint64_t *b, uint32_t K, uint64_t *n_tokens,
                  uint64_t *consumed, cudaStream_t st, uint64_t sparse_limit)
{
    auto al = [](uint64_t x, uint64_t a) { return (x + a - 1) / a * a; };
    // device layout: piece i's bytes at a 16-byte aligned offset; its tokens
    // (at most one per byte) in its own output range, 4-token aligned
    std::vector<uint64_t> in_off(K), out_off(K), cap(K);
    uint64_t in_total = 0, out_total = 0, largest = 0;
    uint32_t big = 0;
    for (uint32_t i = 0; i < K; i++) {
        const uint64_t len = b[i + 1] - b[i];
        in_off[i] = in_total;
        in_total = al(in_total + len, 16);
        cap[i] = al(len + 1, 4);
        out_off[i] = out_total;
        out_total += cap[i];
        if (len > largest) largest = len, big = i;
    }
    int rc = grow(&c->d_in, &c->d_in_bytes, in_total + 16);
    if (rc == LX_OK) rc = grow(&c->d_out, &c->d_out_bytes, 6 * out_total + 64);
    if (rc == LX_OK) rc = grow_host(&c->h_scratch, &c->h_scratch_bytes, sizeof(WResult) * (size_t)K);
    if (rc != LX_OK) return rc;
    uint8_t *d_in = static_cast<uint8_t *>(c->d_in);
    uint32_t *d_lens = static_cast<uint32_t *>(c->d_out);
    uint16_t *d_kinds = reinterpret_cast<uint16_t *>(d_lens + out_total);
    WResult *h_res = static_cast<WResult *>(c->h_scratch);
    WResult *h_res_dev = nullptr;   // the same pinned records, as the device sees them
    if (cudaHostGetDevicePointer(reinterpret_cast<void **>(&h_res_dev), c->h_scratch, 0) != cudaSuccess)
        return LX_E_CUDA;
    // the scratch and spill slots grow for the largest piece first: no
    // reallocation once launches are queued
    WarpLaunch L;
    rc = warp_prepare(c, ts, d_in + in_off[big], largest, mode, d_kinds + out_off[big], d_lens + out_off[big],
                      cap[big], sparse_limit, L);
    if (rc != LX_OK) return rc;
    const bool dense = L.dense;
    // the pieces in, each on its own event
    for (uint32_t i = 0; i < K; i++) {
        rc = cuda_err(cudaMemcpyAsync(d_in + in_off[i], h_in + b[i], b[i + 1] - b[i], cudaMemcpyHostToDevice, c->s_in));
        if (rc == LX_OK) rc = cuda_err(cudaEventRecord(c->ev_in[i], c->s_in));
        if (rc != LX_OK) return rc;
    }
    // the launches, in order on the caller's stream (one scratch, reused)
    if (c->timing) cudaEventRecord(c->ev[0], st);
    for (uint32_t i = 0; i < K; i++) {
        rc = warp_prepare(c, ts, d_in + in_off[i], b[i + 1] - b[i], mode, d_kinds + out_off[i], d_lens + out_off[i],
                          cap[i], sparse_limit, L);
        if (rc == LX_OK && L.dense != dense) rc = LX_E_CUDA;   // one geometry per call
        if (rc == LX_OK) rc = cuda_err(cudaStreamWaitEvent(st, c->ev_in[i], 0));
        if (rc == LX_OK) rc = cuda_err(cudaMemsetAsync(c->scratch, 0, L.need, st));
        if (rc != LX_OK) return rc;
        warp_launch(L, st);
        copy_wrecord<<<1, 32, 0, st>>>(L.P.res, h_res_dev + i);
        rc = cuda_err(cudaGetLastError());
        if (rc == LX_OK) rc = cuda_err(cudaEventRecord(c->ev_lex[i], st));
        if (rc != LX_OK) return rc;
    }
    if (c->timing) cudaEventRecord(c->ev[1], st);
    // each piece's tokens out as soon as it is lexed, after the previous pieces'
    uint64_t out = 0, con = n, tokens = 0, n_tiles = 0;
    uint32_t long_tiles = 0;
    bool failed = false;
    for (uint32_t i = 0; i < K && !failed && rc == LX_OK; i++) {
        rc = cuda_err(cudaEventSynchronize(c->ev_lex[i]));
        if (rc != LX_OK) break;
        const WResult r = h_res[i];
        if (r.error & ERR_LOOKAHEAD) rc = LX_LOOKAHEAD;   // the caller lexes the input another way
        else if (r.error & ERR_SPARSE) rc = LX_SPARSE;
        else if (r.error & ERR_TIMEOUT) rc = LX_E_TIMEOUT;
        else if (r.error) rc = LX_E_TOOBIG;
        if (rc != LX_OK) break;
        uint64_t m = r.total;
        if (r.inv_fail_pos) {   // Corollary 1: the first failing piece ends the stream
            m = ~r.inv_fail_tok;
            con = b[i] + ~r.inv_fail_pos;
            failed = true;
        }
        const uint64_t lo = std::min(out, capacity), hi = std::min(out + m, capacity);
        if (hi > lo) {
            rc = cuda_err(cudaMemcpyAsync(h_kinds + lo, d_kinds + out_off[i], (hi - lo) * 2, cudaMemcpyDeviceToHost,
                                          c->s_out));
            if (rc == LX_OK)
                rc = cuda_err(cudaMemcpyAsync(h_lens + lo, d_lens + out_off[i], (hi - lo) * 4,
                                              cudaMemcpyDeviceToHost, c->s_out));
        }
        out += m;
        tokens += r.total;
        n_tiles += (b[i + 1] - b[i] + WT - 1) / WT;
        long_tiles += r.long_tiles;
    }
    int r2 = cuda_err(cudaStreamSynchronize(c->s_out));
    if (rc == LX_OK) rc = r2;
    r2 = cuda_err(cudaStreamSynchronize(st));
    if (rc == LX_OK) rc = r2;
    if (rc != LX_OK) return rc;
    if (!failed && c->warp_geometry == LX_WARP_GEOMETRY_AUTO) note_geometry(c, ts, mode, tokens, n_tiles, long_tiles);
    *n_tokens = out;
    *consumed = con;
    return out > capacity ? LX_E_CAPACITY : LX_OK;
}

// ---------------------------------------------------------------------------
// batches: every document of every token set in one launch
// ---------------------------------------------------------------------------
namespace {

// The combined table of a batch's token sets (class form): all rows first,
// each set's entries moved by its row offset, then one acceptance byte per
// row, then per set its kind map, class map (256-aligned) and cut map, then
// the WSet array.
struct Combined {
    std::vector<uint8_t> blob;
    uint32_t rows_bytes = 0, acc_off = 0, sets_off = 0;
};

const WalkTable *class_walk(const lx_tokenset *ts, int mode)
{
    const WalkTable &w = ts->walk[mode];
    if (w.status == LX_OK && w.form == FORM_CLASS) return &w;
    const WalkTable &wc = ts->walk_cls[mode];
    return wc.status == LX_OK ? &wc : nullptr;
}

// Rows of all sets must share one 16-bit shared-address window; the first
// kilobyte of the window may be reserved.
constexpr uint32_t BATCH_ROWS_MAX = 65536 - 1024;

int combine(const lx_tokenset *const *sets, uint32_t n_sets, int mode, Combined &out)
{
    auto al = [](uint32_t x, uint32_t a) { return (x + a - 1) / a * a; };
    std::vector<const WalkTable *> w(n_sets);
    uint32_t rows = 0;
    for (uint32_t s = 0; s < n_sets; s++) {
        w[s] = class_walk(sets[s], mode);
        if (!w[s] || w[s]->n_ctx) return LX_E_TOOBIG;   // tables with split-window contexts stay single
        rows += w[s]->rows_bytes;
    }
    if (rows > BATCH_ROWS_MAX) return LX_E_TOOBIG;
    const uint32_t n_rows = rows >> 8;
    out.rows_bytes = rows;
    out.acc_off = rows;
    uint32_t o = al(rows + n_rows, 256);
    std::vector<uint32_t> base(n_sets), maps(n_sets);
    uint32_t rb = 0;
    for (uint32_t s = 0; s < n_sets; s++) {
        base[s] = rb;
        rb += w[s]->rows_bytes;
        maps[s] = o;   // kmap (256 B), cmap (256 B, 256-aligned), cut (256 B), context map (256 B, zero)
        o += 1024;
    }
    out.sets_off = o;
    out.blob.assign(al(o + (uint32_t)sizeof(WSet) * n_sets, 16), 0);
    std::vector<WSet> ws(n_sets);
    for (uint32_t s = 0; s < n_sets; s++) {
        const WalkTable &t = *w[s];
        const uint16_t *src = reinterpret_cast<const uint16_t *>(t.blob.data());
        uint16_t *dst = reinterpret_cast<uint16_t *>(out.blob.data() + base[s]);
        for (uint32_t k = 0; k < t.rows_bytes / 2; k++) dst[k] = (uint16_t)(src[k] + base[s]);   // rows move by base
        std::memcpy(out.blob.data() + out.acc_off + (base[s] >> 8), t.blob.data() + t.acc_off, t.n_rows);
        std::memcpy(out.blob.data() + maps[s], t.blob.data() + t.kmap_off, 256);
        std::memcpy(out.blob.data() + maps[s] + 256, t.blob.data() + t.cmap_off, 256);
        std::memcpy(out.blob.data() + maps[s] + 512, t.blob.data() + t.cut_off, 256);
        ws[s] = WSet{base[s] + t.p_start, base[s] + t.p_pre, base[s], maps[s], maps[s] + 256, maps[s] + 512,
                     maps[s] + 768, 0};
    }
    std::memcpy(out.blob.data() + out.sets_off, ws.data(), sizeof(WSet) * n_sets);
    return LX_OK;
}

}  // namespace

int lex_batch_warp(lx_ctx *c, const lx_tokenset *const *sets, uint32_t n_sets, const lx_doc *docs, uint32_t n_docs,
                   int mode, uint16_t *d_kinds, uint32_t *d_lens, uint64_t capacity, lx_doc_result *results,
                   uint64_t *n_total, cudaStream_t st)
{
    // applicable: class-form tables that share the address window, aligned documents
    if (n_sets == 0 || n_sets > 16) return LX_SPARSE;
    for (uint32_t i = 0; i < n_docs; i++)
        if (docs[i].n && (reinterpret_cast<uintptr_t>(docs[i].data) & 15u)) return LX_SPARSE;
    std::vector<uint64_t> key = {0xB47C4ull, (uint64_t)mode, n_sets};
    for (uint32_t s = 0; s < n_sets; s++) key.push_back(sets[s]->serial);
    if (key != c->wb_key) {
        Combined cb;
        const int rc = combine(sets, n_sets, mode, cb);
        if (rc == LX_E_TOOBIG) return LX_SPARSE;
        if (rc != LX_OK) return rc;
        int r2 = grow(&c->wb_dev, &c->wb_dev_bytes, cb.blob.size());
        if (r2 != LX_OK) return r2;
        r2 = cuda_err(cudaMemcpy(c->wb_dev, cb.blob.data(), cb.blob.size(), cudaMemcpyHostToDevice));
        if (r2 != LX_OK) return r2;
        c->wb_key = key;
        c->wb_blob_bytes = (uint32_t)cb.blob.size();
        c->wb_rows = cb.rows_bytes;
        c->wb_acc_off = cb.acc_off;
        c->wb_sets_off = cb.sets_off;
    }

    // documents in their order; empty ones take no tile
    std::vector<WDoc> hd;
    std::vector<uint32_t> idx;
    uint64_t TT = 0;
    for (uint32_t i = 0; i < n_docs; i++) {
        if (!docs[i].n) continue;
        hd.push_back(WDoc{docs[i].data, docs[i].n, (uint32_t)TT, docs[i].set});
        idx.push_back(i);
        TT += (docs[i].n + WT - 1) / WT;
        if (TT > 0xFFFFFFF0ull) return LX_E_INVAL;
    }
    if (hd.empty()) return LX_OK;
    const uint32_t D = (uint32_t)hd.size(), n_tiles = (uint32_t)TT, n_groups = (n_tiles + GS - 1) / GS;

    uint32_t smem = 0;
    const uint32_t nwarps = warps_for(c->warps, c->wb_blob_bytes, &smem);
    if (nwarps < 1) return LX_SPARSE;
    int occ = 0;
    int rc = warp_occupancy(c, FORM_CLASS, true, 32 * nwarps, smem, &occ);
    if (rc == LX_E_TOOBIG) return LX_SPARSE;
    if (rc != LX_OK) return rc;
    const uint32_t grid = (uint32_t)std::min<uint64_t>((uint64_t)occ * c->num_sms, (n_tiles + nwarps - 1) / nwarps);

    // device scratch: [zeroed: record, counter, statuses, group words, document records][documents][tile map]
    auto al = [](size_t x, size_t a) { return (x + a - 1) / a * a; };
    const size_t o_status = 64, o_gstatus = al(o_status + 8 * (size_t)n_tiles, 64);
    const size_t o_gdone = al(o_gstatus + 8 * (size_t)n_groups, 64), o_dres = al(o_gdone + 4 * (size_t)n_groups, 64);
    const size_t zero_end = o_dres + sizeof(WDocRes) * D;
    const size_t o_docs = al(zero_end, 256), o_tdoc = al(o_docs + sizeof(WDoc) * D, 256);
    const size_t dev_total = o_tdoc + 4 * (size_t)n_tiles;
    // pinned staging: documents up, then the record and the document records down
    const size_t h_down = al(sizeof(WDoc) * D, 64), host_total = h_down + zero_end;
    bool moved = false;
    {
        void *od = c->b_dev, *oh = c->b_host;
        rc = grow(&c->b_dev, &c->b_dev_bytes, dev_total);
        if (rc == LX_OK) rc = grow_host(&c->b_host, &c->b_host_bytes, host_total);
        if (rc != LX_OK) return rc;
        moved = od != c->b_dev || oh != c->b_host;
    }
    uint32_t *spill = nullptr;
    rc = warp_spill(c, grid, nwarps, &spill);
    if (rc != LX_OK) return rc;
    uint8_t *dv = static_cast<uint8_t *>(c->b_dev);
    uint8_t *hs = static_cast<uint8_t *>(c->b_host);
    std::memcpy(hs, hd.data(), sizeof(WDoc) * D);

    std::vector<uint64_t> gkey = {0xB47C5ull, D, TT, (uint64_t)mode, (uint64_t)(uintptr_t)d_kinds,
                                  (uint64_t)(uintptr_t)d_lens, capacity, (uint64_t)(uintptr_t)dv,
                                  (uint64_t)(uintptr_t)hs, c->timeout_ns, grid, nwarps,
                                  (uint64_t)(uintptr_t)c->wb_dev, (uint64_t)(uintptr_t)spill};
    gkey.insert(gkey.end(), key.begin(), key.end());
    if (moved || gkey != c->b_key || !c->b_exec) {
        if (c->b_exec) cudaGraphExecDestroy(c->b_exec);
        c->b_exec = nullptr;
        c->b_key.clear();
        if (!c->b_stream && cudaStreamCreateWithFlags(&c->b_stream, cudaStreamNonBlocking) != cudaSuccess)
            return LX_E_CUDA;
        cudaStream_t cs = c->b_stream;
        WParams P{};
        P.in = nullptr;
        P.n = 0;
        P.blob = static_cast<const uint8_t *>(c->wb_dev);
        P.blob_bytes = c->wb_blob_bytes;
        P.rows_bytes = c->wb_rows;
        P.row_shift = 8;
        P.acc_off = c->wb_acc_off;
        P.out_kinds = d_kinds;
        P.out_lens = d_lens;
        P.cap = capacity;
        P.spill = spill;
        P.res = reinterpret_cast<WResult *>(dv);
        P.tile_counter = reinterpret_cast<unsigned int *>(dv + sizeof(WResult));
        P.status = reinterpret_cast<unsigned long long *>(dv + o_status);
        P.gstatus = reinterpret_cast<unsigned long long *>(dv + o_gstatus);
        P.gdone = reinterpret_cast<unsigned int *>(dv + o_gdone);
        P.n_tiles = n_tiles;
        P.timeout_ns = c->timeout_ns;
        P.withhold = NONE;
        P.sparse_limit = 0;   // long chunks are walked byte by byte: no document leaves the launch
        P.docs = reinterpret_cast<const WDoc *>(dv + o_docs);
        P.tile_doc = reinterpret_cast<const uint32_t *>(dv + o_tdoc);
        P.dres = reinterpret_cast<WDocRes *>(dv + o_dres);
        P.sets_off = c->wb_sets_off;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return LX_E_CUDA;
        cudaMemsetAsync(dv, 0, zero_end, cs);
        cudaMemcpyAsync(dv + o_docs, hs, sizeof(WDoc) * D, cudaMemcpyHostToDevice, cs);
        bt_tile_docs<<<(D + 7) / 8, 256, 0, cs>>>(P.docs, D, const_cast<uint32_t *>(P.tile_doc));
        lex_warps<FORM_CLASS, true><<<grid, 32 * nwarps, smem, cs>>>(P);
        cudaMemcpyAsync(hs + h_down, dv, zero_end, cudaMemcpyDeviceToHost, cs);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&c->b_exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            c->b_exec = nullptr;
            cudaGetLastError();
            return LX_E_CUDA;
        }
        c->b_key = gkey;
    }
    if (c->timing) cudaEventRecord(c->ev[0], st);
    rc = cuda_err(cudaGraphLaunch(c->b_exec, st));
    if (c->timing) cudaEventRecord(c->ev[1], st);
    if (rc == LX_OK) rc = cuda_err(cudaStreamSynchronize(st));
    if (rc != LX_OK) return rc;

    const WResult r = *reinterpret_cast<const WResult *>(hs + h_down);
    if (r.error & ERR_TIMEOUT) return LX_E_TIMEOUT;
    if (r.error & ERR_SMEM) return LX_SPARSE;   // the rows did not fit the window after all
    if (r.error) return LX_E_CUDA;
    const WDocRes *dres = reinterpret_cast<const WDocRes *>(hs + h_down + o_dres);
    for (uint32_t j = 0; j < D; j++) {
        const WDocRes &x = dres[j];
        lx_doc_result &o = results[idx[j]];
        if (x.out_off1 == 0) return LX_E_CUDA;   // every document's first tile reports its offset
        o.out_off = x.out_off1 - 1;
        if (x.inv_fail_pos) {
            o.consumed = ~x.inv_fail_pos;
            o.n_tokens = ~x.inv_fail_tok - o.out_off;
        } else {
            o.consumed = hd[j].n;
            o.n_tokens = x.total;
        }
    }
    *n_total = r.total;
    return r.total > capacity ? LX_E_CAPACITY : LX_OK;
}

}  // namespace lx
