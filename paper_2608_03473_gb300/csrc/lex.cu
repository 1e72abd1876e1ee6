// lex.cu -- GB300 (sm_103a) certified-split lexing: the tile kernel and the
// lx_lex / lx_ctx entry points.
//
// One persistent CTA per resident slot loops over tiles of TILE input bytes.
// Per tile:
//   (a) stage: a 1-D bulk copy (cp.async.bulk, TMA) brings the tile plus a
//       halo into shared memory; it is issued as soon as the previous tile's
//       aggregate is published, so it overlaps that tile's output writes;
//   (b) plan:  each of NT threads owns the equal-division target of its
//       SEG-byte segment and slides it forward to the first byte of the
//       mode's certified set in the segment (the planner of Section 6 with
//       k = one target per thread); a segment holding no certified byte
//       yields no chunk and the previous chunk runs on;
//   (c) walk:  all lanes run the longest-match loop of Section 3 in lockstep
//       over the shared-memory walk table (internal.h), every certified byte
//       ending the token in progress, each from its chunk start to the next
//       chunk start (or the end of the input); token ends go to per-thread
//       record columns, compacted in place and spilled to a per-CTA global
//       region when a range has more tokens than a column holds;
//   (d) emit:  a CTA scan of kept-token counts, the tile's aggregate published
//       at once for a decoupled look-back over per-tile status words; the
//       kept tokens wait in a shared stage and are written (coalesced kinds
//       u16, lengths u32) one iteration later, once the look-back has
//       resolved the tile's output offset.  The first lexing failure
//       (Corollary 1) is combined with device atomics.
// Every device-side wait is bounded by a %globaltimer budget.

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>

#include "devutil.cuh"
#include "internal.h"
#include "runtime.h"

namespace lx {

constexpr int NT = 256;                 // threads per CTA
constexpr int NW = NT / 32;
constexpr int SEG = 68;                 // bytes per thread target (17 words: odd stride)
constexpr int TILE = NT * SEG;          // 17408 input bytes per tile
constexpr int HALO = 1024;              // extra staged bytes for ranges that run past the tile
constexpr int BUF = TILE + HALO;        // 18432, a multiple of 16
constexpr uint32_t KS_DEFAULT = 40;     // token-end records per thread (the column height), unless tuned
constexpr uint32_t KS_MIN = LX_KS_MIN;  // make_room needs half a column of at least 8 words
constexpr int STAGE_CAP = 4096;         // kept tokens per tile that take the deferred coalesced path
constexpr int SPILL_WORDS = 8192;       // global spill region per CTA (kept tokens of long ranges)
constexpr uint64_t NOPOS = ~0ull;
constexpr uint32_t NONE32 = 0xFFFFFFFFu;

constexpr unsigned ERR_TIMEOUT = 1u;
constexpr unsigned ERR_SMEM = 2u;


// One launch's record.  With a single document it is also that document's
// record (the first three fields are laid out as in DocResult).
struct Result {
    unsigned long long total;          // kept tokens over all chunks (atomicAdd)
    unsigned long long inv_fail_pos;   // ~min failure offset (atomicMax), 0 = none
    unsigned long long inv_fail_tok;   // ~min output index at the failure
    unsigned int error;
    unsigned int pad;
};

// A document of a batched launch: its tiles are consecutive in the launch's
// tile sequence, starting at first_tile.
struct DocDesc {
    const uint8_t *in;
    uint64_t n;
    uint32_t first_tile;
    uint32_t tma;           // input 16-byte aligned: tiles are staged by TMA
};

struct DocResult {
    unsigned long long total;          // kept tokens of the document, including any after a failure
    unsigned long long inv_fail_pos;   // ~min failure offset within the document, 0 = none
    unsigned long long inv_fail_tok;   // ~min output index at the failure
    unsigned long long out_off1;       // output index of its first token + 1 (0 = not yet written)
};

struct Params {
    DocDesc one;                 // the document when docs == nullptr
    const DocDesc *docs;         // batched: documents of this launch
    const uint32_t *tile_doc;    // batched: document index of every tile
    DocResult *dres;             // batched: per-document records
    const Result *prev;          // batched: records of the launches before this one
    uint32_t n_prev;             // (their token totals offset this launch's output)
    const uint8_t *blob;
    uint32_t blob_bytes, table_bytes, kind_off, cmap_off, cert_off;
    uint32_t ncols;
    uint32_t p_start, p_flag, p_slow, p_pre;
    uint16_t *out_kinds;
    uint32_t *out_lens;
    uint64_t cap;
    unsigned long long *status;
    unsigned int *tile_counter;
    Result *res;
    uint32_t n_tiles;
    uint64_t timeout_ns;
    uint32_t *spill;       // per-CTA spill regions for long ranges' kept tokens
    uint32_t spill_cap;    // words per CTA (0: no spilling)
    uint32_t ks;           // record column height (words per thread)
    uint32_t withhold;     // failure-detection tests: this tile never publishes (NONE32: off)
};

// ---- shared-memory layout (bytes from the dynamic shared base) ----
// [walk tables][input tile + halo, one TMA buffer][per-lane record columns]
// [stage: the previous tile's kept tokens, waiting for its output offset][misc]
struct Layout {
    uint32_t buf, slots, stage, misc, total;
};

__host__ __device__ inline uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) & ~(a - 1); }

__host__ __device__ inline Layout make_layout(uint32_t blob_bytes, uint32_t ks)
{
    Layout L;                                    // blob first: + up to 511 bytes to 512-align the table
    L.buf = align_up(512 + blob_bytes, 128);
    L.slots = L.buf + BUF;
    L.stage = L.slots + ks * NT * 4;
    L.misc = L.stage + STAGE_CAP * 4;
    L.total = L.misc + 256 + 12 * NW;
    return L;
}

// misc region offsets
constexpr uint32_t M_WARP = 256;    // u64[NW] warp totals -> exclusive offsets
constexpr uint32_t M_MBAR = 64;     // u64
constexpr uint32_t M_TILE = 80;     // u32: next tile id
constexpr uint32_t M_X = 84;        // u32: first cut at or past the tile end (relative)
constexpr uint32_t M_G = 96;        // u64: resolved output offset
constexpr uint32_t M_TOT = 104;     // u64: this tile's kept total
constexpr uint32_t M_FPOS = 112;    // u64: this tile's first failure offset (NOPOS = none)
constexpr uint32_t M_FIDX = 120;    // u64: kept tokens before it, within the tile
constexpr uint32_t M_WMIN = 256 + 8 * NW;   // u32[NW]: per-warp minimum chunk start
constexpr uint32_t M_PTILE = 160;   // u32: pending tile (NONE32 = none)
constexpr uint32_t M_PTOT = 168;    // u64: pending tile's kept total
constexpr uint32_t M_PFPOS = 176;   // u64: pending tile's failure offset
constexpr uint32_t M_PFIDX = 184;   // u64: pending tile's kept tokens before the failure
constexpr uint32_t M_FLAGS = 192;   // u32: this tile: bit0 synchronous
constexpr uint32_t M_SPILL = 196;   // u32: words of this CTA's spill region used by this tile
constexpr uint32_t M_PDOC = 200;    // u32: pending tile's document
constexpr uint32_t M_PFIRST = 204;  // u32: pending tile is its document's first
constexpr uint32_t M_TREF = 208;    // TileRef of the claimed tile (40 bytes)

// ---- PTX helpers (shared ones in devutil.cuh) ----
__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Thread 0 only: bulk-copy `bytes` (multiple of 16, both addresses 16-aligned)
// global -> shared, completing on `mbar`.
__device__ __forceinline__ void tma_load(uint32_t dst, const uint8_t *src, uint32_t bytes, uint32_t mbar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
    for (uint32_t o = 0; o < bytes; o += 8192) {
        uint32_t sz = bytes - o < 8192 ? bytes - o : 8192;
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst + o),
            "l"(src + o), "r"(sz), "r"(mbar)
            : "memory");
    }
}
// Bounded wait on an mbarrier phase; false when the time budget runs out.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, uint64_t timeout_ns)
{
    uint64_t t0 = 0;
    for (uint32_t it = 0;; it++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 15) == 0) {
            uint64_t t = globaltimer();
            if (it == 0) t0 = t;
            else if (t - t0 > timeout_ns) return false;
        }
    }
}

// ---- tables ----
struct Env {
    uint32_t buf;          // shared address of the staged tile
    uint64_t tile_base;    // input offset of buf[0]
    uint64_t sm_end;       // input offset one past the last staged byte
    const uint8_t *in;
    uint64_t n;
    uint32_t P_start, P_flag, P_slow, P_pre;
    uint32_t tbase, kind_s, cmap_s, cert_s, kcol2;
    uint32_t *spill;            // this CTA's spill region (global)
    uint32_t spill_cap;         // its size in words
    uint32_t ks;                // record column height
    unsigned *spill_used;       // shared allocation counter, reset per tile
};

__device__ __forceinline__ uint32_t byte_at(const Env &E, uint64_t p)
{
    return p < E.sm_end ? lds_u8(E.buf + (uint32_t)(p - E.tile_base)) : (uint32_t)__ldg(E.in + p);
}

template <int FORM>
__device__ __forceinline__ uint32_t step(const Env &E, uint32_t e, uint32_t b)
{
    if (FORM == FORM_BYTE) return lds_u16(e ^ (b << 1));
    uint32_t c = lds_u8(E.cmap_s + b);
    return lds_u16(e + (c << 1));
}

// Step on byte K of a little-endian word: the byte-indexed form folds the
// extraction and the row address into one shift and one LOP3.
template <int FORM, int K>
__device__ __forceinline__ uint32_t step_w(const Env &E, uint32_t e, uint32_t w)
{
    if (FORM == FORM_BYTE) {
        uint32_t x = K == 0 ? (w << 1) : (w >> (8 * K - 1));
        return lds_u16(e ^ (x & 0x1FEu));
    }
    uint32_t c = lds_u8(E.cmap_s + ((w >> (8 * K)) & 0xFFu));
    return lds_u16(e + (c << 1));
}

template <int FORM>
__device__ __forceinline__ uint32_t kind_of(const Env &E, uint32_t e)
{
    if (FORM == FORM_BYTE) return lds_u16(E.kind_s + (((e - E.tbase) >> 9) << 1));
    return lds_u16(e + E.kcol2);
}

__device__ __forceinline__ bool is_cut(const Env &E, uint32_t b) { return lds_u8(E.cert_s + b) != 0; }

// ---- generic walker (64-bit offsets, reads past the staged bytes) ----
// Counts kept tokens; `big` is set when one does not fit the packed staging
// word (kind << 20 | length: kind < 4096, length < 2^20).
struct CountEmit {
    uint64_t count = 0;
    bool big = false;
    __device__ __forceinline__ void operator()(uint32_t kw, uint64_t len)
    {
        if (!(kw & KIND_KEEP)) return;
        count++;
        big |= (kw & 0x7FFFu) >= 4096u || len >= (1ull << 20);
    }
};

// Writes kept tokens, packed, to consecutive shared staging words.
struct StageEmit {
    uint32_t *stage;
    __device__ __forceinline__ void operator()(uint32_t kw, uint64_t len)
    {
        if (!(kw & KIND_KEEP)) return;
        *stage++ = ((kw & 0x7FFFu) << 20) | (uint32_t)len;
    }
};

struct DirectEmit {
    uint16_t *kinds;
    uint32_t *lens;
    uint64_t cap;
    uint64_t idx;
    __device__ __forceinline__ void operator()(uint32_t kw, uint64_t len)
    {
        if (!(kw & KIND_KEEP)) return;
        if (idx < cap) {
            kinds[idx] = (uint16_t)(kw & 0x7FFFu);
            lens[idx] = (uint32_t)len;
        }
        idx++;
    }
};

// Longest-match walk of the chunks that start at `start` (a certified byte,
// or offset 0) and run until a certified byte at or past `seg_end`, or the
// end of the input.  Returns the failure offset (Section 3: the scan halts
// where no positive-length accepting prefix exists) or NOPOS.  Used for
// ranges that leave the staged bytes or overflow their records.
template <int FORM, class Emit>
__device__ uint64_t walk(const Env &E, uint64_t start, uint64_t seg_end, Emit &emit)
{
    uint64_t p = start, tok = start;
    uint32_t e = E.P_start;
    for (;;) {
        bool slow;
        if (p == E.n) {
            if (e == E.P_start) return NOPOS;
            uint32_t kw = kind_of<FORM>(E, e);
            if ((kw & 0x7FFFu) != KIND_NONE) {
                emit(kw, p - tok);
                return NOPOS;
            }
            slow = true;
        } else {
            uint32_t b = byte_at(E, p);
            uint32_t e2 = step<FORM>(E, e, b);
            slow = false;
            if (e2 == E.P_slow) {
                slow = true;
            } else if (e2 >= E.P_flag) {
                emit(kind_of<FORM>(E, e), p - tok);   // token [tok, p) ends before byte p
                tok = p;
                if (p >= seg_end && is_cut(E, b)) return NOPOS;
            }
            if (!slow) {
                e = e2;
                p++;
                continue;
            }
        }
        // Slow path: replay [tok, p) from q0 to find the last accepting
        // position (longest match with backtracking).
        uint32_t q = E.P_start, rk = 0;
        uint64_t r = NOPOS;
        for (uint64_t j = tok; j < p; j++) {
            q = step<FORM>(E, q, byte_at(E, j));
            uint32_t kw = kind_of<FORM>(E, q);
            if ((kw & 0x7FFFu) != KIND_NONE) {
                r = j + 1;
                rk = kw;
            }
        }
        if (r == NOPOS) return tok;   // halts: lexing error at tok
        emit(rk, r - tok);
        tok = p = r;
        e = E.P_start;
        if (r == E.n) return NOPOS;
        if (r >= seg_end && is_cut(E, byte_at(E, r))) return NOPOS;
    }
}

// One lockstep iteration of a lane: four byte steps over the word `w` (bytes
// base .. base+3), as branch-free PTX.  The loop-carried chain per byte is
// only the row address (one LOP3 or LEA) and the shared-memory load of the
// next row; the token-end test, the record packing (PRMT) and its predicated
// store hang off that chain:
//   a_k   = e_k ^ ((w >> 8k) << 1 & 0x1FE)       (byte form)
//   a_k   = e_k + 2 * class(byte k)               (class form, class loaded off-chain)
//   e_k+1 = [a_k]
//   if e_k+1 >= P_flag: record (e_k << 16 | base + k); sp += 4 NT
template <int FORM>
__device__ __forceinline__ void walk_word(const Env &E, uint32_t &e, uint32_t &sp, uint32_t w, uint32_t base)
{
    const uint32_t P_flag = E.P_flag;
    if (FORM == FORM_BYTE) {
#define LX_PSTEP(K, XOP)                                           \
        XOP                                                        \
        "and.b32 x, x, 0x1FE;\n\t"                                 \
        "xor.b32 a, %0, x;\n\t"                                    \
        "ld.shared.u16 e2, [a];\n\t"                               \
        "setp.ge.u32 pf, e2, %3;\n\t"                              \
        "add.u32 t, %4, " #K ";\n\t"                               \
        "prmt.b32 v, t, %0, 0x5410;\n\t"                           \
        "@pf st.shared.u32 [%1], v;\n\t"                           \
        "@pf add.u32 %1, %1, %5;\n\t"                              \
        "mov.b32 %0, e2;\n\t"
        asm volatile(
            "{\n\t.reg .pred pf;\n\t.reg .b32 t, x, a, e2, v;\n\t"
            LX_PSTEP(0, "shl.b32 x, %2, 1;\n\t")
            LX_PSTEP(1, "shr.b32 x, %2, 7;\n\t")
            LX_PSTEP(2, "shr.b32 x, %2, 15;\n\t")
            LX_PSTEP(3, "shr.b32 x, %2, 23;\n\t")
            "}"
            : "+r"(e), "+r"(sp)
            : "r"(w), "r"(P_flag), "r"(base), "n"(NT * 4)
            : "memory");
#undef LX_PSTEP
    } else {
        const uint32_t cm = E.cmap_s;
#define LX_CSTEP(K, SH)                                            \
        "bfe.u32 x, %2, " #SH ", 8;\n\t"                           \
        "add.u32 x, x, %6;\n\t"                                    \
        "ld.shared.u8 c, [x];\n\t"                                 \
        "shl.b32 c, c, 1;\n\t"                                     \
        "add.u32 a, %0, c;\n\t"                                    \
        "ld.shared.u16 e2, [a];\n\t"                               \
        "setp.ge.u32 pf, e2, %3;\n\t"                              \
        "add.u32 t, %4, " #K ";\n\t"                               \
        "prmt.b32 v, t, %0, 0x5410;\n\t"                           \
        "@pf st.shared.u32 [%1], v;\n\t"                           \
        "@pf add.u32 %1, %1, %5;\n\t"                              \
        "mov.b32 %0, e2;\n\t"
        asm volatile(
            "{\n\t.reg .pred pf;\n\t.reg .b32 t, x, a, c, e2, v;\n\t"
            LX_CSTEP(0, 0)
            LX_CSTEP(1, 8)
            LX_CSTEP(2, 16)
            LX_CSTEP(3, 24)
            "}"
            : "+r"(e), "+r"(sp)
            : "r"(w), "r"(P_flag), "r"(base), "n"(NT * 4), "r"(cm)
            : "memory");
#undef LX_CSTEP
    }
}

// ---- lockstep walker (staged bytes only, 32-bit offsets) ----
enum { LS_WALK = 0, LS_SLOW = 1, LS_END = 2, LS_TAIL = 3, LS_FULL = 4, LS_DONE = 5, LS_FAIL = 6, LS_OVF = 7 };

// All lanes of a warp walk their ranges in lockstep, two aligned
// shared-memory words (eight bytes) per lane per iteration, with no per-byte
// predicate: a lane whose chunk starts inside a word begins at the word in
// the PRE row (the bytes between the word start and the chunk start are not
// certified, PRE absorbs them), and a lane runs over the word holding its
// range end, whose recorded token ends past that cut are dropped afterwards.
// A lane's range is [start, end]: `end` is the next chunk start (a certified
// byte, whose step ends the last token) or, with `eoi`, the end of the
// input.  Every token end is recorded as (row before the byte << 16 | end
// offset) in the lane's record column `col` (stride NT words).  When the
// column fills, its raw records are compacted in place into kept tokens
// (kind << 20 | length, discarded kinds dropped) and the walk goes on; when
// compacted tokens fill half of it, they move to a block of the CTA's global
// spill region (blocks of one lane are chained: count, next, tokens).  A
// lane that falls into the absorbing SLOW row leaves the lockstep loop and
// replays its current token from q0 to its last accepting position (longest
// match with backtracking), then rejoins; a restart inside a word, and the
// last partial word of the input, are stepped byte by byte.
//
// On return the lane's first `spilled` kept tokens are in the spill blocks
// chained from `sp_first`, the column holds the next `nc` compacted kept
// tokens followed by raw records up to index `cnt`; `prev` is the offset
// where the first of those raw records' tokens begins.
template <int FORM>
__device__ __forceinline__ int lockstep_walk(const Env &E, bool has, uint32_t start, uint32_t end, bool eoi,
                                             uint32_t col, uint32_t &cnt, uint32_t &nc, uint32_t &prev,
                                             uint32_t &fail, uint32_t &sp_first, uint32_t &spilled)
{
    const uint32_t P_flag = E.P_flag, P_slow = E.P_slow;
    const uint32_t col_end = col + E.ks * NT * 4;
    const uint32_t lim = eoi ? end : end + 1;             // bytes [start, lim) are stepped
    const uint32_t mlim = eoi ? (lim & ~3u) : lim;        // whole words while p < mlim
    uint32_t p = start & ~3u;
    uint32_t e = (start & 3u) ? E.P_pre : E.P_start;
    // sp: next record; raw0: first raw record (after nc compacted tokens);
    // sp_lo: first record of the current token run (after the last restart or
    // compaction), tok_base: where that run's first token begins
    uint32_t sp = col, raw0 = col, sp_lo = col, tok_base = start;
    uint32_t ncomp = 0, prev_pos = start;
    uint32_t sp_last = NONE32, nspill = 0;
    sp_first = NONE32;
    int st = !has ? LS_DONE : (p < mlim ? LS_WALK : LS_TAIL);

    // byte-by-byte steps over [p, stop) with the same recording rule
    auto scalar = [&](uint32_t stop) {
        for (; p < stop && e != P_slow; p++) {
            const uint32_t e2 = step<FORM>(E, e, lds_u8(E.buf + p));
            if (e2 >= P_flag) {
                sts_u32(sp, (e << 16) | p);
                sp += NT * 4;
            }
            e = e2;
        }
    };
    // Make room in the column: compact its raw records into kept tokens
    // and, when those fill half of it, move them to a spill block.  False
    // when a kept kind does not pack or the spill region is full.
    auto make_room = [&]() -> bool {
        uint32_t wr = raw0;
        bool big = false;
        for (uint32_t a = raw0; a < sp; a += NT * 4) {
            const uint32_t v = lds_u32(a);
            const uint32_t pos = v & 0xFFFFu;
            const uint32_t kw = kind_of<FORM>(E, v >> 16);
            const uint32_t len = pos - prev_pos;
            prev_pos = pos;
            if (kw & KIND_KEEP) {
                big |= (kw & 0x7FFFu) >= 4096u;
                sts_u32(wr, ((kw & 0x7FFFu) << 20) | len);
                wr += NT * 4;
                ncomp++;
            }
        }
        raw0 = sp = sp_lo = wr;
        tok_base = prev_pos;   // the token in progress began at the last end
        if (big) return false;
        if (sp > col + (E.ks / 2) * NT * 4) {   // move the kept tokens out
            const uint32_t off = atomicAdd(E.spill_used, ncomp + 2);
            if (off + ncomp + 2 > E.spill_cap) return false;
            uint32_t *blk = E.spill + off;
            blk[0] = ncomp;
            blk[1] = NONE32;
            for (uint32_t i = 0; i < ncomp; i++) blk[2 + i] = lds_u32(col + i * NT * 4);
            if (sp_last == NONE32) sp_first = off;
            else E.spill[sp_last + 1] = off;
            sp_last = off;
            nspill += ncomp;
            ncomp = 0;
            raw0 = sp = sp_lo = col;
        }
        return true;
    };
    for (;;) {
        while (__any_sync(0xffffffffu, st == LS_WALK)) {
            if (st == LS_WALK) {
                if (sp + 8 * NT * 4 > col_end) {
                    st = LS_FULL;
                } else {
                    const uint32_t w0 = lds_u32(E.buf + p), w1 = lds_u32(E.buf + p + 4);
                    walk_word<FORM>(E, e, sp, w0, p);
                    p += 4;
                    if (p >= mlim) st = eoi ? (e == P_slow ? LS_SLOW : LS_TAIL) : LS_END;
                    else if (e == P_slow) st = LS_SLOW;
                    else {
                        walk_word<FORM>(E, e, sp, w1, p);
                        p += 4;
                        if (p >= mlim) st = eoi ? (e == P_slow ? LS_SLOW : LS_TAIL) : LS_END;
                        else if (e == P_slow) st = LS_SLOW;
                    }
                }
            }
        }
        // events, one lane at a time where they occur
        if (st == LS_FULL) st = make_room() ? LS_WALK : LS_OVF;
        if (st == LS_TAIL) {   // the input's last partial word, then close at the end
            if (sp + 4 * NT * 4 > col_end && !make_room()) {
                st = LS_OVF;
            } else {
                scalar(lim);
                if (e == P_slow) {
                    st = LS_SLOW;
                } else if (e == E.P_start) {
                    st = LS_DONE;
                } else if ((kind_of<FORM>(E, e) & 0x7FFFu) != KIND_NONE) {
                    sts_u32(sp, (e << 16) | p);
                    sp += NT * 4;
                    st = LS_DONE;
                } else {
                    st = LS_SLOW;
                }
            }
        }
        if (st == LS_END) {   // stepped through the cut at `end` (and maybe past it)
            while (sp > sp_lo && (lds_u32(sp - NT * 4) & 0xFFFFu) > end) sp -= NT * 4;
            if (sp > sp_lo && (lds_u32(sp - NT * 4) & 0xFFFFu) == end) {
                st = LS_DONE;   // the last token ended exactly at the cut
            } else {
                p = end;        // it did not: the state at the cut (or before) is SLOW
                st = LS_SLOW;
            }
        }
        if (st == LS_SLOW) {
            // the token in progress began at the last recorded end (or the
            // last restart); SLOW absorbs, so replaying up to p (never past
            // the range's cut byte) finds the same last accepting position
            const uint32_t tok = sp > sp_lo ? (lds_u32(sp - NT * 4) & 0xFFFFu) : tok_base;
            const uint32_t stop = (!eoi && p > end) ? end : p;
            uint32_t q = E.P_start, r = NONE32, rq = 0;
            for (uint32_t j = tok; j < stop; j++) {
                q = step<FORM>(E, q, lds_u8(E.buf + j));
                if ((kind_of<FORM>(E, q) & 0x7FFFu) != KIND_NONE) {
                    r = j + 1;
                    rq = q;
                }
            }
            if (r == NONE32) {
                fail = tok;
                st = LS_FAIL;
            } else if (sp + 8 * NT * 4 > col_end && !make_room()) {
                st = LS_OVF;
            } else {
                sts_u32(sp, (rq << 16) | r);
                sp += NT * 4;
                sp_lo = sp;
                tok_base = p = r;
                e = E.P_start;
                if (r == end) {
                    st = LS_DONE;
                } else {
                    scalar(((r + 3u) & ~3u) < mlim ? ((r + 3u) & ~3u) : mlim);   // up to a word boundary
                    if (e == P_slow) st = LS_SLOW;
                    else if (p < mlim) st = LS_WALK;
                    else st = eoi ? LS_TAIL : LS_END;
                }
            }
        }
        if (!__any_sync(0xffffffffu, st < LS_DONE)) break;   // no lane walking or with an event
    }
    cnt = (sp - col) / (NT * 4);
    nc = ncomp;
    prev = prev_pos;
    spilled = nspill;
    return st;
}

// Decoupled look-back (devutil.cuh): each tile first publishes its
// aggregate (tile 0 its inclusive prefix) without waiting; later one warp
// resolves the exclusive prefix.
__device__ __forceinline__ void publish_aggregate(const Params &P, uint32_t tile, uint64_t agg)
{
    st_status(&P.status[tile], (tile == 0 ? ST_INCL : ST_AGG) | agg);
}

__device__ __forceinline__ uint64_t resolve_prefix(const Params &P, uint32_t tile, uint64_t agg, bool &timed_out)
{
    return lookback(P.status, tile, agg, P.timeout_ns, &P.res->error, P.withhold, timed_out);
}

// Where global tile g of a launch lies: its document and the document-relative
// offset of its first byte.
struct TileRef {
    const uint8_t *in;
    uint64_t n;
    uint64_t base;
    uint32_t doc;
    uint32_t tma;
    bool first;
};

static_assert(sizeof(TileRef) <= 40, "TileRef must fit its shared slot");

__device__ __forceinline__ TileRef tile_ref(const Params &P, uint32_t g)
{
    uint32_t d = 0;
    const DocDesc D = P.docs ? P.docs[d = P.tile_doc[g]] : P.one;
    TileRef r;
    r.in = D.in;
    r.n = D.n;
    r.doc = d;
    r.tma = D.tma;
    r.base = (uint64_t)(g - D.first_tile) * TILE;
    r.first = g == D.first_tile;
    return r;
}

// 4-bit mask of the certified bytes of a little-endian word.
__device__ __forceinline__ uint32_t cut_mask4(const Env &E, uint32_t w)
{
    return (uint32_t)is_cut(E, w & 0xFFu) | ((uint32_t)is_cut(E, (w >> 8) & 0xFFu) << 1) |
           ((uint32_t)is_cut(E, (w >> 16) & 0xFFu) << 2) | ((uint32_t)is_cut(E, w >> 24) << 3);
}

template <int FORM>
__global__ void __launch_bounds__(NT, 3) lex_tiles(Params P)
{
    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const Layout L = make_layout(P.blob_bytes, P.ks);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t tbase = align_up(sbase, 512);
    uint8_t *misc = smem + L.misc;
    const uint32_t mbar = sbase + L.misc + M_MBAR;
    const uint32_t buf = sbase + L.buf;

    if (tbase + P.table_bytes > 65536u) {   // u16 row pointers must reach every row
        if (tid == 0) atomicOr(&P.res->error, ERR_SMEM);
        return;
    }
    // stage the walk tables; row pointers become shared addresses
    {
        uint8_t *dst = smem + (tbase - sbase);
        const uint16_t *src16 = reinterpret_cast<const uint16_t *>(P.blob);
        uint16_t *dst16 = reinterpret_cast<uint16_t *>(dst);
        const uint32_t n16 = P.blob_bytes / 2, t16 = P.table_bytes / 2;
        for (uint32_t i = tid; i < n16; i += NT) {
            uint32_t v = src16[i];
            bool ptr = i < t16 && (FORM == FORM_BYTE || (i % P.ncols) != P.ncols - 1);
            dst16[i] = (uint16_t)(ptr ? v + tbase : v);
        }
    }
    Env E;
    E.P_start = tbase + P.p_start;
    E.P_flag = tbase + P.p_flag;
    E.P_slow = tbase + P.p_slow;
    E.P_pre = tbase + P.p_pre;
    E.tbase = tbase;
    E.kind_s = tbase + P.kind_off;
    E.cmap_s = tbase + P.cmap_off;
    E.cert_s = tbase + P.cert_off;
    E.kcol2 = 2 * (P.ncols - 1);
    E.buf = buf;
    E.spill = P.spill + (size_t)blockIdx.x * P.spill_cap;
    E.spill_cap = P.spill_cap;
    E.ks = P.ks;
    E.spill_used = reinterpret_cast<unsigned *>(misc + M_SPILL);

    volatile uint32_t *s_tile = reinterpret_cast<volatile uint32_t *>(misc + M_TILE);
    volatile uint32_t *s_x = reinterpret_cast<volatile uint32_t *>(misc + M_X);
    volatile uint32_t *s_flags = reinterpret_cast<volatile uint32_t *>(misc + M_FLAGS);
    uint32_t *s_wmin = reinterpret_cast<uint32_t *>(misc + M_WMIN);
    unsigned long long *s_G = reinterpret_cast<unsigned long long *>(misc + M_G);
    unsigned long long *s_tot = reinterpret_cast<unsigned long long *>(misc + M_TOT);
    unsigned long long *s_fpos = reinterpret_cast<unsigned long long *>(misc + M_FPOS);
    unsigned long long *s_fidx = reinterpret_cast<unsigned long long *>(misc + M_FIDX);
    volatile uint32_t *s_ptile = reinterpret_cast<volatile uint32_t *>(misc + M_PTILE);
    unsigned long long *s_ptot = reinterpret_cast<unsigned long long *>(misc + M_PTOT);
    unsigned long long *s_pfpos = reinterpret_cast<unsigned long long *>(misc + M_PFPOS);
    unsigned long long *s_pfidx = reinterpret_cast<unsigned long long *>(misc + M_PFIDX);
    unsigned long long *warp_tot = reinterpret_cast<unsigned long long *>(misc + M_WARP);
    volatile uint32_t *s_pdoc = reinterpret_cast<volatile uint32_t *>(misc + M_PDOC);
    volatile uint32_t *s_pfirst = reinterpret_cast<volatile uint32_t *>(misc + M_PFIRST);
    // the launch's output starts after the tokens of the launches before it
    uint64_t out_base = 0;
    for (uint32_t k = 0; k < P.n_prev; k++) out_base += P.prev[k].total;
    // per-document record (the launch record itself for a single document)
    auto rec = [&](uint32_t d) -> DocResult * {
        return P.dres ? P.dres + d : reinterpret_cast<DocResult *>(P.res);
    };
    // a resolved tile: its failure and, for a document's first tile, the
    // document's output offset
    auto report = [&](uint32_t d, bool first, uint64_t G, uint64_t fpos, uint64_t fidx) {
        if (fpos != NOPOS) {
            atomicMax(&rec(d)->inv_fail_pos, ~(unsigned long long)fpos);
            atomicMax(&rec(d)->inv_fail_tok, ~(unsigned long long)(out_base + G + fidx));
        }
        if (first && P.dres) P.dres[d].out_off1 = out_base + G + 1;
    };
    uint32_t *stage32 = reinterpret_cast<uint32_t *>(smem + L.stage);
    const uint32_t col = sbase + L.slots + tid * 4;   // this thread's record column

    if (tid == 0) {
        mbar_init(mbar, 1);
        fence_proxy_async();
        *s_ptile = NONE32;
        *E.spill_used = 0;
    }
    __syncthreads();

    TileRef *s_tref = reinterpret_cast<TileRef *>(misc + M_TREF);
    // one thread: claim the next tile, note where it lies, start its copy
    auto claim = [&]() {
        uint32_t t = atomicAdd(P.tile_counter, 1u);
        if (*(volatile unsigned int *)&P.res->error != 0) t = P.n_tiles;   // a wait gave up: stop
        s_tile[0] = t;
        if (t >= P.n_tiles) return;
        const TileRef R = tile_ref(P, t);
        *s_tref = R;
        if (!R.tma) return;
        uint64_t avail = R.n - R.base;
        uint32_t len = (uint32_t)(avail < (uint64_t)BUF ? avail : (uint64_t)BUF) & ~15u;
        if (len) {
            fence_proxy_async();
            tma_load(buf, R.in + R.base, len, mbar);
        }
    };
    // Resolve the pending tile's output offset (warp 0), then write its
    // staged kept tokens with coalesced stores (all threads).
    auto flush_pending = [&]() {
        const uint32_t pt = *s_ptile;
        if (pt == NONE32) return;
        if (wid == 0) {
            bool to = false;
            const uint64_t G = resolve_prefix(P, pt, *s_ptot, to);
            if (lane == 0) {
                if (to) atomicOr(&P.res->error, ERR_TIMEOUT);
                *s_G = G;
                report(*s_pdoc, *s_pfirst != 0, G, *s_pfpos, *s_pfidx);
            }
        }
        __syncthreads();
        const uint64_t G = *s_G, tot = *s_ptot;
        for (uint32_t i = tid; i < tot; i += NT) {
            const uint64_t idx = out_base + G + i;
            if (idx < P.cap) {
                const uint32_t v = stage32[i];
                P.out_kinds[idx] = (uint16_t)(v >> 20);
                P.out_lens[idx] = v & 0xFFFFFu;
            }
        }
        __syncthreads();
        if (tid == 0) *s_ptile = NONE32;
    };

    if (tid == 0) claim();
    __syncthreads();
    uint32_t tile = s_tile[0];
    uint32_t par = 0;

    while (tile < P.n_tiles) {
        const TileRef T = *s_tref;
        const uint64_t tile_base = T.base;   // offsets below are relative to the document
        const uint64_t avail = T.n - tile_base;
        E.in = T.in;
        E.n = T.n;
        uint32_t staged;
        bool bad = false;
        if (T.tma) {
            staged = (uint32_t)(avail < (uint64_t)BUF ? avail : (uint64_t)BUF) & ~15u;
            if (staged) {
                bad = !mbar_wait(mbar, par, P.timeout_ns);
                par ^= 1;
            }
        } else {
            staged = (uint32_t)(avail < (uint64_t)BUF ? avail : (uint64_t)BUF);
            uint8_t *b = smem + L.buf;
            for (uint32_t i = tid; i < staged; i += NT) b[i] = T.in[tile_base + i];
        }
        if (__syncthreads_or(bad)) {
            if (tid == 0) atomicOr(&P.res->error, ERR_TIMEOUT);
            break;
        }
        if (tid == 0) *E.spill_used = 0;   // the previous tile's spill blocks are staged (seen after the plan)
        E.tile_base = tile_base;
        E.sm_end = tile_base + staged;
        const uint32_t n_rel = avail < 0x7FFFFFFFull ? (uint32_t)avail : 0x7FFFFFFFu;

        // (b) plan: the first certified byte of this thread's segment, tested
        // a word at a time
        const uint32_t seg0 = (uint32_t)tid * SEG;
        uint32_t start = NONE32;
        if (T.first && tid == 0) {
            start = 0;
        } else if (seg0 + SEG <= staged) {
            for (uint32_t k = 0; k < SEG / 4; k++) {
                const uint32_t m = cut_mask4(E, lds_u32(buf + seg0 + 4 * k));
                if (m) { start = seg0 + 4 * k + __ffs(m) - 1; break; }
            }
            if (start >= n_rel) start = NONE32;
        } else {
            const uint32_t lim = seg0 + SEG < n_rel ? seg0 + SEG : n_rel;
            for (uint32_t p = seg0; p < lim; p++) {
                uint32_t b = p < staged ? lds_u8(buf + p) : (uint32_t)__ldg(T.in + tile_base + p);
                if (is_cut(E, b)) { start = p; break; }
            }
        }
        if (wid == NW - 1) {   // first cut at or past the tile end, within the staged halo
            const uint32_t hl = staged < n_rel ? staged : n_rel;
            uint32_t x = NONE32;
            for (uint32_t b0 = TILE; b0 < hl; b0 += 32) {
                const uint32_t p = b0 + lane;
                const unsigned m = __ballot_sync(0xffffffffu, p < hl && is_cut(E, lds_u8(buf + p)));
                if (m) { x = b0 + __ffs(m) - 1; break; }
            }
            if (x == NONE32 && hl >= n_rel) x = n_rel;
            if (lane == 0) *s_x = x;
        }
        // next chunk start after this thread's: suffix minimum over the starts
        uint32_t smin = start;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_down_sync(0xffffffffu, smin, o);
            if (lane + o < 32) smin = min(smin, y);
        }
        uint32_t nxt = __shfl_down_sync(0xffffffffu, smin, 1);
        if (lane == 31) nxt = NONE32;
        if (lane == 0) s_wmin[wid] = smin;
        __syncthreads();
        for (int w = wid + 1; w < NW && nxt == NONE32; w++) nxt = s_wmin[w];
        if (nxt == NONE32) nxt = *s_x;   // may still be NONE32: the range leaves the halo

        // (c) walk
        uint32_t cnt = 0, kept = 0;
        uint64_t kept_generic = 0;
        uint64_t fail = NOPOS;
        bool generic = false;   // this lane's tokens come from the generic walker
        bool big = false;       // ... and one of them does not fit a staging word
        const bool has = start != NONE32;
        const bool eoi = nxt == n_rel;
        const bool fast = has && nxt != NONE32 && (eoi ? n_rel <= staged : nxt < staged);
        uint32_t f32 = 0, ncomp = 0, prev0 = start, sp_first = NONE32, spilled = 0;
        const int st = lockstep_walk<FORM>(E, fast, start, fast ? nxt : 0u, eoi, col, cnt, ncomp, prev0, f32,
                                           sp_first, spilled);
        if (fast && st == LS_FAIL) fail = tile_base + f32;
        if (has && (!fast || st == LS_OVF)) {
            generic = true;
            sp_first = NONE32;   // blocks spilled before the overflow are not used
            spilled = 0;
            CountEmit ce;
            fail = walk<FORM>(E, tile_base + start, tile_base + seg0 + SEG, ce);
            kept_generic = ce.count;
            big = ce.big;
        } else if (has) {
            // kinds, discard filter and lengths of the recorded token ends,
            // compacted in place in the column as kind << 20 | length
            uint32_t prev = prev0;
            kept = ncomp;
            for (uint32_t k = ncomp; k < cnt; k++) {
                const uint32_t v = lds_u32(col + k * NT * 4);
                const uint32_t pos = v & 0xFFFFu;
                const uint32_t kw = kind_of<FORM>(E, v >> 16);
                const uint32_t len = pos - prev;
                prev = pos;
                if (kw & KIND_KEEP) {
                    if ((kw & 0x7FFFu) >= 4096u) generic = big = true;
                    sts_u32(col + kept * NT * 4, ((kw & 0x7FFFu) << 20) | len);
                    kept++;
                }
            }
            if (generic) kept_generic = kept;
        }
        const uint32_t count32 = generic ? 0u : kept;

        // (d) CTA scan of kept-token counts
        const uint64_t mycount = generic ? kept_generic : (uint64_t)(spilled + kept);
        uint64_t x = mycount;
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        const uint64_t lane_excl = x - mycount;
        if (lane == 31) warp_tot[wid] = x;
        if (tid == 0) *s_fpos = NOPOS;
        const int any_big = __syncthreads_or(big);
        if (tid == 0) {
            unsigned long long run = 0;
            for (int w = 0; w < NW; w++) {
                unsigned long long t = warp_tot[w];
                warp_tot[w] = run;
                run += t;
            }
            *s_tot = run;
            *s_flags = (any_big || run > (unsigned long long)STAGE_CAP) ? 1u : 0u;
            // publish this tile's aggregate at once
            if (tile != P.withhold) publish_aggregate(P, tile, run);
            if (run) {
                atomicAdd(&rec(T.doc)->total, run);
                if (P.dres) atomicAdd(&P.res->total, run);
            }
            // claim the next tile now that this one's aggregate is out, and
            // stage it while this tile's output is written
            claim();
        }
        const int any_fail = __syncthreads_or(fail != NOPOS);
        const uint64_t my_off = warp_tot[wid] + lane_excl;   // within the tile
        if (any_fail) {   // the first failure of the tile and the kept tokens before it
            if (fail != NOPOS) atomicMin(s_fpos, (unsigned long long)fail);
            __syncthreads();
            if (fail != NOPOS && *s_fpos == fail) *s_fidx = my_off + mycount;
            __syncthreads();
        }

        // the previous tile's output: its predecessors have had a whole walk
        // to publish, so its look-back rarely waits
        flush_pending();

        // this lane's packed kept tokens in order: spill blocks, then the column
        auto for_lane_tokens = [&](auto put) {
            uint32_t i = 0;
            for (uint32_t off = sp_first; off != NONE32;) {
                const uint32_t *blk = E.spill + off;
                const uint32_t nb = blk[0];
                for (uint32_t j = 0; j < nb; j++) put(i++, blk[2 + j]);
                off = blk[1];
            }
            for (uint32_t k = 0; k < count32; k++) put(i++, lds_u32(col + k * NT * 4));
        };
        E.sm_end = E.tile_base;   // the staged buffer now receives the next tile: re-walks read global
        const bool sync_tile = *s_flags != 0;
        if (!sync_tile) {
            // stage this tile's kept tokens; they are written after the next walk.
            // A lane whose range overflowed its records or left the staged
            // bytes walks it again, writing straight into the stage (the
            // input tile is still staged).
            if (!generic) {
                for_lane_tokens([&](uint32_t i, uint32_t v) { stage32[my_off + i] = v; });
            } else {
                StageEmit se{stage32 + my_off};
                walk<FORM>(E, tile_base + start, tile_base + seg0 + SEG, se);
            }
            if (tid == 0) {
                *s_ptot = *s_tot;
                *s_pfpos = *s_fpos;
                *s_pfidx = *s_fidx;
                *s_pdoc = T.doc;
                *s_pfirst = T.first ? 1u : 0u;
                *s_ptile = tile;
            }
        } else {
            // rare: stage overflow or a token that does not pack -- resolve
            // now and write directly
            if (wid == 0) {
                bool to = false;
                const uint64_t G = resolve_prefix(P, tile, *s_tot, to);
                if (lane == 0) {
                    if (to) atomicOr(&P.res->error, ERR_TIMEOUT);
                    *s_G = G;
                    report(T.doc, T.first, G, *s_fpos, *s_fidx);
                }
            }
            __syncthreads();
            const uint64_t G = *s_G;
            if (!generic) {
                for_lane_tokens([&](uint32_t i, uint32_t v) {
                    const uint64_t idx = out_base + G + my_off + i;
                    if (idx < P.cap) {
                        P.out_kinds[idx] = (uint16_t)(v >> 20);
                        P.out_lens[idx] = v & 0xFFFFFu;
                    }
                });
            } else {
                DirectEmit de{P.out_kinds, P.out_lens, P.cap, out_base + G + my_off};
                walk<FORM>(E, tile_base + start, tile_base + seg0 + SEG, de);
            }
        }
        __syncthreads();   // records, stage and spill blocks are free
        tile = s_tile[0];
    }
    flush_pending();
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int cuda_err(cudaError_t e)
{
    if (e == cudaSuccess) return LX_OK;
    return e == cudaErrorMemoryAllocation ? LX_E_NOMEM : LX_E_CUDA;
}

}  // namespace lx

using namespace lx;

int lx::ensure_device_tables(const lx_tokenset *cts, int device, DeviceTables *out)
{
    lx_tokenset *ts = const_cast<lx_tokenset *>(cts);
    std::lock_guard<std::mutex> g(ts->mu);
    for (auto &d : ts->dev)
        if (d.device == device) {
            *out = d;
            return LX_OK;
        }
    DeviceTables dt;
    dt.device = device;
    auto upload = [](const std::vector<uint8_t> &blob, void **dst) {
        int rc = cuda_err(cudaMalloc(dst, blob.size()));
        if (rc == LX_OK) rc = cuda_err(cudaMemcpy(*dst, blob.data(), blob.size(), cudaMemcpyHostToDevice));
        return rc;
    };
    int rc = LX_OK;
    for (int m = 0; m < 3 && rc == LX_OK; m++) {
        if (ts->tab[m].status == LX_OK) rc = upload(ts->tab[m].blob, &dt.d_blob[m]);
        if (rc == LX_OK && ts->tab_cls[m].status == LX_OK && !ts->tab_cls[m].blob.empty())
            rc = upload(ts->tab_cls[m].blob, &dt.d_blob_cls[m]);
    }
    if (rc == LX_OK && ts->scan.status == LX_OK) rc = upload(ts->scan.blob, &dt.d_scan);
    for (int m = 0; m < 3 && rc == LX_OK; m++)
        if (ts->walk[m].status == LX_OK) rc = upload(ts->walk[m].blob, &dt.d_walk[m]);
    if (rc == LX_OK && ts->liveness.status == LX_OK) rc = upload(ts->liveness.blob, &dt.d_live);
    if (rc != LX_OK) {
        for (int m = 0; m < 3; m++) {
            if (dt.d_blob[m]) cudaFree(dt.d_blob[m]);
            if (dt.d_blob_cls[m]) cudaFree(dt.d_blob_cls[m]);
            if (dt.d_walk[m]) cudaFree(dt.d_walk[m]);
        }
        if (dt.d_scan) cudaFree(dt.d_scan);
        if (dt.d_live) cudaFree(dt.d_live);
        return rc;
    }
    ts->dev.push_back(dt);
    *out = dt;
    return LX_OK;
}

extern "C" void lx_tokenset_free(lx_tokenset *ts)
{
    if (!ts) return;
    int cur = -1;
    cudaGetDevice(&cur);
    for (auto &d : ts->dev) {
        cudaSetDevice(d.device);
        for (int m = 0; m < 3; m++) {
            if (d.d_blob[m]) cudaFree(d.d_blob[m]);
            if (d.d_blob_cls[m]) cudaFree(d.d_blob_cls[m]);
            if (d.d_walk[m]) cudaFree(d.d_walk[m]);
        }
        if (d.d_scan) cudaFree(d.d_scan);
        if (d.d_live) cudaFree(d.d_live);
    }
    if (cur >= 0 && !ts->dev.empty()) cudaSetDevice(cur);
    delete ts;
}

extern "C" int lx_ctx_create(lx_ctx **out)
{
    if (!out) return LX_E_INVAL;
    *out = nullptr;
    int dev = 0, n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        return LX_E_CUDA;
    }
    if (cudaGetDevice(&dev) != cudaSuccess) return LX_E_CUDA;
    lx_ctx *c = new (std::nothrow) lx_ctx();
    if (!c) return LX_E_NOMEM;
    c->device = dev;
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaMallocHost(&c->h_res, std::max(sizeof(Result), LAUNCH_RECORD_BYTES)) != cudaSuccess) {
        delete c;
        return LX_E_CUDA;
    }
    *out = c;
    return LX_OK;
}

extern "C" void lx_ctx_free(lx_ctx *c)
{
    if (!c) return;
    cudaDeviceSynchronize();
    if (c->scratch) cudaFree(c->scratch);
    if (c->b_exec) cudaGraphExecDestroy(c->b_exec);
    if (c->b_stream) cudaStreamDestroy(c->b_stream);
    if (c->b_dev) cudaFree(c->b_dev);
    if (c->e_dev) cudaFree(c->e_dev);
    if (c->lv_dev) cudaFree(c->lv_dev);
    if (c->wb_dev) cudaFree(c->wb_dev);
    if (c->w_spill) cudaFree(c->w_spill);
    if (c->b_host) cudaFreeHost(c->b_host);
    if (c->d_in) cudaFree(c->d_in);
    if (c->h_scratch) cudaFreeHost(c->h_scratch);
    if (c->s_in) cudaStreamDestroy(c->s_in);
    if (c->s_out) cudaStreamDestroy(c->s_out);
    for (auto e : c->ev_in) cudaEventDestroy(e);
    for (auto e : c->ev_lex) cudaEventDestroy(e);
    if (c->d_out) cudaFree(c->d_out);
    if (c->h_res) cudaFreeHost(c->h_res);
    for (auto &e : c->ev)
        if (e) cudaEventDestroy(e);
    delete c;
}

extern "C" int lx_ctx_enable_timing(lx_ctx *c, int on)
{
    if (!c) return LX_E_INVAL;
    if (on && !c->ev[0]) {
        if (cudaEventCreate(&c->ev[0]) != cudaSuccess || cudaEventCreate(&c->ev[1]) != cudaSuccess) return LX_E_CUDA;
    }
    c->timing = on != 0;
    return LX_OK;
}

extern "C" int lx_ctx_last_kernel_ms(lx_ctx *c, float *ms)
{
    if (!c || !ms || !c->ev[0]) return LX_E_INVAL;
    return cuda_err(cudaEventElapsedTime(ms, c->ev[0], c->ev[1]));
}

extern "C" int lx_ctx_set_kernel(lx_ctx *c, int kernel)
{
    if (!c || kernel < LX_KERNEL_AUTO || kernel > LX_KERNEL_WARP) return LX_E_INVAL;
    c->kernel = kernel;
    return LX_OK;
}

extern "C" int lx_ctx_set_warps(lx_ctx *c, uint32_t warps)
{
    if (!c || warps > 20) return LX_E_INVAL;
    c->warps = warps;
    return LX_OK;
}

extern "C" int lx_ctx_set_warp_geometry(lx_ctx *c, int geometry)
{
    if (!c || geometry < LX_WARP_GEOMETRY_AUTO || geometry > LX_WARP_GEOMETRY_DENSE) return LX_E_INVAL;
    c->warp_geometry = geometry;
    return LX_OK;
}

extern "C" int lx_lex_async(lx_ctx *c, const lx_tokenset *ts, const uint8_t *d_in, uint64_t n, int mode,
                            uint16_t *d_kinds, uint32_t *d_lens, uint64_t capacity, lx_async_result *d_result,
                            void *stream)
{
    if (!c || !ts || !d_result || (n && !d_in)) return LX_E_INVAL;
    if (mode < LX_FULL_EXACT || mode > LX_FILTERED_MODULO) return LX_E_MODE;
    if (capacity && (!d_kinds || !d_lens)) return LX_E_INVAL;
    if (!warp_path_ok(ts, mode, d_in)) return LX_E_INVAL;
    return lex_warp_async(c, ts, d_in, n, mode, d_kinds, d_lens, capacity, d_result,
                          static_cast<cudaStream_t>(stream));
}

extern "C" int lx_ctx_debug_withhold(lx_ctx *c, uint32_t tile)
{
    if (!c) return LX_E_INVAL;
    c->withhold = tile;
    return LX_OK;
}

extern "C" int lx_ctx_set_timeout_ms(lx_ctx *c, uint32_t ms)
{
    if (!c || ms == 0) return LX_E_INVAL;
    c->timeout_ns = (uint64_t)ms * 1000000ull;
    return LX_OK;
}

int lx::grow(void **p, size_t *have, size_t need)
{
    if (*have >= need) return LX_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *have = 0;
    int rc = cuda_err(cudaMalloc(p, need));   // exactly what is asked: buffers are sized per call
    if (rc == LX_OK) *have = need;
    return rc;
}

// CTAs per SM of the tile kernel for a table form and dynamic shared size
// (also raises the kernel's dynamic shared-memory limit on first use).
static int occupancy_for(lx_ctx *c, int form, uint32_t smem, int *occ)
{
    const uint64_t key = ((uint64_t)form << 32) | smem;
    for (auto &kv : c->occupancy)
        if (kv.first == key) {
            *occ = kv.second;
            return LX_OK;
        }
    cudaError_t e;
    int o = 0;
    if (form == FORM_BYTE) {
        e = cudaFuncSetAttribute(lex_tiles<FORM_BYTE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, lex_tiles<FORM_BYTE>, NT, smem);
    } else {
        e = cudaFuncSetAttribute(lex_tiles<FORM_CLASS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, lex_tiles<FORM_CLASS>, NT, smem);
    }
    if (e != cudaSuccess) return LX_E_CUDA;
    if (o < 1) o = 1;
    c->occupancy.emplace_back(key, o);
    *occ = o;
    return LX_OK;
}

// Table fields of the launch parameters for one token set and mode.
static void set_table_params(Params &P, const HostTable &h, const void *blob)
{
    P.blob = static_cast<const uint8_t *>(blob);
    P.blob_bytes = (uint32_t)h.blob.size();
    P.table_bytes = h.table_bytes;
    P.kind_off = h.kind_off;
    P.cmap_off = h.cmap_off;
    P.cert_off = h.cert_off;
    P.ncols = h.ncols;
    P.p_start = h.p_start;
    P.p_flag = h.p_flag;
    P.p_slow = h.p_slow;
    P.p_pre = h.p_pre;
}

static void launch_tiles(int form, uint32_t grid, uint32_t smem, cudaStream_t st, const Params &P)
{
    if (form == FORM_BYTE) lex_tiles<FORM_BYTE><<<grid, NT, smem, st>>>(P);
    else lex_tiles<FORM_CLASS><<<grid, NT, smem, st>>>(P);
}

struct LaunchCfg {
    uint32_t ks = KS_DEFAULT;
    uint32_t ctas = 0;   // CTAs per SM; 0 = as many as fit
    uint32_t cls = 0;    // 1: the class-indexed table (when the default is byte-indexed)
};

static bool has_class_table(const lx_tokenset *ts, int mode)
{
    return ts->tab_cls[mode].status == LX_OK && !ts->tab_cls[mode].blob.empty();
}

static const HostTable &table_for(const lx_tokenset *ts, int mode, const LaunchCfg &g)
{
    return g.cls && has_class_table(ts, mode) ? ts->tab_cls[mode] : ts->tab[mode];
}

static const lx_tuned *tuned_for(const lx_ctx *c, const lx_tokenset *ts, int mode)
{
    for (const lx_tuned &t : c->tuned)
        if (t.ts == ts && t.mode == mode) return &t;
    return nullptr;
}

uint32_t lx::warps_setting(const lx_ctx *c, const lx_tokenset *ts, int mode)
{
    if (c->warps) return c->warps;
    const lx_tuned *t = tuned_for(c, ts, mode);
    return t ? t->warps : 0u;
}

static LaunchCfg config_for(lx_ctx *c, const lx_tokenset *ts, int mode)
{
    LaunchCfg g;
    for (const lx_tuned &t : c->tuned)
        if (t.ts == ts && t.mode == mode) {
            g.ks = t.ks;
            g.ctas = t.ctas;
            g.cls = t.cls;
            return g;
        }
    // default: the byte-indexed table (one LOP3 per step) unless the smaller
    // class-indexed one lets more CTAs share an SM with a column of >= 32
    if (!has_class_table(ts, mode)) return g;
    int occ_b = 0, occ_c = 0;
    if (occupancy_for(c, ts->tab[mode].form, make_layout((uint32_t)ts->tab[mode].blob.size(), KS_DEFAULT).total,
                      &occ_b) != LX_OK)
        return g;
    for (uint32_t ks = KS_DEFAULT; ks >= 32; ks -= 2) {
        if (occupancy_for(c, FORM_CLASS, make_layout((uint32_t)ts->tab_cls[mode].blob.size(), ks).total, &occ_c) !=
            LX_OK)
            return g;
        if (occ_c > occ_b) {
            g.ks = ks;
            g.cls = 1;
            return g;
        }
    }
    return g;
}

// Grid of the tile kernel for a configuration: CTAs per SM as asked, never
// above what fits (shared memory, registers).
static int grid_for(lx_ctx *c, int form, uint32_t smem, const LaunchCfg &g, uint64_t n_tiles, uint32_t *grid)
{
    int occ = 0;
    int rc = occupancy_for(c, form, smem, &occ);
    if (rc != LX_OK) return rc;
    const uint64_t per_sm = g.ctas ? std::min<uint64_t>(g.ctas, (uint64_t)occ) : (uint64_t)occ;
    *grid = (uint32_t)std::min<uint64_t>(n_tiles, per_sm * c->num_sms);
    return LX_OK;
}

// A chunk the warp-tile kernel walks byte by byte beyond this length makes
// lx_lex switch to the enumerative path.
constexpr uint64_t SPARSE_LIMIT = 32 * 1024;

// Whether the mode's cut set (useful exact certificate for the exact modes,
// modulo-I certificate for LX_FILTERED_MODULO) holds any byte.
static bool mode_has_cuts(const lx_tokenset *ts, int mode)
{
    const uint32_t *m = mode == LX_FILTERED_MODULO ? ts->modulo : ts->exact;
    for (int i = 0; i < 8; i++)
        if (m[i]) return true;
    return false;
}

// The same for the warp-tile kernel, whose walk table also cuts at certified
// two-byte windows in the exact modes.
static bool warp_has_cuts(const lx_tokenset *ts, int mode)
{
    return mode_has_cuts(ts, mode) || (ts->walk[mode].status == LX_OK && ts->walk[mode].n_ctx > 0);
}

// Launch the tile kernel and read back its result record.
static int lex_device(lx_ctx *c, const lx_tokenset *ts, const uint8_t *d_in, uint64_t n, int mode,
                      uint16_t *d_kinds, uint32_t *d_lens, uint64_t capacity, uint64_t *n_tokens,
                      uint64_t *consumed, cudaStream_t st, const LaunchCfg *force = nullptr)
{
    // Hybrid plan (Section 9): certified cuts where certified bytes occur;
    // where the mode certifies no byte, or certified bytes turn out too far
    // apart, entry contexts are enumerated instead (lx_lex_enumerative), so
    // no call degenerates to one lane walking the input.
    const bool can_enumerate = !force && c->kernel == LX_KERNEL_AUTO && ts->scan.status == LX_OK;
    const lx_tuned *tu = tuned_for(c, ts, mode);
    const bool tuned_tile = c->kernel == LX_KERNEL_AUTO && tu && tu->kernel == LX_KERNEL_TILE;
    const bool warp_ok = !force && c->kernel != LX_KERNEL_TILE && warp_path_ok(ts, mode, d_in);
    // the tile kernel cuts at single certified bytes only; the warp kernel also at windows
    const bool warp_windows = warp_ok && !mode_has_cuts(ts, mode) && warp_has_cuts(ts, mode);
    if (can_enumerate && !mode_has_cuts(ts, mode) && !warp_windows)
        return lx_lex_enumerative(c, ts, d_in, n, mode, d_kinds, d_lens, capacity, n_tokens, consumed, st);
    if (warp_ok && (!tuned_tile || warp_windows)) {
        const int rc = lex_warp_device(c, ts, d_in, n, mode, d_kinds, d_lens, capacity, n_tokens, consumed, st,
                                       can_enumerate ? SPARSE_LIMIT : 0);
        if (rc != LX_SPARSE && rc != LX_LOOKAHEAD) return rc;
        return lex_enumerative_device(c, ts, d_in, n, mode, d_kinds, d_lens, capacity, n_tokens, consumed, st,
                                      rc == LX_LOOKAHEAD);
    }
    if (!force && c->kernel == LX_KERNEL_WARP && n) return LX_E_INVAL;   // asked for, not available here
    if (ts->tab[mode].status != LX_OK) return ts->tab[mode].status;
    const LaunchCfg g = force ? *force : config_for(c, ts, mode);
    const HostTable &h = table_for(ts, mode, g);
    if (n == 0) {
        *n_tokens = 0;
        *consumed = 0;
        return LX_OK;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != c->device) return LX_E_INVAL;
    DeviceTables dt;
    int rc = ensure_device_tables(ts, dev, &dt);
    if (rc != LX_OK) return rc;
    void *blob = &h == &ts->tab_cls[mode] ? dt.d_blob_cls[mode] : dt.d_blob[mode];

    const uint64_t n_tiles64 = (n + TILE - 1) / TILE;
    if (n_tiles64 > 0xFFFFFFF0ull) return LX_E_INVAL;
    const uint32_t n_tiles = (uint32_t)n_tiles64;
    const size_t need = 64 + sizeof(unsigned long long) * (size_t)n_tiles;   // zeroed per call
    const size_t spill_off = (need + 255) & ~(size_t)255;

    Params P;
    P.one.in = d_in;
    P.one.n = n;
    P.one.first_tile = 0;
    P.one.tma = ((reinterpret_cast<uintptr_t>(d_in) & 15u) == 0) ? 1u : 0u;
    P.docs = nullptr;
    P.tile_doc = nullptr;
    P.dres = nullptr;
    P.prev = nullptr;
    P.n_prev = 0;
    set_table_params(P, h, blob);
    P.out_kinds = d_kinds;
    P.out_lens = d_lens;
    P.cap = capacity;
    P.n_tiles = n_tiles;
    P.timeout_ns = c->timeout_ns;
    P.ks = g.ks;
    P.withhold = c->withhold;

    const Layout L = make_layout(P.blob_bytes, P.ks);
    const int form = h.form;
    uint32_t grid = 0;
    rc = grid_for(c, form, L.total, g, n_tiles, &grid);
    if (rc != LX_OK) return rc;

    // scratch: result record, tile counter, status words, then the spill regions
    rc = grow(&c->scratch, &c->scratch_bytes, spill_off + sizeof(uint32_t) * (size_t)SPILL_WORDS * grid);
    if (rc != LX_OK) return rc;
    uint8_t *scr = static_cast<uint8_t *>(c->scratch);
    P.res = reinterpret_cast<Result *>(scr);
    P.tile_counter = reinterpret_cast<unsigned int *>(scr + 32);
    P.status = reinterpret_cast<unsigned long long *>(scr + 64);
    P.spill = reinterpret_cast<uint32_t *>(scr + spill_off);
    P.spill_cap = SPILL_WORDS;

    rc = cuda_err(cudaMemsetAsync(c->scratch, 0, need, st));
    if (rc != LX_OK) return rc;
    if (c->timing) cudaEventRecord(c->ev[0], st);
    launch_tiles(form, grid, L.total, st, P);
    rc = cuda_err(cudaGetLastError());
    if (c->timing) cudaEventRecord(c->ev[1], st);
    if (rc != LX_OK) return rc;
    rc = cuda_err(cudaMemcpyAsync(c->h_res, P.res, sizeof(Result), cudaMemcpyDeviceToHost, st));
    if (rc == LX_OK) rc = cuda_err(cudaStreamSynchronize(st));
    if (rc != LX_OK) return rc;
    const Result r = *static_cast<const Result *>(c->h_res);
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

static int check_args(lx_ctx *c, const lx_tokenset *ts, const void *in, uint64_t n, int mode, const void *k,
                      const void *l, uint64_t cap, uint64_t *n_tokens, uint64_t *consumed)
{
    if (!c || !ts || !n_tokens || !consumed) return LX_E_INVAL;
    if (mode < LX_FULL_EXACT || mode > LX_FILTERED_MODULO) return LX_E_MODE;
    if (n && !in) return LX_E_INVAL;
    if (cap && (!k || !l)) return LX_E_INVAL;
    return LX_OK;
}

extern "C" int lx_lex(lx_ctx *c, const lx_tokenset *ts, const uint8_t *d_in, uint64_t n, int mode,
                      uint16_t *d_kinds, uint32_t *d_lens, uint64_t capacity, uint64_t *n_tokens,
                      uint64_t *consumed, void *stream)
{
    int rc = check_args(c, ts, d_in, n, mode, d_kinds, d_lens, capacity, n_tokens, consumed);
    if (rc != LX_OK) return rc;
    return lex_device(c, ts, d_in, n, mode, d_kinds, d_lens, capacity, n_tokens, consumed,
                      static_cast<cudaStream_t>(stream));
}

// lx_lex_host splits inputs of at least 2 * HOST_PIECE bytes into up to
// HOST_PIECES pieces at certified bytes (the planner of Section 6 on the
// host: each equal-division target slides forward to the next byte of the
// mode's cut set, within HOST_SLIDE bytes), so that the copy of one piece in,
// the lexing of another and the copy of a third's tokens out overlap.  Each
// piece is lexed by its own launch, in order on the caller's stream, its
// output placed after the previous pieces' tokens (device-side totals).
constexpr uint64_t HOST_PIECE = 32ull << 20;
constexpr uint32_t HOST_PIECES = 8;
constexpr uint64_t HOST_SLIDE = 4ull << 20;

// A piece's record is written into pinned host memory by a one-warp kernel
// rather than a device-to-host copy, which would queue on the copy engine
// behind the previous piece's tokens.
__global__ void copy_record(const Result *src, Result *dst)
{
    if (threadIdx.x < sizeof(Result) / 8)
        reinterpret_cast<volatile unsigned long long *>(dst)[threadIdx.x] =
            reinterpret_cast<const volatile unsigned long long *>(src)[threadIdx.x];
}

static std::vector<uint64_t> host_pieces(const HostTable &h, const uint8_t *in, uint64_t n)
{
    std::vector<uint64_t> b{0};
    const uint8_t *cert = h.blob.data() + h.cert_off;
    uint32_t k = (uint32_t)std::min<uint64_t>(HOST_PIECES, n / HOST_PIECE);
    bool any = false;
    for (uint32_t x = 0; x < 256; x++) any |= cert[x] != 0;
    if (!any || k < 2) k = 1;
    for (uint32_t i = 1; i < k; i++) {
        uint64_t t = n / k * i;
        const uint64_t lim = std::min(n, t + HOST_SLIDE);
        while (t < lim && !cert[in[t]]) t++;
        if (t < lim && t > b.back()) b.push_back(t);
    }
    b.push_back(n);
    return b;
}

extern "C" int lx_lex_host(lx_ctx *c, const lx_tokenset *ts, const uint8_t *h_in, uint64_t n, int mode,
                           uint16_t *h_kinds, uint32_t *h_lens, uint64_t capacity, uint64_t *n_tokens,
                           uint64_t *consumed, void *stream)
{
    int rc = check_args(c, ts, h_in, n, mode, h_kinds, h_lens, capacity, n_tokens, consumed);
    if (rc != LX_OK) return rc;
    if (ts->tab[mode].status != LX_OK) return ts->tab[mode].status;
    const LaunchCfg g = config_for(c, ts, mode);
    const HostTable &h = table_for(ts, mode, g);
    *n_tokens = 0;
    *consumed = 0;
    if (n == 0) return LX_OK;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != c->device) return LX_E_INVAL;
    DeviceTables dt;
    rc = ensure_device_tables(ts, dev, &dt);
    if (rc != LX_OK) return rc;
    void *blob = &h == &ts->tab_cls[mode] ? dt.d_blob_cls[mode] : dt.d_blob[mode];
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rc = grow(&c->d_in, &c->d_in_bytes, n);
    if (rc == LX_OK) rc = grow(&c->d_out, &c->d_out_bytes, capacity ? capacity * 6 + 16 : 16);
    if (rc != LX_OK) return rc;
    cudaStream_t st0 = static_cast<cudaStream_t>(stream);
    // the whole input in, one device-side call, the tokens out
    auto whole = [&](bool enumerate) -> int {
        int r = grow(&c->d_in, &c->d_in_bytes, n);
        if (r == LX_OK) r = grow(&c->d_out, &c->d_out_bytes, capacity ? capacity * 6 + 16 : 16);
        if (r == LX_OK) r = cuda_err(cudaMemcpyAsync(c->d_in, h_in, n, cudaMemcpyHostToDevice, st0));
        if (r != LX_OK) return r;
        uint32_t *dl = static_cast<uint32_t *>(c->d_out);
        uint16_t *dk = reinterpret_cast<uint16_t *>(dl + capacity);
        const uint8_t *di = static_cast<const uint8_t *>(c->d_in);
        uint64_t nt = 0, con = 0;
        r = enumerate ? lx_lex_enumerative(c, ts, di, n, mode, dk, dl, capacity, &nt, &con, stream)
                      : lex_device(c, ts, di, n, mode, dk, dl, capacity, &nt, &con, st0);
        if (r != LX_OK && r != LX_E_CAPACITY) return r;
        const uint64_t m = std::min(nt, capacity);
        int r2 = LX_OK;
        if (m) r2 = cuda_err(cudaMemcpyAsync(h_kinds, dk, 2 * m, cudaMemcpyDeviceToHost, st0));
        if (m && r2 == LX_OK) r2 = cuda_err(cudaMemcpyAsync(h_lens, dl, 4 * m, cudaMemcpyDeviceToHost, st0));
        if (r2 == LX_OK) r2 = cuda_err(cudaStreamSynchronize(st0));
        if (r2 != LX_OK) return r2;
        *n_tokens = nt;
        *consumed = con;
        return r;
    };
    // the warp-tile kernel where it applies (it also cuts at certified windows)
    const bool warp = c->kernel != LX_KERNEL_TILE && ts->walk[mode].status == LX_OK;
    if (c->kernel == LX_KERNEL_WARP && !warp) return LX_E_INVAL;   // as lx_lex: asked for a kernel that cannot serve
    const bool can_enumerate = c->kernel == LX_KERNEL_AUTO && ts->scan.status == LX_OK;
    if (can_enumerate && !(warp ? warp_has_cuts(ts, mode) : mode_has_cuts(ts, mode)))
        return whole(true);   // no certified byte: the enumerative path

    const std::vector<uint64_t> b = host_pieces(h, h_in, n);
    const uint32_t K = (uint32_t)b.size() - 1;
    if (!c->s_in && (cudaStreamCreateWithFlags(&c->s_in, cudaStreamNonBlocking) != cudaSuccess ||
                     cudaStreamCreateWithFlags(&c->s_out, cudaStreamNonBlocking) != cudaSuccess))
        return LX_E_CUDA;
    while (c->ev_in.size() < K) {
        cudaEvent_t e1 = nullptr, e2 = nullptr;
        if (cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&e2, cudaEventDisableTiming) != cudaSuccess)
            return LX_E_CUDA;
        c->ev_in.push_back(e1);
        c->ev_lex.push_back(e2);
    }
    if (warp) {
        rc = lex_warp_host(c, ts, h_in, n, mode, h_kinds, h_lens, capacity, b.data(), K, n_tokens, consumed, st,
                           can_enumerate ? SPARSE_LIMIT : 0);
        if (rc != LX_SPARSE && rc != LX_LOOKAHEAD) return rc;
        // certified bytes too far apart, or failed lookahead, in some piece:
        // the whole input through lx_lex's plan
        return whole(false);
    }
    uint32_t *d_lens = static_cast<uint32_t *>(c->d_out);
    uint16_t *d_kinds = reinterpret_cast<uint16_t *>(d_lens + capacity);
    const uint8_t *d_in = static_cast<const uint8_t *>(c->d_in);

    // scratch: one record + tile counter per piece, status words, spill regions
    const Layout L = make_layout((uint32_t)h.blob.size(), g.ks);
    uint32_t grid_max = 0;
    std::vector<uint32_t> tiles(K), grid(K);
    uint64_t tiles_total = 0;
    for (uint32_t i = 0; i < K; i++) {
        tiles[i] = (uint32_t)((b[i + 1] - b[i] + TILE - 1) / TILE);
        rc = grid_for(c, h.form, L.total, g, tiles[i], &grid[i]);
        if (rc != LX_OK) return rc;
        grid_max = std::max(grid_max, grid[i]);
        tiles_total += tiles[i];
    }
    const size_t o_cnt = (sizeof(Result) * K + 63) & ~(size_t)63, o_status = o_cnt + 64 * (size_t)K;
    const size_t zero = o_status + 8 * tiles_total;
    const size_t o_spill = (zero + 255) & ~(size_t)255;
    rc = grow(&c->scratch, &c->scratch_bytes, o_spill + sizeof(uint32_t) * (size_t)SPILL_WORDS * grid_max);
    if (rc == LX_OK) rc = grow_host(&c->h_scratch, &c->h_scratch_bytes, sizeof(Result) * (size_t)K);
    if (rc != LX_OK) return rc;
    uint8_t *scr = static_cast<uint8_t *>(c->scratch);
    Result *res = reinterpret_cast<Result *>(scr);   // one record per piece
    Result *h_res = static_cast<Result *>(c->h_scratch);
    Result *h_res_dev = nullptr;   // the same pinned records, as the device sees them
    if (cudaHostGetDevicePointer(reinterpret_cast<void **>(&h_res_dev), c->h_scratch, 0) != cudaSuccess)
        return LX_E_CUDA;
    uint8_t *d_in_w = static_cast<uint8_t *>(c->d_in);
    rc = cuda_err(cudaMemsetAsync(scr, 0, zero, st));
    if (rc != LX_OK) return rc;
    // the pieces in, each on its own event
    for (uint32_t i = 0; i < K; i++) {
        rc = cuda_err(cudaMemcpyAsync(d_in_w + b[i], h_in + b[i], b[i + 1] - b[i], cudaMemcpyHostToDevice, c->s_in));
        if (rc == LX_OK) rc = cuda_err(cudaEventRecord(c->ev_in[i], c->s_in));
        if (rc != LX_OK) return rc;
    }
    // the launches, in order on the caller's stream
    if (c->timing) cudaEventRecord(c->ev[0], st);
    uint64_t tile_off = 0;
    for (uint32_t i = 0; i < K; i++) {
        Params P;
        P.one = DocDesc{d_in + b[i], b[i + 1] - b[i], 0,
                        ((reinterpret_cast<uintptr_t>(d_in + b[i]) & 15u) == 0) ? 1u : 0u};
        P.docs = nullptr;
        P.tile_doc = nullptr;
        P.dres = nullptr;
        P.prev = res;
        P.n_prev = i;
        set_table_params(P, h, blob);
        P.out_kinds = d_kinds;
        P.out_lens = d_lens;
        P.cap = capacity;
        P.n_tiles = tiles[i];
        P.timeout_ns = c->timeout_ns;
        P.ks = g.ks;
        P.withhold = NONE32;
        P.res = res + i;
        P.tile_counter = reinterpret_cast<unsigned int *>(scr + o_cnt + 64 * (size_t)i);
        P.status = reinterpret_cast<unsigned long long *>(scr + o_status) + tile_off;
        P.spill = reinterpret_cast<uint32_t *>(scr + o_spill);
        P.spill_cap = SPILL_WORDS;
        tile_off += tiles[i];
        rc = cuda_err(cudaStreamWaitEvent(st, c->ev_in[i], 0));
        if (rc != LX_OK) return rc;
        launch_tiles(h.form, grid[i], L.total, st, P);
        copy_record<<<1, 32, 0, st>>>(P.res, h_res_dev + i);
        rc = cuda_err(cudaGetLastError());
        if (rc == LX_OK) rc = cuda_err(cudaEventRecord(c->ev_lex[i], st));
        if (rc != LX_OK) return rc;
    }
    if (c->timing) cudaEventRecord(c->ev[1], st);
    // each piece's tokens out as soon as it is lexed
    uint64_t out = 0, con = n;
    bool failed = false;
    for (uint32_t i = 0; i < K && !failed && rc == LX_OK; i++) {
        rc = cuda_err(cudaEventSynchronize(c->ev_lex[i]));
        if (rc != LX_OK) break;
        const Result r = h_res[i];
        if (r.error & ERR_TIMEOUT) rc = LX_E_TIMEOUT;
        if (r.error & ERR_SMEM) rc = LX_E_TOOBIG;
        if (rc != LX_OK) break;
        uint64_t end = out + r.total;
        if (r.inv_fail_pos) {   // Corollary 1: the first failing piece ends the stream
            end = ~r.inv_fail_tok;
            con = b[i] + ~r.inv_fail_pos;
            failed = true;
        }
        const uint64_t lo = std::min(out, capacity), hi = std::min(end, capacity);
        if (hi > lo) {
            rc = cuda_err(cudaMemcpyAsync(h_kinds + lo, d_kinds + lo, (hi - lo) * 2, cudaMemcpyDeviceToHost, c->s_out));
            if (rc == LX_OK)
                rc = cuda_err(cudaMemcpyAsync(h_lens + lo, d_lens + lo, (hi - lo) * 4, cudaMemcpyDeviceToHost, c->s_out));
        }
        out = end;
    }
    int r2 = cuda_err(cudaStreamSynchronize(c->s_out));
    if (rc == LX_OK) rc = r2;
    r2 = cuda_err(cudaStreamSynchronize(st));
    if (rc == LX_OK) rc = r2;
    if (rc != LX_OK) return rc;
    *n_tokens = out;
    *consumed = con;
    return out > capacity ? LX_E_CAPACITY : LX_OK;
}


// ---------------------------------------------------------------------------
// lx_lex_batch
// ---------------------------------------------------------------------------
namespace {

struct BatchGroup {
    uint32_t set;
    uint32_t doc_begin, doc_end;   // range in the grouped document order
    uint32_t tile_begin, n_tiles;  // range in the concatenated status / tile_doc arrays
};

// Byte offsets of the batch scratch (device) and staging (pinned host).
struct BatchLayout {
    size_t res, cnt, dres, status, zero_end;   // zeroed per call: [0, zero_end)
    size_t docs, tdoc, up_end;                 // uploaded per call: [docs, up_end)
    size_t spill, dev_total;
    // host staging: [0, up_bytes) descriptors, then [down, down + zero_end) records
    size_t up_bytes, down, host_total;
};

BatchLayout batch_layout(uint32_t G, uint32_t D, uint64_t TT, uint32_t grid)
{
    auto al = [](size_t x, size_t a) { return (x + a - 1) / a * a; };
    BatchLayout B;
    B.res = 0;
    B.cnt = al(sizeof(Result) * G, 64);
    B.dres = al(B.cnt + 4 * (size_t)G, 64);
    B.status = al(B.dres + sizeof(DocResult) * D, 64);
    B.zero_end = B.status + 8 * TT;
    B.docs = al(B.zero_end, 256);
    B.tdoc = al(B.docs + sizeof(DocDesc) * D, 64);
    B.up_end = B.tdoc + 4 * TT;
    B.spill = al(B.up_end, 256);
    B.dev_total = B.spill + sizeof(uint32_t) * (size_t)SPILL_WORDS * grid;
    B.up_bytes = B.up_end - B.docs;
    B.down = al(B.up_bytes, 64);
    B.host_total = B.down + B.status;
    return B;
}


}  // namespace

int lx::grow_host(void **p, size_t *have, size_t need)
{
    if (*have >= need) return LX_OK;
    if (*p) cudaFreeHost(*p);
    *p = nullptr;
    *have = 0;
    if (cudaMallocHost(p, need) != cudaSuccess) return LX_E_NOMEM;
    *have = need;
    return LX_OK;
}

extern "C" int lx_lex_batch(lx_ctx *c, const lx_tokenset *const *sets, uint32_t n_sets, const lx_doc *docs,
                            uint32_t n_docs, int mode, uint16_t *d_kinds, uint32_t *d_lens, uint64_t capacity,
                            lx_doc_result *results, uint64_t *n_total, void *stream)
{
    if (!c || !n_total || (n_docs && (!docs || !results)) || (n_sets && !sets)) return LX_E_INVAL;
    if (mode < LX_FULL_EXACT || mode > LX_FILTERED_MODULO) return LX_E_MODE;
    if (capacity && (!d_kinds || !d_lens)) return LX_E_INVAL;
    for (uint32_t s = 0; s < n_sets; s++)
        if (!sets[s]) return LX_E_INVAL;
    for (uint32_t i = 0; i < n_docs; i++) {
        if (docs[i].set >= n_sets || docs[i].reserved != 0) return LX_E_INVAL;
        if (docs[i].n && !docs[i].data) return LX_E_INVAL;
        results[i] = lx_doc_result{0, 0, 0};
    }
    *n_total = 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != c->device) return LX_E_INVAL;
    if (c->kernel != LX_KERNEL_TILE) {   // one launch for every document of every set
        const int rc = lex_batch_warp(c, sets, n_sets, docs, n_docs, mode, d_kinds, d_lens, capacity, results,
                                      n_total, st);
        if (rc != LX_SPARSE) return rc;
        for (uint32_t i = 0; i < n_docs; i++) results[i] = lx_doc_result{0, 0, 0};
        *n_total = 0;
    }
    for (uint32_t s = 0; s < n_sets; s++)
        if (sets[s]->tab[mode].status != LX_OK) return sets[s]->tab[mode].status;

    // group the non-empty documents by token set, keeping their order
    std::vector<uint32_t> order;
    std::vector<BatchGroup> groups;
    uint64_t TT = 0;
    for (uint32_t s = 0; s < n_sets; s++) {
        BatchGroup g{s, (uint32_t)order.size(), 0, (uint32_t)0, 0};
        uint64_t tiles = 0;
        for (uint32_t i = 0; i < n_docs; i++)
            if (docs[i].set == s && docs[i].n) {
                order.push_back(i);
                tiles += (docs[i].n + TILE - 1) / TILE;
            }
        g.doc_end = (uint32_t)order.size();
        if (g.doc_end == g.doc_begin) continue;
        if (tiles > 0xFFFFFFF0ull || TT + tiles > 0xFFFFFFF0ull) return LX_E_INVAL;
        g.tile_begin = (uint32_t)TT;
        g.n_tiles = (uint32_t)tiles;
        TT += tiles;
        groups.push_back(g);
    }
    if (groups.empty()) return LX_OK;
    const uint32_t G = (uint32_t)groups.size(), D = (uint32_t)order.size();

    // tables, occupancy and grid per group
    std::vector<void *> blob(G);
    std::vector<uint32_t> grid(G), smem(G);
    std::vector<LaunchCfg> cfg(G);
    uint32_t grid_max = 0;
    for (uint32_t k = 0; k < G; k++) {
        const lx_tokenset *ts = sets[groups[k].set];
        DeviceTables dt;
        int rc = ensure_device_tables(ts, dev, &dt);
        if (rc != LX_OK) return rc;
        cfg[k] = config_for(c, ts, mode);
        const HostTable &h = table_for(ts, mode, cfg[k]);
        blob[k] = &h == &ts->tab_cls[mode] ? dt.d_blob_cls[mode] : dt.d_blob[mode];
        smem[k] = make_layout((uint32_t)h.blob.size(), cfg[k].ks).total;
        rc = grid_for(c, h.form, smem[k], cfg[k], groups[k].n_tiles, &grid[k]);
        if (rc != LX_OK) return rc;
        grid_max = std::max(grid_max, grid[k]);
    }
    const BatchLayout B = batch_layout(G, D, TT, grid_max);
    bool moved = false;
    {
        void *old_d = c->b_dev, *old_h = c->b_host;
        int rc = grow(&c->b_dev, &c->b_dev_bytes, B.dev_total);
        if (rc == LX_OK) rc = grow_host(&c->b_host, &c->b_host_bytes, B.host_total);
        if (rc != LX_OK) return rc;
        moved = old_d != c->b_dev || old_h != c->b_host;
    }
    uint8_t *dv = static_cast<uint8_t *>(c->b_dev);
    uint8_t *hs = static_cast<uint8_t *>(c->b_host);

    // descriptors into the pinned staging area
    DocDesc *h_docs = reinterpret_cast<DocDesc *>(hs);
    uint32_t *h_tdoc = reinterpret_cast<uint32_t *>(hs + (B.tdoc - B.docs));
    for (const BatchGroup &g : groups) {
        uint32_t t = 0;
        for (uint32_t j = g.doc_begin; j < g.doc_end; j++) {
            const lx_doc &d = docs[order[j]];
            const uint32_t nt = (uint32_t)((d.n + TILE - 1) / TILE);
            h_docs[j] = DocDesc{d.data, d.n, t, (reinterpret_cast<uintptr_t>(d.data) & 15u) == 0 ? 1u : 0u};
            for (uint32_t k = 0; k < nt; k++) h_tdoc[g.tile_begin + t + k] = j - g.doc_begin;
            t += nt;
        }
    }

    // the graph's shape: everything baked into its nodes
    std::vector<uint64_t> key = {G, D, TT, (uint64_t)mode, (uint64_t)(uintptr_t)d_kinds, (uint64_t)(uintptr_t)d_lens,
                                 capacity, (uint64_t)(uintptr_t)dv, (uint64_t)(uintptr_t)hs, c->timeout_ns};
    for (uint32_t k = 0; k < G; k++) {
        key.push_back((uint64_t)(uintptr_t)blob[k]);
        key.push_back(groups[k].doc_begin);
        key.push_back(groups[k].n_tiles);
        key.push_back(grid[k]);
        key.push_back(cfg[k].ks);
    }
    if (moved || key != c->b_key || !c->b_exec) {
        if (c->b_exec) cudaGraphExecDestroy(c->b_exec);
        c->b_exec = nullptr;
        c->b_key.clear();
        if (!c->b_stream && cudaStreamCreateWithFlags(&c->b_stream, cudaStreamNonBlocking) != cudaSuccess)
            return LX_E_CUDA;
        cudaStream_t cs = c->b_stream;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return LX_E_CUDA;
        cudaMemsetAsync(dv, 0, B.zero_end, cs);
        cudaMemcpyAsync(dv + B.docs, hs, B.up_bytes, cudaMemcpyHostToDevice, cs);
        Result *res = reinterpret_cast<Result *>(dv + B.res);
        for (uint32_t k = 0; k < G; k++) {
            const BatchGroup &g = groups[k];
            const HostTable &h = table_for(sets[g.set], mode, cfg[k]);
            Params P;
            P.one = DocDesc{nullptr, 0, 0, 0};
            P.docs = reinterpret_cast<const DocDesc *>(dv + B.docs) + g.doc_begin;
            P.tile_doc = reinterpret_cast<const uint32_t *>(dv + B.tdoc) + g.tile_begin;
            P.dres = reinterpret_cast<DocResult *>(dv + B.dres) + g.doc_begin;
            P.prev = res;
            P.n_prev = k;
            set_table_params(P, h, blob[k]);
            P.out_kinds = d_kinds;
            P.out_lens = d_lens;
            P.cap = capacity;
            P.status = reinterpret_cast<unsigned long long *>(dv + B.status) + g.tile_begin;
            P.tile_counter = reinterpret_cast<unsigned int *>(dv + B.cnt) + k;
            P.res = res + k;
            P.n_tiles = g.n_tiles;
            P.spill = reinterpret_cast<uint32_t *>(dv + B.spill);
            P.spill_cap = SPILL_WORDS;
            P.timeout_ns = c->timeout_ns;
            P.ks = cfg[k].ks;
            P.withhold = NONE32;
            launch_tiles(h.form, grid[k], smem[k], cs, P);
        }
        cudaMemcpyAsync(hs + B.down, dv, B.zero_end - 8 * TT, cudaMemcpyDeviceToHost, cs);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&c->b_exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            c->b_exec = nullptr;
            cudaGetLastError();
            return LX_E_CUDA;
        }
        c->b_key = key;
    }
    if (c->timing) cudaEventRecord(c->ev[0], st);
    int rc = cuda_err(cudaGraphLaunch(c->b_exec, st));
    if (c->timing) cudaEventRecord(c->ev[1], st);
    if (rc == LX_OK) rc = cuda_err(cudaStreamSynchronize(st));
    if (rc != LX_OK) return rc;

    // records
    const Result *h_res = reinterpret_cast<const Result *>(hs + B.down + B.res);
    const DocResult *h_dres = reinterpret_cast<const DocResult *>(hs + B.down + B.dres);
    uint64_t total = 0;
    for (uint32_t k = 0; k < G; k++) {
        if (h_res[k].error & ERR_TIMEOUT) return LX_E_TIMEOUT;
        if (h_res[k].error & ERR_SMEM) return LX_E_TOOBIG;
        total += h_res[k].total;
    }
    for (uint32_t j = 0; j < D; j++) {
        const DocResult &r = h_dres[j];
        const lx_doc &d = docs[order[j]];
        lx_doc_result &o = results[order[j]];
        if (r.out_off1 == 0) return LX_E_CUDA;   // every document's first tile reports its offset
        o.out_off = r.out_off1 - 1;
        if (r.inv_fail_pos) {
            o.consumed = ~r.inv_fail_pos;
            o.n_tokens = ~r.inv_fail_tok - o.out_off;
        } else {
            o.consumed = d.n;
            o.n_tokens = r.total;
        }
    }
    *n_total = total;
    return total > capacity ? LX_E_CAPACITY : LX_OK;
}

// ---------------------------------------------------------------------------
// launch configuration: set by hand or measured
// ---------------------------------------------------------------------------
static void store_config(lx_ctx *c, const lx_tokenset *ts, int mode, const LaunchCfg &g, float ms)
{
    bool found = false;
    for (lx_tuned &t : c->tuned)
        if (t.ts == ts && t.mode == mode) {
            t.ks = g.ks;
            t.ctas = g.ctas;
            t.cls = g.cls;
            t.ms = ms;
            t.kernel = 0;   // a configuration set by hand: the default kernel choice again
            t.warps = 0;
            found = true;
        }
    if (!found) c->tuned.push_back(lx_tuned{ts, mode, g.ks, g.ctas, g.cls, ms, 0, 0});
    if (c->b_exec) {   // a cached batch graph may hold the old configuration
        cudaGraphExecDestroy(c->b_exec);
        c->b_exec = nullptr;
        c->b_key.clear();
    }
}

extern "C" int lx_ctx_set_config(lx_ctx *c, const lx_tokenset *ts, int mode, uint32_t ks, uint32_t ctas_per_sm,
                                 uint32_t class_table)
{
    if (!c || !ts) return LX_E_INVAL;
    if (mode < LX_FULL_EXACT || mode > LX_FILTERED_MODULO) return LX_E_MODE;
    if (ks < KS_MIN || ks > LX_KS_MAX || class_table > 1) return LX_E_INVAL;
    LaunchCfg g;
    g.ks = ks;
    g.ctas = ctas_per_sm;
    g.cls = class_table && has_class_table(ts, mode) ? 1u : 0u;
    if (make_layout((uint32_t)table_for(ts, mode, g).blob.size(), ks).total > 200u * 1024u) return LX_E_TOOBIG;
    store_config(c, ts, mode, g, 0.0f);
    return LX_OK;
}

extern "C" int lx_ctx_get_config(lx_ctx *c, const lx_tokenset *ts, int mode, uint32_t *ks, uint32_t *ctas_per_sm,
                                 uint32_t *class_table, float *ms)
{
    if (!c || !ts) return LX_E_INVAL;
    if (mode < LX_FULL_EXACT || mode > LX_FILTERED_MODULO) return LX_E_MODE;
    const LaunchCfg g = config_for(c, ts, mode);
    float t = 0.0f;
    for (const lx_tuned &x : c->tuned)
        if (x.ts == ts && x.mode == mode) t = x.ms;
    if (ks) *ks = g.ks;
    if (ctas_per_sm) *ctas_per_sm = g.ctas;
    if (class_table) *class_table = table_for(ts, mode, g).form == FORM_CLASS ? 1u : 0u;
    if (ms) *ms = t;
    return LX_OK;
}

extern "C" int lx_autotune(lx_ctx *c, const lx_tokenset *ts, int mode, const uint8_t *d_sample, uint64_t n,
                           uint16_t *d_kinds, uint32_t *d_lens, uint64_t capacity, void *stream)
{
    uint64_t unused_t = 0, unused_c = 0;
    int rc = check_args(c, ts, d_sample, n, mode, d_kinds, d_lens, capacity, &unused_t, &unused_c);
    if (rc != LX_OK || n == 0) return rc == LX_OK ? LX_E_INVAL : rc;
    if (ts->tab[mode].status != LX_OK) return ts->tab[mode].status;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return LX_E_CUDA;
    }
    const bool timing = c->timing;
    c->timing = false;
    float best = 1e30f;
    LaunchCfg best_g;
    uint64_t ref_tokens = ~0ull, ref_con = ~0ull;
    static const uint32_t ks_list[] = {24, 32, 36, 40, 48, 56, 64};
    for (uint32_t cls = 0; cls < (has_class_table(ts, mode) ? 2u : 1u) && rc == LX_OK; cls++) {
        for (uint32_t ks : ks_list) {
            LaunchCfg g0;
            g0.ks = ks;
            g0.cls = cls;
            const HostTable &h = table_for(ts, mode, g0);
            const uint32_t smem = make_layout((uint32_t)h.blob.size(), ks).total;
            if (smem > 200u * 1024u) continue;
            int occ = 0;
            rc = occupancy_for(c, h.form, smem, &occ);
            if (rc != LX_OK) break;
            for (uint32_t ctas : {(uint32_t)occ, 1u}) {
                if (ctas == 1 && occ == 1) continue;
                LaunchCfg g = g0;
                g.ctas = ctas;
                uint64_t nt = 0, con = 0;
                float total = 0.0f;
                for (int rep = 0; rep < 4 && rc == LX_OK; rep++) {
                    cudaEventRecord(e0, st);
                    rc = lex_device(c, ts, d_sample, n, mode, d_kinds, d_lens, capacity, &nt, &con, st, &g);
                    cudaEventRecord(e1, st);
                    if (rc == LX_E_CAPACITY) rc = LX_OK;
                    if (rc != LX_OK) break;
                    cudaEventSynchronize(e1);
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep) total += ms;   // the first run warms up
                }
                if (rc != LX_OK) break;
                if (ref_tokens == ~0ull) {
                    ref_tokens = nt;
                    ref_con = con;
                } else if (nt != ref_tokens || con != ref_con) {
                    rc = LX_E_CUDA;   // every configuration must give the same result
                    break;
                }
                if (total / 3 < best) {
                    best = total / 3;
                    best_g = g;
                }
            }
            if (rc != LX_OK) break;
        }
    }
    // the warp-tile kernel at several warps per CTA, when it applies
    float best_w = 1e30f;
    uint32_t best_nw = 0;
    const uint32_t saved_warps = c->warps;
    if (rc == LX_OK && warp_path_ok(ts, mode, d_sample)) {
        for (uint32_t nw : {4u, 8u, 12u, 16u, 20u}) {
            c->warps = nw;
            uint64_t nt = 0, con = 0;
            float total = 0.0f;
            for (int rep = 0; rep < 4 && rc == LX_OK; rep++) {
                cudaEventRecord(e0, st);
                rc = lex_warp_device(c, ts, d_sample, n, mode, d_kinds, d_lens, capacity, &nt, &con, st, 0);
                cudaEventRecord(e1, st);
                if (rc == LX_E_CAPACITY) rc = LX_OK;
                if (rc != LX_OK) break;
                cudaEventSynchronize(e1);
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep) total += ms;
            }
            if (rc != LX_OK) break;
            if (ref_tokens == ~0ull) {
                ref_tokens = nt;
                ref_con = con;
            } else if (nt != ref_tokens || con != ref_con) {
                rc = LX_E_CUDA;
                break;
            }
            if (total / 3 < best_w) {
                best_w = total / 3;
                best_nw = nw;
            }
        }
    }
    c->warps = saved_warps;
    c->timing = timing;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != LX_OK) return rc;
    store_config(c, ts, mode, best_g, best);
    for (lx_tuned &t : c->tuned)
        if (t.ts == ts && t.mode == mode) {
            t.kernel = best_nw && best_w < best ? LX_KERNEL_WARP : LX_KERNEL_TILE;
            t.warps = best_nw;
            if (t.kernel == LX_KERNEL_WARP) t.ms = best_w;
        }
    return LX_OK;
}

extern "C" const char *lx_strerror(int code)
{
    switch (code) {
    case LX_OK: return "ok";
    case LX_E_INVAL: return "invalid argument or automaton";
    case LX_E_NOMEM: return "out of memory";
    case LX_E_CAPACITY: return "output capacity too small";
    case LX_E_CUDA: return "CUDA runtime error";
    case LX_E_TIMEOUT: return "device-side wait timed out";
    case LX_E_MODE: return "invalid lexing mode";
    case LX_E_TOOBIG: return "automaton too large for shared-memory tables";
    default: return "unknown error";
    }
}

// ---------------------------------------------------------------------------
// lx_lex_noalloc: the same tile kernel, with every piece of scratch in one
// fixed device array instead of context allocations.
// ---------------------------------------------------------------------------
namespace lx {

constexpr size_t NA_TABLE_BYTES = 64 * 1024;            // walk-table blob of one mode
constexpr size_t NA_RESULT = NA_TABLE_BYTES;            // Result, then the tile counter
constexpr size_t NA_STATUS = NA_TABLE_BYTES + 64;       // one u64 status word per tile
constexpr uint64_t NA_MAX_TILES = (LX_NOALLOC_SCRATCH_BYTES - NA_STATUS) / 8;
static_assert(NA_MAX_TILES * TILE == LX_NOALLOC_MAX_INPUT, "LX_NOALLOC_MAX_INPUT out of date");
// the largest walk-table blob (rows, byte-form kind words, class map and cut
// table, 16-byte padding) fits the table slot, so it never reaches the status words
static_assert(MAX_TABLE_BYTES + 2 * (MAX_BYTE_FORM_BYTES / 512) + 16 + 256 + 256 + 16 <= NA_TABLE_BYTES,
              "walk tables can overrun the no-alloc table slot");

static __device__ __align__(256) unsigned char g_noalloc_scratch[LX_NOALLOC_SCRATCH_BYTES];

constexpr int NA_MAX_DEVICES = 64;
struct NoallocDevice {
    bool ready = false;
    unsigned char *scratch = nullptr;   // device address of g_noalloc_scratch on this device
    int num_sms = 0;
};
static std::mutex g_noalloc_mu;
static NoallocDevice g_noalloc_dev[NA_MAX_DEVICES];

// One-time set-up on the current device: the host-side name of the array is
// not a device address, so ask the runtime for it.
static int noalloc_setup(int dev, NoallocDevice &d)
{
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (d.ready) return LX_OK;
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) return LX_E_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LX_E_CUDA;
    if (cudaFuncSetAttribute(lex_tiles<FORM_BYTE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
            cudaSuccess ||
        cudaFuncSetAttribute(lex_tiles<FORM_CLASS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
            cudaSuccess)
        return LX_E_CUDA;
    d.scratch = static_cast<unsigned char *>(ptr);
    d.num_sms = sms;
    d.ready = true;
    return LX_OK;
}

}  // namespace lx

extern "C" int lx_lex_noalloc(const lx_tokenset *ts, const uint8_t *d_in, uint64_t n, int mode, uint16_t *d_kinds,
                              uint32_t *d_lens, uint64_t capacity, uint64_t *n_tokens, uint64_t *consumed,
                              void *stream)
{
    if (!ts || !n_tokens || !consumed) return LX_E_INVAL;
    if (mode < LX_FULL_EXACT || mode > LX_FILTERED_MODULO) return LX_E_MODE;
    if (n && !d_in) return LX_E_INVAL;
    if (capacity && (!d_kinds || !d_lens)) return LX_E_INVAL;
    if (n > LX_NOALLOC_MAX_INPUT) return LX_E_INVAL;
    const HostTable &h = ts->tab[mode];
    if (h.status != LX_OK) return h.status;
    if (h.blob.size() > NA_TABLE_BYTES) return LX_E_TOOBIG;
    if (n == 0) {
        *n_tokens = 0;
        *consumed = 0;
        return LX_OK;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return LX_E_CUDA;
    NoallocDevice &d = g_noalloc_dev[dev];
    int rc = noalloc_setup(dev, d);
    if (rc != LX_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    const uint32_t n_tiles = (uint32_t)((n + TILE - 1) / TILE);
    unsigned char *scr = d.scratch;
    // zero the result record, the tile counter and this call's status words;
    // bring in this token set's tables for `mode`
    rc = cuda_err(cudaMemsetAsync(scr + NA_RESULT, 0, 64 + 8 * (size_t)n_tiles, st));
    if (rc == LX_OK)
        rc = cuda_err(cudaMemcpyAsync(scr, h.blob.data(), h.blob.size(), cudaMemcpyHostToDevice, st));
    if (rc != LX_OK) return rc;

    Params P;
    P.one.in = d_in;
    P.one.n = n;
    P.one.first_tile = 0;
    P.one.tma = ((reinterpret_cast<uintptr_t>(d_in) & 15u) == 0) ? 1u : 0u;
    P.docs = nullptr;
    P.tile_doc = nullptr;
    P.dres = nullptr;
    P.prev = nullptr;
    P.n_prev = 0;
    set_table_params(P, h, scr);
    P.out_kinds = d_kinds;
    P.out_lens = d_lens;
    P.cap = capacity;
    P.res = reinterpret_cast<Result *>(scr + NA_RESULT);
    P.tile_counter = reinterpret_cast<unsigned int *>(scr + NA_RESULT + 32);
    P.status = reinterpret_cast<unsigned long long *>(scr + NA_STATUS);
    P.spill = nullptr;   // no spill region: long ranges take the generic walker
    P.spill_cap = 0;
    P.ks = KS_DEFAULT;
    P.withhold = NONE32;
    P.n_tiles = n_tiles;
    P.timeout_ns = 20ull * 1000 * 1000 * 1000;

    const Layout L = make_layout(P.blob_bytes, P.ks);
    int occ = 0;
    cudaError_t e = h.form == FORM_BYTE
                        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lex_tiles<FORM_BYTE>, NT, L.total)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lex_tiles<FORM_CLASS>, NT, L.total);
    if (e != cudaSuccess) return LX_E_CUDA;
    if (occ < 1) occ = 1;
    const uint32_t grid = (uint32_t)std::min<uint64_t>(n_tiles, (uint64_t)occ * d.num_sms);
    if (h.form == FORM_BYTE) lex_tiles<FORM_BYTE><<<grid, NT, L.total, st>>>(P);
    else lex_tiles<FORM_CLASS><<<grid, NT, L.total, st>>>(P);
    rc = cuda_err(cudaGetLastError());
    if (rc != LX_OK) return rc;
    Result r;
    rc = cuda_err(cudaMemcpyAsync(&r, P.res, sizeof(Result), cudaMemcpyDeviceToHost, st));
    if (rc == LX_OK) rc = cuda_err(cudaStreamSynchronize(st));
    if (rc != LX_OK) return rc;
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
