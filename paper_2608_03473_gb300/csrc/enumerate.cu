// enumerate.cu -- lx_lex_enumerative: splitting an input whose token set
// certifies no byte (the paper's refused sets, Table 2), by enumerating the
// entry context of every chunk.
//
// The serial scan of Section 3 at an offset p is either at a token boundary
// or inside a token, in the DFA state reached from q0 over the token's bytes
// before p.  Scanning on from that state finds the same token end (the
// longest match keeps the last accepting position), so a chunk entered in
// the right context yields exactly the serial tokens that start in it.  The
// context right after a byte b is BOUNDARY or one of delta+(q, b), q in Q+;
// the planner puts every chunk start after a byte with few such candidates.
//   (1) plan:      per CHUNK-byte target, the start in its first WIN bytes
//                  after the byte with the fewest candidates (none when every
//                  byte there has more than KMAX);
//   (2) enumerate: per chunk and candidate, scan the chunk from that context:
//                  kept-token count, exit context at the next chunk start
//                  (the chunk reads past its end to finish its last token),
//                  or the failure offset;
//   (3) resolve:   the chain of exits from BOUNDARY at offset 0: runs of 16
//                  chunks summarised per candidate (one thread each), groups of
//                  runs composed and linked in one CTA, then each run labelled:
//                  every chunk's true entry context and output offset, and the
//                  first failure (Corollary 1);
//   (4) emit:      per chunk, scan once more from its true context and write
//                  its tokens at its offset.
// The result is tok(w) (or pi_I(tok(w))) and con(w) exactly.

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "internal.h"
#include "runtime.h"

namespace lx {
namespace {

constexpr uint32_t CHUNK = 4096;       // bytes per chunk target
constexpr uint32_t WIN = 256;          // a chunk start is searched in the target's first WIN bytes
constexpr uint32_t KMAX = 8;           // candidate contexts per chunk start (BOUNDARY included)
constexpr int EN_NT = 256;             // threads of the plan / enumerate / emit kernels
constexpr int RS_NT = 1024;            // threads of the resolve kernel
constexpr int SO_NT = 1024;            // threads of the offset kernels (one chunk each)
constexpr uint32_t R1 = 16;            // chunks per run of the resolve kernels
constexpr uint32_t SPEC_ROUNDS = 8;    // speculative rounds before the enumerative judge (a round that
                                       // rescans nothing costs two short launches; the judge a whole enumeration)
constexpr uint32_t STEP_BUDGET = 32 * 4096;   // steps of one unguarded chunk scan before the guard is called for
constexpr unsigned EN_ERR_STATE = 1u;  // the resolve step met an impossible chain (never on valid tables)
constexpr unsigned EN_ERR_LOOKAHEAD = 2u;   // a scan ran past STEP_BUDGET
constexpr uint64_t NOPOS64 = ~0ull;
constexpr uint32_t NONE32_EN = 0xFFFFFFFFu;
constexpr uint16_t CTX_B = 0xFFFEu;    // context: at a token boundary
constexpr uint16_t CTX_BAD = 0xFFFFu;  // context: none (failure, or an impossible entry)

struct ChunkRes {          // one (chunk, candidate) scan
    uint64_t fail;         // failure offset, NOPOS64 = none
    uint32_t count;        // kept tokens starting in the chunk (before a failure)
    uint16_t exit;         // context at the next chunk start
    uint16_t pad;
};

struct ChunkOut {          // the resolved chunk
    uint64_t off;          // output index of its first token
    uint16_t entry;        // its true entry context
    uint16_t live;         // 1: emit its tokens
    uint32_t pad;
};

struct EnResult {
    unsigned long long total;   // kept tokens up to con(w)
    unsigned long long fail;    // con(w) when < n, else NOPOS64
    unsigned int error;
    unsigned int pad;
};

struct Summary {           // a run of chunks entered with one candidate
    unsigned long long count;
    uint32_t fail_chunk;   // chunk where the run fails (state 2)
    uint16_t exit;         // context after the run (state 1)
    uint8_t state;         // 0 broken, 1 ok, 2 fails
    uint8_t fail_k;        // candidate index at the failing chunk
};

struct EnParams {
    const uint8_t *in;
    uint64_t n;
    const uint8_t *blob;         // ScanTable blob
    uint32_t blob_bytes, S, q0, next_off, acc_off, cbeg_off, cand_off;
    uint32_t keep_all;           // full stream: every token is kept
    // the failed-lookahead guard: the liveness automaton's state at every
    // offset and its member bitsets (live == nullptr: unguarded, each scan
    // within a step budget)
    const uint8_t *live;
    const uint32_t *lmem;
    uint32_t lw;                 // member words per automaton state
    uint32_t budget;             // steps of an unguarded scan (~0u: no limit)
    uint32_t M;                  // chunk targets
    uint64_t *start;             // [M] chunk start offset, NOPOS64 = no chunk
    uint32_t *cinfo;             // [M] byte before the start << 8 | candidates
    ChunkRes *res;               // [M * KMAX]
    ChunkOut *out;               // [M]
    EnResult *rec;
    uint16_t *kinds;
    uint32_t *lens;
    uint64_t cap;
    // speculative scans
    uint16_t *ctx;               // [M] assumed entry context of each chunk
    uint32_t *prev;              // [M] previous chunk with a start
    uint8_t *dirty;              // [M] chunk to (re)scan from ctx
    unsigned int *changed;       // a fix-up round changed some ctx
    unsigned int *rescans;       // chunks scanned again after the first round
    unsigned int *rounds_used;   // fix-up rounds that changed some entry
    const uint16_t *guess;       // [M] predicted entry contexts (nullptr: BOUNDARY)
    uint16_t *st_kinds;          // [n] a chunk's kept tokens from its latest scan, at its start offset
    uint32_t *st_lens;           // [n]
    unsigned long long *blk_sum; // [ceil(M / SO_NT)] kept tokens of each block of chunks, to its first failure
    unsigned long long *blk_off; // [ceil(M / SO_NT)] output offset of each block (~0: after the failure)
    uint32_t *blk_fail;          // [ceil(M / SO_NT)] first failing chunk of each block (NONE32_EN: none)
    // resolve: runs of R1 consecutive chunks
    uint32_t nr1;                // number of runs
    Summary *sum1;               // [nr1 * KMAX] each run from each candidate of its first chunk
    uint32_t *first1;            // [nr1] first chunk with a start (NONE32_EN: none)
    uint32_t *entry1;            // [nr1] resolved candidate index (NONE32_EN: nothing emitted)
    unsigned long long *prefix1; // [nr1] output offset of the run
};

// Shared-memory view of the scan table.
struct ScanEnv {
    uint32_t cls_s, next_s;   // shared-window addresses of the class map and next table
    const uint8_t *cls;
    const uint16_t *next, *acc, *cbeg, *cand;
    uint32_t S, q0, keep_all;
    const uint8_t *in;
    uint64_t n;
    const uint8_t *live;
    const uint32_t *lmem;
    uint32_t lw, budget;
    unsigned int *error;
};

__device__ __forceinline__ ScanEnv stage_scan(const EnParams &P, uint8_t *smem)
{
    const uint4 *src = reinterpret_cast<const uint4 *>(P.blob);
    uint4 *dst = reinterpret_cast<uint4 *>(smem);
    for (uint32_t i = threadIdx.x; i < P.blob_bytes / 16; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    ScanEnv E;
    E.cls = smem;
    E.cls_s = (uint32_t)__cvta_generic_to_shared(smem);
    E.next_s = E.cls_s + P.next_off;
    E.next = reinterpret_cast<const uint16_t *>(smem + P.next_off);
    E.acc = reinterpret_cast<const uint16_t *>(smem + P.acc_off);
    E.cbeg = reinterpret_cast<const uint16_t *>(smem + P.cbeg_off);
    E.cand = reinterpret_cast<const uint16_t *>(smem + P.cand_off);
    E.S = P.S;
    E.q0 = P.q0;
    E.keep_all = P.keep_all;
    E.in = P.in;
    E.n = P.n;
    E.live = P.live;
    E.lmem = P.lmem;
    E.lw = P.lw;
    E.budget = P.budget;
    E.error = &P.rec->error;
    return E;
}

// Whether state q has an accepting position ahead of offset k (the guard).
__device__ __forceinline__ bool lv_has(const ScanEnv &E, uint32_t q, uint64_t k)
{
    const uint32_t r = __ldg(E.live + k);
    return (__ldg(E.lmem + r * E.lw + (q >> 5)) >> (q & 31)) & 1u;
}

// A lane's view of the input: a 16-byte block of its chunk held in
// registers, the next block loaded as soon as the lane enters one (its
// latency hidden behind sixteen steps).  Lanes of a warp read different
// chunks, so byte loads through L1 would bring a sector per lane and step;
// a block per lane cuts that sixteenfold.  Unaligned inputs and the last
// partial block are read byte by byte.
struct Bytes {
    const uint8_t *in;
    uint64_t n;
    bool wide;   // `in` 16-byte aligned
    uint64_t base = ~0ull, nbase = ~0ull;
    unsigned long long c0 = 0, c1 = 0, n0 = 0, n1 = 0;
    __device__ __forceinline__ void load(uint64_t b, unsigned long long &w0, unsigned long long &w1) const
    {
        if (wide && b + 16 <= n) {
            const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(in + b));
            w0 = v.x;
            w1 = v.y;
        } else {
            w0 = w1 = 0;
            for (uint32_t k = 0; k < 16 && b + k < n; k++) {
                const unsigned long long x = (unsigned long long)__ldg(in + b + k);
                if (k < 8) w0 |= x << (8 * k);
                else w1 |= x << (8 * (k - 8));
            }
        }
    }
    __device__ __forceinline__ uint32_t operator()(uint64_t p)
    {
        const uint64_t b = p & ~15ull;
        if (b != base) {
            if (b == nbase) {
                c0 = n0;
                c1 = n1;
            } else {
                load(b, c0, c1);
            }
            base = b;
            nbase = b + 16;
            if (nbase < n) load(nbase, n0, n1);
        }
        const unsigned long long w = (p & 8) ? c1 : c0;
        return (uint32_t)(w >> (8 * (uint32_t)(p & 7))) & 0xFFu;
    }
};

__device__ __forceinline__ uint32_t delta(const ScanEnv &E, uint32_t q, uint32_t b)
{
    uint32_t c, t;
    asm("ld.shared.u8 %0, [%1];" : "=r"(c) : "r"(E.cls_s + b));
    asm("ld.shared.u16 %0, [%1];" : "=r"(t) : "r"(E.next_s + 2u * (c * E.S + q)));
    return t;
}

struct CountTok {
    uint32_t count = 0;
    __device__ __forceinline__ void operator()(uint32_t, uint64_t) { count++; }
};

// The kept tokens of a chunk starting at p0 go to st[p0 + i]: tokens start
// at distinct offsets in [p0, p1), so a chunk's run of entries ends before
// the next chunk's begins.
struct StageTok {
    uint16_t *kinds;
    uint32_t *lens;
    uint64_t base;
    uint32_t count = 0;
    __device__ __forceinline__ void operator()(uint32_t kind, uint64_t len)
    {
        kinds[base + count] = (uint16_t)kind;
        lens[base + count] = (uint32_t)len;
        count++;
    }
};

struct WriteTok {
    uint16_t *kinds;
    uint32_t *lens;
    uint64_t cap, idx;
    __device__ __forceinline__ void operator()(uint32_t kind, uint64_t len)
    {
        if (idx < cap) {
            kinds[idx] = (uint16_t)kind;
            lens[idx] = (uint32_t)len;
        }
        idx++;
    }
};

// The chunk [p0, p1) entered in context `ctx`: emits the kept tokens that
// start in it (a token straddling p0 belongs to the previous chunk, one
// straddling p1 to this one) and returns the context at p1; on a failure
// returns CTX_BAD with `fail` set; for an entry from which no accepting
// position past p0 is reachable (never the true context) returns CTX_BAD
// with `fail` = NOPOS64.
//
// All 32 lanes of a warp call it together (`has` false: no chunk, result
// unused) and step in lockstep, up to four steps per lane between warp
// votes, so that their byte loads and table lookups issue together.  Each
// step is one DFA transition, or the end of a run: the run from `tok` in
// start state `qs` keeps its last accepting end, and when no transition is
// defined its token is [tok, last).  The entry run (from `ctx`) ends a token
// that began before p0 and is not emitted.  The state at p1 of the run that
// crosses it is kept: when the last token runs past p1, that state is the
// context at p1.
//
// Guarded (E.live set): a run also ends where its state has no accepting
// position ahead (it has passed its last one, so the token is the same), and
// an entry run that reaches p1 with one ahead stops there: its token runs
// past p1, so the context at p1 is its state.  Every token then costs its own
// length plus one step.  Unguarded, a lane that takes more than STEP_BUDGET
// steps gives up and flags EN_ERR_LOOKAHEAD; the caller runs again guarded.
template <bool GUARDED, class Emit>
__device__ __forceinline__ uint16_t chunk_scan_t(const ScanEnv &E, bool has, uint64_t p0, uint64_t p1, uint16_t ctx,
                                                 Emit &emit, uint64_t &fail)
{
    fail = NOPOS64;
    Bytes by{E.in, E.n, (reinterpret_cast<uintptr_t>(E.in) & 15u) == 0};
    const bool entered = ctx != CTX_B;
    uint16_t res = CTX_B;
    bool run = has && (entered || p0 < p1);
    uint64_t tok = p0, j = p0, last = NOPOS64;
    uint32_t qs = entered ? ctx : E.q0, q = qs, lq = 0, qp1 = qs, steps = 0;
    bool first = entered;
    while (__any_sync(0xffffffffu, run)) {
#pragma unroll
        for (int u = 0; u < 4; u++) {
            if (!run) break;
            uint32_t t = j < E.n ? delta(E, q, by(j)) : (uint32_t)SCAN_NONE;
            if (GUARDED) {
                if (!lv_has(E, q, j)) {
                    t = SCAN_NONE;   // no accepting position ahead: the run ends here
                } else if (first && j == p1) {
                    res = (uint16_t)q;   // the entered token runs past p1
                    run = false;
                    continue;
                }
            } else if (++steps > E.budget) {   // past the budget: give up, the caller reruns guarded
                atomicOr(E.error, EN_ERR_LOOKAHEAD);
                res = CTX_BAD;
                run = false;
                continue;
            }
            if (t != SCAN_NONE) {
                q = t & ~(uint32_t)SCAN_ACCEPT;
                j++;
                if (j == p1) qp1 = q;
                if (t & SCAN_ACCEPT) {
                    last = j;
                    lq = q;
                }
            } else if (last == NOPOS64) {   // no accepting end: a failure, or an impossible entry
                if (!first) fail = tok;
                res = CTX_BAD;
                run = false;
            } else {
                if (!first) {
                    const uint32_t acc = E.acc[lq];
                    if (E.keep_all || (acc & KIND_KEEP)) emit(acc & 0x7FFFu, last - tok);
                }
                if (last >= p1) {
                    if (last > p1) res = (uint16_t)qp1;
                    run = false;
                } else {
                    tok = j = last;
                    q = qs = E.q0;
                    last = NOPOS64;
                    first = false;
                }
            }
        }
    }
    if (!GUARDED && steps > E.budget) fail = NOPOS64;
    return res;
}

// The unguarded scan (with its step budget) or, once the liveness prepass
// has run, the guarded one; the choice is uniform over the launch.
template <class Emit>
__device__ __forceinline__ uint16_t chunk_scan(const ScanEnv &E, bool has, uint64_t p0, uint64_t p1, uint16_t ctx,
                                               Emit &emit, uint64_t &fail)
{
    if (E.live) return chunk_scan_t<true>(E, has, p0, p1, ctx, emit, fail);
    return chunk_scan_t<false>(E, has, p0, p1, ctx, emit, fail);
}

__device__ __forceinline__ uint32_t n_cand(const ScanEnv &E, uint32_t b)
{
    return 1u + E.cbeg[b + 1] - E.cbeg[b];
}

// Candidate k (0 = BOUNDARY) after byte b.
__device__ __forceinline__ uint16_t cand_ctx(const ScanEnv &E, uint32_t b, uint32_t k)
{
    return k == 0 ? CTX_B : E.cand[E.cbeg[b] + k - 1];
}

// Index of context x among the candidates after byte b, or -1.
__device__ __forceinline__ int cand_index(const ScanEnv &E, uint32_t b, uint16_t x)
{
    if (x == CTX_B) return 0;
    uint32_t lo = E.cbeg[b], hi = E.cbeg[b + 1];
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        const uint16_t v = E.cand[mid];
        if (v == x) return (int)(mid - E.cbeg[b]) + 1;
        if (v < x) lo = mid + 1;
        else hi = mid;
    }
    return -1;
}

// Next chunk start after target j, or n.
__device__ __forceinline__ uint64_t next_start(const EnParams &P, uint32_t j, uint32_t *jn)
{
    for (uint32_t k = j + 1; k < P.M; k++)
        if (P.start[k] != NOPOS64) {
            *jn = k;
            return P.start[k];
        }
    *jn = P.M;
    return P.n;
}

// (1) plan
__global__ void __launch_bounds__(EN_NT) en_plan(EnParams P)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const ScanEnv E = stage_scan(P, smem);
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < P.M; j += gridDim.x * blockDim.x) {
        if (j == 0) {
            P.start[0] = 0;
            P.cinfo[0] = 1;
            continue;
        }
        const uint64_t lo = (uint64_t)j * CHUNK;
        const uint64_t hi = min(lo + WIN, P.n);
        uint64_t best = NOPOS64;
        uint32_t bk = KMAX + 1, bb = 0;
        for (uint64_t p = lo; p < hi; p++) {
            const uint32_t b = __ldg(E.in + p - 1);
            const uint32_t k = n_cand(E, b);
            if (k < bk) {
                bk = k;
                bb = b;
                best = p;
                if (k == 1) break;
            }
        }
        P.start[j] = best;
        P.cinfo[j] = best == NOPOS64 ? 0u : (bb << 8 | bk);
    }
}

// (2) enumerate
__global__ void __launch_bounds__(EN_NT) en_enumerate(EnParams P)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const ScanEnv E = stage_scan(P, smem);
    // one lane per (candidate k, chunk j), candidate-major so that a warp
    // holds one candidate of 32 consecutive chunks and warps past every
    // chunk's candidate count skip; block-uniform loop
    const uint64_t total = (uint64_t)KMAX * P.M;
    for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x; i0 < total; i0 += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = i0 + threadIdx.x;
        const uint32_t k = (uint32_t)(i / P.M), j = (uint32_t)(i % P.M);
        const uint64_t p0 = i < total ? P.start[j] : NOPOS64;
        const bool has = p0 != NOPOS64 && k < (P.cinfo[j] & 0xFFu);
        if (!__any_sync(0xffffffffu, has)) continue;
        uint64_t p1 = 0;
        uint16_t c = CTX_B;
        if (has) {
            uint32_t jn;
            p1 = next_start(P, j, &jn);
            c = cand_ctx(E, P.cinfo[j] >> 8, k);
        }
        CountTok ct;
        uint64_t fail;
        const uint16_t x = chunk_scan(E, has, p0, p1, c, ct, fail);
        if (has) {
            ChunkRes r;
            r.fail = fail;
            r.count = ct.count;
            r.exit = x;
            r.pad = 0;
            P.res[(size_t)j * KMAX + k] = r;
        }
    }
}

// (3) resolve, three launches.  en_sum: one thread per run of R1 chunks
// follows the run from every candidate of its first chunk (count, exit
// context, or failure).  en_link (one CTA of RS_NT threads): each thread
// composes its group of runs from every candidate of the group's first chunk;
// thread 0 links the groups from BOUNDARY at offset 0 and finds the first
// failure (Corollary 1); each thread then gives each run of its group its
// true candidate and output offset.  en_label: one thread per run labels its
// chunks with their entry contexts and output offsets.

// Follow the chunks from candidate k of chunk j up to chunk j1 (exclusive);
// with `label`, give each its true entry context and output offset.
__device__ Summary follow_run(const EnParams &P, const ScanEnv &E, uint32_t j, uint32_t k, uint32_t j1, bool label,
                              unsigned long long base)
{
    Summary s{0, 0, CTX_BAD, 0, 0};
    unsigned long long cnt = 0;
    for (;;) {
        const ChunkRes r = P.res[(size_t)j * KMAX + k];
        if (label) {
            ChunkOut o;
            o.off = base + cnt;
            o.entry = cand_ctx(E, P.cinfo[j] >> 8, k);
            o.live = 1;
            o.pad = 0;
            P.out[j] = o;
        }
        if (r.fail != NOPOS64) {
            s.state = 2;
            s.count = cnt + r.count;
            s.fail_chunk = j;
            s.fail_k = (uint8_t)k;
            return s;
        }
        if (r.exit == CTX_BAD) return s;   // broken: not the true chain
        cnt += r.count;
        uint32_t jn;
        next_start(P, j, &jn);
        if (jn >= j1) {
            s.state = 1;
            s.count = cnt;
            s.exit = r.exit;
            return s;
        }
        const int ki = cand_index(E, P.cinfo[jn] >> 8, r.exit);
        if (ki < 0) return s;
        j = jn;
        k = (uint32_t)ki;
    }
}

__global__ void __launch_bounds__(EN_NT) en_sum(EnParams P)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const ScanEnv E = stage_scan(P, smem);
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= P.nr1) return;
    const uint32_t j0 = r * R1, j1 = min(P.M, j0 + R1);
    uint32_t f = NONE32_EN;
    for (uint32_t j = j0; j < j1; j++)
        if (P.start[j] != NOPOS64) {
            f = j;
            break;
        }
    P.first1[r] = f;
    if (f == NONE32_EN) return;
    const uint32_t K = P.cinfo[f] & 0xFFu;
    for (uint32_t k = 0; k < K; k++) P.sum1[(size_t)r * KMAX + k] = follow_run(P, E, f, k, j1, false, 0);
}

__global__ void __launch_bounds__(RS_NT) en_link(EnParams P)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const ScanEnv E = stage_scan(P, smem);
    Summary *sum = reinterpret_cast<Summary *>(smem + ((P.blob_bytes + 15u) & ~15u));
    uint32_t *first = reinterpret_cast<uint32_t *>(sum + RS_NT * KMAX);   // first run with a chunk
    uint32_t *entry = first + RS_NT;                                      // resolved candidate index
    unsigned long long *prefix = reinterpret_cast<unsigned long long *>(entry + RS_NT);
    const uint32_t t = threadIdx.x;
    const uint32_t per = (P.nr1 + RS_NT - 1) / RS_NT;
    const uint32_t g0 = min(P.nr1, t * per), g1 = min(P.nr1, g0 + per);

    // compose the runs [r, g1) entered with candidate k of run r's first chunk
    auto compose = [&](uint32_t r, uint32_t k) -> Summary {
        Summary a{0, 0, CTX_BAD, 0, 0};
        unsigned long long cnt = 0;
        uint16_t ctx = CTX_B;
        for (bool head = true; r < g1; r++) {
            if (P.first1[r] == NONE32_EN) continue;
            if (!head) {
                const int ki = cand_index(E, P.cinfo[P.first1[r]] >> 8, ctx);
                if (ki < 0) return a;
                k = (uint32_t)ki;
            }
            head = false;
            const Summary s = P.sum1[(size_t)r * KMAX + k];
            if (s.state == 2) {
                a = s;
                a.count += cnt;
                return a;
            }
            if (s.state != 1) return a;
            cnt += s.count;
            ctx = s.exit;
        }
        a.state = 1;
        a.count = cnt;
        a.exit = ctx;
        return a;
    };

    uint32_t f = NONE32_EN;
    for (uint32_t r = g0; r < g1; r++)
        if (P.first1[r] != NONE32_EN) {
            f = r;
            break;
        }
    first[t] = f;
    if (f != NONE32_EN) {
        const uint32_t K = P.cinfo[P.first1[f]] & 0xFFu;
        for (uint32_t k = 0; k < K; k++) sum[t * KMAX + k] = compose(f, k);
    }
    __syncthreads();

    if (t == 0) {   // link the groups from BOUNDARY at offset 0
        uint16_t ctx = CTX_B;
        unsigned long long run = 0;
        uint32_t r = 0;
        bool failed = false;
        for (; r < RS_NT; r++) {
            entry[r] = NONE32_EN;
            prefix[r] = run;
            if (first[r] == NONE32_EN) continue;
            const int k = cand_index(E, P.cinfo[P.first1[first[r]]] >> 8, ctx);
            if (k < 0) {
                P.rec->error |= EN_ERR_STATE;
                break;
            }
            const Summary s = sum[r * KMAX + k];
            entry[r] = (uint32_t)k;
            if (s.state == 2) {
                P.rec->fail = P.res[(size_t)s.fail_chunk * KMAX + s.fail_k].fail;
                P.rec->total = run + s.count;
                failed = true;
                r++;
                break;
            }
            if (s.state != 1) {
                P.rec->error |= EN_ERR_STATE;
                break;
            }
            run += s.count;
            ctx = s.exit;
        }
        for (; r < RS_NT; r++) entry[r] = NONE32_EN;   // after the failure: nothing is emitted
        if (!failed) {
            P.rec->total = run;
            P.rec->fail = NOPOS64;
        }
    }
    __syncthreads();

    // each run of the group: its true candidate and output offset
    uint32_t k = entry[t];
    unsigned long long pre = prefix[t];
    uint16_t ctx = CTX_B;
    bool live = k != NONE32_EN, head = true;
    for (uint32_t r = g0; r < g1; r++) {
        const uint32_t fc = P.first1[r];
        if (!live || fc == NONE32_EN) {
            P.entry1[r] = NONE32_EN;
            continue;
        }
        if (!head) {
            const int ki = cand_index(E, P.cinfo[fc] >> 8, ctx);
            if (ki < 0) {
                live = false;
                P.entry1[r] = NONE32_EN;
                continue;
            }
            k = (uint32_t)ki;
        }
        head = false;
        const Summary s = P.sum1[(size_t)r * KMAX + k];
        P.entry1[r] = k;
        P.prefix1[r] = pre;
        if (s.state != 1) {   // the failing run (or a break): nothing after it
            live = false;
            continue;
        }
        pre += s.count;
        ctx = s.exit;
    }
}

__global__ void __launch_bounds__(EN_NT) en_label(EnParams P)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const ScanEnv E = stage_scan(P, smem);
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= P.nr1) return;
    const uint32_t j0 = r * R1, j1 = min(P.M, j0 + R1);
    for (uint32_t j = j0; j < j1; j++) {
        ChunkOut o{0, CTX_BAD, 0, 0};
        P.out[j] = o;
    }
    const uint32_t k = P.entry1[r];
    if (k != NONE32_EN) follow_run(P, E, P.first1[r], k, j1, true, P.prefix1[r]);
}

// (4) emit
__global__ void __launch_bounds__(EN_NT) en_emit(EnParams P)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const ScanEnv E = stage_scan(P, smem);
    for (uint32_t j0 = blockIdx.x * blockDim.x; j0 < P.M; j0 += gridDim.x * blockDim.x) {
        const uint32_t j = j0 + threadIdx.x;
        ChunkOut o{0, CTX_B, 0, 0};
        if (j < P.M) o = P.out[j];
        uint64_t p0 = 0, p1 = 0;
        if (o.live) {
            uint32_t jn;
            p0 = P.start[j];
            p1 = next_start(P, j, &jn);
        }
        WriteTok wt{P.kinds, P.lens, P.cap, o.off};
        uint64_t fail;
        chunk_scan(E, o.live != 0, p0, p1, o.entry, wt, fail);
    }
}

// ---- speculative scans: one context per chunk, fixed up round by round ----
// A chunk's result is final once its entry equals the exit of its
// predecessor under the predecessor's (final) entry; chunk 0 enters at
// BOUNDARY.  Each round scans the chunks whose assumed entry changed, then
// every chunk takes its predecessor's exit as its entry.  At the fixed point
// the chain from offset 0 is consistent, so every entry is the true context.
__global__ void __launch_bounds__(EN_NT) sp_init(EnParams P)
{
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < P.M; j += gridDim.x * blockDim.x) {
        const bool has = P.start[j] != NOPOS64;
        uint16_t c = CTX_B;
        if (j > 0 && has && P.guess) c = P.guess[j];
        P.ctx[j] = c;
        P.dirty[j] = has ? 1 : 0;
        uint32_t q = NONE32_EN;
        for (uint32_t k = j; k-- > 0;)
            if (P.start[k] != NOPOS64) {
                q = k;
                break;
            }
        P.prev[j] = q;
    }
}

__global__ void __launch_bounds__(EN_NT) sp_scan(EnParams P, uint32_t round)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const ScanEnv E = stage_scan(P, smem);
    for (uint32_t j0 = blockIdx.x * blockDim.x; j0 < P.M; j0 += gridDim.x * blockDim.x) {
        const uint32_t j = j0 + threadIdx.x;
        const bool has = j < P.M && P.dirty[j];
        // a warp with no dirty chunk skips the scan as a whole
        if (!__any_sync(0xffffffffu, has)) continue;
        uint64_t p0 = 0, p1 = 0;
        uint16_t c = CTX_B;
        if (has) {
            uint32_t jn;
            p0 = P.start[j];
            p1 = next_start(P, j, &jn);
            c = P.ctx[j];
        }
        StageTok ct{P.st_kinds, P.st_lens, p0};
        uint64_t fail;
        const uint16_t x = chunk_scan(E, has, p0, p1, c, ct, fail);
        if (has) {
            ChunkRes r;
            r.fail = fail;
            r.count = ct.count;
            r.exit = x;
            r.pad = 0;
            P.res[(size_t)j * KMAX] = r;
            P.dirty[j] = 0;
            if (round > 0) atomicAdd(P.rescans, 1u);
        }
    }
}

__global__ void __launch_bounds__(EN_NT) sp_fix(EnParams P)
{
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < P.M; j += gridDim.x * blockDim.x) {
        const uint32_t q = P.prev[j];
        if (P.start[j] == NOPOS64 || q == NONE32_EN) continue;
        const ChunkRes r = P.res[(size_t)q * KMAX];
        if (r.fail != NOPOS64 || r.exit == CTX_BAD) continue;   // failed, or not settled yet
        if (r.exit != P.ctx[j]) {
            P.ctx[j] = r.exit;
            P.dirty[j] = 1;
            *P.changed = 1;
        }
    }
}

// Counts the rounds whose fix-up changed some entry (one thread).
__global__ void sp_count(EnParams P)
{
    if (*P.changed) atomicAdd(P.rounds_used, 1u);
}

// The judge: after a full enumeration (en_enumerate .. en_label) every live
// chunk takes its true entry context.  A chunk whose latest speculative scan
// already ran from it keeps that scan (its staged tokens are valid; its
// result, which the enumeration overwrote in slot 0, is copied back from the
// slot of that candidate); every other live chunk is marked for one more scan.
__global__ void __launch_bounds__(EN_NT) jd_apply(EnParams P)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const ScanEnv E = stage_scan(P, smem);
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < P.M; j += gridDim.x * blockDim.x) {
        if (P.start[j] == NOPOS64) continue;
        const ChunkOut o = P.out[j];
        if (!o.live) {
            P.dirty[j] = 0;
            continue;
        }
        if (P.dirty[j] || P.ctx[j] != o.entry) {
            P.ctx[j] = o.entry;
            P.dirty[j] = 1;
        } else {
            const int ki = cand_index(E, P.cinfo[j] >> 8, o.entry);
            if (ki > 0) P.res[(size_t)j * KMAX] = P.res[(size_t)j * KMAX + ki];
        }
    }
}

// Chunk starts and their true entry contexts (after en_label), per target.
__global__ void __launch_bounds__(EN_NT) ctx_export(EnParams P, uint64_t *starts, uint16_t *ctx)
{
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < P.M; j += gridDim.x * blockDim.x) {
        const ChunkOut o = P.out[j];
        starts[j] = o.live ? P.start[j] : NOPOS64;
        ctx[j] = o.live ? o.entry : CTX_BAD;
    }
}

// The settled chunks' staged tokens to their output offsets, one warp per
// chunk, coalesced: the last scan of every chunk ran from its true entry
// context, so no chunk is walked again to emit.
__global__ void __launch_bounds__(EN_NT) sp_copy(EnParams P)
{
    const uint32_t lane = threadIdx.x & 31u, nw = gridDim.x * (blockDim.x / 32u);
    for (uint32_t j = (blockIdx.x * blockDim.x + threadIdx.x) / 32u; j < P.M; j += nw) {
        const ChunkOut o = P.out[j];
        if (!o.live) continue;
        const uint64_t base = P.start[j];
        const uint32_t cnt = P.res[(size_t)j * KMAX].count;
        for (uint32_t i = lane; i < cnt; i += 32u) {
            const uint64_t idx = o.off + i;
            if (idx < P.cap) {
                P.kinds[idx] = P.st_kinds[base + i];
                P.lens[idx] = P.st_lens[base + i];
            }
        }
    }
}

// Output offsets along the settled chain: the kept-token counts of the chunks
// in order, up to and including the first failing chunk (Corollary 1: the
// chunks after it emit nothing).  Three launches, one chunk per thread: the
// blocks' sums (so_block), the blocks' offsets (so_top, one CTA), each
// chunk's offset (so_out).

// Inclusive block-wide scan of v over SO_NT threads; `total` = the block's sum.
__device__ __forceinline__ unsigned long long so_scan(unsigned long long v, unsigned long long *sh,
                                                      unsigned long long &total)
{
    const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= (uint32_t)o) v += y;
    }
    if (lane == 31) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        unsigned long long x = sh[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= (uint32_t)o) x += y;
        }
        sh[lane] = x;
    }
    __syncthreads();
    if (w > 0) v += sh[w - 1];
    total = sh[31];
    __syncthreads();
    return v;
}

// A chunk's kept-token count and whether it fails (0, false for no chunk).
__device__ __forceinline__ unsigned long long so_count(const EnParams &P, uint32_t j, bool &fails)
{
    fails = false;
    if (j >= P.M || P.start[j] == NOPOS64) return 0;
    const ChunkRes r = P.res[(size_t)j * KMAX];
    fails = r.fail != NOPOS64;
    return r.count;
}

__global__ void __launch_bounds__(SO_NT) so_block(EnParams P)
{
    __shared__ unsigned long long sh[32];
    __shared__ uint32_t s_first;
    __shared__ unsigned long long s_at;
    const uint32_t t = threadIdx.x, j = blockIdx.x * SO_NT + t;
    if (t == 0) s_first = NONE32_EN;
    __syncthreads();
    bool fails;
    const unsigned long long v = so_count(P, j, fails);
    if (fails) atomicMin(&s_first, t);
    unsigned long long total;
    const unsigned long long incl = so_scan(v, sh, total);
    const uint32_t f = s_first;
    if (t == f) s_at = incl;
    __syncthreads();
    if (t == 0) {
        P.blk_sum[blockIdx.x] = f == NONE32_EN ? total : s_at;
        P.blk_fail[blockIdx.x] = f == NONE32_EN ? NONE32_EN : blockIdx.x * SO_NT + f;
    }
}

__global__ void __launch_bounds__(SO_NT) so_top(EnParams P, uint32_t nb)
{
    __shared__ unsigned long long sh[32];
    __shared__ uint32_t s_first;
    __shared__ unsigned long long s_at;
    const uint32_t t = threadIdx.x;
    unsigned long long carry = 0;
    bool dead = false;
    uint32_t fail_chunk = NONE32_EN;
    for (uint32_t b0 = 0; b0 < nb; b0 += SO_NT) {
        const uint32_t i = b0 + t;
        if (t == 0) s_first = NONE32_EN;
        __syncthreads();
        const unsigned long long v = i < nb ? P.blk_sum[i] : 0ull;
        if (i < nb && P.blk_fail[i] != NONE32_EN) atomicMin(&s_first, t);
        unsigned long long total;
        const unsigned long long incl = so_scan(v, sh, total);
        const uint32_t f = s_first;
        if (i < nb) P.blk_off[i] = (dead || t > f) ? ~0ull : carry + incl - v;
        if (t == f) s_at = incl;
        __syncthreads();
        if (!dead) {
            if (f != NONE32_EN) {
                carry += s_at;
                fail_chunk = P.blk_fail[b0 + f];
                dead = true;
            } else {
                carry += total;
            }
        }
        __syncthreads();
    }
    if (t == 0) {
        P.rec->total = carry;
        P.rec->fail = fail_chunk == NONE32_EN ? NOPOS64 : P.res[(size_t)fail_chunk * KMAX].fail;
    }
}

__global__ void __launch_bounds__(SO_NT) so_out(EnParams P)
{
    __shared__ unsigned long long sh[32];
    __shared__ uint32_t s_first;
    const uint32_t t = threadIdx.x, j = blockIdx.x * SO_NT + t;
    if (t == 0) s_first = NONE32_EN;
    __syncthreads();
    bool fails;
    const unsigned long long v = so_count(P, j, fails);
    if (fails) atomicMin(&s_first, t);
    unsigned long long total;
    const unsigned long long incl = so_scan(v, sh, total);
    const unsigned long long boff = P.blk_off[blockIdx.x];
    if (j < P.M) {
        ChunkOut o{0, CTX_BAD, 0, 0};
        if (P.start[j] != NOPOS64 && boff != ~0ull && t <= s_first) {
            o.off = boff + incl - v;
            o.entry = P.ctx[j];
            o.live = 1;
        }
        P.out[j] = o;
    }
}

}  // namespace
}  // namespace lx

using namespace lx;

namespace {

// Everything a run over one input needs: parameters, launch shapes, stream.
struct EnRun {
    EnParams P;
    uint32_t grid = 0, egrid = 0, smem = 0, rs_smem = 0;
    cudaStream_t s = nullptr;
    uint16_t *guess_buf = nullptr;   // [M] scratch for predicted contexts
};

// Validate, upload tables, size the scratch and fill the parameters.
int en_setup(lx_ctx *c, const lx_tokenset *ts, const uint8_t *d_in, uint64_t n, int mode, uint16_t *d_kinds,
             uint32_t *d_lens, uint64_t capacity, void *stream, EnRun &R, bool stage = false)
{
    if (!c || !ts) return LX_E_INVAL;
    if (mode < LX_FULL_EXACT || mode > LX_FILTERED_MODULO) return LX_E_MODE;
    if (n && !d_in) return LX_E_INVAL;
    if (capacity && (!d_kinds || !d_lens)) return LX_E_INVAL;
    const ScanTable &st = ts->scan;
    if (st.status != LX_OK) return st.status;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != c->device) return LX_E_INVAL;
    DeviceTables dt;
    int rc = ensure_device_tables(ts, dev, &dt);
    if (rc != LX_OK) return rc;
    void *scan = dt.d_scan;
    const uint64_t M64 = (n + CHUNK - 1) / CHUNK;
    if (M64 > 0xFFFFFFF0ull) return LX_E_INVAL;
    const uint32_t M = (uint32_t)M64;

    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_rec = 0, o_flags = 128, o_start = 256, o_cinfo = al(o_start + 8 * (size_t)M);
    const size_t o_res = al(o_cinfo + 4 * (size_t)M), o_out = al(o_res + sizeof(ChunkRes) * KMAX * (size_t)M);
    const size_t o_ctx = al(o_out + sizeof(ChunkOut) * (size_t)M), o_prev = al(o_ctx + 2 * (size_t)M);
    const size_t o_dirty = al(o_prev + 4 * (size_t)M), o_guess = al(o_dirty + (size_t)M);
    const size_t o_stk = al(o_guess + 2 * (size_t)M), o_stl = al(o_stk + (stage ? 2 * (size_t)n : 0));
    const size_t nb = (M + SO_NT - 1) / SO_NT;
    const size_t o_bsum = al(o_stl + (stage ? 4 * (size_t)n : 0)), o_boff = al(o_bsum + 8 * nb);
    const size_t o_bfail = al(o_boff + 8 * nb);
    const size_t nr1 = (M + R1 - 1) / R1;
    const size_t o_sum1 = al(o_bfail + 4 * nb), o_first1 = al(o_sum1 + sizeof(Summary) * KMAX * nr1);
    const size_t o_entry1 = al(o_first1 + 4 * nr1), o_prefix1 = al(o_entry1 + 4 * nr1);
    const size_t total = al(o_prefix1 + 8 * nr1);
    rc = grow(&c->e_dev, &c->e_dev_bytes, total);
    if (rc != LX_OK) return rc;
    uint8_t *d = static_cast<uint8_t *>(c->e_dev);

    EnParams &P = R.P;
    P.in = d_in;
    P.n = n;
    P.blob = static_cast<const uint8_t *>(scan);
    P.blob_bytes = (uint32_t)st.blob.size();
    P.S = st.S;
    P.q0 = st.q0;
    P.next_off = st.next_off;
    P.acc_off = st.acc_off;
    P.cbeg_off = st.cbeg_off;
    P.cand_off = st.cand_off;
    P.keep_all = mode == LX_FULL_EXACT ? 1u : 0u;
    P.M = M;
    P.rec = reinterpret_cast<EnResult *>(d + o_rec);
    P.start = reinterpret_cast<uint64_t *>(d + o_start);
    P.cinfo = reinterpret_cast<uint32_t *>(d + o_cinfo);
    P.res = reinterpret_cast<ChunkRes *>(d + o_res);
    P.out = reinterpret_cast<ChunkOut *>(d + o_out);
    P.kinds = d_kinds;
    P.lens = d_lens;
    P.cap = capacity;
    P.ctx = reinterpret_cast<uint16_t *>(d + o_ctx);
    P.prev = reinterpret_cast<uint32_t *>(d + o_prev);
    P.dirty = d + o_dirty;
    P.changed = reinterpret_cast<unsigned int *>(d + o_flags);
    P.rescans = reinterpret_cast<unsigned int *>(d + o_flags + 4);
    P.rounds_used = reinterpret_cast<unsigned int *>(d + o_flags + 8);
    P.guess = nullptr;
    P.live = nullptr;
    P.lmem = nullptr;
    P.lw = 0;
    P.budget = STEP_BUDGET;
    P.st_kinds = stage ? reinterpret_cast<uint16_t *>(d + o_stk) : nullptr;
    P.st_lens = stage ? reinterpret_cast<uint32_t *>(d + o_stl) : nullptr;
    P.blk_sum = reinterpret_cast<unsigned long long *>(d + o_bsum);
    P.blk_off = reinterpret_cast<unsigned long long *>(d + o_boff);
    P.blk_fail = reinterpret_cast<uint32_t *>(d + o_bfail);
    P.nr1 = (uint32_t)nr1;
    P.sum1 = reinterpret_cast<Summary *>(d + o_sum1);
    P.first1 = reinterpret_cast<uint32_t *>(d + o_first1);
    P.entry1 = reinterpret_cast<uint32_t *>(d + o_entry1);
    P.prefix1 = reinterpret_cast<unsigned long long *>(d + o_prefix1);
    R.guess_buf = reinterpret_cast<uint16_t *>(d + o_guess);

    R.smem = P.blob_bytes;
    R.rs_smem = ((R.smem + 15u) & ~15u) + sizeof(Summary) * RS_NT * KMAX + 8u * RS_NT + 8u * RS_NT;
    static bool attr_done[64] = {false};
    if (dev < 64 && !attr_done[dev]) {
        const size_t lim = 64 * 1024;
        if (cudaFuncSetAttribute(en_plan, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess ||
            cudaFuncSetAttribute(en_enumerate, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess ||
            cudaFuncSetAttribute(en_emit, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess ||
            cudaFuncSetAttribute(jd_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess ||
            cudaFuncSetAttribute(sp_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess ||
            cudaFuncSetAttribute(en_sum, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess ||
            cudaFuncSetAttribute(en_label, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess ||
            cudaFuncSetAttribute(en_link, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024) != cudaSuccess)
            return LX_E_CUDA;
        attr_done[dev] = true;
    }
    if (R.rs_smem > 220u * 1024u) return LX_E_TOOBIG;
    R.grid = (uint32_t)std::min<uint64_t>((M + EN_NT - 1) / EN_NT, 4ull * c->num_sms);
    R.egrid = (uint32_t)std::min<uint64_t>(((uint64_t)KMAX * M + EN_NT - 1) / EN_NT, 8ull * c->num_sms);
    R.s = static_cast<cudaStream_t>(stream);
    return cuda_err(cudaMemsetAsync(d, 0, 256, R.s));
}

// Read back the record: status, token count and con(w).
// rescans (optional): chunks scanned again after the first round, then the
// fix-up rounds that changed some entry (two words).
int en_finish(lx_ctx *c, const EnRun &R, uint64_t capacity, uint64_t *n_tokens, uint64_t *consumed,
              unsigned int *rescans = nullptr)
{
    int rc = cuda_err(cudaGetLastError());
    if (rc != LX_OK) return rc;
    uint8_t buf[256];
    rc = cuda_err(cudaMemcpyAsync(c->h_res, R.P.rec, sizeof(EnResult), cudaMemcpyDeviceToHost, R.s));
    if (rc == LX_OK && rescans) rc = cuda_err(cudaMemcpyAsync(rescans, R.P.rescans, 8, cudaMemcpyDeviceToHost, R.s));
    if (rc == LX_OK) rc = cuda_err(cudaStreamSynchronize(R.s));
    if (rc != LX_OK) return rc;
    std::memcpy(buf, c->h_res, sizeof(EnResult));
    EnResult r;
    std::memcpy(&r, buf, sizeof r);
    if (r.error & EN_ERR_LOOKAHEAD) return LX_LOOKAHEAD;
    if (r.error) return LX_E_CUDA;
    *n_tokens = r.total;
    *consumed = r.fail == NOPOS64 ? R.P.n : r.fail;
    return r.total > capacity ? LX_E_CAPACITY : LX_OK;
}

// After a scan flagged EN_ERR_LOOKAHEAD: the guard's prepass over the input,
// and the record cleared for the next run.  Without a liveness automaton the
// next run goes unguarded with no step budget (exact, possibly quadratic).
int en_guard(lx_ctx *c, const lx_tokenset *ts, EnRun &R)
{
    const uint8_t *live = nullptr;
    const uint32_t *member = nullptr;
    const int rc = liveness_device(c, ts, R.P.in, R.P.n, nullptr, R.s, &live, &member);
    if (rc == LX_OK) {
        R.P.live = live;
        R.P.lmem = member;
        R.P.lw = ts->liveness.W;
    } else if (rc == LX_E_TOOBIG) {
        R.P.budget = ~0u;
    } else {
        return rc;
    }
    return cuda_err(cudaMemsetAsync(R.P.rec, 0, 256, R.s));
}

// The enumerative pipeline (plan .. emit) on a prepared run.
void en_pipeline(const EnRun &R)
{
    en_plan<<<R.grid, EN_NT, R.smem, R.s>>>(R.P);
    en_enumerate<<<R.egrid, EN_NT, R.smem, R.s>>>(R.P);
    en_sum<<<(R.P.nr1 + EN_NT - 1) / EN_NT, EN_NT, R.smem, R.s>>>(R.P);
    en_link<<<1, RS_NT, R.rs_smem, R.s>>>(R.P);
    en_label<<<(R.P.nr1 + EN_NT - 1) / EN_NT, EN_NT, R.smem, R.s>>>(R.P);
    en_emit<<<R.grid, EN_NT, R.smem, R.s>>>(R.P);
}

// The speculative pipeline (plan .. copy) on a prepared run; the record's
// status as en_finish reads it.
int spec_pipeline(lx_ctx *c, EnRun &R, lx_model *model, uint64_t capacity, uint64_t *n_tokens, uint64_t *consumed,
                  lx_spec_stats *stats)
{
    int rc = LX_OK;
    en_plan<<<R.grid, EN_NT, R.smem, R.s>>>(R.P);
    if (model) {
        rc = model_predict(model, R.P.in, R.P.n, R.P.start, R.P.cinfo, R.P.blob, R.P.cbeg_off, R.P.cand_off,
                           R.P.M, R.guess_buf, R.s);
        if (rc != LX_OK) return rc;
        R.P.guess = R.guess_buf;
    }
    sp_init<<<R.grid, EN_NT, 0, R.s>>>(R.P);
    // SPEC_ROUNDS rounds back to back on the device (a round with nothing
    // to rescan costs two short launches), one read-back; what is still
    // unsettled then goes to the judge
    for (uint32_t r = 0; r < SPEC_ROUNDS; r++) {
        sp_scan<<<R.grid, EN_NT, R.smem, R.s>>>(R.P, r);
        rc = cuda_err(cudaMemsetAsync(R.P.changed, 0, 4, R.s));
        if (rc != LX_OK) return rc;
        sp_fix<<<R.grid, EN_NT, 0, R.s>>>(R.P);
        sp_count<<<1, 1, 0, R.s>>>(R.P);
    }
    unsigned int *h_flag = static_cast<unsigned int *>(c->h_res);
    rc = cuda_err(cudaMemcpyAsync(h_flag, R.P.changed, 4, cudaMemcpyDeviceToHost, R.s));
    if (rc == LX_OK) rc = cuda_err(cudaStreamSynchronize(R.s));
    if (rc != LX_OK) return rc;
    const bool judged = *h_flag != 0;
    if (judged) {
        // the enumerative scan of every chunk from every candidate context
        // settles all chains at once; one more round rescans the chunks whose
        // true entry differs from their latest scan
        en_enumerate<<<R.egrid, EN_NT, R.smem, R.s>>>(R.P);
        en_sum<<<(R.P.nr1 + EN_NT - 1) / EN_NT, EN_NT, R.smem, R.s>>>(R.P);
        en_link<<<1, RS_NT, R.rs_smem, R.s>>>(R.P);
        en_label<<<(R.P.nr1 + EN_NT - 1) / EN_NT, EN_NT, R.smem, R.s>>>(R.P);
        jd_apply<<<R.grid, EN_NT, R.smem, R.s>>>(R.P);
        sp_scan<<<R.grid, EN_NT, R.smem, R.s>>>(R.P, SPEC_ROUNDS);
    }
    const uint32_t nb = (R.P.M + SO_NT - 1) / SO_NT;
    so_block<<<nb, SO_NT, 0, R.s>>>(R.P);
    so_top<<<1, SO_NT, 0, R.s>>>(R.P, nb);
    so_out<<<nb, SO_NT, 0, R.s>>>(R.P);
    sp_copy<<<R.grid * (EN_NT / 32), EN_NT, 0, R.s>>>(R.P);
    if (c->timing) cudaEventRecord(c->ev[1], R.s);
    unsigned int rr[2] = {0, 0};
    rc = en_finish(c, R, capacity, n_tokens, consumed, rr);
    if (stats) {
        stats->chunks = R.P.M;
        stats->rounds = 1 + rr[1];
        stats->rescanned = rr[0];
        stats->judged = judged ? 1u : 0u;
    }
    return rc;
}

}  // namespace

int lx::lex_enumerative_device(lx_ctx *c, const lx_tokenset *ts, const uint8_t *d_in, uint64_t n, int mode,
                               uint16_t *d_kinds, uint32_t *d_lens, uint64_t capacity, uint64_t *n_tokens,
                               uint64_t *consumed, cudaStream_t stream, bool guard)
{
    if (!n_tokens || !consumed) return LX_E_INVAL;
    *n_tokens = 0;
    *consumed = 0;
    EnRun R;
    int rc = en_setup(c, ts, d_in, n, mode, d_kinds, d_lens, capacity, stream, R);
    if (rc != LX_OK || n == 0) return rc;
    if (c->timing) cudaEventRecord(c->ev[0], R.s);
    if (guard && (rc = en_guard(c, ts, R)) != LX_OK) return rc;
    for (;;) {
        en_pipeline(R);
        if (c->timing) cudaEventRecord(c->ev[1], R.s);
        rc = en_finish(c, R, capacity, n_tokens, consumed);
        if (rc != LX_LOOKAHEAD) return rc;
        if (R.P.live || R.P.budget == ~0u) return LX_E_CUDA;   // a guarded run never flags it
        if ((rc = en_guard(c, ts, R)) != LX_OK) return rc;
    }
}

extern "C" int lx_lex_enumerative(lx_ctx *c, const lx_tokenset *ts, const uint8_t *d_in, uint64_t n, int mode,
                                  uint16_t *d_kinds, uint32_t *d_lens, uint64_t capacity, uint64_t *n_tokens,
                                  uint64_t *consumed, void *stream)
{
    return lex_enumerative_device(c, ts, d_in, n, mode, d_kinds, d_lens, capacity, n_tokens, consumed,
                                  static_cast<cudaStream_t>(stream), false);
}

extern "C" int lx_chunk_contexts(lx_ctx *c, const lx_tokenset *ts, const uint8_t *d_in, uint64_t n,
                                 uint64_t *d_starts, uint16_t *d_ctx, uint64_t cap, uint64_t *count, void *stream)
{
    if (!count || (cap && (!d_starts || !d_ctx))) return LX_E_INVAL;
    *count = 0;
    EnRun R;
    int rc = en_setup(c, ts, d_in, n, LX_FULL_EXACT, nullptr, nullptr, 0, stream, R);
    if (rc != LX_OK || n == 0) return rc;
    *count = R.P.M;
    if (cap < R.P.M) return LX_E_CAPACITY;
    for (;;) {
        en_plan<<<R.grid, EN_NT, R.smem, R.s>>>(R.P);
        en_enumerate<<<R.egrid, EN_NT, R.smem, R.s>>>(R.P);
        en_sum<<<(R.P.nr1 + EN_NT - 1) / EN_NT, EN_NT, R.smem, R.s>>>(R.P);
        en_link<<<1, RS_NT, R.rs_smem, R.s>>>(R.P);
        en_label<<<(R.P.nr1 + EN_NT - 1) / EN_NT, EN_NT, R.smem, R.s>>>(R.P);
        ctx_export<<<R.grid, EN_NT, 0, R.s>>>(R.P, d_starts, d_ctx);
        uint64_t nt, con;
        rc = en_finish(c, R, ~0ull, &nt, &con);
        if (rc != LX_LOOKAHEAD) return rc;
        if (R.P.live || R.P.budget == ~0u) return LX_E_CUDA;
        if ((rc = en_guard(c, ts, R)) != LX_OK) return rc;
    }
}

extern "C" int lx_lex_speculative(lx_ctx *c, const lx_tokenset *ts, lx_model *model, const uint8_t *d_in,
                                  uint64_t n, int mode, uint16_t *d_kinds, uint32_t *d_lens, uint64_t capacity,
                                  uint64_t *n_tokens, uint64_t *consumed, lx_spec_stats *stats, void *stream)
{
    if (!n_tokens || !consumed) return LX_E_INVAL;
    *n_tokens = 0;
    *consumed = 0;
    if (stats) *stats = lx_spec_stats{0, 0, 0, 0};
    EnRun R;
    int rc = en_setup(c, ts, d_in, n, mode, d_kinds, d_lens, capacity, stream, R, true);
    if (rc != LX_OK || n == 0) return rc;
    if (model && model_contexts(model) != ts->scan.S + 1) return LX_E_INVAL;
    if (c->timing) cudaEventRecord(c->ev[0], R.s);
    for (;;) {
        rc = spec_pipeline(c, R, model, capacity, n_tokens, consumed, stats);
        if (rc != LX_LOOKAHEAD) return rc;
        if (R.P.live || R.P.budget == ~0u) return LX_E_CUDA;   // a guarded run never flags it
        if ((rc = en_guard(c, ts, R)) != LX_OK) return rc;
    }
}
