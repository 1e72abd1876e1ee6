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
//   (3) resolve:   one CTA follows the chain of exits from BOUNDARY at offset
//                  0 (1024 threads compose their runs of chunks, one thread
//                  links the runs, then each thread labels its run): every
//                  chunk's true entry context and output offset, and the first
//                  failure (Corollary 1);
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

struct EnParams {
    const uint8_t *in;
    uint64_t n;
    const uint8_t *blob;         // ScanTable blob
    uint32_t blob_bytes, S, q0, next_off, acc_off, cbeg_off, cand_off;
    uint32_t keep_all;           // full stream: every token is kept
    uint32_t M;                  // chunk targets
    uint64_t *start;             // [M] chunk start offset, NOPOS64 = no chunk
    uint32_t *cinfo;             // [M] byte before the start << 8 | candidates
    ChunkRes *res;               // [M * KMAX]
    ChunkOut *out;               // [M]
    EnResult *rec;
    uint16_t *kinds;
    uint32_t *lens;
    uint64_t cap;
};

// Shared-memory view of the scan table.
struct ScanEnv {
    const uint8_t *cls;
    const uint16_t *next, *acc, *cbeg, *cand;
    uint32_t S, q0, keep_all;
    const uint8_t *in;
    uint64_t n;
};

__device__ __forceinline__ ScanEnv stage_scan(const EnParams &P, uint8_t *smem)
{
    const uint4 *src = reinterpret_cast<const uint4 *>(P.blob);
    uint4 *dst = reinterpret_cast<uint4 *>(smem);
    for (uint32_t i = threadIdx.x; i < P.blob_bytes / 16; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    ScanEnv E;
    E.cls = smem;
    E.next = reinterpret_cast<const uint16_t *>(smem + P.next_off);
    E.acc = reinterpret_cast<const uint16_t *>(smem + P.acc_off);
    E.cbeg = reinterpret_cast<const uint16_t *>(smem + P.cbeg_off);
    E.cand = reinterpret_cast<const uint16_t *>(smem + P.cand_off);
    E.S = P.S;
    E.q0 = P.q0;
    E.keep_all = P.keep_all;
    E.in = P.in;
    E.n = P.n;
    return E;
}

__device__ __forceinline__ uint32_t byte_at(const ScanEnv &E, uint64_t p) { return __ldg(E.in + p); }

__device__ __forceinline__ uint32_t delta(const ScanEnv &E, uint32_t q, uint32_t b)
{
    return E.next[(uint32_t)E.cls[b] * E.S + q];
}

// The DFA run from state q before byte j while transitions are defined: the
// last accepting end (> j) and its accept word, or NOPOS64.
__device__ __forceinline__ uint64_t run_last_accept(const ScanEnv &E, uint32_t q, uint64_t j, uint32_t &acc)
{
    uint64_t last = NOPOS64;
    while (j < E.n) {
        const uint32_t t = delta(E, q, byte_at(E, j));
        if (t == SCAN_NONE) break;
        q = t;
        j++;
        const uint32_t a = E.acc[q];
        if ((a & 0x7FFFu) != KIND_NONE) {
            last = j;
            acc = a;
        }
    }
    return last;
}

__device__ __forceinline__ uint32_t state_after(const ScanEnv &E, uint32_t q, uint64_t lo, uint64_t hi)
{
    for (uint64_t j = lo; j < hi; j++) q = delta(E, q, byte_at(E, j));
    return q;
}

struct CountTok {
    uint32_t count = 0;
    __device__ __forceinline__ void operator()(uint32_t, uint64_t) { count++; }
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
template <class Emit>
__device__ uint16_t chunk_scan(const ScanEnv &E, uint64_t p0, uint64_t p1, uint16_t ctx, Emit &emit,
                               uint64_t &fail)
{
    fail = NOPOS64;
    uint64_t pos = p0;
    uint32_t acc = 0;
    if (ctx != CTX_B) {
        const uint64_t e = run_last_accept(E, ctx, p0, acc);
        if (e == NOPOS64) return CTX_BAD;
        if (e >= p1) return e == p1 ? CTX_B : (uint16_t)state_after(E, ctx, p0, p1);
        pos = e;
    }
    while (pos < p1) {
        const uint64_t e = run_last_accept(E, E.q0, pos, acc);
        if (e == NOPOS64) {
            fail = pos;
            return CTX_BAD;
        }
        if (E.keep_all || (acc & KIND_KEEP)) emit(acc & 0x7FFFu, e - pos);
        if (e >= p1) return e == p1 ? CTX_B : (uint16_t)state_after(E, E.q0, pos, p1);
        pos = e;
    }
    return CTX_B;
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
            const uint32_t b = byte_at(E, p - 1);
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
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < P.M; j += gridDim.x * blockDim.x) {
        const uint64_t p0 = P.start[j];
        if (p0 == NOPOS64) continue;
        uint32_t jn;
        const uint64_t p1 = next_start(P, j, &jn);
        const uint32_t b = P.cinfo[j] >> 8, K = P.cinfo[j] & 0xFFu;
        for (uint32_t k = 0; k < K; k++) {
            CountTok ct;
            uint64_t fail;
            const uint16_t x = chunk_scan(E, p0, p1, cand_ctx(E, b, k), ct, fail);
            ChunkRes r;
            r.fail = fail;
            r.count = ct.count;
            r.exit = x;
            r.pad = 0;
            P.res[(size_t)j * KMAX + k] = r;
        }
    }
}

// (3) resolve: one CTA of RS_NT threads
struct Summary {           // a thread's run of chunks entered with one candidate
    unsigned long long count;
    uint32_t fail_chunk;   // chunk where the run fails (state 2)
    uint16_t exit;         // context after the run (state 1)
    uint8_t state;         // 0 broken, 1 ok, 2 fails
    uint8_t fail_k;        // candidate index at the failing chunk
};

__global__ void __launch_bounds__(RS_NT) en_resolve(EnParams P)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const ScanEnv E = stage_scan(P, smem);
    Summary *sum = reinterpret_cast<Summary *>(smem + ((P.blob_bytes + 15u) & ~15u));
    uint32_t *first = reinterpret_cast<uint32_t *>(sum + RS_NT * KMAX);   // first chunk of each run
    uint32_t *entry = first + RS_NT;                                      // resolved candidate index
    unsigned long long *prefix = reinterpret_cast<unsigned long long *>(entry + RS_NT);
    const uint32_t t = threadIdx.x;
    const uint32_t per = (P.M + RS_NT - 1) / RS_NT;
    const uint32_t j0 = min(P.M, t * per), j1 = min(P.M, j0 + per);

    // follow the run [j0, j1) from candidate k of its first chunk
    auto follow = [&](uint32_t j, uint32_t k, bool label, unsigned long long base) -> Summary {
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
    };

    uint32_t f = NONE32_EN;
    for (uint32_t j = j0; j < j1; j++)
        if (P.start[j] != NOPOS64) {
            f = j;
            break;
        }
    first[t] = f;
    if (f != NONE32_EN) {
        const uint32_t K = P.cinfo[f] & 0xFFu;
        for (uint32_t k = 0; k < K; k++) sum[t * KMAX + k] = follow(f, k, false, 0);
    }
    __syncthreads();

    if (t == 0) {   // link the runs from BOUNDARY at offset 0
        uint16_t ctx = CTX_B;
        unsigned long long run = 0;
        uint32_t r = 0;
        bool failed = false;
        for (; r < RS_NT; r++) {
            entry[r] = NONE32_EN;
            prefix[r] = run;
            if (first[r] == NONE32_EN) continue;
            const int k = cand_index(E, P.cinfo[first[r]] >> 8, ctx);
            if (k < 0) {
                P.rec->error = 1;
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
                P.rec->error = 1;
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

    // label this run's chunks with their entry contexts and offsets
    for (uint32_t j = j0; j < j1; j++) {
        ChunkOut o{0, CTX_BAD, 0, 0};
        P.out[j] = o;
    }
    if (entry[t] != NONE32_EN) follow(first[t], entry[t], true, prefix[t]);
}

// (4) emit
__global__ void __launch_bounds__(EN_NT) en_emit(EnParams P)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const ScanEnv E = stage_scan(P, smem);
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < P.M; j += gridDim.x * blockDim.x) {
        const ChunkOut o = P.out[j];
        if (!o.live) continue;
        uint32_t jn;
        const uint64_t p1 = next_start(P, j, &jn);
        WriteTok wt{P.kinds, P.lens, P.cap, o.off};
        uint64_t fail;
        chunk_scan(E, P.start[j], p1, o.entry, wt, fail);
    }
}

}  // namespace
}  // namespace lx

using namespace lx;

extern "C" int lx_lex_enumerative(lx_ctx *c, const lx_tokenset *ts, const uint8_t *d_in, uint64_t n, int mode,
                                  uint16_t *d_kinds, uint32_t *d_lens, uint64_t capacity, uint64_t *n_tokens,
                                  uint64_t *consumed, void *stream)
{
    if (!c || !ts || !n_tokens || !consumed) return LX_E_INVAL;
    if (mode < LX_FULL_EXACT || mode > LX_FILTERED_MODULO) return LX_E_MODE;
    if (n && !d_in) return LX_E_INVAL;
    if (capacity && (!d_kinds || !d_lens)) return LX_E_INVAL;
    const ScanTable &st = ts->scan;
    if (st.status != LX_OK) return st.status;
    *n_tokens = 0;
    *consumed = 0;
    if (n == 0) return LX_OK;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != c->device) return LX_E_INVAL;
    void *blobs[3], *scan = nullptr;
    int rc = ensure_device_tables(ts, dev, blobs, &scan);
    if (rc != LX_OK) return rc;
    const uint64_t M64 = (n + CHUNK - 1) / CHUNK;
    if (M64 > 0xFFFFFFF0ull) return LX_E_INVAL;
    const uint32_t M = (uint32_t)M64;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_rec = 0, o_start = 256, o_cinfo = al(o_start + 8 * (size_t)M);
    const size_t o_res = al(o_cinfo + 4 * (size_t)M), o_out = al(o_res + sizeof(ChunkRes) * KMAX * (size_t)M);
    const size_t total = al(o_out + sizeof(ChunkOut) * (size_t)M);
    rc = grow(&c->e_dev, &c->e_dev_bytes, total);
    if (rc != LX_OK) return rc;
    uint8_t *d = static_cast<uint8_t *>(c->e_dev);

    EnParams P;
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

    const uint32_t smem = P.blob_bytes;
    const uint32_t rs_smem = ((smem + 15u) & ~15u) + sizeof(Summary) * RS_NT * KMAX + 8u * RS_NT + 8u * RS_NT;
    static bool attr_done[64] = {false};
    if (dev < 64 && !attr_done[dev]) {
        if (cudaFuncSetAttribute(en_plan, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024) != cudaSuccess ||
            cudaFuncSetAttribute(en_enumerate, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024) !=
                cudaSuccess ||
            cudaFuncSetAttribute(en_emit, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024) != cudaSuccess ||
            cudaFuncSetAttribute(en_resolve, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024) !=
                cudaSuccess)
            return LX_E_CUDA;
        attr_done[dev] = true;
    }
    if (rs_smem > 220u * 1024u) return LX_E_TOOBIG;
    const uint32_t grid = (uint32_t)std::min<uint64_t>((M + EN_NT - 1) / EN_NT, 4ull * c->num_sms);

    rc = cuda_err(cudaMemsetAsync(d, 0, 256, s));
    if (rc != LX_OK) return rc;
    if (c->timing) cudaEventRecord(c->ev[0], s);
    en_plan<<<grid, EN_NT, smem, s>>>(P);
    en_enumerate<<<grid, EN_NT, smem, s>>>(P);
    en_resolve<<<1, RS_NT, rs_smem, s>>>(P);
    en_emit<<<grid, EN_NT, smem, s>>>(P);
    rc = cuda_err(cudaGetLastError());
    if (c->timing) cudaEventRecord(c->ev[1], s);
    if (rc != LX_OK) return rc;
    EnResult r;
    rc = cuda_err(cudaMemcpyAsync(c->h_res, P.rec, sizeof(EnResult), cudaMemcpyDeviceToHost, s));
    if (rc == LX_OK) rc = cuda_err(cudaStreamSynchronize(s));
    if (rc != LX_OK) return rc;
    std::memcpy(&r, c->h_res, sizeof r);
    if (r.error) return LX_E_CUDA;
    *n_tokens = r.total;
    *consumed = r.fail == NOPOS64 ? n : r.fail;
    return r.total > capacity ? LX_E_CAPACITY : LX_OK;
}
