// lex.cu -- GB300 (sm_103a) certified-split lexing: the tile kernel and the
// lx_lex / lx_ctx entry points.
//
// One persistent CTA per resident slot loops over tiles of TILE input bytes.
// Per tile:
//   (a) stage: a 1-D bulk copy (cp.async.bulk, TMA) brings the tile plus a
//       halo into shared memory, double-buffered against the previous tile;
//   (b) plan:  each of NT threads owns the equal-division target of its
//       SEG-byte segment and slides it forward to the first byte of the
//       mode's certified set in the segment (the planner of Section 6 with
//       k = one target per thread); a segment holding no certified byte
//       yields no chunk and the previous chunk runs on;
//   (c) walk:  from its start each thread runs the longest-match loop of
//       Section 3 from q0 over the shared-memory walk table (internal.h),
//       every certified byte ending the token in progress, until it reaches
//       a certified byte at or past its segment end (the next chunk start) or
//       the end of the input; tokens go to per-thread shared slots;
//   (d) emit:  a CTA scan of kept-token counts, a decoupled look-back over
//       per-tile status words for the global offset, compaction through a
//       shared staging array and coalesced writes of kinds (u16) and
//       lengths (u32).  The first lexing failure (Corollary 1) is combined
//       with device atomics.
// Every device-side wait is bounded by a %globaltimer budget.

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>

#include "internal.h"

namespace lx {

constexpr int NT = 256;                 // threads per CTA
constexpr int SEG = 68;                 // bytes per thread target (17 words: odd stride)
constexpr int TILE = NT * SEG;          // 17408 input bytes per tile
constexpr int HALO = 1024;              // extra staged bytes for walks that run past the tile
constexpr int BUF = TILE + HALO;        // 18432, a multiple of 16
constexpr int KSLOT = 20;               // shared token slots per thread
constexpr int STAGE_CAP = 4096;         // tokens per tile that take the coalesced path
constexpr uint64_t NOPOS = ~0ull;

constexpr unsigned ERR_TIMEOUT = 1u;
constexpr unsigned ERR_SMEM = 2u;

constexpr unsigned long long ST_AGG = 1ull << 62;
constexpr unsigned long long ST_INCL = 2ull << 62;
constexpr unsigned long long ST_VAL = (1ull << 62) - 1;

struct Result {
    unsigned long long total;          // kept tokens over all chunks (atomicAdd)
    unsigned long long inv_fail_pos;   // ~min failure offset (atomicMax), 0 = none
    unsigned long long inv_fail_tok;   // ~min token index at the failure
    unsigned int error;
    unsigned int pad;
};

struct Params {
    const uint8_t *in;
    uint64_t n;
    const uint8_t *blob;
    uint32_t blob_bytes, table_bytes, kind_off, cmap_off, cert_off;
    uint32_t ncols;
    uint32_t p_start, p_flag, p_slow;
    uint16_t *out_kinds;
    uint32_t *out_lens;
    uint64_t cap;
    unsigned long long *status;
    unsigned int *tile_counter;
    Result *res;
    uint32_t n_tiles;
    int tma;
    uint64_t timeout_ns;
};

// ---- shared-memory layout (bytes from the dynamic shared base) ----
struct Layout {
    uint32_t blob, buf0, buf1, slots, stage, misc, total;
};

__host__ __device__ inline uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) & ~(a - 1); }

__host__ __device__ inline Layout make_layout(uint32_t blob_bytes)
{
    Layout L;
    L.blob = 0;                                   // + up to 511 bytes to 512-align the table
    L.buf0 = align_up(512 + blob_bytes, 128);
    L.buf1 = L.buf0 + BUF;
    L.slots = L.buf1 + BUF;
    L.stage = L.slots + KSLOT * NT * 4;
    L.misc = L.stage + STAGE_CAP * 4;
    L.total = L.misc + 256;
    return L;
}

// misc region offsets
constexpr uint32_t M_WARP = 0;      // u64[8] warp totals -> exclusive offsets
constexpr uint32_t M_MBAR = 64;     // u64[2]
constexpr uint32_t M_TILE = 80;     // u32[2]: next tile id, flags
constexpr uint32_t M_G = 96;        // u64: tile's global output offset
constexpr uint32_t M_TOT = 104;     // u64: tile total
constexpr uint32_t M_FLAG = 112;    // u32: CTA flags

// ---- PTX helpers ----
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
__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
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

// ---- the walk ----
struct Env {
    uint32_t buf;          // shared address of the staged tile
    uint64_t tile_base;    // input offset of buf[0]
    uint64_t sm_end;       // input offset one past the last staged byte
    const uint8_t *in;
    uint64_t n;
    uint32_t P_start, P_flag, P_slow;
    uint32_t tbase, kind_s, cmap_s, cert_s, kcol2;
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

template <int FORM>
__device__ __forceinline__ uint32_t kind_of(const Env &E, uint32_t e)
{
    if (FORM == FORM_BYTE) return lds_u16(E.kind_s + (((e - E.tbase) >> 9) << 1));
    return lds_u16(e + E.kcol2);
}

__device__ __forceinline__ bool is_cut(const Env &E, uint32_t b) { return lds_u8(E.cert_s + b) != 0; }

// Emission into shared slots (first pass).
struct SlotEmit {
    uint32_t slots;   // shared address of this thread's slot column
    uint32_t count;
    bool ovf;
    __device__ __forceinline__ void operator()(uint32_t kw, uint64_t len)
    {
        if (!(kw & KIND_KEEP)) return;
        uint32_t k = kw & 0x7FFFu;
        if (count < KSLOT && len < (1u << 20) && k < 4096u) {
            uint32_t v = (k << 20) | (uint32_t)len;
            asm volatile("st.shared.u32 [%0], %1;" ::"r"(slots + count * NT * 4), "r"(v) : "memory");
        } else {
            ovf = true;
        }
        count++;
    }
};

// Emission straight to global memory (tiles that overflow their slots).
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
// where no positive-length accepting prefix exists) or NOPOS.
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
            if (e2 >= E.P_flag) {
                if (e2 >= E.P_slow) {
                    slow = true;
                } else {
                    emit(kind_of<FORM>(E, e), p - tok);   // token [tok, p) ends before byte p
                    tok = p;
                    if (p >= seg_end && is_cut(E, b)) return NOPOS;
                }
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

// Decoupled look-back (thread 0): publish this tile's aggregate, accumulate
// predecessors until an inclusive prefix, publish ours.  Bounded spin.
__device__ uint64_t lookback(const Params &P, uint32_t tile, uint64_t agg, bool need, bool &timed_out)
{
    if (tile == 0) {
        st_release(&P.status[0], ST_INCL | agg);
        return 0;
    }
    st_release(&P.status[tile], ST_AGG | agg);
    if (!need) return 0;
    uint64_t G = 0;
    uint32_t k = tile - 1;
    uint64_t t0 = globaltimer();
    uint32_t spins = 0;
    for (;;) {
        unsigned long long v = ld_acquire(&P.status[k]);
        unsigned long long f = v & ~ST_VAL;
        if (f == 0) {
            if ((++spins & 15) == 0 && globaltimer() - t0 > P.timeout_ns) {
                timed_out = true;
                break;
            }
            __nanosleep(64);
            continue;
        }
        G += v & ST_VAL;
        if (f == ST_INCL) break;
        k--;
    }
    st_release(&P.status[tile], ST_INCL | (G + agg));
    return G;
}

template <int FORM>
__global__ void __launch_bounds__(NT, 2) lex_tiles(Params P)
{
    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const Layout L = make_layout(P.blob_bytes);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t tbase = align_up(sbase, 512);
    uint8_t *misc = smem + L.misc;
    const uint32_t misc_s = sbase + L.misc;
    const uint32_t mbar[2] = {misc_s + M_MBAR, misc_s + M_MBAR + 8};
    const uint32_t bufs[2] = {sbase + L.buf0, sbase + L.buf1};

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
    E.in = P.in;
    E.n = P.n;
    E.P_start = tbase + P.p_start;
    E.P_flag = tbase + P.p_flag;
    E.P_slow = tbase + P.p_slow;
    E.tbase = tbase;
    E.kind_s = tbase + P.kind_off;
    E.cmap_s = tbase + P.cmap_off;
    E.cert_s = tbase + P.cert_off;
    E.kcol2 = 2 * (P.ncols - 1);

    volatile uint32_t *s_tile = reinterpret_cast<volatile uint32_t *>(misc + M_TILE);
    if (tid == 0) {
        mbar_init(mbar[0], 1);
        mbar_init(mbar[1], 1);
        fence_proxy_async();
    }
    __syncthreads();

    auto issue = [&](uint32_t tile, int which) {   // thread 0
        uint64_t base = (uint64_t)tile * TILE;
        uint64_t avail = P.n - base;
        uint32_t len = (uint32_t)(avail < (uint64_t)BUF ? avail : (uint64_t)BUF) & ~15u;
        if (len) {
            fence_proxy_async();
            tma_load(bufs[which], P.in + base, len, mbar[which]);
        }
    };

    if (tid == 0) {
        uint32_t t = atomicAdd(P.tile_counter, 1u);
        s_tile[0] = t;
        if (t < P.n_tiles && P.tma) issue(t, 0);
    }
    __syncthreads();
    uint32_t tile = s_tile[0];
    uint32_t parity[2] = {0, 0};
    int cur = 0;
    uint32_t *slots32 = reinterpret_cast<uint32_t *>(smem + L.slots);
    uint32_t *stage32 = reinterpret_cast<uint32_t *>(smem + L.stage);
    unsigned long long *warp_tot = reinterpret_cast<unsigned long long *>(misc + M_WARP);

    while (tile < P.n_tiles) {
        __syncthreads();   // everyone has read s_tile
        if (tid == 0) {
            uint32_t t = atomicAdd(P.tile_counter, 1u);
            s_tile[0] = t;
            if (t < P.n_tiles && P.tma) issue(t, cur ^ 1);
        }
        const uint64_t tile_base = (uint64_t)tile * TILE;
        const uint64_t avail = P.n - tile_base;
        uint32_t staged;
        bool bad = false;
        if (P.tma) {
            staged = (uint32_t)(avail < (uint64_t)BUF ? avail : (uint64_t)BUF) & ~15u;
            if (staged) {
                bad = !mbar_wait(mbar[cur], parity[cur], P.timeout_ns);
                parity[cur] ^= 1;
            }
        } else {
            staged = (uint32_t)(avail < (uint64_t)BUF ? avail : (uint64_t)BUF);
            uint8_t *b = smem + (bufs[cur] - sbase);
            for (uint32_t i = tid; i < staged; i += NT) b[i] = P.in[tile_base + i];
        }
        if (__syncthreads_or(bad)) {
            if (tid == 0) atomicOr(&P.res->error, ERR_TIMEOUT);
            break;
        }
        E.buf = bufs[cur];
        E.tile_base = tile_base;
        E.sm_end = tile_base + staged;

        // (b) plan: first certified byte of this thread's segment
        const uint64_t seg_start = tile_base + (uint64_t)tid * SEG;
        const uint64_t seg_end = seg_start + SEG;
        uint64_t start = NOPOS;
        if (tile == 0 && tid == 0) {
            start = 0;
        } else {
            uint64_t lim = seg_end < P.n ? seg_end : P.n;
            for (uint64_t p = seg_start; p < lim; p++)
                if (is_cut(E, byte_at(E, p))) { start = p; break; }
        }
        // (c) walk
        SlotEmit se{smem_u32(slots32 + tid), 0, false};
        uint64_t fail = NOPOS;
        if (start != NOPOS) fail = walk<FORM>(E, start, seg_end, se);

        // (d) CTA scan of kept-token counts
        uint32_t x = se.count;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        const uint32_t lane_excl = x - se.count;
        if (lane == 31) warp_tot[wid] = x;
        const int any_ovf = __syncthreads_or(se.ovf);
        const int any_fail = __syncthreads_or(fail != NOPOS);
        if (tid == 0) {
            unsigned long long acc = 0;
            for (int w = 0; w < NT / 32; w++) {
                unsigned long long t = warp_tot[w];
                warp_tot[w] = acc;
                acc += t;
            }
            bool to = false;
            uint64_t G = lookback(P, tile, acc, acc > 0 || any_fail, to);
            if (to) atomicOr(&P.res->error, ERR_TIMEOUT);
            if (acc) atomicAdd(&P.res->total, acc);
            *reinterpret_cast<unsigned long long *>(misc + M_G) = G;
            *reinterpret_cast<unsigned long long *>(misc + M_TOT) = acc;
        }
        __syncthreads();
        const uint64_t G = *reinterpret_cast<unsigned long long *>(misc + M_G);
        const uint64_t cta_total = *reinterpret_cast<unsigned long long *>(misc + M_TOT);
        const uint64_t my_off = warp_tot[wid] + lane_excl;   // within the tile

        if (!any_ovf && cta_total <= (uint64_t)STAGE_CAP) {
            for (uint32_t k = 0; k < se.count; k++) stage32[my_off + k] = slots32[k * NT + tid];
            __syncthreads();
            for (uint32_t i = tid; i < cta_total; i += NT) {
                uint64_t idx = G + i;
                if (idx < P.cap) {
                    uint32_t v = stage32[i];
                    P.out_kinds[idx] = (uint16_t)(v >> 20);
                    P.out_lens[idx] = v & 0xFFFFFu;
                }
            }
        } else if (se.count) {
            if (!se.ovf) {
                for (uint32_t k = 0; k < se.count; k++) {
                    uint64_t idx = G + my_off + k;
                    if (idx < P.cap) {
                        uint32_t v = slots32[k * NT + tid];
                        P.out_kinds[idx] = (uint16_t)(v >> 20);
                        P.out_lens[idx] = v & 0xFFFFFu;
                    }
                }
            } else {
                DirectEmit de{P.out_kinds, P.out_lens, P.cap, G + my_off};
                walk<FORM>(E, start, seg_end, de);
            }
        }
        if (fail != NOPOS) {
            atomicMax(&P.res->inv_fail_pos, ~(unsigned long long)fail);
            atomicMax(&P.res->inv_fail_tok, ~(unsigned long long)(G + my_off + se.count));
        }
        __syncthreads();   // slots, stage and this buffer are free again
        tile = s_tile[0];
        cur ^= 1;
    }
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

struct lx_ctx {
    int device = 0;
    int num_sms = 0;
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    Result *h_res = nullptr;   // pinned
    uint64_t timeout_ns = 20ull * 1000 * 1000 * 1000;
    int occupancy[2] = {0, 0};
    // device buffers of lx_lex_host
    void *d_in = nullptr;
    size_t d_in_bytes = 0;
    void *d_out = nullptr;
    size_t d_out_bytes = 0;
    // optional kernel timing
    bool timing = false;
    cudaEvent_t ev[2] = {nullptr, nullptr};
};

static int ensure_device_tables(const lx_tokenset *cts, int device, void **out_blobs)
{
    lx_tokenset *ts = const_cast<lx_tokenset *>(cts);
    std::lock_guard<std::mutex> g(ts->mu);
    for (auto &d : ts->dev)
        if (d.device == device) {
            for (int m = 0; m < 3; m++) out_blobs[m] = d.d_blob[m];
            return LX_OK;
        }
    DeviceTables dt;
    dt.device = device;
    for (int m = 0; m < 3; m++) {
        const HostTable &h = ts->tab[m];
        if (h.status != LX_OK) continue;
        int rc = cuda_err(cudaMalloc(&dt.d_blob[m], h.blob.size()));
        if (rc == LX_OK) rc = cuda_err(cudaMemcpy(dt.d_blob[m], h.blob.data(), h.blob.size(), cudaMemcpyHostToDevice));
        if (rc != LX_OK) {
            for (int k = 0; k <= m; k++) cudaFree(dt.d_blob[k]);
            return rc;
        }
    }
    ts->dev.push_back(dt);
    for (int m = 0; m < 3; m++) out_blobs[m] = dt.d_blob[m];
    return LX_OK;
}

extern "C" void lx_tokenset_free(lx_tokenset *ts)
{
    if (!ts) return;
    int cur = -1;
    cudaGetDevice(&cur);
    for (auto &d : ts->dev) {
        cudaSetDevice(d.device);
        for (int m = 0; m < 3; m++)
            if (d.d_blob[m]) cudaFree(d.d_blob[m]);
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
        cudaMallocHost(reinterpret_cast<void **>(&c->h_res), sizeof(Result)) != cudaSuccess) {
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
    if (c->d_in) cudaFree(c->d_in);
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

extern "C" int lx_ctx_set_timeout_ms(lx_ctx *c, uint32_t ms)
{
    if (!c || ms == 0) return LX_E_INVAL;
    c->timeout_ns = (uint64_t)ms * 1000000ull;
    return LX_OK;
}

static int grow(void **p, size_t *have, size_t need)
{
    if (*have >= need) return LX_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *have = 0;
    size_t sz = std::max(need, *have * 2);
    int rc = cuda_err(cudaMalloc(p, sz));
    if (rc == LX_OK) *have = sz;
    return rc;
}

// Launch the tile kernel and read back its result record.
static int lex_device(lx_ctx *c, const lx_tokenset *ts, const uint8_t *d_in, uint64_t n, int mode,
                      uint16_t *d_kinds, uint32_t *d_lens, uint64_t capacity, uint64_t *n_tokens,
                      uint64_t *consumed, cudaStream_t st)
{
    const HostTable &h = ts->tab[mode];
    if (h.status != LX_OK) return h.status;
    if (n == 0) {
        *n_tokens = 0;
        *consumed = 0;
        return LX_OK;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != c->device) return LX_E_INVAL;
    void *blobs[3];
    int rc = ensure_device_tables(ts, dev, blobs);
    if (rc != LX_OK) return rc;

    const uint64_t n_tiles64 = (n + TILE - 1) / TILE;
    if (n_tiles64 > 0xFFFFFFF0ull) return LX_E_INVAL;
    const uint32_t n_tiles = (uint32_t)n_tiles64;
    const size_t need = 64 + sizeof(unsigned long long) * (size_t)n_tiles;
    rc = grow(&c->scratch, &c->scratch_bytes, need);
    if (rc != LX_OK) return rc;

    Params P;
    P.in = d_in;
    P.n = n;
    P.blob = static_cast<const uint8_t *>(blobs[mode]);
    P.blob_bytes = (uint32_t)h.blob.size();
    P.table_bytes = h.table_bytes;
    P.kind_off = h.kind_off;
    P.cmap_off = h.cmap_off;
    P.cert_off = h.cert_off;
    P.ncols = h.ncols;
    P.p_start = h.p_start;
    P.p_flag = h.p_flag;
    P.p_slow = h.p_slow;
    P.out_kinds = d_kinds;
    P.out_lens = d_lens;
    P.cap = capacity;
    uint8_t *scr = static_cast<uint8_t *>(c->scratch);
    P.res = reinterpret_cast<Result *>(scr);
    P.tile_counter = reinterpret_cast<unsigned int *>(scr + 32);
    P.status = reinterpret_cast<unsigned long long *>(scr + 64);
    P.n_tiles = n_tiles;
    P.tma = ((reinterpret_cast<uintptr_t>(d_in) & 15u) == 0) ? 1 : 0;
    P.timeout_ns = c->timeout_ns;

    const Layout L = make_layout(P.blob_bytes);
    const int form = h.form;
    if (!c->occupancy[form]) {
        cudaError_t e;
        if (form == FORM_BYTE) {
            e = cudaFuncSetAttribute(lex_tiles<FORM_BYTE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->occupancy[form], lex_tiles<FORM_BYTE>, NT, L.total);
        } else {
            e = cudaFuncSetAttribute(lex_tiles<FORM_CLASS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->occupancy[form], lex_tiles<FORM_CLASS>, NT, L.total);
        }
        if (e != cudaSuccess) return LX_E_CUDA;
        if (c->occupancy[form] < 1) c->occupancy[form] = 1;
    }
    const uint32_t grid = (uint32_t)std::min<uint64_t>(n_tiles, (uint64_t)c->occupancy[form] * c->num_sms);

    rc = cuda_err(cudaMemsetAsync(c->scratch, 0, need, st));
    if (rc != LX_OK) return rc;
    if (c->timing) cudaEventRecord(c->ev[0], st);
    if (form == FORM_BYTE) lex_tiles<FORM_BYTE><<<grid, NT, L.total, st>>>(P);
    else lex_tiles<FORM_CLASS><<<grid, NT, L.total, st>>>(P);
    rc = cuda_err(cudaGetLastError());
    if (c->timing) cudaEventRecord(c->ev[1], st);
    if (rc != LX_OK) return rc;
    rc = cuda_err(cudaMemcpyAsync(c->h_res, P.res, sizeof(Result), cudaMemcpyDeviceToHost, st));
    if (rc == LX_OK) rc = cuda_err(cudaStreamSynchronize(st));
    if (rc != LX_OK) return rc;
    const Result r = *c->h_res;
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

extern "C" int lx_lex_host(lx_ctx *c, const lx_tokenset *ts, const uint8_t *h_in, uint64_t n, int mode,
                           uint16_t *h_kinds, uint32_t *h_lens, uint64_t capacity, uint64_t *n_tokens,
                           uint64_t *consumed, void *stream)
{
    int rc = check_args(c, ts, h_in, n, mode, h_kinds, h_lens, capacity, n_tokens, consumed);
    if (rc != LX_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rc = grow(&c->d_in, &c->d_in_bytes, n ? n : 1);
    if (rc == LX_OK) rc = grow(&c->d_out, &c->d_out_bytes, capacity ? capacity * 6 + 16 : 16);
    if (rc != LX_OK) return rc;
    uint32_t *d_lens = static_cast<uint32_t *>(c->d_out);
    uint16_t *d_kinds = reinterpret_cast<uint16_t *>(d_lens + capacity);
    if (n) {
        rc = cuda_err(cudaMemcpyAsync(c->d_in, h_in, n, cudaMemcpyHostToDevice, st));
        if (rc != LX_OK) return rc;
    }
    rc = lex_device(c, ts, static_cast<const uint8_t *>(c->d_in), n, mode, d_kinds, d_lens, capacity,
                    n_tokens, consumed, st);
    if (rc != LX_OK && rc != LX_E_CAPACITY) return rc;
    uint64_t m = std::min(*n_tokens, capacity);
    if (m) {
        int r2 = cuda_err(cudaMemcpyAsync(h_kinds, d_kinds, m * 2, cudaMemcpyDeviceToHost, st));
        if (r2 == LX_OK) r2 = cuda_err(cudaMemcpyAsync(h_lens, d_lens, m * 4, cudaMemcpyDeviceToHost, st));
        if (r2 == LX_OK) r2 = cuda_err(cudaStreamSynchronize(st));
        if (r2 != LX_OK) return r2;
    }
    return rc;
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
