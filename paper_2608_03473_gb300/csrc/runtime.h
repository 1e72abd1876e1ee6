// runtime.h -- host-side runtime shared by the CUDA translation units: the
// context (scratch, pinned staging, graph cache, timing events) and the
// helpers that size its buffers and upload token-set tables.  Not part of the
// C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <utility>
#include <vector>

#include "internal.h"

// A launch configuration of the tile kernel for one token set and mode:
// the record column height and the CTAs per SM (capped by occupancy).
struct lx_tuned {
    const lx_tokenset *ts;
    int mode;
    uint32_t ks, ctas, cls;   // cls: class-indexed table
    float ms;   // measured by lx_autotune (0 when set by hand)
    int kernel = 0;           // LX_KERNEL_TILE or _WARP when lx_autotune chose one (0: not chosen)
    uint32_t warps = 0;       // warps per CTA it chose for the warp-tile kernel (0: as many as fit)
};

// Bytes of the pinned buffer for a kernel's launch record (lx_ctx::h_res).
constexpr size_t LAUNCH_RECORD_BYTES = 64;

struct lx_ctx {
    int device = 0;
    int num_sms = 0;
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    void *h_res = nullptr;   // pinned: the launch record read back by lx_lex (LAUNCH_RECORD_BYTES)
    uint64_t timeout_ns = 20ull * 1000 * 1000 * 1000;
    uint32_t withhold = 0xFFFFFFFFu;   // failure-detection tests (lx_ctx_debug_withhold)
    std::vector<std::pair<uint64_t, int>> occupancy;   // (form << 32 | shared bytes) -> CTAs per SM
    std::vector<lx_tuned> tuned;                       // per (token set, mode); default otherwise
    // lx_lex_batch: device scratch, pinned staging (descriptors up, records
    // down), the capture stream and the cached graph with its shape key
    void *b_dev = nullptr;
    size_t b_dev_bytes = 0;
    void *b_host = nullptr;
    size_t b_host_bytes = 0;
    cudaStream_t b_stream = nullptr;
    cudaGraphExec_t b_exec = nullptr;
    std::vector<uint64_t> b_key;
    // lx_lex_enumerative: device scratch
    void *e_dev = nullptr;
    size_t e_dev_bytes = 0;
    // device buffers of lx_lex_host, its copy streams, per-piece events and
    // pinned per-piece records
    void *d_in = nullptr;
    size_t d_in_bytes = 0;
    void *d_out = nullptr;
    size_t d_out_bytes = 0;
    void *h_scratch = nullptr;   // pinned
    size_t h_scratch_bytes = 0;
    cudaStream_t s_in = nullptr, s_out = nullptr;
    std::vector<cudaEvent_t> ev_in, ev_lex;
    // the failed-lookahead guard's prepass (liveness.cu): device scratch
    void *lv_dev = nullptr;
    size_t lv_dev_bytes = 0;
    // lx_lex kernel choice (lx_ctx_set_kernel): LX_KERNEL_AUTO, _TILE or _WARP
    int kernel = 0;
    // warps per CTA of the warp-tile kernel (0: as many as shared memory holds)
    uint32_t warps = 0;
    // lx_lex_batch on the warp-tile kernel: the combined table of the last
    // batch's token sets (key: mode and the sets' serial numbers)
    void *wb_dev = nullptr;
    size_t wb_dev_bytes = 0;
    std::vector<uint64_t> wb_key;
    uint32_t wb_blob_bytes = 0, wb_rows = 0, wb_acc_off = 0, wb_sets_off = 0;
    // the warp-tile kernel's geometry (lx_ctx_set_warp_geometry) and, in
    // LX_WARP_GEOMETRY_AUTO, the choice per (token set serial * 8 + mode)
    int warp_geometry = 0;
    std::vector<std::pair<uint64_t, bool>> warp_dense;
    // the warp-tile kernel's per-warp spill slots (kept tokens of a tile beyond its shared stage)
    void *w_spill = nullptr;
    size_t w_spill_bytes = 0;
    // optional kernel timing
    bool timing = false;
    cudaEvent_t ev[2] = {nullptr, nullptr};
};

namespace lx {

// lx_lex_host on the warp-tile kernel (lexwarp.cu): the K pieces [b[i],
// b[i+1]) of the host input (cut at certified bytes) each copied to a
// 16-byte aligned place on the device, lexed by their own launch with their
// own output range, and their tokens copied out after the previous pieces'
// once their records are in (same contract as lx_lex_host).  Uses the
// context's s_in / s_out streams and K of its ev_in / ev_lex events.  With
// sparse_limit != 0, LX_SPARSE or LX_LOOKAHEAD as lex_warp_device (some
// piece stopped early; the host buffers then hold nothing defined).
int lex_warp_host(lx_ctx *c, const lx_tokenset *ts, const uint8_t *h_in, uint64_t n, int mode, uint16_t *h_kinds,
                  uint32_t *h_lens, uint64_t capacity, const uint64_t *b, uint32_t K, uint64_t *n_tokens,
                  uint64_t *consumed, cudaStream_t st, uint64_t sparse_limit);
// LX_OK, LX_E_NOMEM for an allocation failure, LX_E_CUDA otherwise.
int cuda_err(cudaError_t e);
// Grow a device (grow) or pinned host (grow_host) buffer to at least `need`
// bytes; contents are not kept.
int grow(void **p, size_t *have, size_t need);
int grow_host(void **p, size_t *have, size_t need);
// The token set's tables on `device` (uploaded on first use): the walk-table
// blobs of each mode (both forms where both exist) and the plain scan table
// (nullptr where a table does not exist for this token set).
int ensure_device_tables(const lx_tokenset *ts, int device, DeviceTables *out);
// The warp-tile kernel (lexwarp.cu): whether lx_lex can take it for this
// token set, mode and input pointer (an event-code walk table and a 16-byte
// aligned input), and the call itself (same contract as lx_lex).  With
// sparse_limit != 0 a chunk longer than that many bytes (certified bytes too
// far apart) makes the call stop early and return LX_SPARSE, and backtracking
// steps beyond a budget proportional to n (failed lookahead) make it return
// LX_LOOKAHEAD, leaving the input to the enumerative path (guarded).
constexpr int LX_SPARSE = -100;   // internal status, never returned by the C ABI
bool warp_path_ok(const lx_tokenset *ts, int mode, const uint8_t *d_in);
// Warps per CTA for the warp-tile kernel on (ts, mode): the context's
// setting, else lx_autotune's choice, else 0 (as many as fit).
uint32_t warps_setting(const lx_ctx *c, const lx_tokenset *ts, int mode);
// lx_lex_async (lexwarp.cu): the warp-tile kernel and a status kernel that
// writes the result record to device memory; no synchronization, no fallback.
int lex_warp_async(lx_ctx *c, const lx_tokenset *ts, const uint8_t *d_in, uint64_t n, int mode, uint16_t *d_kinds,
                   uint32_t *d_lens, uint64_t capacity, lx_async_result *d_result, cudaStream_t st);
// lx_lex_batch in one launch of the warp-tile kernel (lexwarp.cu): every
// document of every token set, the sets' class-form tables side by side in
// shared memory, the output in document order.  LX_SPARSE when not
// applicable (a table without a class form, rows beyond the 16-bit window,
// an unaligned document): the caller takes the per-set tile kernels.
int lex_batch_warp(lx_ctx *c, const lx_tokenset *const *sets, uint32_t n_sets, const lx_doc *docs, uint32_t n_docs,
                   int mode, uint16_t *d_kinds, uint32_t *d_lens, uint64_t capacity, lx_doc_result *results,
                   uint64_t *n_total, cudaStream_t st);
int lex_warp_device(lx_ctx *c, const lx_tokenset *ts, const uint8_t *d_in, uint64_t n, int mode, uint16_t *d_kinds,
                    uint32_t *d_lens, uint64_t capacity, uint64_t *n_tokens, uint64_t *consumed, cudaStream_t st,
                    uint64_t sparse_limit);
// Internal status: a scan ran past its step budget (failed lookahead, or a
// token spanning many chunks); the caller runs the input again with the
// failed-lookahead guard.  Never returned by the C ABI.
constexpr int LX_LOOKAHEAD = -101;
// lx_lex_enumerative (enumerate.cu) with the failed-lookahead guard from the
// start when `guard` (the caller saw a scan run past its budget already).
int lex_enumerative_device(lx_ctx *c, const lx_tokenset *ts, const uint8_t *d_in, uint64_t n, int mode,
                           uint16_t *d_kinds, uint32_t *d_lens, uint64_t capacity, uint64_t *n_tokens,
                           uint64_t *consumed, cudaStream_t stream, bool guard);
// The guard's prepass (liveness.cu): the liveness automaton's state at every
// offset 0..n of the input into d_out[n + 1] (nullptr: the context's scratch);
// *live receives the array, *member the automaton's member bitsets on the
// device.  LX_E_TOOBIG when the token set has no liveness automaton.
int liveness_device(lx_ctx *c, const lx_tokenset *ts, const uint8_t *d_in, uint64_t n, uint8_t *d_out,
                    cudaStream_t s, const uint8_t **live, const uint32_t **member);
// The entry-context model (model.cu): number of contexts it scores, and the
// BF16 prediction of the entry context of every chunk start (0xFFFE =
// BOUNDARY) into guess[M], restricted to the candidates of the byte before.
uint32_t model_contexts(const lx_model *m);
int model_predict(lx_model *m, const uint8_t *in, uint64_t n, const uint64_t *start, const uint32_t *cinfo,
                  const uint8_t *scan_blob, uint32_t cbeg_off, uint32_t cand_off, uint32_t M, uint16_t *guess,
                  cudaStream_t s);

}  // namespace lx
