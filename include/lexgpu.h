/*
 * lexgpu.h -- C ABI of the GB300 certified-split lexer.
 *
 * Longest-match (maximal munch), table-driven DFA lexing of one large byte
 * buffer on one GPU, split at certified split symbols and rejoined by ordered
 * concatenation, after "Certified Split Points for Parallel Lexing: Exact and
 * Modulo Discarded Tokens".  Paper references below are to its sections,
 * definitions and theorems.
 *
 * Conventions
 *   - Every function returns LX_OK (0) or a negative LX_E_* code.  A lexing
 *     error in the input is NOT a status error: it is reported through
 *     *consumed (Section 3: con(w)); the input is completely tokenizable iff
 *     *consumed == n.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory of the current device.  The caller owns every buffer it
 *     passes; the library never frees or retains them past the call.
 *   - Streams are passed as `void *` holding a cudaStream_t (NULL = the legacy
 *     default stream).  Work is stream-ordered.
 *   - Objects (lx_tokenset, lx_ctx) are owned by the library and released
 *     with the matching *_free call.  A token set is immutable after
 *     compilation and may be shared by several contexts and threads; a
 *     context must not be used by two host threads at once.
 */
#ifndef LEXGPU_H
#define LEXGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define LX_OK 0
#define LX_E_INVAL (-1)    /* malformed argument or automaton                  */
#define LX_E_NOMEM (-2)    /* host or device allocation failed                 */
#define LX_E_CAPACITY (-3) /* output capacity too small; *n_tokens = required  */
#define LX_E_CUDA (-4)     /* a CUDA runtime call failed                       */
#define LX_E_TIMEOUT (-5)  /* a bounded device-side wait ran out               */
#define LX_E_MODE (-6)     /* mode not allowed (e.g. full stream, modulo cuts) */
#define LX_E_TOOBIG (-7)   /* automaton too large for the shared-memory tables */

#define LX_NONE 0xFFFFFFFFu /* undefined transition in lx_dfa.next             */
#define LX_NO_KIND 0xFFFFu  /* non-accepting state in lx_dfa.accept_kind       */

/*
 * A compiled token set, A = (Q, Sigma, delta, q0, tau) of Section 3, in the
 * class-compressed physical form `state = table[row(byte) + state]` of
 * Section 1.  All arrays are host memory, read during lx_compile_tokenset
 * only (copied).
 *   n_states     |Q| >= 1
 *   n_classes    number of byte classes, 1..256
 *   q0           initial state, < n_states
 *   n_kinds      number of token kinds, 1..32767
 *   byte_class   [256]: class of each byte value, < n_classes
 *   next         [n_classes * n_states]: next[c * n_states + q] = delta(q, b)
 *                for any byte b of class c, or LX_NONE when undefined
 *   accept_kind  [n_states]: tau(q), or LX_NO_KIND (tau is partial; any
 *                same-length tie is already resolved, Section 3)
 */
typedef struct lx_dfa {
    uint32_t n_states;
    uint32_t n_classes;
    uint32_t q0;
    uint32_t n_kinds;
    const uint8_t *byte_class;
    const uint32_t *next;
    const uint16_t *accept_kind;
} lx_dfa;

typedef struct lx_tokenset lx_tokenset;
typedef struct lx_ctx lx_ctx;

/* Output modes of lx_lex. */
enum {
    LX_FULL_EXACT = 0,      /* tok(w) in full, cuts at exact certificates (Theorem 1)          */
    LX_FILTERED_EXACT = 1,  /* pi_I(tok(w)), cuts at exact certificates (Theorem 1, Section 5) */
    LX_FILTERED_MODULO = 2  /* pi_I(tok(w)), cuts at certificates modulo I (Theorem 3)         */
};

/*
 * lx_compile_tokenset -- validate the automaton and derive both certificates
 * (Sections 4 and 6; Section 6.1 for the modulo condition) in time linear in
 * the table: predecessor index, co-accessibility, reachability, re-entrancy
 * (Definition 1), the exact map (Definition 2) and the map modulo the
 * discarded set I (Definition 3), each restricted to useful bytes
 * (Corollary 2, Proposition 2).  I is fixed here, not per call (Section 6.1).
 *   dfa          host, read only during the call
 *   discarded    host array of n_discarded kind ids (< dfa->n_kinds), may be
 *                NULL when n_discarded == 0; duplicates allowed
 *   out          receives a new token set; release with lx_tokenset_free
 * Pure host code: needs no GPU.  Device tables are uploaded lazily by the
 * first lx_lex on each device.
 * Errors: LX_E_INVAL (bad sizes, out-of-range entries), LX_E_NOMEM.
 */
int lx_compile_tokenset(const lx_dfa *dfa, const uint16_t *discarded, uint32_t n_discarded,
                        lx_tokenset **out);

/*
 * lx_compile_tokenset_framed -- lx_compile_tokenset for documents framed at
 * the producer (Section 7.1, Framing at the producer).  The reserved byte
 * `frame_byte` (conventionally 0x1E, RECORD SEPARATOR) gets a rule of its own:
 * a new token kind, numbered dfa->n_kinds, of that one byte from q0; every
 * other state of `dfa` rejects the byte, so no other token admits it at any
 * position.  Its only live consumption is then from q0, and with q0 not
 * re-entrant Definition 2 certifies it: a document whose producer emits the
 * byte only at token boundaries (escaping it inside tokens) splits at every
 * occurrence, whatever the rest of the token set certifies.  With
 * frame_discarded != 0 the frame kind joins the discarded set.  The
 * automaton gains one state and, when the byte shares its class, one class.
 * Errors as lx_compile_tokenset; LX_E_INVAL for frame_byte > 255.
 */
int lx_compile_tokenset_framed(const lx_dfa *dfa, const uint16_t *discarded, uint32_t n_discarded,
                               uint32_t frame_byte, int frame_discarded, lx_tokenset **out);

/*
 * lx_certificates -- the useful certified bytes (Corollary 2) and the useful
 * bytes certified modulo I (Proposition 2).  Bit (b & 31) of word (b >> 5) is
 * byte b.  Either output pointer may be NULL.  Host only.
 */
int lx_certificates(const lx_tokenset *ts, uint32_t exact_useful[8], uint32_t modulo_useful[8]);

/* lx_tokenset_info -- sizes of the compiled set: n_states, live states (|Q+|),
 * re-entrancy of q0 (Definition 1) as 0/1, and the shared-memory table form
 * chosen for `mode` (0 = byte-indexed, 1 = class-indexed) with its row count.
 * Any output pointer may be NULL. */
int lx_tokenset_info(const lx_tokenset *ts, int mode, uint32_t *n_states, uint32_t *n_live,
                     int *reentrant, int *table_form, uint32_t *table_rows);

/*
 * lx_tokenset_table -- the packed shared-memory walk table built for `mode`
 * (for inspection and host-side tests).  Copies min(cap, size) bytes of the
 * blob to `out` (host, may be NULL) and fills the first meta_len (<= 12)
 * entries of meta (host, may be NULL):
 *   { blob bytes, table_form, n_rows, ncols, row_bytes, table_bytes,
 *     p_start, p_flag, p_slow, kind_off | cmap_off << 16, cert_off, p_pre }.
 * Row pointers in the blob are offsets from the start of the blob.
 */
int lx_tokenset_table(const lx_tokenset *ts, int mode, void *out, uint32_t cap, uint32_t *meta,
                      uint32_t meta_len);
/* The same for the class-indexed table of `mode` (the default table when
 * that is class-indexed already). */
int lx_tokenset_class_table(const lx_tokenset *ts, int mode, void *out, uint32_t cap, uint32_t *meta,
                            uint32_t meta_len);

/*
 * lx_tokenset_walk_table -- the event-code walk table of `mode` that the
 * warp-tile kernel of lx_lex stages in shared memory (for inspection and
 * host-side tests).  Copies min(cap, size) bytes of the blob to `out` (host,
 * may be NULL) and fills the first meta_len (<= 12) entries of meta:
 *   { blob bytes, table_form, n_rows, row_shift, p_start, p_pre,
 *     acc_off, kmap_off, cmap_off, cut_off, n_ctx, ctx_off }
 * (n_ctx, ctx_off: the split-window context classes, lx_window_certificates).
 * Entries are u16: target row offset (from the blob start) | event code << 1
 * (code 0: no token ended before the byte; 1: a discarded token ended;
 * c >= 2: a kept token of kind kind_map[c] ended).  Byte form: row r holds
 * the entry of byte b at r * 512 + 2b; class form: of class c at
 * r * 256 + 2c, with cmap2[b] = 2 class(b).  Returns LX_E_TOOBIG when the
 * automaton has no such table for `mode` (more than 126 kept kinds, or rows
 * beyond the shared-memory budget); lx_lex then takes the tile kernel.
 */
int lx_tokenset_walk_table(const lx_tokenset *ts, int mode, void *out, uint32_t cap, uint32_t *meta,
                           uint32_t meta_len);

/*
 * lx_window_certificates -- two-byte split windows, the generalisation of the
 * exact certificate (Definition 2) to a byte in one byte of left context that
 * Sections 1 and 9 mention (the paper defines no window certificate; this is
 * the library's, written in the header so that it can be checked):
 *   Z(a)      = { delta+(q, a) : q in Q+ }   (the states right after reading a)
 *   cert(a,b) = q0 not re-entrant, delta+(q0, b) defined, and no state of Z(a)
 *               has a transition on b into Q+.
 * With q0 not re-entrant no token can read a and then b, so every occurrence
 * of a b has a token boundary between the bytes: a cut before b is exact
 * (Theorem 1's argument applies unchanged).  b is exact-certified iff (a, b)
 * is certified for every a.  Fills pairs[a * 8 + (b >> 5)] bit (b & 31) for
 * every pair (256 x 8 words, host).  In the exact modes the warp-tile kernel
 * also cuts at certified windows: its walk table gains PRE_k rows (PRE in the
 * context class k of the byte before), meta[10] = number of context classes K
 * and meta[11] = offset of the u8[256] context map; the cut table at cut_off
 * then has K + 1 rows of 256 bytes (row k: a chunk may start at byte b after a
 * byte of context k).  Returns LX_OK.
 */
int lx_window_certificates(const lx_tokenset *ts, uint32_t *pairs);

/*
 * lx_tokenset_liveness -- the liveness automaton of the failed-lookahead guard
 * (for inspection and tests).  Read from right to left over the input, its
 * state after w[k..n) stands for the set
 *   live_k = { q in Q+ : delta+*(q, w[k..m)) is accepting for some m > k }
 * (empty at k = n): the states from which a scan at offset k still has an
 * accepting position ahead.  A scan whose state is outside live_k has passed
 * its last accepting position and may end its token at once -- the memo of
 * failed (state, position) pairs of Reps' maximal-munch scanner, computed in
 * one pass before the scan.  Its states are the distinct sets reachable from
 * the empty set under F_c(X) = { q in Q+ : delta+(q, c) accepts or lies in X }.
 * Copies min(cap, size) bytes of the blob to `out` (host, may be NULL) and
 * fills meta[0..7] = { blob bytes, R (automaton states), C (classes), S (DFA
 * states), W (member words per state), next offset, reset offset, member
 * offset }.  Blob: byte_class u8[256]; next u8[C * R] (state r on class c at
 * c * R + r; state 0 is the empty set); reset u8[C] (1: F_c is the same for
 * every state); member u32[R * W] (bit q of state r's words: q in the set).
 * LX_E_TOOBIG when more than 255 sets are reachable (no guard: the scans then
 * run unguarded, exact and possibly quadratic).
 */
int lx_tokenset_liveness(const lx_tokenset *ts, void *out, uint32_t cap, uint32_t *meta, uint32_t meta_len);

/* Release a token set (NULL is a no-op).  Frees its device tables. */
void lx_tokenset_free(lx_tokenset *ts);

/*
 * lx_tokenset_scan_table -- copy the plain DFA scan table that
 * lx_lex_enumerative stages in shared memory (for host-side inspection and
 * tests): up to `cap` bytes into `out`, and meta[0..8] = {bytes, states,
 * classes, q0, next offset, accept offset, candidate-begin offset, candidate
 * offset, longest candidate list}.  Layout: class u8[256]; next u16[C*S]
 * (0xFFFF = undefined or leaving Q+; else the target state, | 0x8000 when it
 * accepts); accept u16[S] (kind | 0x8000 when not
 * discarded, 0x7FFF = not accepting); cand_begin u16[257]; cand u16[...]:
 * for byte b the ascending states delta+(q, b), q in Q+, at
 * [cand_begin[b], cand_begin[b+1]).  Returns LX_E_TOOBIG when no such table
 * was built (too large), else LX_OK.
 */
int lx_tokenset_scan_table(const lx_tokenset *ts, void *out, uint32_t cap, uint32_t *meta, uint32_t meta_len);

/*
 * lx_ctx_create -- a lexing context bound to the current CUDA device.  It owns
 * the scratch memory of lx_lex (per-tile look-back status words, a tile
 * counter and a result record), grown on demand with cudaMalloc.
 * Errors: LX_E_CUDA (no device), LX_E_NOMEM.
 */
int lx_ctx_create(lx_ctx **out);

/* Release a context (NULL is a no-op).  Synchronizes its device first. */
void lx_ctx_free(lx_ctx *ctx);

/* Bound, in milliseconds, of every device-side wait of later calls (the
 * look-back spin and the shared-memory load barrier).  Default 20000.
 * A wait that runs out makes the call return LX_E_TIMEOUT. */
int lx_ctx_set_timeout_ms(lx_ctx *ctx, uint32_t ms);

/* Kernel timing: when enabled, lx_lex (and the other lexing calls) record a
 * CUDA event pair on the stream around their kernel launches;
 * lx_ctx_last_kernel_ms returns the elapsed time of the most recent call's
 * launches (milliseconds, host out).  Off by default. */
int lx_ctx_enable_timing(lx_ctx *ctx, int on);
int lx_ctx_last_kernel_ms(lx_ctx *ctx, float *ms);

/*
 * lx_ctx_set_kernel -- which kernel lx_lex uses on this context.
 *   LX_KERNEL_AUTO (default): the warp-tile kernel (every warp owns 6144-byte
 *     tiles, event codes in the walk table) when the token set has an
 *     event-code walk table for the mode (lx_tokenset_walk_table) and d_in is
 *     16-byte aligned; the tile kernel (CTAs of 256 threads over 17408-byte
 *     tiles, per-lane token records) otherwise;
 *   LX_KERNEL_TILE: always the tile kernel;
 *   LX_KERNEL_WARP: always the warp-tile kernel; lx_lex returns LX_E_INVAL
 *     for a call it cannot serve.
 * Both produce the same stream (tests compare them).  Returns LX_E_INVAL
 * for another value.  lx_lex_host follows the same choice; lx_lex_batch
 * takes the one-launch warp-tile batch unless LX_KERNEL_TILE is set.
 */
#define LX_KERNEL_AUTO 0
#define LX_KERNEL_TILE 1
#define LX_KERNEL_WARP 2
int lx_ctx_set_kernel(lx_ctx *ctx, int kernel);

/*
 * lx_ctx_set_warps -- warps per CTA of the warp-tile kernel on this context
 * (1..20; 0 = as many as the shared-memory budget holds next to the table,
 * the default).  Each warp owns one 6144-byte tile at a time, so the setting
 * trades resident warps (latency hiding) against L1 left beside shared
 * memory.  Same tokens either way; lx_autotune chooses it.  LX_E_INVAL for a
 * value above 20.
 */
int lx_ctx_set_warps(lx_ctx *ctx, uint32_t warps);

/*
 * lx_ctx_set_warp_geometry -- the warp-tile kernel's per-warp geometry on
 * this context.
 *   LX_WARP_GEOMETRY_SPARSE: a chunk may end up to 512 bytes past its tile
 *     and 1536 kept tokens per tile are staged in shared memory;
 *   LX_WARP_GEOMETRY_DENSE: 2048 bytes and 768 staged tokens, the rest of a
 *     tile's tokens staged in global memory (for inputs whose certified
 *     bytes lie far apart, or with many kept tokens per tile);
 *   LX_WARP_GEOMETRY_AUTO (default): sparse for the first call on a token
 *     set and mode; later calls take what the previous call on them showed:
 *     dense if it kept more than 1536 tokens per tile on average, or if
 *     more than one tile in 20000 had its last chunk end past 512 bytes.
 * Same tokens either way (a chunk that ends past the halo is walked by one
 * lane, which is slow, not wrong).  LX_E_INVAL for another value.
 */
#define LX_WARP_GEOMETRY_AUTO 0
#define LX_WARP_GEOMETRY_SPARSE 1
#define LX_WARP_GEOMETRY_DENSE 2
int lx_ctx_set_warp_geometry(lx_ctx *ctx, int geometry);

/*
 * lx_ctx_debug_withhold -- failure-detection test hook.  In later lx_lex
 * calls on this context, the CTA that processes tile `tile` (17 408-byte
 * tiles) never publishes its look-back aggregate, so the bounded look-back
 * waits of its successors run out: the call returns LX_E_TIMEOUT after about
 * the context's timeout (lx_ctx_set_timeout_ms), every CTA stops claiming
 * tiles once one wait has given up, and the context stays usable.
 * 0xFFFFFFFF turns it off (the default).  No GPU fault is involved.
 */
int lx_ctx_debug_withhold(lx_ctx *ctx, uint32_t tile);

/*
 * lx_lex -- lex n bytes at d_in (device) on the context's device.
 *
 * The input is cut before occurrences of the certified bytes that `mode`
 * selects (Definition 2 or Definition 3), every chunk is scanned from q0 by
 * the longest-match loop of Section 3, and the chunk streams are concatenated
 * in order (Section 6).  By Theorem 1 (exact cuts) the result equals the
 * serial tok(w); by Theorem 3 (modulo cuts) it equals pi_I(tok(w)).
 *
 *   d_in       device, n bytes, read only.  16-byte alignment enables the
 *              bulk-copy (TMA) staging path; other alignments are accepted.
 *   mode       LX_FULL_EXACT, LX_FILTERED_EXACT or LX_FILTERED_MODULO.
 *   d_kinds    device, capacity entries: token kind of each emitted token.
 *   d_lens     device, capacity entries: its length in bytes.
 *   capacity   entries available in d_kinds / d_lens.
 *   n_tokens   host out: tokens emitted (or required, on LX_E_CAPACITY).
 *   consumed   host out: con(w), the offset after the last emitted token;
 *              < n iff the scan halts on malformed input.  The tokens
 *              returned are then exactly those before the failure
 *              (Corollary 1; with modulo cuts the same holds for
 *              pi_I: every serial token ends at or before con(w), so the
 *              one-cut argument of Theorem 3 covers every cut below it and
 *              the chunk holding con(w) halts there).
 *   stream     cudaStream_t.  The call synchronizes this stream once, to
 *              read back the 32-byte result record.
 * Errors: LX_E_INVAL, LX_E_MODE (LX_FULL_EXACT needs exact cuts: modulo
 * cuts only preserve pi_I, Theorem 3), LX_E_CAPACITY (entries beyond
 * capacity are not written), LX_E_TOOBIG, LX_E_CUDA, LX_E_TIMEOUT, LX_E_NOMEM.
 */
int lx_lex(lx_ctx *ctx, const lx_tokenset *ts, const uint8_t *d_in, uint64_t n, int mode,
           uint16_t *d_kinds, uint32_t *d_lens, uint64_t capacity, uint64_t *n_tokens,
           uint64_t *consumed, void *stream);

/*
 * lx_lex_async -- lx_lex without a host round trip: the warp-tile kernel, then
 * a one-thread kernel that writes the call's result record to *d_result
 * (device memory, caller-owned) in stream order.  Nothing synchronizes and
 * nothing falls back: chunks whose certified bytes lie far apart are walked
 * byte by byte, and backtracking carries no step budget (same tokens as
 * lx_lex, possibly slower on such inputs).  Needs the warp-tile kernel
 * (an event-code walk table for the mode and a 16-byte aligned d_in):
 * LX_E_INVAL otherwise, returned at once, like every argument error.
 * d_result->status is LX_OK, LX_E_CAPACITY, LX_E_TIMEOUT or LX_E_TOOBIG;
 * n_tokens and consumed as in lx_lex.  Calls on one context must share one
 * stream (they reuse the context's scratch in order).
 */
typedef struct {
    int32_t status;
    uint32_t reserved;
    uint64_t n_tokens;
    uint64_t consumed;
} lx_async_result;
int lx_lex_async(lx_ctx *ctx, const lx_tokenset *ts, const uint8_t *d_in, uint64_t n, int mode,
                 uint16_t *d_kinds, uint32_t *d_lens, uint64_t capacity, lx_async_result *d_result, void *stream);

/*
 * lx_lex_host -- lx_lex on HOST buffers: copies h_in to the device, lexes it
 * and copies the tokens back into h_kinds / h_lens (host, capacity entries),
 * using device buffers owned by the context.  Same results and errors as
 * lx_lex.  Inputs of 64 MiB or more with a non-empty cut set are split on the
 * host into up to 8 pieces at certified bytes (the planner of Section 6) and
 * piece copies overlap the lexing of other pieces (two context-owned copy
 * streams; the launches run in order on `stream`).  On the warp-tile kernel
 * each piece is copied to a 16-byte aligned place and lexed into its own
 * output range, and its tokens are copied out behind the previous pieces';
 * if some piece's certified bytes lie too far apart, or its backtracking
 * runs past the step budget (failed lookahead), the whole input is copied
 * in again and lexed by lx_lex's plan.  Host buffers should be pinned for
 * full copy speed.  Returns after all copies have completed.
 */
int lx_lex_host(lx_ctx *ctx, const lx_tokenset *ts, const uint8_t *h_in, uint64_t n, int mode,
                uint16_t *h_kinds, uint32_t *h_lens, uint64_t capacity, uint64_t *n_tokens,
                uint64_t *consumed, void *stream);

/*
 * Launch configuration of the tile kernel per (token set, mode), held by the
 * context (chunk targets stay 68 bytes, 256 threads per CTA):
 *   ks          -- token-end records per thread held in shared memory before
 *                  compaction / spilling (LX_KS_MIN .. LX_KS_MAX; default 40);
 *   ctas_per_sm -- resident CTAs per SM (0 = as many as fit; capped by what
 *                  fits);
 *   class_table -- 1: walk the class-indexed table even where the
 *                  byte-indexed one fits (one more lookup per byte, a far
 *                  smaller table, so more CTAs per SM).
 * Without a configuration the context takes the byte-indexed table and ks 40
 * unless the class-indexed table with some ks >= 32 fits more CTAs per SM.
 * Every configuration gives the same tokens; only speed differs.
 * lx_ctx_set_config sets one (LX_E_TOOBIG if its shared memory exceeds the
 * kernel's budget); lx_ctx_get_config reads the one in force (ms = the time
 * lx_autotune measured for it, 0 if set by hand or default).
 * lx_autotune times every ks in {24, 32, 36, 40, 48, 56, 64} on each table form,
 * with the largest and the smallest CTA count, on `d_sample` (a device buffer representative
 * of the inputs to come, n bytes; outputs go to d_kinds / d_lens), then the
 * warp-tile kernel (where it applies to the sample) at 4, 8, 12, 16 and 20
 * warps per CTA; checks that all give the same result, keeps the fastest
 * tile configuration and, for lx_lex on LX_KERNEL_AUTO, the faster kernel
 * with its warps per CTA (lx_ctx_set_warps overrides the latter; setting a
 * configuration by hand clears the choice).  Synchronizes `stream`.
 * The tile configuration also applies to lx_lex_batch groups of that token set.
 */
#define LX_KS_MIN 16u
#define LX_KS_MAX 96u
int lx_ctx_set_config(lx_ctx *ctx, const lx_tokenset *ts, int mode, uint32_t ks, uint32_t ctas_per_sm,
                      uint32_t class_table);
int lx_ctx_get_config(lx_ctx *ctx, const lx_tokenset *ts, int mode, uint32_t *ks, uint32_t *ctas_per_sm,
                      uint32_t *class_table, float *ms);
int lx_autotune(lx_ctx *ctx, const lx_tokenset *ts, int mode, const uint8_t *d_sample, uint64_t n,
                uint16_t *d_kinds, uint32_t *d_lens, uint64_t capacity, void *stream);

/*
 * lx_lex_enumerative -- lx_lex for token sets that certify no byte (the
 * paper's refused sets, Table 2, where lx_lex can only run one chunk).
 *
 * The input is split every 4096 bytes, each start placed within the first
 * 256 bytes of its target right after the byte with the fewest possible entry
 * contexts (at most 8: BOUNDARY or a state delta+(q, b) of Q+).  Every chunk
 * is scanned from every candidate context (counting kept tokens, recording
 * the context at the next start); the chain of exit contexts from BOUNDARY at
 * offset 0 then fixes each chunk's true context and output offset, and each
 * chunk is scanned once more to write its tokens.  Output and errors as
 * lx_lex: tok(w) with LX_FULL_EXACT, pi_I(tok(w)) with either filtered mode
 * (the certificates play no part), con(w) in *consumed (Corollary 1).
 * Works for any token set; LX_E_TOOBIG when its plain DFA table exceeds the
 * shared-memory budget.  Synchronizes `stream`.
 *
 * Failed-lookahead guard (Section 9): a chunk scan that takes more than
 * 32 x 4096 steps (failed lookahead repeated at successive token starts, as
 * over the tokens a, a+b and ; on a^n, or a token spanning many chunks) makes
 * the call run again with the liveness prepass (lx_liveness): every scan then
 * ends its token as soon as no accepting position lies ahead, and a chunk
 * entered inside a token that runs past its end stops there, so the work is
 * linear in n.  Same output; lx_lex takes this route too when its own
 * backtracking exceeds a budget linear in the chunk lengths.
 */
int lx_lex_enumerative(lx_ctx *ctx, const lx_tokenset *ts, const uint8_t *d_in, uint64_t n, int mode,
                       uint16_t *d_kinds, uint32_t *d_lens, uint64_t capacity, uint64_t *n_tokens,
                       uint64_t *consumed, void *stream);

/*
 * lx_liveness -- the guard's prepass on its own: the state of the liveness
 * automaton (lx_tokenset_liveness) at every offset 0..n of the device buffer
 * d_in into d_live[0..n] (device, n + 1 bytes, caller-owned; d_live[n] = 0,
 * the empty set).  The run from right to left is split into 4096-byte pieces:
 * each piece's map from its end state to its start state (runs that meet a
 * reset class merge), composed in groups and linked from offset n, then
 * every piece run from its end state.  Stream-ordered, no synchronization.
 * LX_E_TOOBIG when the token set has no liveness automaton.
 */
int lx_liveness(lx_ctx *ctx, const lx_tokenset *ts, const uint8_t *d_in, uint64_t n, uint8_t *d_live,
                void *stream);

/*
 * lx_chunk_contexts -- the chunk starts lx_lex_enumerative plans for `d_in`
 * and the true entry context of each (0..states-1: inside a token in that
 * DFA state; 0xFFFE: at a token boundary), resolved by enumeration.  One
 * entry per 4096-byte target into d_starts / d_ctx (device, cap entries;
 * offset ~0 and context 0xFFFF where a target has no start, or after a
 * lexing error); *count = number of targets (LX_E_CAPACITY if cap < count).
 * These are the labels the entry-context model is trained on.
 */
int lx_chunk_contexts(lx_ctx *ctx, const lx_tokenset *ts, const uint8_t *d_in, uint64_t n, uint64_t *d_starts,
                      uint16_t *d_ctx, uint64_t cap, uint64_t *count, void *stream);

/*
 * Entry-context model (opaque, lives on the device that created it): a
 * byte-window network over the 64 bytes around a chunk start (32 before, 32
 * after; a padding value outside the input) scoring n_contexts = states + 1
 * classes (class states = BOUNDARY): byte embedding (257 x 8), a 1D
 * convolution of 32 filters of width 5 with ReLU, max pooling by 4 (16
 * positions x 32 filters = 512 features), a hidden layer of `hidden` ReLU
 * units and a linear output (49 915 parameters for hidden 64 and the 211
 * contexts of the refused C-like set).  Every product reads BF16 weights
 * and accumulates in FP32; the FP32 master parameters are trained with AdamW
 * (beta 0.9 / 0.999, eps 1e-8, decoupled weight decay 0.01 on the
 * convolution and dense weight matrices) on mean softmax cross-entropy.
 * Predictions take the argmax over the candidate contexts of the byte before
 * the start.  Parameters are exchanged as one FP32 array in the order:
 * embedding [257][8], conv weights [32][5][8], conv bias [32], W1
 * [512][hidden] (feature u * 32 + f), b1 [hidden], W2 [hidden][n_contexts],
 * b2 [n_contexts].  Windows are u16 arrays of 64 byte values (256 = pad),
 * labels u16 class indices.
 */
typedef struct lx_model lx_model;
int lx_model_create(uint32_t n_contexts, uint32_t hidden, uint64_t seed, lx_model **out);
void lx_model_free(lx_model *m);
int lx_model_info(const lx_model *m, uint32_t *n_contexts, uint32_t *hidden, uint32_t *window, uint32_t *embed,
                  uint64_t *n_params);
int lx_model_get_params(const lx_model *m, float *host, uint64_t count);
int lx_model_set_params(lx_model *m, const float *host, uint64_t count);
/* windows around the offsets d_pos[0..count) of d_in (all device buffers) */
int lx_model_windows(const uint8_t *d_in, uint64_t n, const uint64_t *d_pos, uint32_t count, uint16_t *d_windows,
                     void *stream);
/* FP32 logits [batch][n_contexts] (device) */
int lx_model_forward(lx_model *m, const uint16_t *d_windows, uint32_t batch, float *d_logits, void *stream);
/* gradient of the mean loss w.r.t. the parameters (host, parameter order) and the loss */
int lx_model_gradient(lx_model *m, const uint16_t *d_windows, const uint16_t *d_labels, uint32_t batch,
                      float *host_grad, uint64_t count, float *loss, void *stream);
/* one AdamW step on a batch (see above); returns its loss before the step */
int lx_model_train_step(lx_model *m, const uint16_t *d_windows, const uint16_t *d_labels, uint32_t batch,
                        float lr, float *loss, void *stream);

/*
 * lx_lex_speculative -- lx_lex_enumerative with one scan per chunk: chunks
 * start where lx_lex_enumerative puts them, each is scanned from a predicted
 * entry context (the model's, or BOUNDARY with model == NULL), then rounds of
 * fix-up give every chunk its predecessor's exit context and rescan the
 * chunks whose entry changed, until the chain from offset 0 is consistent:
 * the result is exact whatever the predictions.  Same output and errors as
 * lx_lex_enumerative; LX_E_INVAL when the model does not score states + 1
 * contexts of this token set.  At most 8 fix-up rounds run (on the device,
 * with one read-back after them); chunks still unsettled then are decided by
 * the enumerative scan of lx_lex_enumerative as the judge (every chunk from
 * every candidate context, chains resolved from BOUNDARY at offset 0), after
 * which one more round rescans the chunks whose entry it changed.  stats
 * (optional): chunk targets, rounds that scanned chunks (the first, the
 * fix-up rounds that changed an entry, and the round after the judge), chunks
 * scanned again after the first round, judged = 1 when the judge ran.  Each
 * scan also stages the chunk's kept tokens in context scratch (6 bytes of
 * device memory per input byte), so that the settled chunks are copied to the
 * output rather than scanned again.
 */
typedef struct {
    uint64_t chunks;
    uint32_t rounds;
    uint32_t rescanned;
    uint64_t judged;
} lx_spec_stats;
int lx_lex_speculative(lx_ctx *ctx, const lx_tokenset *ts, lx_model *model, const uint8_t *d_in, uint64_t n,
                       int mode, uint16_t *d_kinds, uint32_t *d_lens, uint64_t capacity, uint64_t *n_tokens,
                       uint64_t *consumed, lx_spec_stats *stats, void *stream);

/*
 * lx_lex_batch -- lex many documents, each with its own token set, in one
 * graph launch (the batched form of lx_lex; the paper lexes one input, this
 * applies its method per document).
 *
 * docs[i] names a device buffer of docs[i].n bytes and the index of its
 * token set in sets[0 .. n_sets).  Every document is lexed exactly as
 * lx_lex would lex it alone (cuts at the mode's certificates of its own
 * token set, Theorems 1 and 3; failures per Corollary 1).
 * One launch (the default): the warp-tile kernel runs over the tiles of all
 * documents in their order in docs[], the class-form walk tables of all the
 * sets side by side in shared memory (their rows must share the 16-bit
 * shared-address window, about 250 rows of 256 bytes in all), each tile
 * taking its document's table; the output stream d_kinds / d_lens (capacity
 * entries) holds the documents in their order in docs[].  Long chunks are
 * walked byte by byte inside the launch (no document leaves it).  When that
 * does not apply (a set without a class-form walk table, rows beyond the
 * window, a document not 16-byte aligned, or LX_KERNEL_TILE set), documents
 * are grouped by token set: one persistent tile kernel per set runs over the
 * tiles of all that set's documents, and the stream holds the groups in set
 * order and, within a group, the documents in their order in docs[].  Either
 * way document i's tokens start at results[i].out_off.
 * results[i] (host array of n_docs) receives the output index of document
 * i's first token (out_off), its kept-token count n_tokens (tokens before
 * its first lexing error) and consumed = con(w) of the document; when
 * consumed < n, entries after out_off + n_tokens up to the next document's
 * out_off are unspecified.  *n_total is the length of the whole stream
 * (the end of the last group).  Empty documents get out_off 0, n_tokens 0,
 * consumed 0.
 *
 * The launch sequence (zeroing, descriptor upload, the per-set kernels,
 * result read-back) is captured once into a CUDA graph held by the context
 * and replayed while the batch shape (number of documents and tiles per
 * set, the sets, mode, output buffers and capacity) stays the same; the
 * descriptors themselves (buffers, lengths) may change between calls.
 *
 * Errors: LX_E_INVAL (null arguments, set index out of range, null buffer
 * for a non-empty document), LX_E_MODE, LX_E_TOOBIG, LX_E_NOMEM, LX_E_CUDA,
 * LX_E_TIMEOUT; LX_E_CAPACITY when *n_total > capacity (results[] are
 * still filled, so the caller can size the buffers and call again).
 * Synchronizes `stream` before returning.
 */
typedef struct {
    const uint8_t *data;   /* device pointer to the document's bytes       */
    uint64_t n;            /* its length in bytes                          */
    uint32_t set;          /* index of its token set in `sets`             */
    uint32_t reserved;     /* must be 0                                    */
} lx_doc;

typedef struct {
    uint64_t out_off;      /* output index of the document's first token   */
    uint64_t n_tokens;     /* kept tokens, up to its first lexing error    */
    uint64_t consumed;     /* con(w) of the document                       */
} lx_doc_result;

int lx_lex_batch(lx_ctx *ctx, const lx_tokenset *const *sets, uint32_t n_sets, const lx_doc *docs,
                 uint32_t n_docs, int mode, uint16_t *d_kinds, uint32_t *d_lens, uint64_t capacity,
                 lx_doc_result *results, uint64_t *n_total, void *stream);

/*
 * lx_lex_noalloc -- lx_lex for callers that cannot allocate memory.
 *
 * The paper has no counterpart to this entry point; it exists for library
 * users, not for the method.  Some callers must not allocate device or
 * pinned host memory on the lexing path: a service that hands all device
 * memory to its own allocator under a fixed budget, or latency-sensitive
 * code for which cudaMalloc (which can synchronize the device) is not
 * acceptable.  lx_lex needs a context whose scratch grows with cudaMalloc and
 * uploads each token set's tables to device memory on first use; this entry
 * point does neither.  It calls no cudaMalloc, cudaFree, cudaMallocHost or
 * other allocating routine.
 *
 * Scratch lives in one fixed array of LX_NOALLOC_SCRATCH_BYTES of device
 * memory, defined at file scope in the library, which every GPU that loads
 * the library holds until the process exits.  It holds the token set's walk
 * tables (copied in on each call), the result record, the tile counter and
 * one status word per 17408-byte tile; the parts that must start at zero are
 * cleared on each call.  Hence n must not exceed LX_NOALLOC_MAX_INPUT
 * (larger inputs return LX_E_INVAL before any GPU work).
 *
 * The first call on a device does a one-time set-up with that device
 * current: it looks up the array's device address and sets the kernel's
 * shared-memory attribute.  Under lazy module loading (the CUDA default)
 * that look-up may load the library's module and with it the array itself,
 * so make one warm-up call outside any allocation-sensitive region, and
 * before any stream capture.  Each call copies the token set's tables from
 * pageable host memory into the array with cudaMemcpyAsync; that copy goes
 * through driver-owned staging and is not free of host synchronization.
 * Every call uses the same array and leaves the last call's contents in it,
 * so calls that overlap on the GPU (for example on two streams at once, or
 * from two host threads) race and must be serialized by the caller.
 *
 * Arguments, results and other errors are those of lx_lex (without a
 * context; the device-wait bound is the default 20 s).  The call
 * synchronizes `stream` once to read back the 32-byte result record.
 */
#define LX_NOALLOC_SCRATCH_BYTES (512u * 1024u)
/* (LX_NOALLOC_SCRATCH_BYTES - 64 KiB of tables - 64 B) / 8 status words, 17408 bytes per tile */
#define LX_NOALLOC_MAX_INPUT (57336ull * 17408ull)
int lx_lex_noalloc(const lx_tokenset *ts, const uint8_t *d_in, uint64_t n, int mode, uint16_t *d_kinds,
                   uint32_t *d_lens, uint64_t capacity, uint64_t *n_tokens, uint64_t *consumed, void *stream);

/* Message for a status code (static string). */
const char *lx_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* LEXGPU_H */
