// internal.h -- definitions shared by the host token-set compiler
// (tokenset.cpp) and the device path (lex.cu).  Not part of the C ABI.
#pragma once

#include <cstdint>
#include <mutex>
#include <vector>

#include "lexgpu.h"

namespace lx {

// ---------------------------------------------------------------------------
// Shared-memory walk tables.
//
// The scanner of Section 3 runs as a Moore machine over "rows".  Row R[q] is
// automaton state q while a token is in progress; START is q0 at a token
// start (nothing consumed yet); E[q'] is a copy of R[q'] entered when the
// previous token ended just before the current byte and the new token moved
// q0 -> q' on it; SLOW means "the fast loop cannot decide" (backtrack to the
// last accepting position, or fail) and absorbs every byte.  Rows are ordered
//     SLOW, R[0..S-1], START, PRE, E[...]
// (PRE lets a lane begin at the word-aligned byte before its chunk start: it
// absorbs bytes outside the cut set and on a cut byte moves as START does),
// so "a token ended here" is one comparison of the row pointer with P_flag
// and "take the slow path" one equality with P_slow.  A table entry is the
// 16-bit shared-memory address of the target row (relative offsets here; the
// kernel adds the table's shared base when it stages the blob).
//
// Certified bytes are folded in: from any row but START, a byte in the cut
// set of the mode ends the token in progress (Definition 2 / 3 guarantee the
// serial scan has no accepting position past it), so every occurrence of a
// certified byte is a chunk boundary.
//
// Two physical forms:
//   byte-indexed:  256 u16 columns per row (512 B), row r's entry for byte b
//                  at column b ^ 2*sigma(r); P(r) = 512 r + 4 sigma(r), so the
//                  next address is P ^ (b << 1) -- one LOP3, and the XOR
//                  spreads equal bytes of different rows over banks.
//   class-indexed: n_classes + 1 u16 columns per row; P(r) = 2 (C+1) r; the
//                  next address is P + 2 class(b); column C holds the row's
//                  kind word.
// ---------------------------------------------------------------------------
enum TableForm : int { FORM_BYTE = 0, FORM_CLASS = 1 };

constexpr uint32_t KIND_NONE = 0x7FFFu;   // kind word: bits 0..14 kind, bit 15 kept
constexpr uint32_t KIND_KEEP = 0x8000u;
constexpr uint32_t MAX_TABLE_BYTES = 60u * 1024u;
constexpr uint32_t MAX_BYTE_FORM_BYTES = 40u * 1024u;

struct HostTable {
    int status = LX_OK;          // LX_OK, or LX_E_TOOBIG for this mode
    int form = FORM_BYTE;
    uint32_t n_rows = 0;
    uint32_t ncols = 0;          // 256 (byte form) or C + 1 (class form)
    uint32_t row_bytes = 0;
    uint32_t table_bytes = 0;    // bytes of row entries
    uint32_t p_start = 0, p_flag = 0, p_slow = 0, p_pre = 0;   // relative row pointers
    uint32_t kind_off = 0;       // byte form: u16 kind word per row
    uint32_t cmap_off = 0;       // class form: u8 class per byte
    uint32_t cert_off = 0;       // u8 per byte: 1 = cut byte in this mode
    std::vector<uint8_t> blob;   // everything above, 16-byte padded
};

// Plain DFA tables for scans entered in a context (splitting an input whose
// token set certifies no byte): the class map, the next state per (class,
// state) with targets outside Q+ made undefined (no accepting state is
// reachable from them, so the longest match is unchanged) and bit 15 set when
// the target accepts (a scan tests acceptance without a lookup), an accept word per
// state (bits 0..14 kind or KIND_NONE, bit 15 kept modulo I), and for every
// byte b the ascending list of states delta+(q, b), q in Q+ -- the mid-token
// contexts possible right after b.
//   [class u8 x 256][next u16 x C*S][accept u16 x S][cand_begin u16 x 257][cand u16 ...]
struct ScanTable {
    int status = LX_OK;          // LX_E_TOOBIG when it does not fit shared memory
    uint32_t S = 0, C = 0, q0 = 0;
    uint32_t next_off = 0, acc_off = 0, cbeg_off = 0, cand_off = 0;
    uint32_t max_cand = 0;       // longest candidate list (BOUNDARY not counted)
    std::vector<uint8_t> cand_count;   // [b]: 1 + list length (BOUNDARY counted)
    std::vector<uint8_t> blob;
};
constexpr uint16_t SCAN_NONE = 0xFFFFu;
constexpr uint16_t SCAN_ACCEPT = 0x8000u;   // next-state flag: the target state accepts

// ---------------------------------------------------------------------------
// Event-code walk tables (the warp-tile kernel, lexwarp.cu).
//
// The same scanner as above, with the token end carried by the transition
// itself: every entry is the 16-bit shared address of the target row with
// the EVENT CODE of the transition in bits 1..7 (rows start on 512- or
// 256-byte boundaries, so those bits are free).  Code 0: no token ended
// before this byte; 1: a discarded token ended; 2..127: a kept token of kind
// kind_map[code] ended.  Rows: SLOW (0), R[0..S-1], START, PRE; no E rows.
//   byte-indexed:  512-byte rows, entry of byte b at row + 2b, so the next
//                  address is (entry & ~0x1FE) | (b << 1): one LOP3;
//   class-indexed: 256-byte rows, entry of class c at row + 2c (C <= 127),
//                  with a 256-byte map cmap2[b] = 2 class(b) on a 256-byte
//                  boundary, so the map address is one PRMT and the next
//                  address (entry & ~0xFF) | cmap2[b]: one LOP3.
// Blob: [rows][acc u8 per row][kind_map u16 x 128][cmap2 u8 x 256][cut u8 x 256 x (K+1)][ctx u8 x 256].
// acc[r] is 2 * the code of the kind row r accepts (0: not accepting).
// ---------------------------------------------------------------------------
constexpr uint32_t WALK_CODES = 128;   // codes 0..127: at most 126 kept kinds
constexpr uint32_t WALK_MAX_CTX = 15;  // split-window context classes (PRE_k rows) at most
struct WalkTable {
    int status = LX_E_TOOBIG;
    int form = FORM_BYTE;
    uint32_t n_rows = 0, row_shift = 9, rows_bytes = 0;
    uint32_t p_start = 0, p_pre = 0;      // relative row addresses (SLOW is 0)
    uint32_t acc_off = 0, kmap_off = 0, cmap_off = 0, cut_off = 0;
    uint32_t n_kept = 0;                  // kept kinds (codes 2 .. n_kept + 1)
    // split windows (exact modes): K context classes; PRE_k rows follow PRE;
    // ctx map u8[256] at ctx_off (context class of a byte, 0: none); the cut
    // table at cut_off holds K + 1 rows of 256 bytes (row k: a chunk may start
    // at byte b when the byte before has context k; row 0: single bytes)
    uint32_t n_ctx = 0, ctx_off = 0;
    std::vector<uint8_t> blob;
};

// ---------------------------------------------------------------------------
// Liveness automaton: the failed-lookahead guard (Section 9, the quadratic
// pathology of longest-match scanning).
//
// Read from right to left, its state after w[k..n) is the set
//   live_k = { q in Q+ : delta+*(q, w[k..m)) accepts for some m > k },
// empty at k = n: the states from which a scan at offset k still has an
// accepting position ahead.  A scan whose state is not in live_k has already
// passed its last accepting position, so it may end its token at once; with
// that test every token costs its own length plus one step -- the table of
// failed (state, position) pairs that Reps keeps during the scan, computed
// before it.  Its states are the distinct sets reachable from the empty set;
// on class c a set X goes to F_c(X) = { q in Q+ : delta+(q, c) accepts or
// lies in X }.  A class whose F_c is the same for every state resets it.
// At most LIVE_MAX sets (one-byte ids); otherwise the guard is unavailable.
// Blob (16-byte aligned parts): byte_class u8[256] | next u8[C * R] (next of
// set r on class c at c * R + r) | reset u8[C] | member u32[R * W] (bit q of
// words r * W .. : q in set r).
// ---------------------------------------------------------------------------
constexpr uint32_t LIVE_MAX = 255;
struct LiveTable {
    int status = LX_E_TOOBIG;
    uint32_t R = 0, C = 0, S = 0, W = 0;     // sets, classes, DFA states, member words per set
    uint32_t next_off = 0, reset_off = 0, member_off = 0;
    std::vector<uint8_t> blob;
};

struct DeviceTables {
    int device = -1;
    void *d_blob[3] = {nullptr, nullptr, nullptr};
    void *d_blob_cls[3] = {nullptr, nullptr, nullptr};
    void *d_scan = nullptr;
    void *d_walk[3] = {nullptr, nullptr, nullptr};
    void *d_live = nullptr;
};

}  // namespace lx

struct lx_tokenset {
    uint64_t serial = 0;        // unique per compiled token set (cache keys)
    uint32_t n_states = 0, n_classes = 0, q0 = 0, n_kinds = 0;
    std::vector<uint8_t> byte_class;
    std::vector<uint32_t> next;       // [c * S + q]
    std::vector<uint16_t> accept;     // [q]
    std::vector<uint8_t> discard;     // [kind]
    std::vector<uint8_t> live;        // [q], Q+
    bool reentrant = false;
    uint32_t exact[8] = {0}, modulo[8] = {0};
    // two-byte split windows: win[a * 8 + (b >> 5)] bit b: a cut before b is
    // certified after a (q0 not re-entrant, delta+(q0, b) defined, and no
    // state of delta+(Q+, a) has a live transition on b)
    std::vector<uint32_t> win;
    lx::HostTable tab[3];       // per mode: byte-indexed when it fits, else class-indexed
    lx::HostTable tab_cls[3];   // per mode: class-indexed (only when tab[m] is byte-indexed)
    lx::ScanTable scan;
    lx::WalkTable walk[3];      // per mode: event-code walk table (LX_E_TOOBIG when it does not fit)
    lx::WalkTable walk_cls[3];  // per mode: its class form, when walk[m] is byte-indexed (batches)
    lx::LiveTable liveness;     // the failed-lookahead guard (LX_E_TOOBIG: unavailable)
    std::mutex mu;
    std::vector<lx::DeviceTables> dev;
};
