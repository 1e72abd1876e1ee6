// tokenset.cpp -- lx_compile_tokenset: the linear certificate derivation of
// Sections 4.1, 6 and 6.1, and the packing of the shared-memory walk tables.
// Pure host code.

#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <new>

#include "internal.h"

namespace {

using lx::HostTable;
using lx::ScanTable;

// Predecessor index over the stored (class-compressed) table: one entry per
// defined (state, class) edge, grouped by target (Section 6.1 builds it once
// per class row and reuses it for both closures).
struct PredIndex {
    std::vector<uint32_t> start;   // [S + 1]
    std::vector<uint32_t> src;     // sources, grouped by target
};

PredIndex build_pred(const lx_tokenset &t)
{
    const uint32_t S = t.n_states, C = t.n_classes;
    PredIndex pi;
    pi.start.assign(S + 1, 0);
    for (uint32_t c = 0; c < C; c++)
        for (uint32_t q = 0; q < S; q++) {
            uint32_t d = t.next[(size_t)c * S + q];
            if (d != LX_NONE) pi.start[d + 1]++;
        }
    for (uint32_t q = 0; q < S; q++) pi.start[q + 1] += pi.start[q];
    pi.src.resize(pi.start[S]);
    std::vector<uint32_t> fill(pi.start.begin(), pi.start.end() - 1);
    for (uint32_t c = 0; c < C; c++)
        for (uint32_t q = 0; q < S; q++) {
            uint32_t d = t.next[(size_t)c * S + q];
            if (d != LX_NONE) pi.src[fill[d]++] = q;
        }
    return pi;
}

// Reverse closure from `seed` states along edges accepted by `edge_ok`.
template <class EdgeOk>
std::vector<uint8_t> reverse_closure(const PredIndex &pi, std::vector<uint32_t> work,
                                     uint32_t S, EdgeOk edge_ok)
{
    std::vector<uint8_t> mark(S, 0);
    for (uint32_t q : work) mark[q] = 1;
    while (!work.empty()) {
        uint32_t t = work.back();
        work.pop_back();
        for (uint32_t k = pi.start[t]; k < pi.start[t + 1]; k++) {
            uint32_t p = pi.src[k];
            if (!mark[p] && edge_ok(p, t)) {
                mark[p] = 1;
                work.push_back(p);
            }
        }
    }
    return mark;
}

void derive_certificates(lx_tokenset &t)
{
    const uint32_t S = t.n_states, C = t.n_classes, q0 = t.q0;
    auto nx = [&](uint32_t c, uint32_t q) { return t.next[(size_t)c * S + q]; };
    PredIndex pi = build_pred(t);

    // co-accessibility: accepting states seed a worklist over predecessors
    std::vector<uint32_t> seeds;
    for (uint32_t q = 0; q < S; q++)
        if (t.accept[q] != LX_NO_KIND) seeds.push_back(q);
    std::vector<uint8_t> coacc = reverse_closure(pi, seeds, S, [](uint32_t, uint32_t) { return true; });

    // reachability: forward sweep from q0
    std::vector<uint8_t> reach(S, 0);
    std::vector<uint32_t> stack{q0};
    reach[q0] = 1;
    while (!stack.empty()) {
        uint32_t q = stack.back();
        stack.pop_back();
        for (uint32_t c = 0; c < C; c++) {
            uint32_t d = nx(c, q);
            if (d != LX_NONE && !reach[d]) {
                reach[d] = 1;
                stack.push_back(d);
            }
        }
    }
    t.live.assign(S, 0);
    for (uint32_t q = 0; q < S; q++) t.live[q] = reach[q] && coacc[q];
    const std::vector<uint8_t> &live = t.live;
    auto live_edge = [&](uint32_t c, uint32_t q) -> uint32_t {   // delta+(q, c)
        if (!live[q]) return LX_NONE;
        uint32_t d = nx(c, q);
        return (d != LX_NONE && live[d]) ? d : LX_NONE;
    };

    // re-entrancy: any live transition into q0 (the equivalent test below
    // Definition 1)
    t.reentrant = false;
    for (uint32_t c = 0; c < C && !t.reentrant; c++)
        for (uint32_t q = 0; q < S; q++)
            if (live_edge(c, q) == q0) { t.reentrant = true; break; }

    // T(q) subset of I  <=>  q not reached by the reverse closure seeded with
    // live accepting states whose kind is kept (Section 6.1)
    std::vector<uint32_t> kept;
    for (uint32_t q = 0; q < S; q++)
        if (live[q] && t.accept[q] != LX_NO_KIND && !t.discard[t.accept[q]]) kept.push_back(q);
    std::vector<uint8_t> keeps = reverse_closure(pi, kept, S, [&](uint32_t p, uint32_t d) {
        return live[p] && live[d];
    });

    std::memset(t.exact, 0, sizeof t.exact);
    std::memset(t.modulo, 0, sizeof t.modulo);
    if (!live[q0]) return;   // accepts nothing: no useful symbol
    std::vector<uint8_t> ex_c(C), mo_c(C);
    for (uint32_t c = 0; c < C; c++) {
        uint32_t d0 = live_edge(c, q0);
        bool ex = true, mo = true;
        for (uint32_t q = 0; q < S && (ex || mo); q++) {
            uint32_t d = live_edge(c, q);
            if (d == LX_NONE) continue;
            bool A = (q == q0) && !t.reentrant;
            if (!A) ex = false;
            bool Cq = t.accept[q] != LX_NO_KIND && d0 != LX_NONE && d0 == d && !keeps[q];
            if (!(A || Cq)) mo = false;
        }
        ex_c[c] = ex && d0 != LX_NONE;    // useful (Corollary 2)
        mo_c[c] = mo && d0 != LX_NONE;    // useful (Proposition 2)
    }
    for (uint32_t b = 0; b < 256; b++) {
        uint32_t c = t.byte_class[b];
        if (ex_c[c]) t.exact[b >> 5] |= 1u << (b & 31);
        if (mo_c[c]) t.modulo[b >> 5] |= 1u << (b & 31);
    }

    // two-byte split windows (a generalisation of Definition 2 with one byte
    // of left context): Z(a) = delta+(Q+, a); a cut before b after a when no
    // state of Z(a) reads b into Q+ (and b starts a token)
    t.win.assign(256 * 8, 0u);
    if (t.reentrant) return;
    std::vector<uint8_t> wc((size_t)C * C, 0);
    std::vector<uint32_t> Z;
    for (uint32_t ca = 0; ca < C; ca++) {
        Z.clear();
        std::vector<uint8_t> seen(S, 0);
        for (uint32_t q = 0; q < S; q++) {
            const uint32_t d = live_edge(ca, q);
            if (d != LX_NONE && !seen[d]) {
                seen[d] = 1;
                Z.push_back(d);
            }
        }
        for (uint32_t cb = 0; cb < C; cb++) {
            if (live_edge(cb, q0) == LX_NONE) continue;
            bool ok = true;
            for (uint32_t z : Z)
                if (live_edge(cb, z) != LX_NONE) {
                    ok = false;
                    break;
                }
            wc[(size_t)ca * C + cb] = ok ? 1 : 0;
        }
    }
    for (uint32_t a = 0; a < 256; a++)
        for (uint32_t b = 0; b < 256; b++)
            if (wc[(size_t)t.byte_class[a] * C + t.byte_class[b]]) t.win[a * 8 + (b >> 5)] |= 1u << (b & 31);
}

inline bool bit(const uint32_t m[8], uint32_t b) { return (m[b >> 5] >> (b & 31)) & 1u; }

// Walk rows (see internal.h).  target(row, class) -> row.
void build_table(const lx_tokenset &t, int mode, HostTable &ht, bool class_form)
{
    const uint32_t S = t.n_states, C = t.n_classes, q0 = t.q0;
    auto nx = [&](uint32_t c, uint32_t q) { return t.next[(size_t)c * S + q]; };
    const uint32_t *cutmask = (mode == LX_FILTERED_MODULO) ? t.modulo : t.exact;
    std::vector<uint8_t> cut_c(C, 0);
    for (uint32_t b = 0; b < 256; b++)
        if (bit(cutmask, b)) cut_c[t.byte_class[b]] = 1;

    // Row order: SLOW, R[0..S-1], START, PRE, E[...].  SLOW sits below P_flag
    // and absorbs every byte, so a lane that falls into it records nothing
    // more and can be sent to the replay lazily.  PRE lets a lane begin at the
    // aligned word before its chunk start: it absorbs bytes outside the cut
    // set and, on a cut byte, moves as START does.
    const uint32_t SLOW = 0, R0 = 1, START = S + 1, PRE = S + 2;
    std::vector<uint32_t> e_row(S, LX_NONE);
    std::vector<uint32_t> e_state;
    for (uint32_t c = 0; c < C; c++) {
        uint32_t d = nx(c, q0);
        if (d != LX_NONE && e_row[d] == LX_NONE) {
            e_row[d] = S + 3 + (uint32_t)e_state.size();
            e_state.push_back(d);
        }
    }
    const uint32_t R = S + 3 + (uint32_t)e_state.size();

    std::vector<uint32_t> tgt((size_t)R * C);
    auto state_row = [&](uint32_t row, uint32_t s) {
        for (uint32_t c = 0; c < C; c++) {
            uint32_t d0 = nx(c, q0), d = nx(c, s);
            bool acc = t.accept[s] != LX_NO_KIND;
            uint32_t r;
            if (cut_c[c]) r = acc ? e_row[d0] : SLOW;
            else if (d != LX_NONE) r = R0 + d;
            else if (acc && d0 != LX_NONE) r = e_row[d0];
            else r = SLOW;
            tgt[(size_t)row * C + c] = r;
        }
    };
    for (uint32_t s = 0; s < S; s++) state_row(R0 + s, s);
    for (uint32_t c = 0; c < C; c++) {
        uint32_t d0 = nx(c, q0);
        tgt[(size_t)START * C + c] = d0 != LX_NONE ? R0 + d0 : SLOW;
        tgt[(size_t)PRE * C + c] = cut_c[c] ? R0 + d0 : PRE;
        tgt[(size_t)SLOW * C + c] = SLOW;
    }
    for (uint32_t k = 0; k < e_state.size(); k++) state_row(S + 3 + k, e_state[k]);

    std::vector<uint16_t> kind(R, (uint16_t)lx::KIND_NONE);
    auto kind_word = [&](uint32_t s) -> uint16_t {
        uint16_t a = t.accept[s];
        if (a == LX_NO_KIND) return (uint16_t)lx::KIND_NONE;
        bool keep = (mode == LX_FULL_EXACT) || !t.discard[a];
        return (uint16_t)(a | (keep ? lx::KIND_KEEP : 0));
    };
    for (uint32_t s = 0; s < S; s++) kind[R0 + s] = kind_word(s);
    for (uint32_t k = 0; k < e_state.size(); k++) kind[S + 3 + k] = kind_word(e_state[k]);

    ht = HostTable();
    ht.n_rows = R;
    bool byte_form = !class_form && (uint64_t)R * 512 <= lx::MAX_BYTE_FORM_BYTES;
    std::vector<uint32_t> P(R);
    if (byte_form) {
        ht.form = lx::FORM_BYTE;
        ht.ncols = 256;
        ht.row_bytes = 512;
        for (uint32_t r = 0; r < R; r++) P[r] = 512 * r + 4 * (r & 31);
        ht.p_flag = 512 * (S + 3);
        ht.p_slow = P[SLOW];
    } else {
        ht.form = lx::FORM_CLASS;
        ht.ncols = C + 1;
        ht.row_bytes = 2 * (C + 1);
        for (uint32_t r = 0; r < R; r++) P[r] = ht.row_bytes * r;
        ht.p_flag = ht.row_bytes * (S + 3);
        ht.p_slow = P[SLOW];
    }
    ht.p_start = P[START];
    ht.p_pre = P[PRE];
    ht.table_bytes = R * ht.row_bytes;
    if (ht.table_bytes > lx::MAX_TABLE_BYTES) {
        ht.status = LX_E_TOOBIG;
        return;
    }
    uint32_t off = ht.table_bytes;
    if (byte_form) {
        ht.kind_off = off;
        off += 2 * R;
    }
    off = (off + 15) & ~15u;
    ht.cmap_off = off;
    off += 256;
    ht.cert_off = off;
    off += 256;
    off = (off + 15) & ~15u;
    ht.blob.assign(off, 0);
    uint16_t *ent = reinterpret_cast<uint16_t *>(ht.blob.data());
    for (uint32_t r = 0; r < R; r++) {
        if (byte_form) {
            uint32_t sig2 = 2 * (r & 31);
            for (uint32_t b = 0; b < 256; b++)
                ent[(size_t)r * 256 + (b ^ sig2)] = (uint16_t)P[tgt[(size_t)r * C + t.byte_class[b]]];
        } else {
            for (uint32_t c = 0; c < C; c++)
                ent[(size_t)r * (C + 1) + c] = (uint16_t)P[tgt[(size_t)r * C + c]];
            ent[(size_t)r * (C + 1) + C] = kind[r];
        }
    }
    if (byte_form) {
        uint16_t *kw = reinterpret_cast<uint16_t *>(ht.blob.data() + ht.kind_off);
        for (uint32_t r = 0; r < R; r++) kw[r] = kind[r];
    }
    for (uint32_t b = 0; b < 256; b++) {
        ht.blob[ht.cmap_off + b] = t.byte_class[b];
        ht.blob[ht.cert_off + b] = bit(cutmask, b) ? 1 : 0;
    }
}

// Event-code walk table (internal.h).  Same transitions as build_table
// without E rows: the token end and its kind travel in the entry.
void build_walk_table(const lx_tokenset &t, int mode, lx::WalkTable &wt, bool force_class = false)
{
    const uint32_t S = t.n_states, C = t.n_classes, q0 = t.q0;
    auto nx = [&](uint32_t c, uint32_t q) { return t.next[(size_t)c * S + q]; };
    const uint32_t *cutmask = (mode == LX_FILTERED_MODULO) ? t.modulo : t.exact;
    std::vector<uint8_t> cut_c(C, 0);
    for (uint32_t b = 0; b < 256; b++)
        if (bit(cutmask, b)) cut_c[t.byte_class[b]] = 1;
    wt = lx::WalkTable();
    // exact modes: the split windows beyond the single certified bytes, as
    // context classes (bytes whose certified followers are the same set)
    std::vector<uint32_t> ctx_of(C, 0);                  // class -> context (0: none)
    std::vector<std::vector<uint8_t>> foll(1, std::vector<uint8_t>(C, 0));   // context -> follower classes
    if (mode != LX_FILTERED_MODULO && !t.win.empty()) {
        std::vector<uint32_t> rep(C, 256);
        for (uint32_t b = 0; b < 256; b++)
            if (rep[t.byte_class[b]] == 256) rep[t.byte_class[b]] = b;
        for (uint32_t ca = 0; ca < C; ca++) {
            std::vector<uint8_t> f(C, 0);
            bool any = false;
            for (uint32_t cb = 0; cb < C; cb++) {
                const uint32_t a = rep[ca], b = rep[cb];
                f[cb] = ((t.win[a * 8 + (b >> 5)] >> (b & 31)) & 1u) && !cut_c[cb];
                any = any || f[cb];
            }
            if (!any) continue;
            uint32_t k = 1;
            while (k < foll.size() && foll[k] != f) k++;
            if (k == foll.size()) {
                if (foll.size() > lx::WALK_MAX_CTX) continue;   // more contexts than rows: this one is dropped
                foll.push_back(f);
            }
            ctx_of[ca] = k;
        }
    }
    const uint32_t K = (uint32_t)foll.size() - 1;
    // event codes: 1 for a discarded kind, 2.. for kept kinds in state order
    std::vector<uint32_t> code(t.n_kinds, 0);
    std::vector<uint16_t> kmap(lx::WALK_CODES, 0);
    uint32_t next_code = 2;
    for (uint32_t q = 0; q < S; q++) {
        const uint32_t k = t.accept[q];
        if (k == LX_NO_KIND || code[k]) continue;
        if (mode != LX_FULL_EXACT && t.discard[k]) {
            code[k] = 1;
        } else {
            if (next_code >= lx::WALK_CODES) return;   // more kept kinds than codes
            kmap[next_code] = (uint16_t)k;
            code[k] = next_code++;
        }
    }
    wt.n_kept = next_code - 2;
    const uint32_t SLOW = 0, START = S + 1, PRE = S + 2, R = S + 3 + K;   // PRE_k = PRE + k
    auto Rq = [](uint32_t q) { return 1 + q; };
    if (!force_class && (uint64_t)R * 512 <= lx::MAX_BYTE_FORM_BYTES) {
        wt.form = lx::FORM_BYTE;
        wt.row_shift = 9;
    } else if (C <= 127 && (uint64_t)R * 256 <= lx::MAX_TABLE_BYTES) {
        wt.form = lx::FORM_CLASS;
        wt.row_shift = 8;
    } else {
        return;
    }
    const uint32_t row_bytes = 1u << wt.row_shift;
    wt.n_rows = R;
    wt.rows_bytes = R * row_bytes;
    wt.p_start = START * row_bytes;
    wt.p_pre = PRE * row_bytes;
    auto entry = [&](uint32_t row, uint32_t c) -> uint16_t {
        uint32_t to = SLOW, cd = 0;
        const uint32_t d0 = nx(c, q0);
        if (row == SLOW) {
            to = SLOW;
        } else if (row == START) {
            to = d0 != LX_NONE ? Rq(d0) : SLOW;
        } else if (row >= PRE) {   // PRE_k: absorbs bytes up to a certified byte or window
            const uint32_t k = row - PRE;
            to = (cut_c[c] || foll[k][c]) ? (d0 != LX_NONE ? Rq(d0) : SLOW) : PRE + ctx_of[c];
        } else {
            const uint32_t q = row - 1, d = nx(c, q);
            const bool acc = t.accept[q] != LX_NO_KIND;
            if (cut_c[c]) {
                if (acc && d0 != LX_NONE) {
                    to = Rq(d0);
                    cd = code[t.accept[q]];
                }
            } else if (d != LX_NONE) {
                to = Rq(d);
            } else if (acc && d0 != LX_NONE) {
                to = Rq(d0);
                cd = code[t.accept[q]];
            }
        }
        return (uint16_t)((to << wt.row_shift) | (cd << 1));
    };
    auto al = [](uint32_t x, uint32_t a) { return (x + a - 1) / a * a; };
    wt.acc_off = wt.rows_bytes;
    wt.kmap_off = al(wt.acc_off + R, 16);
    wt.cmap_off = al(wt.kmap_off + 2 * lx::WALK_CODES, 256);
    wt.cut_off = wt.cmap_off + 256;
    wt.n_ctx = K;
    wt.ctx_off = wt.cut_off + 256 * (K + 1);
    wt.blob.assign(wt.ctx_off + 256, 0);
    uint16_t *ent = reinterpret_cast<uint16_t *>(wt.blob.data());
    for (uint32_t r = 0; r < R; r++) {
        if (wt.form == lx::FORM_BYTE) {
            for (uint32_t b = 0; b < 256; b++) ent[(size_t)r * 256 + b] = entry(r, t.byte_class[b]);
        } else {
            for (uint32_t c = 0; c < 128; c++) ent[(size_t)r * 128 + c] = c < C ? entry(r, c) : (uint16_t)0;
        }
        const uint32_t q = r - 1;
        if (r >= 1 && r <= S && t.accept[q] != LX_NO_KIND)
            wt.blob[wt.acc_off + r] = (uint8_t)(2 * code[t.accept[q]]);
    }
    std::memcpy(wt.blob.data() + wt.kmap_off, kmap.data(), 2 * lx::WALK_CODES);
    for (uint32_t b = 0; b < 256; b++) {
        const uint32_t c = t.byte_class[b];
        wt.blob[wt.cmap_off + b] = (uint8_t)(2 * c);
        for (uint32_t k = 0; k <= K; k++) wt.blob[wt.cut_off + 256 * k + b] = (cut_c[c] || foll[k][c]) ? 1 : 0;
        wt.blob[wt.ctx_off + b] = (uint8_t)ctx_of[c];
    }
    wt.status = LX_OK;
}

void build_scan_table(const lx_tokenset &t, ScanTable &st)
{
    const uint32_t S = t.n_states, C = t.n_classes;
    st.S = S;
    st.C = C;
    st.q0 = t.q0;
    st.cand_count.assign(256, 1);
    if (S >= lx::SCAN_ACCEPT) {   // state numbers and the accept flag share 16 bits
        st.status = LX_E_TOOBIG;
        return;
    }
    const auto &live = t.live;
    std::vector<std::vector<uint16_t>> cand(256);
    for (uint32_t b = 0; b < 256; b++) {
        const uint32_t c = t.byte_class[b];
        std::vector<uint8_t> seen(S, 0);
        for (uint32_t q = 0; q < S; q++) {
            if (!live[q]) continue;
            const uint32_t d = t.next[(size_t)c * S + q];
            if (d != LX_NONE && live[d] && !seen[d]) {
                seen[d] = 1;
                cand[b].push_back((uint16_t)d);
            }
        }
        std::sort(cand[b].begin(), cand[b].end());
        st.max_cand = std::max<uint32_t>(st.max_cand, (uint32_t)cand[b].size());
        st.cand_count[b] = (uint8_t)std::min<size_t>(255, cand[b].size() + 1);
    }
    auto al = [](uint32_t x) { return (x + 15u) & ~15u; };
    st.next_off = 256;
    st.acc_off = al(st.next_off + 2 * C * S);
    st.cbeg_off = al(st.acc_off + 2 * S);
    st.cand_off = al(st.cbeg_off + 2 * 257);
    uint32_t total = 0;
    for (auto &v : cand) total += (uint32_t)v.size();
    const uint32_t bytes = al(st.cand_off + 2 * total);
    if (bytes > lx::MAX_TABLE_BYTES || total > 0xFFFFu) {
        st.status = LX_E_TOOBIG;
        return;
    }
    st.blob.assign(bytes, 0);
    std::memcpy(st.blob.data(), t.byte_class.data(), 256);
    uint16_t *nx = reinterpret_cast<uint16_t *>(st.blob.data() + st.next_off);
    for (uint32_t c = 0; c < C; c++)
        for (uint32_t q = 0; q < S; q++) {
            const uint32_t d = t.next[(size_t)c * S + q];
            nx[(size_t)c * S + q] = (d != LX_NONE && live[d])
                                        ? (uint16_t)(d | (t.accept[d] != LX_NO_KIND ? lx::SCAN_ACCEPT : 0u))
                                        : lx::SCAN_NONE;
        }
    uint16_t *acc = reinterpret_cast<uint16_t *>(st.blob.data() + st.acc_off);
    for (uint32_t q = 0; q < S; q++) {
        const uint32_t k = t.accept[q];
        acc[q] = k == LX_NO_KIND ? (uint16_t)lx::KIND_NONE : (uint16_t)(k | (t.discard[k] ? 0u : lx::KIND_KEEP));
    }
    uint16_t *cb = reinterpret_cast<uint16_t *>(st.blob.data() + st.cbeg_off);
    uint16_t *cv = reinterpret_cast<uint16_t *>(st.blob.data() + st.cand_off);
    uint32_t o = 0;
    for (uint32_t b = 0; b < 256; b++) {
        cb[b] = (uint16_t)o;
        for (uint16_t v : cand[b]) cv[o++] = v;
    }
    cb[256] = (uint16_t)o;
}

// The liveness automaton (internal.h): breadth-first over the reachable live
// sets from the empty one, at most LIVE_MAX of them.
void build_liveness(const lx_tokenset &t, lx::LiveTable &lt)
{
    const uint32_t S = t.n_states, C = t.n_classes, W = (S + 31) / 32;
    lt.S = S;
    lt.C = C;
    lt.W = W;
    std::map<std::vector<uint32_t>, uint32_t> ids;
    std::vector<std::vector<uint32_t>> sets;
    std::vector<uint8_t> nxt;   // [r * C + c] while building
    sets.emplace_back(W, 0u);
    ids[sets[0]] = 0;
    for (uint32_t r = 0; r < sets.size(); r++) {
        for (uint32_t c = 0; c < C; c++) {
            std::vector<uint32_t> y(W, 0u);
            for (uint32_t q = 0; q < S; q++) {
                if (!t.live[q]) continue;
                const uint32_t d = t.next[(size_t)c * S + q];
                if (d == LX_NONE || !t.live[d]) continue;
                if (t.accept[d] != LX_NO_KIND || ((sets[r][d >> 5] >> (d & 31)) & 1u)) y[q >> 5] |= 1u << (q & 31);
            }
            auto it = ids.find(y);
            uint32_t id;
            if (it != ids.end()) {
                id = it->second;
            } else {
                if (sets.size() >= lx::LIVE_MAX) return;   // too many: no guard
                id = (uint32_t)sets.size();
                ids.emplace(y, id);
                sets.push_back(std::move(y));
            }
            nxt.push_back((uint8_t)id);
        }
    }
    const uint32_t R = (uint32_t)sets.size();
    auto al = [](uint32_t x) { return (x + 15u) & ~15u; };
    lt.R = R;
    lt.next_off = 256;
    lt.reset_off = al(lt.next_off + C * R);
    lt.member_off = al(lt.reset_off + C);
    lt.blob.assign(al(lt.member_off + 4 * R * W), 0);
    std::memcpy(lt.blob.data(), t.byte_class.data(), 256);
    for (uint32_t c = 0; c < C; c++) {
        bool same = true;
        for (uint32_t r = 0; r < R; r++) {
            lt.blob[lt.next_off + c * R + r] = nxt[(size_t)r * C + c];
            same = same && nxt[(size_t)r * C + c] == nxt[c];
        }
        lt.blob[lt.reset_off + c] = same ? 1 : 0;
    }
    uint32_t *mem = reinterpret_cast<uint32_t *>(lt.blob.data() + lt.member_off);
    for (uint32_t r = 0; r < R; r++)
        for (uint32_t w = 0; w < W; w++) mem[r * W + w] = sets[r][w];
    lt.status = LX_OK;
}

}  // namespace

extern "C" int lx_compile_tokenset(const lx_dfa *dfa, const uint16_t *discarded,
                                   uint32_t n_discarded, lx_tokenset **out)
{
    if (!dfa || !out) return LX_E_INVAL;
    *out = nullptr;
    const uint32_t S = dfa->n_states, C = dfa->n_classes;
    if (S == 0 || S > (1u << 20) || C == 0 || C > 256 || dfa->q0 >= S || dfa->n_kinds == 0 ||
        dfa->n_kinds > 32767 || !dfa->byte_class || !dfa->next || !dfa->accept_kind)
        return LX_E_INVAL;
    if (n_discarded && !discarded) return LX_E_INVAL;
    for (uint32_t b = 0; b < 256; b++)
        if (dfa->byte_class[b] >= C) return LX_E_INVAL;
    for (size_t k = 0; k < (size_t)S * C; k++)
        if (dfa->next[k] != LX_NONE && dfa->next[k] >= S) return LX_E_INVAL;
    for (uint32_t q = 0; q < S; q++)
        if (dfa->accept_kind[q] != LX_NO_KIND && dfa->accept_kind[q] >= dfa->n_kinds) return LX_E_INVAL;
    for (uint32_t k = 0; k < n_discarded; k++)
        if (discarded[k] >= dfa->n_kinds) return LX_E_INVAL;

    lx_tokenset *t = new (std::nothrow) lx_tokenset();
    if (!t) return LX_E_NOMEM;
    static std::atomic<uint64_t> next_serial{1};
    t->serial = next_serial++;
    try {
        t->n_states = S;
        t->n_classes = C;
        t->q0 = dfa->q0;
        t->n_kinds = dfa->n_kinds;
        t->byte_class.assign(dfa->byte_class, dfa->byte_class + 256);
        t->next.assign(dfa->next, dfa->next + (size_t)S * C);
        t->accept.assign(dfa->accept_kind, dfa->accept_kind + S);
        t->discard.assign(dfa->n_kinds, 0);
        for (uint32_t k = 0; k < n_discarded; k++) t->discard[discarded[k]] = 1;
        derive_certificates(*t);
        for (int m = 0; m < 3; m++) {
            build_table(*t, m, t->tab[m], false);
            // the class-indexed form as well when the default is byte-indexed:
            // far smaller, so more CTAs fit per SM
            if (t->tab[m].form == lx::FORM_BYTE) build_table(*t, m, t->tab_cls[m], true);
            build_walk_table(*t, m, t->walk[m]);
            // the class form as well, for batches that hold several tables
            if (t->walk[m].status == LX_OK && t->walk[m].form == lx::FORM_BYTE)
                build_walk_table(*t, m, t->walk_cls[m], true);
        }
        build_scan_table(*t, t->scan);
        build_liveness(*t, t->liveness);
    } catch (const std::bad_alloc &) {
        delete t;
        return LX_E_NOMEM;
    }
    *out = t;
    return LX_OK;
}

// Framing at the producer (Section 7.1): the reserved byte gets a rule of its
// own -- a new kind n_kinds, one byte long, from q0 -- and no other token
// admits it at any position, so its only live consumption is from q0.
extern "C" int lx_compile_tokenset_framed(const lx_dfa *dfa, const uint16_t *discarded, uint32_t n_discarded,
                                          uint32_t frame_byte, int frame_discarded, lx_tokenset **out)
{
    if (!dfa || !out || frame_byte > 255 || !dfa->byte_class || !dfa->next || !dfa->accept_kind) return LX_E_INVAL;
    const uint32_t S = dfa->n_states, C = dfa->n_classes;
    if (S == 0 || S >= (1u << 20) || C == 0 || C > 256 || dfa->q0 >= S || dfa->n_kinds >= 32767 ||
        (n_discarded && !discarded))
        return LX_E_INVAL;
    const uint32_t cr = dfa->byte_class[frame_byte];
    if (cr >= C) return LX_E_INVAL;
    uint32_t share = 0;   // other bytes in the reserved byte's class
    for (uint32_t b = 0; b < 256; b++) share += (b != frame_byte && dfa->byte_class[b] == cr);
    const uint32_t C2 = share ? C + 1 : C, c_new = share ? C : cr, F = S;   // F: the new accepting state
    if (C2 > 256) return LX_E_INVAL;
    try {
        std::vector<uint8_t> cls(dfa->byte_class, dfa->byte_class + 256);
        cls[frame_byte] = (uint8_t)c_new;
        std::vector<uint32_t> nx((size_t)C2 * (S + 1), LX_NONE);
        for (uint32_t c = 0; c < C; c++)
            for (uint32_t q = 0; q < S; q++)
                if (c != c_new) nx[(size_t)c * (S + 1) + q] = dfa->next[(size_t)c * S + q];
        nx[(size_t)c_new * (S + 1) + dfa->q0] = F;   // the frame token; every other state rejects the byte
        std::vector<uint16_t> acc(dfa->accept_kind, dfa->accept_kind + S);
        acc.push_back((uint16_t)dfa->n_kinds);
        std::vector<uint16_t> disc(discarded, discarded + n_discarded);
        if (frame_discarded) disc.push_back((uint16_t)dfa->n_kinds);
        lx_dfa d{S + 1, C2, dfa->q0, dfa->n_kinds + 1, cls.data(), nx.data(), acc.data()};
        return lx_compile_tokenset(&d, disc.empty() ? nullptr : disc.data(), (uint32_t)disc.size(), out);
    } catch (const std::bad_alloc &) {
        return LX_E_NOMEM;
    }
}

extern "C" int lx_certificates(const lx_tokenset *ts, uint32_t exact_useful[8], uint32_t modulo_useful[8])
{
    if (!ts) return LX_E_INVAL;
    if (exact_useful) std::memcpy(exact_useful, ts->exact, sizeof ts->exact);
    if (modulo_useful) std::memcpy(modulo_useful, ts->modulo, sizeof ts->modulo);
    return LX_OK;
}

extern "C" int lx_tokenset_info(const lx_tokenset *ts, int mode, uint32_t *n_states, uint32_t *n_live,
                                int *reentrant, int *table_form, uint32_t *table_rows)
{
    if (!ts || mode < 0 || mode > 2) return LX_E_INVAL;
    if (n_states) *n_states = ts->n_states;
    if (n_live) *n_live = (uint32_t)std::count(ts->live.begin(), ts->live.end(), (uint8_t)1);
    if (reentrant) *reentrant = ts->reentrant ? 1 : 0;
    if (table_form) *table_form = ts->tab[mode].form;
    if (table_rows) *table_rows = ts->tab[mode].n_rows;
    return ts->tab[mode].status;
}

static int table_out(const HostTable &h, void *out, uint32_t cap, uint32_t *meta, uint32_t meta_len);

extern "C" int lx_tokenset_table(const lx_tokenset *ts, int mode, void *out, uint32_t cap, uint32_t *meta,
                                 uint32_t meta_len)
{
    if (!ts || mode < 0 || mode > 2) return LX_E_INVAL;
    return table_out(ts->tab[mode], out, cap, meta, meta_len);
}

extern "C" int lx_tokenset_class_table(const lx_tokenset *ts, int mode, void *out, uint32_t cap, uint32_t *meta,
                                       uint32_t meta_len)
{
    if (!ts || mode < 0 || mode > 2) return LX_E_INVAL;
    const bool own = ts->tab_cls[mode].status == LX_OK && !ts->tab_cls[mode].blob.empty();
    return table_out(own ? ts->tab_cls[mode] : ts->tab[mode], out, cap, meta, meta_len);
}

static int table_out(const HostTable &h, void *out, uint32_t cap, uint32_t *meta, uint32_t meta_len)
{
    if (out && cap) std::memcpy(out, h.blob.data(), std::min<size_t>(cap, h.blob.size()));
    const uint32_t m[12] = {(uint32_t)h.blob.size(), (uint32_t)h.form, h.n_rows, h.ncols, h.row_bytes,
                            h.table_bytes, h.p_start, h.p_flag, h.p_slow, h.kind_off | (h.cmap_off << 16),
                            h.cert_off, h.p_pre};
    if (meta) std::memcpy(meta, m, sizeof(uint32_t) * std::min<uint32_t>(meta_len, 12));
    return h.status;
}

extern "C" int lx_tokenset_walk_table(const lx_tokenset *ts, int mode, void *out, uint32_t cap, uint32_t *meta,
                                      uint32_t meta_len)
{
    if (!ts || mode < 0 || mode > 2) return LX_E_INVAL;
    const lx::WalkTable &w = ts->walk[mode];
    if (out && cap) std::memcpy(out, w.blob.data(), std::min<size_t>(cap, w.blob.size()));
    const uint32_t m[12] = {(uint32_t)w.blob.size(), (uint32_t)w.form, w.n_rows, w.row_shift, w.p_start,
                            w.p_pre, w.acc_off, w.kmap_off, w.cmap_off, w.cut_off, w.n_ctx, w.ctx_off};
    if (meta) std::memcpy(meta, m, sizeof(uint32_t) * std::min<uint32_t>(meta_len, 12));
    return w.status;
}

extern "C" int lx_window_certificates(const lx_tokenset *ts, uint32_t *pairs)
{
    if (!ts || !pairs) return LX_E_INVAL;
    if (ts->win.size() == 256 * 8) std::memcpy(pairs, ts->win.data(), sizeof(uint32_t) * 256 * 8);
    else std::memset(pairs, 0, sizeof(uint32_t) * 256 * 8);
    return LX_OK;
}

extern "C" int lx_tokenset_liveness(const lx_tokenset *ts, void *out, uint32_t cap, uint32_t *meta,
                                    uint32_t meta_len)
{
    if (!ts) return LX_E_INVAL;
    const lx::LiveTable &lt = ts->liveness;
    if (out && cap) std::memcpy(out, lt.blob.data(), std::min<size_t>(cap, lt.blob.size()));
    const uint32_t m[8] = {(uint32_t)lt.blob.size(), lt.R, lt.C, lt.S, lt.W, lt.next_off, lt.reset_off, lt.member_off};
    if (meta) std::memcpy(meta, m, sizeof(uint32_t) * std::min<uint32_t>(meta_len, 8));
    return lt.status;
}

extern "C" int lx_tokenset_scan_table(const lx_tokenset *ts, void *out, uint32_t cap, uint32_t *meta,
                                      uint32_t meta_len)
{
    if (!ts) return LX_E_INVAL;
    const lx::ScanTable &st = ts->scan;
    if (out && cap) std::memcpy(out, st.blob.data(), std::min<size_t>(cap, st.blob.size()));
    const uint32_t m[9] = {(uint32_t)st.blob.size(), st.S, st.C, st.q0, st.next_off, st.acc_off,
                           st.cbeg_off, st.cand_off, st.max_cand};
    if (meta) std::memcpy(meta, m, sizeof(uint32_t) * std::min<uint32_t>(meta_len, 9));
    return st.status;
}
