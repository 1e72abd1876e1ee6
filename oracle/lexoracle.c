/*
 * lexoracle.c -- plain, slow, obviously correct CPU reference for
 * certified-split lexing ("Certified Split Points for Parallel Lexing:
 * Exact and Modulo Discarded Tokens").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * bench's CPU-baseline / reference arm may load this file.  It shares no
 * code, header, table or helper with the GPU library.
 *
 * The automaton is given as a full table delta[q*256 + b] (-1 = undefined)
 * and tau[q] (-1 = not accepting), exactly the A = (Q, Sigma, delta, q0, tau)
 * of Section 3.  Every function follows the definition it cites, written
 * set-wise, with no reuse of the linear derivation of Section 6.
 *
 * Parity pins: see tests/test_oracle_*.py (worked examples of the paper,
 * brute force on tiny token sets, Python re.fullmatch cross-check).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define UNDEF (-1)

/* ---------------------------------------------------------------------- */
/* Section 3: the longest-match scanner.                                   */
/* At offset i start in q0, consume bytes while delta is defined, remember */
/* the last position (after >= 1 byte) at which tau is defined, emit that  */
/* token and restart there in q0.  With no accepting position the scan     */
/* halts at i; con(w) is the final committed offset.                       */
/* Returns the number of tokens (all of them, even beyond `cap`; only the  */
/* first `cap` are stored).                                                */
/* ---------------------------------------------------------------------- */
int64_t orc_lex(int32_t n_states, int32_t q0, const int32_t *delta, const int32_t *tau,
                const uint8_t *w, int64_t n, int32_t *kinds, int64_t *lens, int64_t cap,
                int64_t *con_out)
{
    (void)n_states;
    int64_t i = 0, count = 0;
    while (i < n) {
        int32_t q = q0;
        int64_t last = -1;
        int32_t last_kind = UNDEF;
        for (int64_t j = i; j < n; j++) {
            int32_t t = delta[(int64_t)q * 256 + w[j]];
            if (t == UNDEF)
                break;
            q = t;
            if (tau[q] != UNDEF) { /* eligible only after >= 1 byte */
                last = j + 1;
                last_kind = tau[q];
            }
        }
        if (last < 0)
            break; /* halt: no positive-length accepting prefix */
        if (count < cap) {
            kinds[count] = last_kind;
            lens[count] = last - i;
        }
        count++;
        i = last;
    }
    *con_out = i;
    return count;
}

/* Section 5: pi_I deletes every pair whose token lies in I. */
int64_t orc_filter(const int32_t *kinds, const int64_t *lens, int64_t n, const uint8_t *in_I,
                   int32_t n_kinds, int32_t *out_kinds, int64_t *out_lens)
{
    int64_t m = 0;
    for (int64_t k = 0; k < n; k++) {
        int32_t t = kinds[k];
        if (t >= 0 && t < n_kinds && in_I[t])
            continue;
        out_kinds[m] = t;
        out_lens[m] = lens[k];
        m++;
    }
    return m;
}

/* ---------------------------------------------------------------------- */
/* Section 4 / Section 5: certificates, written set-wise.                  */
/* ---------------------------------------------------------------------- */

/* Reachable states: breadth-first search from q0 over defined delta. */
static void reach_from(int32_t S, const int32_t *delta, int32_t q0, uint8_t *reach)
{
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(S > 0 ? S : 1));
    memset(reach, 0, (size_t)S);
    int32_t head = 0, tail = 0;
    reach[q0] = 1;
    queue[tail++] = q0;
    while (head < tail) {
        int32_t q = queue[head++];
        for (int b = 0; b < 256; b++) {
            int32_t t = delta[(int64_t)q * 256 + b];
            if (t != UNDEF && !reach[t]) {
                reach[t] = 1;
                queue[tail++] = t;
            }
        }
    }
    free(queue);
}

/* Co-accessible states: the least set containing every accepting state and
 * every state with a transition into the set (iterated to a fixpoint). */
static void coaccessible(int32_t S, const int32_t *delta, const int32_t *tau, uint8_t *coacc)
{
    for (int32_t q = 0; q < S; q++)
        coacc[q] = tau[q] != UNDEF;
    int changed = 1;
    while (changed) {
        changed = 0;
        for (int32_t q = 0; q < S; q++) {
            if (coacc[q])
                continue;
            for (int b = 0; b < 256; b++) {
                int32_t t = delta[(int64_t)q * 256 + b];
                if (t != UNDEF && coacc[t]) {
                    coacc[q] = 1;
                    changed = 1;
                    break;
                }
            }
        }
    }
}

/* delta+(q, b): defined when delta(q, b) is defined and lands in Q+ (Section 4);
 * only asked for q in Q+. */
static int32_t delta_plus(const int32_t *delta, const uint8_t *live, int32_t q, int b)
{
    if (!live[q])
        return UNDEF;
    int32_t t = delta[(int64_t)q * 256 + b];
    if (t == UNDEF || !live[t])
        return UNDEF;
    return t;
}

/* States reachable from q by (delta+)^* including q itself; marks into `seen`. */
static void closure_plus(int32_t S, const int32_t *delta, const uint8_t *live, int32_t q,
                         uint8_t *seen, int32_t *queue)
{
    memset(seen, 0, (size_t)S);
    int32_t head = 0, tail = 0;
    seen[q] = 1;
    queue[tail++] = q;
    while (head < tail) {
        int32_t p = queue[head++];
        for (int b = 0; b < 256; b++) {
            int32_t t = delta_plus(delta, live, p, b);
            if (t != UNDEF && !seen[t]) {
                seen[t] = 1;
                queue[tail++] = t;
            }
        }
    }
}

/*
 * Outputs (each a 256-entry 0/1 array indexed by byte):
 *   exact_raw   -- Definition 2 (certified split symbol)
 *   modulo_raw  -- Definition 3 (certified modulo I)
 *   exact_use   -- Corollary 2: exact_raw and delta+(q0, b) defined
 *   modulo_use  -- Proposition 2: modulo_raw and delta+(q0, b) defined
 * live_out[S]: membership of Q+ (reachable and co-accessible, Section 4).
 * *reentrant_out: Definition 1, (delta+)^*(q0, u) = q0 for some nonempty u.
 * If q0 is not in Q+ the token set accepts nothing and no symbol is useful.
 * in_I[n_kinds] marks the discarded kinds.
 */
int orc_certificates(int32_t S, int32_t q0, const int32_t *delta, const int32_t *tau,
                     const uint8_t *in_I, int32_t n_kinds,
                     uint8_t *exact_raw, uint8_t *modulo_raw, uint8_t *exact_use,
                     uint8_t *modulo_use, uint8_t *live_out, int32_t *reentrant_out)
{
    if (S <= 0 || q0 < 0 || q0 >= S)
        return -1;
    uint8_t *reach = (uint8_t *)malloc((size_t)S);
    uint8_t *coacc = (uint8_t *)malloc((size_t)S);
    uint8_t *live = (uint8_t *)malloc((size_t)S);
    uint8_t *seen = (uint8_t *)malloc((size_t)S);
    uint8_t *only_I = (uint8_t *)malloc((size_t)S); /* T(q) subset of I */
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)S);

    reach_from(S, delta, q0, reach);
    coaccessible(S, delta, tau, coacc);
    for (int32_t q = 0; q < S; q++)
        live[q] = reach[q] && coacc[q];
    if (live_out)
        memcpy(live_out, live, (size_t)S);

    /* Definition 1 literally: run (delta+)^* from the successors of q0 and
     * ask whether q0 comes back (a nonempty word returning to q0). */
    int reentrant = 0;
    if (live[q0]) {
        uint8_t *back = (uint8_t *)calloc((size_t)S, 1);
        int32_t head = 0, tail = 0;
        for (int b = 0; b < 256; b++) {
            int32_t t = delta_plus(delta, live, q0, b);
            if (t != UNDEF && !back[t]) {
                back[t] = 1;
                queue[tail++] = t;
            }
        }
        while (head < tail) {
            int32_t p = queue[head++];
            for (int b = 0; b < 256; b++) {
                int32_t t = delta_plus(delta, live, p, b);
                if (t != UNDEF && !back[t]) {
                    back[t] = 1;
                    queue[tail++] = t;
                }
            }
        }
        reentrant = back[q0];
        free(back);
    }
    *reentrant_out = reentrant;

    /* T(q) = { tau(p) : p in (delta+)^*(q, v) } ; only_I[q] iff T(q) subset of I. */
    for (int32_t q = 0; q < S; q++) {
        only_I[q] = 0;
        if (!live[q])
            continue;
        closure_plus(S, delta, live, q, seen, queue);
        int ok = 1;
        for (int32_t p = 0; p < S && ok; p++) {
            if (!seen[p] || tau[p] == UNDEF)
                continue;
            int32_t t = tau[p];
            if (!(t >= 0 && t < n_kinds && in_I[t]))
                ok = 0;
        }
        only_I[q] = (uint8_t)ok;
    }

    for (int b = 0; b < 256; b++) {
        int32_t d0 = delta_plus(delta, live, q0, b);
        /* Definition 2: every q in Q+ with delta+(q, b) defined is q0, and if
         * delta+(q0, b) is defined then q0 is not re-entrant. */
        int ex = 1;
        /* Definition 3: every q in Q+ with delta+(q, b) defined satisfies A(q) or C(q). */
        int mo = 1;
        for (int32_t q = 0; q < S; q++) {
            if (!live[q])
                continue;
            int32_t t = delta_plus(delta, live, q, b);
            if (t == UNDEF)
                continue;
            if (q != q0)
                ex = 0;
            int A = (q == q0) && !reentrant;
            int C = (tau[q] != UNDEF) && (d0 != UNDEF) && (d0 == t) && only_I[q];
            if (!(A || C))
                mo = 0;
        }
        if (d0 != UNDEF && reentrant)
            ex = 0;
        if (!live[q0]) { /* accepts nothing: raw conditions hold vacuously, none useful */
            ex = 1;
            mo = 1;
        }
        exact_raw[b] = (uint8_t)ex;
        modulo_raw[b] = (uint8_t)mo;
        exact_use[b] = (uint8_t)(ex && d0 != UNDEF);
        modulo_use[b] = (uint8_t)(mo && d0 != UNDEF);
    }

    free(reach);
    free(coacc);
    free(live);
    free(seen);
    free(only_I);
    free(queue);
    return 0;
}
