/*
 * corpus.c -- seeded synthetic corpora for the lexing workloads.
 *
 * Part of the input generators: it writes bytes only and holds none of the
 * lexing method.  Every generator is deterministic for a given seed and size
 * on any host: integer RNG (xoshiro256**), no libm, and the floating-point
 * helpers below use only + - * / (compile with -ffp-contract=off).
 *
 *   gen_arith   identifiers, integers, operators, parens, ';', space runs, newlines
 *   gen_json    newline-delimited nested JSON values (depth <= 8)
 *   gen_clike   C-like statement lines (strings, chars, '//' comments, operators)
 *   gen_clike_block  gen_clike plus multi-line block comments and strings
 *
 * Each returns the number of bytes written (always exactly n).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------- RNG ---------------- */
typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix(uint64_t *x)
{
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static void rng_seed(rng_t *r, uint64_t seed)
{
    for (int i = 0; i < 4; i++) r->s[i] = splitmix(&seed);
}
static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static uint64_t next64(rng_t *r)
{
    uint64_t *s = r->s;
    uint64_t res = rotl(s[1] * 5, 7) * 9, t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3]; s[2] ^= t; s[3] = rotl(s[3], 45);
    return res;
}
static uint32_t below(rng_t *r, uint32_t n) { return (uint32_t)((next64(r) >> 32) * (uint64_t)n >> 32); }
static double unif(rng_t *r) { return (double)(next64(r) >> 11) * (1.0 / 9007199254740992.0); }
static int chance(rng_t *r, double p) { return unif(r) < p; }

/* Geometric on {0,1,...} with mean m. */
static uint32_t geom(rng_t *r, double mean)
{
    double p = 1.0 / (1.0 + mean);
    uint32_t k = 0;
    while (!chance(r, p) && k < 4096) k++;
    return k;
}

/* exp(x) from range reduction and a Taylor polynomial, + - * / only. */
static double det_exp(double x)
{
    const double LN2 = 0.69314718055994530942;
    int k = 0;
    while (x > 0.5 * LN2) { x -= LN2; k++; }
    while (x < -0.5 * LN2) { x += LN2; k--; }
    double term = 1.0, sum = 1.0;
    for (int i = 1; i < 20; i++) { term = term * x / (double)i; sum += term; }
    while (k > 0) { sum *= 2.0; k--; }
    while (k < 0) { sum *= 0.5; k++; }
    return sum;
}
/* Approximately standard normal (Irwin-Hall, 12 uniforms). */
static double normal(rng_t *r)
{
    double s = 0;
    for (int i = 0; i < 12; i++) s += unif(r);
    return s - 6.0;
}
static uint32_t lognormal_len(rng_t *r, double median, double sigma, uint32_t lo, uint32_t hi)
{
    double v = median * det_exp(sigma * normal(r));
    uint32_t L = (uint32_t)(v + 0.5);
    if (L < lo) L = lo;
    if (L > hi) L = hi;
    return L;
}

/* ---------------- byte sink ---------------- */
typedef struct { uint8_t *p; uint64_t n, cap; int full; } sink_t;
static void put(sink_t *s, uint8_t c)
{
    if (s->n < s->cap) s->p[s->n++] = c; else s->full = 1;
}
static void puts_(sink_t *s, const char *t) { while (*t) put(s, (uint8_t)*t++); }

static const uint8_t LOWER[] = "abcdefghijklmnopqrstuvwxyz";
static const char ALNUM[] = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ0123456789";
static const char HEX[] = "0123456789abcdefABCDEF";

/* =============================== arith =============================== */
/* Kinds uniform over the 13 kinds of the arith token set; identifier and
 * integer lengths 1 + Geom (mean 6 total); space runs 1 + Geom(p = 0.5). */
uint64_t gen_arith(uint64_t seed, uint8_t *out, uint64_t n)
{
    rng_t r; rng_seed(&r, seed);
    sink_t s = {out, 0, n, 0};
    static const char *ops[] = {"+", "-", "*", "/", "=", "==", "(", ")", ";"};
    while (s.n < n) {
        uint32_t k = below(&r, 13);
        if (k == 0) {
            uint32_t L = 1 + geom(&r, 5.0);
            put(&s, (uint8_t)(chance(&r, 0.1) ? '_' : LOWER[below(&r, 26)]));
            for (uint32_t i = 1; i < L; i++) {
                uint32_t c = below(&r, 37);
                put(&s, (uint8_t)(c < 26 ? LOWER[c] : c < 36 ? '0' + (c - 26) : '_'));
            }
        } else if (k == 1) {
            uint32_t L = 1 + geom(&r, 5.0);
            for (uint32_t i = 0; i < L; i++) put(&s, (uint8_t)('0' + below(&r, 10)));
        } else if (k <= 10) {
            puts_(&s, ops[k - 2]);
        } else if (k == 11) {
            uint32_t L = 1 + geom(&r, 1.0);
            for (uint32_t i = 0; i < L; i++) put(&s, ' ');
        } else {
            put(&s, '\n');
        }
    }
    return s.n;
}

/* =============================== JSON =============================== */
typedef struct { rng_t *r; sink_t *s; } jctx;

static void json_string(jctx *c, double median)
{
    rng_t *r = c->r;
    uint32_t L = lognormal_len(r, median, 0.75, 0, 4096);
    int with_escape = chance(r, 0.20);
    uint32_t esc_at = with_escape ? below(r, L + 1) : 0xFFFFFFFFu;
    put(c->s, '"');
    for (uint32_t i = 0; i <= L; i++) {
        if (i == esc_at) {
            uint32_t e = below(r, 3);
            if (e == 0) puts_(c->s, "\\\"");
            else if (e == 1) puts_(c->s, "\\\\");
            else {
                puts_(c->s, "\\u");
                for (int h = 0; h < 4; h++) put(c->s, (uint8_t)HEX[below(r, 22)]);
            }
        }
        if (i == L) break;
        uint32_t q = below(r, 100);
        if (q < 12) put(c->s, ' ');
        else if (q < 90) put(c->s, (uint8_t)ALNUM[below(r, 62)]);
        else {
            static const char P[] = "!#$%&'()*+,-./:;<=>?@[]^_`{|}~";
            put(c->s, (uint8_t)P[below(r, sizeof(P) - 1)]);
        }
    }
    put(c->s, '"');
}

static void json_number(jctx *c)
{
    rng_t *r = c->r;
    if (chance(r, 0.3)) put(c->s, '-');
    if (chance(r, 0.1)) put(c->s, '0');
    else {
        uint32_t L = 1 + geom(r, 3.0);
        put(c->s, (uint8_t)('1' + below(r, 9)));
        for (uint32_t i = 1; i < L; i++) put(c->s, (uint8_t)('0' + below(r, 10)));
    }
    if (chance(r, 0.35)) {
        put(c->s, '.');
        uint32_t L = 1 + geom(r, 3.0);
        for (uint32_t i = 0; i < L; i++) put(c->s, (uint8_t)('0' + below(r, 10)));
    }
    if (chance(r, 0.15)) {
        put(c->s, chance(r, 0.5) ? 'e' : 'E');
        uint32_t sg = below(r, 3);
        if (sg == 1) put(c->s, '+');
        if (sg == 2) put(c->s, '-');
        uint32_t L = 1 + geom(r, 1.0);
        for (uint32_t i = 0; i < L; i++) put(c->s, (uint8_t)('0' + below(r, 10)));
    }
}

static void json_newline(jctx *c)
{
    /* mostly '\n'; a few CRLF and tab-indented lines keep \r and \t in play */
    uint32_t q = below(c->r, 100);
    if (q < 2) puts_(c->s, "\r\n");
    else put(c->s, '\n');
    if (q == 2) put(c->s, '\t');
}

static void json_value(jctx *c, int depth)
{
    rng_t *r = c->r;
    double p_container = depth >= 8 ? 0.0 : (depth == 0 ? 1.0 : 0.42 / (double)(depth + 1));
    if (c->s->full) return;
    if (chance(r, p_container)) {
        int obj = chance(r, 0.65);
        put(c->s, obj ? '{' : '[');
        json_newline(c);
        uint32_t m = 1 + geom(r, depth == 0 ? 6.0 : 3.0);
        if (chance(r, 0.05)) m = 0;
        for (uint32_t i = 0; i < m; i++) {
            if (obj) {
                json_string(c, 8.0);
                puts_(c->s, chance(r, 0.8) ? ": " : ":");
            }
            json_value(c, depth + 1);
            if (i + 1 < m) put(c->s, ',');
            json_newline(c);
        }
        put(c->s, obj ? '}' : ']');
        return;
    }
    uint32_t q = below(r, 100);
    if (q < 50) json_string(c, 12.0);
    else if (q < 85) json_number(c);
    else if (q < 92) puts_(c->s, chance(r, 0.5) ? "true" : "false");
    else puts_(c->s, "null");
}

/* A stream of top-level values, each followed by a newline; the tail that no
 * further whole value fits into is padded with newlines to exactly n bytes. */
uint64_t gen_json(uint64_t seed, uint8_t *out, uint64_t n)
{
    rng_t r; rng_seed(&r, seed);
    uint64_t tmp_cap = 4u << 20;
    uint8_t *tmp = (uint8_t *)malloc(tmp_cap);
    uint64_t pos = 0;
    for (;;) {
        sink_t s = {tmp, 0, tmp_cap, 0};
        jctx c = {&r, &s};
        json_value(&c, 0);
        put(&s, '\n');
        if (s.full) continue; /* discard oversize values */
        if (pos + s.n > n) break;
        memcpy(out + pos, tmp, s.n);
        pos += s.n;
    }
    while (pos < n) out[pos++] = '\n';
    free(tmp);
    return pos;
}

/* =============================== C-like =============================== */
static const char *KW_TYPES[] = {"int", "char", "long", "short", "unsigned", "signed", "float",
                                 "double", "void", "const", "static", "extern", "register",
                                 "volatile", "auto"};
static const char *BINOPS[] = {"+", "-", "*", "/", "%", "<<", ">>", "<", ">", "<=", ">=", "==",
                               "!=", "&", "^", "|", "&&", "||"};
static const char *ASSIGNOPS[] = {"=", "*=", "/=", "%=", "+=", "-=", "<<=", ">>=", "&=", "^=", "|="};

typedef struct { rng_t *r; sink_t *s; int block; } cctx;

static void c_ident(cctx *c)
{
    rng_t *r = c->r;
    uint32_t L = lognormal_len(r, 5.0, 0.6, 1, 40);
    static const char FIRST[] = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ_";
    static const char REST[] = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ_0123456789";
    put(c->s, (uint8_t)FIRST[below(r, sizeof(FIRST) - 1)]);
    for (uint32_t i = 1; i < L; i++) put(c->s, (uint8_t)REST[below(r, sizeof(REST) - 1)]);
}

static void c_string_body(cctx *c, uint32_t L, char quote)
{
    rng_t *r = c->r;
    for (uint32_t i = 0; i < L; i++) {
        uint32_t q = below(r, 100);
        if (q < 5) {
            static const char E[] = "ntr0\\\"'a";
            put(c->s, '\\');
            put(c->s, (uint8_t)E[below(r, sizeof(E) - 1)]);
        } else if (q < 18) put(c->s, ' ');
        else if (q < 88) put(c->s, (uint8_t)ALNUM[below(r, 62)]);
        else {
            static const char P[] = "!#$%&()*+,-./:;<=>?@[]^_`{|}~";
            char ch = P[below(r, sizeof(P) - 1)];
            put(c->s, (uint8_t)ch);
        }
        (void)quote;
    }
}

static void c_literal(cctx *c)
{
    rng_t *r = c->r;
    uint32_t q = below(r, 100);
    if (q < 40) {
        uint32_t L = 1 + geom(r, 2.0);
        for (uint32_t i = 0; i < L; i++) put(c->s, (uint8_t)('0' + below(r, 10)));
    } else if (q < 55) {
        puts_(c->s, chance(r, 0.5) ? "0x" : "0X");
        uint32_t L = 1 + geom(r, 3.0);
        for (uint32_t i = 0; i < L; i++) put(c->s, (uint8_t)HEX[below(r, 22)]);
    } else if (q < 70) {
        uint32_t L = 1 + geom(r, 1.0);
        for (uint32_t i = 0; i < L; i++) put(c->s, (uint8_t)('0' + below(r, 10)));
        put(c->s, '.');
        L = geom(r, 2.0);
        for (uint32_t i = 0; i < L; i++) put(c->s, (uint8_t)('0' + below(r, 10)));
        if (chance(r, 0.3)) {
            put(c->s, 'e');
            if (chance(r, 0.5)) put(c->s, '-');
            put(c->s, (uint8_t)('1' + below(r, 9)));
        }
    } else if (q < 88) {
        put(c->s, '"');
        c_string_body(c, lognormal_len(r, 10.0, 0.7, 0, 200), '"');
        if (c->block && chance(r, 0.04)) { /* a string spanning a line */
            put(c->s, '\n');
            c_string_body(c, lognormal_len(r, 10.0, 0.7, 0, 200), '"');
        }
        put(c->s, '"');
    } else {
        put(c->s, '\'');
        if (chance(r, 0.3)) {
            put(c->s, '\\');
            put(c->s, (uint8_t)"ntr0\\'"[below(r, 6)]);
        } else put(c->s, (uint8_t)ALNUM[below(r, 62)]);
        put(c->s, '\'');
    }
}

static void c_expr(cctx *c, int depth)
{
    rng_t *r = c->r;
    uint32_t q = below(r, 100);
    if (depth > 2 || q < 35) {
        if (chance(r, 0.55)) c_ident(c); else c_literal(c);
    } else if (q < 65) {
        c_expr(c, depth + 1);
        if (chance(r, 0.8)) put(c->s, ' ');
        const char *op = BINOPS[below(r, sizeof(BINOPS) / sizeof(BINOPS[0]))];
        puts_(c->s, op);
        /* with block comments, '/' directly before a unary '*' would open one */
        if (chance(r, 0.8) || (c->block && op[0] == '/')) put(c->s, ' ');
        c_expr(c, depth + 1);
    } else if (q < 75) {
        put(c->s, '(');
        c_expr(c, depth + 1);
        put(c->s, ')');
    } else if (q < 85) {
        c_ident(c);
        put(c->s, '(');
        uint32_t m = geom(r, 1.5);
        for (uint32_t i = 0; i < m; i++) {
            if (i) puts_(c->s, ", ");
            c_expr(c, depth + 1);
        }
        put(c->s, ')');
    } else if (q < 92) {
        c_ident(c);
        uint32_t k = below(r, 3);
        if (k == 0) { put(c->s, '['); c_expr(c, depth + 1); put(c->s, ']'); }
        else if (k == 1) { puts_(c->s, "->"); c_ident(c); }
        else { put(c->s, '.'); c_ident(c); }
    } else {
        static const char *UN[] = {"!", "~", "-", "++", "--", "*", "&"};
        puts_(c->s, UN[below(r, 7)]);
        c_ident(c);
    }
}

static void c_line(cctx *c, int *indent)
{
    rng_t *r = c->r;
    for (int i = 0; i < *indent; i++) put(c->s, ' ');
    uint32_t q = below(r, 100);
    if (q < 22) {
        puts_(c->s, KW_TYPES[below(r, sizeof(KW_TYPES) / sizeof(KW_TYPES[0]))]);
        put(c->s, ' ');
        if (chance(r, 0.2)) put(c->s, '*');
        c_ident(c);
        if (chance(r, 0.7)) { puts_(c->s, " = "); c_expr(c, 0); }
        put(c->s, ';');
    } else if (q < 50) {
        c_ident(c);
        put(c->s, ' ');
        puts_(c->s, ASSIGNOPS[below(r, sizeof(ASSIGNOPS) / sizeof(ASSIGNOPS[0]))]);
        put(c->s, ' ');
        c_expr(c, 0);
        put(c->s, ';');
    } else if (q < 62) {
        c_ident(c);
        put(c->s, '(');
        uint32_t m = geom(r, 2.0);
        for (uint32_t i = 0; i < m; i++) {
            if (i) puts_(c->s, ", ");
            c_expr(c, 1);
        }
        puts_(c->s, ");");
    } else if (q < 74 && *indent < 16) {
        uint32_t k = below(r, 4);
        if (k == 0) { puts_(c->s, "if ("); c_expr(c, 0); puts_(c->s, ") {"); }
        else if (k == 1) { puts_(c->s, "while ("); c_expr(c, 0); puts_(c->s, ") {"); }
        else if (k == 2) {
            puts_(c->s, "for ("); c_ident(c); puts_(c->s, " = 0; "); c_expr(c, 1);
            puts_(c->s, "; ++"); c_ident(c); puts_(c->s, ") {");
        } else { puts_(c->s, "switch ("); c_ident(c); puts_(c->s, ") {"); }
        *indent += 4;
    } else if (q < 86 && *indent >= 4) {
        *indent -= 4;
        /* undo the indentation already written for this line */
        c->s->n -= (c->s->n >= 4 ? 4 : c->s->n);
        puts_(c->s, chance(r, 0.2) ? "} else {" : "}");
        if (c->s->p[c->s->n - 1] == '{') *indent += 4;
    } else {
        static const char *J[] = {"return ", "break;", "continue;", "goto ", "case 1:", "default:"};
        uint32_t k = below(r, 6);
        puts_(c->s, J[k]);
        if (k == 0) { c_expr(c, 0); put(c->s, ';'); }
        if (k == 3) { c_ident(c); put(c->s, ';'); }
    }
    if (chance(r, 0.10)) {
        puts_(c->s, " // ");
        c_string_body(c, lognormal_len(r, 14.0, 0.6, 0, 120), 0);
    }
    put(c->s, '\n');
}

static void c_block_comment(cctx *c)
{
    rng_t *r = c->r;
    uint32_t lines = 1 + geom(r, 3.0);
    puts_(c->s, "/*");
    for (uint32_t i = 0; i < lines; i++) {
        put(c->s, ' ');
        uint32_t L = lognormal_len(r, 30.0, 0.5, 0, 200);
        for (uint32_t k = 0; k < L; k++) {
            uint32_t q = below(r, 100);
            uint8_t ch = q < 15 ? ' ' : q < 90 ? (uint8_t)ALNUM[below(r, 62)]
                                     : (uint8_t)"(){};,.+-=\"'/"[below(r, 13)];
            /* never close the comment early */
            if (ch == '/' && c->s->n && c->s->p[c->s->n - 1] == '*') ch = 'x';
            put(c->s, ch);
        }
        if (i + 1 < lines) put(c->s, '\n');
    }
    puts_(c->s, " */\n");
}

/* block: unrestricted block comments; frame: the producer puts the record
 * separator 0x1E before every unit (a statement line or a block comment),
 * which is always a token boundary of its output (Section 7.1). */
static uint64_t gen_c_common(uint64_t seed, uint8_t *out, uint64_t n, int block, int frame)
{
    rng_t r; rng_seed(&r, seed);
    uint64_t tmp_cap = 1u << 16;
    uint8_t *tmp = (uint8_t *)malloc(tmp_cap);
    uint64_t pos = 0;
    int indent = 0;
    for (;;) {
        sink_t s = {tmp, 0, tmp_cap, 0};
        cctx c = {&r, &s, block};
        if (frame) put(&s, 0x1E);
        if (block && chance(&r, 0.025)) c_block_comment(&c);
        else c_line(&c, &indent);
        if (s.full) continue;
        if (pos + s.n > n) break;
        memcpy(out + pos, tmp, s.n);
        pos += s.n;
    }
    while (pos < n) out[pos++] = '\n';
    free(tmp);
    return pos;
}

uint64_t gen_clike(uint64_t seed, uint8_t *out, uint64_t n) { return gen_c_common(seed, out, n, 0, 0); }
uint64_t gen_clike_block(uint64_t seed, uint8_t *out, uint64_t n) { return gen_c_common(seed, out, n, 1, 0); }
uint64_t gen_clike_block_framed(uint64_t seed, uint8_t *out, uint64_t n) { return gen_c_common(seed, out, n, 1, 1); }
