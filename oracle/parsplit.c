/*
 * parsplit.c -- the paper's CPU method as a timed baseline: the planner and
 * executor of Section 6 on host threads.
 *
 * TEST AND BENCH INFRASTRUCTURE ONLY (like lexoracle.c): only the test suite
 * and the bench's CPU-baseline leg load it.  It shares no code, header,
 * table or helper with the GPU library.  It is not an oracle: the tests check
 * it against the serial scan of lexoracle.c.
 *
 * Planner (Section 6): the k-1 equal-division targets t_i = floor(i n / k)
 * each slide forward to the next byte of the useful certified set; targets
 * that reach the end of the input, or land on a cut already taken, add no
 * chunk.  Executor: one thread per chunk runs the longest-match scanner of
 * Section 3 from q0 over its chunk (Theorems 1 and 3 make the result the
 * serial one), deleting discarded kinds as it emits (pi_I of Section 5, for
 * the filtered modes); then the per-chunk streams are concatenated in order,
 * one thread per chunk copying its stream to its prefix offset.
 * The first chunk (in order) that does not consume its whole slice ends the
 * stream at its halting offset (Corollary 1).
 *
 * Output format is the GPU library's: kinds u16, lengths u32.
 */
#define _POSIX_C_SOURCE 200809L
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#define UNDEF (-1)

typedef struct {
    /* automaton and input (shared, read only) */
    const int32_t *delta;
    const int32_t *tau;
    const uint8_t *in_I;      /* NULL: keep every kind */
    int32_t n_kinds, q0;
    const uint8_t *w;
    int64_t lo, hi;           /* this chunk */
    /* per-chunk stream */
    uint16_t *k;
    uint32_t *l;
    int64_t count, cap;
    int64_t con;              /* offset (relative to lo) where the scan halted */
    int oom;
    /* concatenation: this chunk's stream goes to out[out_off, out_off + out_n) */
    int64_t out_off, out_n;
    uint16_t *out_k;
    uint32_t *out_l;
} chunk_job;

static int push(chunk_job *j, int32_t kind, int64_t len)
{
    if (j->count == j->cap) {
        int64_t nc = j->cap ? 2 * j->cap : 4096;
        uint16_t *k = (uint16_t *)realloc(j->k, sizeof(uint16_t) * (size_t)nc);
        if (!k) return -1;
        j->k = k;
        uint32_t *l = (uint32_t *)realloc(j->l, sizeof(uint32_t) * (size_t)nc);
        if (!l) return -1;
        j->l = l;
        j->cap = nc;
    }
    j->k[j->count] = (uint16_t)kind;
    j->l[j->count] = (uint32_t)len;
    j->count++;
    return 0;
}

/* Section 3 scanner over [lo, hi), emitting kept tokens only. */
static void scan_chunk(chunk_job *j)
{
    const int32_t *delta = j->delta, *tau = j->tau;
    const uint8_t *w = j->w;
    int64_t i = j->lo;
    const int64_t n = j->hi;
    while (i < n) {
        int32_t q = j->q0;
        int64_t last = -1;
        int32_t last_kind = UNDEF;
        for (int64_t p = i; p < n; p++) {
            int32_t t = delta[(int64_t)q * 256 + w[p]];
            if (t == UNDEF) break;
            q = t;
            if (tau[q] != UNDEF) {
                last = p + 1;
                last_kind = tau[q];
            }
        }
        if (last < 0) break;
        if (!(j->in_I && last_kind >= 0 && last_kind < j->n_kinds && j->in_I[last_kind]))
            if (push(j, last_kind, last - i)) {
                j->oom = 1;
                break;
            }
        i = last;
    }
    j->con = i - j->lo;
}

static void *scan_worker(void *arg)
{
    scan_chunk((chunk_job *)arg);
    return NULL;
}

static void *copy_worker(void *arg)
{
    chunk_job *j = (chunk_job *)arg;
    if (j->out_n > 0) {
        memcpy(j->out_k + j->out_off, j->k, sizeof(uint16_t) * (size_t)j->out_n);
        memcpy(j->out_l + j->out_off, j->l, sizeof(uint32_t) * (size_t)j->out_n);
    }
    return NULL;
}

/* Run fn on every job, one thread each (a job whose thread cannot start runs
 * on the calling thread), and wait for all of them. */
static void run_all(chunk_job *jobs, int32_t m, pthread_t *th, uint8_t *started, void *(*fn)(void *))
{
    for (int32_t c = 0; c < m; c++) {
        started[c] = pthread_create(&th[c], NULL, fn, &jobs[c]) == 0;
        if (!started[c]) fn(&jobs[c]);
    }
    for (int32_t c = 0; c < m; c++)
        if (started[c]) pthread_join(th[c], NULL);
}

static double now_s(void)
{
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

/*
 * Lex w[0, n) with k chunks (k threads).  useful[b] != 0 marks the useful
 * certified bytes of the mode; in_I (or NULL) the discarded kinds.  Returns
 * the number of output tokens (all of them; the first `cap` are stored),
 * *con_out = con(w), *chunks_out = chunks planned, *seconds = wall time from
 * the start of planning to the end of the concatenation; -1 on failure to
 * allocate or start threads.
 */
int64_t par_lex(int32_t q0, const int32_t *delta, const int32_t *tau, const uint8_t *useful,
                const uint8_t *in_I, int32_t n_kinds, const uint8_t *w, int64_t n, int32_t k,
                uint16_t *out_k, uint32_t *out_l, int64_t cap, int64_t *con_out, int32_t *chunks_out,
                double *seconds)
{
    if (k < 1) k = 1;
    int64_t *cut = (int64_t *)malloc(sizeof(int64_t) * (size_t)(k + 1));
    chunk_job *jobs = (chunk_job *)calloc((size_t)k, sizeof(chunk_job));
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)k);
    uint8_t *started = (uint8_t *)malloc((size_t)k);
    int64_t total = -1;
    if (!cut || !jobs || !th || !started) goto out;
    const double t0 = now_s();
    /* planner */
    int32_t m = 0;
    cut[m++] = 0;
    int any = 0;
    for (int b = 0; b < 256; b++) any |= useful[b] != 0;
    for (int32_t i = 1; any && i < k && n > 0; i++) {
        int64_t t = (int64_t)((__int128)n * i / k);
        while (t < n && !useful[w[t]]) t++;
        if (t > cut[m - 1] && t < n) cut[m++] = t;
    }
    cut[m] = n;
    for (int32_t c = 0; c < m; c++) {
        chunk_job *j = &jobs[c];
        j->delta = delta;
        j->tau = tau;
        j->in_I = in_I;
        j->n_kinds = n_kinds;
        j->q0 = q0;
        j->w = w;
        j->lo = cut[c];
        j->hi = cut[c + 1];
        j->out_k = out_k;
        j->out_l = out_l;
    }
    run_all(jobs, m, th, started, scan_worker);
    /* ordered concatenation, up to and including the first chunk that halted */
    int64_t off = 0, con = n;
    int stop = 0, oom = 0;
    for (int32_t c = 0; c < m; c++) {
        chunk_job *j = &jobs[c];
        oom |= j->oom;
        if (stop) continue;
        j->out_off = off;
        j->out_n = off >= cap ? 0 : (off + j->count <= cap ? j->count : cap - off);
        off += j->count;
        if (j->lo + j->con < j->hi) {
            con = j->lo + j->con;
            stop = 1;
        }
    }
    run_all(jobs, m, th, started, copy_worker);
    const double t1 = now_s();
    for (int32_t c = 0; c < m; c++) {
        free(jobs[c].k);
        free(jobs[c].l);
    }
    if (!oom) {
        total = off;
        *con_out = con;
        *chunks_out = m;
        *seconds = t1 - t0;
    }
out:
    free(cut);
    free(jobs);
    free(th);
    free(started);
    return total;
}
