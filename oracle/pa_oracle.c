/*
 * CPU oracle for the GF(2) Toeplitz hash of length-compatible privacy
 * amplification (Wang, Zhang, Yu, Guo, arXiv 1805.02372).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, calls or
 * includes this file; only the tests, the smoke check and the bench's CPU
 * baseline use it. It shares no code with the CUDA path.
 *
 * What it computes (Sec. 2.1, Eq. 1 and Sec. 2.3): the Toeplitz matrix T is
 * diagonal-constant, T[i][j] = T[i+1][j+1], so the m x n matrix is fixed by the
 * n+m-1 bits of its first column and first row. This library reads those bits
 * from one seed string s with
 *
 *        T[i][j] = s[n-1+i-j]         (0 <= i < m, 0 <= j < n)
 *
 * and returns y = T x mod 2, i.e. y[i] = XOR over j of (x[j] AND s[n-1+i-j]).
 * This is the plain definition of the hash written out; every GPU path must
 * reach exactly this result (the method is exact, not an approximation).
 *
 * Packing: bit j of a string is bit (j & 63) of 64-bit word (j >> 6). Key bits at
 * positions >= n and seed bits at positions >= n+m-1 are ignored; output bits
 * at positions >= m are written as zero.
 *
 * Two row evaluators are given:
 *   oracle_row_bitloop  one AND per matrix entry, bit by bit (tiny sizes);
 *   oracle_row_packed   row i of T taken as 64-bit windows of the reversed seed
 *                       (T[i][j] = r[m-1-i+j] with r[t] = s[n+m-2-t]), ANDed
 *                       with the key words, XOR-accumulated, parity of the
 *                       population count at the end.
 * The full hash runs the packed evaluator over row ranges on POSIX threads.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL -1
#define ORACLE_ENOMEM -3

static int get_bit(const uint64_t *v, uint64_t i) { return (int)((v[i >> 6] >> (i & 63)) & 1u); }

static void set_bit(uint64_t *v, uint64_t i) { v[i >> 6] |= (uint64_t)1 << (i & 63); }

static int parity64(uint64_t v) {
    int c = 0;
    while (v) { v &= v - 1; c ^= 1; }
    return c;
}

/* y[i] straight from the definition, one bit product at a time. */
int oracle_row_bitloop(uint64_t n, uint64_t m, const uint64_t *seed, const uint64_t *key,
                       uint64_t i) {
    int acc = 0;
    (void)m;
    for (uint64_t j = 0; j < n; ++j)
        acc ^= get_bit(key, j) & get_bit(seed, n - 1 + i - j);
    return acc;
}

/* Reversed seed r[t] = s[n+m-2-t] for t < n+m-1, zero beyond, plus 2 spare words. */
static uint64_t *reversed_seed(uint64_t n, uint64_t m, const uint64_t *seed, uint64_t *nwords) {
    uint64_t len = n + m - 1;
    uint64_t w = (len + 63) / 64 + 2;
    uint64_t *r = (uint64_t *)calloc(w, sizeof(uint64_t));
    if (!r) return NULL;
    for (uint64_t t = 0; t < len; ++t)
        if (get_bit(seed, len - 1 - t)) set_bit(r, t);
    *nwords = w;
    return r;
}

/* Key words with the bits at positions >= n cleared. */
static uint64_t *masked_key(uint64_t n, const uint64_t *key) {
    uint64_t w = (n + 63) / 64;
    uint64_t *k = (uint64_t *)malloc(w * sizeof(uint64_t));
    if (!k) return NULL;
    memcpy(k, key, w * sizeof(uint64_t));
    if (n & 63) k[w - 1] &= ((uint64_t)1 << (n & 63)) - 1;
    return k;
}

/* 64 bits of r starting at bit o (bits past the array read as zero). */
static uint64_t window64(const uint64_t *r, uint64_t nwords, uint64_t o) {
    uint64_t q = o >> 6, b = o & 63;
    uint64_t lo = q < nwords ? r[q] : 0;
    uint64_t hi = q + 1 < nwords ? r[q + 1] : 0;
    return b ? (lo >> b) | (hi << (64 - b)) : lo;
}

/* Row i of T is r[m-1-i .. m-1-i+n); y[i] = parity(row AND key). */
static int row_packed(uint64_t n, uint64_t m, const uint64_t *r, uint64_t rw, const uint64_t *k,
                      uint64_t i) {
    uint64_t kw = (n + 63) / 64, acc = 0, off = m - 1 - i;
    for (uint64_t w = 0; w < kw; ++w) acc ^= k[w] & window64(r, rw, off + 64 * w);
    return parity64(acc);
}

typedef struct {
    uint64_t n, m, rw;
    const uint64_t *r, *k;
    /* full mode: rows [lo, hi) into out; rows mode: list entries [lo, hi) into bits */
    uint64_t lo, hi;
    uint64_t *out;
    const uint64_t *rows;
    uint8_t *bits;
} job_t;

static void *run_job(void *p) {
    job_t *j = (job_t *)p;
    for (uint64_t t = j->lo; t < j->hi; ++t) {
        if (j->rows) {
            j->bits[t] = (uint8_t)row_packed(j->n, j->m, j->r, j->rw, j->k, j->rows[t]);
        } else if (row_packed(j->n, j->m, j->r, j->rw, j->k, t)) {
            j->out[t >> 6] |= (uint64_t)1 << (t & 63); /* ranges are 64-row aligned */
        }
    }
    return NULL;
}

static int run_threads(job_t *proto, uint64_t total, uint64_t align, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    job_t jobs[256];
    uint64_t units = (total + align - 1) / align;
    uint64_t per = (units + (uint64_t)nthreads - 1) / (uint64_t)nthreads;
    int started = 0;
    for (int t = 0; t < nthreads; ++t) {
        uint64_t lo = (uint64_t)t * per * align, hi = lo + per * align;
        if (lo >= total) break;
        if (hi > total) hi = total;
        jobs[t] = *proto;
        jobs[t].lo = lo;
        jobs[t].hi = hi;
        if (nthreads == 1 || pthread_create(&th[t], NULL, run_job, &jobs[t]) != 0) {
            run_job(&jobs[t]);
            th[t] = 0;
        }
        started = t + 1;
    }
    for (int t = 0; t < started; ++t)
        if (th[t]) pthread_join(th[t], NULL);
    return ORACLE_OK;
}

/* y = T x mod 2 for all m rows; out has ceil(m/64) words, bits >= m zero. */
int oracle_hash(uint64_t n, uint64_t m, const uint64_t *seed, const uint64_t *key, uint64_t *out,
                int nthreads) {
    if (n == 0 || m == 0 || !seed || !key || !out) return ORACLE_EINVAL;
    uint64_t rw;
    uint64_t *r = reversed_seed(n, m, seed, &rw);
    uint64_t *k = masked_key(n, key);
    if (!r || !k) { free(r); free(k); return ORACLE_ENOMEM; }
    memset(out, 0, ((m + 63) / 64) * sizeof(uint64_t));
    job_t proto = {n, m, rw, r, k, 0, 0, out, NULL, NULL};
    int rc = run_threads(&proto, m, 64, nthreads);
    free(r);
    free(k);
    return rc;
}

/* y[rows[t]] for t < count, one byte (0/1) each. */
int oracle_rows(uint64_t n, uint64_t m, const uint64_t *seed, const uint64_t *key,
                const uint64_t *rows, uint64_t count, uint8_t *bits, int nthreads) {
    if (n == 0 || m == 0 || !seed || !key || (count && (!rows || !bits))) return ORACLE_EINVAL;
    for (uint64_t t = 0; t < count; ++t)
        if (rows[t] >= m) return ORACLE_EINVAL;
    uint64_t rw;
    uint64_t *r = reversed_seed(n, m, seed, &rw);
    uint64_t *k = masked_key(n, key);
    if (!r || !k) { free(r); free(k); return ORACLE_ENOMEM; }
    job_t proto = {n, m, rw, r, k, 0, 0, NULL, rows, bits};
    int rc = run_threads(&proto, count, 1, nthreads);
    free(r);
    free(k);
    return rc;
}

/* Same rows, by the bit-by-bit evaluator (single thread; tiny sizes only). */
int oracle_rows_bitloop(uint64_t n, uint64_t m, const uint64_t *seed, const uint64_t *key,
                        const uint64_t *rows, uint64_t count, uint8_t *bits) {
    if (n == 0 || m == 0 || !seed || !key || (count && (!rows || !bits))) return ORACLE_EINVAL;
    for (uint64_t t = 0; t < count; ++t) {
        if (rows[t] >= m) return ORACLE_EINVAL;
        bits[t] = (uint8_t)oracle_row_bitloop(n, m, seed, key, rows[t]);
    }
    return ORACLE_OK;
}
