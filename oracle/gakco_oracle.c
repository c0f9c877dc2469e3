/*
 * CPU oracle for the gapped k-mer string kernel (GaKCo, arXiv 1704.07468).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code with the CUDA library.
 *
 * What it computes is the plain definition, written out by brute force:
 *
 *   Definition 1 (Section 2.1): a g-pair_m(x, y) is a pair of g-mers, one
 *   from x and one from y, at Hamming distance exactly m.  The g-mers of a
 *   sequence of length l are its l - g + 1 contiguous windows (Eq. 5, where
 *   the i-th g-mer starts at position i); a sequence shorter than g has none.
 *
 *   Mismatch profile N_m(x, y) (Eq. 7, Table 1) = number of g-pair_m(x, y),
 *   counted over ALL ordered window pairs (i, j), including i == j when
 *   x == y.
 *
 * For every requested row x and every column y the oracle visits every
 * window pair, counts the positions where the two windows differ, and
 * increments N_d(x, y) when that count d is at most maxd.  Accumulation is
 * in int64.  The kernel K = sum_m h_m N_m (Eq. 6 and Eq. 7) and the
 * normalisation are applied on top of these counts by the Python wrapper.
 *
 * Rows are split across POSIX threads; each thread owns whole output rows,
 * so no synchronisation is needed beyond the final join.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    const uint8_t *xcodes;
    const int64_t *xoff;
    const int32_t *rows;
    int32_t nrows;
    const uint8_t *ycodes;
    const int64_t *yoff;
    int32_t ny;
    int32_t g;
    int32_t maxd;
    int64_t *out; /* (maxd + 1) x nrows x ny */
    int32_t first_row;
    int32_t stride;
} job_t;

static int64_t n_windows(int64_t len, int32_t g) {
    return len >= g ? len - g + 1 : 0;
}

/* Hamming distance of two g-long windows, stopping early once it passes
 * maxd (the count then no longer matters, only that it exceeds maxd). */
static int32_t hamming_capped(const uint8_t *a, const uint8_t *b, int32_t g,
                              int32_t maxd) {
    int32_t d = 0;
    for (int32_t p = 0; p < g; ++p) {
        if (a[p] != b[p]) {
            if (++d > maxd) return d;
        }
    }
    return d;
}

static void profile_one_row(const job_t *jb, int32_t r) {
    const int32_t x = jb->rows[r];
    const uint8_t *xs = jb->xcodes + jb->xoff[x];
    const int64_t wx = n_windows(jb->xoff[x + 1] - jb->xoff[x], jb->g);
    const int64_t plane = (int64_t)jb->nrows * jb->ny;
    for (int32_t y = 0; y < jb->ny; ++y) {
        const uint8_t *ys = jb->ycodes + jb->yoff[y];
        const int64_t wy = n_windows(jb->yoff[y + 1] - jb->yoff[y], jb->g);
        int64_t *cell = jb->out + (int64_t)r * jb->ny + y;
        for (int64_t i = 0; i < wx; ++i) {
            for (int64_t j = 0; j < wy; ++j) {
                int32_t d = hamming_capped(xs + i, ys + j, jb->g, jb->maxd);
                if (d <= jb->maxd) cell[(int64_t)d * plane] += 1;
            }
        }
    }
}

static void *worker(void *arg) {
    const job_t *jb = (const job_t *)arg;
    for (int32_t r = jb->first_row; r < jb->nrows; r += jb->stride)
        profile_one_row(jb, r);
    return NULL;
}

/*
 * Mismatch profile of rows `rows[0..nrows)` of dataset X against every
 * sequence of dataset Y.
 *
 *   xcodes/xoff : dataset X (codes concatenated, offsets of length nx + 1)
 *   rows        : indices into X of the rows to compute
 *   ycodes/yoff : dataset Y (for a Gram matrix, the same arrays as X)
 *   g           : g-mer length (>= 1)
 *   maxd        : largest distance histogrammed (0 <= maxd <= g)
 *   nthreads    : worker threads (>= 1)
 *   out         : int64 (maxd + 1) x nrows x ny, zeroed here
 *
 * Returns 0, or -1 on an invalid argument.
 */
int oracle_profile(const uint8_t *xcodes, const int64_t *xoff,
                   const int32_t *rows, int32_t nrows, const uint8_t *ycodes,
                   const int64_t *yoff, int32_t ny, int32_t g, int32_t maxd,
                   int32_t nthreads, int64_t *out) {
    if (g < 1 || maxd < 0 || maxd > g || nrows < 0 || ny < 0 || nthreads < 1)
        return -1;
    memset(out, 0, sizeof(int64_t) * (size_t)(maxd + 1) * (size_t)nrows *
                       (size_t)ny);
    if (nthreads > nrows) nthreads = nrows > 0 ? nrows : 1;
    pthread_t *tid = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
    job_t *jobs = (job_t *)malloc(sizeof(job_t) * nthreads);
    if (!tid || !jobs) {
        free(tid);
        free(jobs);
        return -1;
    }
    for (int32_t t = 0; t < nthreads; ++t) {
        job_t j = {xcodes, xoff, rows, nrows, ycodes, yoff, ny, g, maxd,
                   out,    t,    nthreads};
        jobs[t] = j;
    }
    for (int32_t t = 1; t < nthreads; ++t)
        pthread_create(&tid[t], NULL, worker, &jobs[t]);
    worker(&jobs[0]);
    for (int32_t t = 1; t < nthreads; ++t) pthread_join(tid[t], NULL);
    free(tid);
    free(jobs);
    return 0;
}

/*
 * Self profile N_d(x, x) for every sequence x of one dataset: the diagonal
 * of the Gram mismatch profile, which normalisation needs for every column
 * even when only a sample of rows is computed.
 *
 *   out : int64 (maxd + 1) x n, zeroed here.
 */
int oracle_self_profile(const uint8_t *codes, const int64_t *off, int32_t n,
                        int32_t g, int32_t maxd, int64_t *out) {
    if (g < 1 || maxd < 0 || maxd > g || n < 0) return -1;
    memset(out, 0, sizeof(int64_t) * (size_t)(maxd + 1) * (size_t)n);
    for (int32_t x = 0; x < n; ++x) {
        const uint8_t *s = codes + off[x];
        const int64_t w = n_windows(off[x + 1] - off[x], g);
        for (int64_t i = 0; i < w; ++i)
            for (int64_t j = 0; j < w; ++j) {
                int32_t d = hamming_capped(s + i, s + j, g, maxd);
                if (d <= maxd) out[(int64_t)d * n + x] += 1;
            }
    }
    return 0;
}
