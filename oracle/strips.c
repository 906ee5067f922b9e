/*
 * strips.c -- the oracle's monotone chain run strip-parallel on the host
 * cores (the CPU baseline of the measurements).
 *
 * TEST INFRASTRUCTURE ONLY, like oracle.c: only tests/, smoke() and
 * bench.py's CPU baseline may call it. It shares no code with the CUDA
 * library.
 *
 * The sorted input is cut into T contiguous strips, one per thread. Each
 * thread runs oracle_upper_hull on its strip; then one more monotone chain
 * runs over the concatenation of the strip hoods, in order. The hood of a
 * union of blocks equals the hood of the union of their hoods (a point below
 * the hood of its own block is below the hood of the whole set), which is
 * the identity the paper's merge schedule rests on (Section 2). The result
 * is the same index list as oracle_upper_hull on the whole input:
 *   - a point that is not a corner of its strip's hood lies on or below a
 *     segment between two points of the strip, so it is not a corner of the
 *     whole hood either;
 *   - repeats: copies of one point are consecutive in sorted order, so a
 *     copy that starts strip k + 1 follows its first occurrence, which ends
 *     strip k and is therefore a corner of strip k's hood; the final chain
 *     meets the first occurrence first and skips the copy, as the single
 *     scan does.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

int64_t oracle_upper_hull(const int32_t *kx, const int32_t *ky, int64_t n,
                          int32_t *out);

struct strip_job {
    const int32_t *kx, *ky;
    int64_t a, b;     /* strip [a, b) of the input */
    int32_t *out;     /* its hood, as strip-relative indices */
    int64_t h;
};

static void *strip_run(void *arg)
{
    struct strip_job *j = (struct strip_job *)arg;
    j->h = oracle_upper_hull(j->kx + j->a, j->ky + j->a, j->b - j->a, j->out);
    return NULL;
}

/*
 * Writes the corners of the hood of kx/ky[0..n) to out[0..h) and returns h,
 * using `threads` strips (clamped to [1, 256] and to n). Returns -1 if
 * memory or a thread could not be had.
 */
int64_t oracle_upper_hull_strips(const int32_t *kx, const int32_t *ky,
                                 int64_t n, int32_t *out, int threads)
{
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    if (n < (int64_t)threads * 2) threads = 1;
    if (threads == 1) return oracle_upper_hull(kx, ky, n, out);

    struct strip_job jobs[256];
    pthread_t tid[256];
    int32_t *scratch = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!scratch) return -1;
    for (int t = 0; t < threads; ++t) {
        jobs[t].kx = kx;
        jobs[t].ky = ky;
        jobs[t].a = n * t / threads;
        jobs[t].b = n * (t + 1) / threads;
        jobs[t].out = scratch + jobs[t].a;
        jobs[t].h = 0;
    }
    int started = 0, failed = 0;
    for (int t = 1; t < threads; ++t) {
        if (pthread_create(&tid[t], NULL, strip_run, &jobs[t]) != 0) {
            failed = 1;
            break;
        }
        ++started;
    }
    strip_run(&jobs[0]);
    for (int t = 1; t <= started; ++t) pthread_join(tid[t], NULL);
    if (failed) {
        free(scratch);
        return -1;
    }

    /* concatenate the strip hoods: their points and global indices */
    int64_t m = 0;
    for (int t = 0; t < threads; ++t) m += jobs[t].h;
    int32_t *cx = (int32_t *)malloc((size_t)m * sizeof(int32_t));
    int32_t *cy = (int32_t *)malloc((size_t)m * sizeof(int32_t));
    int32_t *gi = (int32_t *)malloc((size_t)m * sizeof(int32_t));
    int32_t *ci = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    if (!cx || !cy || !gi || !ci) {
        free(cx); free(cy); free(gi); free(ci); free(scratch);
        return -1;
    }
    int64_t k = 0;
    for (int t = 0; t < threads; ++t)
        for (int64_t i = 0; i < jobs[t].h; ++i) {
            const int64_t g = jobs[t].a + jobs[t].out[i];
            cx[k] = kx[g];
            cy[k] = ky[g];
            gi[k] = (int32_t)g;
            ++k;
        }
    const int64_t h = oracle_upper_hull(cx, cy, m, ci);
    for (int64_t i = 0; i < h; ++i) out[i] = gi[ci[i]];
    free(cx); free(cy); free(gi); free(ci); free(scratch);
    return h;
}

void oracle_upper_hull_batched(const int32_t *kx, const int32_t *ky,
                               const int64_t *offsets, int64_t num_sets,
                               int32_t *out, int32_t *counts);

struct batch_job {
    const int32_t *kx, *ky;
    const int64_t *offsets;
    int64_t s0, s1;  /* sets [s0, s1) */
    int32_t *out, *counts;
};

static void *batch_run(void *arg)
{
    struct batch_job *j = (struct batch_job *)arg;
    oracle_upper_hull_batched(j->kx, j->ky, j->offsets + j->s0, j->s1 - j->s0,
                              j->out, j->counts + j->s0);
    return NULL;
}

/*
 * The batched form on `threads` threads: each takes a contiguous range of
 * sets (ranges of about equal point counts) and runs the single-set chain on
 * each of its sets. Same output as oracle_upper_hull_batched. Returns 0, or
 * -1 if a thread could not be started.
 */
int oracle_upper_hull_batched_threads(const int32_t *kx, const int32_t *ky,
                                      const int64_t *offsets, int64_t num_sets,
                                      int32_t *out, int32_t *counts, int threads)
{
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    if (num_sets < threads) threads = num_sets > 0 ? (int)num_sets : 1;
    struct batch_job jobs[256];
    pthread_t tid[256];
    const int64_t total = num_sets > 0 ? offsets[num_sets] - offsets[0] : 0;
    int64_t s = 0;
    for (int t = 0; t < threads; ++t) {
        /* sets until the point count reaches (t + 1) / threads of the total */
        const int64_t goal = offsets[0] + total * (t + 1) / threads;
        int64_t e = s;
        while (e < num_sets && (t == threads - 1 || offsets[e] < goal)) ++e;
        jobs[t].kx = kx;
        jobs[t].ky = ky;
        jobs[t].offsets = offsets;
        jobs[t].s0 = s;
        jobs[t].s1 = e;
        jobs[t].out = out;
        jobs[t].counts = counts;
        s = e;
    }
    int started = 0, failed = 0;
    for (int t = 1; t < threads; ++t) {
        if (pthread_create(&tid[t], NULL, batch_run, &jobs[t]) != 0) {
            failed = 1;
            break;
        }
        ++started;
    }
    batch_run(&jobs[0]);
    for (int t = 1; t <= started; ++t) pthread_join(tid[t], NULL);
    return failed ? -1 : 0;
}
