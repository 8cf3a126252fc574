/* Multi-threaded CPU compaction, timed by the benchmark for context beside
 * the oracle. It is NOT the oracle: the oracle is the plain sequential loop in
 * ka_oracle.c. This is test and benchmark infrastructure; the product library
 * never uses it.
 *
 * keep x < t, stable order (the order-preserving compaction of Sec. 4.1), in
 * three phases over `threads` contiguous chunks: each thread counts the kept
 * entries of its chunk; one thread turns the counts into chunk offsets (an
 * exclusive prefix sum); each thread copies its chunk's kept entries to its
 * offset. Returns the number of kept entries. */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

typedef struct {
    const uint32_t *x;
    uint32_t *y;
    uint64_t lo, hi;
    uint32_t t;
    uint64_t count, offset;
    int phase;
} job_t;

static void *work(void *arg) {
    job_t *j = (job_t *)arg;
    if (j->phase == 0) {
        uint64_t c = 0;
        for (uint64_t i = j->lo; i < j->hi; ++i) c += j->x[i] < j->t;
        j->count = c;
    } else {
        uint32_t *o = j->y + j->offset;
        for (uint64_t i = j->lo; i < j->hi; ++i)
            if (j->x[i] < j->t) *o++ = j->x[i];
    }
    return NULL;
}

static int run_phase(job_t *jobs, int threads, int phase) {
    pthread_t *tid = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
    if (!tid) return -1;
    int started = 0, rc = 0;
    for (int i = 0; i < threads; ++i) {
        jobs[i].phase = phase;
        if (pthread_create(&tid[i], NULL, work, &jobs[i]) != 0) {
            rc = -1;
            break;
        }
        ++started;
    }
    for (int i = 0; i < started; ++i) pthread_join(tid[i], NULL);
    free(tid);
    return rc;
}

/* Returns the kept count, or UINT64_MAX if threads could not be started. */
uint64_t cpu_mt_compact_lt(const uint32_t *x, uint64_t n, uint32_t t, uint32_t *y, int threads) {
    if (threads < 1) threads = 1;
    if ((uint64_t)threads > n && n > 0) threads = (int)n;
    if (n == 0) return 0;
    job_t *jobs = (job_t *)calloc((size_t)threads, sizeof(job_t));
    if (!jobs) return UINT64_MAX;
    const uint64_t per = (n + (uint64_t)threads - 1) / (uint64_t)threads;
    for (int i = 0; i < threads; ++i) {
        jobs[i].x = x;
        jobs[i].y = y;
        jobs[i].t = t;
        jobs[i].lo = per * (uint64_t)i < n ? per * (uint64_t)i : n;
        jobs[i].hi = per * (uint64_t)(i + 1) < n ? per * (uint64_t)(i + 1) : n;
    }
    uint64_t total = UINT64_MAX;
    if (run_phase(jobs, threads, 0) == 0) {
        total = 0;
        for (int i = 0; i < threads; ++i) {
            jobs[i].offset = total;
            total += jobs[i].count;
        }
        if (run_phase(jobs, threads, 1) != 0) total = UINT64_MAX;
    }
    free(jobs);
    return total;
}
