/*
 * oracle_threads.c -- runs the single-threaded oracle (vsbpp_oracle.c) on many
 * independent instances, one instance at a time per host thread.
 *
 * TEST INFRASTRUCTURE ONLY (parity tests and the CPU-baseline timing).  It
 * adds no arithmetic of its own: each instance is one plain call of
 * oracle_pack_ext; threads only take the next instance index from a shared
 * counter.  Instances are independent problems (Section 6.1), so the result
 * does not depend on the thread count.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

int oracle_pack_ext(const int32_t *w, int64_t m, const int32_t *B, int32_t n,
                    int32_t heuristic, int32_t criterion, int64_t sublist_size,
                    int32_t preopen, uint64_t seed, int32_t flags, int64_t max_open,
                    int32_t *bin_of_item, int32_t *bin_type,
                    int64_t *num_bins, int64_t *total_capacity);

typedef struct {
    int64_t N;
    const int32_t *w_all;
    const int64_t *w_off;
    const int32_t *B_all;
    const int32_t *B_off;
    int32_t heuristic, criterion, preopen, flags;
    int64_t sublist_size;
    int64_t max_open;
    uint64_t seed;
    int32_t *bin_of_item_all;
    int32_t *bin_type_all;
    int64_t *num_bins;
    int64_t *total;
    int32_t *status;
    int64_t next;                      /* shared work counter */
    pthread_mutex_t lock;
} or_many_job;

static void *or_many_worker(void *arg)
{
    or_many_job *job = (or_many_job *)arg;
    for (;;) {
        pthread_mutex_lock(&job->lock);
        const int64_t i = job->next++;
        pthread_mutex_unlock(&job->lock);
        if (i >= job->N)
            break;
        const int64_t a = job->w_off[i];
        const int64_t m = job->w_off[i + 1] - a;
        const int32_t b0 = job->B_off[i];
        const int32_t n = job->B_off[i + 1] - b0;
        job->status[i] = oracle_pack_ext(job->w_all + a, m, job->B_all + b0, n,
                                         job->heuristic, job->criterion,
                                         job->sublist_size, job->preopen, job->seed, job->flags,
                                         job->max_open,
                                         job->bin_of_item_all + a,
                                           job->bin_type_all + a,
                                           &job->num_bins[i], &job->total[i]);
    }
    return NULL;
}

int oracle_pack_many(int64_t N, const int32_t *w_all, const int64_t *w_off,
                     const int32_t *B_all, const int32_t *B_off,
                     int32_t heuristic, int32_t criterion, int64_t sublist_size,
                     int32_t preopen, uint64_t seed, int32_t flags, int64_t max_open,
                     int32_t *bin_of_item_all, int32_t *bin_type_all,
                     int64_t *num_bins, int64_t *total, int32_t *status,
                     int32_t nthreads)
{
    if (N < 0 || nthreads < 1)
        return -1;
    or_many_job job;
    job.N = N;
    job.w_all = w_all; job.w_off = w_off;
    job.B_all = B_all; job.B_off = B_off;
    job.heuristic = heuristic; job.criterion = criterion; job.preopen = preopen; job.flags = flags;
    job.sublist_size = sublist_size; job.seed = seed; job.max_open = max_open;
    job.bin_of_item_all = bin_of_item_all; job.bin_type_all = bin_type_all;
    job.num_bins = num_bins; job.total = total; job.status = status;
    job.next = 0;
    pthread_mutex_init(&job.lock, NULL);
    if (nthreads == 1) {
        or_many_worker(&job);
    } else {
        pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
        if (!th) {
            pthread_mutex_destroy(&job.lock);
            return -3;
        }
        int32_t started = 0;
        for (int32_t t = 0; t < nthreads; ++t) {
            if (pthread_create(&th[t], NULL, or_many_worker, &job) != 0)
                break;
            ++started;
        }
        if (started == 0)
            or_many_worker(&job);
        for (int32_t t = 0; t < started; ++t)
            pthread_join(th[t], NULL);
        free(th);
    }
    pthread_mutex_destroy(&job.lock);
    return 0;
}
