/*
 * vsbpp.h -- C ABI of the GB300 (sm_103a) engine for the hybrid-P-system
 * heuristics for the Variable Sized Bin Packing Problem (VSBPP) of Alenezi,
 * Aboelfotoh, Albdaiwi & Almulla (arXiv:1602.08735).
 *
 * The problem (Section 1 "Formal Definition", Section 6.1): n bin types with
 * capacities B_1 > B_2 > ... > B_n > 0 in unlimited supply, a list of m
 * indivisible items with integer weights 1 <= w_j <= B_1; pack every item and
 * minimise the total capacity of the bins used.
 *
 * The method (Sections 6.2-6.4): a "hybrid P system" in which every open bin
 * is a membrane whose label carries (bin index, type) and whose polarity
 * carries the load.  Items leave their sublist membrane one per step (Rule 3)
 * in list order, every bin membrane tests whether the item fits (Rule 4),
 * first-fit / best-fit / worst-fit (Section 1) picks one bin, the lowest
 * creation index winning ties, the bin's load grows by w, and a bin whose
 * load first reaches half its capacity divides off one empty bin of its type
 * (Rule 5).  When no bin has room, a bin of the smallest type that holds the
 * item is opened.  The second heuristic (Section 6.4) packs every
 * permutation of each small sublist and keeps the cheapest.
 *
 * Conventions shared by every entry point:
 *   - all integers are exact; no floating point anywhere on the path;
 *   - capacities B[0..n) are given largest first; "type t" is index t into B
 *     (type 0 = B_1);  1 <= n <= VSBPP_MAX_TYPES;
 *   - bin ids are dense, 0-based, in creation order among used bins (bins
 *     with at least one item); with several sublists, the bins of sublist g
 *     follow those of sublist g-1;
 *   - a packing of m items uses at most m bins, so bin_type needs room for m
 *     entries;
 *   - total_capacity is the sum of B[type] over the used bins (int64);
 *   - the library never allocates or frees caller-owned buffers; all output
 *     buffers are written in full on success;
 *   - no C++ exception crosses this interface; every function returns a
 *     status code (VSBPP_OK or a negative VSBPP_E* value).
 *
 * Validation (identical for every entry point, first failing check wins):
 *   m >= 0; 1 <= n <= VSBPP_MAX_TYPES; B strictly decreasing and > 0;
 *   parameters in range; then the items in list order: w_j < 1 gives
 *   VSBPP_EINVAL, w_j > B_1 gives VSBPP_ETOOBIG.  m = 0 is valid and gives
 *   zero bins and total 0.  On an error the output arrays of that instance
 *   are unspecified and num_bins = total = 0.
 *
 * Threading: every entry point may be called from any host thread.  Calls on
 * different streams (or devices) proceed at the same time; calls on the same
 * stream or on the same plan are serialised by the library.  Host-memory
 * calls (vsbpp_pack, vsbpp_pack_batch_host) from several threads also proceed
 * at the same time: each borrows a stream, 16 MB of pinned staging and
 * scratch of the current device for its length (created when all are in use,
 * kept for reuse until the process exits).  The launch configuration and the counter and
 * timing switches are process-wide.  Device entry points are asynchronous
 * with respect to the host and ordered on the caller's stream.
 *
 * Parameter layout changed in 1.1.0: `reserved` became `flags` and `max_open`
 * was appended (struct size 40 bytes).
 */
#ifndef VSBPP_H
#define VSBPP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VSBPP_VERSION 10100          /* 1.1.0 */
#define VSBPP_MAX_TYPES 32           /* bin types per instance */
#define VSBPP_MAX_OPEN 32            /* largest bound of the bounded-space variant */

/* Option flags (vsbpp_params.flags). */
#define VSBPP_REMARK3 1   /* Rule 5 with Remark 3 of Section 6.3 read as a condition: a bin of a
                             type divides off a new one only if every bin of that type then
                             holds at least half its capacity (a consequence of Rule 5 under the
                             literal Rule 2, not once a bin can open below half)               */
#define VSBPP_PRESORT 2   /* offline pre-sort: the list is packed in non-increasing weight order
                             (equal weights keep their list order), as the decreasing-order
                             heuristics of the prior work in Section 5 do; bin_of_item is still
                             reported per item at its original position, RANDOM keys are the
                             sorted positions, and validation still reports the first
                             offending item in the caller's order                               */
#define VSBPP_H2_MAX_SUBLIST 12      /* s <= 6: Section 6.4 (s! <= 720); 7..12: exhaustive search */

/* Selection criterion of Rule 3 / Rule 4 (Section 1 defines FF, BF, WF). */
typedef enum {
    VSBPP_FF = 0,      /* lowest-index bin with room                          */
    VSBPP_BF = 1,      /* bin with the least room left that fits; lowest index */
    VSBPP_WF = 2,      /* bin with the most room left; lowest index            */
    VSBPP_RANDOM = 3   /* per item, c = SplitMix64(seed, key) mod 3 (0=FF,1=BF,2=WF);
                          key = item index within the instance (first heuristic),
                          (sublist*720 + permutation rank)*8 + step (second, s <= 6)
                          or (sublist*12! + rank)*16 + step (second, s = 7..12) */
} vsbpp_criterion;

/* The two heuristics of Section 6. */
typedef enum {
    VSBPP_H1 = 1,      /* Section 6.3: each sublist packed in list order        */
    VSBPP_H2 = 2       /* Section 6.4: best permutation of each small sublist   */
} vsbpp_heuristic;

/* Run parameters.  Zero-initialise and set what you need. */
typedef struct {
    int32_t  heuristic;     /* VSBPP_H1 or VSBPP_H2                                     */
    int32_t  criterion;     /* vsbpp_criterion                                          */
    int64_t  sublist_size;  /* Rule 1 sublist length s.  H1: 0 means s = m (one membrane
                               system per instance).  H2: 0 means 5; at most 12 (s <= 6
                               is Section 6.4's block per sublist; 7..12 runs every one
                               of the s! permutations across the whole GPU, the
                               exhaustive search Section 7 compares against, and
                               requires preopen = 0, else EINVAL).  The
                               list is cut into contiguous chunks of s items in order.   */
    int32_t  preopen;       /* 0: no bin open at the start (a bin opens when nothing
                               fits).  1: literal Rule 2, one empty bin of every type,
                               types in order, before the first item.                    */
    int32_t  flags;         /* VSBPP_REMARK3 | VSBPP_PRESORT, or 0; other bits: EINVAL.
                               Both apply to every heuristic and sublist size (the
                               exhaustive 7..12-item search included); VSBPP_REMARK3
                               with max_open > 0: EINVAL                                 */
    uint64_t seed;          /* used by VSBPP_RANDOM only                                 */
    int64_t  max_open;      /* 0: no bound (the method as the paper states it).  K >= 1:
                               the bounded-space variant of Section 1's FF / BF / WF
                               ("keeps only a specific number of bins open"): only the K or
                               fewer open bins take part in Rule 4's fit test, a bin
                               closes as soon as it is completely filled, and before a bin
                               is created (no open bin holds the item, a Rule 5 division,
                               a Rule 2 bin) while K are open, the open bin with the lowest
                               creation index closes.  Closed bins keep their items and
                               count in the objective.  First heuristic with one membrane
                               system per instance (sublist_size 0 or >= every m), without
                               VSBPP_REMARK3, else EINVAL; K <= VSBPP_MAX_OPEN, else
                               VSBPP_ECAPACITY; K < 0: EINVAL.                           */
} vsbpp_params;

/* Status codes. */
enum {
    VSBPP_OK = 0,
    VSBPP_EINVAL = -1,      /* malformed instance or parameter                     */
    VSBPP_ETOOBIG = -2,     /* an item heavier than B_1                            */
    VSBPP_ENOMEM = -3,      /* device or host memory could not be obtained         */
    VSBPP_ECUDA = -4,       /* a CUDA call failed (see vsbpp_last_cuda_error)      */
    VSBPP_ETIMEDOUT = -5,   /* a bounded wait ran out                              */
    VSBPP_EBUSY = -6,       /* serving: no slot or memory budget available now     */
    VSBPP_ENOTFOUND = -7,   /* serving: unknown ticket                             */
    VSBPP_ECAPACITY = -8    /* an instance exceeds a size limit of the entry point */
};

/* Human-readable name of a status code (static string, never NULL). */
const char *vsbpp_strerror(int code);

/* Library version, VSBPP_VERSION of the build. */
int vsbpp_version(void);

/* Last CUDA error code seen by the library on this process (cudaError_t as int). */
int vsbpp_last_cuda_error(void);

/*
 * vsbpp_pack -- pack one instance held in HOST memory; synchronous.
 *
 *   w[m]            item weights (host, int32), list order
 *   B[n]            capacities, strictly decreasing (host, int32)
 *   p               run parameters (host); NULL means H1, BF, s = m, no preopen
 *   bin_of_item[m]  out (host): dense bin id of each item
 *   bin_type[m]     out (host): type of bin k for k < *num_bins
 *   num_bins        out (host): number of used bins
 *   total_capacity  out (host): sum of B[bin_type[k]]
 *
 * Copies the instance to the device, runs the same kernels as
 * vsbpp_pack_device on the library's own stream, copies the result back and
 * returns when it is complete.  Returns the instance's status code.
 */
int vsbpp_pack(const int32_t *w, int64_t m, const int32_t *B, int32_t n,
               const vsbpp_params *p,
               int32_t *bin_of_item, int32_t *bin_type,
               int64_t *num_bins, int64_t *total_capacity);

/*
 * vsbpp_pack_device -- pack one instance held in DEVICE memory; asynchronous.
 *
 * Same arguments as vsbpp_pack, but w, B and every output pointer are device
 * pointers (e.g. the data pointers of CUDA tensors) and the work is enqueued
 * on `stream` (a cudaStream_t; NULL = legacy default stream).  The return
 * value only reports host-side argument checks (m, n, p, pointers); the
 * instance's own status (including weight checks) is written to the device
 * word *status when the stream reaches it.  Library scratch belongs to the
 * stream and grows in stream order, as for vsbpp_pack_batch below: calls on
 * different streams never wait for each other on the host.
 */
int vsbpp_pack_device(const int32_t *w, int64_t m, const int32_t *B, int32_t n,
                      const vsbpp_params *p,
                      int32_t *bin_of_item, int32_t *bin_type,
                      int64_t *num_bins, int64_t *total_capacity,
                      int32_t *status, void *stream);

/*
 * vsbpp_pack_batch -- pack N independent instances in one persistent,
 * work-stealing launch; asynchronous on `stream`.  All array arguments are
 * DEVICE pointers in CSR form:
 *
 *   w_all[w_off[N]]     item weights, instance i = w_all[w_off[i] .. w_off[i+1])
 *   w_off[N+1]          int64 offsets, w_off[0] = 0, non-decreasing
 *   B_all[B_off[N]]     capacities, instance i = B_all[B_off[i] .. B_off[i+1])
 *   B_off[N+1]          int32 offsets
 *   max_m               host-side upper bound on any instance's m (sizes the
 *                       on-chip state); an instance with m > max_m gets status
 *                       VSBPP_ECAPACITY
 *   bin_of_item_all     out [w_off[N]]: dense bin ids, aligned with w_all
 *   bin_type_all        out [w_off[N]]: instance i's bin types at
 *                       bin_type_all[w_off[i] .. w_off[i] + num_bins[i])
 *   num_bins[N], total[N], status[N]   out, per instance
 *
 * Instances are handed out largest first to resident thread groups through an
 * atomic queue (work stealing).  The first call for a given shape may
 * allocate scratch memory and should not be made while `stream` is being
 * captured; vsbpp_plan_* below pre-allocates and records a CUDA graph.
 * Scratch belongs to the stream and grows with the stream-ordered allocator
 * (cudaMallocFromPoolAsync / cudaFreeAsync on `stream`, from a library pool
 * that keeps freed memory), so growing it never waits on other streams'
 * work.  Returns a host-side status.
 */
int vsbpp_pack_batch(int64_t N, const int32_t *w_all, const int64_t *w_off,
                     const int32_t *B_all, const int32_t *B_off, int64_t max_m,
                     const vsbpp_params *p,
                     int32_t *bin_of_item_all, int32_t *bin_type_all,
                     int64_t *num_bins, int64_t *total, int32_t *status,
                     void *stream);

/*
 * vsbpp_pack_batch_host -- vsbpp_pack_batch for a batch held in HOST memory;
 * synchronous.  Same CSR arguments and results as vsbpp_pack_batch, but every
 * array is a host pointer (pinned, e.g. from cudaHostAlloc, or pageable).
 * The library copies the inputs to device buffers it owns on the current
 * device, packs them with the same kernels on a stream of its own that the
 * call holds alone, copies the results back and returns when they are in
 * place: the whole host-to-host path in one call.  Calls from several host
 * threads run side by side on the GPU.  Pinned buffers are copied directly;
 * pageable ones are staged through the library's pinned buffers.  max_m: as
 * for vsbpp_pack_batch (0 lets the library read it off w_off).  Returns a
 * host-side status; per-instance codes are in status[].
 */
int vsbpp_pack_batch_host(int64_t N, const int32_t *w_all, const int64_t *w_off,
                          const int32_t *B_all, const int32_t *B_off, int64_t max_m,
                          const vsbpp_params *p,
                          int32_t *bin_of_item_all, int32_t *bin_type_all,
                          int64_t *num_bins, int64_t *total, int32_t *status);

/*
 * vsbpp_pack_batch_noalloc -- vsbpp_pack_batch for callers that cannot
 * allocate device memory.  (The paper has no counterpart: this is a property
 * of the library, not of the method.)
 *
 * Who needs it: code that owns a fixed device-memory reservation or runs
 * inside another allocator's arena, where a library allocation would bypass
 * the owner's accounting; latency-critical loops that cannot afford an
 * allocation, or the device-wide synchronisation a cudaFree implies, on
 * their path.  This call allocates nothing: its scratch (about 0.5 MiB) is
 * one static array in the library's device image, shared by every call on a
 * device and held by every GPU that loads the library until the process
 * exits.
 *
 * Arguments and results as vsbpp_pack_batch, restricted to the first
 * heuristic with one membrane system per instance (sublist_size 0 or
 * >= max_m), without option flags or a bound (flags = max_open = 0, else
 * VSBPP_EINVAL): N <= VSBPP_NOALLOC_MAX_INSTANCES and max_m <=
 * VSBPP_NOALLOC_MAX_ITEMS, else VSBPP_ECAPACITY; other parameters as in
 * vsbpp_pack_batch, a second-heuristic request gives VSBPP_EINVAL.
 * Instances with B_1 > 32767 get status VSBPP_ECAPACITY.
 *
 * The first call on a device looks up the scratch array's device address
 * (with that device current) and keeps it until the process exits; make that
 * first call before any stream capture begins, and make no call after a
 * cudaDeviceReset of that device (the kept address would be stale).
 * `stream` must belong to the current device (else VSBPP_EINVAL).  Every
 * call on a device uses the same scratch: calls whose GPU work may overlap
 * in time (for example on two streams) race and must be ordered by the
 * caller.  Each call clears what must start at zero.  The work counters
 * (vsbpp_counters_*) include this call's work; kernel timing
 * (vsbpp_kernel_timing_*) does not record it.
 */
#define VSBPP_NOALLOC_MAX_INSTANCES 65536
#define VSBPP_NOALLOC_MAX_ITEMS 16384
int vsbpp_pack_batch_noalloc(int64_t N, const int32_t *w_all, const int64_t *w_off,
                             const int32_t *B_all, const int32_t *B_off, int64_t max_m,
                             const vsbpp_params *p,
                             int32_t *bin_of_item_all, int32_t *bin_type_all,
                             int64_t *num_bins, int64_t *total, int32_t *status,
                             void *stream);

/*
 * vsbpp_shard -- split one batch across `world` processes, one per GPU, for
 * the multi-GPU path (instances are independent problems, Section 6.1, so
 * they shard with no collective on the data).  Longest processing time
 * first: instances in decreasing m (equal m: lower index first) each go to
 * the rank holding the fewest items so far (equal: lowest rank).  m is the
 * cost: each membrane system is one warp's chain of m dependent item steps.
 *   w_off[N+1]            host, CSR offsets of the batch
 *   rank_of[N]            out (host): the rank that packs instance i
 *   items_of_rank[world]  out (host, may be NULL): items assigned per rank
 * Host-only and deterministic (every rank computes the same split); no CUDA
 * call.  EINVAL for N < 0, world < 1, null arrays or decreasing offsets.
 */
int vsbpp_shard(int64_t N, const int64_t *w_off, int32_t world, int32_t *rank_of,
                int64_t *items_of_rank);

/*
 * vsbpp_pack_plain -- the same batch, packed the plain way: one kernel launch
 * per instance, one instance after another on `stream`, each launch a single
 * thread block with the per-instance kernel.  Same arguments and results as
 * vsbpp_pack_batch; kept as the baseline the batched path is measured
 * against.
 */
int vsbpp_pack_plain(int64_t N, const int32_t *w_all, const int64_t *w_off,
                     const int32_t *B_all, const int32_t *B_off, int64_t max_m,
                     const vsbpp_params *p,
                     int32_t *bin_of_item_all, int32_t *bin_type_all,
                     int64_t *num_bins, int64_t *total, int32_t *status,
                     void *stream);

/*
 * Work counters (tracing).  While enabled, the first-heuristic kernels and
 * the second heuristic's register kernel (no pre-opened bins) add to two
 * device counters: the items they pack, and the fit tests the method
 * performs -- for every item, one per bin membrane alive when it arrives
 * (Rule 4 tests every open bin), whether or not a kernel stops a first-fit
 * scan early; for the second heuristic, summed over every permutation each
 * sublist tries (Section 6.4).  Enabling affects launches made (or plans
 * recorded) afterwards.  vsbpp_counters_read synchronises the device, copies
 * the counters and, if reset != 0, sets them back to zero.
 */
typedef struct {
    uint64_t items;
    uint64_t fit_tests;
} vsbpp_counters;

int vsbpp_counters_enable(int enable);
int vsbpp_counters_read(vsbpp_counters *out, int reset);

/*
 * Kernel timing (measurement).  While enabled, every vsbpp_pack_batch call
 * made on a stream that is not capturing records a CUDA event pair on that
 * stream around its main packing phase: the first-heuristic kernels of the
 * instances held in shared memory (both size classes, from the fork of the
 * second stream to the join), the bounded-space kernel, or the
 * second-heuristic kernel.  Up to 256 pairs are kept (the oldest are overwritten).
 * vsbpp_kernel_timing_read waits for the recorded pairs, writes up to `max`
 * durations in milliseconds to ms[] (oldest first), their number to *count,
 * and forgets them.  Enabling or disabling also forgets them.
 * Errors: EINVAL for a null count or a null ms with max > 0; ECUDA.
 */
int vsbpp_kernel_timing_enable(int enable);
int vsbpp_kernel_timing_read(float *ms, int32_t max, int32_t *count);

/*
 * Plans: a batch shape recorded once into a CUDA graph and replayed.
 *
 * vsbpp_plan_create fixes N, an upper bound total_m >= w_off[N], max_m and
 * the parameters, allocates all scratch memory, and picks the launch
 * configuration (thread-group size per size class, items staged per step)
 * from the autotuner's table.  vsbpp_plan_run records the launch sequence
 * into a CUDA graph the first time it sees a set of pointers and replays the
 * graph on `stream` afterwards (new pointers re-record).  It never allocates;
 * called while `stream` is itself being captured, it adds the launches to the
 * caller's graph directly instead of replaying its own.
 */
typedef struct vsbpp_plan vsbpp_plan;
int vsbpp_plan_create(int64_t N, int64_t total_m, int64_t max_m, const vsbpp_params *p,
                      vsbpp_plan **out);
int vsbpp_plan_run(vsbpp_plan *plan, const int32_t *w_all, const int64_t *w_off,
                   const int32_t *B_all, const int32_t *B_off,
                   int32_t *bin_of_item_all, int32_t *bin_type_all,
                   int64_t *num_bins, int64_t *total, int32_t *status, void *stream);
int vsbpp_plan_destroy(vsbpp_plan *plan);

/*
 * Launch configuration and autotuner.
 *
 * The batched first-heuristic kernel runs thread groups of `warps` warps per
 * instance; in batched calls (device or host memory) and plans, instances
 * with m <= small_m go to single-warp groups whose bin slots are sized for
 * small_m, launched on a second stream beside the larger instances' launch
 * (their blocks take the shared memory the larger ones' warps give back as
 * their queue runs dry).  Single-instance calls pack their instance in the
 * larger groups.  The autotuner times candidate
 * configurations on the caller's batch (device CSR arrays as in
 * vsbpp_pack_batch; the outputs are scratch it may overwrite) and installs
 * the fastest for the batch's heuristic; vsbpp_tune_save/load keep the table
 * in a small JSON file.
 */
typedef struct {
    int32_t large_warps;    /* warps per group for instances with m > small_m (1..32, power of 2) */
    int32_t small_m;        /* instances at or below this size use one warp each (>= 0)           */
    int32_t small_warps_per_block; /* warps per thread block in the single-warp kernel (1, 2, 4,
                               8 or 16)                                                      */
    int32_t chunk;          /* items staged in shared memory per step (multiple of 32)            */
    int32_t slot_pct;       /* bin slots per membrane system in the shared-memory kernels, as a
                               percentage of its items (+64); 200 = the worst case (every item
                               can create two bins).  A system that outgrows its slots is packed
                               again from the start by a worst-case-sized launch, so the result
                               never depends on this value (50..200)                           */
    int32_t h2_blocks_per_sm; /* second heuristic: resident blocks per SM at most (0 = as many as
                               fit; fewer leaves room for work running beside it on another
                               stream, e.g. first-heuristic passes) (0..32)                    */
} vsbpp_config;

int vsbpp_get_config(vsbpp_config *out);
int vsbpp_set_config(const vsbpp_config *cfg);
int vsbpp_autotune(int64_t N, const int32_t *w_all, const int64_t *w_off,
                   const int32_t *B_all, const int32_t *B_off, int64_t max_m,
                   const vsbpp_params *p,
                   int32_t *bin_of_item_all, int32_t *bin_type_all,
                   int64_t *num_bins, int64_t *total, int32_t *status,
                   void *stream, vsbpp_config *best, double *best_ms);
int vsbpp_tune_save(const char *path);
int vsbpp_tune_load(const char *path);

/*
 * Serving: continuous batching of packing requests.
 *
 * vsbpp_server_create starts a server that keeps request state resident on
 * the device.  A request is admitted when a slot is free and its device
 * memory (an upper bound from m and n) fits within device_mem_budget bytes;
 * admitted requests are packed by the same kernels while other requests are
 * in flight, on `lanes` concurrent streams.  Requests submitted while the GPU
 * is busy wait in a host queue until slots and memory free up.
 *
 *   vsbpp_server_submit copies the request (host pointers) and returns a
 *     ticket at once; VSBPP_EBUSY when the host queue is full (max_queued
 *     waiting requests), VSBPP_ECAPACITY when the request alone needs more
 *     device memory than the whole budget.  A request holds
 *     12*m + 4*n bytes (rounded up to 256-byte blocks) plus 256 bytes of
 *     device memory while admitted, on top of the library's per-lane scratch.
 *   vsbpp_server_poll waits up to timeout_us microseconds (0: do not wait,
 *     < 0: wait without limit) for the ticket and copies the result into the
 *     host buffers; VSBPP_ETIMEDOUT if it is not finished in time.  A ticket
 *     is released by the poll that returns its result.
 *   vsbpp_server_stats reports completed requests and latency percentiles
 *     over the last completed requests, in microseconds: submit to
 *     completion, and its two parts -- the wait in the host queue (submit to
 *     admission) and the service time (admission to completion).
 */
typedef struct vsbpp_server vsbpp_server;
typedef struct {
    int64_t completed;
    int64_t items_packed;
    double  p50_us, p99_us, max_us;        /* submit to completion                          */
    double  busy_s;          /* seconds from the first admission to the last completion */
    double  wait_p50_us, wait_p99_us;      /* submit to admission (queueing)                */
    double  service_p50_us, service_p99_us;  /* admission to completion (copies + packing)  */
} vsbpp_server_stats_t;

int vsbpp_server_create(size_t device_mem_budget, int32_t max_slots, int32_t lanes,
                        int32_t max_queued, vsbpp_server **out);
int vsbpp_server_submit(vsbpp_server *srv, const int32_t *w, int64_t m,
                        const int32_t *B, int32_t n, const vsbpp_params *p,
                        uint64_t *ticket);
int vsbpp_server_poll(vsbpp_server *srv, uint64_t ticket,
                      int32_t *bin_of_item, int32_t *bin_type,
                      int64_t *num_bins, int64_t *total_capacity,
                      int64_t timeout_us);
int vsbpp_server_stats(vsbpp_server *srv, vsbpp_server_stats_t *out);
int vsbpp_server_destroy(vsbpp_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* VSBPP_H */
