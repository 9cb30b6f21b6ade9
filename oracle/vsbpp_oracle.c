/*
 * vsbpp_oracle.c -- plain, slow, single-threaded CPU oracle for the hybrid
 * P-system heuristics of Alenezi, Aboelfotoh, Albdaiwi & Almulla,
 * "Heuristics for the Variable Sized Bin Packing Problem Using a Hybrid
 * P System and CUDA Architecture" (arXiv:1602.08735).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header or constant table with
 * the CUDA path: every constant below is restated here on purpose.
 *
 * What it computes (one function per passage of the paper):
 *   - the VSBPP instance and objective (Section 1 "Formal Definition",
 *     Section 6.1): items w_1..w_m, bin types B_1 > ... > B_n > 0, unlimited
 *     supply, minimise the total capacity of the used bins;
 *   - Rule 1 / step 1 of Section 6.3: the item list is split into sublists;
 *     each sublist is an independent membrane system with its own bins
 *     (Rule 2 gives every thread its own bin membranes);
 *   - Rules 3-6 of Section 6.3: items leave the sublist one per step, are
 *     tagged with a criterion FF/BF/WF (Section 1 defines the three), enter
 *     the chosen bin membrane (Rule 4, whose polarity is the bin load), and a
 *     bin whose load reaches half its capacity divides off one empty bin of
 *     the same type (Rule 5);
 *   - Section 6.4: the second heuristic packs every permutation of each small
 *     sublist and keeps the cheapest (ties: lowest permutation index);
 *   - the "second kernel" of Section 7: total capacity of used bins.
 *
 * Readings taken where the paper is silent or garbled (each restated next to
 * the code that implements it):
 *   G1  sublists are contiguous chunks of the list, in list order;
 *   G2  items leave a sublist in list order, one per step;
 *   G3  by default no bin is open at the start; preopen=1 gives the literal
 *       Rule 2 (one empty bin of each type, types in order);
 *   G4  when no open bin has room, a bin of the smallest type that holds the
 *       item is opened and appended (the paper has no rule for this case);
 *   G5  Rule 4 fit test: residual capacity >= w (Remark 2 of Section 6.3);
 *   G6  ties in FF/BF/WF go to the lowest creation index (Section 1);
 *   G7  Rule 5 fires once per bin, when 2*load first reaches >= B (real half);
 *       with flag ORACLE_REMARK3 it fires only if, in addition, every bin of
 *       that type now holds at least half its capacity -- Remark 3 of Section
 *       6.3 read as a condition (a consequence of Rule 5 under the literal
 *       Rule 2, but not once G4 can open bins below half);
 *   G8  "used" bins are those with load > 0; bin ids are dense in creation
 *       order among used bins, sublists concatenated in order;
 *   G9  permutations are enumerated in lexicographic order of positions,
 *       rank 0 = identity;
 *   G10 ties between permutations go to the lowest rank;
 *   G15 (bounded-space variant, Section 1: FF / BF / WF keep a given number
 *       of bins active, and a bin is closed when it is completely filled)
 *       with max_open = K >= 1: only active (open) bin membranes take part
 *       in Rule 4's fit test; a bin closes as soon as its residual reaches
 *       0; whenever a bin must be created (an item that fits no open bin,
 *       a Rule 5 division, or a Rule 2 bin) while K bins are open, the open
 *       bin with the lowest creation index closes first.  Closed bins keep
 *       their items and still count toward the objective.  K = 0 means no
 *       bound (the method as above, nothing ever closes).  First heuristic
 *       only; not combined with Remark 3;
 *   G16 (offline pre-sort, the decreasing order of FFD/BFD that Section 5's
 *       prior work uses) with flag ORACLE_PRESORT: the item list is sorted
 *       by non-increasing weight, ties kept in list order, before Rule 1;
 *       the sorted list is then packed exactly as a caller-given list would
 *       be (RANDOM keys are sorted positions), and each item's bin id is
 *       reported at the item's original position;
 *   G12 the RANDOM criterion draws c = SplitMix64(seed, key) mod 3 with
 *       0=FF, 1=BF, 2=WF; key = item index (first heuristic) or
 *       (sublist*720 + rank)*8 + step (second heuristic, s <= 6), or
 *       (sublist*12! + rank)*16 + step (s = 7..12, the exhaustive search of
 *       Section 7's parallel comparison), s being the run's sublist size
 *       whatever the length of a particular sublist (an instance shorter
 *       than s, or its last sublist).  SplitMix64 is the
 *       published generator of Steele, Lea & Flood (OOPSLA 2014): the
 *       key-th output (0-based) of the stream seeded with `seed`.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* status codes (same numeric values as the library's public interface) */
#define OR_OK       0
#define OR_EINVAL  (-1)
#define OR_ETOOBIG (-2)
#define OR_ENOMEM  (-3)

/* criteria and heuristics */
#define OR_FF 0
#define OR_BF 1
#define OR_WF 2
#define OR_RANDOM 3
#define OR_H1 1
#define OR_H2 2

/* flags of oracle_pack_flags / oracle_pack_ext */
#define ORACLE_REMARK3 1       /* G7 with Remark 3's per-type condition */
#define ORACLE_PRESORT 2       /* G16: non-increasing weight order before packing */

#define OR_H2_DEFAULT_SUBLIST 5
#define OR_H2_MAX_SUBLIST 12   /* s <= 6: Section 6.4; up to 12: Section 7's exhaustive search */
#define OR_FACT12 479001600ull

/* Fit tests of Rule 4 performed by this thread's calls: for every item, one
 * per bin membrane alive when it arrives (summed over every permutation the
 * second heuristic tries).  Read by oracle_fit_tests. */
static _Thread_local uint64_t or_fit_tests;

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea & Flood 2014): state advances by the golden-ratio  */
/* increment; the output is the state passed through the variant-13 mixer.   */
/* The key-th output of the stream seeded with `seed` is therefore the mix of */
/* seed + (key+1)*gamma.                                                      */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t key)
{
    uint64_t z = seed + (key + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static int32_t or_random_criterion(uint64_t seed, uint64_t key)
{
    return (int32_t)(oracle_splitmix64(seed, key) % 3u);
}

/* A bin membrane (b, x, B_type, I) with polarity = load (Rule 4). */
typedef struct {
    int64_t load;
    int32_t type;
} or_bin;

/*
 * One membrane system of Section 6.3 packing the sequence seq[0..k) with the
 * criterion crit[q] for step q.  bins must have room for 2k + n entries (each
 * step appends at most one bin by G4 and one by Rule 5; preopen adds n).
 * raw[q] receives the creation index of the bin that took step q's item.
 * Returns the number of bins created.
 */
/* Remark 3 of Section 6.3: does every bin of type t hold at least half of
 * its capacity? */
static int or_type_all_half(const or_bin *bins, int64_t nb, const int32_t *B, int32_t t)
{
    for (int64_t x = 0; x < nb; ++x)
        if (bins[x].type == t && 2 * bins[x].load < (int64_t)B[t])
            return 0;
    return 1;
}

static int64_t or_membrane_run(const int32_t *seq, const int32_t *crit, int64_t k,
                               const int32_t *B, int32_t n, int32_t preopen,
                               or_bin *bins, int64_t *raw, int32_t remark3)
{
    int64_t nb = 0;
    if (preopen) {                         /* Rule 2 taken literally (G3) */
        for (int32_t i = 0; i < n; ++i) {
            bins[nb].load = 0;
            bins[nb].type = i;
            ++nb;
        }
    }
    for (int64_t q = 0; q < k; ++q) {      /* Rule 3: one item per step (G2) */
        const int64_t w = seq[q];
        const int32_t c = crit[q];
        int64_t chosen = -1;
        int64_t chosen_res = 0;
        /* Rule 4: every bin membrane tests whether w fits (G5); the
         * criterion picks one, lowest creation index on ties (G6). */
        or_fit_tests += (uint64_t)nb;
        for (int64_t x = 0; x < nb; ++x) {
            const int64_t res = (int64_t)B[bins[x].type] - bins[x].load;
            if (res < w)
                continue;
            if (chosen < 0 ||
                (c == OR_BF && res < chosen_res) ||
                (c == OR_WF && res > chosen_res)) {
                chosen = x;
                chosen_res = res;
            }
            if (c == OR_FF)
                break;
        }
        if (chosen < 0) {
            /* G4: nothing fits; open the smallest type whose capacity holds w.
             * Types are sorted by decreasing capacity, so that is the last
             * index i with B[i] >= w. */
            int32_t t = 0;
            for (int32_t i = 0; i < n; ++i)
                if (B[i] >= w)
                    t = i;
            bins[nb].load = 0;
            bins[nb].type = t;
            chosen = nb;
            ++nb;
        }
        {
            const int64_t cap = B[bins[chosen].type];
            const int64_t before = bins[chosen].load;
            const int64_t after = before + w;
            bins[chosen].load = after;     /* Rule 4: polarity k -> k + w */
            /* Rule 5 (G7): the bin divides when its load first reaches half
             * of its capacity, i.e. 2*before < cap <= 2*after. */
            if (2 * before < cap && cap <= 2 * after) {
                if (!remark3 || or_type_all_half(bins, nb, B, bins[chosen].type)) {
                    bins[nb].load = 0;
                    bins[nb].type = bins[chosen].type;
                    ++nb;
                }
            }
        }
        raw[q] = chosen;
    }
    return nb;
}

/* G15: open bin number `at` of the list (creation order) closes. */
static void or_close_at(int64_t *active, int64_t *na, int64_t at)
{
    for (int64_t a = at + 1; a < *na; ++a)
        active[a - 1] = active[a];
    --*na;
}

/* G15: before a bin is created while max_open bins are open, the open bin
 * with the lowest creation index (the first of the list) closes. */
static void or_make_room(int64_t *active, int64_t *na, int64_t max_open)
{
    if (*na >= max_open)
        or_close_at(active, na, 0);
}

/*
 * The bounded-space variant of one membrane system (reading G15): at most
 * max_open bin membranes are active at a time.  active[0..na) lists the open
 * bins by creation index (new bins are appended, so the list stays in
 * creation order and its first entry is the oldest open bin).  Same
 * arguments and result as or_membrane_run; active needs room for max_open
 * entries.
 */
static int64_t or_membrane_run_bounded(const int32_t *seq, const int32_t *crit, int64_t k,
                                       const int32_t *B, int32_t n, int32_t preopen,
                                       or_bin *bins, int64_t *raw, int64_t max_open,
                                       int64_t *active)
{
    int64_t nb = 0, na = 0;
    if (preopen) {                         /* Rule 2 taken literally (G3) */
        for (int32_t i = 0; i < n; ++i) {
            or_make_room(active, &na, max_open);
            bins[nb].load = 0;
            bins[nb].type = i;
            active[na++] = nb;
            ++nb;
        }
    }
    for (int64_t q = 0; q < k; ++q) {      /* Rule 3: one item per step (G2) */
        const int64_t w = seq[q];
        const int32_t c = crit[q];
        int64_t chosen = -1, chosen_at = -1;
        int64_t chosen_res = 0;
        /* Rule 4 over the open bins only, in creation order (G5, G6) */
        or_fit_tests += (uint64_t)na;
        for (int64_t a = 0; a < na; ++a) {
            const int64_t x = active[a];
            const int64_t res = (int64_t)B[bins[x].type] - bins[x].load;
            if (res < w)
                continue;
            if (chosen < 0 ||
                (c == OR_BF && res < chosen_res) ||
                (c == OR_WF && res > chosen_res)) {
                chosen = x;
                chosen_at = a;
                chosen_res = res;
            }
            if (c == OR_FF)
                break;
        }
        if (chosen < 0) {
            /* G4: a bin of the smallest type that holds w, after closing the
             * oldest open bin if max_open are open */
            int32_t t = 0;
            for (int32_t i = 0; i < n; ++i)
                if (B[i] >= w)
                    t = i;
            or_make_room(active, &na, max_open);
            bins[nb].load = 0;
            bins[nb].type = t;
            chosen = nb;
            chosen_at = na;
            active[na++] = nb;
            ++nb;
        }
        {
            const int64_t cap = B[bins[chosen].type];
            const int64_t before = bins[chosen].load;
            const int64_t after = before + w;
            bins[chosen].load = after;     /* Rule 4: polarity k -> k + w */
            if (after == cap)              /* completely filled: the bin closes */
                or_close_at(active, &na, chosen_at);
            /* Rule 5 (G7), after a full bin has closed */
            if (2 * before < cap && cap <= 2 * after) {
                or_make_room(active, &na, max_open);
                bins[nb].load = 0;
                bins[nb].type = bins[chosen].type;
                active[na++] = nb;
                ++nb;
            }
        }
        raw[q] = chosen;
    }
    return nb;
}

/*
 * Objective of Section 1 over one membrane system (G8): dense[x] receives the
 * rank of bin x among used bins in creation order (or -1 when unused).
 * Returns the number of used bins; *cap_sum receives their total capacity.
 */
static int64_t or_used_bins(const or_bin *bins, int64_t nb, const int32_t *B,
                            int64_t *dense, int64_t *cap_sum)
{
    int64_t used = 0, sum = 0;
    for (int64_t x = 0; x < nb; ++x) {
        if (bins[x].load > 0) {
            dense[x] = used++;
            sum += B[bins[x].type];
        } else {
            dense[x] = -1;
        }
    }
    *cap_sum = sum;
    return used;
}

/* Lexicographic successor of a permutation (Narayana Pandita's method).
 * Returns 0 when p is the last permutation. */
static int or_next_permutation(int32_t *p, int32_t k)
{
    int32_t i = k - 2;
    while (i >= 0 && p[i] >= p[i + 1])
        --i;
    if (i < 0)
        return 0;
    int32_t j = k - 1;
    while (p[j] <= p[i])
        --j;
    int32_t t = p[i]; p[i] = p[j]; p[j] = t;
    for (int32_t a = i + 1, b = k - 1; a < b; ++a, --b) {
        t = p[a]; p[a] = p[b]; p[b] = t;
    }
    return 1;
}

/* Validation of the instance and parameters (Section 6.1 assumptions). */
static int or_validate(const int32_t *w, int64_t m, const int32_t *B, int32_t n,
                       int32_t heuristic, int32_t criterion, int64_t sublist_size,
                       int32_t preopen)
{
    if (m < 0 || n < 1 || !B || (m > 0 && !w))
        return OR_EINVAL;
    if (heuristic != OR_H1 && heuristic != OR_H2)
        return OR_EINVAL;
    if (criterion < OR_FF || criterion > OR_RANDOM)
        return OR_EINVAL;
    if (preopen != 0 && preopen != 1)
        return OR_EINVAL;
    if (sublist_size < 0)
        return OR_EINVAL;
    if (heuristic == OR_H2 && sublist_size > OR_H2_MAX_SUBLIST)
        return OR_EINVAL;
    for (int32_t i = 0; i < n; ++i) {
        if (B[i] <= 0)
            return OR_EINVAL;
        if (i > 0 && B[i] >= B[i - 1])
            return OR_EINVAL;          /* B_1 > B_2 > ... > B_n > 0 */
    }
    for (int64_t j = 0; j < m; ++j) {   /* first offending item decides */
        if (w[j] < 1)
            return OR_EINVAL;
        if (w[j] > B[0])
            return OR_ETOOBIG;          /* w_max <= B_1 is assumed */
    }
    return OR_OK;
}

/* G16: one item of the pre-sort, its weight and its position in the list. */
typedef struct {
    int32_t w;
    int64_t pos;
} or_sort_item;

/* Non-increasing weight; equal weights keep their list order. */
static int or_sort_cmp(const void *a, const void *b)
{
    const or_sort_item *x = (const or_sort_item *)a, *y = (const or_sort_item *)b;
    if (x->w != y->w)
        return x->w > y->w ? -1 : 1;
    return x->pos < y->pos ? -1 : (x->pos > y->pos ? 1 : 0);
}

/*
 * Pack one instance.  bin_of_item[m] receives dense bin ids, bin_type[<= m]
 * receives the 0-based type of each used bin (0 = largest capacity).
 * flags: ORACLE_REMARK3 (reading G7 with Remark 3's condition) and/or
 * ORACLE_PRESORT (reading G16).  max_open: 0, or the bound K of the
 * bounded-space variant (reading G15; first heuristic, without Remark 3).
 */
int oracle_pack_ext(const int32_t *w, int64_t m, const int32_t *B, int32_t n,
                    int32_t heuristic, int32_t criterion, int64_t sublist_size,
                    int32_t preopen, uint64_t seed, int32_t flags, int64_t max_open,
                    int32_t *bin_of_item, int32_t *bin_type,
                    int64_t *num_bins, int64_t *total_capacity)
{
    if (num_bins) *num_bins = 0;
    if (total_capacity) *total_capacity = 0;
    int rc = or_validate(w, m, B, n, heuristic, criterion, sublist_size, preopen);
    if (rc != OR_OK)
        return rc;
    if (flags & ~(ORACLE_REMARK3 | ORACLE_PRESORT))
        return OR_EINVAL;
    const int32_t remark3 = (flags & ORACLE_REMARK3) ? 1 : 0;
    if (max_open < 0 || (max_open > 0 && (heuristic != OR_H1 || remark3)))
        return OR_EINVAL;
    if (m == 0)
        return OR_OK;

    if (flags & ORACLE_PRESORT) {
        /* G16: pack the list sorted by non-increasing weight (stable), then
         * report each item's bin at its original position */
        or_sort_item *it = (or_sort_item *)malloc(sizeof(or_sort_item) * (size_t)m);
        int32_t *ws = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
        int32_t *bs = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
        if (!it || !ws || !bs) {
            free(it); free(ws); free(bs);
            return OR_ENOMEM;
        }
        for (int64_t j = 0; j < m; ++j) {
            it[j].w = w[j];
            it[j].pos = j;
        }
        qsort(it, (size_t)m, sizeof(or_sort_item), or_sort_cmp);
        for (int64_t j = 0; j < m; ++j)
            ws[j] = it[j].w;
        rc = oracle_pack_ext(ws, m, B, n, heuristic, criterion, sublist_size, preopen, seed,
                             flags & ~ORACLE_PRESORT, max_open, bs, bin_type, num_bins,
                             total_capacity);
        if (rc == OR_OK)
            for (int64_t j = 0; j < m; ++j)
                bin_of_item[it[j].pos] = bs[j];
        free(it); free(ws); free(bs);
        return rc;
    }

    int64_t s;
    if (heuristic == OR_H1)
        s = sublist_size == 0 ? m : sublist_size;        /* default: one system */
    else
        s = sublist_size == 0 ? OR_H2_DEFAULT_SUBLIST : sublist_size;
    /* G12: the RANDOM key layout follows the run's sublist size, also for an
     * instance shorter than it */
    const int64_t s_run = s;
    if (s > m)
        s = m;

    const int64_t bin_room = 2 * s + n;
    or_bin *bins = (or_bin *)malloc(sizeof(or_bin) * (size_t)bin_room);
    int64_t *raw = (int64_t *)malloc(sizeof(int64_t) * (size_t)s);
    int64_t *dense = (int64_t *)malloc(sizeof(int64_t) * (size_t)bin_room);
    int32_t *seq = (int32_t *)malloc(sizeof(int32_t) * (size_t)s);
    int32_t *crit = (int32_t *)malloc(sizeof(int32_t) * (size_t)s);
    int64_t *best_item_bin = (int64_t *)malloc(sizeof(int64_t) * (size_t)s);
    int32_t *best_types = (int32_t *)malloc(sizeof(int32_t) * (size_t)bin_room);
    int64_t *active = max_open > 0 ? (int64_t *)malloc(sizeof(int64_t) * (size_t)max_open) : NULL;
    if (!bins || !raw || !dense || !seq || !crit || !best_item_bin || !best_types ||
        (max_open > 0 && !active)) {
        free(bins); free(raw); free(dense); free(seq); free(crit);
        free(best_item_bin); free(best_types); free(active);
        return OR_ENOMEM;
    }

    int64_t bin_offset = 0;      /* bins of earlier sublists (G11) */
    int64_t total = 0;
    for (int64_t g = 0; g * s < m; ++g) {
        const int64_t a = g * s;
        const int64_t k = (m - a < s) ? (m - a) : s;
        if (heuristic == OR_H1) {
            for (int64_t q = 0; q < k; ++q) {
                seq[q] = w[a + q];
                crit[q] = criterion == OR_RANDOM
                              ? or_random_criterion(seed, (uint64_t)(a + q))
                              : criterion;
            }
            const int64_t nb = max_open > 0
                ? or_membrane_run_bounded(seq, crit, k, B, n, preopen, bins, raw, max_open, active)
                : or_membrane_run(seq, crit, k, B, n, preopen, bins, raw, remark3);
            int64_t cap_sum = 0;
            const int64_t used = or_used_bins(bins, nb, B, dense, &cap_sum);
            for (int64_t q = 0; q < k; ++q)
                bin_of_item[a + q] = (int32_t)(bin_offset + dense[raw[q]]);
            for (int64_t x = 0; x < nb; ++x)
                if (dense[x] >= 0)
                    bin_type[bin_offset + dense[x]] = bins[x].type;
            bin_offset += used;
            total += cap_sum;
        } else {
            /* Section 6.4: every permutation of the sublist packs with
             * Rules 2-6; the cheapest one wins, lowest rank on ties. */
            int32_t perm[OR_H2_MAX_SUBLIST];
            for (int32_t q = 0; q < (int32_t)k; ++q)
                perm[q] = q;
            int64_t best_total = -1, best_used = 0;
            int64_t rank = 0;
            do {
                for (int64_t q = 0; q < k; ++q) {
                    seq[q] = w[a + perm[q]];
                    crit[q] = criterion == OR_RANDOM
                                  ? or_random_criterion(
                                        seed, s_run <= 6
                                                  ? (uint64_t)((g * 720 + rank) * 8 + q)
                                                  : ((uint64_t)g * OR_FACT12 + (uint64_t)rank) * 16u + (uint64_t)q)
                                  : criterion;
                }
                const int64_t nb = or_membrane_run(seq, crit, k, B, n, preopen, bins, raw, remark3);
                int64_t cap_sum = 0;
                const int64_t used = or_used_bins(bins, nb, B, dense, &cap_sum);
                if (best_total < 0 || cap_sum < best_total) {
                    best_total = cap_sum;
                    best_used = used;
                    for (int64_t q = 0; q < k; ++q)
                        best_item_bin[perm[q]] = dense[raw[q]];
                    for (int64_t x = 0; x < nb; ++x)
                        if (dense[x] >= 0)
                            best_types[dense[x]] = bins[x].type;
                }
                ++rank;
            } while (or_next_permutation(perm, (int32_t)k));
            for (int64_t q = 0; q < k; ++q)
                bin_of_item[a + q] = (int32_t)(bin_offset + best_item_bin[q]);
            for (int64_t d = 0; d < best_used; ++d)
                bin_type[bin_offset + d] = best_types[d];
            bin_offset += best_used;
            total += best_total;
        }
    }

    free(bins); free(raw); free(dense); free(seq); free(crit);
    free(best_item_bin); free(best_types); free(active);
    if (num_bins) *num_bins = bin_offset;
    if (total_capacity) *total_capacity = total;
    return OR_OK;
}

/* oracle_pack_ext without the bounded-space variant (max_open = 0). */
int oracle_pack_flags(const int32_t *w, int64_t m, const int32_t *B, int32_t n,
                      int32_t heuristic, int32_t criterion, int64_t sublist_size,
                      int32_t preopen, uint64_t seed, int32_t flags,
                      int32_t *bin_of_item, int32_t *bin_type,
                      int64_t *num_bins, int64_t *total_capacity)
{
    return oracle_pack_ext(w, m, B, n, heuristic, criterion, sublist_size, preopen, seed, flags, 0,
                           bin_of_item, bin_type, num_bins, total_capacity);
}

/* oracle_pack_flags with flags = 0: the readings G1-G12 as stated above. */
int oracle_pack(const int32_t *w, int64_t m, const int32_t *B, int32_t n,
                int32_t heuristic, int32_t criterion, int64_t sublist_size,
                int32_t preopen, uint64_t seed,
                int32_t *bin_of_item, int32_t *bin_type,
                int64_t *num_bins, int64_t *total_capacity)
{
    return oracle_pack_flags(w, m, B, n, heuristic, criterion, sublist_size, preopen, seed, 0,
                             bin_of_item, bin_type, num_bins, total_capacity);
}

/*
 * The number of Rule 4 fit tests (one per bin membrane alive when an item
 * arrives; every permutation counted for the second heuristic) that
 * oracle_pack performs for this instance.  Returns 0 on invalid input.
 */
uint64_t oracle_fit_tests_ext(const int32_t *w, int64_t m, const int32_t *B, int32_t n,
                              int32_t heuristic, int32_t criterion, int64_t sublist_size,
                              int32_t preopen, uint64_t seed, int32_t flags, int64_t max_open)
{
    int32_t *boi = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    int32_t *bt = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    if (!boi || !bt) {
        free(boi); free(bt);
        return 0;
    }
    or_fit_tests = 0;
    int64_t nb = 0, tot = 0;
    const int rc = oracle_pack_ext(w, m, B, n, heuristic, criterion, sublist_size, preopen, seed,
                                   flags, max_open, boi, bt, &nb, &tot);
    free(boi); free(bt);
    return rc == OR_OK ? or_fit_tests : 0;
}

uint64_t oracle_fit_tests(const int32_t *w, int64_t m, const int32_t *B, int32_t n,
                          int32_t heuristic, int32_t criterion, int64_t sublist_size,
                          int32_t preopen, uint64_t seed)
{
    return oracle_fit_tests_ext(w, m, B, n, heuristic, criterion, sublist_size, preopen, seed, 0, 0);
}

/*
 * Exact VSBPP optimum (Section 1 "Formal Definition") by dynamic programming
 * over item subsets: a packing is a partition of the items into groups, each
 * group costing the smallest capacity B_i that holds its weight.  With
 * f(S) = min over groups T containing the lowest item of S of
 * cap(sum T) + f(S \ T), OPT = f(all items).  O(3^m); m <= 20 accepted.
 * Returns -1 on invalid input.
 */
int64_t oracle_opt_bruteforce(const int32_t *w, int32_t m, const int32_t *B, int32_t n)
{
    if (m < 0 || m > 20 || n < 1)
        return -1;
    if (m == 0)
        return 0;
    const uint32_t full = (1u << m) - 1u;
    int64_t *sum = (int64_t *)malloc(sizeof(int64_t) * ((size_t)full + 1));
    int64_t *cap = (int64_t *)malloc(sizeof(int64_t) * ((size_t)full + 1));
    int64_t *f = (int64_t *)malloc(sizeof(int64_t) * ((size_t)full + 1));
    if (!sum || !cap || !f) {
        free(sum); free(cap); free(f);
        return -1;
    }
    sum[0] = 0;
    for (uint32_t S = 1; S <= full; ++S) {
        uint32_t low = S & (~S + 1u);
        int32_t bit = 0;
        while ((1u << bit) != low)
            ++bit;
        sum[S] = sum[S ^ low] + w[bit];
    }
    for (uint32_t S = 0; S <= full; ++S) {
        cap[S] = -1;                            /* -1: no type holds it */
        for (int32_t i = n - 1; i >= 0; --i) {  /* smallest capacity first */
            if ((int64_t)B[i] >= sum[S]) {
                cap[S] = B[i];
                break;
            }
        }
    }
    const int64_t INF = INT64_MAX / 4;
    f[0] = 0;
    for (uint32_t S = 1; S <= full; ++S) {
        const uint32_t low = S & (~S + 1u);
        const uint32_t rest = S ^ low;
        int64_t best = INF;
        uint32_t sub = rest;
        for (;;) {
            const uint32_t T = sub | low;
            if (cap[T] > 0 && f[S ^ T] < INF) {
                const int64_t v = cap[T] + f[S ^ T];
                if (v < best)
                    best = v;
            }
            if (sub == 0)
                break;
            sub = (sub - 1u) & rest;
        }
        f[S] = best;
    }
    const int64_t out = f[full] >= INF ? -1 : f[full];
    free(sum); free(cap); free(f);
    return out;
}
