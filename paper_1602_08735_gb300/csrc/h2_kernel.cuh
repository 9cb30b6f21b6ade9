// h2_kernel.cuh -- the second heuristic of Section 6.4.
//
// Each sublist of k <= 6 items is one thread block's job; thread r packs the
// permutation of lexicographic rank r (rank 0 = list order) with Rules 2-6,
// exactly as the first heuristic packs a sublist, on its own bin membranes.
// The block then takes the permutation with the smallest total capacity, the
// lowest rank winning ties, and that thread writes the sublist's result in
// sublist-local form (bin ids from 0, types, count, capacity); the compose
// pass concatenates sublists.  A thread's bins live in shared memory laid out
// bin-major ([bin][thread]) so a block's threads touch consecutive words.
#pragma once

#include "h2_params.cuh"

namespace vsbpp {

__device__ __forceinline__ int h2_factorial(int k) {
    int f = 1;
    for (int x = 2; x <= k; ++x) f *= x;
    return f;
}

__global__ void h2_pack_kernel(const H2Params p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int T = static_cast<int>(blockDim.x);
    const int tid = static_cast<int>(threadIdx.x);
    const int lane = tid & 31, warp = tid >> 5, nwarps = T >> 5;
    uint32_t* res = reinterpret_cast<uint32_t*>(smem);                   // [max_bins][T]
    uint8_t* typ = smem + static_cast<size_t>(p.max_bins) * T * 4;        // [max_bins][T]
    unsigned long long* wbest =
        reinterpret_cast<unsigned long long*>(smem + static_cast<size_t>(p.max_bins) * T * 5);
    wbest = reinterpret_cast<unsigned long long*>((reinterpret_cast<uintptr_t>(wbest) + 7) & ~uintptr_t(7));

    int64_t u_begin = 0, u_end = p.units.unit_base[p.in.N];
    if (p.only_instance >= 0) {
        u_begin = p.units.unit_base[p.only_instance];
        u_end = p.units.unit_base[p.only_instance + 1];
    }
    for (int64_t uid = u_begin + blockIdx.x; uid < u_end; uid += gridDim.x) {
        const int64_t i = p.units.instance_of(uid, p.in.N);
        if (p.out.status[i] != VSBPP_OK) continue;
        const int64_t m = p.in.m(i);
        const int64_t g = uid - p.units.unit_base[i];
        const int64_t a = g * p.sublist;
        const int k = static_cast<int>((m - a) < p.sublist ? (m - a) : p.sublist);
        const int nperm = h2_factorial(k);
        const int64_t wb = p.in.w_begin(i);
        const int32_t* w = p.in.w_all + wb + a;
        const int32_t n = p.in.n(i);
        const int32_t* B = p.in.B_all + p.in.B_begin(i);
        const uint32_t Bl = lane < n ? static_cast<uint32_t>(B[lane]) : 0u;

        unsigned long long key = ~0ull;
        int perm[6];
        int raw[6];
        int L = 0;
        const bool active = tid < nperm;
        if (active) {
            // lexicographic rank -> permutation (factorial number system)
            int rem = tid;
            unsigned used = 0;
            for (int q = 0; q < k; ++q) {
                const int f = h2_factorial(k - 1 - q);
                int d = rem / f;
                rem -= d * f;
                int x = 0;
                for (;; ++x) {
                    if (!(used & (1u << x))) {
                        if (d == 0) break;
                        --d;
                    }
                }
                used |= 1u << x;
                perm[q] = x;
            }
            if (p.preopen) {
                for (int t = 0; t < n; ++t) {
                    res[t * T + tid] = static_cast<uint32_t>(B[t]);
                    typ[t * T + tid] = static_cast<uint8_t>(t);
                }
                L = n;
            }
            for (int q = 0; q < k; ++q) {
                const uint32_t wj = static_cast<uint32_t>(w[perm[q]]);
                const int c = pick_criterion(p.criterion, p.seed,
                                             static_cast<uint64_t>((g * 720 + tid) * 8 + q));
                int chosen = -1;
                uint32_t chosen_r = 0;
                for (int x = 0; x < L; ++x) {                 // Rule 4 fit test
                    const uint32_t r = res[x * T + tid];
                    if (r < wj) continue;
                    if (chosen < 0 || (c == kBF && r < chosen_r) || (c == kWF && r > chosen_r)) {
                        chosen = x;
                        chosen_r = r;
                    }
                    if (c == kFF) break;
                }
                uint32_t t;
                if (chosen < 0) {                             // smallest type holding w
                    t = 0;
                    for (int x = 0; x < n; ++x)
                        if (static_cast<uint32_t>(B[x]) >= wj) t = static_cast<uint32_t>(x);
                    chosen = L++;
                    chosen_r = static_cast<uint32_t>(B[t]);
                    res[chosen * T + tid] = chosen_r;
                    typ[chosen * T + tid] = static_cast<uint8_t>(t);
                } else {
                    t = typ[chosen * T + tid];
                }
                const uint64_t Bt = static_cast<uint32_t>(B[t]);
                const uint64_t r_old = chosen_r, r_new = chosen_r - wj;
                res[chosen * T + tid] = static_cast<uint32_t>(r_new);
                bool fire = Bt < 2 * r_old && 2 * r_new <= Bt;       // Rule 5
                if (fire && p.remark3) {
                    // Remark 3: every bin of type t must now hold at least half
                    for (int x = 0; x < L; ++x)
                        fire = fire && !(typ[x * T + tid] == t && Bt < 2ull * res[x * T + tid]);
                }
                if (fire) {
                    res[L * T + tid] = static_cast<uint32_t>(Bt);
                    typ[L * T + tid] = static_cast<uint8_t>(t);
                    ++L;
                }
                raw[q] = chosen;
            }
            uint64_t tot = 0;
            for (int x = 0; x < L; ++x) {
                const uint32_t cap = static_cast<uint32_t>(B[typ[x * T + tid]]);
                if (res[x * T + tid] < cap) tot += cap;
            }
            key = (static_cast<unsigned long long>(tot) << 10) | static_cast<unsigned long long>(tid);
        }
        (void)Bl;
        key = warp_min_u64(key);
        if (lane == 0) wbest[warp] = key;
        __syncthreads();
        unsigned long long best = ~0ull;
        for (int x = 0; x < nwarps; ++x) best = wbest[x] < best ? wbest[x] : best;
        const int winner = static_cast<int>(best & 1023ull);
        if (active && tid == winner) {
            // dense ids of used bins in creation order; results in sublist-local form
            int dense[2 * 6 + kMaxTypes];
            int cnt = 0;
            for (int x = 0; x < L; ++x) {
                const int t = typ[x * T + tid];
                if (res[x * T + tid] < static_cast<uint32_t>(B[t])) {
                    dense[x] = cnt;
                    p.out.local_types[wb + a + cnt] = t;
                    ++cnt;
                } else {
                    dense[x] = -1;
                }
            }
            for (int q = 0; q < k; ++q) p.out.bin_of_item[wb + a + perm[q]] = dense[raw[q]];
            p.out.unit_count[uid] = cnt;
            p.out.unit_total[uid] = static_cast<int64_t>(best >> 10);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Register version (no preopen): the sublist size S is a compile-time
// constant, so every loop below has a constant trip count -- at step q at
// most 2q bins exist -- and one thread's bins, permutation and assignment
// stay in registers.  Capacities and each item's fallback type (the smallest
// type holding it) are staged in shared memory once per sublist.
__device__ __forceinline__ int h2_fact_small(int v) {
    return v <= 1 ? 1 : v == 2 ? 2 : v == 3 ? 6 : v == 4 ? 24 : v == 5 ? 120 : 720;
}

// Permutation of lexicographic rank `rank` over k <= S positions.
template <int S>
__device__ __forceinline__ void h2_decode(int rank, int k, int (&perm)[S]) {
    unsigned used = 0;
#pragma unroll
    for (int q = 0; q < S; ++q) {
        perm[q] = 0;
        if (q < k) {
            const int f = h2_fact_small(k - 1 - q);
            int d = rank / f;
            rank -= d * f;
            int x = 0;
#pragma unroll
            for (int y = S - 1; y >= 0; --y) {       // the d-th unused index, ascending
                if (y < k && !((used >> y) & 1u)) {
                    int below = 0;
#pragma unroll
                    for (int z = 0; z < S; ++z)
                        if (z < y && z < k && !((used >> z) & 1u)) ++below;
                    if (below == d) x = y;
                }
            }
            used |= 1u << x;
            perm[q] = x;
        }
    }
}

// ---------------------------------------------------------------------------
// Register kernel (no pre-opened bins): one warp per sublist.
//
// Lane l of the warp packs the permutations of rank l, l+32, ... (rounds of
// 32), keeping the best (least total, then least rank) it has seen; one warp
// minimum names the winner, whose lane writes the sublist's result.  No block
// barrier is taken per sublist.  A lane's bins are fixed slots: the bin
// opened at item step q (nothing fits) is slot 2q and the bin divided off at
// step q (Rule 5) is slot 2q+1, so slot order is creation order and a new
// bin's slot is known at compile time; a slot never created reads as an
// empty word that never fits and is never used.
//
// Capacities <= 2047 and n <= 16 (narrow): one word per slot, v =
// (residual << 20) | (slot << 16) | (type << 12) | capacity, so each
// selection is one operation pair per slot
//   FF  the lowest fitting slot (v >= w << 20),
//   BF  min(v - (w << 20)): a slot that does not fit wraps above 2^31,
//   WF  min(v ^ 0xFFF00000): the largest residual, then the lowest slot,
// and the chosen word carries the bin's residual, slot, type and capacity.
// Larger capacities (wide): residual and capacity words per slot, 64-bit
// selection keys.
// Permutations are packed 3 bits per position, one table per sublist
// length k <= S in shared memory (lexicographic rank order).

__host__ __device__ constexpr int h2_fact_c(int v) { return v <= 1 ? 1 : v * h2_fact_c(v - 1); }
__host__ __device__ constexpr int h2_table_size(int S) { return S < 0 ? 0 : h2_fact_c(S) + h2_table_size(S - 1); }
__device__ __forceinline__ int h2_table_off(int k) {      // entries of lengths 0 .. k-1
    return k <= 0 ? 0 : k == 1 ? 1 : k == 2 ? 2 : k == 3 ? 4 : k == 4 ? 10 : k == 5 ? 34 : 154;
}

// Minimum of t[0..cnt) (cnt a compile-time constant after unrolling) as a
// balanced tree; all-ones when cnt = 0.
template <int N>
__device__ __forceinline__ uint32_t h2_min_tree(uint32_t (&t)[N], int cnt) {
#pragma unroll
    for (int x = 0; x < N; ++x) if (x >= cnt) t[x] = 0xFFFFFFFFu;
#pragma unroll
    for (int step = 1; step < N; step *= 2) {
#pragma unroll
        for (int x = 0; x + step < N; x += 2 * step) t[x] = min(t[x], t[x + step]);
    }
    return t[0];
}

// Pack one permutation, narrow slot words.  Returns the used capacity (a
// bin's capacity counts from the item that finds it empty); rawp gets the
// slot of the item at step q in bits 4q..4q+3.  K > 0: exactly K items
// Item steps Q0 .. Q1-1 of one permutation, narrow slot words (running
// state: slots v, slot per step rawp, used capacity tot; with COUNT, fit
// tests fit and bins alive).  K > 0: exactly K items (compile time); K = 0:
// k items.
template <int S, int CRIT, int Q0, int Q1, int K, bool COUNT>
__device__ __forceinline__ void h2_steps_narrow(uint32_t perm, int k, const uint32_t* wsub, const uint32_t* bnew,
                                                uint64_t seed, int64_t g, int rank, uint32_t (&v)[2 * S],
                                                uint32_t& rawp, uint32_t& tot, uint32_t& fit, uint32_t& alive) {
    constexpr int kSlots = 2 * S;
    constexpr uint32_t kNo = 0xFFFFFFFFu;
#pragma unroll
    for (int q = Q0; q < Q1; ++q) {
        if (K > 0 ? q < K : q < k) {
            const uint32_t it = (perm >> (3 * q)) & 7u;
            const uint32_t wq = wsub[it], bnp = bnew[it];     // bnp = new bin's (type << 12) | capacity
            const uint32_t bn = bnp & 0xFFFu;
            const uint32_t W = wq << 20;
            const int c = CRIT == kRandom
                              ? pick_criterion(kRandom, seed, static_cast<uint64_t>((g * 720 + rank) * 8 + q))
                              : CRIT;
            uint32_t best;
            bool hit;
            if (c == kFF) {
                best = kNo;
#pragma unroll
                for (int x = 2 * q - 1; x >= 0; --x) best = v[x] >= W ? v[x] : best;
                hit = best != kNo;
            } else if (c == kBF) {
                uint32_t t[kSlots];
#pragma unroll
                for (int x = 0; x < 2 * q; ++x) t[x] = v[x] - W;
                const uint32_t m = h2_min_tree<kSlots>(t, 2 * q);
                hit = m < 0x80000000u;
                best = m + W;
            } else {
                uint32_t t[kSlots];
#pragma unroll
                for (int x = 0; x < 2 * q; ++x) t[x] = v[x] ^ 0xFFF00000u;
                best = h2_min_tree<kSlots>(t, 2 * q) ^ 0xFFF00000u;
                hit = (best >> 20) >= wq;
            }
            const uint32_t xs = hit ? (best >> 16) & 15u : static_cast<uint32_t>(2 * q);
            const uint32_t r_old = hit ? best >> 20 : bn;
            const uint32_t tc = hit ? best & 0xFFFFu : bnp;    // (type << 12) | capacity
            const uint32_t cap = tc & 0xFFFu;
            const uint32_t r_new = r_old - wq;
            const bool fire = (cap < 2u * r_old) && (2u * r_new <= cap);     // Rule 5
            tot += r_old == cap ? cap : 0u;        // the bin's first item: it becomes used
            if (COUNT) {
                fit += alive;
                alive += (hit ? 0u : 1u) + (fire ? 1u : 0u);
            }
#pragma unroll
            for (int x = 0; x < 2 * q; ++x) v[x] = xs == static_cast<uint32_t>(x) ? v[x] - W : v[x];
            v[2 * q] = hit ? 0u : (r_new << 20) | (static_cast<uint32_t>(2 * q) << 16) | tc;
            v[2 * q + 1] = fire ? (cap << 20) | (static_cast<uint32_t>(2 * q + 1) << 16) | tc : 0u;
            rawp |= xs << (4 * q);
        }
    }
}

template <int S, int CRIT, int K, bool COUNT>
__device__ __forceinline__ uint32_t h2_pack_narrow(uint32_t perm, int k, const uint32_t* wsub,
                                                   const uint32_t* bnew, uint64_t seed, int64_t g, int rank,
                                                   uint32_t (&v)[2 * S], uint32_t& rawp, uint32_t& fit) {
#pragma unroll
    for (int x = 0; x < 2 * S; ++x) v[x] = 0u;
    rawp = 0;
    uint32_t tot = 0, alive = 0;
    fit = 0;
    h2_steps_narrow<S, CRIT, 0, S, K, COUNT>(perm, k, wsub, bnew, seed, g, rank, v, rawp, tot, fit, alive);
    return tot;
}

// Pack one permutation, wide slots (residual r[x], capacity c[x]).
template <int S, int CRIT>
__device__ __forceinline__ uint64_t h2_pack_wide(uint32_t perm, int k, const uint32_t* wsub, const uint32_t* bnew,
                                                 uint64_t seed, int64_t g, int rank, uint32_t (&r)[2 * S],
                                                 uint32_t (&cp)[2 * S], uint32_t& rawp, uint32_t& fit) {
    constexpr int kSlots = 2 * S;
    constexpr uint64_t kNo = ~0ull;
#pragma unroll
    for (int x = 0; x < kSlots; ++x) { r[x] = 0u; cp[x] = 0u; }
    rawp = 0;
    fit = 0;
    uint32_t alive = 0;
#pragma unroll
    for (int q = 0; q < S; ++q) {
        if (q < k) {
            const uint32_t it = (perm >> (3 * q)) & 7u;
            const uint32_t wq = wsub[it], bn = bnew[it];
            const int c = CRIT == kRandom
                              ? pick_criterion(kRandom, seed, static_cast<uint64_t>((g * 720 + rank) * 8 + q))
                              : CRIT;
            uint64_t key = kNo;                // (measure << 4) | slot, least wins
#pragma unroll
            for (int x = 0; x < 2 * q; ++x) {
                const bool fit = r[x] >= wq;
                const uint64_t m = c == kFF ? 0ull : c == kBF ? static_cast<uint64_t>(r[x] - wq)
                                                              : static_cast<uint64_t>(~r[x]);
                const uint64_t kx = (m << 4) | static_cast<uint64_t>(x);
                key = fit && kx < key ? kx : key;
            }
            const bool hit = key != kNo;
            const uint32_t xs = hit ? static_cast<uint32_t>(key & 15ull) : static_cast<uint32_t>(2 * q);
            uint32_t r_old = bn, cap = bn;
#pragma unroll
            for (int x = 0; x < 2 * q; ++x) {
                r_old = xs == static_cast<uint32_t>(x) ? r[x] : r_old;
                cap = xs == static_cast<uint32_t>(x) ? cp[x] : cap;
            }
            const uint32_t r_new = r_old - wq;
            const bool fire = (static_cast<uint64_t>(cap) < 2ull * r_old) &&
                              (2ull * r_new <= static_cast<uint64_t>(cap));     // Rule 5
            fit += alive;                      // Rule 4 fit tests (counters)
            alive += (hit ? 0u : 1u) + (fire ? 1u : 0u);
#pragma unroll
            for (int x = 0; x < 2 * q; ++x) r[x] = xs == static_cast<uint32_t>(x) ? r_new : r[x];
            r[2 * q] = hit ? 0u : r_new;
            cp[2 * q] = hit ? 0u : cap;
            r[2 * q + 1] = fire ? cap : 0u;
            cp[2 * q + 1] = fire ? cap : 0u;
            rawp |= xs << (4 * q);
        }
    }
    uint64_t tot = 0;
#pragma unroll
    for (int x = 0; x < kSlots; ++x) tot += r[x] < cp[x] ? cp[x] : 0u;
    return tot;
}

// The winner's result in sublist-local form: used slots (load > 0) get
// dense ids in slot order (= creation order).
template <int S>
__device__ __forceinline__ void h2_write_winner(const H2Params& p, const uint32_t (&typ)[2 * S],
                                                uint32_t used, uint32_t rawp, uint32_t perm, int k,
                                                int64_t uid, int64_t base, uint64_t total) {
    int cnt = 0;
#pragma unroll
    for (int x = 0; x < 2 * S; ++x) {
        if ((used >> x) & 1u) {
            p.out.local_types[base + cnt] = static_cast<int32_t>(typ[x]);
            ++cnt;
        }
    }
#pragma unroll
    for (int q = 0; q < S; ++q) {
        if (q < k) {
            const uint32_t slot = (rawp >> (4 * q)) & 15u;
            p.out.bin_of_item[base + ((perm >> (3 * q)) & 7u)] = __popc(used & ((1u << slot) - 1u));
        }
    }
    p.out.unit_count[uid] = cnt;
    p.out.unit_total[uid] = static_cast<int64_t>(total);
}

template <int S, int CRIT>
__global__ void __launch_bounds__(128) h2_pack_kernel_reg(const H2Params p) {
    constexpr int kWarps = 4;
    constexpr int kRun = 16;                 // sublists per run
    constexpr int kSlots = 2 * S;
    __shared__ uint32_t permtab[h2_table_size(S)];
    __shared__ uint32_t Bs[kMaxTypes];
    __shared__ uint32_t wrun[kRun * S];
    __shared__ uint32_t brun[kRun * S];
    const int tid = static_cast<int>(threadIdx.x);
    const int lane = tid & 31, warp = tid >> 5;

    // permutation tables: entry off(k) + rank = rank's permutation of k items
    for (int e = tid; e < h2_table_size(S); e += blockDim.x) {
        int k = 0;
        while (k < S && e >= h2_table_off(k + 1)) ++k;
        int perm[S];
        h2_decode<S>(e - h2_table_off(k), k, perm);
        uint32_t packed = 0;
        for (int q = 0; q < k; ++q) packed |= static_cast<uint32_t>(perm[q]) << (3 * q);
        permtab[e] = packed;
    }
    __syncthreads();

    int64_t u_begin = 0, u_end = p.units.unit_base[p.in.N];
    if (p.only_instance >= 0) {
        u_begin = p.units.unit_base[p.only_instance];
        u_end = p.units.unit_base[p.only_instance + 1];
    }
    // Each block takes runs of kRun consecutive sublists (numbered instance
    // by instance), in segments, one per instance a run touches: a segment's
    // items are consecutive in w_all and are staged in shared memory once,
    // each with the capacity of the smallest type holding it; the warps then
    // take the segment's sublists in turn.
    for (int64_t r0 = u_begin + static_cast<int64_t>(blockIdx.x) * kRun; r0 < u_end;
         r0 += static_cast<int64_t>(gridDim.x) * kRun) {
        const int64_t r1 = (r0 + kRun) < u_end ? (r0 + kRun) : u_end;
        int64_t i = p.units.instance_of(r0, p.in.N);
        int64_t uid = r0;
        while (uid < r1) {
            while (uid >= p.units.unit_base[i + 1]) ++i;     // instance of this segment
            const int64_t ub = p.units.unit_base[i];
            const int64_t seg_end = p.units.unit_base[i + 1] < r1 ? p.units.unit_base[i + 1] : r1;
            if (p.out.status[i] != VSBPP_OK) { uid = seg_end; continue; }
            const int64_t m = p.in.m(i), wb = p.in.w_begin(i);
            const int32_t n = p.in.n(i);
            const int32_t* B = p.in.B_all + p.in.B_begin(i);
            const int64_t a0 = (uid - ub) * S;
            const int64_t a1 = (seg_end - ub) * S < m ? (seg_end - ub) * S : m;
            const int cnt = static_cast<int>(a1 - a0);
            if (tid < kMaxTypes) Bs[tid] = tid < n ? static_cast<uint32_t>(B[tid]) : 0u;
            const bool narrow = static_cast<uint32_t>(B[0]) <= 2047u && n <= 16;
            for (int t = tid; t < cnt; t += blockDim.x) {
                const uint32_t x = static_cast<uint32_t>(p.in.w_all[wb + a0 + t]);
                uint32_t bn = 0, tn = 0;                   // smallest type holding x
                for (int y = 0; y < n; ++y) {
                    const uint32_t c = static_cast<uint32_t>(B[y]);
                    tn = c >= x ? static_cast<uint32_t>(y) : tn;
                    bn = c >= x ? c : bn;
                }
                wrun[t] = x;
                brun[t] = narrow ? (tn << 12) | bn : bn;
            }
            __syncthreads();
            for (int64_t u = uid + warp; u < seg_end; u += kWarps) {
                const int64_t g = u - ub;
                const int64_t a = g * S;
                const int k = static_cast<int>((m - a) < S ? (m - a) : S);
                const int nperm = h2_fact_small(k);
                const uint32_t* ws = wrun + (a - a0);
                const uint32_t* bs = brun + (a - a0);
                const uint32_t* tab = permtab + h2_table_off(k);
                if (narrow) {
                    uint32_t bestkey = 0xFFFFFFFFu, bv[kSlots], brawp = 0, bperm = 0;
#pragma unroll
                    for (int x = 0; x < kSlots; ++x) bv[x] = 0u;
                    // Full sublists, fixed criterion: permutations 2e and 2e+1
                    // share their first S-2 items (they differ in the order of
                    // the last two), so a lane packs that prefix once and
                    // finishes both from copies of its state.
                    constexpr bool kShare = CRIT != kRandom && S >= 3;
                    const int nlane = (kShare && k == S) ? nperm / 2 : 0;
                    for (int rb = 0; rb < nlane; rb += 32) {
                        const int e = rb + lane;
                        const bool active = e < nlane;
                        const uint32_t pa = tab[active ? 2 * e : 0], pb = tab[active ? 2 * e + 1 : 1];
                        uint32_t va[kSlots], rawa = 0, tota = 0, fita = 0, alivea = 0;
#pragma unroll
                        for (int x = 0; x < kSlots; ++x) va[x] = 0u;
                        if (p.counters)
                            h2_steps_narrow<S, CRIT, 0, S - 2, S, true>(pa, k, ws, bs, p.seed, g, 2 * e, va, rawa,
                                                                     tota, fita, alivea);
                        else
                            h2_steps_narrow<S, CRIT, 0, S - 2, S, false>(pa, k, ws, bs, p.seed, g, 2 * e, va, rawa,
                                                                      tota, fita, alivea);
                        uint32_t vb[kSlots], rawb = rawa, totb = tota, fitb = fita, aliveb = alivea;
#pragma unroll
                        for (int x = 0; x < kSlots; ++x) vb[x] = va[x];
                        if (p.counters) {
                            h2_steps_narrow<S, CRIT, S - 2, S, S, true>(pa, k, ws, bs, p.seed, g, 2 * e, va, rawa,
                                                                     tota, fita, alivea);
                            h2_steps_narrow<S, CRIT, S - 2, S, S, true>(pb, k, ws, bs, p.seed, g, 2 * e + 1, vb,
                                                                     rawb, totb, fitb, aliveb);
                            const uint32_t f = __reduce_add_sync(kFull, active ? fita + fitb : 0u);
                            if (lane == 0) atomicAdd(p.counters + 1, static_cast<unsigned long long>(f));
                        } else {
                            h2_steps_narrow<S, CRIT, S - 2, S, S, false>(pa, k, ws, bs, p.seed, g, 2 * e, va, rawa,
                                                                      tota, fita, alivea);
                            h2_steps_narrow<S, CRIT, S - 2, S, S, false>(pb, k, ws, bs, p.seed, g, 2 * e + 1, vb,
                                                                      rawb, totb, fitb, aliveb);
                        }
                        const uint32_t ka = active ? (tota << 10) | static_cast<uint32_t>(2 * e) : 0xFFFFFFFFu;
                        const uint32_t kb = active ? (totb << 10) | static_cast<uint32_t>(2 * e + 1) : 0xFFFFFFFFu;
                        const bool ba = ka < bestkey && ka < kb;       // ka < kb: equal totals go to the lower rank
                        const bool bb = !ba && kb < bestkey;
                        bestkey = ba ? ka : bb ? kb : bestkey;
                        brawp = ba ? rawa : bb ? rawb : brawp;
                        bperm = ba ? pa : bb ? pb : bperm;
#pragma unroll
                        for (int x = 0; x < kSlots; ++x) bv[x] = ba ? va[x] : bb ? vb[x] : bv[x];
                    }
                    for (int rb = nlane > 0 ? nperm : 0; rb < nperm; rb += 32) {
                        const int rank = rb + lane;
                        const bool active = rank < nperm;
                        const uint32_t perm = tab[active ? rank : 0];
                        uint32_t v[kSlots], rawp, fit = 0;
                        uint32_t tot;
                        if (p.counters) {
                            tot = h2_pack_narrow<S, CRIT, 0, true>(perm, k, ws, bs, p.seed, g, rank, v, rawp, fit);
                            fit = __reduce_add_sync(kFull, active ? fit : 0u);
                            if (lane == 0) atomicAdd(p.counters + 1, static_cast<unsigned long long>(fit));
                        } else if (k == S) {
                            tot = h2_pack_narrow<S, CRIT, S, false>(perm, k, ws, bs, p.seed, g, rank, v, rawp, fit);
                        } else {
                            tot = h2_pack_narrow<S, CRIT, 0, false>(perm, k, ws, bs, p.seed, g, rank, v, rawp, fit);
                        }
                        const uint32_t key = active ? (tot << 10) | static_cast<uint32_t>(rank) : 0xFFFFFFFFu;
                        const bool better = key < bestkey;
                        bestkey = better ? key : bestkey;
                        brawp = better ? rawp : brawp;
                        bperm = better ? perm : bperm;
#pragma unroll
                        for (int x = 0; x < kSlots; ++x) bv[x] = better ? v[x] : bv[x];
                    }
                    if (p.counters && lane == 0) atomicAdd(p.counters, static_cast<unsigned long long>(k));
                    const uint32_t wkey = __reduce_min_sync(kFull, bestkey);
                    if (bestkey == wkey) {
                        uint32_t used = 0, typx[kSlots];
#pragma unroll
                        for (int x = 0; x < kSlots; ++x) {
                            typx[x] = (bv[x] >> 12) & 15u;
                            used |= ((bv[x] >> 20) < (bv[x] & 0xFFFu) ? 1u : 0u) << x;
                        }
                        h2_write_winner<S>(p, typx, used, brawp, bperm, k, u, wb + a, wkey >> 10);
                    }
                } else {
                    uint64_t bestkey = ~0ull;
                    uint32_t br[kSlots], bc[kSlots], brawp = 0, bperm = 0;
#pragma unroll
                    for (int x = 0; x < kSlots; ++x) { br[x] = 0u; bc[x] = 0u; }
                    for (int rb = 0; rb < nperm; rb += 32) {
                        const int rank = rb + lane;
                        const bool active = rank < nperm;
                        const uint32_t perm = tab[active ? rank : 0];
                        uint32_t r[kSlots], c[kSlots], rawp, fit;
                        const uint64_t tot = h2_pack_wide<S, CRIT>(perm, k, ws, bs, p.seed, g, rank, r, c, rawp, fit);
                        if (p.counters) {
                            fit = __reduce_add_sync(kFull, active ? fit : 0u);
                            if (lane == 0) atomicAdd(p.counters + 1, static_cast<unsigned long long>(fit));
                        }
                        const uint64_t key = active ? (tot << 10) | static_cast<uint64_t>(rank) : ~0ull;
                        const bool better = key < bestkey;
                        bestkey = better ? key : bestkey;
                        brawp = better ? rawp : brawp;
                        bperm = better ? perm : bperm;
#pragma unroll
                        for (int x = 0; x < kSlots; ++x) {
                            br[x] = better ? r[x] : br[x];
                            bc[x] = better ? c[x] : bc[x];
                        }
                    }
                    if (p.counters && lane == 0) atomicAdd(p.counters, static_cast<unsigned long long>(k));
                    const uint64_t wkey = warp_min_u64(bestkey);
                    if (bestkey == wkey) {
                        uint32_t used = 0, typx[kSlots];
#pragma unroll
                        for (int x = 0; x < kSlots; ++x) {
                            used |= (br[x] < bc[x] ? 1u : 0u) << x;
                            uint32_t t = 0;
                            for (int y = 0; y < n; ++y) t = Bs[y] == bc[x] ? static_cast<uint32_t>(y) : t;
                            typx[x] = t;
                        }
                        h2_write_winner<S>(p, typx, used, brawp, bperm, k, u, wb + a, wkey >> 10);
                    }
                }
            }
            __syncthreads();                         // staged items are reused by the next segment
            uid = seg_end;
        }
    }
}

}  // namespace vsbpp
