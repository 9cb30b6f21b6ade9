// h2x_kernel.cuh -- the second heuristic with sublists of 7..12 items: every
// one of the s! permutations of each sublist packed with Rules 2-6 and the
// cheapest kept, the exhaustive search Section 7 compares the second
// heuristic against (its "parallel implementation": a thread per permutation,
// the least capacity found per block, then over the grid).
//
// s! outgrows a block (5040 .. 479,001,600 permutations), so the search runs
// across the whole GPU: a task is (sublist, chunk of kChunk consecutive
// lexicographic ranks); warps take tasks from an atomic counter, each lane
// packs every 32nd rank of the chunk, and the warp's least (total, rank) key
// goes to the sublist's slot with a 64-bit atomicMin on (total << 29) |
// rank (12! < 2^29; a total is at most 12 used bins below 2^31 each) -- the
// least total, ties to the least rank, as in Section 6.4.  A second kernel packs each
// sublist's winning permutation again and writes the sublist-local result
// (bin ids from 0 in creation order, types, count, capacity) for the
// composition pass.
//
// A lane's bins are fixed slots as in h2_kernel.cuh (the bin opened at item
// step q is slot 2q, the one divided off at step q slot 2q + 1, so slot order
// is creation order); residual and capacity words per slot, 64-bit
// selection keys (measure << 5 | slot).
#pragma once

#include "h2_params.cuh"

namespace vsbpp {

constexpr int kH2XChunk = 512;               // ranks per task
constexpr uint64_t kFact12 = 479001600ull;   // RANDOM key stride for s = 7..12

__host__ __device__ constexpr int64_t h2x_fact(int v) {
    return v <= 1 ? 1 : v == 2 ? 2 : v == 3 ? 6 : v == 4 ? 24 : v == 5 ? 120 : v == 6 ? 720 : v == 7 ? 5040
         : v == 8 ? 40320 : v == 9 ? 362880 : v == 10 ? 3628800 : v == 11 ? 39916800 : 479001600;
}

// Permutation of lexicographic rank `rank` over k <= S positions.
template <int S>
__device__ __forceinline__ void h2x_decode(uint32_t rank, int k, int (&perm)[S]) {
    uint32_t used = 0;
#pragma unroll
    for (int q = 0; q < S; ++q) {
        perm[q] = 0;
        if (q < k) {
            const uint32_t f = static_cast<uint32_t>(h2x_fact(k - 1 - q));
            uint32_t d = rank / f;
            rank -= d * f;
            // the d-th position (ascending) not used yet
            int x = 0;
#pragma unroll
            for (int y = 0; y < S; ++y) {
                const bool free = y < k && !((used >> y) & 1u);
                if (free && d == 0u) { x = y; d = 0xFFFFFFFFu; }
                else if (free && d != 0xFFFFFFFFu) --d;
            }
            used |= 1u << x;
            perm[q] = x;
        }
    }
}

// Pack the permutation `perm` of the sublist's k items (weights ws, capacity
// of the smallest type holding each in bs).  Returns the used capacity; r, cp
// the slots' residuals and capacities; slot[q] the slot that took step q's
// item; fit the method's fit tests (bins alive when each item arrives).
template <int S, int CRIT>
__device__ __forceinline__ uint64_t h2x_pack(const int (&perm)[S], int k, const uint32_t* ws, const uint32_t* bs,
                                             uint64_t seed, int64_t g, uint32_t rank, uint32_t (&r)[2 * S],
                                             uint32_t (&cp)[2 * S], uint32_t (&slot)[S], uint32_t& fit,
                                             bool remark3) {
    constexpr int kSlots = 2 * S;
    constexpr uint64_t kNo = ~0ull;
#pragma unroll
    for (int x = 0; x < kSlots; ++x) { r[x] = 0u; cp[x] = 0u; }
    uint64_t tot = 0;
    uint32_t alive = 0;
    fit = 0;
#pragma unroll
    for (int q = 0; q < S; ++q) {
        slot[q] = 0;
        if (q < k) {
            const uint32_t wq = ws[perm[q]], bn = bs[perm[q]];
            const int c = CRIT == kRandom
                              ? pick_criterion(kRandom, seed,
                                               (static_cast<uint64_t>(g) * kFact12 + rank) * 16ull + q)
                              : CRIT;
            uint64_t key = kNo;              // (measure << 5) | slot, least wins (lowest slot on ties)
#pragma unroll
            for (int x = 0; x < 2 * q; ++x) {
                const bool fits = r[x] >= wq;
                const uint64_t mes = c == kFF ? 0ull : c == kBF ? static_cast<uint64_t>(r[x] - wq)
                                                                : static_cast<uint64_t>(~r[x]);
                const uint64_t kx = (mes << 5) | static_cast<uint64_t>(x);
                key = fits && kx < key ? kx : key;
            }
            const bool hit = key != kNo;
            const uint32_t xs = hit ? static_cast<uint32_t>(key & 31ull) : static_cast<uint32_t>(2 * q);
            uint32_t r_old = bn, cap = bn;
#pragma unroll
            for (int x = 0; x < 2 * q; ++x) {
                r_old = xs == static_cast<uint32_t>(x) ? r[x] : r_old;
                cap = xs == static_cast<uint32_t>(x) ? cp[x] : cap;
            }
            const uint32_t r_new = r_old - wq;
            bool fire = (static_cast<uint64_t>(cap) < 2ull * r_old) &&
                        (2ull * r_new <= static_cast<uint64_t>(cap));           // Rule 5
            if (remark3 && fire) {
                // Remark 3: no other bin of this type (capacities are distinct)
                // may be below half; the chosen one holds half now
#pragma unroll
                for (int x = 0; x < 2 * q; ++x)
                    fire = fire && !(static_cast<uint32_t>(x) != xs && cp[x] == cap &&
                                     static_cast<uint64_t>(cap) < 2ull * r[x]);
            }
            tot += r_old == cap ? cap : 0u;            // the bin's first item: it becomes used
            fit += alive;
            alive += (hit ? 0u : 1u) + (fire ? 1u : 0u);
#pragma unroll
            for (int x = 0; x < 2 * q; ++x) r[x] = xs == static_cast<uint32_t>(x) ? r_new : r[x];
            r[2 * q] = hit ? 0u : r_new;
            cp[2 * q] = hit ? 0u : cap;
            r[2 * q + 1] = fire ? cap : 0u;
            cp[2 * q + 1] = fire ? cap : 0u;
            slot[q] = xs;
        }
    }
    return tot;
}

// The instance holding unit u and the sublist's place in it.
__device__ __forceinline__ bool h2x_unit(const H2XParams& p, int64_t u, int64_t& i, int64_t& a, int& k,
                                         int64_t& g) {
    i = p.units.instance_of(u, p.in.N);
    if (p.out.status[i] != VSBPP_OK) return false;
    g = u - p.units.unit_base[i];
    a = g * p.sublist;
    const int64_t m = p.in.m(i);
    k = static_cast<int>((m - a) < p.sublist ? (m - a) : p.sublist);
    return k > 0;
}

// Stage the sublist's k items: weight, and the capacity of the smallest type
// holding it (the new bin when nothing fits).
__device__ __forceinline__ void h2x_stage(const H2XParams& p, int64_t i, int64_t a, int k, int lane,
                                          uint32_t* ws, uint32_t* bs) {
    if (lane < k) {
        const uint32_t x = static_cast<uint32_t>(p.in.w_all[p.in.w_begin(i) + a + lane]);
        const int32_t n = p.in.n(i);
        const int32_t* B = p.in.B_all + p.in.B_begin(i);
        uint32_t bn = 0;
        for (int y = 0; y < n; ++y) {
            const uint32_t c = static_cast<uint32_t>(B[y]);
            bn = c >= x ? c : bn;
        }
        ws[lane] = x;
        bs[lane] = bn;
    }
    __syncwarp();
}

template <int S, int CRIT>
__global__ void __launch_bounds__(128) h2x_search_kernel(const H2XParams p) {
    __shared__ uint32_t items[4][2][16];
    const int lane = static_cast<int>(threadIdx.x) & 31, warp = static_cast<int>(threadIdx.x) >> 5;
    uint32_t* ws = items[warp][0];
    uint32_t* bs = items[warp][1];
    int64_t u_begin = 0, u_end = p.seg_units[1];
    if (p.only_instance >= 0) {
        u_begin = p.units.unit_base[p.only_instance];
        u_end = p.units.unit_base[p.only_instance + 1];
    }
    const int64_t chunks = (h2x_fact(S) + kH2XChunk - 1) / kH2XChunk;
    const int64_t tasks = (u_end - u_begin) * chunks;
    int64_t last_u = -1;
    bool ok = false;
    int64_t i = 0, a = 0, g = 0;
    int k = 0;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(p.queue, 1ull);
        t = __shfl_sync(kFull, t, 0);
        if (static_cast<int64_t>(t) >= tasks) break;
        const int64_t u = u_begin + static_cast<int64_t>(t) / chunks;
        const int64_t c = static_cast<int64_t>(t) % chunks;
        if (u != last_u) {
            __syncwarp();
            ok = h2x_unit(p, u, i, a, k, g);
            if (ok) h2x_stage(p, i, a, k, lane, ws, bs);
            last_u = u;
        }
        if (!ok) continue;
        const int64_t nperm = h2x_fact(k);
        const int64_t r0 = c * kH2XChunk;
        if (r0 >= nperm) continue;
        const int64_t r1 = (r0 + kH2XChunk) < nperm ? (r0 + kH2XChunk) : nperm;
        unsigned long long best = ~0ull;
        uint32_t fits = 0;
        for (int64_t rr = r0 + lane; rr < r1; rr += 32) {
            int perm[S];
            h2x_decode<S>(static_cast<uint32_t>(rr), k, perm);
            uint32_t r[2 * S], cp[2 * S], slot[S], fit;
            const uint64_t tot = h2x_pack<S, CRIT>(perm, k, ws, bs, p.seed, g, static_cast<uint32_t>(rr), r, cp,
                                                   slot, fit, p.remark3 != 0);
            const unsigned long long key = (tot << 29) | static_cast<unsigned long long>(rr);
            best = key < best ? key : best;
            fits += fit;
        }
        best = warp_min_u64(best);
        if (lane == 0) atomicMin(p.best + u, best);
        if (p.counters) {
            const unsigned long long f = warp_sum_u64(fits);
            if (lane == 0) atomicAdd(p.counters + 1, f);
        }
    }
}

// One warp per sublist: lane 0 packs the winning permutation again and writes
// the sublist-local result.
template <int S, int CRIT>
__global__ void __launch_bounds__(128) h2x_write_kernel(const H2XParams p) {
    __shared__ uint32_t items[4][2][16];
    __shared__ uint32_t Bs[4][kMaxTypes];
    const int lane = static_cast<int>(threadIdx.x) & 31, warp = static_cast<int>(threadIdx.x) >> 5;
    uint32_t* ws = items[warp][0];
    uint32_t* bs = items[warp][1];
    int64_t u_begin = 0, u_end = p.seg_units[1];
    if (p.only_instance >= 0) {
        u_begin = p.units.unit_base[p.only_instance];
        u_end = p.units.unit_base[p.only_instance + 1];
    }
    const int64_t wid = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t u = u_begin + wid; u < u_end; u += nw) {
        int64_t i, a, g;
        int k;
        if (!h2x_unit(p, u, i, a, k, g)) continue;
        h2x_stage(p, i, a, k, lane, ws, bs);
        const int32_t n = p.in.n(i);
        Bs[warp][lane] = lane < n ? static_cast<uint32_t>(p.in.B_all[p.in.B_begin(i) + lane]) : 0u;
        __syncwarp();
        if (lane == 0) {
            const unsigned long long key = p.best[u];
            const uint32_t rank = static_cast<uint32_t>(key & ((1ull << 29) - 1ull));
            int perm[S];
            h2x_decode<S>(rank, k, perm);
            uint32_t r[2 * S], cp[2 * S], slot[S], fit;
            const uint64_t tot = h2x_pack<S, CRIT>(perm, k, ws, bs, p.seed, g, rank, r, cp, slot, fit,
                                                   p.remark3 != 0);
            const int64_t base = p.in.w_begin(i) + a;
            uint32_t used = 0;
            int cnt = 0;
#pragma unroll
            for (int x = 0; x < 2 * S; ++x) {
                if (r[x] < cp[x]) {
                    used |= 1u << x;
                    int t = 0;
                    for (int y = 0; y < n; ++y) t = Bs[warp][y] == cp[x] ? y : t;
                    p.out.local_types[base + cnt] = t;
                    ++cnt;
                }
            }
#pragma unroll
            for (int q = 0; q < S; ++q)
                if (q < k) p.out.bin_of_item[base + perm[q]] = __popc(used & ((1u << slot[q]) - 1u));
            p.out.unit_count[u] = cnt;
            p.out.unit_total[u] = static_cast<int64_t>(tot);
            if (p.counters) atomicAdd(p.counters, static_cast<unsigned long long>(k));
        }
        __syncwarp();
    }
}

}  // namespace vsbpp
