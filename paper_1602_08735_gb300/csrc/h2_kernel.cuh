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
                if (Bt < 2 * r_old && 2 * r_new <= Bt) {      // Rule 5
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

template <int S, int CRIT>
__global__ void __launch_bounds__(768) h2_pack_kernel_reg(const H2Params p) {
    constexpr int kBins = 2 * S;
    __shared__ unsigned long long wbest[32];
    __shared__ uint32_t Bs[kMaxTypes];
    __shared__ uint32_t wsub[8];
    __shared__ uint32_t tstar[8];
    const int T = static_cast<int>(blockDim.x);
    const int tid = static_cast<int>(threadIdx.x);
    const int lane = tid & 31, warp = tid >> 5, nwarps = T >> 5;
    int pfull[S];
    h2_decode<S>(tid, S, pfull);                     // this thread's permutation of S items

    int64_t u_begin = 0, u_end = p.units.unit_base[p.in.N];
    if (p.only_instance >= 0) {
        u_begin = p.units.unit_base[p.only_instance];
        u_end = p.units.unit_base[p.only_instance + 1];
    }
    // Each block takes runs of kRun consecutive sublists, so the instance is
    // found once per run and its metadata reloaded only when the run crosses
    // into the next instance (sublists are numbered instance by instance).
    constexpr int kRun = 16;
    for (int64_t r0 = u_begin + static_cast<int64_t>(blockIdx.x) * kRun; r0 < u_end;
         r0 += static_cast<int64_t>(gridDim.x) * kRun) {
        const int64_t r1 = (r0 + kRun) < u_end ? (r0 + kRun) : u_end;
        int64_t i = p.units.instance_of(r0, p.in.N);
        int64_t ub = p.units.unit_base[i], ub_next = p.units.unit_base[i + 1];
        int32_t st = p.out.status[i];
        int64_t m = p.in.m(i), wb = p.in.w_begin(i);
        int32_t n = p.in.n(i);
        const int32_t* B = p.in.B_all + p.in.B_begin(i);
        for (int64_t uid = r0; uid < r1; ++uid) {
            while (uid >= ub_next) {                 // next instance with sublists
                ++i;
                ub = ub_next;
                ub_next = p.units.unit_base[i + 1];
                st = p.out.status[i];
                m = p.in.m(i);
                wb = p.in.w_begin(i);
                n = p.in.n(i);
                B = p.in.B_all + p.in.B_begin(i);
            }
            if (st != VSBPP_OK) continue;
            const int64_t g = uid - ub;
            const int64_t a = g * S;
            const int k = static_cast<int>((m - a) < S ? (m - a) : S);
            const int nperm = h2_fact_small(k);
            const int32_t* w = p.in.w_all + wb + a;
            if (tid < kMaxTypes) Bs[tid] = tid < n ? static_cast<uint32_t>(B[tid]) : 0u;
            if (tid < k) {
                const int32_t x = w[tid];
                uint32_t t = 0;
                for (int y = 0; y < n; ++y)
                    if (B[y] >= x) t = static_cast<uint32_t>(y);
                wsub[tid] = static_cast<uint32_t>(x);
                tstar[tid] = t;
            }
            __syncthreads();

            unsigned long long key = ~0ull;
            int perm[S], raw[S];
            uint32_t res[kBins], typ[kBins];
    #pragma unroll
            for (int x = 0; x < kBins; ++x) { res[x] = 0; typ[x] = 0; }
            int L = 0;
            const bool active = tid < nperm;
            if (active) {
                if (k == S) {
    #pragma unroll
                    for (int q = 0; q < S; ++q) perm[q] = pfull[q];
                } else {
                    h2_decode<S>(tid, k, perm);
                }
    #pragma unroll
                for (int q = 0; q < S; ++q) {
                    raw[q] = 0;
                    if (q < k) {
                        const int item = perm[q];
                        const uint32_t wj = wsub[item];
                        const int c = CRIT == kRandom
                                          ? pick_criterion(kRandom, p.seed,
                                                           static_cast<uint64_t>((g * 720 + tid) * 8 + q))
                                          : CRIT;
                        int chosen = -1;
                        uint32_t cr = 0, ct = 0;             // residual and type of the choice
    #pragma unroll
                        for (int x = 0; x < 2 * q; ++x) {        // Rule 4 over the live bins
                            const uint32_t r = res[x];
                            if (x < L && r >= wj &&
                                (chosen < 0 || (c == kBF && r < cr) || (c == kWF && r > cr))) {
                                chosen = x;
                                cr = r;
                                ct = typ[x];
                            }
                        }
                        const bool opened = chosen < 0;
                        if (opened) {                           // smallest type holding w
                            ct = tstar[item];
                            cr = Bs[ct];
                            chosen = L;
                            ++L;
                        }
                        const uint32_t Bt = Bs[ct];
                        const uint32_t r_new = cr - wj;
                        const bool fire = (static_cast<uint64_t>(Bt) < 2ull * cr) &&
                                          (2ull * r_new <= static_cast<uint64_t>(Bt));   // Rule 5
    #pragma unroll
                        for (int x = 0; x < 2 * q + 2 && x < kBins; ++x) {
                            if (x == chosen) res[x] = r_new;
                            if ((opened && x == chosen) || (fire && x == L)) typ[x] = ct;
                            if (fire && x == L) res[x] = Bt;
                        }
                        if (fire) ++L;
                        raw[q] = chosen;
                    }
                }
                unsigned long long tot = 0;
    #pragma unroll
                for (int x = 0; x < kBins; ++x) {
                    const uint32_t cap = Bs[typ[x]];
                    if (x < L && res[x] < cap) tot += cap;
                }
                key = (tot << 10) | static_cast<unsigned long long>(tid);
            }
            key = warp_min_u64(key);
            if (lane == 0) wbest[warp] = key;
            __syncthreads();
            unsigned long long best = ~0ull;
            for (int x = 0; x < nwarps; ++x) best = wbest[x] < best ? wbest[x] : best;
            if (active && tid == static_cast<int>(best & 1023ull)) {
                // the winning permutation's result, in sublist-local form
                bool used[kBins];
                int cnt = 0;
    #pragma unroll
                for (int x = 0; x < kBins; ++x) {
                    used[x] = x < L && res[x] < Bs[typ[x]];
                    if (used[x]) {
                        p.out.local_types[wb + a + cnt] = static_cast<int32_t>(typ[x]);
                        ++cnt;
                    }
                }
    #pragma unroll
                for (int q = 0; q < S; ++q) {
                    if (q < k) {
                        int d = 0;
    #pragma unroll
                        for (int x = 0; x < kBins; ++x)
                            if (x < raw[q] && used[x]) ++d;
                        p.out.bin_of_item[wb + a + perm[q]] = d;
                    }
                }
                p.out.unit_count[uid] = cnt;
                p.out.unit_total[uid] = static_cast<int64_t>(best >> 10);
            }
            __syncthreads();
        }
    }
}

}  // namespace vsbpp
