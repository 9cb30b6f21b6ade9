// device_common.cuh -- device-side helpers shared by the packing kernels.
//
// Everything here is integer arithmetic.  The batch layout is CSR (see
// include/vsbpp.h); a "unit" is one membrane system of Section 6.3: an
// instance when the sublist size s covers the whole list, otherwise one
// contiguous sublist of s items (Rule 1 reading: chunks in list order).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "vsbpp.h"

namespace vsbpp {

constexpr int kFF = VSBPP_FF;
constexpr int kBF = VSBPP_BF;
constexpr int kWF = VSBPP_WF;
constexpr int kRandom = VSBPP_RANDOM;
constexpr int kMaxTypes = VSBPP_MAX_TYPES;
constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr uint32_t kH16MaxB = 255;   // B_1 limit of the one-warp kernel's 16-bit slot form

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the key-th output of the
// stream seeded with `seed` is the variant-13 mix of seed + (key+1)*gamma.
// Rule 3 of Section 6.3 draws the criterion "with equal probabilities"; the
// RANDOM criterion takes this output modulo 3 (0 = FF, 1 = BF, 2 = WF).
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t key) {
    uint64_t z = seed + (key + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ int pick_criterion(int crit, uint64_t seed, uint64_t key) {
    return crit == kRandom ? static_cast<int>(splitmix64(seed, key) % 3ull) : crit;
}

// Remark 3 of Section 6.3 read as a condition on Rule 5 (option
// VSBPP_REMARK3): a bin divides off a new one only if every bin of its type
// then holds at least half its capacity.  `below` is lane-distributed: lane t
// (capacity Bl = B[t], 0 past the types) holds the number of type-t bins
// below half.  A bin opened because nothing fits starts below half (opened);
// `cross` says the chosen bin's load has just reached half (the Rule 5
// condition), so it leaves the count; the division then fires only when no
// bin of its type (capacity Bt) is still below half, and the empty bin it
// divides off joins the count.  Called by all 32 lanes with uniform
// arguments (other than Bl and below).
__device__ __forceinline__ bool remark3_divide(uint32_t& below, uint32_t Bl, bool opened, uint64_t Bt,
                                               bool cross) {
    const bool mine = static_cast<uint64_t>(Bl) == Bt;
    below += (opened && mine) ? 1u : 0u;
    below -= (cross && mine) ? 1u : 0u;
    const bool fire = cross && !__any_sync(kFull, mine && below != 0u);
    below += (fire && mine) ? 1u : 0u;
    return fire;
}

// Read-only view of a CSR batch.  A null offset array means a single
// instance whose size is given directly (used by the single-instance calls).
struct BatchView {
    int64_t N;
    const int32_t* w_all;
    const int64_t* w_off;
    int64_t m_single;
    const int32_t* B_all;
    const int32_t* B_off;
    int32_t n_single;

    __device__ __forceinline__ int64_t w_begin(int64_t i) const { return w_off ? w_off[i] : 0; }
    __device__ __forceinline__ int64_t m(int64_t i) const {
        return w_off ? (w_off[i + 1] - w_off[i]) : m_single;
    }
    __device__ __forceinline__ int32_t B_begin(int64_t i) const { return B_off ? B_off[i] : 0; }
    __device__ __forceinline__ int32_t n(int64_t i) const {
        return B_off ? (B_off[i + 1] - B_off[i]) : n_single;
    }
};

// Where a packing's results go.  In direct mode (one unit per instance) the
// unit writes the instance outputs.  In compose mode (several sublists per
// instance) each unit writes sublist-local bin ids into bin_of_item, its bin
// types into local_types at its own item positions, and its bin count and
// capacity into unit_count / unit_total; a compose pass then concatenates.
struct OutView {
    int32_t* bin_of_item;
    int32_t* bin_type;
    int64_t* num_bins;
    int64_t* total;
    int32_t* status;
    int32_t* local_types;   // compose mode only
    int32_t* unit_count;    // compose mode only
    int64_t* unit_total;    // compose mode only
};

// Units: one per instance when unit_base is null, else unit_base[i] ..
// unit_base[i+1] are instance i's sublists of `sublist` items.
struct UnitMap {
    const int64_t* unit_base;   // [N+1] or null
    int64_t sublist;            // items per sublist (compose mode)
    int64_t num_units;

    // instance of unit u (binary search over the prefix array)
    __device__ __forceinline__ int64_t instance_of(int64_t u, int64_t N) const {
        if (!unit_base) return u;
        int64_t lo = 0, hi = N;          // unit_base[lo] <= u < unit_base[hi]
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (unit_base[mid] <= u) lo = mid; else hi = mid;
        }
        return lo;
    }
};

// Exclusive warp scan (sum) of a 32-bit value.
__device__ __forceinline__ uint32_t warp_exclusive_scan(uint32_t v, int lane) {
    uint32_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, d);
        if (lane >= d) x += y;
    }
    return x - v;
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
    return v;
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long o = __shfl_xor_sync(kFull, v, d);
        v = o < v ? o : v;
    }
    return v;
}

// Named barrier over `nthreads` threads (a multiple of 32).
__device__ __forceinline__ void named_barrier(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

}  // namespace vsbpp
