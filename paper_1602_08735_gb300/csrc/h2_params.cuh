// h2_params.cuh -- launch parameters of the second-heuristic kernel
// (Section 6.4); the kernel itself is in h2_kernel.cuh.
#pragma once

#include "device_common.cuh"

namespace vsbpp {

struct H2Params {
    BatchView in;
    OutView out;          // compose-mode fields are used
    UnitMap units;
    int32_t criterion;
    int32_t preopen;
    int32_t remark3;      // 1: Rule 5 with Remark 3's per-type condition (generic kernel only)
    uint64_t seed;
    int32_t sublist;      // s (1..6)
    int32_t perms;        // s!
    int32_t max_bins;     // 2*s + (preopen ? 32 : 0)
    int64_t only_instance;  // -1: every unit; else only that instance's sublists
    unsigned long long* counters;   // null, or {items, fit tests} to add to (register kernel)
};

// Exhaustive second heuristic (sublists of 7..12 items, h2x_kernel.cuh).
struct H2XParams {
    BatchView in;
    OutView out;                    // compose-mode fields are used
    UnitMap units;
    int32_t criterion;
    int32_t remark3;                // 1: Rule 5 with Remark 3's per-type condition
    int32_t sublist;                // s (7..12)
    uint64_t seed;
    const int64_t* seg_units;       // [1] = number of sublists (device)
    unsigned long long* best;       // per sublist: least (total << 29) | rank
    unsigned long long* queue;      // task counter (zero at the start)
    unsigned long long* counters;   // null, or {items, fit tests} to add to
    int64_t only_instance;          // -1: every sublist; else that instance's
};

__host__ __device__ inline int h2_smem_bytes(int threads, int max_bins) {
    return max_bins * threads * 4      // residuals
         + max_bins * threads          // types
         + 32 * 8                      // per-warp best keys
         + 16;
}

}  // namespace vsbpp
