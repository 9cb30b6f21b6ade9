// variants_params.cuh -- launch parameters of the offline pre-sort and the
// bounded-space kernels (variants_kernels.cuh).
#pragma once

#include "device_common.cuh"

namespace vsbpp {

// Pre-sort (VSBPP_PRESORT) and its inverse.
struct PresortParams {
    BatchView in;            // the caller's batch
    int32_t* w_sorted;       // [w_off[N]] weights in packing order (CSR as in.w_all)
    int32_t* perm;           // [w_off[N]] original index (within the instance) per sorted position
    int32_t* tmp;            // [w_off[N]] radix ping-pong buffer
    int32_t* status0;        // [N] validation status of the caller's order
    int32_t* bin_of_item;    // caller's output (unpermute)
    const int32_t* boi_sorted;   // bin ids per sorted position (unpermute)
    int32_t* status;         // caller's status (unpermute)
    int64_t* num_bins;
    int64_t* total;
};

constexpr int kPresortWarps = 4;

// Bounded-space first heuristic (max_open = K <= 32).
struct BKParams {
    BatchView in;
    OutView out;
    int32_t criterion;
    int32_t preopen;
    int32_t max_open;        // K, 1..32
    uint64_t seed;
    // Work list: positions [seg[segment], seg[segment+1]) naming instances
    // order[x], pulled through the atomic counter queue; or, with seg null,
    // instances [range_begin, range_end) taken round robin by the warps.
    const int32_t* order;
    const int64_t* seg;
    int32_t segment;
    unsigned long long* queue;
    int64_t range_begin, range_end;
    int32_t* rec;            // per created bin: type | kUsed; instance i at 2*w_off[i] + 32*i
    unsigned long long* counters;
};

constexpr int kBKWarps = 4;
constexpr int32_t kBKUsed = 0x100;     // record flag: the bin holds an item

}  // namespace vsbpp
