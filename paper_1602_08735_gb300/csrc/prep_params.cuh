// prep_params.cuh -- parameters of the validation, ordering and compose
// kernels (prep_kernels.cuh).
#pragma once

#include "device_common.cuh"

namespace vsbpp {

constexpr int kClassLarge = 0;   // narrow slots, one multi-warp group per instance
constexpr int kClassSmall = 1;   // narrow slots, one warp per instance
constexpr int kClassWide = 2;    // wide slots
constexpr int kClassHuge = 3;    // bins in global memory, tile summaries (kc_kernel)
constexpr int kClassNone = 4;    // nothing to pack (error, empty, or composed)
constexpr int kClasses = 4;
constexpr int kBuckets = 64;

struct PrepParams {
    BatchView in;
    OutView out;
    int32_t classify;        // 1: first heuristic with one unit per instance
    int32_t one_class;       // 1 (with classify): every packable instance in the large class
                             // (the bounded-space kernel holds any size)
    int64_t small_m;         // m <= small_m -> small class
    int64_t narrow_cap;      // largest m the narrow kernels hold
    int64_t small_cap;       // largest m the single-warp kernel holds
    int64_t wide_cap;        // largest m the wide kernel holds
    int64_t huge_cap;        // largest m the global-memory kernel holds (0: none)
    int64_t huge_max_B1;     // largest B_1 the global-memory kernel holds
    int64_t narrow_max_B;    // B_1 limit of the narrow slots
    int64_t narrow_bins;     // worst-case bins (2m + preopen n) the narrow classes accept
    int64_t narrow_cap16;    // largest m the one-warp kernel's 16-bit slots take (B_1 <= 255; 0: none)
    int32_t preopen;
    int32_t* cls;            // [N]
    uint32_t* hist;          // [kClasses * kBuckets]
    int64_t* nu;             // [N] sublists per instance (compose mode) or null
    int64_t sublist;         // sublist size (compose mode)
};

struct ComposeParams {
    BatchView in;
    OutView out;
    const int64_t* unit_base;
    int64_t sublist;
    int64_t only_instance;   // -1: all
};

}  // namespace vsbpp
