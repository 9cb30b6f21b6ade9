// kc_params.cuh -- launch parameters and shared-memory layout of the
// global-memory first-heuristic kernel (kc_kernel.cuh).
#pragma once

#include "device_common.cuh"

namespace vsbpp {

constexpr int kTileBins = 2048;            // bins per tile
constexpr int kTileQuadsPerLane = kTileBins / 4 / 32;   // 16 uint4 per lane
constexpr int kMaxTiles = 1024;            // 2^21 bins per membrane system
constexpr int kSupers = kMaxTiles / 32;

struct KCParams {
    BatchView in;
    OutView out;
    int32_t criterion;
    int32_t preopen;
    int32_t remark3;         // 1: Rule 5 with Remark 3's per-type condition
    uint64_t seed;
    const int32_t* order;
    const int64_t* seg;
    int32_t segment;
    unsigned long long* queue;
    uint32_t* slots_all;     // [grid][bin_cap]
    int64_t bin_cap;         // bins of scratch per block (multiple of kTileBins)
    int32_t max_B1;          // largest B_1 the shared-memory layout holds
    int32_t pres_words;      // words per residual in pres (ceil(tiles/32))
    unsigned long long* counters;
};

// Shared-memory bytes: tile_max, sup_max, B, gp bitmap, pres bitmap.
__host__ __device__ inline int kc_smem_bytes(int max_B1, int pres_words) {
    const int gp_words = (max_B1 + 1 + 31) / 32;
    return kMaxTiles * 2 + kSupers * 2 + kMaxTypes * 4 + gp_words * 4 +
           (max_B1 + 1) * pres_words * 4 + 64;
}

}  // namespace vsbpp
