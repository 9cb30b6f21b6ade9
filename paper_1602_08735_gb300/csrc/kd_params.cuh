// kd_params.cuh -- launch parameters and shared-memory layout of the
// cluster kernel for membrane systems of hundreds of thousands of bins
// (kd_kernel.cuh).
#pragma once

#include "device_common.cuh"

namespace vsbpp {

constexpr int kKDSeg = 512;                         // bins per segment (16-bit slots: 1 KB)
constexpr int kKDSegBytes = kKDSeg * 2;
constexpr int kKDMaxSegs = 1024;                    // 2^19 bins per membrane system
constexpr int kKDMaxBins = kKDMaxSegs * kKDSeg;
constexpr int kKDTiles = kKDMaxSegs / 32;           // 32 segments per tile
constexpr int kKDMaxB1 = 2047;                      // 11-bit residuals
constexpr int kKDGpWords = (kKDMaxB1 + 1) / 32;     // 64

struct KDParams {
    BatchView in;
    OutView out;
    int32_t criterion;
    int32_t preopen;
    int32_t remark3;
    uint64_t seed;
    const int32_t* order;          // work list: positions [seg[segment], seg[segment+1]) of order
    const int64_t* seg;
    int32_t segment;
    unsigned long long* queue;
    int32_t* spill_list;           // systems this kernel does not hold (count in spill_seg[1])
    int64_t* spill_seg;
    uint16_t* over;                // [clusters][over_bins]: bins past the two CTAs' shared memory
    int64_t over_bins;
    int32_t* dense;                // [clusters][kKDMaxBins]: dense id per bin (epilogue)
    int32_t max_B1;                // largest B_1 the presence rows hold (BF items)
    int32_t pres;                  // 1: BF items occur (presence rows laid out)
    int32_t segs0, segs1;          // segments held by CTA 0 and CTA 1
    int32_t smem;                  // dynamic shared memory per CTA
    unsigned long long* counters;
};

// CTA 0's layout: segment maxima, tile maxima, capacities, residual-present
// bitmap, per-residual segment bitmaps (BF), then its bins.
constexpr int kKDOffSegmax = 0;
constexpr int kKDOffTilemax = kKDOffSegmax + 2 * kKDMaxSegs;
constexpr int kKDOffBs = kKDOffTilemax + 2 * kKDTiles;
constexpr int kKDOffGp = kKDOffBs + 4 * kMaxTypes;
constexpr int kKDOffPres = kKDOffGp + 4 * kKDGpWords;

__host__ __device__ inline int kd_pres_bytes(int max_B1, int pres) {
    return pres ? (max_B1 + 1) * 32 * 4 : 0;
}

__host__ __device__ inline int kd_bins_offset(int max_B1, int pres) {
    return (kKDOffPres + kd_pres_bytes(max_B1, pres) + 127) & ~127;
}

}  // namespace vsbpp
