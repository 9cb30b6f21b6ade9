// kd_params.cuh -- launch parameters and shared-memory layout of the
// cluster kernel for membrane systems of hundreds of thousands of bins
// (kd_kernel.cuh).
#pragma once

#include "device_common.cuh"

namespace vsbpp {

constexpr int kKDSeg = 512;                         // bins per segment (16-bit slots: 1 KB), BF presence unit
constexpr int kKDSegBytes = kKDSeg * 2;
constexpr int kKDSub = 128;                         // bins per sub-segment (8 bytes a lane), FF / WF scan unit
constexpr int kKDMaxSegs = 1024;                    // 2^19 bins per membrane system
constexpr int kKDMaxBins = kKDMaxSegs * kKDSeg;
constexpr int kKDMaxSubs = kKDMaxBins / kKDSub;     // 4096
constexpr int kKDTiles = kKDMaxSubs / 32;           // 128 tiles of 32 sub-segments (4 per lane)
constexpr int kKDMaxB1 = 2047;                      // 11-bit residuals
constexpr int kKDMaxB1Idx = 1023;                   // with BF items: one present-residual word per lane

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

// CTA 0's layout: sub-segment maxima (FF / WF items), capacities,
// per-residual segment bitmaps (BF items), then its bins.
constexpr int kKDOffSubmax = 0;
constexpr int kKDOffBs = kKDOffSubmax + 2 * kKDMaxSubs;
constexpr int kKDOffPres = kKDOffBs + 4 * kMaxTypes;

__host__ __device__ inline int kd_pres_bytes(int max_B1, int pres) {
    return pres ? (max_B1 + 1) * 32 * 4 : 0;
}

__host__ __device__ inline int kd_bins_offset(int max_B1, int pres) {
    return (kKDOffPres + kd_pres_bytes(max_B1, pres) + 127) & ~127;
}

}  // namespace vsbpp
