// noalloc.cu -- vsbpp_pack_batch_noalloc: the batched first-heuristic pack
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the moment they need a packing: code
// that runs under a fixed device-memory reservation or inside another
// allocator's arena (where a library allocation would go around the owner's
// accounting), and latency-critical loops that cannot afford an allocation,
// or the device-wide synchronisation of a cudaFree, on their path.  This
// entry point takes its scratch from one file-scope __device__ array instead
// of the library's per-stream scratch, and calls no allocating routine.
//
// The scratch array is a host-side symbol; host code may not pass its name to
// a kernel.  Its device address is obtained with cudaGetSymbolAddress once
// per device, with that device current, by the first call on that device,
// and cached until the process ends: after a cudaDeviceReset the cached
// address is stale, so calls must not be made after a reset.  Every call on a
// device shares the array: calls whose GPU work overlaps in time (on
// different streams) race on it and must be serialised by the caller.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace vsbpp {
namespace {

constexpr int64_t kNoallocMaxInstances = VSBPP_NOALLOC_MAX_INSTANCES;

// Layout: class per instance, work order, histogram, cursors, segment bounds,
// queue counters.  Sized for kNoallocMaxInstances; about 0.5 MiB per device.
constexpr size_t kOffCls = 0;
constexpr size_t kOffOrder = kOffCls + 4 * kNoallocMaxInstances;
constexpr size_t kOffHist = kOffOrder + 4 * kNoallocMaxInstances;
constexpr size_t kOffCursor = kOffHist + 4 * kClasses * kBuckets;
constexpr size_t kOffSeg = kOffCursor + 8 * kClasses * kBuckets;
constexpr size_t kOffQueue = kOffSeg + 8 * 8;
constexpr size_t kScratchBytes = kOffQueue + 8 * 8;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_ptr[kMaxDevices] = {};

}  // namespace
}  // namespace vsbpp

using namespace vsbpp;

extern "C" int vsbpp_pack_batch_noalloc(int64_t N, const int32_t* w_all, const int64_t* w_off,
                                        const int32_t* B_all, const int32_t* B_off, int64_t max_m,
                                        const vsbpp_params* p, int32_t* bin_of_item_all,
                                        int32_t* bin_type_all, int64_t* num_bins, int64_t* total,
                                        int32_t* status, void* stream) {
    if (N < 0 || max_m < 0) return VSBPP_EINVAL;
    if (N == 0) return VSBPP_OK;
    if (!w_off || !B_all || !B_off || !bin_of_item_all || !bin_type_all || !num_bins || !total || !status)
        return VSBPP_EINVAL;
    vsbpp_params prm;
    std::memset(&prm, 0, sizeof(prm));
    prm.heuristic = VSBPP_H1;
    prm.criterion = VSBPP_BF;
    if (p) prm = *p;
    if (prm.heuristic != VSBPP_H1 || prm.criterion < VSBPP_FF || prm.criterion > VSBPP_RANDOM ||
        (prm.preopen & ~1) || prm.flags != 0 || prm.max_open != 0 || prm.sublist_size < 0)
        return VSBPP_EINVAL;
    // one membrane system per instance only (sublists need per-sublist scratch)
    if (prm.sublist_size != 0 && prm.sublist_size < max_m) return VSBPP_ECAPACITY;
    if (N > kNoallocMaxInstances || max_m > VSBPP_NOALLOC_MAX_ITEMS) return VSBPP_ECAPACITY;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return VSBPP_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (st) {
        // the scratch address and the SM count are the current device's: a
        // stream of another device would run on the wrong GPU's scratch
        int sdev = -1;
        if (cudaStreamGetDevice(st, &sdev) != cudaSuccess) return VSBPP_ECUDA;
        if (sdev != dev) return VSBPP_EINVAL;
    }
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* ptr = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr) return VSBPP_ECUDA;
            g_noalloc_ptr[dev] = static_cast<unsigned char*>(ptr);
        }
        base = g_noalloc_ptr[dev];
    }
    int32_t* cls = reinterpret_cast<int32_t*>(base + kOffCls);
    int32_t* order = reinterpret_cast<int32_t*>(base + kOffOrder);
    uint32_t* hist = reinterpret_cast<uint32_t*>(base + kOffHist);
    int64_t* cursor = reinterpret_cast<int64_t*>(base + kOffCursor);
    int64_t* seg = reinterpret_cast<int64_t*>(base + kOffSeg);
    unsigned long long* queue = reinterpret_cast<unsigned long long*>(base + kOffQueue);

    // launch shape: the block-group kernel with narrow slots for every instance
    vsbpp_config cfg;
    if (vsbpp_get_config(&cfg) != VSBPP_OK) return VSBPP_ECUDA;
    int sms = 0, smax = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return VSBPP_ECUDA;
    const int64_t cap_m = std::max<int64_t>(max_m, 1);
    const int slot_cap = static_cast<int>((2 * cap_m + kMaxTypes + 127) & ~int64_t(127));
    const int smem = h1_group_bytes(slot_cap, cfg.chunk, 4);
    if (smem > smax) return VSBPP_ECAPACITY;
    const int occ = h1_blocks_per_sm(false, cfg.large_warps, 1, smem);
    if (occ <= 0) return VSBPP_ECUDA;
    const int grid = static_cast<int>(std::min<int64_t>(int64_t(occ) * sms, N));

    BatchView in{N, w_all, w_off, 0, B_all, B_off, 0};
    OutView out{bin_of_item_all, bin_type_all, num_bins, total, status, nullptr, nullptr, nullptr};
    // the histogram must start at zero; the previous call left whatever it left
    if (cudaMemsetAsync(hist, 0, 4 * kClasses * kBuckets, st) != cudaSuccess) return VSBPP_ECUDA;
    PrepParams pp;
    std::memset(&pp, 0, sizeof(pp));
    pp.in = in;
    pp.out = out;
    pp.classify = 1;
    pp.small_m = 0;
    pp.narrow_cap = cap_m;
    pp.narrow_bins = 65536;
    pp.small_cap = 0;
    pp.wide_cap = 0;
    pp.huge_cap = 0;
    pp.narrow_max_B = 32767;
    pp.preopen = prm.preopen;
    pp.cls = cls;
    pp.hist = hist;
    const int prep_grid = static_cast<int>(std::min<int64_t>(int64_t(sms) * 8, (N + 7) / 8));
    if (validate_launch(pp, prep_grid, st) != cudaSuccess) return VSBPP_ECUDA;
    if (order_launch(hist, cursor, seg, queue, nullptr, st) != cudaSuccess) return VSBPP_ECUDA;
    if (scatter_launch(in, cls, cursor, order, prep_grid, st) != cudaSuccess) return VSBPP_ECUDA;
    H1Params hp;
    std::memset(&hp, 0, sizeof(hp));
    hp.in = in;
    hp.out = out;
    hp.criterion = prm.criterion;
    hp.preopen = prm.preopen;
    hp.seed = prm.seed;
    hp.order = order;
    hp.seg = seg;
    hp.segment = kClassLarge;
    hp.queue = queue + kClassLarge;
    hp.chunk = cfg.chunk;
    hp.slot_cap = slot_cap;
    hp.group_bytes = smem;
    hp.counters = counters_ptr();       // work counters, when enabled
    if (h1_launch(false, hp, cfg.large_warps, 1, grid, smem, st) != cudaSuccess) return VSBPP_ECUDA;
    return VSBPP_OK;
}
