// api.cu -- the C ABI of include/vsbpp.h: argument checks, scratch memory,
// launch planning (thread-group sizes, shared-memory capacities, persistent
// grids), CUDA-graph plans, and the host-memory convenience call.
//
// Every pack goes through the same device pipeline:
//   validate -> (first heuristic, one system per instance)
//                 order by size class and log2(m), largest first
//                 -> large-group kernel, single-warp kernel, wide-slot kernel
//            -> (sublists: first heuristic with s < m, or second heuristic)
//                 sublist prefix sums -> per-sublist kernel -> compose
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <numeric>
#include <queue>
#include <vector>

#include "internal.h"

using namespace vsbpp;

namespace {

// Locks.  g_mu guards the process-wide tables (launch configuration, work
// counters, the per-stream scratch map, per-device pools and host contexts)
// and is held only while they are read or changed.  Each stream's scratch,
// each plan and each device's host context has a lock of its own, held for
// a whole call, so calls on different streams or devices proceed at once.
std::recursive_mutex g_mu;
std::mutex g_timing_mu;          // the kernel-timing ring
std::atomic<int> g_last_cuda{0};
unsigned long long* g_counters = nullptr;   // device {items, fit tests} or null

// Kernel timing: a ring of CUDA event pairs recorded around the main
// packing launch of calls made outside stream capture.
struct KernelTiming {
    static constexpr int kRing = 256;
    bool on = false;
    int dev = -1;
    cudaEvent_t ev[kRing][2] = {};
    int head = 0, count = 0;       // pairs recorded since the last read (oldest at head - count)
} g_timing;

// Records the start event of the main launch on `st` when timing applies.
bool timing_begin(cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_timing_mu);
    if (!g_timing.on) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return false;
    int dev = 0;
    cudaGetDevice(&dev);
    if (g_timing.dev != dev) {
        for (auto& pr : g_timing.ev)
            for (auto& e : pr)
                if (e) { cudaEventDestroy(e); e = nullptr; }
        g_timing.dev = dev;
        g_timing.head = g_timing.count = 0;
    }
    auto& pr = g_timing.ev[g_timing.head];
    for (auto& e : pr)
        if (!e && cudaEventCreate(&e) != cudaSuccess) return false;
    return cudaEventRecord(pr[0], st) == cudaSuccess;
}

void timing_end(bool started, cudaStream_t st) {
    if (!started) return;
    std::lock_guard<std::mutex> lk(g_timing_mu);
    auto& pr = g_timing.ev[g_timing.head];
    if (cudaEventRecord(pr[1], st) != cudaSuccess) return;
    g_timing.head = (g_timing.head + 1) % KernelTiming::kRing;
    if (g_timing.count < KernelTiming::kRing) ++g_timing.count;
}

struct DeviceInfo {
    int dev = -1;
    int sms = 0;
    int max_smem_optin = 0;
};

// Attributes of the current device (cached per device).
DeviceInfo device_info() {
    static std::mutex mu;
    static std::map<int, DeviceInfo> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    DeviceInfo& di = cache[dev];
    if (di.dev != dev) {
        di.dev = dev;
        cudaDeviceGetAttribute(&di.sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&di.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    }
    return di;
}

// Defaults: the autotuner's choice on the 4096-instance benchmark batch
// (one warp per membrane system; systems of up to 6000 items in the smaller
// single-warp shape, beside the large class on a second stream).
vsbpp_config g_cfg = {
    /*large_warps=*/1,
    /*small_m=*/6000,
    /*small_warps_per_block=*/1,
    /*chunk=*/512,
    /*slot_pct=*/80,
    /*h2_blocks_per_sm=*/0,
};

int record(cudaError_t e) {
    if (e == cudaSuccess) return VSBPP_OK;
    g_last_cuda.store(static_cast<int>(e));
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? VSBPP_ENOMEM : VSBPP_ECUDA;
}

#define VS_TRY(expr)                              \
    do {                                          \
        const int _rc = record(expr);             \
        if (_rc != VSBPP_OK) return _rc;          \
    } while (0)

// The memory pool of stream-ordered scratch on the current device: memory a
// stream frees is kept for reuse (no release threshold), and is handed to
// another stream only once the free has completed, never by making that
// stream wait on the freeing one.  Null where pools are unsupported.
cudaMemPool_t scratch_pool() {
    static std::map<int, cudaMemPool_t> pools;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    auto it = pools.find(dev);
    if (it != pools.end()) return it->second;
    cudaMemPool_t pool = nullptr;
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        pool = nullptr;
    } else {
        uint64_t keep = ~0ull;
        int no = 0;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
    }
    pools[dev] = pool;
    return pool;
}

// Scratch owned by the library for one stream (or one plan).
//
// Scratch bound to a stream (the per-stream scratch of the batched and
// single-instance calls) grows with the stream-ordered allocator on that
// stream: freeing an outgrown buffer then waits only for that stream's earlier
// work, where cudaFree would wait for the whole device, every other stream's
// kernels included (a server packing on several streams would stall its
// admissions behind its longest request).  Plan scratch (read by recorded
// graphs), and buffers made while the stream is being captured, come from
// cudaMalloc; an outgrown buffer met under capture is set aside and freed by
// the next call made outside capture.
struct Scratch {
    std::shared_ptr<std::recursive_mutex> mu = std::make_shared<std::recursive_mutex>();   // held for a call
    bool ordered = false;            // grows in stream order on `ord`
    cudaStream_t ord = nullptr;
    std::vector<void*> sync_bufs;    // cudaMalloc buffers of an ordered scratch
    std::vector<void*> retired;      // outgrown under capture, not yet freed

    int32_t* cls = nullptr;        int64_t cap_cls = 0;
    int32_t* order = nullptr;      int64_t cap_order = 0;
    int64_t* nu = nullptr;         int64_t cap_nu = 0;
    int64_t* unit_base = nullptr;  int64_t cap_unit_base = 0;
    int32_t* unit_count = nullptr; int64_t cap_unit_count = 0;
    int64_t* unit_total = nullptr; int64_t cap_unit_total = 0;
    int32_t* local_types = nullptr; int64_t cap_local_types = 0;
    uint8_t* fixed = nullptr;      // histogram, cursors, segments, queues
    // host-memory call staging
    int32_t* h_w = nullptr;    int64_t cap_h_w = 0;
    int32_t* h_B = nullptr;    int64_t cap_h_B = 0;
    int32_t* h_boi = nullptr;  int64_t cap_h_boi = 0;
    int32_t* h_bt = nullptr;   int64_t cap_h_bt = 0;
    int64_t* h_small = nullptr; int64_t cap_h_small = 0;   // num_bins, total, status

    uint32_t* kc_slots = nullptr; int64_t cap_kc_slots = 0;   // global-memory bins
    int32_t* spill_list = nullptr; int64_t cap_spill_list = 0;  // systems to repack at full size
    int32_t* spill_list2 = nullptr; int64_t cap_spill_list2 = 0;  // ... and those beyond it (global memory)
    unsigned long long* h2x_best = nullptr; int64_t cap_h2x_best = 0;  // exhaustive search: best key per sublist
    // offline pre-sort: sorted weights, permutation, radix buffer, sorted-order bin ids, caller-order status
    int32_t* ps_w = nullptr;    int64_t cap_ps_w = 0;
    int32_t* ps_perm = nullptr; int64_t cap_ps_perm = 0;
    int32_t* ps_tmp = nullptr;  int64_t cap_ps_tmp = 0;
    int32_t* ps_boi = nullptr;  int64_t cap_ps_boi = 0;
    int32_t* ps_stat = nullptr; int64_t cap_ps_stat = 0;
    int32_t* bk_rec = nullptr;  int64_t cap_bk_rec = 0;     // bounded space: per-bin records
    uint16_t* kd_over = nullptr; int64_t cap_kd_over = 0;  // cluster kernel: bins past shared memory
    // a second stream for the single-warp class, forked from and joined to
    // the caller's stream by events (captured into graphs as fork / join)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int32_t* kd_dense = nullptr; int64_t cap_kd_dense = 0; // cluster kernel: dense id per bin
    // host-memory batch call: device copies of the CSR offsets and the per-instance outputs
    int64_t* hb_woff = nullptr; int64_t cap_hb_woff = 0;
    int32_t* hb_Boff = nullptr; int64_t cap_hb_Boff = 0;
    int64_t* hb_nb = nullptr;   int64_t cap_hb_nb = 0;
    int64_t* hb_tot = nullptr;  int64_t cap_hb_tot = 0;
    int32_t* hb_st = nullptr;   int64_t cap_hb_st = 0;

    uint32_t* hist() const { return reinterpret_cast<uint32_t*>(fixed); }
    int64_t* cursor() const { return reinterpret_cast<int64_t*>(fixed + kClasses * kBuckets * 4); }
    int64_t* seg() const { return cursor() + kClasses * kBuckets; }
    int64_t* seg_units() const { return seg() + 8; }
    unsigned long long* queue() const { return reinterpret_cast<unsigned long long*>(seg_units() + 8); }
    int64_t* spill_seg() const { return reinterpret_cast<int64_t*>(queue() + 8); }
    static size_t fixed_bytes() { return kClasses * kBuckets * 4 + kClasses * kBuckets * 8 + 32 * 8; }

    bool stream_order() const {
        if (!ordered) return false;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        return cudaStreamIsCapturing(ord, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
    }
    int alloc(void** q, size_t bytes) {
        *q = nullptr;
        if (stream_order()) {
            cudaMemPool_t pool = scratch_pool();
            return record(pool ? cudaMallocFromPoolAsync(q, bytes, pool, ord) : cudaMallocAsync(q, bytes, ord));
        }
        const cudaError_t e = cudaMalloc(q, bytes);
        if (e == cudaSuccess && ordered) sync_bufs.push_back(*q);
        return record(e);
    }
    // Frees now: in stream order for a stream-ordered buffer.
    void free_buf(void* q) {
        if (!q) return;
        auto it = std::find(sync_bufs.begin(), sync_bufs.end(), q);
        if (!ordered || it != sync_bufs.end()) {
            if (it != sync_bufs.end()) sync_bufs.erase(it);
            cudaFree(q);
        } else {
            cudaFreeAsync(q, ord);
        }
    }
    // An outgrown buffer: freed now, or set aside while the stream is captured.
    void drop(void* q) {
        if (!q) return;
        if (ordered && !stream_order()) retired.push_back(q);
        else free_buf(q);
    }
    void free_retired() {
        if (retired.empty() || !stream_order()) return;
        for (void* q : retired) free_buf(q);
        retired.clear();
    }
    template <typename T>
    int grow(T*& p, int64_t& cap, int64_t need) {
        if (need <= cap && p) return VSBPP_OK;
        int64_t n = std::max<int64_t>(need, 1);
        n = std::max<int64_t>(n, cap + cap / 2);
        drop(p);
        p = nullptr;
        cap = 0;
        void* q = nullptr;
        const int rc = alloc(&q, static_cast<size_t>(n) * sizeof(T));
        if (rc != VSBPP_OK) return rc;
        p = static_cast<T*>(q);
        cap = n;
        return VSBPP_OK;
    }

    int ensure_side() {
        if (side) return VSBPP_OK;
        VS_TRY(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
        VS_TRY(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
        return record(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
    }

    int ensure_fixed() {
        if (fixed) return VSBPP_OK;
        void* q = nullptr;
        int rc = alloc(&q, fixed_bytes());
        if (rc != VSBPP_OK) return rc;
        const cudaError_t e = stream_order() ? cudaMemsetAsync(q, 0, fixed_bytes(), ord)
                                             : cudaMemset(q, 0, fixed_bytes());
        if (e != cudaSuccess) {
            free_buf(q);
            return record(e);
        }
        fixed = static_cast<uint8_t*>(q);
        return VSBPP_OK;
    }

    void release() {
        void* bufs[] = {cls, order, nu, unit_base, unit_count, unit_total, local_types, fixed, kc_slots,
                        spill_list, spill_list2, h2x_best, h_w, h_B, h_boi, h_bt, h_small,
                        ps_w, ps_perm, ps_tmp, ps_boi, ps_stat, bk_rec, hb_woff, hb_Boff, hb_nb,
                        hb_tot, hb_st, kd_over, kd_dense};
        for (void* q : bufs) free_buf(q);
        for (void* q : retired) free_buf(q);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (side) cudaStreamDestroy(side);
        auto keep = mu;
        *this = Scratch();
        mu = keep;
    }
};

std::map<cudaStream_t, Scratch>& stream_scratch() {
    static std::map<cudaStream_t, Scratch> m;
    return m;
}

// The scratch of stream `st` (created on first use, growing in stream order).
// The map's nodes never move, so the reference stays valid; the caller holds
// the scratch's own lock while it uses it.
Scratch& scratch_for(cudaStream_t st) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    auto& m = stream_scratch();
    auto it = m.find(st);
    if (it == m.end()) {
        it = m.emplace(st, Scratch()).first;
        it->second.ordered = true;
        it->second.ord = st;
    }
    return it->second;
}

// The library's own stream and pinned staging on one device, for the calls
// that take host buffers (vsbpp_pack, vsbpp_pack_batch_host).  Pageable host
// memory is copied through two pinned chunks, so the host copy of one chunk
// overlaps the transfer of the other.
struct HostCtx {
    static constexpr size_t kChunk = size_t(8) << 20;
    int dev = -1;
    bool ready = false;              // every resource below exists
    cudaStream_t st = nullptr;
    void* pin[2] = {nullptr, nullptr};
    cudaEvent_t ev[2] = {nullptr, nullptr};

    // Creates whatever is still missing (a failed earlier attempt is
    // completed, not taken for done).
    int init() {
        if (ready) return VSBPP_OK;
        if (!st) {
            cudaStream_t x = nullptr;
            VS_TRY(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
            st = x;
        }
        for (int k = 0; k < 2; ++k) {
            if (!pin[k]) {
                void* x = nullptr;
                VS_TRY(cudaHostAlloc(&x, kChunk, cudaHostAllocDefault));
                pin[k] = x;
            }
            if (!ev[k]) {
                cudaEvent_t x = nullptr;
                VS_TRY(cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
                ev[k] = x;
            }
        }
        ready = true;
        return VSBPP_OK;
    }
    static bool pinned(const void* p) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return a.type == cudaMemoryTypeHost;
    }
    // host -> device, enqueued on st (pageable sources go through the chunks)
    int to_device(void* dst, const void* src, size_t bytes) {
        if (bytes == 0) return VSBPP_OK;
        if (pinned(src)) return record(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
        int k = 0;
        for (size_t off = 0; off < bytes; off += kChunk, k ^= 1) {
            const size_t n = std::min(kChunk, bytes - off);
            VS_TRY(cudaEventSynchronize(ev[k]));          // the chunk's previous transfer is done
            std::memcpy(pin[k], static_cast<const char*>(src) + off, n);
            VS_TRY(cudaMemcpyAsync(static_cast<char*>(dst) + off, pin[k], n, cudaMemcpyHostToDevice, st));
            VS_TRY(cudaEventRecord(ev[k], st));
        }
        return VSBPP_OK;
    }
    // device -> host after the work enqueued on st; returns when the copy is done
    int to_host(void* dst, const void* src, size_t bytes) {
        if (bytes == 0) return VSBPP_OK;
        if (pinned(dst)) return record(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st));
        int k = 0;
        size_t prev_off = 0, prev_n = 0;
        for (size_t off = 0; off < bytes; off += kChunk, k ^= 1) {
            const size_t n = std::min(kChunk, bytes - off);
            VS_TRY(cudaMemcpyAsync(pin[k], static_cast<const char*>(src) + off, n, cudaMemcpyDeviceToHost, st));
            VS_TRY(cudaEventRecord(ev[k], st));
            if (prev_n) {                                  // the other chunk, copied while this one moves
                VS_TRY(cudaEventSynchronize(ev[k ^ 1]));
                std::memcpy(static_cast<char*>(dst) + prev_off, pin[k ^ 1], prev_n);
            }
            prev_off = off;
            prev_n = n;
        }
        VS_TRY(cudaEventSynchronize(ev[k ^ 1]));
        std::memcpy(static_cast<char*>(dst) + prev_off, pin[k ^ 1], prev_n);
        return VSBPP_OK;
    }
};

// Host contexts of each device.  A host-memory call borrows one for its
// whole length (a free one, or a new one when all are in use) and gives it
// back at the end, so calls from several host threads run side by side, each
// on its own stream with its own staging and scratch.  Contexts are kept for
// reuse until the process exits.
struct HostPool {
    std::deque<HostCtx> all;        // stable addresses
    std::vector<HostCtx*> free_list;
};

std::map<int, HostPool>& host_pools() {
    static std::map<int, HostPool> pools;
    return pools;
}

void host_ctx_release(HostCtx* c) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    host_pools()[c->dev].free_list.push_back(c);
}

// A context of the current device, held until the lease ends.
struct HostLease {
    HostCtx* c = nullptr;
    HostLease() {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return;
        HostCtx* got = nullptr;
        {
            std::lock_guard<std::recursive_mutex> lk(g_mu);
            HostPool& pool = host_pools()[dev];
            if (!pool.free_list.empty()) {
                got = pool.free_list.back();
                pool.free_list.pop_back();
            } else {
                pool.all.emplace_back();
                got = &pool.all.back();
                got->dev = dev;
            }
        }
        if (got->init() != VSBPP_OK) {
            host_ctx_release(got);
            return;
        }
        c = got;
    }
    ~HostLease() {
        if (c) host_ctx_release(c);
    }
    HostLease(const HostLease&) = delete;
    HostLease& operator=(const HostLease&) = delete;
};

// ------------------------------------------------------------ launch plan
struct Mode {
    int heuristic;
    int compose;          // 1: sublists (first heuristic with s < max_m, or second heuristic)
    int64_t s;            // sublist size in compose mode
};

struct H1Shape {
    int G, groups;
    int chunk;
    int bf_index;         // BF residual index laid out in shared memory
    int slot_cap;
    int smem;
    int grid;
    int64_t cap_m;        // largest membrane system (items) the shape holds
    bool warp_kernel;     // the one-warp kernel (G = 1, narrow, <= 32768 bins)
};

// Global-memory kernel for membrane systems beyond shared memory.
struct KCShape {
    bool enabled = false;
    int64_t cap_m = 0;        // largest m it holds
    int64_t bin_cap = 0;      // bins of scratch per block
    int pres_words = 0;       // 0 unless the criterion needs residual presence (BF, RANDOM)
    int max_B1 = 0;
    int smem = 0;
    int grid = 0;
};

// Cluster kernel for the systems beyond shared memory whose B_1 and bins fit
// its 16-bit slots (the rest go to the global-memory kernel).
struct KDShape {
    bool enabled = false;
    int smem = 0;
    int segs0 = 0, segs1 = 0;
    int max_B1 = 0;
    int pres = 0;
    int clusters = 0;
    int64_t over_bins = 0;
};

struct LaunchPlan {
    Mode mode;
    unsigned long long* counters = nullptr;   // work counters when the plan was made (or null)
    KDShape kd{};
    vsbpp_config cfg;
    H1Shape large{}, small{}, wide{}, sub{};
    H1Shape full{};       // worst-case slots: repacks systems that outgrew large/small
    int64_t large16_cap_m = 0;   // one-warp 16-bit slots (B_1 <= 255): largest m taken (0: none)
    KCShape kc{};
    int h2_threads = 0, h2_smem = 0, h2_grid = 0, h2_max_bins = 0;
    bool h2x = false;     // sublists of 7..12 items: the exhaustive search
    bool h2_generic = false;   // second heuristic in the one-thread-per-permutation kernel
    bool presort = false;      // VSBPP_PRESORT: sort, pack the sorted copy, scatter back
    bool remark3 = false;      // VSBPP_REMARK3
    bool bounded = false;      // max_open > 0: the bounded-space kernel
    int bk_grid = 0;
    int prep_grid = 0;
};

// The process-wide settings a launch plan reads, copied under g_mu.
struct Snapshot {
    vsbpp_config cfg;
    unsigned long long* counters;
};

Snapshot snapshot() {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    return Snapshot{g_cfg, g_counters};
}

int round4(int64_t x) { return static_cast<int>((x + 3) & ~int64_t(3)); }
// Shared-memory kernels read whole 128-bin segments.
int round128(int64_t x) { return static_cast<int>((x + 127) & ~int64_t(127)); }

// Shared memory of one group: the one-warp kernel's layout where it applies
// (h1w_ok: the one-warp kernel may be used).
int group_bytes(bool wide, int G, int slot_cap, int chunk, int bf_index, bool h1w_ok) {
    if (h1w_ok && !wide && G == 1 && h1w_supported(slot_cap)) return h1w_bytes(slot_cap, bf_index);
    return h1_group_bytes(slot_cap, chunk, wide ? 8 : 4, G, bf_index);
}

// Largest m whose group footprint fits `budget` bytes (slot_cap = 2m + 32).
int64_t cap_for_budget(int budget, bool wide, int chunk, int G, int bf_index, bool h1w_ok) {
    int64_t lo = 0, hi = 1 << 22;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) / 2;
        const int64_t sc = round128(2 * mid + kMaxTypes);
        const int64_t bytes = group_bytes(wide, G, static_cast<int>(std::min<int64_t>(sc, 1 << 26)), chunk,
                                          bf_index, h1w_ok);
        if (bytes <= budget) lo = mid; else hi = mid;
    }
    return lo;
}

// cap_m = the largest system whose worst case (2m + 32 slots) the shape could
// hold; slot_cap = pct% of that plus 64 (never above the worst case).
int make_shape(H1Shape& sh, bool wide, int G, int groups, int64_t want_m, int chunk, int smem_max,
               int sms, int64_t hard_cap, int pct, int bf_index, int criterion, bool spills = false,
               bool h1w_ok = true) {
    sh.chunk = chunk;
    sh.bf_index = bf_index;
    int64_t cap = std::min<int64_t>(want_m, cap_for_budget(smem_max / groups, wide, chunk, G, bf_index, h1w_ok));
    if (spills && h1w_ok && !wide && G == 1) {
        // The one-warp kernel spills a system that outgrows its slots (it is
        // packed again by the worst-case shape, or in global memory), so its
        // reach is set by the pct estimate rather than the worst case.
        int64_t lo = cap, hi = want_m + 1;
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) / 2;
            const int64_t sc = round128(mid * pct / 100 + 64);
            const bool fits = h1w_supported(static_cast<int>(std::min<int64_t>(sc, 1 << 30))) &&
                              group_bytes(false, 1, static_cast<int>(sc), chunk, bf_index, true) <=
                                                         smem_max / groups;
            if (fits) lo = mid; else hi = mid;
        }
        cap = lo;
    }
    cap = std::min<int64_t>(cap, hard_cap);
    cap = std::max<int64_t>(cap, 1);
    sh.G = G;
    sh.groups = groups;
    sh.cap_m = cap;
    sh.slot_cap = std::min(round128(2 * cap + kMaxTypes), round128(cap * pct / 100 + 64));
    sh.warp_kernel = h1w_ok && !wide && G == 1 && h1w_supported(sh.slot_cap);
    sh.smem = group_bytes(wide, G, sh.slot_cap, chunk, bf_index, h1w_ok) * groups;
    if (sh.smem > smem_max) return VSBPP_ECAPACITY;
    const int occ = sh.warp_kernel ? h1w_blocks_per_sm(sh.slot_cap, criterion, groups, sh.smem)
                                   : h1_blocks_per_sm(wide, G, groups, sh.smem);
    if (occ <= 0) return record(cudaErrorInvalidConfiguration);
    sh.grid = occ * sms;
    return VSBPP_OK;
}

// Launch one shape's kernel.
cudaError_t launch_shape(const H1Shape& sh, bool wide, const H1Params& p, int groups, int grid,
                         cudaStream_t st) {
    if (sh.warp_kernel && !wide) return h1w_launch(p, groups, grid, sh.smem, st);
    return h1_launch(wide, p, sh.G, groups, grid, sh.smem, st);
}

int check_params(const vsbpp_params* p) { return check_params_public(p); }

vsbpp_params defaults(const vsbpp_params* p) {
    vsbpp_params q;
    std::memset(&q, 0, sizeof(q));
    q.heuristic = VSBPP_H1;
    q.criterion = VSBPP_BF;
    if (p) q = *p;
    return q;
}

// Persistent grids never need more groups than there are units of work.
void cap_grid(H1Shape& sh, int64_t units) {
    const int64_t blocks = (std::max<int64_t>(units, 1) + sh.groups - 1) / sh.groups;
    if (blocks < sh.grid) sh.grid = static_cast<int>(blocks);
}

int build_plan(const vsbpp_params& prm, int64_t max_m, int64_t N, LaunchPlan& lp, const Snapshot& snap) {
    const DeviceInfo di = device_info();
    if (di.sms <= 0) return record(cudaErrorNoDevice);
    lp.cfg = snap.cfg;
    lp.counters = snap.counters;
    const int chunk = lp.cfg.chunk;
    const int smax = di.max_smem_optin;
    max_m = std::max<int64_t>(max_m, 1);
    lp.prep_grid = di.sms * 8;
    lp.presort = (prm.flags & VSBPP_PRESORT) != 0;
    lp.remark3 = (prm.flags & VSBPP_REMARK3) != 0;
    if (prm.heuristic == VSBPP_H2) {
        const int s = static_cast<int>(prm.sublist_size == 0 ? 5 : prm.sublist_size);
        lp.mode = {VSBPP_H2, 1, s};
        if (s >= 7) {
            // s! permutations per sublist searched across the GPU (no
            // pre-opened bins on this path)
            if (prm.preopen) return VSBPP_EINVAL;
            lp.h2x = true;
            const int occ = h2x_blocks_per_sm(s, prm.criterion);
            if (occ <= 0) return record(cudaErrorInvalidConfiguration);
            lp.h2_grid = occ * di.sms;
            return VSBPP_OK;
        }
        int f = 1;
        for (int x = 2; x <= s; ++x) f *= x;
        // literal Rule 2 start or Remark 3: one thread per permutation
        // (shared-memory bins); otherwise four warps per block, one sublist
        // per warp, bins in registers
        lp.h2_generic = prm.preopen || lp.remark3;
        lp.h2_threads = lp.h2_generic ? std::max(32, (f + 31) / 32 * 32) : 128;
        lp.h2_max_bins = 2 * s + (prm.preopen ? kMaxTypes : 0);
        lp.h2_smem = h2_smem_bytes(lp.h2_threads, lp.h2_max_bins);
        int occ = lp.h2_generic ? h2_blocks_per_sm(lp.h2_threads, lp.h2_smem)
                                : h2_blocks_per_sm_reg(lp.h2_threads, s, prm.criterion);
        if (lp.cfg.h2_blocks_per_sm > 0) occ = std::min(occ, lp.cfg.h2_blocks_per_sm);
        if (occ <= 0) return record(cudaErrorInvalidConfiguration);
        lp.h2_grid = occ * di.sms;
        const int64_t units = N * ((max_m + s - 1) / s);
        if (units < lp.h2_grid) lp.h2_grid = static_cast<int>(std::max<int64_t>(units, 1));
        return VSBPP_OK;
    }
    const int64_t s = prm.sublist_size;
    if (prm.max_open > 0) {
        // bounded space: one membrane system per instance, one warp each,
        // the open bins in registers
        if (s > 0 && s < max_m) return VSBPP_EINVAL;
        lp.mode = {VSBPP_H1, 0, 0};
        lp.bounded = true;
        const int occ = bk_blocks_per_sm();
        if (occ <= 0) return record(cudaErrorInvalidConfiguration);
        lp.bk_grid = static_cast<int>(std::max<int64_t>(
            1, std::min<int64_t>(int64_t(occ) * di.sms, (N + kBKWarpsPerBlock - 1) / kBKWarpsPerBlock)));
        return VSBPP_OK;
    }
    if (s > 0 && s < max_m) {
        lp.mode = {VSBPP_H1, 1, s};
        const bool one_warp = s <= lp.cfg.small_m;
        const int G = one_warp ? 1 : lp.cfg.large_warps;
        const int groups = one_warp ? lp.cfg.small_warps_per_block : 1;
        const int sub_chunk = one_warp ? std::min(chunk, 256) : chunk;
        const int bfi = prm.criterion == VSBPP_BF || prm.criterion == VSBPP_RANDOM;
        int rc = make_shape(lp.sub, true, G, groups, s, sub_chunk, smax, di.sms, 1 << 30, 200, bfi,
                            prm.criterion);
        if (rc != VSBPP_OK) return rc;
        if (lp.sub.cap_m < s) return VSBPP_ECAPACITY;
        cap_grid(lp.sub, N * ((max_m + s - 1) / s));
        return VSBPP_OK;
    }
    lp.mode = {VSBPP_H1, 0, 0};
    // the BF residual index is laid out when BF items can occur
    const int bfi = prm.criterion == VSBPP_BF || prm.criterion == VSBPP_RANDOM;
    // the one-warp kernel takes every option (Remark 3 in kernels of their
    // own: a lane-distributed count of each type's bins below half)
    const bool h1w_ok = true;
    int rc = make_shape(lp.full, false, lp.cfg.large_warps, 1, max_m, chunk, smax, di.sms, 32752, 200, bfi,
                        prm.criterion, false, h1w_ok);
    if (rc != VSBPP_OK) return rc;
    rc = make_shape(lp.large, false, lp.cfg.large_warps, 1, max_m, chunk, smax, di.sms, 1 << 30,
                    lp.cfg.slot_pct, bfi, prm.criterion, true, h1w_ok);
    if (rc != VSBPP_OK) return rc;
    rc = make_shape(lp.small, false, 1, lp.cfg.small_warps_per_block,
                    std::min<int64_t>(max_m, std::max(1, lp.cfg.small_m)), std::min(chunk, 256), smax,
                    di.sms, 32752, lp.cfg.slot_pct, bfi, prm.criterion, true, h1w_ok);
    if (rc != VSBPP_OK) return rc;
    rc = make_shape(lp.wide, true, lp.cfg.large_warps, 1, max_m, chunk, smax, di.sms, 1 << 30, 200, bfi,
                    prm.criterion);
    if (rc != VSBPP_OK) return rc;
    // systems with B_1 <= 255 past the large shape's reach (only the largest
    // one-warp shape has any) take 16-bit slots in the same warp's shared
    // memory, grown to the 16-bit layout (one warp per SM either way),
    // admitted while 60% of their items would fill the slots; those that
    // outgrow them go to global memory
    lp.large16_cap_m = 0;
    if (lp.large.warp_kernel && lp.large.groups == 1 && h1w_segment_words(lp.large.slot_cap) == 8) {
        const int64_t cap16 = std::min<int64_t>(max_m, (h1w16_slots() - 64) * 100 / 60);
        const int bytes16 = h1w16_bytes(bfi);
        if (cap16 > lp.large.cap_m && bytes16 <= smax) {
            lp.large16_cap_m = cap16;
            if (bytes16 > lp.large.smem) {
                lp.large.smem = bytes16;
                const int occ = h1w_blocks_per_sm(lp.large.slot_cap, prm.criterion, 1, bytes16);
                if (occ <= 0) return record(cudaErrorInvalidConfiguration);
                lp.large.grid = occ * di.sms;
            }
        }
    }
    cap_grid(lp.large, N);
    cap_grid(lp.small, N);
    cap_grid(lp.wide, N);
    cap_grid(lp.full, N);
    // global memory for systems beyond the shared-memory classes, and for
    // those that outgrow even the worst-case shape after a spill
    if (max_m > std::min(lp.large.cap_m, lp.full.cap_m)) {
        KCShape& kc = lp.kc;
        kc.enabled = true;
        const int64_t want_bins = std::min<int64_t>(2 * max_m + kMaxTypes, int64_t(kMaxTiles) * kTileBins);
        kc.bin_cap = (want_bins + kTileBins - 1) / kTileBins * kTileBins;
        kc.cap_m = (kc.bin_cap - kMaxTypes) / 2;
        const int tiles = static_cast<int>(kc.bin_cap / kTileBins);
        const bool track = prm.criterion == VSBPP_BF || prm.criterion == VSBPP_RANDOM;
        kc.pres_words = track ? (tiles + 31) / 32 : 0;
        int b1 = 32767;
        while (b1 > 0 && kc_smem_bytes(b1, kc.pres_words) > smax) b1 = b1 * 7 / 8;
        kc.max_B1 = b1;
        kc.smem = kc_smem_bytes(kc.max_B1, kc.pres_words);
        const int occ = kc_blocks_per_sm(kc.smem);
        if (occ <= 0) return record(cudaErrorInvalidConfiguration);
        kc.grid = static_cast<int>(std::min<int64_t>(int64_t(occ) * di.sms, std::max<int64_t>(N, 1)));
    }
    if (!lp.kc.enabled) lp.large16_cap_m = 0;     // no global-memory fallback for its spills
    if (lp.kc.enabled) {
        // the systems of the global-memory class go to two-CTA clusters first:
        // 16-bit slots in both CTAs' shared memory (B_1 <= 1023 with BF items,
        // whose presence rows take 128 KB of CTA 0; else B_1 <= 2047)
        KDShape& kd = lp.kd;
        kd.pres = bfi;
        kd.max_B1 = kd.pres ? kKDMaxB1Idx : kKDMaxB1;
        kd.smem = smax;
        kd.segs1 = kd.smem / kKDSegBytes;
        kd.segs0 = (kd.smem - kd_bins_offset(kd.max_B1, kd.pres)) / kKDSegBytes;
        kd.over_bins = std::max<int64_t>(0, int64_t(kKDMaxBins) - int64_t(kd.segs0 + kd.segs1) * kKDSeg);
        const int mc = kd.segs0 > 0 ? kd_max_clusters(prm.criterion, kd.smem) : 0;
        kd.clusters = static_cast<int>(std::min<int64_t>(mc, std::max<int64_t>(N, 1)));
        kd.enabled = kd.clusters > 0;
    }
    return VSBPP_OK;
}

int ensure_scratch(Scratch& sc, const LaunchPlan& lp, int64_t N, int64_t total_m) {
    sc.free_retired();
    int rc = sc.ensure_fixed();
    if (rc) return rc;
    if ((rc = sc.grow(sc.cls, sc.cap_cls, N))) return rc;
    if (lp.presort) {
        if ((rc = sc.grow(sc.ps_w, sc.cap_ps_w, total_m))) return rc;
        if ((rc = sc.grow(sc.ps_perm, sc.cap_ps_perm, total_m))) return rc;
        if ((rc = sc.grow(sc.ps_tmp, sc.cap_ps_tmp, total_m))) return rc;
        if ((rc = sc.grow(sc.ps_boi, sc.cap_ps_boi, total_m))) return rc;
        if ((rc = sc.grow(sc.ps_stat, sc.cap_ps_stat, N))) return rc;
    }
    if (!lp.mode.compose) {
        if (lp.bounded && (rc = sc.grow(sc.bk_rec, sc.cap_bk_rec, 2 * total_m + int64_t(kMaxTypes) * N)))
            return rc;
        if (lp.cfg.small_m > 0 && (rc = sc.ensure_side())) return rc;
        if ((rc = sc.grow(sc.order, sc.cap_order, N))) return rc;
        if ((rc = sc.grow(sc.spill_list, sc.cap_spill_list, N))) return rc;
        if ((rc = sc.grow(sc.spill_list2, sc.cap_spill_list2, N))) return rc;
        if (lp.kc.enabled && (rc = sc.grow(sc.kc_slots, sc.cap_kc_slots, int64_t(lp.kc.grid) * lp.kc.bin_cap)))
            return rc;
        if (lp.kd.enabled) {
            if ((rc = sc.grow(sc.kd_over, sc.cap_kd_over, std::max<int64_t>(1, lp.kd.clusters * lp.kd.over_bins))))
                return rc;
            if ((rc = sc.grow(sc.kd_dense, sc.cap_kd_dense, int64_t(lp.kd.clusters) * kKDMaxBins))) return rc;
        }
        return VSBPP_OK;
    }
    const int64_t U = total_m / std::max<int64_t>(lp.mode.s, 1) + N;   // >= sum ceil(m_i/s)
    if ((rc = sc.grow(sc.nu, sc.cap_nu, N))) return rc;
    if ((rc = sc.grow(sc.unit_base, sc.cap_unit_base, N + 1))) return rc;
    if ((rc = sc.grow(sc.unit_count, sc.cap_unit_count, U))) return rc;
    if (lp.h2x && (rc = sc.grow(sc.h2x_best, sc.cap_h2x_best, U))) return rc;
    if ((rc = sc.grow(sc.unit_total, sc.cap_unit_total, U))) return rc;
    if ((rc = sc.grow(sc.local_types, sc.cap_local_types, total_m))) return rc;
    return VSBPP_OK;
}

H1Params h1_params(const BatchView& in, const OutView& out, const vsbpp_params& prm,
                   const H1Shape& sh, unsigned long long* counters) {
    H1Params p;
    std::memset(&p, 0, sizeof(p));
    p.in = in;
    p.out = out;
    p.units.unit_base = nullptr;
    p.units.sublist = 0;
    p.units.num_units = 0;
    p.criterion = prm.criterion;
    p.preopen = prm.preopen;
    p.remark3 = (prm.flags & VSBPP_REMARK3) ? 1 : 0;
    p.no_trend = (prm.flags & VSBPP_PRESORT) ? 1 : 0;
    p.seed = prm.seed;
    p.chunk = sh.chunk;
    p.slot_cap = sh.slot_cap;
    p.group_bytes = sh.smem / sh.groups;
    p.cls = nullptr;
    p.want_cls = 0;
    p.counters = counters;
    p.bf_index = sh.bf_index;
    return p;
}

// The large class's 16-bit slot systems: m past the 32-bit reach, B_1 <= 255;
// those that outgrow the slots are listed for global memory.
void set_h16(H1Params& p, const LaunchPlan& lp, Scratch& sc) {
    if (lp.large16_cap_m <= 0 || !lp.kc.enabled) return;
    p.h16_min_m = lp.large.cap_m + 1;
    p.spill_list2 = sc.spill_list2;
    p.spill_seg2 = sc.spill_seg() + 2;
}

// Enqueue the whole pipeline on `st`.  plain = one launch per instance.
// split: the single-warp class may run on the second stream (batched device
// calls and plans; see the caller).
int enqueue_core(const LaunchPlan& lp, Scratch& sc, const BatchView& in, const OutView& out0,
                 const vsbpp_params& prm, bool plain, cudaStream_t st, bool split_ok) {
    if (in.N == 0) return VSBPP_OK;
    OutView out = out0;
    PrepParams pp;
    std::memset(&pp, 0, sizeof(pp));
    pp.in = in;
    pp.out = out;
    pp.preopen = prm.preopen;
    pp.cls = sc.cls;
    pp.hist = sc.hist();
    pp.narrow_max_B = SlotTraits<uint32_t>::kMaxCap;
    const int prep_grid = static_cast<int>(std::min<int64_t>(lp.prep_grid, (in.N + 7) / 8));

    // the single-warp class runs beside the large one on the second stream,
    // or not at all (every system in the large class)
    const bool split = !plain && split_ok && lp.cfg.small_m > 0 && sc.side;
    if (!lp.mode.compose) {
        pp.classify = 1;
        pp.small_m = split ? lp.cfg.small_m : 0;
        pp.narrow_cap = lp.large.cap_m;
        pp.narrow_bins = lp.large.warp_kernel ? (int64_t(1) << 40) : 65536;   // one-warp shapes spill instead
        pp.narrow_cap16 = lp.large16_cap_m;
        pp.small_cap = lp.small.cap_m;
        pp.wide_cap = lp.wide.cap_m;
        pp.huge_cap = lp.kc.enabled ? lp.kc.cap_m : 0;
        pp.huge_max_B1 = lp.kc.max_B1;
        pp.one_class = lp.bounded ? 1 : 0;
        VS_TRY(validate_launch(pp, prep_grid, st));
        VS_TRY(order_launch(sc.hist(), sc.cursor(), sc.seg(), sc.queue(), sc.spill_seg(), st));
        VS_TRY(scatter_launch(in, sc.cls, sc.cursor(), sc.order, prep_grid, st));
        if (lp.bounded) {
            // bounded space: one warp per membrane system, largest first
            BKParams bp;
            std::memset(&bp, 0, sizeof(bp));
            bp.in = in;
            bp.out = out;
            bp.criterion = prm.criterion;
            bp.preopen = prm.preopen;
            bp.max_open = static_cast<int32_t>(prm.max_open);
            bp.seed = prm.seed;
            bp.rec = sc.bk_rec;
            bp.counters = lp.counters;
            if (plain) {
                for (int64_t i = 0; i < in.N; ++i) {       // one single-warp launch per instance
                    bp.range_begin = i;
                    bp.range_end = i + 1;
                    VS_TRY(bk_launch(bp, 1, st));
                }
                return VSBPP_OK;
            }
            bp.order = sc.order;
            bp.seg = sc.seg();
            bp.segment = kClassLarge;
            bp.queue = sc.queue() + kClassLarge;
            const bool timed = timing_begin(st);
            VS_TRY(bk_launch(bp, lp.bk_grid, st));
            timing_end(timed, st);
            return VSBPP_OK;
        }
        const H1Shape* shapes[3] = {&lp.large, &lp.small, &lp.wide};
        // the single-warp class (smaller slots, more warps per SM) runs beside
        // the large one on a second stream: its blocks take the shared memory
        // the large class's warps give back as its queue runs dry
        const bool fork = split;
        // kernel timing brackets the whole packing phase: both classes, from
        // the fork to the join
        const bool timed = !plain && timing_begin(st);
        if (fork) {
            VS_TRY(cudaEventRecord(sc.ev_fork, st));
            VS_TRY(cudaStreamWaitEvent(sc.side, sc.ev_fork, 0));
        }
        for (int c = 0; c < 3; ++c) {
            const H1Shape& sh = *shapes[c];
            const cudaStream_t cs = (fork && c == kClassSmall) ? sc.side : st;
            if (plain && c == kClassLarge) {
                // the plain path: one single-block launch per instance, in turn
                for (int64_t i = 0; i < in.N; ++i) {
                    H1Params p = h1_params(in, out, prm, sh, lp.counters);
                    p.range_begin = i;
                    p.range_end = i + 1;
                    p.cls = sc.cls;
                    p.want_cls = kClassLarge;
                    p.spill_list = sc.spill_list;
                    p.spill_seg = sc.spill_seg();
                    set_h16(p, lp, sc);
                    VS_TRY(launch_shape(sh, false, p, 1, 1, st));
                }
                continue;
            }
            // (plain path: the rare wide-slot and global-memory instances
            // share one work-stealing launch per class)
            H1Params p = h1_params(in, out, prm, sh, lp.counters);
            p.order = sc.order;
            p.seg = sc.seg();
            p.segment = c;
            p.queue = sc.queue() + c;
            if (c != kClassWide) {
                p.spill_list = sc.spill_list;
                p.spill_seg = sc.spill_seg();
            }
            if (c == kClassLarge) set_h16(p, lp, sc);
            VS_TRY(launch_shape(sh, c == kClassWide, p, sh.groups, sh.grid, cs));
        }
        if (fork) {
            VS_TRY(cudaEventRecord(sc.ev_join, sc.side));
            VS_TRY(cudaStreamWaitEvent(st, sc.ev_join, 0));
        }
        timing_end(timed, st);
        {
            // systems that outgrew their slots, repacked from the start at full
            // size; a system that outgrows that too is listed for global memory
            H1Params p = h1_params(in, out, prm, lp.full, lp.counters);
            p.order = sc.spill_list;
            p.seg = sc.spill_seg();
            p.segment = 0;
            p.queue = sc.queue() + kClasses;
            p.spill_list = sc.spill_list2;
            p.spill_seg = sc.spill_seg() + 2;
            VS_TRY(launch_shape(lp.full, false, p, 1, lp.full.grid, st));
        }
        if (lp.kc.enabled) {
            KCParams kp;
            std::memset(&kp, 0, sizeof(kp));
            kp.in = in;
            kp.out = out;
            kp.criterion = prm.criterion;
            kp.preopen = prm.preopen;
            kp.remark3 = lp.remark3 ? 1 : 0;
            kp.seed = prm.seed;
            kp.order = sc.order;
            kp.seg = sc.seg();
            kp.segment = kClassHuge;
            kp.queue = sc.queue() + kClassHuge;
            kp.slots_all = sc.kc_slots;
            kp.bin_cap = lp.kc.bin_cap;
            kp.max_B1 = lp.kc.max_B1;
            kp.pres_words = lp.kc.pres_words;
            kp.counters = lp.counters;
            if (lp.kd.enabled) {
                // the class in two-CTA clusters; the systems they cannot hold
                // join the list the global-memory kernel packs next
                KDParams dp;
                std::memset(&dp, 0, sizeof(dp));
                dp.in = in;
                dp.out = out;
                dp.criterion = prm.criterion;
                dp.preopen = prm.preopen;
                dp.remark3 = lp.remark3 ? 1 : 0;
                dp.seed = prm.seed;
                dp.order = sc.order;
                dp.seg = sc.seg();
                dp.segment = kClassHuge;
                dp.queue = sc.queue() + kClassHuge;
                dp.spill_list = sc.spill_list2;
                dp.spill_seg = sc.spill_seg() + 2;
                dp.over = sc.kd_over;
                dp.over_bins = lp.kd.over_bins;
                dp.dense = sc.kd_dense;
                dp.max_B1 = lp.kd.max_B1;
                dp.pres = lp.kd.pres;
                dp.segs0 = lp.kd.segs0;
                dp.segs1 = lp.kd.segs1;
                dp.smem = lp.kd.smem;
                dp.counters = lp.counters;
                VS_TRY(kd_launch(dp, lp.kd.clusters, st));
            } else {
                VS_TRY(kc_launch(kp, lp.kc.grid, lp.kc.smem, st));
            }
            // systems that outgrew the worst-case shared-memory shape (or the clusters)
            kp.order = sc.spill_list2;
            kp.seg = sc.spill_seg() + 2;
            kp.segment = 0;
            kp.queue = sc.queue() + kClasses + 1;
            VS_TRY(kc_launch(kp, lp.kc.grid, lp.kc.smem, st));
        }
        return VSBPP_OK;
    }

    // compose mode: sublists of s items
    out.local_types = sc.local_types;
    out.unit_count = sc.unit_count;
    out.unit_total = sc.unit_total;
    pp.out = out;
    pp.classify = 0;
    pp.nu = sc.nu;
    pp.sublist = lp.mode.s;
    pp.cls = nullptr;
    VS_TRY(validate_launch(pp, prep_grid, st));
    VS_TRY(unit_scan_launch(in.N, sc.nu, sc.unit_base, sc.seg_units(), sc.queue(), st));
    ComposeParams cp;
    cp.in = in;
    cp.out = out;
    cp.unit_base = sc.unit_base;
    cp.sublist = lp.mode.s;
    cp.only_instance = -1;
    const int64_t instances = plain ? in.N : 1;
    if (lp.h2x)      // exhaustive search: every best key starts above every key
        VS_TRY(cudaMemsetAsync(sc.h2x_best, 0xFF, sizeof(unsigned long long) * sc.cap_h2x_best, st));
    for (int64_t it = 0; it < instances; ++it) {
        const int64_t only = plain ? it : -1;
        if (lp.mode.heuristic == VSBPP_H2 && lp.h2x) {
            H2XParams xp;
            std::memset(&xp, 0, sizeof(xp));
            xp.in = in;
            xp.out = out;
            xp.units.unit_base = sc.unit_base;
            xp.units.sublist = lp.mode.s;
            xp.criterion = prm.criterion;
            xp.remark3 = lp.remark3 ? 1 : 0;
            xp.sublist = static_cast<int32_t>(lp.mode.s);
            xp.seed = prm.seed;
            xp.seg_units = sc.seg_units();
            xp.best = sc.h2x_best;
            xp.queue = sc.queue();
            xp.counters = lp.counters;
            xp.only_instance = only;
            VS_TRY(cudaMemsetAsync(sc.queue(), 0, sizeof(unsigned long long), st));     // task counter
            const bool timed = !plain && timing_begin(st);
            VS_TRY(h2x_launch(xp, plain ? 1 : lp.h2_grid, st));
            timing_end(timed, st);
        } else if (lp.mode.heuristic == VSBPP_H2) {
            H2Params hp;
            std::memset(&hp, 0, sizeof(hp));
            hp.in = in;
            hp.out = out;
            hp.units.unit_base = sc.unit_base;
            hp.units.sublist = lp.mode.s;
            hp.criterion = prm.criterion;
            hp.preopen = prm.preopen;
            hp.remark3 = lp.remark3 ? 1 : 0;
            hp.seed = prm.seed;
            hp.sublist = static_cast<int32_t>(lp.mode.s);
            hp.max_bins = lp.h2_max_bins;
            hp.only_instance = only;
            hp.counters = lp.counters;
            const bool timed = !plain && timing_begin(st);
            VS_TRY(h2_launch(hp, lp.h2_threads, plain ? 1 : lp.h2_grid, lp.h2_smem, st));
            timing_end(timed, st);
        } else {
            H1Params p = h1_params(in, out, prm, lp.sub, lp.counters);
            p.units.unit_base = sc.unit_base;
            p.units.sublist = lp.mode.s;
            p.compose = 1;
            if (plain) {
                // one launch for this instance's sublists: positions from unit_base
                p.seg = sc.unit_base;
                p.segment = static_cast<int32_t>(it);
                VS_TRY(h1_launch(true, p, lp.sub.G, lp.sub.groups, 1, lp.sub.smem, st));
            } else {
                p.seg = sc.seg_units();
                p.segment = 0;
                p.queue = sc.queue();
                VS_TRY(h1_launch(true, p, lp.sub.G, lp.sub.groups, lp.sub.grid, lp.sub.smem, st));
            }
        }
        cp.only_instance = only;
        VS_TRY(compose_launch(cp, plain ? 1 : prep_grid, st));
    }
    return VSBPP_OK;
}

// The pipeline, with the offline pre-sort around it when asked for: the
// instances' weights are sorted into scratch (caller-order validation kept
// aside), the sorted copy is packed, and each sorted position's bin id goes
// back to the item's original position.
//
// split_ok: the size-class split (small_m) with its second stream pays off
// for batches (batched device calls, plans and their graphs, the host-buffer
// batch call: config 3's BF pass through the host call 3.65 -> 3.40 ms) and
// is measured to cost more than it gains for single-instance calls (the
// serving lanes), which pack their one system in the large class instead.
int enqueue(const LaunchPlan& lp, Scratch& sc, const BatchView& in, const OutView& out,
            const vsbpp_params& prm, bool plain, cudaStream_t st, bool split_ok = true) {
    if (!lp.presort) return enqueue_core(lp, sc, in, out, prm, plain, st, split_ok);
    if (in.N == 0) return VSBPP_OK;
    PresortParams pp;
    std::memset(&pp, 0, sizeof(pp));
    pp.in = in;
    pp.w_sorted = sc.ps_w;
    pp.perm = sc.ps_perm;
    pp.tmp = sc.ps_tmp;
    pp.status0 = sc.ps_stat;
    pp.bin_of_item = out.bin_of_item;
    pp.boi_sorted = sc.ps_boi;
    pp.status = out.status;
    pp.num_bins = out.num_bins;
    pp.total = out.total;
    const int grid = static_cast<int>(std::min<int64_t>(lp.prep_grid, (in.N + kPresortWarps - 1) / kPresortWarps));
    VS_TRY(presort_launch(pp, grid, st));
    BatchView sorted = in;
    sorted.w_all = sc.ps_w;
    OutView out2 = out;
    out2.bin_of_item = sc.ps_boi;
    const int rc = enqueue_core(lp, sc, sorted, out2, prm, plain, st, split_ok);
    if (rc != VSBPP_OK) return rc;
    VS_TRY(unpermute_launch(pp, static_cast<int>(std::min<int64_t>(lp.prep_grid, (in.N + 7) / 8)), st));
    return VSBPP_OK;
}

// Items the per-item scratch must hold when only N and max_m are known on the
// host (the offsets live on the device): N * max_m bounds w_off[N].
int64_t scratch_items(const LaunchPlan& lp, int64_t N, int64_t max_m) {
    const bool per_item = lp.mode.compose || lp.presort || lp.bounded;
    return per_item ? N * std::max<int64_t>(max_m, 1) : 0;
}

int check_instance_args(int64_t m, int32_t n, const void* w, const void* B) {
    if (m < 0 || n < 1 || n > VSBPP_MAX_TYPES) return VSBPP_EINVAL;
    if (!B || (m > 0 && !w)) return VSBPP_EINVAL;
    return VSBPP_OK;
}

int batch_common(int64_t N, const int32_t* w_all, const int64_t* w_off, const int32_t* B_all,
                 const int32_t* B_off, int64_t max_m, const vsbpp_params* p, int32_t* boi,
                 int32_t* bt, int64_t* nb, int64_t* tot, int32_t* status, void* stream, bool plain) {
    try {
        if (N < 0 || max_m < 0) return VSBPP_EINVAL;
        if (N == 0) return VSBPP_OK;
        if (!w_off || !B_all || !B_off || !nb || !tot || !status || !boi || !bt) return VSBPP_EINVAL;
        int rc = check_params(p);
        if (rc) return rc;
        const vsbpp_params prm = defaults(p);
        LaunchPlan lp;
        if ((rc = build_plan(prm, max_m, N, lp, snapshot()))) return rc;
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        Scratch& sc = scratch_for(st);
        std::lock_guard<std::recursive_mutex> lk(*sc.mu);
        // sublist scratch is sized from the host-side bound N * max_m, so the call
        // never has to read the device offsets back
        const int64_t total_m = scratch_items(lp, N, max_m);
        if ((rc = ensure_scratch(sc, lp, N, total_m))) return rc;
        BatchView in{N, w_all, w_off, 0, B_all, B_off, 0};
        OutView out{boi, bt, nb, tot, status, nullptr, nullptr, nullptr};
        return enqueue(lp, sc, in, out, prm, plain, st);
    } catch (...) {
        return VSBPP_ENOMEM;      // no exception crosses the C interface
    }
}

// A recorded batch shape (vsbpp_plan_*).
struct PlanImpl {
    int64_t N = 0, total_m = 0, max_m = 0;
    vsbpp_params prm{};
    LaunchPlan lp;
    Scratch sc;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void* key[10] = {};
    int graphs_recorded = 0;
};

// Times one configuration on a batch: best of `reps` device-timed runs.
int time_config(const vsbpp_config& cfg, int64_t N, const int32_t* w_all, const int64_t* w_off,
                const int32_t* B_all, const int32_t* B_off, int64_t max_m, const vsbpp_params& prm,
                int32_t* boi, int32_t* bt, int64_t* nb, int64_t* tot, int32_t* status,
                cudaStream_t st, int reps, double* ms_out) {
    LaunchPlan lp;
    Snapshot snap = snapshot();
    snap.cfg = cfg;                            // the candidate, not the installed table
    int rc = build_plan(prm, max_m, N, lp, snap);
    if (rc) return rc;
    Scratch& sc = scratch_for(st);
    std::lock_guard<std::recursive_mutex> lk(*sc.mu);
    const int64_t total_m = scratch_items(lp, N, max_m);
    if ((rc = ensure_scratch(sc, lp, N, total_m))) return rc;
    BatchView in{N, w_all, w_off, 0, B_all, B_off, 0};
    OutView out{boi, bt, nb, tot, status, nullptr, nullptr, nullptr};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e30;
    for (int r = 0; r <= reps && rc == VSBPP_OK; ++r) {
        cudaEventRecord(e0, st);
        rc = enqueue(lp, sc, in, out, prm, false, st);
        cudaEventRecord(e1, st);
        if (rc == VSBPP_OK) rc = record(cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0) best = std::min(best, static_cast<double>(ms));   // first run warms up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_out = best;
    return rc;
}

}  // namespace

int vsbpp::check_params_public(const vsbpp_params* p) {
    if (!p) return VSBPP_OK;
    if (p->heuristic != VSBPP_H1 && p->heuristic != VSBPP_H2) return VSBPP_EINVAL;
    if (p->criterion < VSBPP_FF || p->criterion > VSBPP_RANDOM) return VSBPP_EINVAL;
    if (p->preopen != 0 && p->preopen != 1) return VSBPP_EINVAL;
    if (p->flags & ~(VSBPP_REMARK3 | VSBPP_PRESORT)) return VSBPP_EINVAL;
    if (p->sublist_size < 0) return VSBPP_EINVAL;
    if (p->heuristic == VSBPP_H2 && p->sublist_size > VSBPP_H2_MAX_SUBLIST) return VSBPP_EINVAL;
    if (p->max_open < 0) return VSBPP_EINVAL;
    if (p->max_open > 0) {
        // bounded space: first heuristic, without Remark 3
        if (p->heuristic != VSBPP_H1 || (p->flags & VSBPP_REMARK3)) return VSBPP_EINVAL;
        if (p->max_open > VSBPP_MAX_OPEN) return VSBPP_ECAPACITY;
    }
    return VSBPP_OK;
}

unsigned long long* vsbpp::counters_ptr() {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    return g_counters;
}

// ================================================================== C ABI
extern "C" {

const char* vsbpp_strerror(int code) {
    switch (code) {
        case VSBPP_OK: return "ok";
        case VSBPP_EINVAL: return "invalid argument or instance";
        case VSBPP_ETOOBIG: return "an item is heavier than the largest bin capacity";
        case VSBPP_ENOMEM: return "out of memory";
        case VSBPP_ECUDA: return "CUDA error";
        case VSBPP_ETIMEDOUT: return "timed out";
        case VSBPP_EBUSY: return "busy: no slot or memory budget available";
        case VSBPP_ENOTFOUND: return "unknown ticket";
        case VSBPP_ECAPACITY: return "instance exceeds a size limit of this entry point";
        default: return "unknown status code";
    }
}

int vsbpp_version(void) { return VSBPP_VERSION; }

int vsbpp_last_cuda_error(void) { return g_last_cuda.load(); }

int vsbpp_pack_device(const int32_t* w, int64_t m, const int32_t* B, int32_t n, const vsbpp_params* p,
                      int32_t* bin_of_item, int32_t* bin_type, int64_t* num_bins,
                      int64_t* total_capacity, int32_t* status, void* stream) {
    try {
        int rc = check_instance_args(m, n, w, B);
        if (rc) return rc;
        if (!num_bins || !total_capacity || !status || (m > 0 && (!bin_of_item || !bin_type)))
            return VSBPP_EINVAL;
        if ((rc = check_params(p))) return rc;
        const vsbpp_params prm = defaults(p);
        LaunchPlan lp;
        if ((rc = build_plan(prm, std::max<int64_t>(m, 1), 1, lp, snapshot()))) return rc;
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        Scratch& sc = scratch_for(st);
        std::lock_guard<std::recursive_mutex> lk(*sc.mu);
        if ((rc = ensure_scratch(sc, lp, 1, m))) return rc;
        BatchView in{1, w, nullptr, m, B, nullptr, n};
        OutView out{bin_of_item, bin_type, num_bins, total_capacity, status, nullptr, nullptr, nullptr};
        return enqueue(lp, sc, in, out, prm, false, st, false);
    } catch (...) {
        return VSBPP_ENOMEM;      // no exception crosses the C interface
    }
}

int vsbpp_pack(const int32_t* w, int64_t m, const int32_t* B, int32_t n, const vsbpp_params* p,
               int32_t* bin_of_item, int32_t* bin_type, int64_t* num_bins, int64_t* total_capacity) {
    try {
        int rc = check_instance_args(m, n, w, B);
        if (rc) return rc;
        if (!num_bins || !total_capacity || (m > 0 && (!bin_of_item || !bin_type))) return VSBPP_EINVAL;
        if ((rc = check_params(p))) return rc;
        *num_bins = 0;
        *total_capacity = 0;
        HostLease lease;                          // a stream and staging of this device, this call's alone
        HostCtx* hc = lease.c;
        if (!hc) return VSBPP_ECUDA;
        cudaStream_t own = hc->st;
        Scratch& sc = scratch_for(own);
        std::lock_guard<std::recursive_mutex> lk(*sc.mu);
        if ((rc = sc.grow(sc.h_w, sc.cap_h_w, m))) return rc;
        if ((rc = sc.grow(sc.h_B, sc.cap_h_B, n))) return rc;
        if ((rc = sc.grow(sc.h_boi, sc.cap_h_boi, m))) return rc;
        if ((rc = sc.grow(sc.h_bt, sc.cap_h_bt, m))) return rc;
        if ((rc = sc.grow(sc.h_small, sc.cap_h_small, 3))) return rc;
        if ((rc = hc->to_device(sc.h_w, w, sizeof(int32_t) * m))) return rc;
        if ((rc = hc->to_device(sc.h_B, B, sizeof(int32_t) * n))) return rc;
        int32_t* d_status = reinterpret_cast<int32_t*>(sc.h_small + 2);
        rc = vsbpp_pack_device(sc.h_w, m, sc.h_B, n, p, sc.h_boi, sc.h_bt, sc.h_small, sc.h_small + 1,
                               d_status, own);
        if (rc) return rc;
        int64_t small[3] = {0, 0, 0};
        VS_TRY(cudaMemcpyAsync(small, sc.h_small, sizeof(small), cudaMemcpyDeviceToHost, own));
        VS_TRY(cudaStreamSynchronize(own));
        const int32_t st = static_cast<int32_t>(small[2] & 0xFFFFFFFF);
        if (st != VSBPP_OK) return st;
        if (m > 0) {
            if ((rc = hc->to_host(bin_of_item, sc.h_boi, sizeof(int32_t) * m))) return rc;
            if (small[0] > 0 && (rc = hc->to_host(bin_type, sc.h_bt, sizeof(int32_t) * small[0]))) return rc;
            VS_TRY(cudaStreamSynchronize(own));
        }
        *num_bins = small[0];
        *total_capacity = small[1];
        return VSBPP_OK;
    } catch (...) {
        return VSBPP_ENOMEM;      // no exception crosses the C interface
    }
}

int vsbpp_pack_batch_host(int64_t N, const int32_t* w_all, const int64_t* w_off, const int32_t* B_all,
                          const int32_t* B_off, int64_t max_m, const vsbpp_params* p,
                          int32_t* bin_of_item_all, int32_t* bin_type_all, int64_t* num_bins,
                          int64_t* total, int32_t* status) {
    try {
        if (N < 0 || max_m < 0) return VSBPP_EINVAL;
        if (N == 0) return VSBPP_OK;
        if (!w_off || !B_all || !B_off || !num_bins || !total || !status) return VSBPP_EINVAL;
        int rc = check_params(p);
        if (rc) return rc;
        // the CSR offsets are on the host here: check them and take max_m
        if (w_off[0] != 0 || B_off[0] != 0) return VSBPP_EINVAL;
        int64_t mm = 0;
        for (int64_t i = 0; i < N; ++i) {
            const int64_t mi = w_off[i + 1] - w_off[i];
            if (mi < 0 || B_off[i + 1] < B_off[i]) return VSBPP_EINVAL;
            mm = std::max(mm, mi);
        }
        const int64_t total_m = w_off[N];
        const int64_t total_B = B_off[N];
        if (total_m > 0 && (!w_all || !bin_of_item_all || !bin_type_all)) return VSBPP_EINVAL;
        if (max_m == 0) max_m = mm;
        if (mm > max_m) return VSBPP_EINVAL;
        const vsbpp_params prm = defaults(p);
        HostLease lease;                          // a stream and staging of this device, this call's alone
        HostCtx* hc = lease.c;
        if (!hc) return VSBPP_ECUDA;
        cudaStream_t st = hc->st;
        LaunchPlan lp;
        if ((rc = build_plan(prm, max_m, N, lp, snapshot()))) return rc;
        Scratch& sc = scratch_for(st);
        std::lock_guard<std::recursive_mutex> lk(*sc.mu);
        if ((rc = ensure_scratch(sc, lp, N, std::max<int64_t>(total_m, 1)))) return rc;
        if ((rc = sc.grow(sc.h_w, sc.cap_h_w, total_m))) return rc;
        if ((rc = sc.grow(sc.h_B, sc.cap_h_B, total_B))) return rc;
        if ((rc = sc.grow(sc.h_boi, sc.cap_h_boi, total_m))) return rc;
        if ((rc = sc.grow(sc.h_bt, sc.cap_h_bt, total_m))) return rc;
        if ((rc = sc.grow(sc.hb_woff, sc.cap_hb_woff, N + 1))) return rc;
        if ((rc = sc.grow(sc.hb_Boff, sc.cap_hb_Boff, N + 1))) return rc;
        if ((rc = sc.grow(sc.hb_nb, sc.cap_hb_nb, N))) return rc;
        if ((rc = sc.grow(sc.hb_tot, sc.cap_hb_tot, N))) return rc;
        if ((rc = sc.grow(sc.hb_st, sc.cap_hb_st, N))) return rc;
        if ((rc = hc->to_device(sc.h_w, w_all, sizeof(int32_t) * total_m)) ||
            (rc = hc->to_device(sc.hb_woff, w_off, sizeof(int64_t) * (N + 1))) ||
            (rc = hc->to_device(sc.h_B, B_all, sizeof(int32_t) * total_B)) ||
            (rc = hc->to_device(sc.hb_Boff, B_off, sizeof(int32_t) * (N + 1))))
            return rc;
        BatchView in{N, sc.h_w, sc.hb_woff, 0, sc.h_B, sc.hb_Boff, 0};
        OutView out{sc.h_boi, sc.h_bt, sc.hb_nb, sc.hb_tot, sc.hb_st, nullptr, nullptr, nullptr};
        if ((rc = enqueue(lp, sc, in, out, prm, false, st, true))) return rc;
        if ((rc = hc->to_host(bin_of_item_all, sc.h_boi, sizeof(int32_t) * total_m)) ||
            (rc = hc->to_host(bin_type_all, sc.h_bt, sizeof(int32_t) * total_m)) ||
            (rc = hc->to_host(num_bins, sc.hb_nb, sizeof(int64_t) * N)) ||
            (rc = hc->to_host(total, sc.hb_tot, sizeof(int64_t) * N)) ||
            (rc = hc->to_host(status, sc.hb_st, sizeof(int32_t) * N)))
            return rc;
        VS_TRY(cudaStreamSynchronize(st));
        return VSBPP_OK;
    } catch (...) {
        return VSBPP_ENOMEM;      // no exception crosses the C interface
    }
}

int vsbpp_pack_batch(int64_t N, const int32_t* w_all, const int64_t* w_off, const int32_t* B_all,
                     const int32_t* B_off, int64_t max_m, const vsbpp_params* p,
                     int32_t* bin_of_item_all, int32_t* bin_type_all, int64_t* num_bins,
                     int64_t* total, int32_t* status, void* stream) {
    return batch_common(N, w_all, w_off, B_all, B_off, max_m, p, bin_of_item_all, bin_type_all,
                        num_bins, total, status, stream, false);
}

int vsbpp_pack_plain(int64_t N, const int32_t* w_all, const int64_t* w_off, const int32_t* B_all,
                     const int32_t* B_off, int64_t max_m, const vsbpp_params* p,
                     int32_t* bin_of_item_all, int32_t* bin_type_all, int64_t* num_bins,
                     int64_t* total, int32_t* status, void* stream) {
    return batch_common(N, w_all, w_off, B_all, B_off, max_m, p, bin_of_item_all, bin_type_all,
                        num_bins, total, status, stream, true);
}

int vsbpp_shard(int64_t N, const int64_t* w_off, int32_t world, int32_t* rank_of, int64_t* items_of_rank) {
    try {
        if (N < 0 || world < 1 || !w_off || (N > 0 && !rank_of)) return VSBPP_EINVAL;
        for (int64_t i = 0; i < N; ++i)
            if (w_off[i + 1] < w_off[i]) return VSBPP_EINVAL;
        std::vector<int64_t> idx(static_cast<size_t>(N));
        std::iota(idx.begin(), idx.end(), int64_t(0));
        std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) {
            return w_off[a + 1] - w_off[a] > w_off[b + 1] - w_off[b];
        });
        // least-loaded rank first, lowest rank on ties
        using Load = std::pair<int64_t, int32_t>;
        std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
        for (int32_t r = 0; r < world; ++r) heap.push(Load(0, r));
        std::vector<int64_t> load(static_cast<size_t>(world), 0);
        for (int64_t i : idx) {
            Load top = heap.top();
            heap.pop();
            rank_of[i] = top.second;
            top.first += w_off[i + 1] - w_off[i];
            load[static_cast<size_t>(top.second)] = top.first;
            heap.push(top);
        }
        if (items_of_rank)
            for (int32_t r = 0; r < world; ++r) items_of_rank[r] = load[static_cast<size_t>(r)];
        return VSBPP_OK;
    } catch (...) {
        return VSBPP_ENOMEM;      // no exception crosses the C interface
    }
}

int vsbpp_counters_enable(int enable) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (!enable) {
        g_counters = nullptr;      // the buffer is kept for later reads
        return VSBPP_OK;
    }
    static unsigned long long* buf = nullptr;
    if (!buf) {
        void* q = nullptr;
        VS_TRY(cudaMalloc(&q, 2 * sizeof(unsigned long long)));
        VS_TRY(cudaMemset(q, 0, 2 * sizeof(unsigned long long)));
        buf = static_cast<unsigned long long*>(q);
    }
    g_counters = buf;
    return VSBPP_OK;
}

int vsbpp_counters_read(vsbpp_counters* out, int reset) {
    if (!out) return VSBPP_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    out->items = 0;
    out->fit_tests = 0;
    if (!g_counters) return VSBPP_OK;
    unsigned long long v[2] = {0, 0};
    VS_TRY(cudaDeviceSynchronize());
    VS_TRY(cudaMemcpy(v, g_counters, sizeof(v), cudaMemcpyDeviceToHost));
    if (reset) VS_TRY(cudaMemset(g_counters, 0, sizeof(v)));
    out->items = v[0];
    out->fit_tests = v[1];
    return VSBPP_OK;
}

int vsbpp_kernel_timing_enable(int enable) {
    std::lock_guard<std::mutex> lk(g_timing_mu);
    g_timing.on = enable != 0;
    g_timing.count = 0;
    return VSBPP_OK;
}

int vsbpp_kernel_timing_read(float* ms, int32_t max, int32_t* count) {
    try {
        if (!count || max < 0 || (max > 0 && !ms)) return VSBPP_EINVAL;
        std::lock_guard<std::mutex> lk(g_timing_mu);
        *count = 0;
        const int have = g_timing.count;
        const int first = (g_timing.head - have + KernelTiming::kRing) % KernelTiming::kRing;
        for (int x = 0; x < have && x < max; ++x) {
            auto& pr = g_timing.ev[(first + x) % KernelTiming::kRing];
            VS_TRY(cudaEventSynchronize(pr[1]));
            float t = 0.f;
            VS_TRY(cudaEventElapsedTime(&t, pr[0], pr[1]));
            ms[x] = t;
            ++*count;
        }
        g_timing.count = 0;
        return VSBPP_OK;
    } catch (...) {
        return VSBPP_ENOMEM;      // no exception crosses the C interface
    }
}

int vsbpp_get_config(vsbpp_config* out) {
    if (!out) return VSBPP_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    *out = g_cfg;
    return VSBPP_OK;
}

int vsbpp_set_config(const vsbpp_config* cfg) {
    if (!cfg) return VSBPP_EINVAL;
    if (!h1_shape_supported(cfg->large_warps, 1)) return VSBPP_EINVAL;
    if (!h1_shape_supported(1, cfg->small_warps_per_block)) return VSBPP_EINVAL;
    if (cfg->small_m < 0 || cfg->chunk < 32 || cfg->chunk % 32 != 0 || cfg->chunk > 8192)
        return VSBPP_EINVAL;
    if (cfg->slot_pct < 50 || cfg->slot_pct > 200) return VSBPP_EINVAL;
    if (cfg->h2_blocks_per_sm < 0 || cfg->h2_blocks_per_sm > 32) return VSBPP_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    g_cfg = *cfg;
    return VSBPP_OK;
}

int vsbpp_plan_create(int64_t N, int64_t total_m, int64_t max_m, const vsbpp_params* p,
                      vsbpp_plan** out) {
    try {
        if (!out) return VSBPP_EINVAL;
        *out = nullptr;
        if (N < 0 || total_m < 0 || max_m < 0) return VSBPP_EINVAL;
        int rc = check_params(p);
        if (rc) return rc;
        PlanImpl* pl = new (std::nothrow) PlanImpl();
        if (!pl) return VSBPP_ENOMEM;
        pl->N = N;
        pl->total_m = total_m;
        pl->max_m = max_m;
        pl->prm = defaults(p);
        if ((rc = build_plan(pl->prm, max_m, N, pl->lp, snapshot())) ||
            (rc = ensure_scratch(pl->sc, pl->lp, N, std::max<int64_t>(total_m, 1))) ||
            (rc = record(cudaStreamCreateWithFlags(&pl->cap, cudaStreamNonBlocking)))) {
            pl->sc.release();
            delete pl;
            return rc;
        }
        *out = reinterpret_cast<vsbpp_plan*>(pl);
        return VSBPP_OK;
    } catch (...) {
        return VSBPP_ENOMEM;      // no exception crosses the C interface
    }
}

int vsbpp_plan_run(vsbpp_plan* plan, const int32_t* w_all, const int64_t* w_off, const int32_t* B_all,
                   const int32_t* B_off, int32_t* boi, int32_t* bt, int64_t* nb, int64_t* tot,
                   int32_t* status, void* stream) {
    try {
        if (!plan) return VSBPP_EINVAL;
        PlanImpl* pl = reinterpret_cast<PlanImpl*>(plan);
        if (pl->N == 0) return VSBPP_OK;
        if (!w_off || !B_all || !B_off || !boi || !bt || !nb || !tot || !status) return VSBPP_EINVAL;
        std::lock_guard<std::recursive_mutex> lk(*pl->sc.mu);   // one call per plan at a time
        cudaStream_t ust = static_cast<cudaStream_t>(stream);
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        VS_TRY(cudaStreamIsCapturing(ust, &cs));
        if (cs == cudaStreamCaptureStatusActive) {
            // The caller is recording its own graph: put the launches straight into
            // it (everything is pre-allocated, so nothing here allocates).
            BatchView in{pl->N, w_all, w_off, 0, B_all, B_off, 0};
            OutView out{boi, bt, nb, tot, status, nullptr, nullptr, nullptr};
            return enqueue(pl->lp, pl->sc, in, out, pl->prm, false, ust);
        }
        const void* key[10] = {w_all, w_off, B_all, B_off, boi, bt, nb, tot, status, nullptr};
        if (!pl->exec || std::memcmp(key, pl->key, sizeof(key)) != 0) {
            BatchView in{pl->N, w_all, w_off, 0, B_all, B_off, 0};
            OutView out{boi, bt, nb, tot, status, nullptr, nullptr, nullptr};
            cudaGraph_t g = nullptr;
            VS_TRY(cudaStreamBeginCapture(pl->cap, cudaStreamCaptureModeRelaxed));
            const int rc = enqueue(pl->lp, pl->sc, in, out, pl->prm, false, pl->cap);
            const cudaError_t ce = cudaStreamEndCapture(pl->cap, &g);
            if (rc != VSBPP_OK) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            VS_TRY(ce);
            cudaGraphExec_t ex = nullptr;
            const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            VS_TRY(ie);
            if (pl->exec) cudaGraphExecDestroy(pl->exec);
            pl->exec = ex;
            std::memcpy(pl->key, key, sizeof(key));
            ++pl->graphs_recorded;
        }
        VS_TRY(cudaGraphLaunch(pl->exec, ust));
        return VSBPP_OK;
    } catch (...) {
        return VSBPP_ENOMEM;      // no exception crosses the C interface
    }
}

int vsbpp_plan_destroy(vsbpp_plan* plan) {
    if (!plan) return VSBPP_OK;
    PlanImpl* pl = reinterpret_cast<PlanImpl*>(plan);
    { std::lock_guard<std::recursive_mutex> lk(*pl->sc.mu); }    // no call of this plan is running
    cudaDeviceSynchronize();
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->cap) cudaStreamDestroy(pl->cap);
    pl->sc.release();
    delete pl;
    return VSBPP_OK;
}

int vsbpp_autotune(int64_t N, const int32_t* w_all, const int64_t* w_off, const int32_t* B_all,
                   const int32_t* B_off, int64_t max_m, const vsbpp_params* p, int32_t* boi,
                   int32_t* bt, int64_t* nb, int64_t* tot, int32_t* status, void* stream,
                   vsbpp_config* best, double* best_ms) {
    try {
        if (N <= 0 || !w_off || !B_all || !B_off || !boi || !bt || !nb || !tot || !status)
            return VSBPP_EINVAL;
        int rc = check_params(p);
        if (rc) return rc;
        const vsbpp_params prm = defaults(p);
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        std::lock_guard<std::recursive_mutex> lk(*scratch_for(st).mu);
        // Coordinate descent over the knobs, starting from the current table.
        vsbpp_config cur = snapshot().cfg;
        double cur_ms = 0;
        if ((rc = time_config(cur, N, w_all, w_off, B_all, B_off, max_m, prm, boi, bt, nb, tot, status,
                              st, 3, &cur_ms)))
            return rc;
        const int warps[] = {1, 2, 4, 8, 16, 32};
        // the single-warp class's size bound and block size are searched as
        // pairs: its blocks only fit beside the large class's warps when small
        const int smalls[] = {0, 1000, 2000, 4000, 5000, 6000, 7000, 8000};
        const int wpb[] = {1, 2, 4, 16};
        const int chunks[] = {256, 512, 1024, 2048};
        const int pcts[] = {60, 70, 80, 100, 130, 200};
        for (int pass = 0; pass < 2; ++pass) {
            for (int knob = 0; knob < 4; ++knob) {
                const int* vals = knob == 0 ? warps : knob == 2 ? chunks : pcts;
                const int nv = knob == 0 ? 6 : knob == 1 ? 8 * 4 : knob == 2 ? 4 : 6;
                for (int v = 0; v < nv; ++v) {
                    vsbpp_config c = cur;
                    if (knob == 0) c.large_warps = vals[v];
                    if (knob == 1) {
                        c.small_m = smalls[v / 4];
                        c.small_warps_per_block = wpb[v % 4];
                    }
                    if (knob == 2) c.chunk = vals[v];
                    if (knob == 3) c.slot_pct = vals[v];
                    if (std::memcmp(&c, &cur, sizeof(c)) == 0) continue;
                    double ms = 0;
                    const int r2 = time_config(c, N, w_all, w_off, B_all, B_off, max_m, prm, boi, bt, nb,
                                               tot, status, st, 3, &ms);
                    if (r2 == VSBPP_ECAPACITY) continue;   // shape does not fit this batch
                    if (r2) return r2;
                    if (ms < cur_ms) {
                        cur = c;
                        cur_ms = ms;
                    }
                }
            }
        }
        {
            std::lock_guard<std::recursive_mutex> lkg(g_mu);
            g_cfg = cur;
        }
        if (best) *best = cur;
        if (best_ms) *best_ms = cur_ms;
        return VSBPP_OK;
    } catch (...) {
        return VSBPP_ENOMEM;      // no exception crosses the C interface
    }
}

int vsbpp_tune_save(const char* path) {
    if (!path) return VSBPP_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    FILE* f = std::fopen(path, "w");
    if (!f) return VSBPP_EINVAL;
    std::fprintf(f,
                 "{\"large_warps\": %d, \"small_m\": %d, \"small_warps_per_block\": %d, \"chunk\": %d, "
                 "\"slot_pct\": %d, \"h2_blocks_per_sm\": %d}\n",
                 g_cfg.large_warps, g_cfg.small_m, g_cfg.small_warps_per_block, g_cfg.chunk, g_cfg.slot_pct,
                 g_cfg.h2_blocks_per_sm);
    std::fclose(f);
    return VSBPP_OK;
}

int vsbpp_tune_load(const char* path) {
    if (!path) return VSBPP_EINVAL;
    FILE* f = std::fopen(path, "r");
    if (!f) return VSBPP_EINVAL;
    char buf[512] = {0};
    const size_t n = std::fread(buf, 1, sizeof(buf) - 1, f);
    std::fclose(f);
    buf[n] = 0;
    vsbpp_config c = g_cfg;
    const char* names[6] = {"\"large_warps\"", "\"small_m\"", "\"small_warps_per_block\"", "\"chunk\"",
                            "\"slot_pct\"", "\"h2_blocks_per_sm\""};
    int* fields[6] = {&c.large_warps, &c.small_m, &c.small_warps_per_block, &c.chunk, &c.slot_pct,
                      &c.h2_blocks_per_sm};
    for (int k = 0; k < 6; ++k) {
        const char* q = std::strstr(buf, names[k]);
        if (!q && k == 5) continue;            // files written before the field existed
        if (!q) return VSBPP_EINVAL;
        q = std::strchr(q, ':');
        if (!q) return VSBPP_EINVAL;
        *fields[k] = static_cast<int>(std::strtol(q + 1, nullptr, 10));
    }
    return vsbpp_set_config(&c);
}

}  // extern "C"
