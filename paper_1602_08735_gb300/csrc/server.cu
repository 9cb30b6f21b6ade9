// server.cu -- continuous batching of packing requests (vsbpp_server_*).
//
// A request is a whole VSBPP instance (host memory).  Submit copies it into a
// pinned staging buffer and queues it.  One worker thread admits queued
// requests in arrival order whenever a slot is free and the request's device
// memory fits in the remaining budget; an admitted request gets its own
// device buffers (stream-ordered allocator) and is packed by the same kernels
// as vsbpp_pack_device on one of several streams ("lanes", the one with the
// fewest items in flight), so requests that arrive while others run are
// packed concurrently with them.  A host callback
// at the end of each request's stream work time-stamps completion and returns
// its slot and memory, which lets the next waiting request in.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Device bytes one request holds while admitted: weights, capacities, two
// int32 result arrays and three 64-bit result words.
size_t request_bytes(int64_t m, int32_t n) {
    return align256(4 * static_cast<size_t>(m)) + align256(4 * static_cast<size_t>(n)) +
           2 * align256(4 * static_cast<size_t>(std::max<int64_t>(m, 1))) + 256;
}

// Pinned host buffers reused across requests, by power-of-two size class.
struct PinnedPool {
    std::mutex mu;
    std::map<size_t, std::vector<void*>> free_;

    static size_t cls(size_t bytes) {
        size_t c = 4096;
        while (c < bytes) c <<= 1;
        return c;
    }
    void* get(size_t bytes) {
        const size_t c = cls(bytes);
        {
            std::lock_guard<std::mutex> lk(mu);
            auto& v = free_[c];
            if (!v.empty()) {
                void* p = v.back();
                v.pop_back();
                return p;
            }
        }
        void* p = nullptr;
        if (cudaMallocHost(&p, c) != cudaSuccess) return nullptr;
        return p;
    }
    void put(void* p, size_t bytes) {
        if (!p) return;
        std::lock_guard<std::mutex> lk(mu);
        free_[cls(bytes)].push_back(p);
    }
    void release() {
        std::lock_guard<std::mutex> lk(mu);
        for (auto& kv : free_)
            for (void* p : kv.second) cudaFreeHost(p);
        free_.clear();
    }
};

struct Req;

}  // namespace

struct vsbpp_server {
    size_t budget = 0;
    int max_slots = 1, nlanes = 1, max_queued = 1;
    int device = 0;
    std::vector<cudaStream_t> lanes;
    // Request buffers: freed memory is kept (release threshold = budget) and
    // reused by another lane only once its free has completed, never by making
    // that lane wait on the freeing one.
    cudaMemPool_t pool = nullptr;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req*> waiting;
    std::unordered_map<uint64_t, Req*> tickets;
    size_t in_use = 0;
    int in_flight = 0;
    std::vector<int64_t> lane_items;   // items in flight per lane
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    PinnedPool pinned;
    std::vector<double> lat_us, wait_us, svc_us;    // submit->done, submit->admit, admit->done
    int64_t completed = 0, items = 0;
    Clock::time_point t_first{}, t_last{};
    bool any = false;
};

namespace {

struct Req {
    vsbpp_server* srv = nullptr;
    uint64_t ticket = 0;
    int64_t m = 0;
    int32_t n = 0;
    vsbpp_params prm{};
    size_t need = 0;
    size_t in_bytes = 0, out_bytes = 0;
    int32_t* h_in = nullptr;     // pinned: w[m], B[n]
    int32_t* h_out = nullptr;    // pinned: bin_of_item[m], bin_type[m], 3 x int64
    void* d_buf = nullptr;
    int status = VSBPP_OK;
    int lane = 0;
    bool done = false;
    Clock::time_point t_submit, t_admit, t_done;

    int64_t* h_small() const {
        return reinterpret_cast<int64_t*>(reinterpret_cast<char*>(h_out) +
                                          align256(8 * static_cast<size_t>(std::max<int64_t>(m, 1))));
    }
};

void finish(Req* r, int status) {
    vsbpp_server* s = r->srv;
    const Clock::time_point now = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    r->t_done = now;
    if (status != VSBPP_OK) r->status = status;
    r->done = true;
    s->in_flight -= 1;
    s->in_use -= r->need;
    s->lane_items[r->lane] -= std::max<int64_t>(r->m, 1);
    s->completed += 1;
    s->items += r->m;
    s->t_last = now;
    auto keep = [](std::vector<double>& v, double x) {
        if (v.size() >= 200000) v.erase(v.begin(), v.begin() + 100000);
        v.push_back(x);
    };
    keep(s->lat_us, std::chrono::duration<double, std::micro>(now - r->t_submit).count());
    keep(s->wait_us, std::chrono::duration<double, std::micro>(r->t_admit - r->t_submit).count());
    keep(s->svc_us, std::chrono::duration<double, std::micro>(now - r->t_admit).count());
    s->cv.notify_all();
}

void CUDART_CB on_done(void* arg) { finish(static_cast<Req*>(arg), VSBPP_OK); }

// Enqueue one admitted request on its lane (worker thread, no server lock held).
int launch(Req* r, cudaStream_t st) {
    const int64_t m = r->m;
    const int32_t n = r->n;
    const size_t ow = align256(4 * static_cast<size_t>(m));
    const size_t oB = align256(4 * static_cast<size_t>(n));
    const size_t om = align256(4 * static_cast<size_t>(std::max<int64_t>(m, 1)));
    cudaError_t e = cudaMallocFromPoolAsync(&r->d_buf, r->need, r->srv->pool, st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? VSBPP_ENOMEM : VSBPP_ECUDA;
    char* d = static_cast<char*>(r->d_buf);
    int32_t* d_w = reinterpret_cast<int32_t*>(d);
    int32_t* d_B = reinterpret_cast<int32_t*>(d + ow);
    int32_t* d_boi = reinterpret_cast<int32_t*>(d + ow + oB);
    int32_t* d_bt = reinterpret_cast<int32_t*>(d + ow + oB + om);
    int64_t* d_small = reinterpret_cast<int64_t*>(d + ow + oB + 2 * om);
    if (m > 0) e = cudaMemcpyAsync(d_w, r->h_in, 4 * static_cast<size_t>(m), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_B, r->h_in + m, 4 * static_cast<size_t>(n), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_small, 0, 3 * sizeof(int64_t), st);
    if (e != cudaSuccess) {
        cudaFreeAsync(r->d_buf, st);
        return VSBPP_ECUDA;
    }
    int rc = vsbpp_pack_device(d_w, m, d_B, n, &r->prm, d_boi, d_bt, d_small, d_small + 1,
                               reinterpret_cast<int32_t*>(d_small + 2), st);
    if (rc == VSBPP_OK) {
        int32_t* h_boi = r->h_out;
        int32_t* h_bt = r->h_out + std::max<int64_t>(m, 1);
        if (m > 0) {
            e = cudaMemcpyAsync(h_boi, d_boi, 4 * static_cast<size_t>(m), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h_bt, d_bt, 4 * static_cast<size_t>(m), cudaMemcpyDeviceToHost, st);
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(r->h_small(), d_small, 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = VSBPP_ECUDA;
    }
    cudaFreeAsync(r->d_buf, st);
    if (rc != VSBPP_OK) return rc;
    e = cudaLaunchHostFunc(st, on_done, r);
    return e == cudaSuccess ? VSBPP_OK : VSBPP_ECUDA;
}

void worker_main(vsbpp_server* s) {
    cudaSetDevice(s->device);
    for (;;) {
        Req* r = nullptr;
        cudaStream_t st = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] {
                if (s->stop) return true;
                if (s->waiting.empty() || s->in_flight >= s->max_slots) return false;
                return s->in_use + s->waiting.front()->need <= s->budget;
            });
            if (s->stop) return;
            r = s->waiting.front();
            s->waiting.pop_front();
            r->t_admit = Clock::now();
            s->in_flight += 1;
            s->in_use += r->need;
            // the lane with the fewest items in flight
            int best = 0;
            for (int l = 1; l < s->nlanes; ++l)
                if (s->lane_items[l] < s->lane_items[best]) best = l;
            r->lane = best;
            s->lane_items[best] += std::max<int64_t>(r->m, 1);
            st = s->lanes[best];
            if (!s->any) {
                s->any = true;
                s->t_first = Clock::now();
            }
        }
        const int rc = launch(r, st);
        if (rc != VSBPP_OK) finish(r, rc);
    }
}

void release_req(vsbpp_server* s, Req* r) {
    s->pinned.put(r->h_in, r->in_bytes);
    s->pinned.put(r->h_out, r->out_bytes);
    delete r;
}

}  // namespace

extern "C" {

int vsbpp_server_create(size_t device_mem_budget, int32_t max_slots, int32_t lanes, int32_t max_queued,
                        vsbpp_server** out) {
    try {
        if (!out) return VSBPP_EINVAL;
        *out = nullptr;
        if (device_mem_budget == 0 || max_slots < 1 || lanes < 1 || lanes > 64 || max_queued < 1)
            return VSBPP_EINVAL;
        vsbpp_server* s = new (std::nothrow) vsbpp_server();
        if (!s) return VSBPP_ENOMEM;
        s->budget = device_mem_budget;
        s->max_slots = max_slots;
        s->nlanes = lanes;
        s->max_queued = max_queued;
        cudaGetDevice(&s->device);
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = s->device;
        if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) {
            delete s;
            return VSBPP_ECUDA;
        }
        uint64_t keep = device_mem_budget;
        int no = 0;
        cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        cudaMemPoolSetAttribute(s->pool, cudaMemPoolReuseAllowInternalDependencies, &no);
        for (int i = 0; i < lanes; ++i) {
            cudaStream_t st = nullptr;
            if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
                for (cudaStream_t x : s->lanes) cudaStreamDestroy(x);
                cudaMemPoolDestroy(s->pool);
                delete s;
                return VSBPP_ECUDA;
            }
            s->lanes.push_back(st);
        }
        s->lane_items.assign(static_cast<size_t>(lanes), 0);
        s->worker = std::thread(worker_main, s);
        *out = s;
        return VSBPP_OK;
    } catch (...) {
        return VSBPP_ENOMEM;      // no exception crosses the C interface
    }
}

int vsbpp_server_submit(vsbpp_server* s, const int32_t* w, int64_t m, const int32_t* B, int32_t n,
                        const vsbpp_params* p, uint64_t* ticket) {
    try {
        if (!s || !ticket || !B || m < 0 || (m > 0 && !w) || n < 1 || n > VSBPP_MAX_TYPES)
            return VSBPP_EINVAL;
        const int prc = vsbpp::check_params_public(p);
        if (prc != VSBPP_OK) return prc;
        const size_t need = request_bytes(m, n);
        if (need > s->budget) return VSBPP_ECAPACITY;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (static_cast<int>(s->waiting.size()) >= s->max_queued) return VSBPP_EBUSY;
        }
        Req* r = new (std::nothrow) Req();
        if (!r) return VSBPP_ENOMEM;
        r->srv = s;
        r->m = m;
        r->n = n;
        std::memset(&r->prm, 0, sizeof(r->prm));
        r->prm.heuristic = VSBPP_H1;
        r->prm.criterion = VSBPP_BF;
        if (p) r->prm = *p;
        r->need = need;
        r->in_bytes = 4 * (static_cast<size_t>(m) + static_cast<size_t>(n));
        r->out_bytes = align256(8 * static_cast<size_t>(std::max<int64_t>(m, 1))) + 64;
        r->h_in = static_cast<int32_t*>(s->pinned.get(r->in_bytes));
        r->h_out = static_cast<int32_t*>(s->pinned.get(r->out_bytes));
        if (!r->h_in || !r->h_out) {
            release_req(s, r);
            return VSBPP_ENOMEM;
        }
        if (m > 0) std::memcpy(r->h_in, w, 4 * static_cast<size_t>(m));
        std::memcpy(r->h_in + m, B, 4 * static_cast<size_t>(n));
        std::lock_guard<std::mutex> lk(s->mu);
        if (static_cast<int>(s->waiting.size()) >= s->max_queued) {
            release_req(s, r);
            return VSBPP_EBUSY;
        }
        r->ticket = s->next_ticket++;
        r->t_submit = Clock::now();
        s->tickets[r->ticket] = r;
        s->waiting.push_back(r);
        s->cv.notify_all();
        *ticket = r->ticket;
        return VSBPP_OK;
    } catch (...) {
        return VSBPP_ENOMEM;      // no exception crosses the C interface
    }
}

int vsbpp_server_poll(vsbpp_server* s, uint64_t ticket, int32_t* bin_of_item, int32_t* bin_type,
                      int64_t* num_bins, int64_t* total_capacity, int64_t timeout_us) {
    try {
        if (!s) return VSBPP_EINVAL;
        std::unique_lock<std::mutex> lk(s->mu);
        auto it = s->tickets.find(ticket);
        if (it == s->tickets.end()) return VSBPP_ENOTFOUND;
        Req* r = it->second;
        if (!r->done) {
            if (timeout_us == 0) return VSBPP_ETIMEDOUT;
            if (timeout_us < 0) {
                s->cv.wait(lk, [&] { return r->done; });
            } else if (!s->cv.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return r->done; })) {
                return VSBPP_ETIMEDOUT;
            }
        }
        s->tickets.erase(it);
        lk.unlock();
        int rc = r->status;
        if (rc == VSBPP_OK) {
            const int64_t* sm = r->h_small();
            rc = static_cast<int32_t>(static_cast<uint32_t>(sm[2] & 0xFFFFFFFF));
            if (rc == VSBPP_OK) {
                if ((r->m > 0 && (!bin_of_item || !bin_type)) || !num_bins || !total_capacity) {
                    rc = VSBPP_EINVAL;
                } else {
                    if (r->m > 0) {
                        std::memcpy(bin_of_item, r->h_out, 4 * static_cast<size_t>(r->m));
                        std::memcpy(bin_type, r->h_out + std::max<int64_t>(r->m, 1), 4 * static_cast<size_t>(sm[0]));
                    }
                    *num_bins = sm[0];
                    *total_capacity = sm[1];
                }
            }
        }
        release_req(s, r);
        return rc;
    } catch (...) {
        return VSBPP_ENOMEM;      // no exception crosses the C interface
    }
}

int vsbpp_server_stats(vsbpp_server* s, vsbpp_server_stats_t* out) {
    try {
        if (!s || !out) return VSBPP_EINVAL;
        std::vector<double> v, wv, sv;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            v = s->lat_us;
            wv = s->wait_us;
            sv = s->svc_us;
            out->completed = s->completed;
            out->items_packed = s->items;
            out->busy_s = s->any ? std::chrono::duration<double>(s->t_last - s->t_first).count() : 0.0;
        }
        // nearest-rank percentile of a sorted copy (0 when empty)
        auto q = [](std::vector<double>& x, double f) {
            if (x.empty()) return 0.0;
            const size_t k = static_cast<size_t>(f * static_cast<double>(x.size() - 1) + 0.5);
            return x[std::min(k, x.size() - 1)];
        };
        std::sort(v.begin(), v.end());
        std::sort(wv.begin(), wv.end());
        std::sort(sv.begin(), sv.end());
        out->p50_us = q(v, 0.50);
        out->p99_us = q(v, 0.99);
        out->max_us = v.empty() ? 0.0 : v.back();
        out->wait_p50_us = q(wv, 0.50);
        out->wait_p99_us = q(wv, 0.99);
        out->service_p50_us = q(sv, 0.50);
        out->service_p99_us = q(sv, 0.99);
        return VSBPP_OK;
    } catch (...) {
        return VSBPP_ENOMEM;      // no exception crosses the C interface
    }
}

int vsbpp_server_destroy(vsbpp_server* s) {
    if (!s) return VSBPP_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    for (cudaStream_t st : s->lanes) cudaStreamSynchronize(st);
    for (cudaStream_t st : s->lanes) cudaStreamDestroy(st);
    cudaMemPoolDestroy(s->pool);
    for (auto& kv : s->tickets) release_req(s, kv.second);
    s->tickets.clear();
    s->pinned.release();
    delete s;
    return VSBPP_OK;
}

}  // extern "C"
