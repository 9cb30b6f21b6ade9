// variants_kernels.cuh -- two variants of the first heuristic around the
// method of Section 6.3:
//
//  presort_kernel    offline pre-sort (VSBPP_PRESORT): each instance's items
//                    in non-increasing weight order, equal weights in list
//                    order (the decreasing order of the FFD / BFD heuristics
//                    of Section 5's prior work).  One warp per instance: a
//                    stable LSD radix sort of the key B_1 - w in 8-bit digits
//                    (1 pass when B_1 <= 256, 2 when <= 65536, ...), each
//                    pass a 256-bucket histogram, a warp scan and an
//                    in-order scatter in which lanes holding equal digits
//                    take consecutive places (__match_any_sync + rank).  The
//                    sorted weights go to a scratch copy of the batch that
//                    the usual pipeline packs; the validation status of the
//                    caller's order (first offending item) is kept aside.
//  unpermute_kernel  moves each sorted position's bin id to the item's
//                    original position and restores the caller-order
//                    validation status.
//  bk_pack_kernel    the bounded-space variant (max_open = K <= 32; Section
//                    1: FF / BF / WF keep a given number of bins open, a bin
//                    is closed when completely filled).  One warp per
//                    membrane system; open bin number l (creation order) is
//                    held in lane l's registers (residual, capacity, type,
//                    creation index), so an item's fit test is one compare
//                    per lane and FF / BF / WF one ballot or one warp
//                    reduction; closing bin l shifts lanes l+1.. down by one
//                    (shuffles), creating a bin writes lane `open`.  Every
//                    bin ever created gets a record (type, used) in scratch;
//                    the epilogue turns records into dense ids in creation
//                    order (Section 1's objective over used bins).
#pragma once

#include "variants_params.cuh"

namespace vsbpp {


// Status of the caller's order (Section 6.1 assumptions, first offending item
// decides; the same checks as the validation kernel) and B_1.
__device__ __forceinline__ int presort_validate(const BatchView& in, int64_t i, int lane, uint32_t& B1) {
    const int64_t m = in.m(i);
    const int32_t n = in.n(i);
    B1 = 0;
    if (m < 0 || n < 1 || n > kMaxTypes) return VSBPP_EINVAL;
    const int32_t* B = in.B_all + in.B_begin(i);
    const int32_t b = lane < n ? B[lane] : 1;
    const int32_t prev = (lane > 0 && lane < n) ? B[lane - 1] : 0x7FFFFFFF;
    const bool bad = lane < n && (b <= 0 || (lane > 0 && prev <= b));
    if (__any_sync(kFull, bad)) return VSBPP_EINVAL;
    B1 = static_cast<uint32_t>(__shfl_sync(kFull, b, 0));
    const int32_t* w = in.w_all + in.w_begin(i);
    unsigned long long first = ~0ull;
    for (int64_t j = lane; j < m; j += 32) {
        const int32_t x = __ldg(w + j);
        const int e = x < 1 ? 1 : (static_cast<uint32_t>(x) > B1 ? 2 : 0);
        const unsigned long long key = (static_cast<unsigned long long>(j) << 2) | static_cast<unsigned>(e);
        first = (e != 0 && key < first) ? key : first;
    }
    first = warp_min_u64(first);
    if (first == ~0ull) return VSBPP_OK;
    return (first & 3ull) == 1ull ? VSBPP_EINVAL : VSBPP_ETOOBIG;
}

__global__ void __launch_bounds__(32 * kPresortWarps) presort_kernel(const PresortParams p) {
    __shared__ uint32_t hist_all[kPresortWarps][256];
    const int lane = threadIdx.x & 31;
    const int wl = threadIdx.x >> 5;
    uint32_t* hist = hist_all[wl];
    const unsigned lt = (1u << lane) - 1u;
    const int64_t nw = static_cast<int64_t>(gridDim.x) * kPresortWarps;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kPresortWarps + wl; i < p.in.N; i += nw) {
        uint32_t B1 = 0;
        const int code = presort_validate(p.in, i, lane, B1);
        if (lane == 0) p.status0[i] = code;
        const int64_t m = p.in.m(i);
        if (m <= 0) continue;
        const int64_t a = p.in.w_begin(i);
        const int32_t* w = p.in.w_all + a;
        int32_t* ws = p.w_sorted + a;
        int32_t* perm = p.perm + a;
        if (code != VSBPP_OK) {
            // the pipeline rejects it anyway; keep the list as it stands
            for (int64_t j = lane; j < m; j += 32) {
                ws[j] = w[j];
                perm[j] = static_cast<int32_t>(j);
            }
            continue;
        }
        // key = B_1 - w in [0, B_1 - 1]: ascending key = non-increasing weight
        const uint32_t top = B1 - 1u;
        const int passes = top < 256u ? 1 : top < 65536u ? 2 : top < (1u << 24) ? 3 : 4;
        // pass q reads src (the identity for q = 0) and writes dst; the
        // buffers alternate so that the last pass writes perm
        int32_t* tmp = p.tmp + a;
        for (int q = 0; q < passes; ++q) {
            const int shift = 8 * q;
            const int32_t* src = q == 0 ? nullptr : (((passes - q + 1) & 1) ? perm : tmp);
            int32_t* dst = ((passes - q) & 1) ? perm : tmp;
            for (int x = lane; x < 256; x += 32) hist[x] = 0u;
            __syncwarp();
            for (int64_t j = lane; j < m; j += 32) {
                const int32_t idx = src ? src[j] : static_cast<int32_t>(j);
                const uint32_t key = B1 - static_cast<uint32_t>(__ldg(w + idx));
                atomicAdd(&hist[(key >> shift) & 255u], 1u);
            }
            __syncwarp();
            // exclusive scan of the 256 buckets, 8 per lane
            uint32_t v[8], run = 0;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                v[u] = hist[lane * 8 + u];
                run += v[u];
            }
            uint32_t ex = warp_exclusive_scan(run, lane);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                hist[lane * 8 + u] = ex;        // cursor of bucket lane*8+u
                ex += v[u];
            }
            __syncwarp();
            // in-order scatter: equal digits take consecutive places in lane order
            for (int64_t j0 = 0; j0 < m; j0 += 32) {
                const int64_t j = j0 + lane;
                const bool ok = j < m;
                const int32_t idx = ok ? (src ? src[j] : static_cast<int32_t>(j)) : 0;
                const uint32_t d = ok ? ((B1 - static_cast<uint32_t>(__ldg(w + idx))) >> shift) & 255u
                                      : 256u + static_cast<uint32_t>(lane);
                const unsigned grp = __match_any_sync(kFull, d);
                const int leader = __ffs(grp) - 1;
                uint32_t base = 0;
                if (lane == leader && ok) base = hist[d];
                base = __shfl_sync(kFull, base, leader);
                if (ok) dst[base + __popc(grp & lt)] = idx;
                __syncwarp();
                if (lane == leader && ok) hist[d] = base + __popc(grp);
                __syncwarp();
            }
        }
        __syncwarp();
        for (int64_t j = lane; j < m; j += 32) ws[j] = __ldg(w + perm[j]);
    }
}

__global__ void unpermute_kernel(const PresortParams p) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t i = wid; i < p.in.N; i += nw) {
        const int code = p.status0[i];
        if (code != VSBPP_OK) {
            // the caller's order decides which offending item is reported
            if (lane == 0) {
                p.status[i] = code;
                p.num_bins[i] = 0;
                p.total[i] = 0;
            }
            continue;
        }
        if (p.status[i] != VSBPP_OK) continue;
        const int64_t a = p.in.w_begin(i), m = p.in.m(i);
        for (int64_t j = lane; j < m; j += 32)
            p.bin_of_item[a + p.perm[a + j]] = p.boi_sorted[a + j];
    }
}

// ----------------------------------------------------------- bounded space

struct BKWarp {
    int lane;
    // open bin `lane` (creation order): residual, capacity, type, creation index
    uint32_t res, cap, typ, id;
    uint32_t open;           // open bins
    uint32_t L;              // bins created so far

    // Open bin number x closes: lanes x+1.. move down one place.
    __device__ __forceinline__ void close_at(uint32_t x) {
        const uint32_t r2 = __shfl_down_sync(kFull, res, 1), c2 = __shfl_down_sync(kFull, cap, 1);
        const uint32_t t2 = __shfl_down_sync(kFull, typ, 1), i2 = __shfl_down_sync(kFull, id, 1);
        if (static_cast<uint32_t>(lane) >= x) {
            res = r2;
            cap = c2;
            typ = t2;
            id = i2;
        }
        --open;
    }

    // A new bin of capacity c, type t (empty); the oldest open bin closes
    // first when K are open.  Returns its place in the open list.
    __device__ __forceinline__ uint32_t create(uint32_t c, uint32_t t, uint32_t K, int32_t* rec) {
        if (open == K) close_at(0);
        if (static_cast<uint32_t>(lane) == open) {
            res = c;
            cap = c;
            typ = t;
            id = L;
        }
        if (lane == 0) rec[L] = static_cast<int32_t>(t);
        ++L;
        return open++;
    }
};

__global__ void __launch_bounds__(32 * kBKWarps) bk_pack_kernel(const BKParams p) {
    const int lane = threadIdx.x & 31;
    const int64_t begin = p.seg ? p.seg[p.segment] : p.range_begin;
    const int64_t end = p.seg ? p.seg[p.segment + 1] : p.range_end;
    const uint32_t K = static_cast<uint32_t>(p.max_open);
    const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t it = 0;; ++it) {
        int64_t u = gw + it * nw;
        if (p.queue) {
            unsigned long long v = 0;
            if (lane == 0) v = atomicAdd(p.queue, 1ull);
            u = static_cast<int64_t>(__shfl_sync(kFull, v, 0));
        }
        if (u >= end - begin) break;
        const int64_t i = p.order ? static_cast<int64_t>(p.order[begin + u]) : begin + u;
        if (p.out.status[i] != VSBPP_OK) continue;
        const int64_t m = p.in.m(i);
        const int64_t wb = p.in.w_begin(i);
        const int32_t* w = p.in.w_all + wb;
        const int32_t n = p.in.n(i);
        const int32_t* B = p.in.B_all + p.in.B_begin(i);
        const uint32_t Bl = lane < n ? static_cast<uint32_t>(B[lane]) : 0u;
        int32_t* rec = p.rec + 2 * wb + 32 * i;
        int32_t* raw = p.out.bin_of_item + wb;

        BKWarp S;
        S.lane = lane;
        S.res = S.cap = S.typ = S.id = 0u;
        S.open = 0u;
        S.L = 0u;
        if (p.preopen)                                 // literal Rule 2
            for (int t = 0; t < n; ++t) S.create(static_cast<uint32_t>(B[t]), static_cast<uint32_t>(t), K, rec);
        unsigned long long fit_tests = 0;
        uint32_t bout = 0;
        for (int64_t j0 = 0; j0 < m; j0 += 32) {
            const int64_t jl = j0 + lane;
            // this block's weights and criteria, one item per lane
            const uint32_t wl = jl < m ? static_cast<uint32_t>(__ldg(w + jl)) : 0u;
            const int cl = pick_criterion(p.criterion, p.seed, static_cast<uint64_t>(jl));
            const int cnt = static_cast<int>(min(static_cast<int64_t>(32), m - j0));
            for (int jj = 0; jj < cnt; ++jj) {
                const uint32_t wj = __shfl_sync(kFull, wl, jj);
                const int c = __shfl_sync(kFull, cl, jj);
                fit_tests += S.open;
                // Rule 4 over the open bins (lane order = creation order)
                const bool fit = static_cast<uint32_t>(lane) < S.open && S.res >= wj;
                int sel;
                if (c == kFF) {
                    const unsigned bal = __ballot_sync(kFull, fit);
                    sel = bal ? __ffs(bal) - 1 : -1;
                } else {
                    const uint32_t mine = fit ? (c == kBF ? S.res : ~S.res) : 0xFFFFFFFFu;
                    const uint32_t best = __reduce_min_sync(kFull, mine);
                    const unsigned bal = __ballot_sync(kFull, fit && mine == best);
                    sel = bal ? __ffs(bal) - 1 : -1;
                }
                if (sel < 0) {
                    // nothing fits: a bin of the smallest type holding w
                    const uint32_t t = 31u - static_cast<uint32_t>(__clz(__ballot_sync(kFull, Bl >= wj)));
                    sel = static_cast<int>(S.create(__shfl_sync(kFull, Bl, static_cast<int>(t)), t, K, rec));
                }
                const uint32_t r_old = __shfl_sync(kFull, S.res, sel);
                const uint32_t cp = __shfl_sync(kFull, S.cap, sel);
                const uint32_t ty = __shfl_sync(kFull, S.typ, sel);
                const uint32_t b = __shfl_sync(kFull, S.id, sel);
                const uint32_t r_new = r_old - wj;
                if (lane == sel) S.res = r_new;
                if (lane == 0) rec[b] = static_cast<int32_t>(ty) | kBKUsed;
                if (r_new == 0u) S.close_at(static_cast<uint32_t>(sel));       // completely filled
                if (static_cast<uint64_t>(cp) < 2ull * r_old && 2ull * r_new <= static_cast<uint64_t>(cp))
                    S.create(cp, ty, K, rec);                                   // Rule 5
                bout = lane == jj ? b : bout;
            }
            if (lane < cnt) raw[j0 + lane] = static_cast<int32_t>(bout);
        }
        __syncwarp();
        // objective and dense ids: used bins in creation order
        uint32_t dbase = 0;
        unsigned long long tot = 0;
        for (uint32_t x0 = 0; x0 < S.L; x0 += 32) {
            const uint32_t x = x0 + static_cast<uint32_t>(lane);
            const int32_t r = x < S.L ? rec[x] : 0;
            const bool used = (r & kBKUsed) != 0;
            const unsigned bal = __ballot_sync(kFull, used);
            const uint32_t d = dbase + __popc(bal & ((1u << lane) - 1u));
            if (used) {
                const uint32_t t = static_cast<uint32_t>(r & 0xFF);
                p.out.bin_type[wb + d] = static_cast<int32_t>(t);
                tot += static_cast<unsigned long long>(B[t]);
            }
            if (x < S.L) rec[x] = used ? static_cast<int32_t>(d) : -1;
            dbase += __popc(bal);
        }
        __syncwarp();
        for (int64_t j = lane; j < m; j += 32) raw[j] = rec[raw[j]];
        tot = warp_sum_u64(tot);
        if (lane == 0) {
            p.out.num_bins[i] = dbase;
            p.out.total[i] = static_cast<int64_t>(tot);
            if (p.counters) {
                atomicAdd(p.counters, static_cast<unsigned long long>(m));
                atomicAdd(p.counters + 1, fit_tests);
            }
        }
        __syncwarp();
    }
}

}  // namespace vsbpp
