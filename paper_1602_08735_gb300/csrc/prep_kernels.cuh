// prep_kernels.cuh -- validation, work ordering and sublist composition.
//
//  validate_kernel   one warp per instance: checks n, B and the items in list
//                    order (Section 6.1 assumptions; first offending item
//                    decides the code), zeroes the instance's counters, and
//                    classifies the instance for the packing kernels
//                    (narrow slots: large / small group; wide slots) with a
//                    log2(m) size bucket.
//  order_kernel      turns the class x bucket histogram into segment bounds
//                    (largest bucket first inside each class) and resets the
//                    work-queue counters.
//  scatter_kernel    writes instance ids into their segment (work order).
//  unit_scan_kernel  prefix sum of sublists per instance (Rule 1 chunks).
//  compose_kernel    concatenates sublist-local results in sublist order
//                    (Section 6.3 step 1: every sublist has its own bins;
//                    Section 6.4: the host accumulates the best results).
#pragma once

#include "prep_params.cuh"

namespace vsbpp {

__device__ __forceinline__ int size_bucket(int64_t m) {
    return m <= 1 ? 0 : 63 - __clzll(static_cast<long long>(m));
}

__global__ void validate_kernel(const PrepParams p) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t i = wid; i < p.in.N; i += nw) {
        const int64_t m = p.in.m(i);
        const int32_t n = p.in.n(i);
        int code = VSBPP_OK;
        if (m < 0 || n < 1 || n > kMaxTypes) code = VSBPP_EINVAL;
        int64_t B1 = 0;
        if (code == VSBPP_OK) {
            const int32_t* B = p.in.B_all + p.in.B_begin(i);
            const int32_t b = lane < n ? B[lane] : 1;
            const int32_t prev = (lane > 0 && lane < n) ? B[lane - 1] : 0x7FFFFFFF;
            const bool bad = lane < n && (b <= 0 || (lane > 0 && prev <= b));
            if (__any_sync(kFull, bad)) code = VSBPP_EINVAL;
            B1 = __shfl_sync(kFull, b, 0);
        }
        if (code == VSBPP_OK) {
            // the first bad weight (in list order) decides the code; eight
            // independent loads per lane per trip keep the loads in flight
            const int32_t* w = p.in.w_all + p.in.w_begin(i);
            unsigned long long first = ~0ull;          // (index << 2) | kind of this lane's first bad weight
            for (int64_t j0 = 0; j0 < m; j0 += 256) {
                int32_t x[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int64_t j = j0 + 32 * u + lane;
                    x[u] = j < m ? __ldg(w + j) : 1;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int64_t j = j0 + 32 * u + lane;
                    const int e = x[u] < 1 ? 1 : (x[u] > B1 ? 2 : 0);
                    const unsigned long long k = (static_cast<unsigned long long>(j) << 2) | static_cast<unsigned>(e);
                    first = (e != 0 && k < first) ? k : first;
                }
            }
            first = warp_min_u64(first);
            if (first != ~0ull) code = (first & 3ull) == 1ull ? VSBPP_EINVAL : VSBPP_ETOOBIG;
        }
        int c = kClassNone;
        if (code == VSBPP_OK && m > 0 && p.classify && p.one_class) {
            c = kClassLarge;
        } else if (code == VSBPP_OK && m > 0 && p.classify) {
            const int64_t bins = 2 * m + (p.preopen ? n : 0);
            if (B1 <= p.narrow_max_B && m <= p.small_m && m <= p.small_cap && bins <= p.narrow_bins) {
                c = kClassSmall;
            } else if (B1 <= p.narrow_max_B && m <= p.narrow_cap && bins <= p.narrow_bins) {
                c = kClassLarge;
            } else if (B1 <= static_cast<int64_t>(kH16MaxB) && m <= p.narrow_cap16) {
                c = kClassLarge;                    // 16-bit slots of the one-warp kernel
            } else if (m <= p.wide_cap) {
                c = kClassWide;
            } else if (m <= p.huge_cap && B1 <= p.huge_max_B1 && bins <= 2 * p.huge_cap + 32) {
                c = kClassHuge;
            } else {
                code = VSBPP_ECAPACITY;
            }
        }
        if (lane == 0) {
            p.out.status[i] = code;
            p.out.num_bins[i] = 0;
            p.out.total[i] = 0;
            if (p.cls) p.cls[i] = c;
            if (c != kClassNone) atomicAdd(&p.hist[c * kBuckets + size_bucket(m)], 1u);
            if (p.nu) p.nu[i] = (code == VSBPP_OK && m > 0) ? (m + p.sublist - 1) / p.sublist : 0;
        }
    }
}

// One warp: histogram -> segment bounds and per-bucket cursors (largest
// bucket first inside each class).  The histogram is cleared for the next
// call; queue counters and the spill segment restart at zero.
__global__ void order_kernel(uint32_t* hist, int64_t* cursor, int64_t* seg,
                             unsigned long long* queue, int64_t* spill_seg) {
    __shared__ uint32_t h[kClasses * kBuckets];
    __shared__ int64_t base[kClasses + 1];
    const int lane = threadIdx.x & 31;
    if (threadIdx.x >= 32 || blockIdx.x != 0) return;
    for (int x = lane; x < kClasses * kBuckets; x += 32) {
        h[x] = hist[x];
        hist[x] = 0;
    }
    __syncwarp();
    // per class: descending-bucket exclusive scan, two buckets per lane
    int64_t run = 0;
    for (int c = 0; c < kClasses; ++c) {
        const int b_hi = kBuckets - 1 - 2 * lane, b_lo = b_hi - 1;    // lane 0: buckets 63, 62
        const uint32_t v_hi = h[c * kBuckets + b_hi], v_lo = h[c * kBuckets + b_lo];
        const uint32_t pair = v_hi + v_lo;
        const uint32_t ex = warp_exclusive_scan(pair, lane);
        cursor[c * kBuckets + b_hi] = run + ex;
        cursor[c * kBuckets + b_lo] = run + ex + v_hi;
        if (lane == 0) base[c] = run;
        run += __shfl_sync(kFull, ex + pair, 31);
    }
    if (lane == 0) {
        for (int c = 0; c < kClasses; ++c) seg[c] = base[c];
        seg[kClasses] = run;
    }
    if (lane <= kClasses + 1) queue[lane] = 0ull;
    if (spill_seg && lane < 4) spill_seg[lane] = 0;
}

__global__ void scatter_kernel(BatchView in, const int32_t* cls, int64_t* cursor, int32_t* order) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < in.N;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int c = cls[i];
        if (c == kClassNone) continue;
        const int64_t pos = static_cast<int64_t>(atomicAdd(
            reinterpret_cast<unsigned long long*>(&cursor[c * kBuckets + size_bucket(in.m(i))]), 1ull));
        order[pos] = static_cast<int32_t>(i);
    }
}

// One block: unit_base[i] = sum of nu[0..i); seg_units = {0, total};
// queue counters restart at zero.
__global__ void unit_scan_kernel(int64_t N, const int64_t* nu, int64_t* unit_base,
                                 int64_t* seg_units, unsigned long long* queue) {
    __shared__ int64_t part[1024];
    const int T = blockDim.x, t = threadIdx.x;
    const int64_t per = (N + T - 1) / T;
    const int64_t a = t * per < N ? t * per : N;
    const int64_t b = (a + per) < N ? (a + per) : N;
    int64_t s = 0;
    for (int64_t i = a; i < b; ++i) s += nu[i];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        int64_t run = 0;
        for (int x = 0; x < T; ++x) {
            const int64_t v = part[x];
            part[x] = run;
            run += v;
        }
        seg_units[0] = 0;
        seg_units[1] = run;
        unit_base[N] = run;
        for (int q = 0; q < 4; ++q) queue[q] = 0ull;
    }
    __syncthreads();
    int64_t run = part[t];
    for (int64_t i = a; i < b; ++i) {
        unit_base[i] = run;
        run += nu[i];
    }
}

// One warp per instance: offsets of each sublist's bins, then the global ids.
__global__ void compose_kernel(const ComposeParams p) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    const int64_t i_first = p.only_instance >= 0 ? p.only_instance : wid;
    const int64_t i_end = p.only_instance >= 0 ? (wid == 0 ? p.only_instance + 1 : 0) : p.in.N;
    const int64_t i_step = p.only_instance >= 0 ? 1 : nw;
    for (int64_t i = i_first; i < i_end; i += i_step) {
        if (p.out.status[i] != VSBPP_OK) continue;
        const int64_t m = p.in.m(i);
        const int64_t wb = p.in.w_begin(i);
        const int64_t ub = p.unit_base[i], ue = p.unit_base[i + 1];
        const int64_t s = p.sublist;
        int64_t off = 0;
        unsigned long long tot = 0;
        for (int64_t u0 = ub; u0 < ue; u0 += 32) {
            const int64_t u = u0 + lane;
            const uint32_t c = u < ue ? static_cast<uint32_t>(p.out.unit_count[u]) : 0u;
            const unsigned long long t = u < ue ? static_cast<unsigned long long>(p.out.unit_total[u]) : 0ull;
            const uint32_t ex = warp_exclusive_scan(c, lane);
            const int64_t my_off = off + ex;
            const int64_t first = (u0 - ub) * s;
            const int64_t last = (first + 32 * s) < m ? (first + 32 * s) : m;
            if (s <= 6) {
                // every load of the chunk is issued before its stores (at most
                // 6 items and 12 bin types per lane)
                int32_t item[6], typ[12];
                int64_t item_off[6];
#pragma unroll
                for (int y = 0; y < 6; ++y) {
                    const int64_t x = first + 32 * y + lane;
                    const bool in = y < s && x < last;
                    const int src = static_cast<int>(in ? (x - first) / s : 0);
                    item_off[y] = __shfl_sync(kFull, my_off, src);
                    item[y] = in ? p.out.bin_of_item[wb + x] : 0;
                }
                const int64_t la = wb + (u - ub) * s;
#pragma unroll
                for (int d = 0; d < 12; ++d) typ[d] = (u < ue && static_cast<uint32_t>(d) < c) ? p.out.local_types[la + d] : 0;
#pragma unroll
                for (int y = 0; y < 6; ++y) {
                    const int64_t x = first + 32 * y + lane;
                    if (y < s && x < last) p.out.bin_of_item[wb + x] = item[y] + static_cast<int32_t>(item_off[y]);
                }
#pragma unroll
                for (int d = 0; d < 12; ++d)
                    if (u < ue && static_cast<uint32_t>(d) < c) p.out.bin_type[wb + my_off + d] = typ[d];
            } else {
                for (int64_t x0 = first; x0 < last; x0 += 32) {
                    const int64_t x = x0 + lane;
                    const int src = static_cast<int>(x < last ? (x - first) / s : 0);
                    const int64_t o = __shfl_sync(kFull, my_off, src);
                    if (x < last) p.out.bin_of_item[wb + x] += static_cast<int32_t>(o);
                }
                if (u < ue) {
                    const int64_t la = wb + (u - ub) * s;
                    for (uint32_t d = 0; d < c; ++d) p.out.bin_type[wb + my_off + d] = p.out.local_types[la + d];
                }
            }
            off += __shfl_sync(kFull, ex + c, 31);
            tot += warp_sum_u64(t);
        }
        if (lane == 0) {
            p.out.num_bins[i] = off;
            p.out.total[i] = static_cast<int64_t>(tot);
        }
    }
}

}  // namespace vsbpp
