// h1w_kernel.cuh -- the first heuristic of Section 6.3, one warp per membrane
// system, for systems of at most 32768 bins with B_1 <= 32767, or of at most
// 65536 bins with B_1 <= 255 (16-bit slots, run16 below).
//
// Same method as h1_kernel.cuh (Rules 2-6: items in list order, fit test
// residual >= w, FF / BF / WF with the lowest creation index winning ties,
// the smallest type holding the item when nothing fits, the Rule 5 division
// when a bin's load first reaches half its capacity), with the per-item work
// arranged so that its dependent chain is as short as one warp can make it:
//
//   slot    one 32-bit word per bin, (residual << 16) | capacity, or
//           (residual << 10) | capacity when B_1 <= 1023.  The bin's index is
//           its position, so a lane knows the index of every slot it reads,
//           and its capacity (hence its type and its Rule 5 threshold)
//           travels with the residual: no second lookup per item.  In the
//           10-bit form a key (index << 20) | slot carries index, residual
//           and capacity at once.
//   segmax  the largest residual of each 128-bin segment, kept in registers:
//           lane l holds segments l, l+32, ... (NS per lane).  FF finds its
//           segment with one warp minimum over (segment, max) keys, WF with
//           one warp maximum over (max, segment) keys.
//   index   (BF, B_1 <= 1023) row[r] = bitmap of the segments holding a bin
//           of residual r (NS words), and the bitmap of residuals present
//           (32 words, word l in lane l's register).  BF takes the least
//           residual >= w present (one warp minimum), then the first segment
//           in its row.  Both bitmaps run from the top bit down (residual or
//           segment 32q + x is bit 31 - x of word q), so one count of leading
//           zeros finds the least member of a word.
//
// Within the chosen segment each lane reads one 16-byte quad; one warp
// minimum over (index, residual or capacity) keys names the bin, and the
// segment's new maximum comes from the same read (count of bins at the old
// maximum and the largest other residual, reduced alongside; for FF one
// maximum over the quad with the chosen slot updated).  Every lane
// makes every shared-memory store of an item with the same value (predicated
// where a store may not apply), so each lane reads back only what it stored
// itself and the item needs no barrier; the spread index rows of the larger
// shapes (one writer lane, other reader lanes) take one __syncwarp() per
// item.  Item weights are read from
// global memory a 32-item block ahead, each lane holding one item's weight
// together with the capacity of the smallest type that holds it.
#pragma once

#include "h1_kernel.cuh"

namespace vsbpp {

constexpr int kWarpMaxSlots = 32768;      // 8 segment words per lane at most
constexpr int kNS16 = 12;                  // 16-bit slots: segment words per lane
constexpr uint32_t kH16Slots = 32u * kNS16 * 256u;   // 98304 bins

// Segment words per lane for a system of slot_cap bins (0: too large).
__host__ __device__ inline int h1w_ns(int slot_cap) {
    return slot_cap <= 4096 ? 1 : slot_cap <= 8192 ? 2 : slot_cap <= 16384 ? 4
         : slot_cap <= kWarpMaxSlots ? 8 : 0;
}

// Shared memory of one warp: slots, a 16-byte pad (the write target of the
// 16-bit form's bin that does not divide), the BF rows (1024 residuals x NS words) and a
// 16-byte pad (the target of index writes that do not apply) when laid out,
// capacities.
__host__ __device__ inline int h1w_group_bytes(int slot_cap, int bf_index) {
    const int ns = h1w_ns(slot_cap);
    return 4 * slot_cap + 16 + (bf_index ? 4 * (kIndexMaxRes + 1) * ns + 16 : 0) + 4 * kMaxTypes;
}

// Shared memory of the 16-bit slot layout (one warp): slots, a 16-byte pad,
// the BF rows (256 residuals x kNS16 words) and a pad when laid out,
// capacities.
__host__ __device__ inline int h1w16_group_bytes(int bf_index) {
    return 2 * static_cast<int>(kH16Slots) + 16 + (bf_index ? 4 * (kH16MaxB + 1) * kNS16 + 16 : 0) +
           4 * kMaxTypes;
}

template <int NS, int CRIT>
struct H1Warp {
    static constexpr bool kSeg = CRIT != kBF;                      // FF or WF items occur
    static constexpr bool kBFItems = CRIT == kBF || CRIT == kRandom;
    static constexpr uint32_t kNoKey = 0xFFFFFFFFu;
    static constexpr uint32_t kRowsPad = (kIndexMaxRes + 1) * NS;   // index word past the rows
    static constexpr bool kLaneRows = NS >= 4;      // index row words spread over the lanes

    uint32_t* slots;
    uint32_t* rows;      // BF index rows (null when not laid out)
    uint32_t* Bs;        // capacities, descending
    int lane;

    // Item weight j (0 past the end of the list).
    __device__ __forceinline__ uint32_t weight(const int32_t* w, int64_t j, int64_t k) const {
        return j < k ? static_cast<uint32_t>(__ldg(w + j)) : 0u;
    }

    // Item descriptor of weight x (item j): x | capacity of the smallest type
    // holding it << 16, criterion bits at 15 and 31 (RANDOM).  0 for x = 0.
    __device__ __forceinline__ uint32_t descriptor(uint32_t x, int64_t j, int n, uint64_t seed,
                                                   int64_t key0) const {
        if (x == 0u) return 0u;
        uint32_t bn = 0;
        for (int t = 0; t < n; ++t) {
            const uint32_t c = Bs[t];
            bn = c >= x ? c : bn;
        }
        uint32_t d = x | (bn << 16);
        if (CRIT == kRandom) {
            const uint32_t c = static_cast<uint32_t>(pick_criterion(kRandom, seed, static_cast<uint64_t>(key0 + j)));
            d |= ((c & 1u) << 15) | ((c >> 1) << 31);
        }
        return d;
    }

    // This lane's part of "residual >= x" in the present-residual bitmap
    // (residual 32 * lane + y at bit 31 - y).
    __device__ __forceinline__ uint32_t present_mask(uint32_t x) const {
        const uint32_t xi = x >> 5, ul = static_cast<uint32_t>(lane);
        return ul < xi ? 0u : ul == xi ? (0xFFFFFFFFu >> (x & 31)) : 0xFFFFFFFFu;
    }

    // Type of a capacity (capacities are distinct and descending).
    __device__ __forceinline__ uint32_t type_of(uint32_t cap, int n) const {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (Bs[mid] > cap) lo = mid + 1; else hi = mid;
        }
        return static_cast<uint32_t>(lo);
    }

    // BF without the index (B_1 > 1023): the full scan over the live segments.
    // key = (r - w) << 15 | index; returns kNoKey when nothing fits.
    template <int kR>
    __device__ __forceinline__ uint32_t bf_scan(uint32_t wj, uint32_t L) const {
        uint32_t key = kNoKey;
        const uint32_t nseg = (L + 127u) >> 7;
        for (uint32_t s = 0; s < nseg; ++s) {
            const uint4 Q = reinterpret_cast<const uint4*>(slots)[32u * s + static_cast<uint32_t>(lane)];
            const uint32_t base = 128u * s + 4u * static_cast<uint32_t>(lane);
            const uint32_t r0 = Q.x >> kR, r1 = Q.y >> kR, r2 = Q.z >> kR, r3 = Q.w >> kR;
            if (r3 >= wj) key = min(key, ((r3 - wj) << 15) | (base + 3u));
            if (r2 >= wj) key = min(key, ((r2 - wj) << 15) | (base + 2u));
            if (r1 >= wj) key = min(key, ((r1 - wj) << 15) | (base + 1u));
            if (r0 >= wj) key = min(key, ((r0 - wj) << 15) | base);
        }
        return __reduce_min_sync(kFull, key);
    }

    // Pack items [0, k) of one system.  Returns false when the system would
    // outgrow slot_cap bins (spill).  IDX: BF items use the residual index
    // (B_1 <= 1023), else the full scan.  The item step is straight-line code:
    // the chosen segment's quad is read whether or not a bin fits, and the
    // fitting / new-bin cases are merged by selects.
    template <bool IDX, bool W10, bool R3>
    __device__ __forceinline__ bool run(const H1Params& p, int64_t i, const int32_t* w, int64_t key0,
                                        uint32_t k, int32_t* raw, int n, uint32_t& L_io,
                                        unsigned long long& fit_tests) const {
        constexpr int kR = W10 ? 10 : 16;                 // residual shift in a slot
        constexpr uint32_t kCap = W10 ? 0x3FFu : 0xFFFFu;   // capacity field
        uint32_t L = L_io;
        const uint32_t cap_bins = static_cast<uint32_t>(p.slot_cap);
        const uint32_t ulane = static_cast<uint32_t>(lane);
        // R3 (Remark 3's reading of Rule 5): lane t counts the type-t bins
        // below half their capacity (a pre-opened bin is empty)
        const uint32_t Bl = R3 ? Bs[ulane] : 0u;
        uint32_t below = (R3 && L > 0 && ulane < static_cast<uint32_t>(n)) ? 1u : 0u;

        uint32_t sm[NS];                 // segment maxima, segment 32q + lane
        uint32_t wb = 0;                 // residuals 32*lane .. 32*lane+31 present, top bit first
#pragma unroll
        for (int q = 0; q < NS; ++q) sm[q] = 0;
        // start state (preopened bins: all in segment 0)
        if (kSeg && L > 0 && lane == 0) sm[0] = Bs[0];
        if (IDX) {
            for (uint32_t t = 0; t < L; ++t) {
                const uint32_t r = Bs[t];
                if ((r >> 5) == ulane) wb |= 0x80000000u >> (r & 31);
            }
        }

        // The index entry of a divided-off bin is written during the next
        // item (its row word read at that item's start, stored before the
        // item reads any row), so the read-modify-write is off the chain.
        uint32_t pend_at = kRowsPad, pend_bit = 0;
        // Items go in blocks of 32: lane l holds the descriptor of item
        // (block + l), and the weights of the next block are loaded a block
        // ahead.
        uint32_t dnext = descriptor(weight(w, ulane, k), ulane, n, p.seed, key0);
        uint32_t wpre = weight(w, 32 + ulane, k);
        for (uint32_t j0 = 0; j0 < k; j0 += 32u) {
            const uint32_t cnt = min(32u, k - j0);
            // an item adds at most two bins: stop before the block could
            // outgrow the slots (a larger shape, or global memory, repacks the
            // system from the start); after 2048 items also stop when the
            // bins so far, extrapolated to all k items, pass 9/8 of the slots
            const bool trend = !p.no_trend && j0 >= 2048u &&
                               static_cast<uint64_t>(L) * k >
                                   static_cast<uint64_t>(cap_bins) * j0 + ((static_cast<uint64_t>(cap_bins) * j0) >> 3);
            if (p.spill_list && (L + 2u * cnt > cap_bins || trend)) {
                if (lane == 0) {
                    const unsigned long long pos = atomicAdd(
                        reinterpret_cast<unsigned long long*>(p.spill_seg + 1), 1ull);
                    p.spill_list[pos] = static_cast<int32_t>(i);
                }
                __syncwarp();
                return false;
            }
            const uint32_t dblk = dnext;
            dnext = descriptor(wpre, static_cast<int64_t>(j0) + 32 + ulane, n, p.seed, key0);
            wpre = weight(w, static_cast<int64_t>(j0) + 64 + ulane, k);
            uint32_t d = __shfl_sync(kFull, dblk, 0);
            uint32_t msk = IDX ? present_mask(d & 0x7FFFu) : 0u;
            uint32_t bout = 0, fit_blk = 0;          // fit tests of the block (< 2^20)
        for (uint32_t jj = 0; jj < cnt; ++jj) {
            // the next item's descriptor and present-residual mask
            // (independent of the packing state, off the item's chain)
            const uint32_t dn = __shfl_sync(kFull, dblk, static_cast<int>((jj + 1u) & 31u));
            const uint32_t mskn = IDX ? present_mask(dn & 0x7FFFu) : 0u;
            const uint32_t wj = d & 0x7FFFu;
            const uint32_t Bn = (d >> 16) & 0x7FFFu;
            const int c = CRIT == kRandom ? static_cast<int>(((d >> 15) & 1u) | ((d >> 30) & 2u)) : CRIT;
            fit_blk += L;
            uint32_t pend_word = 0;
            if (IDX) pend_word = rows[pend_at];

            // 1. the segment holding the answer: sf; Mseg = its largest
            //    residual; R = the residual sought (BF, WF)
            bool hit;
            uint32_t sf = 0, Mseg = 0, R = 0;
            // index rows of r_old and of r_new: all NS words in every lane
            // (NS < 4), or word `lane` in lane `lane` (kLaneRows)
            uint32_t rw[kLaneRows ? 1 : NS], rn[kLaneRows ? 1 : NS];
#pragma unroll
            for (int q = 0; q < (kLaneRows ? 1 : NS); ++q) rw[q] = rn[q] = 0;
            if (kSeg && c == kFF) {
                uint32_t key = kNoKey;
#pragma unroll
                for (int q = NS - 1; q >= 0; --q)
                    key = sm[q] >= wj ? ((32u * q + ulane) << 16) | sm[q] : key;
                key = __reduce_min_sync(kFull, key);
                hit = key != kNoKey;
                sf = hit ? key >> 16 : 0u;
                Mseg = key & 0xFFFFu;
            } else if (kSeg && c == kWF) {
                uint32_t key = 0;
#pragma unroll
                for (int q = 0; q < NS; ++q) key = max(key, (sm[q] << 8) | (255u - (32u * q + ulane)));
                key = __reduce_max_sync(kFull, key);
                Mseg = key >> 8;
                sf = 255u - (key & 255u);
                hit = Mseg >= wj;
                R = Mseg;
            } else if (IDX) {
                // residuals >= w present in this lane's word: the least is the
                // highest bit left
                const uint32_t x = wb & msk;
                uint32_t key = x ? 32u * ulane + static_cast<uint32_t>(__clz(x)) : kNoKey;
                key = __reduce_min_sync(kFull, key);
                hit = key != kNoKey;
                R = hit ? key : 0u;
                // the deferred entry, before any row read
                if (pend_at != kRowsPad) rows[pend_at] = pend_word | pend_bit;
                pend_at = kRowsPad;
                pend_bit = 0;
                // the row the chosen bin leaves and the row it enters, read together
                const uint32_t Rn = (hit ? R : Bn) - wj;
                if constexpr (kLaneRows) {
                    rw[0] = ulane < NS ? rows[R * NS + ulane] : 0u;
                    rn[0] = ulane < NS ? rows[Rn * NS + ulane] : 0u;
                    const uint32_t sk = rw[0] ? 32u * ulane + static_cast<uint32_t>(__clz(rw[0])) : kNoKey;
                    sf = __reduce_min_sync(kFull, sk);
                    sf = hit ? sf : 0u;
                } else {
                    if constexpr (NS == 2) {        // a row is one 8-byte word pair
                        const uint2 ra = *reinterpret_cast<const uint2*>(rows + R * 2u);
                        const uint2 rb = *reinterpret_cast<const uint2*>(rows + Rn * 2u);
                        rw[0] = ra.x;
                        rw[1] = ra.y;
                        rn[0] = rb.x;
                        rn[1] = rb.y;
                    } else {
#pragma unroll
                        for (int q = 0; q < NS; ++q) {
                            rw[q] = rows[R * NS + q];
                            rn[q] = rows[Rn * NS + q];
                        }
                    }
#pragma unroll
                    for (int q = NS - 1; q >= 0; --q)
                        sf = rw[q] ? 32u * q + static_cast<uint32_t>(__clz(rw[q])) : sf;
                }
            } else {
                const uint32_t key = bf_scan<kR>(wj, L);
                hit = key != kNoKey;
                sf = hit ? (key & 0x7FFFu) >> 7 : 0u;
                R = (key >> 15) + wj;
            }
            if (kSeg && c == kBF) {
                // RANDOM: a BF item still keeps the segment maxima exact
                uint32_t v = 0;
#pragma unroll
                for (int q = 0; q < NS; ++q) v = (sf >> 5) == static_cast<uint32_t>(q) ? sm[q] : v;
                Mseg = __shfl_sync(kFull, v, static_cast<int>(sf & 31));
            }

            // 2. in segment sf: the chosen bin (FF: first fitting; BF / WF:
            //    first at residual R) as (index, residual) and (index,
            //    capacity) keys; cR = bins at R, cM = bins at Mseg, M2 = the
            //    largest residual other than Mseg
            const uint4 Q = reinterpret_cast<const uint4*>(slots)[32u * sf + ulane];
            const uint32_t r0 = Q.x >> kR, r1 = Q.y >> kR, r2 = Q.z >> kR, r3 = Q.w >> kR;
            const uint32_t c0 = Q.x & kCap, c1 = Q.y & kCap, c2 = Q.z & kCap, c3 = Q.w & kCap;
            const uint32_t i0 = (4u * ulane) << 16;
            const uint32_t j0 = (4u * ulane) << 20;          // 10-bit form: index field of a key
            uint32_t k1 = kNoKey, k2 = kNoKey, cR = 0, cM = 0, M2 = 0;
            if (kSeg && CRIT != kFF) {      // these need only the quad: issued first
                cM = __reduce_add_sync(kFull, (r0 == Mseg) + (r1 == Mseg) + (r2 == Mseg) + (r3 == Mseg));
                M2 = __reduce_max_sync(kFull, max(max(r0 != Mseg ? r0 : 0u, r1 != Mseg ? r1 : 0u),
                                                  max(r2 != Mseg ? r2 : 0u, r3 != Mseg ? r3 : 0u)));
            }
            if (c == kFF && W10) {
                // keys grow with the index: the first fitting bin is the minimum
                k1 = min(min(r0 >= wj ? j0 | Q.x : kNoKey, r1 >= wj ? (j0 + (1u << 20)) | Q.y : kNoKey),
                         min(r2 >= wj ? (j0 + (2u << 20)) | Q.z : kNoKey, r3 >= wj ? (j0 + (3u << 20)) | Q.w : kNoKey));
            } else if (c == kFF) {
                k1 = min(min(r0 >= wj ? i0 | r0 : kNoKey, r1 >= wj ? (i0 + (1u << 16)) | r1 : kNoKey),
                         min(r2 >= wj ? (i0 + (2u << 16)) | r2 : kNoKey, r3 >= wj ? (i0 + (3u << 16)) | r3 : kNoKey));
                k2 = min(min(r0 >= wj ? i0 | c0 : kNoKey, r1 >= wj ? (i0 + (1u << 16)) | c1 : kNoKey),
                         min(r2 >= wj ? (i0 + (2u << 16)) | c2 : kNoKey, r3 >= wj ? (i0 + (3u << 16)) | c3 : kNoKey));
                k2 = __reduce_min_sync(kFull, k2);
            } else if (W10) {
                k1 = min(min(r0 == R ? j0 | Q.x : kNoKey, r1 == R ? (j0 + (1u << 20)) | Q.y : kNoKey),
                         min(r2 == R ? (j0 + (2u << 20)) | Q.z : kNoKey, r3 == R ? (j0 + (3u << 20)) | Q.w : kNoKey));
                if (IDX) cR = __reduce_add_sync(kFull, (r0 == R) + (r1 == R) + (r2 == R) + (r3 == R));
            } else {
                k1 = min(min(r0 == R ? i0 | c0 : kNoKey, r1 == R ? (i0 + (1u << 16)) | c1 : kNoKey),
                         min(r2 == R ? (i0 + (2u << 16)) | c2 : kNoKey, r3 == R ? (i0 + (3u << 16)) | c3 : kNoKey));
                if (IDX) cR = __reduce_add_sync(kFull, (r0 == R) + (r1 == R) + (r2 == R) + (r3 == R));
            }
            k1 = __reduce_min_sync(kFull, k1);
            uint32_t b, r_old, Bt;
            if (W10) {                                 // (index << 20) | (residual << 10) | capacity
                b = hit ? 128u * sf + (k1 >> 20) : L;
                // a BF or WF item takes a bin at the residual R it sought
                r_old = hit ? (c == kFF ? (k1 >> 10) & 0x3FFu : R) : Bn;
                Bt = hit ? k1 & 0x3FFu : Bn;
            } else {
                b = hit ? 128u * sf + (k1 >> 16) : L;
                r_old = hit ? (c == kFF ? (k1 & 0xFFFFu) : R) : Bn;
                Bt = hit ? ((c == kFF ? k2 : k1) & 0xFFFFu) : Bn;
            }
            const uint32_t r_new = r_old - wj;
            const bool cross = (Bt < 2u * r_old) && (2u * r_new <= Bt);    // Rule 5
            const bool fire = R3 ? remark3_divide(below, Bl, !hit, Bt, cross) : cross;
            const uint32_t Lf = hit ? L : L + 1u;      // where a divided-off bin goes
            // every lane writes the same words (a predicated store for the
            // divided-off bin: no branch, nothing written when it does not
            // divide)
            slots[b] = (r_new << kR) | Bt;
            if (fire) slots[Lf] = (Bt << kR) | Bt;
            // the chosen bin lies in segment sf (or is the new bin L): known
            // before the bin itself, so the updates below need not wait for it
            const uint32_t sb = hit ? sf : (L >> 7), sfire = Lf >> 7;

            // 3. segment maxima
            if (kSeg) {
                uint32_t top;
                if constexpr (CRIT == kFF) {
                    // the new maximum of segment sf by one warp maximum over
                    // the quad with the chosen slot updated: one reduction
                    // fewer per item (WF, whose chosen bin always holds the
                    // maximum, keeps the count at the maximum and the next
                    // largest, issued beside the bin's reduction)
                    const uint32_t pq = b & 127u;
                    const bool mine = hit && ulane == (pq >> 2);
                    const uint32_t e = pq & 3u;
                    const uint32_t u0 = (mine && e == 0u) ? r_new : r0, u1 = (mine && e == 1u) ? r_new : r1;
                    const uint32_t u2 = (mine && e == 2u) ? r_new : r2, u3 = (mine && e == 3u) ? r_new : r3;
                    top = __reduce_max_sync(kFull, max(max(u0, u1), max(u2, u3)));
                } else {
                    top = (r_old != Mseg || cM >= 2u) ? Mseg : max(M2, r_new);
                }
#pragma unroll
                for (int q = 0; q < NS; ++q) {
                    const uint32_t s = 32u * q + ulane;
                    uint32_t v = sm[q];
                    v = s == sb ? (hit ? top : max(v, r_new)) : v;
                    v = (fire && s == sfire) ? max(v, Bt) : v;
                    sm[q] = v;
                }
            }
            // 4. the BF index: r_old leaves segment sb when the chosen bin was
            //    its only bin at r_old; r_new and a divided-off bin's
            //    capacity enter
            if (IDX) {
                if (c != kBF) {
                    // (RANDOM) an FF or WF item: the deferred entry, then the rows
                    rows[pend_at] = pend_word | pend_bit;
                    pend_at = kRowsPad;
                    pend_bit = 0;
                    if constexpr (kLaneRows) {
                        rw[0] = ulane < NS ? rows[r_old * NS + ulane] : 0u;
                        rn[0] = ulane < NS ? rows[r_new * NS + ulane] : 0u;
                    } else {
#pragma unroll
                        for (int q = 0; q < NS; ++q) {
                            rw[q] = rows[r_old * NS + q];
                            rn[q] = rows[r_new * NS + q];
                        }
                    }
                    if (c == kFF)
                        cR = __reduce_add_sync(kFull, (r0 == r_old) + (r1 == r_old) + (r2 == r_old) + (r3 == r_old));
                    else
                        cR = cM;
                }
                // selects and predicated stores only (no branch): a store that
                // does not apply is not made, or writes the pad word
                const bool clear = hit && cR == 1u;
                bool any;
                if constexpr (kLaneRows) {
                    // the lane holding word sb / 32 writes both rows' words
                    const bool here = ulane == (sb >> 5);
                    const uint32_t cl = here ? rw[0] & ~(0x80000000u >> (sb & 31)) : rw[0];
                    any = __any_sync(kFull, cl != 0u);
                    if (here) {
                        rows[clear ? r_old * NS + (sb >> 5) : kRowsPad] = cl;
                        rows[r_new > 0u ? r_new * NS + (sb >> 5) : kRowsPad] = rn[0] | (0x80000000u >> (sb & 31));
                    }
                } else {
                    uint32_t anyw = 0, word = 0, wnew = 0;
#pragma unroll
                    for (int q = 0; q < NS; ++q) {
                        const bool here = (sb >> 5) == static_cast<uint32_t>(q);
                        const uint32_t cl = here ? rw[q] & ~(0x80000000u >> (sb & 31)) : rw[q];
                        word = here ? cl : word;
                        anyw |= cl;
                        wnew = here ? rn[q] : wnew;
                    }
                    any = anyw != 0u;
                    if (clear) rows[r_old * NS + (sb >> 5)] = word;
                    rows[r_new > 0u ? r_new * NS + (sb >> 5) : kRowsPad] = wnew | (0x80000000u >> (sb & 31));
                }
                wb = (clear && !any && (r_old >> 5) == ulane) ? wb & ~(0x80000000u >> (r_old & 31)) : wb;
                wb = (r_new > 0u && (r_new >> 5) == ulane) ? wb | (0x80000000u >> (r_new & 31)) : wb;
                pend_at = fire ? Bt * NS + (sfire >> 5) : kRowsPad;
                pend_bit = fire ? 0x80000000u >> (sfire & 31) : 0u;
                wb = (fire && (Bt >> 5) == ulane) ? wb | (0x80000000u >> (Bt & 31)) : wb;
            }
            L += (hit ? 0u : 1u) + (fire ? 1u : 0u);
            bout = ulane == jj ? b : bout;
            d = dn;
            msk = mskn;
            // with the rows in every lane, each lane stores every word the
            // item changes and reads only words it stored itself; spread
            // rows are written by one lane and read by another
            if constexpr (kLaneRows) __syncwarp();
        }
            if (ulane < cnt) raw[j0 + ulane] = static_cast<int32_t>(bout);
            fit_tests += fit_blk;
        }
        L_io = L;
        return true;
    }

    // 16-bit slots (B_1 <= 255): slot = (residual << 8) | capacity, kH16Slots
    // of them in segments of 256 bins (one 16-byte read per lane still covers
    // a segment; kNS16 segment words per lane), with the BF index rows r16 of
    // 256 residuals after them.  A key (index in the segment << 16) | slot
    // carries index, residual and capacity at once.  BF items use the
    // residual index (IDX: laid out whenever BF items occur).  A system that
    // would outgrow the slots, or whose bins so far, extrapolated to all k
    // items, pass them, is appended to spill_list2 and packed in global
    // memory.
    template <bool IDX, bool R3>
    __device__ __forceinline__ bool run16(const H1Params& p, int64_t i, const int32_t* w, uint32_t k,
                                          int32_t* raw, int n, uint32_t& L_io,
                                          unsigned long long& fit_tests, uint32_t* r16) const {
        constexpr uint32_t kPad16 = (kH16MaxB + 1) * kNS16;     // index word past the rows
        uint16_t* s16 = reinterpret_cast<uint16_t*>(slots);
        uint32_t L = L_io;
        constexpr uint32_t cap_bins = kH16Slots;
        const uint32_t ulane = static_cast<uint32_t>(lane);
        const uint32_t Bl = R3 ? Bs[ulane] : 0u;      // Remark 3 as in run()
        uint32_t below = (R3 && L > 0 && ulane < static_cast<uint32_t>(n)) ? 1u : 0u;

        uint32_t sm[kNS16];                 // segment maxima, segment 32q + lane
        uint32_t wb = 0;                 // residuals 32*lane .. 32*lane+31 present
#pragma unroll
        for (int q = 0; q < kNS16; ++q) sm[q] = 0;
        if (kSeg && L > 0 && lane == 0) sm[0] = Bs[0];
        if (IDX) {
            for (uint32_t t = 0; t < L; ++t) {
                const uint32_t r = Bs[t];
                if ((r >> 5) == ulane) wb |= 1u << (r & 31);
            }
        }
        uint32_t pend_at = kPad16, pend_bit = 0;
        uint32_t dnext = descriptor(weight(w, ulane, k), ulane, n, p.seed, 0);
        uint32_t wpre = weight(w, 32 + ulane, k);
        for (uint32_t j0 = 0; j0 < k; j0 += 32u) {
            const uint32_t cnt = min(32u, k - j0);
            const bool trend = !p.no_trend && j0 >= 2048u &&
                               static_cast<uint64_t>(L) * k > static_cast<uint64_t>(cap_bins) * j0;
            if (L + 2u * cnt > cap_bins || trend) {
                if (lane == 0) {
                    const unsigned long long pos = atomicAdd(
                        reinterpret_cast<unsigned long long*>(p.spill_seg2 + 1), 1ull);
                    p.spill_list2[pos] = static_cast<int32_t>(i);
                }
                __syncwarp();
                return false;
            }
            const uint32_t dblk = dnext;
            dnext = descriptor(wpre, static_cast<int64_t>(j0) + 32 + ulane, n, p.seed, 0);
            wpre = weight(w, static_cast<int64_t>(j0) + 64 + ulane, k);
            uint32_t d = __shfl_sync(kFull, dblk, 0);
            uint32_t bout = 0;
        for (uint32_t jj = 0; jj < cnt; ++jj) {
            const uint32_t dn = __shfl_sync(kFull, dblk, static_cast<int>((jj + 1u) & 31u));
            const uint32_t wj = d & 0x7FFFu;
            const uint32_t Bn = (d >> 16) & 0x7FFFu;
            const int c = CRIT == kRandom ? static_cast<int>(((d >> 15) & 1u) | ((d >> 30) & 2u)) : CRIT;
            fit_tests += L;
            uint32_t pend_word = 0;
            if (IDX) pend_word = r16[pend_at];

            // 1. the segment holding the answer (as in the 32-bit form)
            bool hit = false;
            uint32_t sf = 0, Mseg = 0, R = 0;
            uint32_t rwl = 0, rnl = 0;        // word `lane` of the two index rows
            if (kSeg && c == kFF) {
                uint32_t key = kNoKey;
#pragma unroll
                for (int q = kNS16 - 1; q >= 0; --q)
                    key = sm[q] >= wj ? ((32u * q + ulane) << 16) | sm[q] : key;
                key = __reduce_min_sync(kFull, key);
                hit = key != kNoKey;
                sf = hit ? key >> 16 : 0u;
                Mseg = key & 0xFFFFu;
            } else if (kSeg && c == kWF) {
                uint32_t key = 0;
#pragma unroll
                for (int q = 0; q < kNS16; ++q) key = max(key, (sm[q] << 9) | (511u - (32u * q + ulane)));
                key = __reduce_max_sync(kFull, key);
                Mseg = key >> 9;
                sf = 511u - (key & 511u);
                hit = Mseg >= wj;
                R = Mseg;
            } else if (IDX) {
                const uint32_t wi = wj >> 5;
                const uint32_t x = wb & (ulane < wi ? 0u : ulane == wi ? ~((1u << (wj & 31)) - 1u) : 0xFFFFFFFFu);
                uint32_t key = x ? 32u * ulane + static_cast<uint32_t>(__ffs(x) - 1) : kNoKey;
                key = __reduce_min_sync(kFull, key);
                hit = key != kNoKey;
                R = hit ? key : 0u;
                if (pend_at != kPad16) r16[pend_at] = pend_word | pend_bit;
                pend_at = kPad16;
                pend_bit = 0;
                // the row the chosen bin leaves and the row it enters: word q
                // of each in lane q; the first segment holding R by one
                // warp minimum
                const uint32_t Rn = (hit ? R : Bn) - wj;
                rwl = ulane < kNS16 ? r16[R * kNS16 + ulane] : 0u;
                rnl = ulane < kNS16 ? r16[Rn * kNS16 + ulane] : 0u;
                const uint32_t sk = rwl ? 32u * ulane + static_cast<uint32_t>(__ffs(rwl) - 1) : kNoKey;
                sf = __reduce_min_sync(kFull, sk);
                sf = hit ? sf : 0u;
            }
            if (kSeg && c == kBF) {
                uint32_t v = 0;
#pragma unroll
                for (int q = 0; q < kNS16; ++q) v = (sf >> 5) == static_cast<uint32_t>(q) ? sm[q] : v;
                Mseg = __shfl_sync(kFull, v, static_cast<int>(sf & 31));
            }

            // 2. in segment sf: eight 16-bit slots per lane
            const uint4 Q = reinterpret_cast<const uint4*>(slots)[32u * sf + ulane];
            uint32_t h[8];
            h[0] = Q.x & 0xFFFFu; h[1] = Q.x >> 16; h[2] = Q.y & 0xFFFFu; h[3] = Q.y >> 16;
            h[4] = Q.z & 0xFFFFu; h[5] = Q.z >> 16; h[6] = Q.w & 0xFFFFu; h[7] = Q.w >> 16;
            const uint32_t i0 = (8u * ulane) << 16;
            uint32_t k1 = kNoKey, cR = 0, cM = 0, M2 = 0;
            if (kSeg) {
                uint32_t nm = 0, m2 = 0;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const uint32_t r = h[e] >> 8;
                    nm += r == Mseg ? 1u : 0u;
                    m2 = max(m2, r != Mseg ? r : 0u);
                }
                cM = __reduce_add_sync(kFull, nm);
                M2 = __reduce_max_sync(kFull, m2);
            }
            if (c == kFF) {
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    k1 = min(k1, (h[e] >> 8) >= wj ? (i0 + (static_cast<uint32_t>(e) << 16)) | h[e] : kNoKey);
            } else {
                uint32_t nr = 0;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const bool eq = (h[e] >> 8) == R;
                    k1 = min(k1, eq ? (i0 + (static_cast<uint32_t>(e) << 16)) | h[e] : kNoKey);
                    nr += eq ? 1u : 0u;
                }
                if (IDX) cR = __reduce_add_sync(kFull, nr);
            }
            k1 = __reduce_min_sync(kFull, k1);
            const uint32_t b = hit ? 256u * sf + (k1 >> 16) : L;
            // a BF item takes a bin at the residual R it sought
            const uint32_t r_old = hit ? (c == kBF ? R : (k1 >> 8) & 0xFFu) : Bn;
            const uint32_t Bt = hit ? k1 & 0xFFu : Bn;
            const uint32_t r_new = r_old - wj;
            const bool cross = (Bt < 2u * r_old) && (2u * r_new <= Bt);    // Rule 5
            const bool fire = R3 ? remark3_divide(below, Bl, !hit, Bt, cross) : cross;
            const uint32_t Lf = hit ? L : L + 1u;
            s16[b] = static_cast<uint16_t>((r_new << 8) | Bt);
            if (fire) s16[Lf] = static_cast<uint16_t>((Bt << 8) | Bt);
            // the chosen bin lies in segment sf (or is the new bin L)
            const uint32_t sb = hit ? sf : (L >> 8), sfire = Lf >> 8;

            // 3. segment maxima
            if (kSeg) {
                const uint32_t top = (r_old != Mseg || cM >= 2u) ? Mseg : max(M2, r_new);
#pragma unroll
                for (int q = 0; q < kNS16; ++q) {
                    const uint32_t s = 32u * q + ulane;
                    uint32_t v = sm[q];
                    v = s == sb ? (hit ? top : max(v, r_new)) : v;
                    v = (fire && s == sfire) ? max(v, Bt) : v;
                    sm[q] = v;
                }
            }
            // 4. the BF index
            if (IDX) {
                if (c != kBF) {
                    if (pend_at != kPad16) r16[pend_at] = pend_word | pend_bit;
                    pend_at = kPad16;
                    pend_bit = 0;
                    rwl = ulane < kNS16 ? r16[r_old * kNS16 + ulane] : 0u;
                    rnl = ulane < kNS16 ? r16[r_new * kNS16 + ulane] : 0u;
                    if (c == kFF) {
                        uint32_t nr = 0;
#pragma unroll
                        for (int e = 0; e < 8; ++e) nr += (h[e] >> 8) == r_old ? 1u : 0u;
                        cR = __reduce_add_sync(kFull, nr);
                    } else {
                        cR = cM;
                    }
                }
                // the lane holding word sb / 32 writes both rows' words
                const bool clear = hit && cR == 1u;
                const bool here = ulane == (sb >> 5);
                const uint32_t cl = here ? rwl & ~(1u << (sb & 31)) : rwl;
                const bool any = __any_sync(kFull, cl != 0u);
                if (here) {
                    if (clear) r16[r_old * kNS16 + (sb >> 5)] = cl;
                    r16[r_new > 0u ? r_new * kNS16 + (sb >> 5) : kPad16] = rnl | (1u << (sb & 31));
                }
                wb = (clear && !any && (r_old >> 5) == ulane) ? wb & ~(1u << (r_old & 31)) : wb;
                wb = (r_new > 0u && (r_new >> 5) == ulane) ? wb | (1u << (r_new & 31)) : wb;
                pend_at = fire ? Bt * kNS16 + (sfire >> 5) : kPad16;
                pend_bit = fire ? 1u << (sfire & 31) : 0u;
                wb = (fire && (Bt >> 5) == ulane) ? wb | (1u << (Bt & 31)) : wb;
            }
            L += (hit ? 0u : 1u) + (fire ? 1u : 0u);
            bout = ulane == jj ? b : bout;
            d = dn;
            __syncwarp();
        }
            if (ulane < cnt) raw[j0 + ulane] = static_cast<int32_t>(bout);
        }
        L_io = L;
        return true;
    }
};

// One warp per membrane system; blockDim.x / 32 warps per block, each with
// p.group_bytes of shared memory.  Direct mode only (no sublists).
// R3: Rule 5 with Remark 3's per-type condition (VSBPP_REMARK3), a kernel of
// its own so that the other kernels' item step is unchanged.
template <int NS, int CRIT, bool R3>
__global__ void __launch_bounds__(512, 1) h1w_pack_kernel(const H1Params p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = static_cast<int>(threadIdx.x) & 31;
    const int wid = static_cast<int>(threadIdx.x) >> 5;
    const int groups = static_cast<int>(blockDim.x) >> 5;
    unsigned char* const group = smem + static_cast<size_t>(wid) * static_cast<size_t>(p.group_bytes);
    unsigned char* base = group;
    H1Warp<NS, CRIT> g;
    g.lane = lane;
    g.slots = reinterpret_cast<uint32_t*>(base);
    base += 4 * p.slot_cap + 16;
    g.rows = nullptr;
    if (p.bf_index) {
        g.rows = reinterpret_cast<uint32_t*>(base);
        base += 4 * (kIndexMaxRes + 1) * NS + 16;
    }
    // capacities: the last bytes of the group (past either slot layout)
    g.Bs = reinterpret_cast<uint32_t*>(group + p.group_bytes - 4 * kMaxTypes);
    // the 16-bit layout's BF rows (after its slots)
    uint32_t* const rows16 = reinterpret_cast<uint32_t*>(group + 2 * kH16Slots + 16);
    const bool fits16 = p.group_bytes >= h1w16_group_bytes(p.bf_index);

    int64_t begin, end;
    if (p.seg) {
        begin = p.seg[p.segment];
        end = p.seg[p.segment + 1];
    } else {
        begin = p.range_begin;
        end = p.range_end;
    }
    const int64_t count = end - begin;
    if (count <= 0) return;

    int64_t u = 0;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * groups;
    if (!p.queue) u = static_cast<int64_t>(blockIdx.x) * groups + wid;
    for (;;) {
        if (p.queue) {
            unsigned long long v = 0;
            if (lane == 0) v = atomicAdd(p.queue, 1ull);
            u = static_cast<long long>(__shfl_sync(kFull, v, 0));
        }
        if (u >= count) break;
        const int64_t i = p.order ? static_cast<int64_t>(p.order[begin + u]) : begin + u;
        if (!p.queue) u += stride;

        if (p.out.status[i] != VSBPP_OK) continue;        // rejected by validation
        if (p.cls && p.cls[i] != p.want_cls) continue;
        const int64_t k = p.in.m(i);
        const int64_t wb = p.in.w_begin(i);
        const int32_t* w = p.in.w_all + wb;
        const int n = p.in.n(i);
        const int32_t* B = p.in.B_all + p.in.B_begin(i);
        const uint32_t Bl = lane < n ? static_cast<uint32_t>(B[lane]) : 0u;
        g.Bs[lane] = Bl;
        int32_t* raw = p.out.bin_of_item + wb;
        int32_t* types_out = p.out.bin_type + wb;
        const uint32_t B1 = __shfl_sync(kFull, Bl, 0);
        const bool use_idx = g.rows != nullptr && H1Warp<NS, CRIT>::kBFItems &&
                             B1 <= static_cast<uint32_t>(kIndexMaxRes);
        const bool w10 = B1 <= 1023u;                 // 10-bit slot form
        // 16-bit slot form: systems too large for the 32-bit slots (only the
        // largest shape, NS = 8, has systems past its reach)
        const bool use16 = NS == 8 && fits16 && p.spill_list2 != nullptr && p.h16_min_m > 0 &&
                           B1 <= kH16MaxB && k >= p.h16_min_m &&
                           (!H1Warp<NS, CRIT>::kBFItems || p.bf_index);
        const int kR = use16 ? 8 : w10 ? 10 : 16;
        const uint32_t kCapMask = use16 ? 0xFFu : w10 ? 0x3FFu : 0xFFFFu;
        uint16_t* s16 = reinterpret_cast<uint16_t*>(g.slots);

        // every slot reads as empty until its bin exists; index rows start clear
        const int quads = use16 ? static_cast<int>(kH16Slots / 8) : p.slot_cap / 4;
        for (int q = lane; q < quads; q += 32)
            reinterpret_cast<uint4*>(g.slots)[q] = make_uint4(0u, 0u, 0u, 0u);
        if (use16 && H1Warp<NS, CRIT>::kBFItems)
            for (uint32_t x = static_cast<uint32_t>(lane); x < (B1 + 1u) * kNS16; x += 32u) rows16[x] = 0u;
        else if (use_idx)
            for (uint32_t x = static_cast<uint32_t>(lane); x < (B1 + 1u) * NS; x += 32u) g.rows[x] = 0u;
        __syncwarp();
        uint32_t L = 0;
        if (p.preopen) {                     // literal Rule 2: one empty bin per type
            if (lane < n) {
                if (use16) s16[lane] = static_cast<uint16_t>((Bl << 8) | Bl);
                else g.slots[lane] = (Bl << kR) | Bl;
                if (use16 && H1Warp<NS, CRIT>::kBFItems) atomicOr(&rows16[Bl * kNS16], 1u);   // segment 0
                else if (use_idx) atomicOr(&g.rows[Bl * NS], 0x80000000u);   // segment 0, top bit first
            }
            L = static_cast<uint32_t>(n);
            __syncwarp();
        }
        unsigned long long fit_tests = 0;
        bool done = false;
        const uint32_t k32 = static_cast<uint32_t>(k);
        if (use16) {
            if constexpr (NS == 8)
                done = g.template run16<H1Warp<NS, CRIT>::kBFItems, R3>(p, i, w, k32, raw, n, L, fit_tests, rows16);
        } else if constexpr (H1Warp<NS, CRIT>::kBFItems) {
            done = use_idx ? g.template run<true, true, R3>(p, i, w, 0, k32, raw, n, L, fit_tests)
                 : w10     ? g.template run<false, true, R3>(p, i, w, 0, k32, raw, n, L, fit_tests)
                           : g.template run<false, false, R3>(p, i, w, 0, k32, raw, n, L, fit_tests);
        } else {
            done = w10 ? g.template run<false, true, R3>(p, i, w, 0, k32, raw, n, L, fit_tests)
                       : g.template run<false, false, R3>(p, i, w, 0, k32, raw, n, L, fit_tests);
        }
        if (!done) continue;                 // spilled: a full-size launch repacks it

        // --- objective (Section 1) and dense ids: used bins in creation order ---
        __syncwarp();
        const uint32_t per = (L + 31u) / 32u;
        uint32_t b0 = static_cast<uint32_t>(lane) * per;
        if (b0 > L) b0 = L;
        const uint32_t b1 = (b0 + per) < L ? (b0 + per) : L;
        uint32_t cnt = 0;
        for (uint32_t b = b0; b < b1; ++b) {
            const uint32_t s = use16 ? static_cast<uint32_t>(s16[b]) : g.slots[b];
            cnt += static_cast<uint32_t>((s >> kR) < (s & kCapMask));
        }
        const uint32_t excl = warp_exclusive_scan(cnt, lane);
        const uint32_t used_total = __shfl_sync(kFull, excl + cnt, 31);
        uint32_t dd = excl;
        uint64_t tot = 0;
        for (uint32_t b = b0; b < b1; ++b) {
            const uint32_t s = use16 ? static_cast<uint32_t>(s16[b]) : g.slots[b];
            const uint32_t cap = s & kCapMask;
            if ((s >> kR) < cap) {
                types_out[dd] = static_cast<int32_t>(g.type_of(cap, n));
                if (use16) s16[b] = static_cast<uint16_t>(dd);      // low 16 bits (see below)
                else g.slots[b] = dd;
                tot += cap;
                ++dd;
            }
        }
        __syncwarp();
        // 16-bit slots keep the low 16 bits of a dense id d <= b.  b - d counts
        // the unused bins before b: bins left empty by Rule 5 (each the
        // division of a distinct bin that does hold items, so at most half of
        // the 98304 slots) and the preopened ones, fewer than 65536 in all;
        // so d = b - ((b - low) mod 65536).
        for (int64_t j = lane; j < k; j += 32) {
            const uint32_t b = static_cast<uint32_t>(raw[j]);
            raw[j] = static_cast<int32_t>(use16 ? b - ((b - static_cast<uint32_t>(s16[b])) & 0xFFFFu)
                                                : g.slots[b]);
        }
        tot = warp_sum_u64(tot);
        if (lane == 0) {
            if (p.counters) {
                atomicAdd(p.counters, static_cast<unsigned long long>(k));
                atomicAdd(p.counters + 1, fit_tests);
            }
            p.out.num_bins[i] = static_cast<int64_t>(used_total);
            p.out.total[i] = static_cast<int64_t>(tot);
        }
        __syncwarp();                        // shared memory is reused by the next system
    }
}

}  // namespace vsbpp
