// h1_kernel.cuh -- the first heuristic of Section 6.3 on one GB300 SM.
//
// One thread group (G warps) runs one membrane system at a time: the items
// of a unit are taken in list order (Rule 3); for each item the bin membranes
// are tested for room (Rule 4, residual >= w) and FF / BF / WF (Section 1)
// picks one, the lowest creation index winning ties.  When nothing fits a bin
// of the smallest type holding the item is opened; the chosen bin's residual
// drops by w, and when its load first reaches half its capacity it divides
// off one empty bin of its type (Rule 5).
//
// GB300 layout.  Bin membranes live in shared memory as one packed word per
// bin, slot = (residual << SHIFT) | creation index, so each criterion is one
// unsigned minimum over slots:
//     BF:  min(slot - (w << SHIFT))  -> (r - w, idx); r < w wraps to the top
//          half of the range, so a non-fitting bin never wins
//     WF:  min(slot ^ HI)            -> (~r, idx): most room, lowest index
//     FF:  min over fitting slots of (idx, r)
// Slots are read as 16-byte quads; quad q belongs to thread q mod T of the
// group, the only writer of those four slots.  A segment (128 bins = 32
// consecutive quads) therefore belongs to one warp (segment s to warp
// s mod G), and each warp keeps exact summaries of its own segments:
//     segmax[s]    the largest residual in segment s (FF, WF)
//     segres[s]    bit r set iff segment s holds a bin with residual r
//     wbits[warp]  bit r set iff any of the warp's segments does (BF)
// so a warp answers the flat scan's question for its bins by scanning one
// segment: FF its first segment whose maximum is >= w, WF its first segment
// whose maximum equals its largest, BF -- with r* the least residual >= w in
// wbits -- its first segment holding r*.  The group minimum of the warps'
// keys is the flat scan's answer.  A warp reads only summaries it writes, so
// the only barrier per item is the exchange of per-warp minima (none when
// G = 1).  BF falls back to the full scan when B_1 > 1023 (no index).
// Item weights are streamed into shared memory a chunk at a time with
// cp.async, one chunk ahead of the one being packed.
#pragma once

#include "device_common.cuh"

namespace vsbpp {

template <typename S>
struct SlotTraits;

// Narrow slots: 16-bit residual (B_1 <= 32767) and 16-bit index (<= 65536 bins).
template <>
struct SlotTraits<uint32_t> {
    using S = uint32_t;
    static constexpr int kShift = 16;
    static constexpr S kNone = 0xFFFFFFFFu;
    static constexpr S kHi = 0xFFFF0000u;
    static constexpr S kLo = 0x0000FFFFu;
    static constexpr S kSign = 0x80000000u;
    static constexpr int64_t kMaxCap = 32767;
    static constexpr int64_t kMaxBins = 65536;
    __device__ static __forceinline__ S warp_min(S v) { return __reduce_min_sync(kFull, v); }
    __device__ static __forceinline__ void load_quad(const S* p, uint32_t q, S& a, S& b, S& c, S& d) {
        const uint4 v = reinterpret_cast<const uint4*>(p)[q];
        a = v.x; b = v.y; c = v.z; d = v.w;
    }
    __device__ static __forceinline__ void store_quad(S* p, uint32_t q, S a, S b, S c, S d) {
        reinterpret_cast<uint4*>(p)[q] = make_uint4(a, b, c, d);
    }
};

// Wide slots: 32-bit residual (B_1 < 2^31) and 32-bit index.
template <>
struct SlotTraits<unsigned long long> {
    using S = unsigned long long;
    static constexpr int kShift = 32;
    static constexpr S kNone = ~0ull;
    static constexpr S kHi = 0xFFFFFFFF00000000ull;
    static constexpr S kLo = 0x00000000FFFFFFFFull;
    static constexpr S kSign = 0x8000000000000000ull;
    static constexpr int64_t kMaxCap = 0x7FFFFFFF;
    static constexpr int64_t kMaxBins = 0x7FFFFFFF;
    __device__ static __forceinline__ S warp_min(S v) { return warp_min_u64(v); }
    __device__ static __forceinline__ void load_quad(const S* p, uint32_t q, S& a, S& b, S& c, S& d) {
        const ulonglong2 v0 = reinterpret_cast<const ulonglong2*>(p)[2 * q];
        const ulonglong2 v1 = reinterpret_cast<const ulonglong2*>(p)[2 * q + 1];
        a = v0.x; b = v0.y; c = v1.x; d = v1.y;
    }
    __device__ static __forceinline__ void store_quad(S* p, uint32_t q, S a, S b, S c, S d) {
        reinterpret_cast<ulonglong2*>(p)[2 * q] = make_ulonglong2(a, b);
        reinterpret_cast<ulonglong2*>(p)[2 * q + 1] = make_ulonglong2(c, d);
    }
};

// Launch parameters of the first-heuristic kernel.
struct H1Params {
    BatchView in;
    OutView out;
    UnitMap units;
    int32_t criterion;
    int32_t preopen;
    uint64_t seed;
    // Work list: positions [seg[segment], seg[segment+1]) when seg != null,
    // else [range_begin, range_end); a position x names unit order[x], or
    // unit x itself when order == null.  With queue != null the groups pull
    // positions through an atomic counter (work stealing); otherwise static
    // round robin.  With cls != null a unit whose class differs from
    // want_cls is skipped (single-instance launches of the plain path).
    const int32_t* order;
    const int64_t* seg;
    int32_t segment;
    int64_t range_begin, range_end;
    unsigned long long* queue;
    const int32_t* cls;
    int32_t want_cls;
    // Spill: with spill_list != null, a group whose system would outgrow
    // slot_cap stops and appends the instance to spill_list (count in
    // spill_seg[1]); a worst-case-sized launch packs it again from the start.
    int32_t* spill_list;
    int64_t* spill_seg;
    // One-warp kernel only: a system with B_1 <= 255 and at least h16_min_m
    // items (0: none) packs in 16-bit slots, twice slot_cap of them; one that
    // outgrows those goes to spill_list2 (count in spill_seg2[1]), which
    // global memory packs.
    int64_t h16_min_m;
    int32_t* spill_list2;
    int64_t* spill_seg2;
    unsigned long long* counters;  // null, or {items, fit tests} to add to
    int32_t compose;        // 1: write sublist-local results (see OutView)
    int32_t remark3;        // 1: Rule 5 with Remark 3's per-type condition (VSBPP_REMARK3)
    int32_t no_trend;       // 1: spill only when the slots run out (lists sorted by
                            // decreasing weight open most of their bins first)
    int32_t bf_index;       // 1: the BF residual index is laid out (used when B_1 <= 1023)
    int32_t chunk;          // items staged per step (multiple of 32)
    int32_t slot_cap;       // bins per group (multiple of 128: whole segments)
    int32_t group_bytes;    // shared memory per group
};

// Shared-memory footprint of one group (host and device agree on this).
__host__ __device__ inline int h1_align16(int x) { return (x + 15) & ~15; }
constexpr int kIndexMaxRes = 1023;       // residuals the BF index covers (32 words)

__host__ __device__ inline int h1_group_bytes(int slot_cap, int chunk, int slot_size, int G = 1,
                                              int bf_index = 0) {
    const int nseg = (slot_cap + 127) / 128;
    return h1_align16(slot_cap * slot_size)      // slots
         + h1_align16(slot_cap)                  // bin types (uint8)
         + h1_align16(4 * nseg)                  // per-segment largest residual
         + (bf_index ? nseg * 128 + G * 128 : 0) // residual bitmaps: per segment, per warp
         + 2 * chunk * 4                         // double-buffered weights
         + kMaxTypes * 4                         // capacities
         + 2 * 32 * slot_size                    // per-warp minima, two buffers
         + 32 * 8                                // scan / totals exchange
         + 16;                                   // broadcast words
}

__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int G, int GROUPS, typename S>
struct H1Group {
    using Tr = SlotTraits<S>;
    static constexpr int T = 32 * G;
    static constexpr int kShift = Tr::kShift;

    int tid, lane, warp, gid;
    S* slots;
    uint8_t* typ;
    uint32_t* segmax;    // largest residual of each 128-bin segment (FF/WF)
    uint32_t* segres;    // [32 words][segment]: residuals present in the segment (BF);
                         // word-major so a warp's lanes read consecutive segments
    uint32_t nsegcap;    // segments in the slot array (the segres row length)
    uint32_t* wbits;     // [warp][32 words]: residuals present in the warp's segments (BF)
    int32_t* wst;
    uint32_t* Bs;
    S* red;
    uint64_t* xch;
    long long* bcast;

    __device__ __forceinline__ void sync() const {
        if constexpr (G == 1) {
            __syncwarp();
        } else if constexpr (GROUPS == 1) {
            __syncthreads();
        } else {
            named_barrier(1 + gid, T);
        }
    }

    __device__ __forceinline__ static uint32_t owner(uint32_t b) { return (b >> 2) & (T - 1); }

    // Owner-only: create bin b with residual r and type t.  The first slot of a
    // quad clears the other three so a partial quad never shows stale bins.
    __device__ __forceinline__ void put_new(uint32_t b, uint64_t r, uint32_t t) const {
        const S s = (static_cast<S>(r) << kShift) | static_cast<S>(b);
        if ((b & 3u) == 0u) {
            Tr::store_quad(slots, b >> 2, s, S(0), S(0), S(0));
        } else {
            slots[b] = s;
        }
        typ[b] = static_cast<uint8_t>(t);
    }

    // --- the fit test of Rule 4 over every live bin, one criterion each ---
    __device__ __forceinline__ S scan_bf(uint32_t nq, uint32_t w) const {
        const S W = static_cast<S>(w) << kShift;
        S best = Tr::kNone;
#pragma unroll 4
        for (uint32_t q = tid; q < nq; q += T) {
            S a, b, c, d;
            Tr::load_quad(slots, q, a, b, c, d);
            best = min(best, a - W);
            best = min(best, b - W);
            best = min(best, c - W);
            best = min(best, d - W);
        }
        return best;
    }

    __device__ __forceinline__ static S ff_key(S s) {
        return ((s & Tr::kLo) << kShift) | (s >> kShift);   // (idx, r)
    }

    // --- segment summaries (FF, WF): segment s = bins [128s, 128s+128) is
    // 32 consecutive quads, all owned by warp s mod G, which alone writes its
    // bins and its entry of segmax; a warp reads only its own segments, so
    // the summaries need no barrier.  Each warp returns its own best key.
    __device__ __forceinline__ S seg_ff(uint32_t nseg, uint32_t w) const {
        const S W = static_cast<S>(w) << kShift;
        for (uint32_t k0 = 0; static_cast<uint32_t>(warp) + G * k0 < nseg; k0 += 32) {
            const uint32_t sl = static_cast<uint32_t>(warp) + G * (k0 + static_cast<uint32_t>(lane));
            const uint32_t mx = sl < nseg ? segmax[sl] : 0u;
            const unsigned bal = __ballot_sync(kFull, mx >= w);
            if (bal) {
                const uint32_t sf = static_cast<uint32_t>(warp) + G * (k0 + __ffs(bal) - 1);
                S a, b, c, d;
                Tr::load_quad(slots, 32u * sf + static_cast<uint32_t>(lane), a, b, c, d);
                S cand = Tr::kNone;
                if (a >= W) cand = ff_key(a);
                else if (b >= W) cand = ff_key(b);
                else if (c >= W) cand = ff_key(c);
                else if (d >= W) cand = ff_key(d);
                return cand;
            }
        }
        return Tr::kNone;
    }

    __device__ __forceinline__ S seg_wf(uint32_t nseg) const {
        uint32_t mx = 0;
        for (uint32_t k0 = 0; static_cast<uint32_t>(warp) + G * k0 < nseg; k0 += 32) {
            const uint32_t sl = static_cast<uint32_t>(warp) + G * (k0 + static_cast<uint32_t>(lane));
            if (sl < nseg) mx = max(mx, segmax[sl]);
        }
        mx = __reduce_max_sync(kFull, mx);
        if (mx == 0u) return Tr::kNone;
        for (uint32_t k0 = 0; static_cast<uint32_t>(warp) + G * k0 < nseg; k0 += 32) {
            const uint32_t sl = static_cast<uint32_t>(warp) + G * (k0 + static_cast<uint32_t>(lane));
            const unsigned bal = __ballot_sync(kFull, sl < nseg && segmax[sl] == mx);
            if (bal) {
                const uint32_t sf = static_cast<uint32_t>(warp) + G * (k0 + __ffs(bal) - 1);
                S a, b, c, d;
                Tr::load_quad(slots, 32u * sf + static_cast<uint32_t>(lane), a, b, c, d);
                S best = min(a ^ Tr::kHi, b ^ Tr::kHi);
                best = min(best, min(c ^ Tr::kHi, d ^ Tr::kHi));
                return best;
            }
        }
        return Tr::kNone;
    }

    // BF with the residual index: r* = least residual >= w present in this
    // warp's segments, then the warp's first segment holding r*; in it the BF
    // key minimum is r* at its lowest index (no bin of the warp has a
    // residual in [w, r*)).
    __device__ __forceinline__ S seg_bf(uint32_t nseg, uint32_t w) const {
        const uint32_t* wb = wbits + warp * 32;
        uint32_t word = wb[lane];
        const uint32_t wi = w >> 5;
        if (static_cast<uint32_t>(lane) < wi) word = 0u;
        else if (static_cast<uint32_t>(lane) == wi) word &= ~((1u << (w & 31)) - 1u);
        const unsigned bal = __ballot_sync(kFull, word != 0u);
        if (!bal) return Tr::kNone;
        const int src = __ffs(bal) - 1;
        const uint32_t rs = static_cast<uint32_t>(src) * 32u +
                            static_cast<uint32_t>(__ffs(__shfl_sync(kFull, word, src)) - 1);
        const uint32_t rw = rs >> 5, rbit = 1u << (rs & 31);
        for (uint32_t k0 = 0; static_cast<uint32_t>(warp) + G * k0 < nseg; k0 += 32) {
            const uint32_t sl = static_cast<uint32_t>(warp) + G * (k0 + static_cast<uint32_t>(lane));
            const bool has = sl < nseg && (segres[rw * nsegcap + sl] & rbit);
            const unsigned b2 = __ballot_sync(kFull, has);
            if (b2) {
                const uint32_t sf = static_cast<uint32_t>(warp) + G * (k0 + __ffs(b2) - 1);
                S a, b, c, d;
                Tr::load_quad(slots, 32u * sf + static_cast<uint32_t>(lane), a, b, c, d);
                const S W = static_cast<S>(w) << kShift;
                S best = min(a - W, b - W);
                best = min(best, min(c - W, d - W));
                return best;
            }
        }
        return Tr::kNone;
    }

    // Owner warp of segment sg brings its summaries up to date after the
    // owners' slot writes of this item: the segment maximum (seg), and for the
    // BF index (idx) the removal of r_removed if no bin of the segment holds it
    // any more (and from the warp's bitmap if none of its segments does), and
    // the addition of r_add1 / r_add2 (residual 0 never fits and is not kept).
    __device__ __forceinline__ void seg_update(uint32_t sg, bool seg, bool idx, uint32_t nseg,
                                               int64_t r_removed, uint32_t r_add1,
                                               uint32_t r_add2) const {
        if (static_cast<uint32_t>(warp) != sg % G) return;
        __syncwarp();
        S a, b, c, d;
        Tr::load_quad(slots, 32u * sg + static_cast<uint32_t>(lane), a, b, c, d);
        if (seg) {
            const S top = max(max(a, b), max(c, d));
            const uint32_t r = __reduce_max_sync(kFull, static_cast<uint32_t>(top >> kShift));
            if (lane == 0) segmax[sg] = r;
        }
        if (idx) {
            uint32_t* wb = wbits + warp * 32;
            if (r_removed > 0) {
                const S R = static_cast<S>(r_removed);
                const bool here = (a >> kShift) == R || (b >> kShift) == R || (c >> kShift) == R ||
                                  (d >> kShift) == R;
                if (!__any_sync(kFull, here)) {
                    const uint32_t rw = static_cast<uint32_t>(r_removed) >> 5;
                    const uint32_t rbit = 1u << (static_cast<uint32_t>(r_removed) & 31);
                    if (lane == 0) segres[rw * nsegcap + sg] &= ~rbit;
                    __syncwarp();
                    bool any = false;
                    for (uint32_t k0 = 0; static_cast<uint32_t>(warp) + G * k0 < nseg; k0 += 32) {
                        const uint32_t sl = static_cast<uint32_t>(warp) + G * (k0 + static_cast<uint32_t>(lane));
                        any |= sl < nseg && (segres[rw * nsegcap + sl] & rbit);
                    }
                    if (!__any_sync(kFull, any) && lane == 0) wb[rw] &= ~rbit;
                }
            }
            if (lane == 0) {
                if (r_add1 > 0) {
                    segres[(r_add1 >> 5) * nsegcap + sg] |= 1u << (r_add1 & 31);
                    wb[r_add1 >> 5] |= 1u << (r_add1 & 31);
                }
                if (r_add2 > 0) {
                    segres[(r_add2 >> 5) * nsegcap + sg] |= 1u << (r_add2 & 31);
                    wb[r_add2 >> 5] |= 1u << (r_add2 & 31);
                }
            }
        }
        __syncwarp();
    }

    __device__ __forceinline__ void load_chunk(const int32_t* w, int64_t first, int64_t k,
                                               int buf, int chunk) const {
        int32_t* dst = wst + buf * chunk;
        const int64_t cnt = (k - first) < chunk ? (k - first) : chunk;
        for (int x = tid; x < cnt; x += T) cp_async4(dst + x, w + first + x);
        cp_async_commit();
    }

    // Rules 3-5 over the unit's items for one criterion CRIT (kRandom: drawn
    // per item).  Returns false when the unit outgrows its slots (spill).
    template <int CRIT>
    __device__ __forceinline__ bool item_loop(const H1Params& p, int64_t i, const int32_t* w,
                                              int64_t a, int64_t k, int32_t* raw, uint32_t Bl,
                                              bool use_idx, uint32_t& L_io,
                                              unsigned long long& fit_tests, uint32_t& below) const {
        const int chunk = p.chunk;
        uint32_t L = L_io;
        int jc = 0, buf = 0, par = 0;
        for (int64_t j = 0; j < k; ++j) {
            if (jc == 0) {
                cp_async_wait_all();
                sync();                        // this chunk is in shared memory
                if (j + chunk < k) load_chunk(w, j + chunk, k, buf ^ 1, chunk);
            }
            if (p.spill_list && L + 2u > static_cast<uint32_t>(p.slot_cap)) {
                // this system outgrows its slots (each item adds at most two)
                cp_async_wait_all();
                if (tid == 0) {
                    const unsigned long long pos = atomicAdd(
                        reinterpret_cast<unsigned long long*>(p.spill_seg + 1), 1ull);
                    p.spill_list[pos] = static_cast<int32_t>(i);
                }
                sync();
                return false;
            }
            const uint32_t wj = static_cast<uint32_t>(wst[buf * chunk + jc]);
            const int c = CRIT == kRandom ? pick_criterion(kRandom, p.seed, static_cast<uint64_t>(a + j))
                                          : CRIT;
            const uint32_t nq = (L + 3u) >> 2;
            fit_tests += L;

            constexpr bool kSeg = CRIT != kBF;          // segment maxima kept up to date
            const uint32_t nseg = (L + 127u) >> 7;
            S key;
            if (c == kBF) key = use_idx ? seg_bf(nseg, wj) : scan_bf(nq, wj);
            else if (c == kWF) key = seg_wf(nseg);
            else key = seg_ff(nseg, wj);
            key = Tr::warp_min(key);
            if constexpr (G > 1) {
                if (lane == 0) red[par + warp] = key;
                sync();
                key = Tr::warp_min(red[par + (lane % G)]);
                par ^= G;
            } else {
                __syncwarp();
            }

            // decode the winning slot (uniform across the group)
            bool hit;
            uint32_t b;
            uint64_t r_old;
            if (c == kFF) {
                hit = key != Tr::kNone;
                b = static_cast<uint32_t>(key >> kShift);
                r_old = static_cast<uint64_t>(key & Tr::kLo);
            } else if (c == kBF) {
                hit = key < Tr::kSign;
                b = static_cast<uint32_t>(key & Tr::kLo);
                r_old = static_cast<uint64_t>(key >> kShift) + wj;
            } else {
                r_old = static_cast<uint64_t>(Tr::kLo - (key >> kShift));
                hit = r_old >= wj;
                b = static_cast<uint32_t>(key & Tr::kLo);
            }
            uint32_t t;
            if (hit) {
                t = typ[b];
            } else {                           // nothing fits: smallest type holding w
                t = 31u - static_cast<uint32_t>(__clz(__ballot_sync(kFull, Bl >= wj)));
                b = L;
            }
            const uint64_t Bt = __shfl_sync(kFull, Bl, static_cast<int>(t));
            if (!hit) r_old = Bt;
            const uint64_t r_new = r_old - wj;
            // Rule 5: 2*load_before < B_t <= 2*load_after, in residual terms
            // (with Remark 3's per-type condition when asked for)
            const bool cross = (Bt < 2 * r_old) && (2 * r_new <= Bt);
            const bool fire = p.remark3 ? remark3_divide(below, Bl, !hit, Bt, cross) : cross;
            if (tid == static_cast<int>(owner(b))) {
                if (hit) slots[b] = (static_cast<S>(r_new) << kShift) | static_cast<S>(b);
                else put_new(b, r_new, t);
            }
            uint32_t Ln = L + (hit ? 0u : 1u);
            if (fire) {
                if (tid == static_cast<int>(owner(Ln))) put_new(Ln, Bt, t);
                ++Ln;
            }
            if (kSeg || use_idx) {                     // summaries of the touched segments
                const uint32_t sb = b >> 7, sf = (Ln - 1u) >> 7;
                const uint32_t nseg_after = (Ln + 127u) >> 7;
                const bool same = fire && sf == sb;
                seg_update(sb, kSeg, use_idx, nseg_after, hit ? static_cast<int64_t>(r_old) : -1,
                           static_cast<uint32_t>(r_new), same ? static_cast<uint32_t>(Bt) : 0u);
                if (fire && !same)
                    seg_update(sf, kSeg, use_idx, nseg_after, -1, static_cast<uint32_t>(Bt), 0u);
            }
            if (tid == 0) raw[j] = static_cast<int32_t>(b);
            L = Ln;
            if (++jc == chunk) {
                jc = 0;
                buf ^= 1;
            }
        }
        L_io = L;
        return true;
    }

    // One-warp item loop (G == 1) driven entirely by the summaries: segment
    // maxima for FF/WF items and the residual index for BF items.  The chain
    // per item is short: each lane prepares its candidate's commit data (type,
    // capacity) while the warp reduction runs, the winning lane -- the one that
    // scanned the chosen bin -- writes, and the chosen segment's summaries are
    // updated from the quad already in registers.  With one warp the owner rule
    // is not needed; __syncwarp orders the writes before the next item.
    template <int CRIT>
    __device__ __forceinline__ bool item_loop_warp(const H1Params& p, int64_t i, const int32_t* w,
                                                   int64_t a, int64_t k, int32_t* raw, uint32_t Bl,
                                                   bool B1_indexed, uint32_t& L_io,
                                                   unsigned long long& fit_tests, uint32_t& below) const {
        constexpr bool kSeg = CRIT != kBF;                        // FF or WF items occur
        constexpr bool kIdx = CRIT == kBF || CRIT == kRandom;     // BF items occur
        const int chunk = p.chunk;
        const uint32_t* wb = wbits;
        uint32_t L = L_io;
        int jc = 0, buf = 0;
        for (int64_t j = 0; j < k; ++j) {
            if (jc == 0) {
                cp_async_wait_all();
                __syncwarp();
                if (j + chunk < k) load_chunk(w, j + chunk, k, buf ^ 1, chunk);
            }
            if (p.spill_list && L + 2u > static_cast<uint32_t>(p.slot_cap)) {
                cp_async_wait_all();
                if (lane == 0) {
                    const unsigned long long pos = atomicAdd(
                        reinterpret_cast<unsigned long long*>(p.spill_seg + 1), 1ull);
                    p.spill_list[pos] = static_cast<int32_t>(i);
                }
                __syncwarp();
                return false;
            }
            const uint32_t wj = static_cast<uint32_t>(wst[buf * chunk + jc]);
            const int c = CRIT == kRandom ? pick_criterion(kRandom, p.seed, static_cast<uint64_t>(a + j))
                                          : CRIT;
            fit_tests += L;
            const uint32_t nseg = (L + 127u) >> 7;

            // 1. the segment that holds the answer (uniform), or none
            int sf = -1;
            if (c == kFF) {
                for (uint32_t k0 = 0; k0 < nseg; k0 += 32) {
                    const uint32_t sl = k0 + static_cast<uint32_t>(lane);
                    const unsigned bal = __ballot_sync(kFull, sl < nseg && segmax[sl] >= wj);
                    if (bal) { sf = static_cast<int>(k0) + __ffs(bal) - 1; break; }
                }
            } else if (c == kWF) {
                uint32_t mx = 0;
                for (uint32_t sl = static_cast<uint32_t>(lane); sl < nseg; sl += 32) mx = max(mx, segmax[sl]);
                mx = __reduce_max_sync(kFull, mx);
                if (mx >= wj) {
                    for (uint32_t k0 = 0; k0 < nseg; k0 += 32) {
                        const uint32_t sl = k0 + static_cast<uint32_t>(lane);
                        const unsigned bal = __ballot_sync(kFull, sl < nseg && segmax[sl] == mx);
                        if (bal) { sf = static_cast<int>(k0) + __ffs(bal) - 1; break; }
                    }
                }
            } else {
                uint32_t word = wb[lane];
                const uint32_t wi = wj >> 5;
                if (static_cast<uint32_t>(lane) < wi) word = 0u;
                else if (static_cast<uint32_t>(lane) == wi) word &= ~((1u << (wj & 31)) - 1u);
                const unsigned bal = __ballot_sync(kFull, word != 0u);
                if (bal) {
                    const int src = __ffs(bal) - 1;
                    const uint32_t rs = static_cast<uint32_t>(src) * 32u +
                                        static_cast<uint32_t>(__ffs(__shfl_sync(kFull, word, src)) - 1);
                    const uint32_t* row = segres + (rs >> 5) * nsegcap;
                    const uint32_t rbit = 1u << (rs & 31);
                    for (uint32_t k0 = 0; k0 < nseg; k0 += 32) {
                        const uint32_t sl = k0 + static_cast<uint32_t>(lane);
                        const unsigned b2 = __ballot_sync(kFull, sl < nseg && (row[sl] & rbit));
                        if (b2) { sf = static_cast<int>(k0) + __ffs(b2) - 1; break; }
                    }
                }
            }

            // 2. scan that segment; decode the winner
            const bool hit = sf >= 0;
            const S W = static_cast<S>(wj) << kShift;
            S q0 = 0, q1 = 0, q2 = 0, q3 = 0;
            uint32_t b, r_old, t, Bt;
            int winner = 0;
            if (hit) {
                Tr::load_quad(slots, 32u * static_cast<uint32_t>(sf) + static_cast<uint32_t>(lane), q0, q1, q2, q3);
                S kl;
                if (c == kFF) {
                    kl = Tr::kNone;
                    if (q3 >= W) kl = ff_key(q3);
                    if (q2 >= W) kl = ff_key(q2);
                    if (q1 >= W) kl = ff_key(q1);
                    if (q0 >= W) kl = ff_key(q0);
                } else if (c == kWF) {
                    kl = min(min(q0 ^ Tr::kHi, q1 ^ Tr::kHi), min(q2 ^ Tr::kHi, q3 ^ Tr::kHi));
                } else {
                    kl = min(min(q0 - W, q1 - W), min(q2 - W, q3 - W));
                }
                // this lane's candidate bin: its type and capacity, fetched
                // while the reduction runs
                const uint32_t bl = c == kFF ? static_cast<uint32_t>(kl >> kShift)
                                             : static_cast<uint32_t>(kl & Tr::kLo);
                uint32_t tl = 0;
                if (kl != Tr::kNone) tl = typ[bl];     // a lane without a candidate reads nothing
                const uint32_t Btl = __shfl_sync(kFull, Bl, static_cast<int>(tl));
                const S key = Tr::warp_min(kl);
                if (c == kFF) {
                    b = static_cast<uint32_t>(key >> kShift);
                    r_old = static_cast<uint32_t>(key & Tr::kLo);
                } else if (c == kBF) {
                    b = static_cast<uint32_t>(key & Tr::kLo);
                    r_old = static_cast<uint32_t>(key >> kShift) + wj;
                } else {
                    b = static_cast<uint32_t>(key & Tr::kLo);
                    r_old = static_cast<uint32_t>(Tr::kLo - (key >> kShift));
                }
                winner = static_cast<int>((b >> 2) & 31u);
                t = __shfl_sync(kFull, tl, winner);
                Bt = __shfl_sync(kFull, Btl, winner);
            } else {                                   // nothing fits: smallest type holding w
                t = 31u - static_cast<uint32_t>(__clz(__ballot_sync(kFull, Bl >= wj)));
                Bt = __shfl_sync(kFull, Bl, static_cast<int>(t));
                b = L;
                r_old = Bt;
            }
            const uint32_t r_new = r_old - wj;
            const bool cross = (static_cast<uint64_t>(Bt) < 2ull * r_old) &&
                               (2ull * r_new <= static_cast<uint64_t>(Bt));       // Rule 5
            const bool fire = p.remark3 ? remark3_divide(below, Bl, !hit, Bt, cross) : cross;
            const uint32_t Lf = hit ? L : L + 1u;         // where a divided-off bin goes
            if (lane == winner) {
                slots[b] = (static_cast<S>(r_new) << kShift) | static_cast<S>(b);
                if (!hit) typ[b] = static_cast<uint8_t>(t);
                if (fire) {
                    slots[Lf] = (static_cast<S>(Bt) << kShift) | static_cast<S>(Lf);
                    typ[Lf] = static_cast<uint8_t>(t);
                }
                raw[j] = static_cast<int32_t>(b);
            }

            // 3. summaries of the touched segments
            const uint32_t sb = b >> 7, sfire = Lf >> 7;
            if constexpr (kSeg) {
                if (hit) {
                    // new maximum of segment sb from the quad in registers
                    const S ns = (static_cast<S>(r_new) << kShift) | static_cast<S>(b);
                    S x0 = q0, x1 = q1, x2 = q2, x3 = q3;
                    if (lane == winner) {
                        const uint32_t pos = b & 3u;
                        x0 = pos == 0 ? ns : x0; x1 = pos == 1 ? ns : x1;
                        x2 = pos == 2 ? ns : x2; x3 = pos == 3 ? ns : x3;
                    }
                    uint32_t top = static_cast<uint32_t>(max(max(x0, x1), max(x2, x3)) >> kShift);
                    top = __reduce_max_sync(kFull, top);
                    if (fire && sfire == sb) top = max(top, Bt);
                    if (lane == 0) segmax[sb] = top;
                } else if (lane == 0) {
                    segmax[sb] = max(segmax[sb], r_new);
                    if (fire && sfire == sb) segmax[sb] = max(segmax[sb], Bt);
                }
                if (fire && sfire != sb && lane == 0) segmax[sfire] = max(segmax[sfire], Bt);
            }
            if constexpr (kIdx) {
                if (hit && B1_indexed) {
                    // does segment sb still hold r_old after the update?
                    const S Ro = static_cast<S>(r_old);
                    const uint32_t pos = (lane == winner) ? (b & 3u) : 4u;
                    const bool here = ((q0 >> kShift) == Ro && pos != 0) || ((q1 >> kShift) == Ro && pos != 1) ||
                                      ((q2 >> kShift) == Ro && pos != 2) || ((q3 >> kShift) == Ro && pos != 3);
                    if (!__any_sync(kFull, here)) {
                        uint32_t* row = segres + (r_old >> 5) * nsegcap;
                        const uint32_t rbit = 1u << (r_old & 31);
                        if (lane == 0) row[sb] &= ~rbit;
                        __syncwarp();
                        bool any = false;
                        for (uint32_t sl = static_cast<uint32_t>(lane); sl < nseg; sl += 32) any |= (row[sl] & rbit) != 0u;
                        if (!__any_sync(kFull, any) && lane == 0) wbits[r_old >> 5] &= ~rbit;
                    }
                }
                if (B1_indexed && lane == 0) {
                    if (r_new > 0u) {
                        segres[(r_new >> 5) * nsegcap + sb] |= 1u << (r_new & 31);
                        wbits[r_new >> 5] |= 1u << (r_new & 31);
                    }
                    if (fire) {
                        segres[(Bt >> 5) * nsegcap + sfire] |= 1u << (Bt & 31);
                        wbits[Bt >> 5] |= 1u << (Bt & 31);
                    }
                }
            }
            __syncwarp();
            L += (hit ? 0u : 1u) + (fire ? 1u : 0u);
            if (++jc == chunk) {
                jc = 0;
                buf ^= 1;
            }
        }
        L_io = L;
        return true;
    }

    // Pack one unit; called by all T threads of the group with identical args.
    __device__ void pack_unit(const H1Params& p, int64_t uid) const {
        const int64_t i = p.units.instance_of(uid, p.in.N);
        if (p.out.status[i] != VSBPP_OK) return;        // rejected by validation
        if (p.cls && p.cls[i] != p.want_cls) return;
        const int64_t m = p.in.m(i);
        int64_t a = 0, k = m;
        if (p.units.unit_base) {
            const int64_t g = uid - p.units.unit_base[i];
            a = g * p.units.sublist;
            k = (m - a) < p.units.sublist ? (m - a) : p.units.sublist;
        }
        const int64_t wb = p.in.w_begin(i);
        const int32_t* w = p.in.w_all + wb + a;
        const int32_t n = p.in.n(i);
        const int32_t* B = p.in.B_all + p.in.B_begin(i);
        const uint32_t Bl = lane < n ? static_cast<uint32_t>(B[lane]) : 0u;
        if (warp == 0) Bs[lane] = Bl;
        int32_t* raw = p.out.bin_of_item + wb + a;
        int32_t* types_out = p.compose ? (p.out.local_types + wb + a) : (p.out.bin_type + wb);
        const int chunk = p.chunk;

        const bool use_seg = p.criterion != kBF;
        const bool use_idx = p.bf_index && (p.criterion == kBF || p.criterion == kRandom) &&
                             __shfl_sync(kFull, Bl, 0) <= static_cast<uint32_t>(kIndexMaxRes);
        if (use_seg || use_idx) {
            // Segment reads cover whole 128-bin segments, so every slot must
            // read as empty until its bin exists: each thread clears its own
            // quads, each warp its own segment summaries.
            for (uint32_t q = static_cast<uint32_t>(tid); q < static_cast<uint32_t>(p.slot_cap) / 4u; q += T)
                Tr::store_quad(slots, q, S(0), S(0), S(0), S(0));
            const uint32_t nseg = static_cast<uint32_t>(p.slot_cap) / 128u;
            for (uint32_t sg = static_cast<uint32_t>(warp); sg < nseg; sg += G) {
                if (use_seg && lane == 0) segmax[sg] = 0u;
                if (use_idx) segres[lane * nsegcap + sg] = 0u;
            }
            if (use_idx) wbits[warp * 32 + lane] = 0u;
            __syncwarp();
        }
        uint32_t L = 0;
        if (p.preopen) {                     // literal Rule 2: one empty bin per type
            for (int t = 0; t < n; ++t) {
                if (tid == static_cast<int>(owner(static_cast<uint32_t>(t))))
                    put_new(static_cast<uint32_t>(t), static_cast<uint32_t>(B[t]), static_cast<uint32_t>(t));
            }
            L = static_cast<uint32_t>(n);
            // n <= 32 bins, all in segment 0 (warp 0's): enter them in its summaries
            if (warp == 0 && (use_seg || use_idx)) {
                __syncwarp();
                if (use_seg && lane == 0) segmax[0] = static_cast<uint32_t>(B[0]);
                if (use_idx) {
                    const uint32_t r = lane < n ? static_cast<uint32_t>(B[lane]) : 0u;
                    if (r > 0u) {
                        atomicOr(&segres[(r >> 5) * nsegcap], 1u << (r & 31));   // segment 0
                        atomicOr(&wbits[r >> 5], 1u << (r & 31));
                    }
                }
                __syncwarp();
            }
        }
        if (k > 0) load_chunk(w, 0, k, 0, chunk);
        unsigned long long fit_tests = 0;      // live bins summed over items (counters)
        // Remark 3: type-t bins below half in lane t (the pre-opened empties)
        uint32_t below = (p.preopen && lane < n) ? 1u : 0u;
        bool done;
        if constexpr (G == 1) {
            // one warp: the summary-driven loop whenever every criterion it
            // meets has its summaries (BF needs the residual index)
            if (p.criterion != kBF && p.criterion != kRandom) {
                done = p.criterion == kFF ? item_loop_warp<kFF>(p, i, w, a, k, raw, Bl, use_idx, L, fit_tests, below)
                                          : item_loop_warp<kWF>(p, i, w, a, k, raw, Bl, use_idx, L, fit_tests, below);
                goto packed;
            }
            if (use_idx) {
                done = p.criterion == kBF ? item_loop_warp<kBF>(p, i, w, a, k, raw, Bl, use_idx, L, fit_tests, below)
                                          : item_loop_warp<kRandom>(p, i, w, a, k, raw, Bl, use_idx, L, fit_tests, below);
                goto packed;
            }
        }
        switch (p.criterion) {                 // the item loop, specialised per criterion
            case kFF: done = item_loop<kFF>(p, i, w, a, k, raw, Bl, use_idx, L, fit_tests, below); break;
            case kBF: done = item_loop<kBF>(p, i, w, a, k, raw, Bl, use_idx, L, fit_tests, below); break;
            case kWF: done = item_loop<kWF>(p, i, w, a, k, raw, Bl, use_idx, L, fit_tests, below); break;
            default: done = item_loop<kRandom>(p, i, w, a, k, raw, Bl, use_idx, L, fit_tests, below); break;
        }
    packed:
        if (!done) return;                     // spilled: a full-size launch repacks it

        // --- objective (Section 1) and dense ids: used bins in creation order ---
        sync();
        const uint32_t per = (L + T - 1) / T;
        uint32_t b0 = static_cast<uint32_t>(tid) * per;
        if (b0 > L) b0 = L;
        const uint32_t b1 = (b0 + per) < L ? (b0 + per) : L;
        uint32_t cnt = 0;
        for (uint32_t b = b0; b < b1; ++b)
            cnt += static_cast<uint32_t>((slots[b] >> kShift) < static_cast<S>(Bs[typ[b]]));
        uint32_t excl = warp_exclusive_scan(cnt, lane);
        uint32_t used_total = __shfl_sync(kFull, excl + cnt, 31);
        if constexpr (G > 1) {
            uint32_t* wsum = reinterpret_cast<uint32_t*>(xch);
            if (lane == 31) wsum[warp] = excl + cnt;
            sync();
            uint32_t pre = 0, all = 0;
            for (int x = 0; x < G; ++x) {
                const uint32_t v = wsum[x];
                pre += x < warp ? v : 0u;
                all += v;
            }
            excl += pre;
            used_total = all;
        }
        uint32_t d = excl;
        uint64_t tot = 0;
        for (uint32_t b = b0; b < b1; ++b) {
            const S s = slots[b];
            const uint32_t t = typ[b];
            const uint32_t cap = Bs[t];
            if ((s >> kShift) < static_cast<S>(cap)) {
                slots[b] = ((s >> kShift) << kShift) | static_cast<S>(d);
                types_out[d] = static_cast<int32_t>(t);
                tot += cap;
                ++d;
            }
        }
        sync();
        for (int64_t j = tid; j < k; j += T)
            raw[j] = static_cast<int32_t>(slots[static_cast<uint32_t>(raw[j])] & Tr::kLo);
        tot = warp_sum_u64(tot);
        if constexpr (G > 1) {
            // xch held the warp counts of the scan above; every read of them
            // happened before the barrier that precedes the remap.
            if (lane == 0) xch[warp] = tot;
            sync();
            if (tid == 0) {
                uint64_t s = 0;
                for (int x = 0; x < G; ++x) s += xch[x];
                tot = s;
            }
        }
        if (tid == 0) {
            if (p.counters) {
                atomicAdd(p.counters, static_cast<unsigned long long>(k));
                atomicAdd(p.counters + 1, fit_tests);
            }
            if (p.compose) {
                p.out.unit_count[uid] = static_cast<int32_t>(used_total);
                p.out.unit_total[uid] = static_cast<int64_t>(tot);
            } else {
                p.out.num_bins[i] = static_cast<int64_t>(used_total);
                p.out.total[i] = static_cast<int64_t>(tot);
            }
        }
        sync();                                 // shared memory is reused by the next unit
    }
};

template <int G, int GROUPS, typename S>
__global__ void __launch_bounds__(32 * G * GROUPS)
h1_pack_kernel(const H1Params p) {
    extern __shared__ __align__(16) unsigned char smem[];
    using Grp = H1Group<G, GROUPS, S>;
    Grp g;
    g.gid = static_cast<int>(threadIdx.x) / Grp::T;
    g.tid = static_cast<int>(threadIdx.x) % Grp::T;
    g.lane = g.tid & 31;
    g.warp = g.tid >> 5;
    unsigned char* base = smem + static_cast<size_t>(g.gid) * static_cast<size_t>(p.group_bytes);
    g.slots = reinterpret_cast<S*>(base);
    base += h1_align16(p.slot_cap * static_cast<int>(sizeof(S)));
    g.typ = base;
    base += h1_align16(p.slot_cap);
    g.segmax = reinterpret_cast<uint32_t*>(base);
    base += h1_align16(4 * ((p.slot_cap + 127) / 128));
    g.segres = reinterpret_cast<uint32_t*>(base);
    g.nsegcap = static_cast<uint32_t>((p.slot_cap + 127) / 128);
    g.wbits = g.segres + g.nsegcap * 32;
    if (p.bf_index) base += ((p.slot_cap + 127) / 128) * 128 + G * 128;
    g.wst = reinterpret_cast<int32_t*>(base);
    base += 2 * p.chunk * 4;
    g.Bs = reinterpret_cast<uint32_t*>(base);
    base += kMaxTypes * 4;
    g.red = reinterpret_cast<S*>(base);
    base += 2 * 32 * sizeof(S);
    g.xch = reinterpret_cast<uint64_t*>(base);
    base += 32 * 8;
    g.bcast = reinterpret_cast<long long*>(base);

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

    if (p.queue) {
        for (int iter = 0;; ++iter) {
            long long u;
            if constexpr (G == 1) {
                unsigned long long v = 0;
                if (g.lane == 0) v = atomicAdd(p.queue, 1ull);
                u = static_cast<long long>(__shfl_sync(kFull, v, 0));
            } else {
                if (g.tid == 0) g.bcast[iter & 1] = static_cast<long long>(atomicAdd(p.queue, 1ull));
                g.sync();
                u = g.bcast[iter & 1];
            }
            if (u >= count) break;
            const int64_t uid = p.order ? static_cast<int64_t>(p.order[begin + u]) : begin + u;
            g.pack_unit(p, uid);
        }
    } else {
        const int64_t first = static_cast<int64_t>(blockIdx.x) * GROUPS + g.gid;
        const int64_t stride = static_cast<int64_t>(gridDim.x) * GROUPS;
        for (int64_t u = first; u < count; u += stride) {
            const int64_t uid = p.order ? static_cast<int64_t>(p.order[begin + u]) : begin + u;
            g.pack_unit(p, uid);
        }
    }
}

}  // namespace vsbpp
