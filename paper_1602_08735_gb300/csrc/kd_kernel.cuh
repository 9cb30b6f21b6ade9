// kd_kernel.cuh -- the first heuristic of Section 6.3 for membrane systems of
// hundreds of thousands of bins, with the bins held on chip in the shared
// memory of a two-CTA thread-block cluster.
//
// Same method as every first-heuristic kernel (Rules 2-6: items in list
// order, fit test residual >= w, FF / BF / WF with the lowest creation index
// winning ties, a bin of the smallest type holding the item when nothing
// fits, the Rule 5 division when a bin's load first reaches half its
// capacity); the flat scan's answer is found exactly through summaries:
//
//   slot       16 bits per bin, (residual << 5) | type (B_1 <= 2047, n <= 32);
//              the bin's creation index is its position.  Bins 0.. live in
//              CTA 0's shared memory, the next ones in CTA 1's (read and
//              written through distributed shared memory), the rest in a
//              global-memory overflow area; a system past 2^19 bins goes to
//              the global-memory kernel from the start.
//   segment    512 bins (1 KB), made of four 128-bin sub-segments (8 bytes,
//              four slots, per lane).
//   maxima     (FF and WF items) the largest residual of every sub-segment
//              in shared memory, of every tile of 32 sub-segments in
//              registers (tile l + 32q in lane l).  FF: one warp minimum over
//              (tile, maximum) keys of the tiles whose maximum is >= w, one
//              over the tile's sub-segments; WF: one warp maximum over
//              (maximum, -tile) keys, one minimum over the tile's
//              sub-segments holding that maximum.
//   presence   (BF items, B_1 <= 1023) the residuals present, one 32-bit word
//              per lane in registers; row r in shared memory: one bit per
//              segment holding a bin of residual r.  r* = the least present
//              residual >= w (one warp minimum), then the first segment in row
//              r* (one more): no bin anywhere has a residual in [w, r*), so
//              the first bin of residual r* there is the flat scan's answer.
//
// In the chosen sub-segment (FF, WF) or segment (BF) each lane turns its
// matching slots into (position, slot) keys, and one warp minimum names the
// bin with its residual and type.  The chain per item is straight-line
// arithmetic and warp reductions.  In the FF, BF and WF kernels each slot is
// stored by the lane that reads it, the maximum of sub-segment G by lane
// G % 32 and word q of every presence row by lane q (the BF bitmaps run from
// the top bit down, so a count of leading zeros finds a word's least
// member), so an item needs no barrier; every segment a system can reach is
// cleared when it starts.  The RANDOM kernel, whose items mix the three,
// clears a segment when a bin opens it and orders an item's stores before the
// next item's reads by __syncwarp.  CTA 1's warp only lends its shared
// memory: it waits at the closing cluster barrier.
#pragma once

#include <cooperative_groups.h>

#include "kd_params.cuh"

namespace vsbpp {

namespace cg = cooperative_groups;

struct KDMem {
    unsigned char* bins0;    // CTA 0's segments
    unsigned char* bins1;    // CTA 1's segments (distributed shared memory)
    unsigned char* over;     // global-memory overflow of this cluster
    uint32_t segs0, segs1;

    __device__ __forceinline__ unsigned char* seg(uint32_t S) const {
        if (S < segs0) return bins0 + static_cast<size_t>(S) * kKDSegBytes;
        S -= segs0;
        if (S < segs1) return bins1 + static_cast<size_t>(S) * kKDSegBytes;
        return over + static_cast<size_t>(S - segs1) * kKDSegBytes;
    }
    __device__ __forceinline__ uint16_t* slot(uint32_t b) const {
        return reinterpret_cast<uint16_t*>(seg(b >> 9)) + (b & 511u);
    }
    // the lane's four slots of sub-segment G
    __device__ __forceinline__ uint2 sub(uint32_t G, uint32_t lane) const {
        return reinterpret_cast<const uint2*>(seg(G >> 2) + (G & 3u) * 256u)[lane];
    }
    // a segment reads as empty (residual 0 fits nothing) until its bins exist
    __device__ __forceinline__ void zero(uint32_t S, uint32_t lane) const {
        uint4* q = reinterpret_cast<uint4*>(seg(S));
        q[lane] = make_uint4(0u, 0u, 0u, 0u);
        q[32 + lane] = make_uint4(0u, 0u, 0u, 0u);
    }
    // the same, each lane clearing the bytes it reads (its 8 bytes of every
    // sub-segment): no barrier is needed before its own reads
    __device__ __forceinline__ void zero_own(uint32_t S, uint32_t lane) const {
        unsigned char* q = seg(S);
#pragma unroll
        for (int k = 0; k < 4; ++k) reinterpret_cast<uint2*>(q + 256 * k)[lane] = make_uint2(0u, 0u);
    }
};

// Bit of member x in its 32-bit word of a bitmap: from the top down in the BF
// kernel (a count of leading zeros then finds a word's least member), from
// the bottom up otherwise.
template <bool TOP>
__device__ __forceinline__ uint32_t kd_bit(uint32_t x) {
    return TOP ? 0x80000000u >> (x & 31u) : 1u << (x & 31u);
}

// slot c (0..3) of a lane's 8 bytes
__device__ __forceinline__ uint32_t kd_half(uint2 v, int c) {
    const uint32_t x = c < 2 ? v.x : v.y;
    return (c & 1) ? (x >> 16) : (x & 0xFFFFu);
}

template <int CRIT>
__global__ void __launch_bounds__(32) kd_pack_kernel(const KDParams p) {
    constexpr bool kSeg = CRIT != kBF;                    // FF or WF items occur
    constexpr bool kIdx = CRIT == kBF || CRIT == kRandom;  // BF items occur
    constexpr bool kTop = CRIT == kBF;                    // bitmaps from the top bit down
    constexpr uint32_t kNo = 0xFFFFFFFFu;
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cluster = cg::this_cluster();
    cluster.sync();                                   // both CTAs are running
    if (cluster.block_rank() != 0) {
        cluster.sync();                               // CTA 1 lends its memory until CTA 0 is done
        return;
    }
    const uint32_t lane = threadIdx.x & 31u;
    uint16_t* submax = reinterpret_cast<uint16_t*>(smem + kKDOffSubmax);
    uint32_t* Bs = reinterpret_cast<uint32_t*>(smem + kKDOffBs);
    uint32_t* pres = reinterpret_cast<uint32_t*>(smem + kKDOffPres);
    KDMem M;
    M.bins0 = smem + kd_bins_offset(p.max_B1, p.pres);
    M.bins1 = cluster.map_shared_rank(smem, 1);
    const uint32_t cid = blockIdx.x >> 1;
    M.over = reinterpret_cast<unsigned char*>(p.over + static_cast<size_t>(cid) * static_cast<size_t>(p.over_bins));
    M.segs0 = static_cast<uint32_t>(p.segs0);
    M.segs1 = static_cast<uint32_t>(p.segs1);
    int32_t* dense = p.dense + static_cast<size_t>(cid) * kKDMaxBins;
    const unsigned lt = (1u << lane) - 1u;

    const int64_t begin = p.seg[p.segment], end = p.seg[p.segment + 1];
    for (;;) {
        unsigned long long v = 0;
        if (lane == 0) v = atomicAdd(p.queue, 1ull);
        const int64_t u = static_cast<int64_t>(__shfl_sync(kFull, v, 0));
        if (u >= end - begin) break;
        const int64_t i = p.order[begin + u];
        if (p.out.status[i] != VSBPP_OK) continue;
        const int64_t m = p.in.m(i);
        const int64_t wb = p.in.w_begin(i);
        const int32_t* w = p.in.w_all + wb;
        const int32_t n = p.in.n(i);
        const int32_t* B = p.in.B_all + p.in.B_begin(i);
        const uint32_t Bl = lane < static_cast<uint32_t>(n) ? static_cast<uint32_t>(B[lane]) : 0u;
        const uint32_t B1 = __shfl_sync(kFull, Bl, 0);
        if (B1 > static_cast<uint32_t>(kIdx ? p.max_B1 : kKDMaxB1)) {
            // residuals past the slot or presence layout: the global-memory kernel
            if (lane == 0) {
                const unsigned long long pos = atomicAdd(reinterpret_cast<unsigned long long*>(p.spill_seg + 1), 1ull);
                p.spill_list[pos] = static_cast<int32_t>(i);
            }
            continue;
        }
        Bs[lane] = Bl;
        uint32_t tm[4] = {0u, 0u, 0u, 0u};           // tile maxima: tile lane + 32 t
        uint32_t gw = 0u;                            // residuals 32 lane .. 32 lane + 31 present
        if (kSeg)
            for (uint32_t x = lane; x < static_cast<uint32_t>(kKDMaxSubs / 2); x += 32)
                reinterpret_cast<uint32_t*>(submax)[x] = 0u;
        if (kIdx)
            for (uint32_t x = lane; x < (B1 + 1u) * 32u; x += 32) pres[x] = 0u;
        if constexpr (CRIT != kRandom) {
            // every segment the system can reach (at most 2m + n bins) reads
            // as empty from the start, each lane clearing the bytes it reads:
            // no item has to clear a segment it opens
            const int64_t reach = (2 * m + n + kKDSeg - 1) / kKDSeg + 1;
            const uint32_t nseg = static_cast<uint32_t>(min(reach, static_cast<int64_t>(kKDMaxSegs)));
            for (uint32_t S = 0; S < nseg; ++S) M.zero_own(S, lane);
        }
        __syncwarp();
        int32_t* raw = p.out.bin_of_item + wb;

        uint32_t L = 0;
        uint32_t below = 0;                          // Remark 3: type-t bins below half, lane t
        if (p.preopen) {                             // literal Rule 2: one empty bin per type, sub-segment 0
            M.zero(0, lane);
            __syncwarp();
            if (lane < static_cast<uint32_t>(n)) *M.slot(lane) = static_cast<uint16_t>((Bl << 5) | lane);
            if (kSeg) {
                if (lane == 0) submax[0] = static_cast<uint16_t>(B1);
                tm[0] = lane == 0 ? B1 : 0u;
            }
            if (kIdx) {
                if (lane < static_cast<uint32_t>(n)) atomicOr(&pres[Bl * 32u], kd_bit<kTop>(0));
                for (int t = 0; t < n; ++t) {
                    const uint32_t r = __shfl_sync(kFull, Bl, t);
                    gw |= (r >> 5) == lane ? kd_bit<kTop>(r) : 0u;
                }
            }
            below = lane < static_cast<uint32_t>(n) ? 1u : 0u;
            L = static_cast<uint32_t>(n);
            __syncwarp();
        }
        unsigned long long fit_tests = 0;
        bool spilled = false;
        // weights and criteria a 32-item block ahead (lane l: item block + l)
        uint32_t wcur = lane < m ? static_cast<uint32_t>(__ldg(w + lane)) : 0u;
        int ccur = pick_criterion(p.criterion, p.seed, static_cast<uint64_t>(lane));
        for (int64_t j0 = 0; j0 < m; j0 += 32) {
            if (L + 64u > static_cast<uint32_t>(kKDMaxBins)) {
                // past 2^19 bins: the global-memory kernel packs it from the start
                if (lane == 0) {
                    const unsigned long long pos =
                        atomicAdd(reinterpret_cast<unsigned long long*>(p.spill_seg + 1), 1ull);
                    p.spill_list[pos] = static_cast<int32_t>(i);
                }
                spilled = true;
                break;
            }
            const int64_t jn = j0 + 32 + lane;
            const uint32_t wnext = jn < m ? static_cast<uint32_t>(__ldg(w + jn)) : 0u;
            const int cnext = pick_criterion(p.criterion, p.seed, static_cast<uint64_t>(jn));
            const int cnt = static_cast<int>(min(static_cast<int64_t>(32), m - j0));
            uint32_t bout = 0, fit_blk = 0;          // fit tests of this block (< 2^24)
            // the block adds at most 64 bins (L + 64 <= 2^19 here), so a new
            // or divided-off bin lies in segment s0 or s0 + 1
            const uint32_t s0 = L >> 9;
            uint16_t* const tail0 = reinterpret_cast<uint16_t*>(M.seg(s0));
            uint16_t* const tail1 = reinterpret_cast<uint16_t*>(M.seg(s0 + 1u));
            for (int jj = 0; jj < cnt; ++jj) {
              if constexpr (CRIT == kBF) {
                // BF items only: straight-line, no barrier.  Every slot is
                // stored by the lane that reads it (the lane holding bins
                // 4l..4l+3 of each sub-segment), word q of every presence row
                // by lane q, and a lane reads nothing else.
                const uint32_t wj = __shfl_sync(kFull, wcur, jj);
                fit_blk += L;
                // 1. r* = the least residual >= w present (residual r is bit
                //    31 - (r & 31) of lane r / 32's word)
                const uint32_t wi = wj >> 5;
                const uint32_t mw = gw & (lane < wi ? 0u : lane == wi ? (kNo >> (wj & 31)) : kNo);
                const uint32_t R = __reduce_min_sync(kFull, mw ? 32u * lane + static_cast<uint32_t>(__clz(mw)) : kNo);
                const bool hit = R != kNo;
                // the first segment of row r* and the bins at r* in it; with
                // nothing fitting, row 0 (never set) and segment 0 are read and
                // the results go unused (a segment index is kept below 2^10,
                // the overflow area's reach, whatever the row holds)
                const uint32_t Rc = hit ? R : 0u;
                const uint32_t rowv = pres[Rc * 32u + lane];
                uint32_t S = __reduce_min_sync(kFull, rowv ? 32u * lane + static_cast<uint32_t>(__clz(rowv)) : kNo);
                S = (hit && S < static_cast<uint32_t>(kKDMaxSegs)) ? S : 0u;
                const unsigned char* base = M.seg(S);
                uint2 v[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) v[k] = reinterpret_cast<const uint2*>(base + 256 * k)[lane];
                // the lane's 16 slots of S as 8 words of two: a half matches r*
                // when its residual bits equal r*'s; adding 0x7FFF to the
                // masked difference sets bit 15 (31) exactly when the low
                // (high) half differs (residuals <= 1023 leave bit 15 clear)
                const uint32_t R5 = Rc << 5, RR = R5 | (R5 << 16);
                uint32_t xw[8];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    xw[2 * k] = v[k].x;
                    xw[2 * k + 1] = v[k].y;
                }
                uint32_t mm = 0;                     // word q's low half at bit q, high half at bit 16 + q
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const uint32_t u = ((xw[q] ^ RR) & 0x7FE07FE0u) + 0x7FFF7FFFu;
                    mm |= (~u >> (15 - q)) & (0x00010001u << q);
                }
                // the lane's first match: the least 2 * word + half
                const uint32_t mlo = mm & 0xFFu, mhi = mm >> 16;
                const uint32_t vlo = mlo ? 2u * static_cast<uint32_t>(__ffs(mlo) - 1) : 64u;
                const uint32_t vhi = mhi ? 2u * static_cast<uint32_t>(__ffs(mhi) - 1) + 1u : 64u;
                const uint32_t vv = min(vlo, vhi);
                const uint32_t qw = (vv >> 1) & 7u;
                const uint32_t a0 = (qw & 1u) ? xw[1] : xw[0], a1 = (qw & 1u) ? xw[3] : xw[2];
                const uint32_t a2 = (qw & 1u) ? xw[5] : xw[4], a3 = (qw & 1u) ? xw[7] : xw[6];
                const uint32_t b0 = (qw & 2u) ? a1 : a0, b1 = (qw & 2u) ? a3 : a2;
                const uint32_t cw = (qw & 4u) ? b1 : b0;
                const uint32_t sv = (vv & 1u) ? (cw >> 16) : (cw & 0xFFFFu);
                // position in S: sub-segment vv / 4, slot 4 * lane + vv % 4 in it
                const uint32_t kmin = mm ? (((128u * (vv >> 2) + 4u * lane + (vv & 3u)) << 16) | sv) : kNo;
                // the chosen bin (least position: the flat scan's first bin at
                // r*), the bins at r* in S, and whether r* is in another
                // segment: three collectives issued together
                const uint32_t k3 = __reduce_min_sync(kFull, kmin);
                const uint32_t atR = __reduce_add_sync(kFull, static_cast<uint32_t>(__popc(mm)));
                const uint32_t nw = lane == (S >> 5) ? rowv & ~(0x80000000u >> (S & 31)) : rowv;
                const bool elsewhere = __any_sync(kFull, nw != 0u);
                // nothing fits: a bin of the smallest type holding w
                const uint32_t tyn = 31u - static_cast<uint32_t>(__clz(__ballot_sync(kFull, Bl >= wj)));
                const uint32_t ty = hit ? (k3 & 31u) : tyn;
                const uint32_t b = hit ? S * 512u + ((k3 >> 16) & 511u) : L;
                const uint32_t Bt = __shfl_sync(kFull, Bl, static_cast<int>(ty));
                const uint32_t r_old = hit ? R : Bt;
                const uint32_t r_new = r_old - wj;
                const bool cross = Bt < 2u * r_old && 2u * r_new <= Bt;        // Rule 5
                const bool fire = p.remark3 ? remark3_divide(below, Bl, !hit, Bt, cross) : cross;
                const uint32_t Lf = hit ? L : L + 1u;
                // 2. slots: the chosen bin in S (read above), a new or
                //    divided-off bin in one of the block's tail segments
                uint16_t* const pb = hit ? reinterpret_cast<uint16_t*>(const_cast<unsigned char*>(base))
                                         : ((b >> 9) == s0 ? tail0 : tail1);
                uint16_t* const pf = (Lf >> 9) == s0 ? tail0 : tail1;
                if (lane == ((b & 127u) >> 2)) pb[b & 511u] = static_cast<uint16_t>((r_new << 5) | ty);
                if (fire && lane == ((Lf & 127u) >> 2)) pf[Lf & 511u] = static_cast<uint16_t>((Bt << 5) | ty);
                // 3. presence: r* leaves S when the chosen bin was S's only bin
                //    at r* (and leaves the present set when no other segment
                //    holds it); r_new and a divided-off bin's capacity enter
                const uint32_t Sb = b >> 9, Sf = Lf >> 9;
                const bool leave = hit && atR == 1u;
                if (leave && lane == (S >> 5)) pres[R * 32u + lane] = nw;
                gw &= (leave && !elsewhere && lane == (R >> 5)) ? ~(0x80000000u >> (R & 31)) : kNo;
                if (r_new > 0u && lane == (Sb >> 5)) atomicOr(&pres[r_new * 32u + lane], 0x80000000u >> (Sb & 31));
                gw |= (r_new > 0u && lane == (r_new >> 5)) ? 0x80000000u >> (r_new & 31) : 0u;
                if (fire && lane == (Sf >> 5)) atomicOr(&pres[Bt * 32u + lane], 0x80000000u >> (Sf & 31));
                gw |= (fire && lane == (Bt >> 5)) ? 0x80000000u >> (Bt & 31) : 0u;
                L += (hit ? 0u : 1u) + (fire ? 1u : 0u);
                bout = lane == static_cast<uint32_t>(jj) ? b : bout;
              } else if constexpr (CRIT == kFF || CRIT == kWF) {
                // FF or WF items only: straight-line, no barrier.  Every slot
                // is stored by the lane that reads it, the maximum of
                // sub-segment G by lane G % 32 (the lane that reads it), and a
                // lane reads nothing else.
                const uint32_t wj = __shfl_sync(kFull, wcur, jj);
                fit_blk += L;
                // 1. the tile, then its sub-segment, then the bin (FF: the first
                //    with maximum >= w; WF: the largest maximum, then the first
                //    bin at it); with nothing fitting, sub-segment 0 is read and
                //    the results go unused
                bool hit;
                uint32_t T, Mx = 0u;
                if constexpr (CRIT == kFF) {
                    uint32_t key = kNo;
#pragma unroll
                    for (int t = 3; t >= 0; --t)
                        key = tm[t] >= wj ? ((lane + 32u * t) << 16) | tm[t] : key;
                    key = __reduce_min_sync(kFull, key);
                    hit = key != kNo;
                    T = hit ? (key >> 16) & 127u : 0u;
                } else {
                    uint32_t key = 0u;
#pragma unroll
                    for (int t = 0; t < 4; ++t) key = max(key, (tm[t] << 8) | (127u - (lane + 32u * t)));
                    key = __reduce_max_sync(kFull, key);
                    Mx = key >> 8;
                    hit = Mx >= wj;
                    T = hit ? 127u - (key & 127u) : 0u;
                }
                const uint32_t sv = submax[T * 32u + lane];
                const bool gsel = CRIT == kFF ? sv >= wj : sv == Mx;
                const uint32_t gl = __reduce_min_sync(kFull, gsel ? lane : 32u);
                const uint32_t G = hit ? T * 32u + (gl & 31u) : 0u;
                const unsigned char* gbase = M.seg(G >> 2);
                const uint2 q4 = reinterpret_cast<const uint2*>(gbase + (G & 3u) * 256u)[lane];
                const uint32_t W5 = wj << 5;          // residual >= w  <=>  slot >= w << 5
                uint32_t kk = kNo;
#pragma unroll
                for (int cc = 3; cc >= 0; --cc) {
                    const uint32_t sl4 = kd_half(q4, cc);
                    const bool mt = CRIT == kFF ? sl4 >= W5 : (sl4 >> 5) == Mx;
                    kk = mt ? ((4u * lane + cc) << 16) | sl4 : kk;
                }
                const uint32_t k3 = __reduce_min_sync(kFull, kk);
                // nothing fits: a bin of the smallest type holding w
                const uint32_t tyn = 31u - static_cast<uint32_t>(__clz(__ballot_sync(kFull, Bl >= wj)));
                const uint32_t ty = hit ? (k3 & 31u) : tyn;
                const uint32_t b = hit ? G * 128u + ((k3 >> 16) & 127u) : L;
                const uint32_t Bt = __shfl_sync(kFull, Bl, static_cast<int>(ty));
                const uint32_t r_old = hit ? ((k3 & 0xFFFFu) >> 5) : Bt;
                const uint32_t r_new = r_old - wj;
                const bool cross = Bt < 2u * r_old && 2u * r_new <= Bt;        // Rule 5
                const bool fire = p.remark3 ? remark3_divide(below, Bl, !hit, Bt, cross) : cross;
                const uint32_t Lf = hit ? L : L + 1u;
                // 2. slots: the chosen bin in G's segment, a new or divided-off
                //    bin in one of the block's tail segments
                uint16_t* const pb = hit ? reinterpret_cast<uint16_t*>(const_cast<unsigned char*>(gbase))
                                         : ((b >> 9) == s0 ? tail0 : tail1);
                uint16_t* const pf = (Lf >> 9) == s0 ? tail0 : tail1;
                const uint32_t nsv = (r_new << 5) | ty;
                if (lane == ((b & 127u) >> 2)) pb[b & 511u] = static_cast<uint16_t>(nsv);
                if (fire && lane == ((Lf & 127u) >> 2)) pf[Lf & 511u] = static_cast<uint16_t>((Bt << 5) | ty);
                // 3. sub-segment maxima: G's from its four slots a lane (the
                //    chosen one updated); a new bin's sub-segment from its old
                //    maximum (lane Gb % 32's own word)
                const uint32_t Gb = b >> 7, Gf = Lf >> 7;
                const uint32_t pos = b & 127u;
                uint32_t mx = 0u;
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                    const uint32_t sl4 = (lane == (pos >> 2) && (pos & 3u) == static_cast<uint32_t>(cc)) ? nsv
                                                                                                        : kd_half(q4, cc);
                    mx = max(mx, sl4 >> 5);
                }
                const uint32_t nmh = __reduce_max_sync(kFull, mx);
                const uint32_t rowb = submax[(Gb & ~31u) + lane];
                uint32_t nmb = hit ? nmh : max(rowb, r_new);
                if (fire && Gf == Gb) nmb = max(nmb, Bt);
                if (lane == (Gb & 31u)) submax[Gb] = static_cast<uint16_t>(nmb);
                if (fire && Gf != Gb && lane == (Gf & 31u))
                    submax[Gf] = static_cast<uint16_t>(max(static_cast<uint32_t>(submax[Gf]), Bt));
                // tile maxima from the touched tiles' rows (each lane its own word)
                const uint32_t Tb = Gb >> 5, Tf = Gf >> 5;
                const bool two = fire && Tf != Tb;
                const uint32_t tb = __reduce_max_sync(kFull, static_cast<uint32_t>(submax[Tb * 32u + lane]));
                const uint32_t tf = two ? __reduce_max_sync(kFull, static_cast<uint32_t>(submax[Tf * 32u + lane])) : 0u;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const uint32_t tile = lane + 32u * t;
                    tm[t] = tile == Tb ? tb : tm[t];
                    tm[t] = (two && tile == Tf) ? tf : tm[t];
                }
                L += (hit ? 0u : 1u) + (fire ? 1u : 0u);
                bout = lane == static_cast<uint32_t>(jj) ? b : bout;
              } else {
                const uint32_t wj = __shfl_sync(kFull, wcur, jj);
                const int c = CRIT == kRandom ? __shfl_sync(kFull, ccur, jj) : CRIT;
                fit_blk += L;

                // 1. the chosen bin b and its slot (residual << 5 | type), or none
                bool hit = false;
                uint32_t b = 0, sl = 0;
                uint2 q4 = make_uint2(0u, 0u);        // FF / WF: this lane's slots of sub-segment G
                uint32_t q16[8];                      // BF: this lane's slots of segment S
#pragma unroll
                for (int k = 0; k < 8; ++k) q16[k] = 0u;
                uint32_t rowv = 0u, mcnt = 0u;        // BF: word `lane` of row r*, matches of r* in S
                if (kSeg && c == kFF) {
                    uint32_t key = kNo;
#pragma unroll
                    for (int t = 3; t >= 0; --t)
                        key = tm[t] >= wj ? ((lane + 32u * t) << 16) | tm[t] : key;
                    key = __reduce_min_sync(kFull, key);
                    hit = key != kNo;
                    if (hit) {
                        const uint32_t T = key >> 16;
                        const uint32_t sv = submax[T * 32u + lane];
                        const uint32_t G = T * 32u + __reduce_min_sync(kFull, sv >= wj ? lane : 32u);
                        q4 = M.sub(G, lane);
                        const uint32_t W5 = wj << 5;  // residual >= w  <=>  slot >= w << 5
                        uint32_t k3 = kNo;
#pragma unroll
                        for (int cc = 3; cc >= 0; --cc) {
                            const uint32_t s = kd_half(q4, cc);
                            k3 = s >= W5 ? ((4u * lane + cc) << 16) | s : k3;
                        }
                        k3 = __reduce_min_sync(kFull, k3);
                        b = G * 128u + (k3 >> 16);
                        sl = k3 & 0xFFFFu;
                    }
                } else if (kSeg && c == kWF) {
                    uint32_t key = 0u;
#pragma unroll
                    for (int t = 0; t < 4; ++t) key = max(key, (tm[t] << 8) | (127u - (lane + 32u * t)));
                    key = __reduce_max_sync(kFull, key);
                    const uint32_t Mx = key >> 8;
                    hit = Mx >= wj;
                    if (hit) {
                        const uint32_t T = 127u - (key & 255u);
                        const uint32_t sv = submax[T * 32u + lane];
                        const uint32_t G = T * 32u + __reduce_min_sync(kFull, sv == Mx ? lane : 32u);
                        q4 = M.sub(G, lane);
                        uint32_t k3 = kNo;
#pragma unroll
                        for (int cc = 3; cc >= 0; --cc) {
                            const uint32_t s = kd_half(q4, cc);
                            k3 = (s >> 5) == Mx ? ((4u * lane + cc) << 16) | s : k3;
                        }
                        k3 = __reduce_min_sync(kFull, k3);
                        b = G * 128u + (k3 >> 16);
                        sl = k3 & 0xFFFFu;
                    }
                } else if (kIdx) {
                    const uint32_t wi = wj >> 5;
                    const uint32_t mw = gw & (lane < wi ? 0u : lane == wi ? ~((1u << (wj & 31)) - 1u) : kNo);
                    const uint32_t R = __reduce_min_sync(kFull, mw ? 32u * lane + static_cast<uint32_t>(__ffs(mw) - 1) : kNo);
                    hit = R != kNo;
                    if (hit) {
                        rowv = pres[R * 32u + lane];
                        const uint32_t S = __reduce_min_sync(
                            kFull, rowv ? 32u * lane + static_cast<uint32_t>(__ffs(rowv) - 1) : kNo);
                        const unsigned char* base = M.seg(S);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const uint2 v2 = reinterpret_cast<const uint2*>(base + 256 * k)[lane];
                            q16[2 * k] = v2.x;
                            q16[2 * k + 1] = v2.y;
                        }
                        const uint32_t R5 = R << 5;
                        uint32_t k3 = kNo;
#pragma unroll
                        for (int k = 3; k >= 0; --k) {
#pragma unroll
                            for (int cc = 3; cc >= 0; --cc) {
                                const uint32_t x = q16[2 * k + (cc >> 1)];
                                const uint32_t s = (cc & 1) ? (x >> 16) : (x & 0xFFFFu);
                                const bool hr = (s & 0xFFE0u) == R5;
                                mcnt += hr ? 1u : 0u;
                                k3 = hr ? ((128u * k + 4u * lane + cc) << 16) | s : k3;
                            }
                        }
                        k3 = __reduce_min_sync(kFull, k3);
                        b = S * 512u + (k3 >> 16);
                        sl = k3 & 0xFFFFu;
                    }
                }
                uint32_t r_old, ty;
                if (hit) {
                    r_old = sl >> 5;
                    ty = sl & 31u;
                } else {                              // nothing fits: smallest type holding w
                    ty = 31u - static_cast<uint32_t>(__clz(__ballot_sync(kFull, Bl >= wj)));
                    b = L;
                    r_old = __shfl_sync(kFull, Bl, static_cast<int>(ty));
                }
                const uint32_t Bt = __shfl_sync(kFull, Bl, static_cast<int>(ty));
                const uint32_t r_new = r_old - wj;
                const bool cross = Bt < 2u * r_old && 2u * r_new <= Bt;        // Rule 5
                const bool fire = p.remark3 ? remark3_divide(below, Bl, !hit, Bt, cross) : cross;
                const uint32_t Lf = hit ? L : L + 1u;

                // 2. stores: a segment a new bin opens is cleared first
                if (!hit && (b & 511u) == 0u) M.zero(b >> 9, lane);
                if (fire && (Lf & 511u) == 0u) M.zero(Lf >> 9, lane);
                __syncwarp();
                if (lane == 0) {
                    *M.slot(b) = static_cast<uint16_t>((r_new << 5) | ty);
                    if (fire) *M.slot(Lf) = static_cast<uint16_t>((Bt << 5) | ty);
                }
                __syncwarp();

                // 3. sub-segment and tile maxima (FF / WF items occur)
                if (kSeg) {
                    const uint32_t Gb = b >> 7, Gf = Lf >> 7;
                    const uint32_t nsv = (r_new << 5) | ty;
                    uint32_t nm;
                    if (hit) {
                        // the sub-segment's four slots a lane, the chosen one updated
                        // (a BF item, under RANDOM, holds its segment in q16)
                        const uint32_t pos = b & 127u, k = (b >> 7) & 3u;
                        uint2 v2 = q4;
                        if (c == kBF) {
                            v2.x = k == 0u ? q16[0] : k == 1u ? q16[2] : k == 2u ? q16[4] : q16[6];
                            v2.y = k == 0u ? q16[1] : k == 1u ? q16[3] : k == 2u ? q16[5] : q16[7];
                        }
                        uint32_t mx = 0u;
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc) {
                            const uint32_t s = (lane == (pos >> 2) && (pos & 3u) == static_cast<uint32_t>(cc))
                                                   ? nsv : kd_half(v2, cc);
                            mx = max(mx, s >> 5);
                        }
                        nm = __reduce_max_sync(kFull, mx);
                    } else {
                        nm = max(static_cast<uint32_t>(submax[Gb]), r_new);
                    }
                    if (fire && Gf == Gb) nm = max(nm, Bt);
                    if (lane == 0) {
                        submax[Gb] = static_cast<uint16_t>(nm);
                        if (fire && Gf != Gb) submax[Gf] = static_cast<uint16_t>(max(static_cast<uint32_t>(submax[Gf]), Bt));
                    }
                    __syncwarp();
                    // tile maxima from the touched tiles' rows
                    const uint32_t Tb = Gb >> 5, Tf = Gf >> 5;
                    const bool two = fire && Tf != Tb;
                    const uint32_t tb = __reduce_max_sync(kFull, static_cast<uint32_t>(submax[Tb * 32u + lane]));
                    const uint32_t tf = two ? __reduce_max_sync(kFull, static_cast<uint32_t>(submax[Tf * 32u + lane])) : 0u;
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const uint32_t tile = lane + 32u * t;
                        tm[t] = tile == Tb ? tb : tm[t];
                        tm[t] = (two && tile == Tf) ? tf : tm[t];
                    }
                }

                // 4. residual presence (BF items occur)
                if (kIdx) {
                    const uint32_t Sb = b >> 9, Sf = Lf >> 9;
                    if (hit) {
                        // does segment Sb still hold a bin of residual r_old?  A BF
                        // item counted r* = r_old in the scan (the chosen bin
                        // included); other items count after the store
                        uint32_t cl = mcnt;
                        if (c != kBF) {
                            const unsigned char* base = M.seg(Sb);
                            cl = 0u;
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                const uint2 v2 = reinterpret_cast<const uint2*>(base + 256 * k)[lane];
#pragma unroll
                                for (int cc = 0; cc < 4; ++cc) cl += (kd_half(v2, cc) >> 5) == r_old ? 1u : 0u;
                            }
                            rowv = pres[r_old * 32u + lane];
                        }
                        const uint32_t others = __reduce_add_sync(kFull, cl) - (c == kBF ? 1u : 0u);
                        if (others == 0u) {
                            const uint32_t nw = lane == (Sb >> 5) ? rowv & ~(1u << (Sb & 31)) : rowv;
                            if (lane == (Sb >> 5)) pres[r_old * 32u + lane] = nw;
                            const bool any = __any_sync(kFull, nw != 0u);
                            gw &= (!any && lane == (r_old >> 5)) ? ~(1u << (r_old & 31)) : kNo;
                        }
                        __syncwarp();
                    }
                    if (r_new > 0u) {
                        if (lane == (Sb >> 5)) atomicOr(&pres[r_new * 32u + lane], 1u << (Sb & 31));
                        gw |= lane == (r_new >> 5) ? 1u << (r_new & 31) : 0u;
                    }
                    if (fire) {
                        if (lane == (Sf >> 5)) atomicOr(&pres[Bt * 32u + lane], 1u << (Sf & 31));
                        gw |= lane == (Bt >> 5) ? 1u << (Bt & 31) : 0u;
                    }
                }
                __syncwarp();
                L += (hit ? 0u : 1u) + (fire ? 1u : 0u);
                bout = lane == static_cast<uint32_t>(jj) ? b : bout;
              }
            }
            if (lane < static_cast<uint32_t>(cnt)) raw[j0 + lane] = static_cast<int32_t>(bout);
            fit_tests += fit_blk;
            wcur = wnext;
            ccur = cnext;
        }
        if (spilled) continue;

        // --- objective and dense ids: used bins in creation order
        __syncwarp();
        uint32_t dbase = 0;
        unsigned long long tot = 0;
        for (uint32_t x0 = 0; x0 < L; x0 += 32) {
            const uint32_t x = x0 + lane;
            bool used = false;
            uint32_t t = 0;
            if (x < L) {
                const uint32_t sv = *M.slot(x);
                t = sv & 31u;
                used = (sv >> 5) < Bs[t];
            }
            const unsigned bal = __ballot_sync(kFull, used);
            const uint32_t d = dbase + __popc(bal & lt);
            if (used) {
                p.out.bin_type[wb + d] = static_cast<int32_t>(t);
                tot += Bs[t];
            }
            if (x < L) dense[x] = used ? static_cast<int32_t>(d) : -1;
            dbase += __popc(bal);
        }
        __syncwarp();
        for (int64_t j = lane; j < m; j += 32) raw[j] = dense[raw[j]];
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
    cluster.sync();                                   // CTA 1 may leave now
}

}  // namespace vsbpp
