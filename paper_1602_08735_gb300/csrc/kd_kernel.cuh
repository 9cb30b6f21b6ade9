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
//   slot      16 bits per bin, (residual << 5) | type (B_1 <= 2047, n <= 32);
//             the bin's creation index is its position.  Bins 0.. live in
//             CTA 0's shared memory, the next ones in CTA 1's (read and
//             written through distributed shared memory), the rest in a
//             global-memory overflow area; a system past 2^19 bins is handed
//             to the global-memory kernel.
//   segment   512 bins (1 KB: two 16-byte words per lane).
//   segmax    largest residual of each segment, tilemax of each 32 segments
//             (FF and WF items): FF takes the first tile, then the first
//             segment, whose maximum is >= w; WF the first whose maximum is
//             the largest of all.
//   gp, pres  (BF items) bit r of gp: some bin has residual r; row r of pres:
//             one bit per segment holding a bin of residual r.  BF takes
//             r* = the least residual >= w present, then the first segment in
//             row r*: no bin anywhere has a residual in [w, r*), so the first
//             bin of residual r* there is the flat scan's answer.
//
// Within the chosen segment each lane reads its 16 slots; the first match
// (FF: residual >= w; BF, WF: residual = the one sought) is one ballot per
// half.  Updates (the chosen slot, a divided-off bin, the summaries) are
// made by the one warp of CTA 0, ordered by __syncwarp before the next item.
// CTA 1 only lends its shared memory: it waits at the cluster barrier until
// CTA 0 has packed every system it takes.
#pragma once

#include <cooperative_groups.h>

#include "kd_params.cuh"

namespace vsbpp {

namespace cg = cooperative_groups;

template <int CRIT>
struct KDWarp {
    static constexpr bool kSeg = CRIT != kBF;                    // FF or WF items occur
    static constexpr bool kIdx = CRIT == kBF || CRIT == kRandom;  // BF items occur

    uint32_t lane;
    uint16_t* segmax;
    uint16_t* tilemax;
    uint32_t* Bs;
    uint32_t* gp;
    uint32_t* pres;
    unsigned char* bins0;    // CTA 0's bins
    unsigned char* bins1;    // CTA 1's bins (distributed shared memory)
    unsigned char* over;     // global-memory overflow of this cluster
    uint32_t segs0, segs1;

    __device__ __forceinline__ uint4* seg_ptr(uint32_t S) const {
        if (S < segs0) return reinterpret_cast<uint4*>(bins0 + static_cast<size_t>(S) * kKDSegBytes);
        S -= segs0;
        if (S < segs1) return reinterpret_cast<uint4*>(bins1 + static_cast<size_t>(S) * kKDSegBytes);
        S -= segs1;
        return reinterpret_cast<uint4*>(over + static_cast<size_t>(S) * kKDSegBytes);
    }
    __device__ __forceinline__ uint16_t* slot_ptr(uint32_t b) const {
        return reinterpret_cast<uint16_t*>(seg_ptr(b >> 9)) + (b & 511u);
    }

    // A segment reads as empty (residual 0 fits nothing) until its bins exist.
    __device__ __forceinline__ void zero_seg(uint32_t S) const {
        uint4* p = seg_ptr(S);
        p[lane] = make_uint4(0u, 0u, 0u, 0u);
        p[32 + lane] = make_uint4(0u, 0u, 0u, 0u);
    }

    __device__ __forceinline__ void refresh_tile(uint32_t T) const {
        const uint32_t v = segmax[T * 32 + lane];
        const uint32_t mx = __reduce_max_sync(kFull, v);
        if (lane == 0) tilemax[T] = static_cast<uint16_t>(mx);
    }

    __device__ __forceinline__ void pres_set(uint32_t r, uint32_t S) const {
        if (lane == 0 && r > 0u) {
            pres[r * 32 + (S >> 5)] |= 1u << (S & 31);
            gp[r >> 5] |= 1u << (r & 31);
        }
    }
};

template <int CRIT>
__global__ void __launch_bounds__(32) kd_pack_kernel(const KDParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cluster = cg::this_cluster();
    cluster.sync();                                   // both CTAs are running
    if (cluster.block_rank() != 0) {
        cluster.sync();                               // CTA 1 lends its memory until CTA 0 is done
        return;
    }
    using W = KDWarp<CRIT>;
    W K;
    K.lane = threadIdx.x & 31u;
    const uint32_t lane = K.lane;
    K.segmax = reinterpret_cast<uint16_t*>(smem + kKDOffSegmax);
    K.tilemax = reinterpret_cast<uint16_t*>(smem + kKDOffTilemax);
    K.Bs = reinterpret_cast<uint32_t*>(smem + kKDOffBs);
    K.gp = reinterpret_cast<uint32_t*>(smem + kKDOffGp);
    K.pres = reinterpret_cast<uint32_t*>(smem + kKDOffPres);
    K.bins0 = smem + kd_bins_offset(p.max_B1, p.pres);
    K.bins1 = cluster.map_shared_rank(smem, 1);
    const uint32_t cid = blockIdx.x >> 1;
    K.over = reinterpret_cast<unsigned char*>(p.over + static_cast<size_t>(cid) * static_cast<size_t>(p.over_bins));
    K.segs0 = static_cast<uint32_t>(p.segs0);
    K.segs1 = static_cast<uint32_t>(p.segs1);
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
        if (B1 > static_cast<uint32_t>(W::kIdx ? p.max_B1 : kKDMaxB1)) {
            // residuals past the slot or presence layout: the global-memory kernel
            if (lane == 0) {
                const unsigned long long pos = atomicAdd(reinterpret_cast<unsigned long long*>(p.spill_seg + 1), 1ull);
                p.spill_list[pos] = static_cast<int32_t>(i);
            }
            continue;
        }
        K.Bs[lane] = Bl;
        for (uint32_t x = lane; x < static_cast<uint32_t>(kKDMaxSegs); x += 32) K.segmax[x] = 0;
        K.tilemax[lane] = 0;
        if (W::kIdx) {
            K.gp[lane] = 0u;
            K.gp[32 + lane] = 0u;
            for (uint32_t x = lane; x < (B1 + 1u) * 32u; x += 32) K.pres[x] = 0u;
        }
        __syncwarp();
        int32_t* raw = p.out.bin_of_item + wb;

        uint32_t L = 0;
        uint32_t below = 0;                  // Remark 3: type-t bins below half, lane t
        if (p.preopen) {                     // literal Rule 2: one empty bin per type, segment 0
            K.zero_seg(0);
            __syncwarp();
            if (lane < static_cast<uint32_t>(n)) *K.slot_ptr(lane) = static_cast<uint16_t>((Bl << 5) | lane);
            if (W::kSeg && lane == 0) {
                K.segmax[0] = static_cast<uint16_t>(B1);
                K.tilemax[0] = static_cast<uint16_t>(B1);
            }
            if (W::kIdx && lane < static_cast<uint32_t>(n)) {
                atomicOr(&K.pres[Bl * 32], 1u);
                atomicOr(&K.gp[Bl >> 5], 1u << (Bl & 31));
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
            uint32_t bout = 0, fit_blk = 0;       // fit tests of this block (< 2^24)
            for (int jj = 0; jj < cnt; ++jj) {
                const uint32_t wj = __shfl_sync(kFull, wcur, jj);
                const int c = CRIT == kRandom ? __shfl_sync(kFull, ccur, jj) : CRIT;
                fit_blk += L;
                const uint32_t nseg = (L + 511u) >> 9;
                const uint32_t ntile = (nseg + 31u) >> 5;

                // 1. the segment holding the answer, and the residual sought
                int S = -1;
                uint32_t want = 0;
                if (W::kSeg && c == kFF) {
                    const unsigned bt = __ballot_sync(kFull, lane < ntile && K.tilemax[lane] >= wj);
                    if (bt) {
                        const uint32_t T = static_cast<uint32_t>(__ffs(bt) - 1);
                        const uint32_t s = T * 32u + lane;
                        const unsigned bs = __ballot_sync(kFull, s < nseg && K.segmax[s] >= wj);
                        S = static_cast<int>(T * 32u) + __ffs(bs) - 1;
                    }
                } else if (W::kSeg && c == kWF) {
                    const uint32_t tm = lane < ntile ? static_cast<uint32_t>(K.tilemax[lane]) : 0u;
                    const uint32_t mx = __reduce_max_sync(kFull, tm);
                    if (mx >= wj) {
                        want = mx;
                        const uint32_t T = static_cast<uint32_t>(__ffs(__ballot_sync(kFull, lane < ntile && tm == mx)) - 1);
                        const uint32_t s = T * 32u + lane;
                        const unsigned bs = __ballot_sync(kFull, s < nseg && K.segmax[s] == mx);
                        S = static_cast<int>(T * 32u) + __ffs(bs) - 1;
                    }
                } else if (W::kIdx) {
                    // the least residual >= w present: words lane and 32 + lane of gp
                    const uint32_t wi = wj >> 5, lo = ~((1u << (wj & 31)) - 1u);
                    uint32_t g0 = K.gp[lane], g1 = K.gp[32 + lane];
                    g0 = lane < wi ? 0u : (lane == wi ? g0 & lo : g0);
                    g1 = 32u + lane < wi ? 0u : (32u + lane == wi ? g1 & lo : g1);
                    const unsigned b0 = __ballot_sync(kFull, g0 != 0u), b1 = __ballot_sync(kFull, g1 != 0u);
                    if (b0 | b1) {
                        const int src = b0 ? __ffs(b0) - 1 : __ffs(b1) - 1;
                        const uint32_t word = __shfl_sync(kFull, b0 ? g0 : g1, src);
                        want = static_cast<uint32_t>((b0 ? src : 32 + src) * 32 + __ffs(word) - 1);
                        const uint32_t rv = K.pres[want * 32u + lane];
                        const unsigned bv = __ballot_sync(kFull, rv != 0u);
                        const int s2 = __ffs(bv) - 1;
                        S = s2 * 32 + __ffs(__shfl_sync(kFull, rv, s2)) - 1;
                    }
                }

                // 2. the chosen bin in segment S (first match in slot order), or
                //    a new bin.  Two slots per 32-bit word: halfword compares
                //    give 0xFFFF per matching slot, one flag byte per slot
                //    (byte permute) and __ffs give the first match of each half.
                const bool hit = S >= 0;
                uint32_t b, r_old, ty;
                uint32_t q[8], mk[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) q[k] = mk[k] = 0u;
                uint32_t own = 32u, ok = 16u;         // lane and slot (0..15) of the chosen bin
                if (hit) {
                    const uint4* sp = K.seg_ptr(static_cast<uint32_t>(S));
                    const uint4 qa = sp[lane], qb = sp[32 + lane];
                    q[0] = qa.x; q[1] = qa.y; q[2] = qa.z; q[3] = qa.w;
                    q[4] = qb.x; q[5] = qb.y; q[6] = qb.z; q[7] = qb.w;
                    if (c == kFF) {
                        const uint32_t W2 = (wj << 5) * 0x10001u;      // residual >= w <=> slot >= w << 5
#pragma unroll
                        for (int k = 0; k < 8; ++k) mk[k] = __vcmpgeu2(q[k], W2);
                    } else {
                        const uint32_t R2 = (want << 5) * 0x10001u;
#pragma unroll
                        for (int k = 0; k < 8; ++k) mk[k] = __vcmpeq2(q[k] & 0xFFE0FFE0u, R2);
                    }
                    const uint32_t a0 = __byte_perm(mk[0], mk[1], 0x7531), a1 = __byte_perm(mk[2], mk[3], 0x7531);
                    const uint32_t b0 = __byte_perm(mk[4], mk[5], 0x7531), b1 = __byte_perm(mk[6], mk[7], 0x7531);
                    const int f0 = a0 ? (__ffs(a0) - 1) >> 3 : a1 ? 4 + ((__ffs(a1) - 1) >> 3) : 8;
                    const int f1 = b0 ? (__ffs(b0) - 1) >> 3 : b1 ? 4 + ((__ffs(b1) - 1) >> 3) : 8;
                    const unsigned h0 = __ballot_sync(kFull, f0 < 8);
                    uint32_t idx;
                    if (h0) {
                        own = static_cast<uint32_t>(__ffs(h0) - 1);
                        ok = static_cast<uint32_t>(__shfl_sync(kFull, f0, static_cast<int>(own)));
                        idx = 8u * own + ok;
                    } else {
                        const unsigned h1 = __ballot_sync(kFull, f1 < 8);
                        own = static_cast<uint32_t>(__ffs(h1) - 1);
                        const uint32_t fo = static_cast<uint32_t>(__shfl_sync(kFull, f1, static_cast<int>(own)));
                        idx = 256u + 8u * own + fo;
                        ok = 8u + fo;
                    }
                    // slot `ok` of every lane (ok is uniform), the owner's broadcast
                    const uint32_t o2 = ok >> 1;      // a select tree keeps q in registers
                    const uint32_t wlo = (o2 & 2u) ? ((o2 & 1u) ? q[3] : q[2]) : ((o2 & 1u) ? q[1] : q[0]);
                    const uint32_t whi = (o2 & 2u) ? ((o2 & 1u) ? q[7] : q[6]) : ((o2 & 1u) ? q[5] : q[4]);
                    const uint32_t wsel = (o2 & 4u) ? whi : wlo;
                    const uint32_t sv = __shfl_sync(kFull, (ok & 1u) ? (wsel >> 16) : (wsel & 0xFFFFu),
                                                    static_cast<int>(own));
                    b = static_cast<uint32_t>(S) * 512u + idx;
                    r_old = sv >> 5;
                    ty = sv & 31u;
                } else {
                    ty = 31u - static_cast<uint32_t>(__clz(__ballot_sync(kFull, Bl >= wj)));
                    b = L;
                    r_old = __shfl_sync(kFull, Bl, static_cast<int>(ty));
                }
                const uint32_t Bt = __shfl_sync(kFull, Bl, static_cast<int>(ty));
                const uint32_t r_new = r_old - wj;
                const bool cross = Bt < 2u * r_old && 2u * r_new <= Bt;        // Rule 5
                const bool fire = p.remark3 ? remark3_divide(below, Bl, !hit, Bt, cross) : cross;
                const uint32_t Lf = hit ? L : L + 1u;

                // 3. stores: new segments cleared first, then the slots
                if (!hit && (b & 511u) == 0u) K.zero_seg(b >> 9);
                if (fire && (Lf & 511u) == 0u) K.zero_seg(Lf >> 9);
                __syncwarp();
                if (lane == 0) {
                    *K.slot_ptr(b) = static_cast<uint16_t>((r_new << 5) | ty);
                    if (fire) *K.slot_ptr(Lf) = static_cast<uint16_t>((Bt << 5) | ty);
                }
                const uint32_t Sb = b >> 9, Sf = Lf >> 9;

                // 4. summaries of the touched segments
                if (W::kSeg) {
                    uint32_t nm;
                    if (hit) {
                        // halfword maxima of this lane's words, the chosen slot
                        // holding its new value; the residual is the slot >> 5
                        const uint32_t nsv = (r_new << 5) | ty;
                        uint32_t mx = 0u;
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            uint32_t wv = q[k];
                            if (lane == own && (ok >> 1) == static_cast<uint32_t>(k))
                                wv = (ok & 1u) ? ((wv & 0xFFFFu) | (nsv << 16)) : ((wv & 0xFFFF0000u) | nsv);
                            mx = __vmaxu2(mx, wv);
                        }
                        nm = __reduce_max_sync(kFull, max(mx & 0xFFFFu, mx >> 16) >> 5);
                    } else {
                        nm = max(static_cast<uint32_t>(K.segmax[Sb]), r_new);
                    }
                    if (fire && Sf == Sb) nm = max(nm, Bt);
                    __syncwarp();
                    if (lane == 0) {
                        K.segmax[Sb] = static_cast<uint16_t>(nm);
                        if (fire && Sf != Sb) K.segmax[Sf] = static_cast<uint16_t>(max(static_cast<uint32_t>(K.segmax[Sf]), Bt));
                    }
                    __syncwarp();
                    K.refresh_tile(Sb >> 5);
                    if (fire && (Sf >> 5) != (Sb >> 5)) K.refresh_tile(Sf >> 5);
                }
                if (W::kIdx) {
                    if (hit) {
                        // does segment S still hold a bin of residual r_old?  BF and
                        // WF items matched exactly r_old above (16 mask bits a slot)
                        uint32_t cntl = 0u;
                        if (c != kFF) {
#pragma unroll
                            for (int k = 0; k < 8; ++k) cntl += __popc(mk[k]);
                        } else {
                            const uint32_t R2 = (r_old << 5) * 0x10001u;
#pragma unroll
                            for (int k = 0; k < 8; ++k) cntl += __popc(__vcmpeq2(q[k] & 0xFFE0FFE0u, R2));
                        }
                        const uint32_t others = (__reduce_add_sync(kFull, cntl) >> 4) - 1u;   // the chosen one left
                        if (others == 0u) {
                            if (lane == 0) K.pres[r_old * 32u + (Sb >> 5)] &= ~(1u << (Sb & 31));
                            __syncwarp();
                            const bool any = __any_sync(kFull, K.pres[r_old * 32u + lane] != 0u);
                            if (!any && lane == 0) K.gp[r_old >> 5] &= ~(1u << (r_old & 31));
                        }
                        __syncwarp();
                    }
                    // r_new's bits (lanes 0, 1) and the divided-off bin's (lanes 2, 3) at once
                    if (lane < 4u) {
                        const uint32_t r = lane < 2u ? r_new : (fire ? Bt : 0u);
                        const uint32_t Sx = lane < 2u ? Sb : Sf;
                        if (r > 0u) {
                            if (lane & 1u) atomicOr(&K.gp[r >> 5], 1u << (r & 31));
                            else atomicOr(&K.pres[r * 32u + (Sx >> 5)], 1u << (Sx & 31));
                        }
                    }
                }
                __syncwarp();
                L += (hit ? 0u : 1u) + (fire ? 1u : 0u);
                bout = lane == static_cast<uint32_t>(jj) ? b : bout;
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
                const uint32_t sv = *K.slot_ptr(x);
                t = sv & 31u;
                used = (sv >> 5) < K.Bs[t];
            }
            const unsigned bal = __ballot_sync(kFull, used);
            const uint32_t d = dbase + __popc(bal & lt);
            if (used) {
                p.out.bin_type[wb + d] = static_cast<int32_t>(t);
                tot += K.Bs[t];
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
