// kc_kernel.cuh -- the first heuristic of Section 6.3 for membrane systems too
// large for shared memory (hundreds of thousands of bins).
//
// The result is the same as the flat fit test over every bin (Rule 4: every
// open bin membrane tests the item; FF / BF / WF with the lowest index on
// ties), but one warp answers each item by touching one tile of bins:
//
//   bins        global memory (L2-resident), tiles of TB = 2048 bins; slot =
//               (residual << 16) | (index within the tile << 5) | type, so
//               a key's order is residual, then creation index
//   tile_max    shared: largest residual in each tile; sup_max: largest over
//               each run of 32 tiles
//   pres        shared, BF only: bit (r, tile) set iff the tile holds a bin
//               with residual r; gp: bit r set iff any tile does
//
//   FF: first tile whose max >= w, then the first slot >= w in it.
//   WF: M = max over all tiles; first tile whose max == M; the first slot
//       with residual M in it (the slot key min(slot ^ HI) finds it).
//   BF: r* = least residual >= w present anywhere (gp); first tile holding
//       r*; in it, min(slot - (w << 16)) gives r* at its lowest index --
//       no bin anywhere has a residual in [w, r*).
//
// After the update the tile is still in registers, so its new maximum and
// whether it still holds the old residual are computed from them; no counts
// are kept.  Rule 5 divisions and new bins append at the end as in the flat
// kernel.  One warp per instance, no block barriers.
#pragma once

#include "kc_params.cuh"

namespace vsbpp {

struct KCWarp {
    int lane;
    uint16_t* tile_max;
    uint16_t* sup_max;
    uint32_t* Bs;
    uint32_t* gp;
    uint32_t* pres;
    int gp_words;
    int pw;            // pres words per residual
    bool track;        // BF presence maintained (BF or RANDOM)
    uint32_t* slots;

    __device__ __forceinline__ void pres_set(uint32_t r, uint32_t t) {
        if (lane == 0) {
            pres[r * pw + (t >> 5)] |= 1u << (t & 31);
            gp[r >> 5] |= 1u << (r & 31);
        }
    }

    // After bin(s) of tile t lost residual r: clear the tile's bit when no
    // slot of the tile holds r any more (still_there is warp-uniform).
    __device__ __forceinline__ void pres_drop(uint32_t r, uint32_t t, bool still_there) {
        if (still_there) return;
        if (lane == 0) pres[r * pw + (t >> 5)] &= ~(1u << (t & 31));
        __syncwarp();
        const uint32_t v = lane < pw ? pres[r * pw + lane] : 0u;
        const bool any = __any_sync(kFull, v != 0u);
        if (!any && lane == 0) gp[r >> 5] &= ~(1u << (r & 31));
        __syncwarp();
    }

    __device__ __forceinline__ void refresh_sup(uint32_t t) {
        const uint32_t s = t >> 5;
        const uint32_t v = tile_max[s * 32 + lane];
        const uint32_t mx = __reduce_max_sync(kFull, v);
        if (lane == 0) sup_max[s] = static_cast<uint16_t>(mx);
    }

    // Create bin L (residual r, type t).  A bin that opens a tile clears it.
    __device__ void append(uint32_t L, uint32_t r, uint32_t t) {
        const uint32_t tile = L / kTileBins, idx = L % kTileBins;
        if (idx == 0) {
            uint4* q = reinterpret_cast<uint4*>(slots + static_cast<size_t>(tile) * kTileBins);
            for (int k = lane; k < kTileBins / 4; k += 32) q[k] = make_uint4(0u, 0u, 0u, 0u);
            if (lane == 0) tile_max[tile] = 0;
            __syncwarp();
        }
        if (lane == 0) {
            slots[L] = (r << 16) | (idx << 5) | t;
            if (r > tile_max[tile]) tile_max[tile] = static_cast<uint16_t>(r);
        }
        __syncwarp();
        refresh_sup(tile);
        if (track) pres_set(r, tile);
        __syncwarp();
    }

    // First set bit >= w in gp, or -1.
    __device__ int first_present_at_least(uint32_t w) const {
        for (int base = static_cast<int>(w >> 5); base < gp_words; base += 32) {
            const int wi = base + lane;
            uint32_t v = wi < gp_words ? gp[wi] : 0u;
            if (wi == static_cast<int>(w >> 5)) v &= ~((1u << (w & 31)) - 1u);
            const unsigned bal = __ballot_sync(kFull, v != 0u);
            if (bal) {
                const int src = __ffs(bal) - 1;
                const uint32_t word = __shfl_sync(kFull, v, src);
                return (base + src) * 32 + (__ffs(word) - 1);
            }
        }
        return -1;
    }
};

__global__ void __launch_bounds__(32) kc_pack_kernel(const KCParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    KCWarp W;
    W.lane = threadIdx.x & 31;
    const int lane = W.lane;
    unsigned char* base = smem;
    W.tile_max = reinterpret_cast<uint16_t*>(base);  base += kMaxTiles * 2;
    W.sup_max = reinterpret_cast<uint16_t*>(base);   base += kSupers * 2;
    W.Bs = reinterpret_cast<uint32_t*>(base);        base += kMaxTypes * 4;
    W.gp_words = (p.max_B1 + 1 + 31) / 32;
    W.gp = reinterpret_cast<uint32_t*>(base);        base += W.gp_words * 4;
    W.pres = reinterpret_cast<uint32_t*>(base);
    W.pw = p.pres_words;
    W.slots = p.slots_all + static_cast<size_t>(blockIdx.x) * static_cast<size_t>(p.bin_cap);

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
        const uint32_t Bl = lane < n ? static_cast<uint32_t>(B[lane]) : 0u;
        const uint32_t B1 = __shfl_sync(kFull, Bl, 0);
        W.Bs[lane] = Bl;
        W.track = p.criterion == kBF || p.criterion == kRandom;
        for (int x = lane; x < kSupers; x += 32) W.sup_max[x] = 0;
        for (int x = lane; x < kMaxTiles; x += 32) W.tile_max[x] = 0;
        for (int x = lane; x < W.gp_words; x += 32) W.gp[x] = 0;
        if (W.track)
            for (int x = lane; x < static_cast<int>((B1 + 1) * W.pw); x += 32) W.pres[x] = 0;
        __syncwarp();
        int32_t* raw = p.out.bin_of_item + wb;

        uint32_t L = 0;
        if (p.preopen) {
            for (int t = 0; t < n; ++t) W.append(L++, static_cast<uint32_t>(B[t]), static_cast<uint32_t>(t));
        }
        uint32_t below = (p.preopen && lane < n) ? 1u : 0u;   // Remark 3: type-t bins below half
        unsigned long long fit_tests = 0;
        // weights a 32-item block ahead (lane l holds item block + l); each
        // item's weight is a shuffle off the dependent chain, and the items'
        // bins are written once per block
        uint32_t wcur = lane < m ? static_cast<uint32_t>(__ldg(w + lane)) : 0u;
        uint32_t wnext = 32 + lane < m ? static_cast<uint32_t>(__ldg(w + 32 + lane)) : 0u;
        uint32_t bout = 0;
        for (int64_t j = 0; j < m; ++j) {
            const int jj = static_cast<int>(j & 31);
            const uint32_t wj = __shfl_sync(kFull, wcur, jj);
            const int c = pick_criterion(p.criterion, p.seed, static_cast<uint64_t>(j));
            fit_tests += L;
            const uint32_t ntiles = (L + kTileBins - 1) / kTileBins;
            const uint32_t nsup = (ntiles + 31) / 32;
            // --- choose the tile from the summaries
            int tile = -1;
            uint32_t want = 0;        // BF: r*; WF: M
            if (c == kFF) {
                for (uint32_t s0 = 0; s0 < nsup && tile < 0; s0 += 32) {
                    const uint32_t s = s0 + lane;
                    const unsigned bal = __ballot_sync(kFull, s < nsup && W.sup_max[s] >= wj);
                    if (bal) {
                        const uint32_t sf = s0 + __ffs(bal) - 1;
                        const uint32_t t = sf * 32 + lane;
                        const unsigned b2 = __ballot_sync(kFull, t < ntiles && W.tile_max[t] >= wj);
                        if (b2) tile = static_cast<int>(sf * 32 + __ffs(b2) - 1);
                    }
                }
            } else if (c == kWF) {
                uint32_t mx = 0;
                for (uint32_t s = lane; s < nsup; s += 32) mx = max(mx, static_cast<uint32_t>(W.sup_max[s]));
                mx = __reduce_max_sync(kFull, mx);
                if (ntiles > 0 && mx >= wj) {
                    want = mx;
                    for (uint32_t s0 = 0; s0 < nsup && tile < 0; s0 += 32) {
                        const uint32_t s = s0 + lane;
                        const unsigned bal = __ballot_sync(kFull, s < nsup && W.sup_max[s] == mx);
                        if (bal) {
                            const uint32_t sf = s0 + __ffs(bal) - 1;
                            const uint32_t t = sf * 32 + lane;
                            const unsigned b2 = __ballot_sync(kFull, t < ntiles && W.tile_max[t] == mx);
                            if (b2) tile = static_cast<int>(sf * 32 + __ffs(b2) - 1);
                        }
                    }
                }
            } else {
                const int rs = W.first_present_at_least(wj);
                if (rs >= 0) {
                    want = static_cast<uint32_t>(rs);
                    const uint32_t pv = lane < W.pw ? W.pres[want * W.pw + lane] : 0u;
                    const unsigned bal = __ballot_sync(kFull, pv != 0u);
                    if (bal) {
                        const int src = __ffs(bal) - 1;
                        const uint32_t word = __shfl_sync(kFull, pv, src);
                        tile = src * 32 + __ffs(word) - 1;
                    }
                }
            }

            uint32_t b, r_old, t;
            bool hit = tile >= 0;
            if (hit) {
                // --- scan the chosen tile (Rule 4 over its bins)
                const uint4* q = reinterpret_cast<const uint4*>(W.slots + static_cast<size_t>(tile) * kTileBins);
                uint32_t s[4 * kTileQuadsPerLane];
#pragma unroll
                for (int k = 0; k < kTileQuadsPerLane; ++k) {
                    const uint4 v4 = q[k * 32 + lane];
                    s[4 * k] = v4.x; s[4 * k + 1] = v4.y; s[4 * k + 2] = v4.z; s[4 * k + 3] = v4.w;
                }
                const uint32_t W16 = wj << 16;
                // BF / WF: the least and the second-least key of the tile (the
                // second tells whether another bin has the chosen residual,
                // and for WF the tile's next-largest residual)
                uint32_t key = 0xFFFFFFFFu, sec = 0xFFFFFFFFu;
                if (c == kFF) {
#pragma unroll
                    for (int x = 4 * kTileQuadsPerLane - 1; x >= 0; --x)
                        if (s[x] >= W16) key = ((s[x] & 0xFFFFu) << 16) | (s[x] >> 16);
                } else if (c == kWF) {
#pragma unroll
                    for (int x = 0; x < 4 * kTileQuadsPerLane; ++x) {
                        const uint32_t v = s[x] ^ 0xFFFF0000u;
                        sec = min(sec, max(key, v));
                        key = min(key, v);
                    }
                } else {
#pragma unroll
                    for (int x = 0; x < 4 * kTileQuadsPerLane; ++x) {
                        const uint32_t v = s[x] - W16;
                        sec = min(sec, max(key, v));
                        key = min(key, v);
                    }
                }
                const uint32_t lane_key = key;
                key = __reduce_min_sync(kFull, key);
                const uint32_t key2 = c == kFF ? 0xFFFFFFFFu : __reduce_min_sync(kFull, lane_key == key ? sec : lane_key);
                uint32_t low;
                if (c == kFF) { low = key >> 16; r_old = key & 0xFFFFu; }
                else if (c == kWF) { low = key & 0xFFFFu; r_old = 0xFFFFu - (key >> 16); }
                else { low = key & 0xFFFFu; r_old = (key >> 16) + wj; }
                const uint32_t idx = low >> 5;
                t = low & 31u;
                b = static_cast<uint32_t>(tile) * kTileBins + idx;
                const uint32_t r_new = r_old - wj;
                // Tile maximum and presence of r_old after the update, from the
                // registers.  The updated slot sits in lane (idx/4)%32, register
                // 4*(idx/128) + idx%4.
                const int own_lane = static_cast<int>((idx >> 2) & 31u);
                const int own_reg = static_cast<int>(((idx >> 7) << 2) | (idx & 3u));
                const uint32_t new_slot = (r_new << 16) | low;
                const uint32_t old_max = W.tile_max[tile];
                uint32_t mx = old_max;
                if (c == kWF) {
                    // the chosen bin held the maximum: the new one is the
                    // larger of its new residual and the next-largest
                    mx = max(r_new, 0xFFFFu - (key2 >> 16));
                } else if (r_old == old_max) {     // the chosen bin held the maximum
                    uint32_t top = 0;
#pragma unroll
                    for (int x = 0; x < 4 * kTileQuadsPerLane; ++x) {
                        const uint32_t sl = (lane == own_lane && x == own_reg) ? new_slot : s[x];
                        top = max(top, sl);
                    }
                    mx = __reduce_max_sync(kFull, top) >> 16;
                }
                bool still = true;
                if (W.track && c != kFF) {          // BF / WF keys order by residual
                    still = (key2 >> 16) == (key >> 16);
                } else if (W.track) {               // does the tile still hold r_old?
                    bool other = false;
#pragma unroll
                    for (int x = 0; x < 4 * kTileQuadsPerLane; ++x)
                        other |= (s[x] >> 16) == r_old && !(lane == own_lane && x == own_reg);
                    still = __any_sync(kFull, other);
                }
                if (lane == 0) {
                    W.slots[b] = new_slot;
                    W.tile_max[tile] = static_cast<uint16_t>(mx);
                }
                __syncwarp();
                if (mx != old_max) W.refresh_sup(static_cast<uint32_t>(tile));
                if (W.track) {
                    W.pres_drop(r_old, static_cast<uint32_t>(tile), still);
                    W.pres_set(r_new, static_cast<uint32_t>(tile));
                }
                __syncwarp();
            } else {
                // nothing fits: a bin of the smallest type that holds w
                t = 31u - static_cast<uint32_t>(__clz(__ballot_sync(kFull, Bl >= wj)));
                b = L;
                r_old = __shfl_sync(kFull, Bl, static_cast<int>(t));
                W.append(L, r_old - wj, t);
                ++L;
            }
            const uint32_t Bt = __shfl_sync(kFull, Bl, static_cast<int>(t));
            const uint32_t r_new = r_old - wj;
            const bool cross = Bt < 2 * r_old && 2 * r_new <= Bt;          // Rule 5
            if (p.remark3 ? remark3_divide(below, Bl, !hit, Bt, cross) : cross) {
                W.append(L, Bt, t);
                ++L;
            }
            bout = lane == jj ? b : bout;
            if (jj == 31 || j + 1 == m) {
                if (lane <= jj) raw[j - jj + lane] = static_cast<int32_t>(bout);
                wcur = wnext;
                wnext = j + 33 + lane < m ? static_cast<uint32_t>(__ldg(w + j + 33 + lane)) : 0u;
            }
        }

        // --- objective and dense ids (used bins in creation order)
        __syncwarp();
        uint32_t base_id = 0;
        unsigned long long tot = 0;
        for (uint32_t b0 = 0; b0 < L; b0 += 32) {
            const uint32_t b = b0 + lane;
            bool used = false;
            uint32_t tt = 0;
            if (b < L) {
                const uint32_t sl = W.slots[b];
                tt = sl & 31u;
                used = (sl >> 16) < W.Bs[tt];
            }
            const unsigned bal = __ballot_sync(kFull, used);
            const uint32_t d = base_id + __popc(bal & ((1u << lane) - 1u));
            if (used) {
                W.slots[b] = d;                                  // slot now holds the dense id
                p.out.bin_type[wb + d] = static_cast<int32_t>(tt);
                tot += W.Bs[tt];
            }
            base_id += __popc(bal);
        }
        __syncwarp();
        for (int64_t j = lane; j < m; j += 32) raw[j] = static_cast<int32_t>(W.slots[raw[j]]);
        tot = warp_sum_u64(tot);
        if (lane == 0) {
            p.out.num_bins[i] = base_id;
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
