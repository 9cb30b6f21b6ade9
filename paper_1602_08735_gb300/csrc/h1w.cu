// h1w.cu -- launchers of the one-warp first-heuristic kernel (h1w_kernel.cuh),
// one instantiation per (segment words per lane, criterion); the Remark 3
// instantiations are in h1w_r3.cu.
#include "internal.h"
#include "h1w_kernel.cuh"

namespace vsbpp {

static const void* h1w_kernel_for(int slot_cap, int criterion, bool remark3) {
    if (remark3) return h1w_r3_kernel_for(slot_cap, criterion);
#define H1W(NS)                                                                                \
    case NS:                                                                                   \
        switch (criterion) {                                                                   \
            case kFF: return reinterpret_cast<const void*>(h1w_pack_kernel<NS, kFF, false>);      \
            case kBF: return reinterpret_cast<const void*>(h1w_pack_kernel<NS, kBF, false>);      \
            case kWF: return reinterpret_cast<const void*>(h1w_pack_kernel<NS, kWF, false>);      \
            default: return reinterpret_cast<const void*>(h1w_pack_kernel<NS, kRandom, false>);   \
        }
    switch (h1w_ns(slot_cap)) {
        H1W(1) H1W(2) H1W(4) H1W(8)
        default: return nullptr;
    }
#undef H1W
}

int h1w_supported(int slot_cap) { return h1w_ns(slot_cap) > 0; }

int h1w_bytes(int slot_cap, int bf_index) { return h1w_group_bytes(slot_cap, bf_index); }

int h1w_segment_words(int slot_cap) { return h1w_ns(slot_cap); }

int h1w16_slots() { return static_cast<int>(kH16Slots); }

int h1w16_bytes(int bf_index) { return h1w16_group_bytes(bf_index); }

cudaError_t h1w_launch(const H1Params& p, int groups, int grid, int smem, cudaStream_t st) {
    const void* k = h1w_kernel_for(p.slot_cap, p.criterion, p.remark3 != 0);
    if (!k || groups < 1 || groups > 16 || p.compose) return cudaErrorInvalidValue;
    cudaError_t e = ensure_smem_attr(k, smem);
    if (e != cudaSuccess) return e;
    void* args[] = {const_cast<H1Params*>(&p)};
    return cudaLaunchKernel(k, dim3(grid), dim3(32 * groups), args, static_cast<size_t>(smem), st);
}

int h1w_blocks_per_sm(int slot_cap, int criterion, int groups, int smem) {
    const void* k = h1w_kernel_for(slot_cap, criterion, false);   // the Remark 3 kernel has the same shared memory
    if (!k) return 0;
    if (ensure_smem_attr(k, smem) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, 32 * groups, smem) != cudaSuccess) return 0;
    return nb;
}

}  // namespace vsbpp
