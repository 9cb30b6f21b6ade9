// h1w_r3.cu -- the one-warp first-heuristic kernel (h1w_kernel.cuh) with
// Rule 5 under Remark 3's per-type condition (VSBPP_REMARK3), one
// instantiation per (segment words per lane, criterion); a unit of its own so
// that it compiles beside h1w.cu.
#include "internal.h"
#include "h1w_kernel.cuh"

namespace vsbpp {

const void* h1w_r3_kernel_for(int slot_cap, int criterion) {
#define H1W(NS)                                                                               \
    case NS:                                                                                  \
        switch (criterion) {                                                                  \
            case kFF: return reinterpret_cast<const void*>(h1w_pack_kernel<NS, kFF, true>);      \
            case kBF: return reinterpret_cast<const void*>(h1w_pack_kernel<NS, kBF, true>);      \
            case kWF: return reinterpret_cast<const void*>(h1w_pack_kernel<NS, kWF, true>);      \
            default: return reinterpret_cast<const void*>(h1w_pack_kernel<NS, kRandom, true>);   \
        }
    switch (h1w_ns(slot_cap)) {
        H1W(1) H1W(2) H1W(4) H1W(8)
        default: return nullptr;
    }
#undef H1W
}

}  // namespace vsbpp
