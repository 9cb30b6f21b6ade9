// h2x.cu -- launchers of the exhaustive second heuristic (h2x_kernel.cuh),
// one instantiation per (sublist size 7..12, criterion).
#include "internal.h"
#include "h2x_kernel.cuh"

namespace vsbpp {

template <int S>
static const void* h2x_pick(int criterion, bool writer) {
    switch (criterion) {
        case kFF: return writer ? reinterpret_cast<const void*>(h2x_write_kernel<S, kFF>)
                                : reinterpret_cast<const void*>(h2x_search_kernel<S, kFF>);
        case kBF: return writer ? reinterpret_cast<const void*>(h2x_write_kernel<S, kBF>)
                                : reinterpret_cast<const void*>(h2x_search_kernel<S, kBF>);
        case kWF: return writer ? reinterpret_cast<const void*>(h2x_write_kernel<S, kWF>)
                                : reinterpret_cast<const void*>(h2x_search_kernel<S, kWF>);
        default: return writer ? reinterpret_cast<const void*>(h2x_write_kernel<S, kRandom>)
                               : reinterpret_cast<const void*>(h2x_search_kernel<S, kRandom>);
    }
}

static const void* h2x_kernel_for(int sublist, int criterion, bool writer) {
    switch (sublist) {
        case 7: return h2x_pick<7>(criterion, writer);
        case 8: return h2x_pick<8>(criterion, writer);
        case 9: return h2x_pick<9>(criterion, writer);
        case 10: return h2x_pick<10>(criterion, writer);
        case 11: return h2x_pick<11>(criterion, writer);
        case 12: return h2x_pick<12>(criterion, writer);
        default: return nullptr;
    }
}

cudaError_t h2x_launch(const H2XParams& p, int grid, cudaStream_t st) {
    const void* search = h2x_kernel_for(p.sublist, p.criterion, false);
    const void* write = h2x_kernel_for(p.sublist, p.criterion, true);
    if (!search || !write) return cudaErrorInvalidValue;
    void* args[] = {const_cast<H2XParams*>(&p)};
    cudaError_t e = cudaLaunchKernel(search, dim3(grid), dim3(128), args, 0, st);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernel(write, dim3(grid), dim3(128), args, 0, st);
}

int h2x_blocks_per_sm(int sublist, int criterion) {
    const void* k = h2x_kernel_for(sublist, criterion, false);
    if (!k) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, 128, 0) != cudaSuccess) return 0;
    return nb;
}

}  // namespace vsbpp
