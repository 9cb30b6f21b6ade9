// variants.cu -- launchers of the offline pre-sort and the bounded-space
// kernels (variants_kernels.cuh).
#include "internal.h"
#include "variants_kernels.cuh"

namespace vsbpp {

cudaError_t presort_launch(const PresortParams& p, int grid, cudaStream_t st) {
    presort_kernel<<<grid, 32 * kPresortWarps, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t unpermute_launch(const PresortParams& p, int grid, cudaStream_t st) {
    unpermute_kernel<<<grid, 256, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t bk_launch(const BKParams& p, int grid, cudaStream_t st) {
    bk_pack_kernel<<<grid, 32 * kBKWarps, 0, st>>>(p);
    return cudaGetLastError();
}

int bk_blocks_per_sm() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, bk_pack_kernel, 32 * kBKWarps, 0) != cudaSuccess)
        return 0;
    return nb;
}

}  // namespace vsbpp
