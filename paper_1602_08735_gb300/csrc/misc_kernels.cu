// misc_kernels.cu -- launchers for validation, ordering, composition and the
// second heuristic, plus the dispatch of the first-heuristic kernels.
#include <map>
#include <mutex>
#include <utility>

#include "internal.h"
#include "h2_kernel.cuh"
#include "prep_kernels.cuh"
#include "kc_kernel.cuh"

namespace vsbpp {

cudaError_t h1_launch_narrow_entry(const H1Params&, int, int, int, int, cudaStream_t);
cudaError_t h1_launch_wide_entry(const H1Params&, int, int, int, int, cudaStream_t);
int h1_occ_narrow_entry(int, int, int);
int h1_occ_wide_entry(int, int, int);

cudaError_t ensure_smem_attr(const void* kernel, int smem) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    int& cur = done[std::make_pair(kernel, dev)];
    if (smem <= cur) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) cur = smem;
    return e;
}

bool h1_shape_supported(int G, int groups) {
    if (G == 1) return groups == 1 || groups == 2 || groups == 4 || groups == 8 || groups == 16;
    return groups == 1 && (G == 2 || G == 4 || G == 8 || G == 16 || G == 32);
}

cudaError_t h1_launch(bool wide, const H1Params& p, int G, int groups, int grid, int smem,
                      cudaStream_t st) {
    return wide ? h1_launch_wide_entry(p, G, groups, grid, smem, st)
                : h1_launch_narrow_entry(p, G, groups, grid, smem, st);
}

int h1_blocks_per_sm(bool wide, int G, int groups, int smem) {
    return wide ? h1_occ_wide_entry(G, groups, smem) : h1_occ_narrow_entry(G, groups, smem);
}

static const void* h2_reg_kernel(int sublist, int criterion);

cudaError_t h2_launch(const H2Params& p, int threads, int grid, int smem, cudaStream_t st) {
    if (!p.preopen && !p.remark3) {
        // bins in registers; sublist size and criterion fixed at compile time
        const void* k = h2_reg_kernel(p.sublist, p.criterion);
        if (k) {
            void* args[] = {const_cast<H2Params*>(&p)};
            return cudaLaunchKernel(k, dim3(grid), dim3(threads), args, 0, st);
        }
    }
    cudaError_t e = ensure_smem_attr(reinterpret_cast<const void*>(h2_pack_kernel), smem);
    if (e != cudaSuccess) return e;
    h2_pack_kernel<<<grid, threads, smem, st>>>(p);
    return cudaGetLastError();
}

// Register second-heuristic kernel for (sublist size, criterion).
static const void* h2_reg_kernel(int sublist, int criterion) {
#define H2K(S)                                                                          \
    case S:                                                                             \
        switch (criterion) {                                                            \
            case kFF: return reinterpret_cast<const void*>(h2_pack_kernel_reg<S, kFF>);      \
            case kBF: return reinterpret_cast<const void*>(h2_pack_kernel_reg<S, kBF>);      \
            case kWF: return reinterpret_cast<const void*>(h2_pack_kernel_reg<S, kWF>);      \
            default: return reinterpret_cast<const void*>(h2_pack_kernel_reg<S, kRandom>);   \
        }
    switch (sublist) {
        H2K(1) H2K(2) H2K(3) H2K(4) H2K(5) H2K(6)
        default: return nullptr;
    }
#undef H2K
}

int h2_blocks_per_sm_reg(int threads, int sublist, int criterion) {
    const void* k = h2_reg_kernel(sublist, criterion);
    if (!k) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads, 0) != cudaSuccess) return 0;
    return nb;
}

int h2_blocks_per_sm(int threads, int smem) {
    if (ensure_smem_attr(reinterpret_cast<const void*>(h2_pack_kernel), smem) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, h2_pack_kernel, threads, smem) != cudaSuccess)
        return 0;
    return nb;
}

cudaError_t kc_launch(const KCParams& p, int grid, int smem, cudaStream_t st) {
    cudaError_t e = ensure_smem_attr(reinterpret_cast<const void*>(kc_pack_kernel), smem);
    if (e != cudaSuccess) return e;
    kc_pack_kernel<<<grid, 32, smem, st>>>(p);
    return cudaGetLastError();
}

int kc_blocks_per_sm(int smem) {
    if (ensure_smem_attr(reinterpret_cast<const void*>(kc_pack_kernel), smem) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kc_pack_kernel, 32, smem) != cudaSuccess) return 0;
    return nb;
}

cudaError_t validate_launch(const PrepParams& p, int grid, cudaStream_t st) {
    validate_kernel<<<grid, 256, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t order_launch(uint32_t* hist, int64_t* cursor, int64_t* seg, unsigned long long* queue,
                         int64_t* spill_seg, cudaStream_t st) {
    order_kernel<<<1, 32, 0, st>>>(hist, cursor, seg, queue, spill_seg);
    return cudaGetLastError();
}

cudaError_t scatter_launch(const BatchView& in, const int32_t* cls, int64_t* cursor, int32_t* order,
                           int grid, cudaStream_t st) {
    scatter_kernel<<<grid, 256, 0, st>>>(in, cls, cursor, order);
    return cudaGetLastError();
}

cudaError_t unit_scan_launch(int64_t N, const int64_t* nu, int64_t* unit_base, int64_t* seg_units,
                             unsigned long long* queue, cudaStream_t st) {
    unit_scan_kernel<<<1, 1024, 0, st>>>(N, nu, unit_base, seg_units, queue);
    return cudaGetLastError();
}

cudaError_t compose_launch(const ComposeParams& p, int grid, cudaStream_t st) {
    compose_kernel<<<grid, 256, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace vsbpp
