// kd.cu -- launchers of the cluster kernel (kd_kernel.cuh): two-CTA clusters,
// one warp per CTA, the whole opt-in shared memory of both CTAs.
#include "internal.h"
#include "kd_kernel.cuh"

namespace vsbpp {

static const void* kd_kernel_for(int criterion) {
    switch (criterion) {
        case kFF: return reinterpret_cast<const void*>(kd_pack_kernel<kFF>);
        case kBF: return reinterpret_cast<const void*>(kd_pack_kernel<kBF>);
        case kWF: return reinterpret_cast<const void*>(kd_pack_kernel<kWF>);
        default: return reinterpret_cast<const void*>(kd_pack_kernel<kRandom>);
    }
}

cudaError_t kd_launch(const KDParams& p, int clusters, cudaStream_t st) {
    const void* k = kd_kernel_for(p.criterion);
    cudaError_t e = ensure_smem_attr(k, p.smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(2 * clusters);
    cfg.blockDim = dim3(32);
    cfg.dynamicSmemBytes = static_cast<size_t>(p.smem);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void* args[] = {const_cast<KDParams*>(&p)};
    return cudaLaunchKernelExC(&cfg, k, args);
}

int kd_max_clusters(int criterion, int smem) {
    const void* k = kd_kernel_for(criterion);
    if (ensure_smem_attr(k, smem) != cudaSuccess) return 0;
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(2);
    cfg.blockDim = dim3(32);
    cfg.dynamicSmemBytes = static_cast<size_t>(smem);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace vsbpp
