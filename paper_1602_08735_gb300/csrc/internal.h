// internal.h -- host-side declarations shared by the library's translation
// units (kernel launchers and the C ABI).  Not part of the public interface.
#pragma once

#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

#include "vsbpp.h"
#include "device_common.cuh"
#include "h1_kernel.cuh"
#include "h2_params.cuh"
#include "prep_params.cuh"
#include "kc_params.cuh"
#include "variants_params.cuh"
#include "kd_params.cuh"

namespace vsbpp {

// Checks of vsbpp_params shared by every entry point (null = defaults):
// VSBPP_OK, VSBPP_EINVAL or VSBPP_ECAPACITY (a bound above VSBPP_MAX_OPEN).
int check_params_public(const vsbpp_params* p);

// The device work counters {items, fit tests} while vsbpp_counters_enable is
// on, else null.
unsigned long long* counters_ptr();

// Raises a kernel's dynamic shared-memory limit to `smem` bytes on the current
// device, once per (kernel, device, size) increase.
cudaError_t ensure_smem_attr(const void* kernel, int smem);

// First-heuristic kernel: G warps per group, `groups` groups per block,
// narrow (32-bit) or wide (64-bit) bin slots.  Supported shapes:
// (G=1, groups in {1,2,4,8,16}) and (G in {2,4,8,16,32}, groups=1).
bool h1_shape_supported(int G, int groups);
cudaError_t h1_launch(bool wide, const H1Params& p, int G, int groups, int grid, int smem,
                      cudaStream_t st);
int h1_blocks_per_sm(bool wide, int G, int groups, int smem);

// One-warp first-heuristic kernel (narrow slots, direct mode, at most
// 32768 bins per system): `groups` warps per block, each a system at a time.
int h1w_supported(int slot_cap);
const void* h1w_r3_kernel_for(int slot_cap, int criterion);   // h1w_r3.cu: the VSBPP_REMARK3 kernels
int h1w_bytes(int slot_cap, int bf_index);
cudaError_t h1w_launch(const H1Params& p, int groups, int grid, int smem, cudaStream_t st);
int h1w_blocks_per_sm(int slot_cap, int criterion, int groups, int smem);
// Segment words per lane of a one-warp shape (1, 2, 4, 8; 0: none).  The
// 8-word shapes also take systems with B_1 <= 255 in 16-bit slots: that
// layout's bins and its shared memory per warp.
int h1w_segment_words(int slot_cap);
int h1w16_slots();
int h1w16_bytes(int bf_index);

cudaError_t kc_launch(const KCParams& p, int grid, int smem, cudaStream_t st);
// Cluster kernel (bins in two CTAs' shared memory): `clusters` two-CTA clusters.
cudaError_t kd_launch(const KDParams& p, int clusters, cudaStream_t st);
int kd_max_clusters(int criterion, int smem);
int kc_blocks_per_sm(int smem);

cudaError_t h2_launch(const H2Params& p, int threads, int grid, int smem, cudaStream_t st);
// Exhaustive second heuristic (sublists of 7..12 items): search, then write.
cudaError_t h2x_launch(const H2XParams& p, int grid, cudaStream_t st);
int h2x_blocks_per_sm(int sublist, int criterion);
int h2_blocks_per_sm(int threads, int smem);
int h2_blocks_per_sm_reg(int threads, int sublist, int criterion);   // register kernel (no preopen)

// Offline pre-sort (VSBPP_PRESORT) and its inverse; bounded-space kernel.
cudaError_t presort_launch(const PresortParams& p, int grid, cudaStream_t st);
cudaError_t unpermute_launch(const PresortParams& p, int grid, cudaStream_t st);
cudaError_t bk_launch(const BKParams& p, int grid, cudaStream_t st);
int bk_blocks_per_sm();
constexpr int kBKWarpsPerBlock = kBKWarps;

cudaError_t validate_launch(const PrepParams& p, int grid, cudaStream_t st);
cudaError_t order_launch(uint32_t* hist, int64_t* cursor, int64_t* seg, unsigned long long* queue,
                         int64_t* spill_seg, cudaStream_t st);
cudaError_t scatter_launch(const BatchView& in, const int32_t* cls, int64_t* cursor, int32_t* order,
                           int grid, cudaStream_t st);
cudaError_t unit_scan_launch(int64_t N, const int64_t* nu, int64_t* unit_base, int64_t* seg_units,
                             unsigned long long* queue, cudaStream_t st);
cudaError_t compose_launch(const ComposeParams& p, int grid, cudaStream_t st);

}  // namespace vsbpp
