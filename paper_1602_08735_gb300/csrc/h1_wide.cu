// h1_wide.cu -- first-heuristic kernels with 64-bit bin slots (any B_1 < 2^31).
#include "internal.h"

#define H1_SLOT unsigned long long
#define H1_LAUNCH_NAME h1_launch_wide
#define H1_OCC_NAME h1_occ_wide
#include "h1_launch.inc"

namespace vsbpp {
cudaError_t h1_launch_wide_entry(const H1Params& p, int G, int groups, int grid, int smem,
                                 cudaStream_t st) {
    return h1_launch_wide(p, G, groups, grid, smem, st);
}
int h1_occ_wide_entry(int G, int groups, int smem) { return h1_occ_wide(G, groups, smem); }
}  // namespace vsbpp
