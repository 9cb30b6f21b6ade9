// h1_narrow.cu -- first-heuristic kernels with 32-bit bin slots
// (B_1 <= 32767, at most 65536 bins per membrane system).
#include "internal.h"

#define H1_SLOT uint32_t
#define H1_LAUNCH_NAME h1_launch_narrow
#define H1_OCC_NAME h1_occ_narrow
#include "h1_launch.inc"

namespace vsbpp {
cudaError_t h1_launch_narrow_entry(const H1Params& p, int G, int groups, int grid, int smem,
                                   cudaStream_t st) {
    return h1_launch_narrow(p, G, groups, grid, smem, st);
}
int h1_occ_narrow_entry(int G, int groups, int smem) { return h1_occ_narrow(G, groups, smem); }
}  // namespace vsbpp
