// Gridding kernel instantiations for the real w = 0 kernel (padded tables
// of FP32 real parts; one translation unit per table kind keeps the build
// parallel).
#include "gw_grid_kernel.cuh"

namespace gw {

void launch_grid_r32(const GridArgs& a, int num_sms, cudaStream_t s) {
    launch_grid_kind<kTabRealF32>(a, num_sms, s);
}

}  // namespace gw
