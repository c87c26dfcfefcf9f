// Gridding kernel instantiations for GW_BF16X2 tables (one translation unit
// per table kind keeps the build parallel).
#include "gw_grid_kernel.cuh"

namespace gw {

void launch_grid_bf16(const GridArgs& a, int num_sms, cudaStream_t s) {
    launch_grid_kind<GW_BF16X2>(a, num_sms, s);
}

}  // namespace gw
