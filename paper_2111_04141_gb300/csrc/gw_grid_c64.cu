// Gridding kernel instantiations for GW_C64 tables (one translation unit
// per table kind keeps the build parallel).
#include "gw_grid_kernel.cuh"

namespace gw {

void launch_grid_c64(const GridArgs& a, int num_sms, cudaStream_t s) {
    launch_grid_kind<GW_C64>(a, num_sms, s);
}

}  // namespace gw
