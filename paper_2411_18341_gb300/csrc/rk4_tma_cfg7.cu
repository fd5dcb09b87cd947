// Instantiations of the persistent TMA-fed step kernel for tile
// configuration 7 (4-row x 2-column micro-tiles, 8 warps, 2 CTAs per SM).
#include "rk4_tma_kernel.cuh"

namespace phx {

static_assert(!tma::has_mode3<4, 8, 2>(), "tma_has_drive_reservoir(7)");

cudaError_t launch_tma_cfg7(int mode, bool pot, bool per, bool one, const TileArgs& ta,
                            cudaStream_t s, int grid) {
  return tma::launch_variants<4, 8, 2>(mode, pot, per, one, ta, s, grid);
}

cudaError_t launch_tma_cfg7_ms(int mode, bool pot, bool per, const TileArgs& ta, cudaStream_t s,
                               int grid) {
  return tma::launch_variants_ms<4, 8, 2>(mode, pot, per, ta, s, grid);
}

}  // namespace phx
