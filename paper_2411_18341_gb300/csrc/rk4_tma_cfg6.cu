// Instantiations of the persistent TMA-fed step kernel for tile
// configuration 6 (2-row x 2-column micro-tiles, 16 warps, 2 CTAs per SM).
#include "rk4_tma_kernel.cuh"

namespace phx {

static_assert(!tma::has_mode3<2, 16, 2>(), "tma_has_drive_reservoir(6)");

cudaError_t launch_tma_cfg6(int mode, bool pot, bool per, bool one, const TileArgs& ta,
                            cudaStream_t s, int grid) {
  return tma::launch_variants<2, 16, 2>(mode, pot, per, one, ta, s, grid);
}

}  // namespace phx
