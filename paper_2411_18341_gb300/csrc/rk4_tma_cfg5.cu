// Instantiations of the persistent TMA-fed step kernel for tile
// configuration 5 (2-row x 2-column micro-tiles, 32 warps, 1 CTA per SM).
#include "rk4_tma_kernel.cuh"

namespace phx {

static_assert(!tma::has_mode3<2, 32, 1>(), "tma_has_drive_reservoir(5)");

cudaError_t launch_tma_cfg5(int mode, bool pot, bool per, bool one, const TileArgs& ta,
                            cudaStream_t s, int grid) {
  return tma::launch_variants<2, 32, 1>(mode, pot, per, one, ta, s, grid);
}

}  // namespace phx
