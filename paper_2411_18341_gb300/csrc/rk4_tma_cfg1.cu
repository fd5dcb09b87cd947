// Instantiations of the persistent TMA-fed step kernel for tile
// configuration 1 (4-row x 2-column micro-tiles, 16 warps, 1 CTA per SM).
#include "rk4_tma_kernel.cuh"

namespace phx {

static_assert(!tma::has_mode3<4, 16, 1>(), "tma_has_drive_reservoir(1)");

cudaError_t launch_tma_cfg1(int mode, bool pot, bool per, bool one, const TileArgs& ta,
                            cudaStream_t s, int grid) {
  return tma::launch_variants<4, 16, 1>(mode, pot, per, one, ta, s, grid);
}

}  // namespace phx
