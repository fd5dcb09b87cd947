// Instantiations of the persistent TMA-fed step kernel for tile
// configuration 4 (2-row x 2-column micro-tiles, 24 warps, 1 CTA per SM).
#include "rk4_tma_kernel.cuh"

namespace phx {

static_assert(tma::has_mode3<2, 24, 1>(), "tma_has_drive_reservoir(4)");

cudaError_t launch_tma_cfg4(int mode, bool pot, bool per, bool one, const TileArgs& ta,
                            cudaStream_t s, int grid) {
  return tma::launch_variants<2, 24, 1>(mode, pot, per, one, ta, s, grid);
}

}  // namespace phx
