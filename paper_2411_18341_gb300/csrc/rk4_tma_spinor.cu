// Instantiations and dispatch of the persistent TMA-fed step kernel for the
// FP32 two-component field with reservoirs (configurations 21..23).
#include "rk4_tma_spinor.cuh"

namespace phx {

cudaError_t launch_rk4_tma_spinor(int tile_cfg, bool pot, bool per, bool tetm,
                                  const TileArgs& ta, cudaStream_t s, int grid) {
  const bool one = ta.ninst == 1;
  switch (tile_cfg) {
    case TILE_SPINOR_64x16: return tma::launch_spinor_variants<2, 8>(pot, per, one, tetm, ta, s, grid);
    case TILE_SPINOR_64x24: return tma::launch_spinor_variants<2, 12>(pot, per, one, tetm, ta, s, grid);
    case TILE_SPINOR_64x32: return tma::launch_spinor_variants<2, 16>(pot, per, one, tetm, ta, s, grid);
    default: break;
  }
  return cudaErrorInvalidValue;
}

}  // namespace phx
