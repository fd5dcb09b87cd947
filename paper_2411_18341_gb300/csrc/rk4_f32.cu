// FP32 instantiations of the fused RK4 step.
#include "rk4_generic.cuh"

namespace phx {

cudaError_t launch_rk4_step_f32(const ModelKey& m, const StepArgs<float>& a,
                                cudaStream_t s, int tile) {
  if (m.ncomp == 1) {
    if (m.reservoir) return launch_generic<float, 1, true, false, 32, 32, 256>(a, s);
    return launch_generic<float, 1, false, false, 32, 32, 256>(a, s);
  }
  if (m.tetm) {
    if (m.reservoir) {
      // tile shapes of the spinor + TE-TM kernel (phx_params.tile 10..12;
      // the default 64 x 32 was the fastest at 2048^2)
      if (tile == 10) return launch_generic<float, 2, true, true, 32, 16, 256>(a, s);
      if (tile == 11) return launch_generic<float, 2, true, true, 32, 32, 256>(a, s);
      if (tile == 12) return launch_generic<float, 2, true, true, 64, 16, 256>(a, s);
      return launch_generic<float, 2, true, true, 64, 32, 512>(a, s);
    }
    return launch_generic<float, 2, false, true, 32, 16, 256>(a, s);
  }
  if (m.reservoir) return launch_generic<float, 2, true, false, 32, 16, 256>(a, s);
  return launch_generic<float, 2, false, false, 32, 16, 256>(a, s);
}

}  // namespace phx
