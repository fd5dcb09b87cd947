// FP64 instantiations of the fused RK4 step.
#include "rk4_generic.cuh"

namespace phx {

cudaError_t launch_rk4_step_f64(const ModelKey& m, const StepArgs<double>& a,
                                cudaStream_t s, int tile) {
  if (m.ncomp == 1) {
    if (m.reservoir) {
      // tile shapes of the scalar reservoir kernel (phx_params.tile 10..12).
      // By default 32 x 32 tiles (less halo recompute: the fastest at 1024^2
      // and 2048^2) once the grid gives every SM several of them, else 16 x 16.
      if (tile == 10) return launch_generic<double, 1, true, false, 32, 16, 256>(a, s);
      if (tile == 11) return launch_generic<double, 1, true, false, 16, 16, 128>(a, s);
      if (tile == 12) return launch_generic<double, 1, true, false, 64, 16, 256>(a, s);
      if ((long long)a.geo.nx * a.geo.ny >= 512LL * 512)
        return launch_generic<double, 1, true, false, 32, 32, 256>(a, s);
      return launch_generic<double, 1, true, false, 16, 16, 128>(a, s);
    }
    return launch_generic<double, 1, false, false, 16, 16, 128>(a, s);
  }
  if (m.tetm) {
    if (m.reservoir) return launch_generic<double, 2, true, true, 16, 16, 128>(a, s);
    return launch_generic<double, 2, false, true, 16, 16, 128>(a, s);
  }
  if (m.reservoir) return launch_generic<double, 2, true, false, 16, 16, 128>(a, s);
  return launch_generic<double, 2, false, false, 16, 16, 128>(a, s);
}

}  // namespace phx
