// Host side of the persistent TMA-fed FP32 scalar step: tile shapes, launch
// dispatch over the per-configuration translation units, tensor-map encoding.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstring>

#include "phx_internal.h"
#include "rk4_tma.h"

namespace phx {

// Box shapes the tensor maps must use for a given tile configuration.
TmaBox tma_box(int tile_cfg) {
  TmaBox b;
  int MR = 4, WY = 16;
  if (tile_cfg == TILE_64x48) WY = 12;
  if (tile_cfg == TILE_64x32) WY = 8;
  if (tile_cfg == TILE_64x48_M2) { MR = 2; WY = 24; }
  if (tile_cfg == TILE_64x64_M2) { MR = 2; WY = 32; }
  if (tile_cfg == TILE_64x32_M2_2) { MR = 2; WY = 16; }
  if (tile_cfg == TILE_64x32_M4_2 || tile_cfg == TILE_64x32_M4_2_MS) { MR = 4; WY = 8; }
  if (tile_cfg == TILE_SPINOR_64x16) { MR = 2; WY = 8; }
  if (tile_cfg == TILE_SPINOR_64x24) { MR = 2; WY = 12; }
  if (tile_cfg == TILE_SPINOR_64x32) { MR = 2; WY = 16; }
  const int RW = 64, RH = MR * WY;
  b.psi_w = 2 * (RW + 4);  // floats (interleaved complex)
  b.psi_h = RH + 2;
  b.f_w = RW + 4;
  b.f_h = RH;
  b.tx = RW - 6;
  b.ty = RH - 6;
  return b;
}

int tma_ctas_per_sm(int tile_cfg) {
  return tile_cfg == TILE_64x32_M2_2 || tile_cfg == TILE_64x32_M4_2 ||
                 tile_cfg == TILE_64x32_M4_2_MS
             ? 2
             : 1;
}

cudaError_t launch_rk4_tma_f32(int tile_cfg, int mode, bool pot, bool per,
                               const TileArgs& ta, cudaStream_t s, int grid) {
  const bool one = ta.ninst == 1;
  switch (tile_cfg) {
    case TILE_64x64: return launch_tma_cfg1(mode, pot, per, one, ta, s, grid);
    case TILE_64x48: return launch_tma_cfg2(mode, pot, per, one, ta, s, grid);
    case TILE_64x32: return launch_tma_cfg3(mode, pot, per, one, ta, s, grid);
    case TILE_64x48_M2: return launch_tma_cfg4(mode, pot, per, one, ta, s, grid);
    case TILE_64x64_M2: return launch_tma_cfg5(mode, pot, per, one, ta, s, grid);
    case TILE_64x32_M2_2: return launch_tma_cfg6(mode, pot, per, one, ta, s, grid);
    case TILE_64x32_M4_2:
    case TILE_64x32_M4_2_MS: return launch_tma_cfg7(mode, pot, per, one, ta, s, grid);
    default: break;
  }
  return cudaErrorInvalidValue;
}

bool tma_has_multistep(int tile_cfg) { return tile_cfg == TILE_64x32_M4_2_MS; }

bool tma_has_drive_reservoir(int tile_cfg) {
  return tile_cfg == TILE_64x48 || tile_cfg == TILE_64x32 || tile_cfg == TILE_64x48_M2;
}

cudaError_t launch_rk4_tma_f32_ms(int tile_cfg, int mode, bool pot, bool per,
                                  const TileArgs& ta, cudaStream_t s, int grid) {
  if (tile_cfg == TILE_64x32_M4_2_MS) return launch_tma_cfg7_ms(mode, pot, per, ta, s, grid);
  return cudaErrorInvalidValue;
}

__global__ void clock_advance_kernel(DevClock* c, int parity, int nsteps, double dt) {
  double t = c->t[parity];
  for (int i = 0; i < nsteps; ++i) t += dt;
  c->t[parity ^ 1] = t;
  c->step[parity ^ 1] = c->step[parity] + nsteps;
}

cudaError_t launch_clock_advance(DevClock* clock, int parity, int nsteps, double dt,
                                 cudaStream_t s) {
  clock_advance_kernel<<<1, 1, 0, s>>>(clock, parity, nsteps, dt);
  count_launch();
  return cudaGetLastError();
}

// ---- tensor-map encoding (driver entry point, no libcuda link needed) -----
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                         cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

bool encode_map_f32(CUtensorMap* map, void* base, unsigned long long w,
                    unsigned long long h, unsigned long long planes,
                    unsigned long long row_bytes, unsigned long long plane_bytes,
                    unsigned box_w, unsigned box_h, unsigned box_d) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {w, h, planes};
  cuuint64_t strides[2] = {row_bytes, plane_bytes};
  cuuint32_t box[3] = {box_w, box_h, box_d};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace phx
