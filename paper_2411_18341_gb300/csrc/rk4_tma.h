// Host-side interface of the persistent TMA-fed FP32 scalar RK4 kernel.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "phx_internal.h"

namespace phx {

// Tile configurations (region columns x region rows; output = region - 6).
enum {
  TILE_AUTO = 0,
  TILE_64x64 = 1,     // 4 rows x 2 columns per thread, 16 warps
  TILE_64x48 = 2,     // 4 x 2, 12 warps
  TILE_64x32 = 3,     // 4 x 2, 8 warps
  TILE_64x48_M2 = 4,  // 2 x 2, 24 warps
  TILE_64x64_M2 = 5,  // 2 x 2, 32 warps
  TILE_GENERIC = 9
};

struct TmaMaps {
  CUtensorMap psi, n, P, V;
};

struct TmaBox {
  int psi_w, psi_h;  // psi box in floats (interleaved complex) x rows
  int f_w, f_h;      // n / P / V box
  int tx, ty;        // output tile
};

TmaBox tma_box(int tile_cfg);

bool encode_map_f32(CUtensorMap* map, void* base, unsigned long long w,
                    unsigned long long h, unsigned long long planes,
                    unsigned long long row_bytes, unsigned long long plane_bytes,
                    unsigned box_w, unsigned box_h);

cudaError_t launch_rk4_tma_f32(int tile_cfg, bool res, bool pot, const TmaMaps& m,
                               const StepArgs<float>& a, cudaStream_t s, int* err,
                               int num_sms);

}  // namespace phx
