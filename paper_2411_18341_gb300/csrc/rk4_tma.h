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
  TILE_64x32_M2_2 = 6,  // 2 x 2, 16 warps, two CTAs per SM
  TILE_64x32_M4_2 = 7,  // 4 x 2, 8 warps, two CTAs per SM
  TILE_64x32_M4_2_MS = 8,  // configuration 7, several steps per launch (single handles)
  // two-component field with reservoirs (2 x 2 micro-tiles of both components)
  TILE_SPINOR_64x16 = 21,  // 8 warps
  TILE_SPINOR_64x24 = 22,  // 12 warps
  TILE_SPINOR_64x32 = 23,  // 16 warps
  TILE_GENERIC = 9
};

// One problem instance as the persistent step kernel sees it (device memory,
// read-only during a launch).  A single handle is a one-instance table; a
// batch has one entry per member.  Tensor maps must be 64-byte aligned.
struct alignas(128) TileInst {
  CUtensorMap psi[2];   // load maps of the psi buffers 0 and 1
  CUtensorMap n[2];     // load maps of the n buffers 0 and 1
  CUtensorMap P, V;
  CUtensorMap Er, Ei;   // load maps of the coherent drive's Re / Im planes
  float2* psi_buf[2];   // the psi buffers (outputs go to buffer cur ^ 1)
  float* n_buf[2];
  Geometry geo;
  CoeffsT<float> k;
  NoiseKey noise;
  double dt64;          // FP64 step for the simulated-time accumulator
  double omega;         // drive angular frequency, rad/ps
  int tiles_x, tiles_y; // tiles of this instance for the chosen configuration
  int tile0;            // index of its first tile in the global tile list
};

// The scalar part of one instance, passed by value in the kernel parameters
// when a launch covers a single instance.
struct InstScalars {
  int p_shared;  // two-component field: both components read pump plane 0
  Geometry geo;
  CoeffsT<float> k;
  NoiseKey noise;
  float2* psi_buf[2];
  float* n_buf[2];
  int tiles_x;
};

inline InstScalars scalars_of(const TileInst& I) {
  InstScalars s;
  s.p_shared = 0;
  s.geo = I.geo;
  s.k = I.k;
  s.noise = I.noise;
  s.psi_buf[0] = I.psi_buf[0];
  s.psi_buf[1] = I.psi_buf[1];
  s.n_buf[0] = I.n_buf[0];
  s.n_buf[1] = I.n_buf[1];
  s.tiles_x = I.tiles_x;
  return s;
}

struct TileArgs {
  const TileInst* inst;   // device array of ninst instances
  const int2* tile_info;  // per global tile: (instance, kx | ky << 16); unused if ninst == 1
  InstScalars one;        // scalars of instance 0 (read when ninst == 1)
  int ntiles, ninst;
  int cur;               // input buffer of this step
  DevClock* clock;       // step counter and FP64 time of instance 0
  int parity;
  double* t_inst;        // [2][ninst] FP64 times of all instances, or nullptr
  int* err;              // set when a bounded wait gives up
  int inject_timeout;    // test hook: leave the first tile's barrier unarmed
  // Several steps in one launch (single instance): items (step, tile) in a
  // fixed order, a tile's load issued once its neighbours completed the
  // previous step.  done[ky * tiles_x + kx] = steps of this launch completed
  // by that tile (zeroed before the launch).
  int* done = nullptr;
  int ms_steps = 1;      // steps in this launch
  int tiles_y = 0;
};

struct TmaBox {
  int psi_w, psi_h;  // psi box in floats (interleaved complex) x rows
  int f_w, f_h;      // n / P / V box
  int tx, ty;        // output tile
};

TmaBox tma_box(int tile_cfg);

// Resident CTAs per SM the configuration is built for (the persistent grid
// is this many CTAs per SM).
int tma_ctas_per_sm(int tile_cfg);

bool encode_map_f32(CUtensorMap* map, void* base, unsigned long long w,
                    unsigned long long h, unsigned long long planes,
                    unsigned long long row_bytes, unsigned long long plane_bytes,
                    unsigned box_w, unsigned box_h, unsigned box_d = 1);

// Build the descriptor of one instance (host memory) for a tile
// configuration; false if a tensor map cannot be encoded.
// E: the drive's split Re / Im planes (single-component instances), or nullptr.
bool fill_tile_inst(TileInst& I, const phx_params& p, const Geometry& g, void* const psi[2],
                    void* const n[2], void* P, void* V, int tile_cfg, void* E = nullptr);

// mode: 0 = plain, 1 = reservoir, 2 = coherent drive (single instance).
// per: every instance is periodic in both axes (selects the variant that
// never forces stage values to zero).
cudaError_t launch_rk4_tma_f32(int tile_cfg, int mode, bool pot, bool per, const TileArgs& ta,
                               cudaStream_t s, int grid);

// Two-component field with reservoirs (rk4_tma_spinor.cu); tetm: TE-TM coupling.
cudaError_t launch_rk4_tma_spinor(int tile_cfg, bool pot, bool per, bool tetm,
                                  const TileArgs& ta, cudaStream_t s, int grid);

// One per tile configuration (rk4_tma_cfgN.cu): every model variant of it.
cudaError_t launch_tma_cfg1(int mode, bool pot, bool per, bool one, const TileArgs& ta,
                            cudaStream_t s, int grid);
cudaError_t launch_tma_cfg2(int mode, bool pot, bool per, bool one, const TileArgs& ta,
                            cudaStream_t s, int grid);
cudaError_t launch_tma_cfg3(int mode, bool pot, bool per, bool one, const TileArgs& ta,
                            cudaStream_t s, int grid);
cudaError_t launch_tma_cfg4(int mode, bool pot, bool per, bool one, const TileArgs& ta,
                            cudaStream_t s, int grid);
cudaError_t launch_tma_cfg5(int mode, bool pot, bool per, bool one, const TileArgs& ta,
                            cudaStream_t s, int grid);
cudaError_t launch_tma_cfg6(int mode, bool pot, bool per, bool one, const TileArgs& ta,
                            cudaStream_t s, int grid);
cudaError_t launch_tma_cfg7(int mode, bool pot, bool per, bool one, const TileArgs& ta,
                            cudaStream_t s, int grid);

// Several steps per launch (single instance, mode 0 or 1; ta.done zeroed,
// ta.ms_steps, ta.tiles_y set).  Configurations with such a variant:
bool tma_has_multistep(int tile_cfg);
// Configurations with the reservoir-and-drive variant (mode 3: one CTA per
// SM, two input buffers of six planes within shared memory).
bool tma_has_drive_reservoir(int tile_cfg);
cudaError_t launch_rk4_tma_f32_ms(int tile_cfg, int mode, bool pot, bool per,
                                  const TileArgs& ta, cudaStream_t s, int grid);
cudaError_t launch_tma_cfg7_ms(int mode, bool pot, bool per, const TileArgs& ta, cudaStream_t s,
                               int grid);

// Advance the step counter and FP64 time by nsteps steps (slot parity ->
// parity ^ 1; the time as nsteps sequential additions of dt, like nsteps
// single-step launches).
cudaError_t launch_clock_advance(DevClock* clock, int parity, int nsteps, double dt,
                                 cudaStream_t s);

}  // namespace phx
