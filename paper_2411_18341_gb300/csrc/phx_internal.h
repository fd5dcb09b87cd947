// Internal declarations shared by the host runtime and the kernels.
// Device layout of every field: ncomp planes of (ny + 2*HALO) rows x pitch
// columns, domain site (i, j) stored at row j + HALO, column i + HALO.  The
// HALO-wide ghost ring holds periodic images (periodic axis) or zeros (zero
// axis), so that a tile with a depth-HALO halo is one rectangular box.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/phx.h"

namespace phx {

constexpr int HALO = 4;       // RK4 needs a depth-4 halo (one cell per stage)
constexpr int PITCH_ALIGN = 32;
constexpr double HBAR = 0.6582119569;  // meV ps (CODATA 2018)
constexpr int BC_PERIODIC = 0;
constexpr int BC_ZERO = 1;

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

// Step counter and FP64 simulated time, double-buffered by step parity so a
// launch can read slot p and write slot p^1 without a grid-wide barrier.
struct DevClock {
  long long step[2];
  double t[2];
};

struct Geometry {
  int nx, ny;        // domain
  int pitch;         // padded row length (elements)
  int prow;          // padded rows = ny + 2*HALO
  long long plane;   // pitch * prow
  int bc_x, bc_y;
};

// Coefficients of one RK4 step, pre-scaled by 1/hbar (units ps^-1), in the
// stencil precision R (converted once on the host: a double-to-float
// conversion inside a kernel runs on the FP64 pipe, which is narrow on GB300).
template <typename R>
struct CoeffsT {
  R ax, ay, a0;      // -(k/h)/dx^2, -(k/h)/dy^2, 2(k/h)(1/dx^2 + 1/dy^2)
  R g, gx, gr;       // g/h, g_x/h, g_r/h
  R inv_hbar;        // multiplies V
  R half_R, half_gc; // R/2, gamma_c/2
  R R_, gamma_r;
  R tx, ty, txy;     // Delta/(h dx^2), Delta/(h dy^2), Delta/(2 h dx dy)
  R dt;
  R dt6;             // dt/6 in this precision (the final RK4 combination)
};
using Coeffs = CoeffsT<double>;

template <typename R>
inline CoeffsT<R> cast_coeffs(const Coeffs& c) {
  CoeffsT<R> o;
  o.ax = (R)c.ax; o.ay = (R)c.ay; o.a0 = (R)c.a0;
  o.g = (R)c.g; o.gx = (R)c.gx; o.gr = (R)c.gr;
  o.inv_hbar = (R)c.inv_hbar;
  o.half_R = (R)c.half_R; o.half_gc = (R)c.half_gc;
  o.R_ = (R)c.R_; o.gamma_r = (R)c.gamma_r;
  o.tx = (R)c.tx; o.ty = (R)c.ty; o.txy = (R)c.txy;
  o.dt = (R)c.dt;
  o.dt6 = o.dt / (R)6;  // IEEE division in R: the value a kernel would compute
  return o;
}

struct NoiseKey {
  unsigned long long seed;
  unsigned int instance;
  int on;                 // noise_var > 0 or wigner_nu > 0
  float scale;            // float32(sqrt(noise_var/2)), the fixed-variance mode
  int twa;                // truncated-Wigner variance per site (nu > 0)
  float kw;               // float32(nu dt / (2 dx dy))
  float R, gc, var;       // float32 R, gamma_c, noise_var
};

template <typename R>
struct StepArgs {
  Geometry geo;
  const typename Cx<R>::T* psi_in;
  typename Cx<R>::T* psi_out;
  const R* n_in;
  R* n_out;
  const R* P;             // ncomp planes (plane 1 may alias plane 0)
  long long P_comp_stride;
  const R* V;             // nullptr when absent
  // coherent drive amplitude E_c(r), meV, as split planes: Re E_c at
  // E + c * E_comp_stride, Im E_c one plane further; nullptr when absent
  const R* E = nullptr;
  long long E_comp_stride = 0;           // 2 * plane, or 0 when both components share E_+
  double omega = 0.0;                    // drive angular frequency, rad/ps
  CoeffsT<R> k;
  double dt64;            // FP64 time step for the simulated-time accumulator
  NoiseKey noise;
  DevClock* clock;
  int parity;
  int inject_timeout;     // test hook: leave the first tile's barrier unarmed
};

struct ModelKey {
  int precision;  // 32 | 64
  int ncomp;      // 1 | 2
  int reservoir;  // 0 | 1
  int tetm;       // 0 | 1
};

// ---- launchers (return cudaGetLastError() after the launch) -------------
cudaError_t launch_rk4_step_f32(const ModelKey& m, const StepArgs<float>& a,
                                cudaStream_t s, int tile);
cudaError_t launch_rk4_step_f64(const ModelKey& m, const StepArgs<double>& a,
                                cudaStream_t s, int tile);

// Split `nplanes` padded planes of interleaved complex values (real element
// size esize) into a real and an imaginary plane each (dst planes 2c, 2c+1).
cudaError_t launch_split_complex(const void* src, void* dst, int esize, int nplanes,
                                 const Geometry& g, cudaStream_t s);

// Fill the ghost ring of `nplanes` planes of element size `esize` bytes.
cudaError_t launch_fill_ghosts(void* base, int esize, int nplanes,
                               const Geometry& g, cudaStream_t s);

// Reductions in FP64.  `partials` is device scratch of reduce_partials_len()
// doubles; `out` receives the final sums on the device.
int reduce_blocks(const Geometry& g);
size_t reduce_partials_len(const Geometry& g);

struct ReduceArgs {
  Geometry geo;
  const void* psi;   // padded, precision 32 or 64
  const void* n;     // may be nullptr
  const void* P;
  long long P_comp_stride;
  const void* V;
  double idx2, idy2, ixy4;   // 1/dx^2, 1/dy^2, 1/(4 dx dy)
  double kappa, g, g_x, g_r, delta_lt, R, gamma_c, gamma_r;  // physical units
  int precision, ncomp, reservoir, tetm;
};

// out[0] = sum |psi|^2, out[1] = sum of the energy density (both without dV)
cudaError_t launch_norm_energy(const ReduceArgs& a, double* partials,
                               double* out, cudaStream_t s);
// Two passes: out[0]=S_pp, out[1]=Re S_pK, out[2]=Im S_pK, out[3]=S_fn,
// out[4]=S_nn, out[5]=sum|K + i omega psi|^2, out[6]=omega, out[7]=nonfinite
cudaError_t launch_residual(const ReduceArgs& a, double* partials, double* out,
                            cudaStream_t s);

cudaError_t launch_noise_sample(unsigned long long seed, long long step,
                                unsigned int instance, int ncomp, int nx,
                                int ny, float scale, float* out,
                                cudaStream_t s);

// Test hooks armed by phx_debug_inject (consumed by the next matching event).
enum { INJ_ALLOC = 1, INJ_LAUNCH = 2, INJ_TIMEOUT = 4 };
bool take_injection(unsigned what);

// ---- host helpers shared by handles and batches (common.cpp) -------------
// nullptr if *p is valid (and *dtmax = RK4 stability limit), else a message
const char* check_params(const phx_params* p, double* dtmax);
double spectral_radius(const phx_params& p);
Coeffs make_coeffs(const phx_params& p);
NoiseKey make_noise_key(const phx_params& p);
Geometry padded_geometry(const phx_params& p);
cudaError_t upload_field(void* dst, const void* src, int nplanes, size_t elem,
                         const Geometry& g, int on_device, cudaStream_t s);
cudaError_t download_field(void* dst, const void* src, int nplanes, size_t elem,
                           const Geometry& g, int on_device, cudaStream_t s);
ReduceArgs reduce_args(const phx_params& p, const Geometry& g, const void* psi, const void* n,
                       const void* P, long long P_stride, const void* V);

// Process-wide count of kernel launches issued by this library.
void count_launch(unsigned n = 1);

}  // namespace phx
