// Host-side building blocks shared by single handles and batches: parameter
// validation and the RK4 stability limit, step coefficients, the padded
// device layout, uploads / downloads with ghost-ring refresh, reduction
// arguments and the persistent kernel's instance descriptor.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/phx.h"
#include "phx_internal.h"
#include "rk4_tma.h"

namespace phx {

// Largest |eigenvalue| of the linear Hermitian operator -kappa Lap (+ TE-TM)
// over the grid's modes: periodic axis phases 2 pi m/N, zero axis Dirichlet
// phases pi m/(N+1).  K^2 = (2 - 2cos a)/d^2, s^2 = sin^2(a)/d^2; the TE-TM
// 2x2 block at a mode has eigenvalues kappa(Kx^2+Ky^2) +- Delta
// sqrt((Kx^2-Ky^2)^2 + 4 sx^2 sy^2).
double spectral_radius(const phx_params& p) {
  auto axis = [](int N, int bc, double d, std::vector<double>& K2,
                 std::vector<double>& s2) {
    const double pi = 3.14159265358979323846;
    if (bc == PHX_BC_PERIODIC) {
      for (int m = 0; m <= N / 2; ++m) {  // phases m and N-m coincide in K2, s2
        double a = 2.0 * pi * m / N;
        K2.push_back((2.0 - 2.0 * std::cos(a)) / (d * d));
        s2.push_back(std::sin(a) * std::sin(a) / (d * d));
      }
    } else {
      for (int m = 1; m <= N; ++m) {
        double a = pi * m / (N + 1);
        K2.push_back((2.0 - 2.0 * std::cos(a)) / (d * d));
        s2.push_back(std::sin(a) * std::sin(a) / (d * d));
      }
    }
  };
  std::vector<double> kx, sx, ky, sy;
  double dx = p.lx / p.nx, dy = p.ly / p.ny;
  axis(p.nx, p.bc_x, dx, kx, sx);
  axis(p.ny, p.bc_y, dy, ky, sy);
  const double kap = p.hbar2_over_2m;
  if (!(p.spinor && p.delta_lt != 0.0)) {
    double mx = 0, my = 0;
    for (double v : kx) mx = std::fmax(mx, v);
    for (double v : ky) my = std::fmax(my, v);
    return std::fabs(kap) * (mx + my);
  }
  const double D = std::fabs(p.delta_lt);
  double best = 0.0;
  for (size_t j = 0; j < ky.size(); ++j)
    for (size_t i = 0; i < kx.size(); ++i) {
      double lam = kap * (kx[i] + ky[j]);
      double dd = kx[i] - ky[j];
      double off = D * std::sqrt(dd * dd + 4.0 * sx[i] * sy[j]);
      best = std::fmax(best, std::fmax(std::fabs(lam + off), std::fabs(lam - off)));
    }
  return best;
}

const char* check_params(const phx_params* p, double* dtmax_out) {
  if (!p) return "params is NULL";
  if (p->struct_size != sizeof(phx_params))
    return "params.struct_size mismatch (call phx_params_init)";
  if (p->nx < 1 || p->ny < 1) return "nx, ny must be >= 1";
  if ((long long)p->nx * p->ny > (1ll << 31) - 1) return "nx*ny must be < 2^31";
  if (!(p->lx > 0) || !(p->ly > 0) || !std::isfinite(p->lx) || !std::isfinite(p->ly))
    return "lx, ly must be positive and finite";
  if ((p->bc_x != PHX_BC_PERIODIC && p->bc_x != PHX_BC_ZERO) ||
      (p->bc_y != PHX_BC_PERIODIC && p->bc_y != PHX_BC_ZERO))
    return "bc_x, bc_y must be PHX_BC_PERIODIC or PHX_BC_ZERO";
  if (p->precision != 32 && p->precision != 64) return "precision must be 32 or 64";
  if ((p->spinor != 0 && p->spinor != 1) || (p->reservoir != 0 && p->reservoir != 1))
    return "spinor and reservoir must be 0 or 1";
  const double c[] = {p->hbar2_over_2m, p->g, p->g_x, p->g_r, p->R, p->gamma_c,
                      p->gamma_r, p->delta_lt, p->dt, p->noise_var, p->wigner_nu, p->drive_omega};
  for (double v : c)
    if (!std::isfinite(v)) return "coefficients must be finite";
  if (p->hbar2_over_2m < 0) return "hbar2_over_2m must be >= 0";
  if (!p->spinor && (p->g_x != 0.0 || p->delta_lt != 0.0)) return "g_x and delta_lt need spinor = 1";
  if (p->noise_var < 0) return "noise_var must be >= 0";
  if (p->wigner_nu < 0) return "wigner_nu must be >= 0";
  if (p->integrator != PHX_INTEGRATOR_RK4 && p->integrator != PHX_INTEGRATOR_SPLIT)
    return "integrator must be PHX_INTEGRATOR_RK4 or PHX_INTEGRATOR_SPLIT";
  double lam = spectral_radius(*p);
  double dtmax = lam > 0 ? 2.0 * std::sqrt(2.0) * HBAR / lam : INFINITY;
  if (dtmax_out) *dtmax_out = dtmax;
  return nullptr;
}

Coeffs make_coeffs(const phx_params& p) {
  Coeffs k;
  const double dx = p.lx / p.nx, dy = p.ly / p.ny;
  const double kh = p.hbar2_over_2m / HBAR;
  k.ax = -kh / (dx * dx);
  k.ay = -kh / (dy * dy);
  k.a0 = 2.0 * kh * (1.0 / (dx * dx) + 1.0 / (dy * dy));
  k.g = p.g / HBAR;
  k.gx = p.g_x / HBAR;
  k.gr = p.g_r / HBAR;
  k.inv_hbar = 1.0 / HBAR;
  k.half_R = 0.5 * p.R;
  k.half_gc = 0.5 * p.gamma_c;
  k.R_ = p.R;
  k.gamma_r = p.gamma_r;
  k.tx = p.delta_lt / (HBAR * dx * dx);
  k.ty = p.delta_lt / (HBAR * dy * dy);
  k.txy = p.delta_lt / (2.0 * HBAR * dx * dy);
  k.dt = p.dt;
  k.dt6 = p.dt / 6.0;
  if (p.wigner_nu > 0.0) {
    // truncated-Wigner renormalisation |psi|^2 -> |psi|^2 - 1/dV in the Kerr,
    // cross-Kerr and depletion terms: constant shifts of the diagonal
    const double w = 1.0 / (dx * dy);
    k.a0 -= (p.g + (p.spinor ? p.g_x : 0.0)) * w / HBAR;
    k.gamma_r -= p.R * w;
  }
  return k;
}

NoiseKey make_noise_key(const phx_params& p) {
  NoiseKey z;
  z.seed = p.seed;
  z.instance = p.instance;
  z.on = p.noise_var > 0.0 || p.wigner_nu > 0.0;
  z.scale = (float)std::sqrt(p.noise_var / 2.0);
  z.twa = p.wigner_nu > 0.0;
  const double dx = p.lx / p.nx, dy = p.ly / p.ny;
  z.kw = (float)(p.wigner_nu * p.dt / (2.0 * dx * dy));
  z.R = (float)p.R;
  z.gc = (float)p.gamma_c;
  z.var = (float)p.noise_var;
  return z;
}

Geometry padded_geometry(const phx_params& p) {
  Geometry g;
  g.nx = p.nx;
  g.ny = p.ny;
  g.pitch = ((p.nx + 2 * HALO + PITCH_ALIGN - 1) / PITCH_ALIGN) * PITCH_ALIGN;
  g.prow = p.ny + 2 * HALO;
  g.plane = (long long)g.pitch * g.prow;
  g.bc_x = p.bc_x;
  g.bc_y = p.bc_y;
  return g;
}

// Copy a user array (nplanes planes of ny x nx elements of `elem` bytes) into
// the padded interior of `dst`, then refresh the ghost ring.
cudaError_t upload_field(void* dst, const void* src, int nplanes, size_t elem,
                         const Geometry& g, int on_device, cudaStream_t s) {
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  for (int c = 0; c < nplanes; ++c) {
    char* d = static_cast<char*>(dst) + ((size_t)c * g.plane + (size_t)HALO * g.pitch + HALO) * elem;
    const char* sp = static_cast<const char*>(src) + (size_t)c * g.nx * g.ny * elem;
    cudaError_t e = cudaMemcpy2DAsync(d, (size_t)g.pitch * elem, sp, (size_t)g.nx * elem,
                                      (size_t)g.nx * elem, g.ny, kind, s);
    if (e != cudaSuccess) return e;
  }
  return launch_fill_ghosts(dst, (int)elem, nplanes, g, s);
}

cudaError_t download_field(void* dst, const void* src, int nplanes, size_t elem,
                           const Geometry& g, int on_device, cudaStream_t s) {
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  for (int c = 0; c < nplanes; ++c) {
    const char* sp = static_cast<const char*>(src) +
                     ((size_t)c * g.plane + (size_t)HALO * g.pitch + HALO) * elem;
    char* d = static_cast<char*>(dst) + (size_t)c * g.nx * g.ny * elem;
    cudaError_t e = cudaMemcpy2DAsync(d, (size_t)g.nx * elem, sp, (size_t)g.pitch * elem,
                                      (size_t)g.nx * elem, g.ny, kind, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

ReduceArgs reduce_args(const phx_params& p, const Geometry& g, const void* psi, const void* n,
                       const void* P, long long P_stride, const void* V) {
  ReduceArgs r;
  const double dx = p.lx / p.nx, dy = p.ly / p.ny;
  r.geo = g;
  r.psi = psi;
  r.n = n;
  r.P = P;
  r.P_comp_stride = P_stride;
  r.V = V;
  r.idx2 = 1.0 / (dx * dx);
  r.idy2 = 1.0 / (dy * dy);
  r.ixy4 = 1.0 / (4.0 * dx * dy);
  r.kappa = p.hbar2_over_2m;
  r.g = p.g;
  r.g_x = p.g_x;
  r.g_r = p.g_r;
  r.delta_lt = p.delta_lt;
  r.R = p.R;
  r.gamma_c = p.gamma_c;
  r.gamma_r = p.gamma_r;
  r.precision = p.precision;
  r.ncomp = p.spinor ? 2 : 1;
  r.reservoir = p.reservoir;
  r.tetm = (p.spinor && p.delta_lt != 0.0) ? 1 : 0;
  return r;
}

bool fill_tile_inst(TileInst& I, const phx_params& p, const Geometry& g, void* const psi[2],
                    void* const n[2], void* P, void* V, int tile_cfg, void* E) {
  TmaBox b = tma_box(tile_cfg);
  const int nc = p.spinor ? 2 : 1;
  std::memset(&I, 0, sizeof I);
  for (int k = 0; k < 2; ++k) {
    // the two-component kernel fetches both component planes in one box
    if (!encode_map_f32(&I.psi[k], psi[k], 2ull * g.pitch, g.prow, nc,
                        (unsigned long long)g.pitch * 8, (unsigned long long)g.plane * 8,
                        b.psi_w, b.psi_h, nc))
      return false;
    I.psi_buf[k] = static_cast<float2*>(psi[k]);
    if (p.reservoir) {
      if (!encode_map_f32(&I.n[k], n[k], g.pitch, g.prow, nc, (unsigned long long)g.pitch * 4,
                          (unsigned long long)g.plane * 4, b.f_w, b.f_h, nc))
        return false;
      I.n_buf[k] = static_cast<float*>(n[k]);
    }
  }
  if (p.reservoir &&
      !encode_map_f32(&I.P, P, g.pitch, g.prow, nc, (unsigned long long)g.pitch * 4,
                      (unsigned long long)g.plane * 4, b.f_w, b.f_h, nc))
    return false;
  if (V && !encode_map_f32(&I.V, V, g.pitch, g.prow, 1, (unsigned long long)g.pitch * 4,
                           (unsigned long long)g.plane * 4, b.f_w, b.f_h))
    return false;
  if (E) {  // Re and Im planes of the drive (component 0)
    float* er = static_cast<float*>(E);
    if (!encode_map_f32(&I.Er, er, g.pitch, g.prow, 1, (unsigned long long)g.pitch * 4,
                        (unsigned long long)g.plane * 4, b.f_w, b.f_h) ||
        !encode_map_f32(&I.Ei, er + g.plane, g.pitch, g.prow, 1, (unsigned long long)g.pitch * 4,
                        (unsigned long long)g.plane * 4, b.f_w, b.f_h))
      return false;
  }
  I.omega = p.drive_omega;
  I.geo = g;
  I.k = cast_coeffs<float>(make_coeffs(p));
  I.noise = make_noise_key(p);
  I.dt64 = p.dt;
  I.tiles_x = (g.nx + 1 + b.tx - 1) / b.tx;
  I.tiles_y = (g.ny + b.ty - 1) / b.ty;
  I.tile0 = 0;
  return true;
}

}  // namespace phx
