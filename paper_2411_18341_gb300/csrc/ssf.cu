// Split-step Fourier integrator (the conventional alternative to RK4 the
// paper's conclusions name; no details given): Strang splitting
//   psi <- L(dt/2) K(dt) L(dt/2) psi
// of a field without reservoir (scalar, or two components), with the exact
// local propagator
//   L(tau) psi_c = psi_c e^{-gamma_c tau/2} exp(-(i/hbar)(V tau + (g|psi_c|^2 + g_x|psi_o|^2) F)),
//   F = (1 - e^{-gamma_c tau}) / gamma_c   (F = tau without loss),
// which holds because every |psi_c|^2 only decays under the local equation,
// and the exact linear propagator applied in Fourier space (cuFFT, via the
// FFT pair of kfilter.cu): exp(-(i/hbar) kappa k^2 tau) per component, times
// the exponential of the TE-TM block [[0, a], [a*, 0]], a = -Delta_LT (k_x - i k_y)^2,
// i.e. cos(th) - i sin(th) [[0, u], [u*, 0]], th = Delta_LT k^2 tau / hbar,
// u = a / |a|, for two components.  The second local
// half step of each step also adds the step's noise (same Philox stream as
// the RK4 path) and advances the FP64 device clock.
#include "phx_noise.cuh"
#include "ssf.h"

namespace phx {

namespace {

__device__ __forceinline__ int fft_index_ssf(int i, int n) { return i <= (n - 1) / 2 ? i : i - n; }

template <typename R, typename C, int NC>
__global__ void ssf_local_kernel(C* psi, Geometry g, const R* V, R gF, R gxF, R tau_h, R damp,
                                 NoiseKey nz, DevClock* clock, int parity, int last,
                                 double dt64) {
  const long long sites = (long long)g.nx * g.ny;
  const long long step = clock->step[parity];
  if (last && blockIdx.x == 0 && threadIdx.x == 0) {
    clock->step[parity ^ 1] = step + 1;
    clock->t[parity ^ 1] = clock->t[parity] + dt64;
  }
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < sites;
       t += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(t / g.nx), i = (int)(t - (long long)j * g.nx);
    const long long off = (long long)(j + HALO) * g.pitch + i + HALO;
    C v[NC];
    R a[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      v[c] = psi[c * g.plane + off];
      a[c] = v[c].x * v[c].x + v[c].y * v[c].y;
    }
    float2 xi[2];
    if (last && nz.on) nz_site(nz.seed, nz.instance, step, (uint32_t)t, nz.scale, xi[0], xi[1], NC == 2);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      // angle of exp(-(i/hbar)(V tau + (g|psi_c|^2 + g_x|psi_o|^2) F)):
      // gF = g F / hbar, gxF = g_x F / hbar, tau_h = tau / hbar
      R ph = gF * a[c];
      if (NC == 2) ph += gxF * a[NC - 1 - c];
      if (V) ph += tau_h * V[off];
      R sn, cs;
      sincos(ph, &sn, &cs);
      C o;
      o.x = damp * (v[c].x * cs + v[c].y * sn);
      o.y = damp * (v[c].y * cs - v[c].x * sn);
      if (last && nz.on) {
        o.x = o.x + R(xi[c].x);
        o.y = o.y + R(xi[c].y);
      }
      psi[c * g.plane + off] = o;
    }
  }
}

template <typename R, typename C, int NC>
__global__ void ssf_kinetic_kernel(C* d, int nx, int ny, R dkx, R dky, R c, R cd, R scale) {
  const long long total = (long long)nx * ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(t / nx), i = (int)(t - (long long)j * nx);
    const R kx = dkx * R(fft_index_ssf(i, nx)), ky = dky * R(fft_index_ssf(j, ny));
    const R k2 = ky * ky + kx * kx;
    R sn, cs;
    sincos(c * k2, &sn, &cs);  // exp(-i c k^2) = cs - i sn
    C f[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) f[q] = d[q * total + t];
    if (NC == 2 && cd != R(0) && k2 > R(0)) {
      // cos(th) f - i sin(th) [[0, u], [u*, 0]] f,  u = -(k_x - i k_y)^2 / k^2
      R st, ct;
      sincos(cd * k2, &st, &ct);
      const R ur = -(kx * kx - ky * ky) / k2, ui = R(2) * kx * ky / k2;
      const C w0 = {ur * f[1].x - ui * f[1].y, ur * f[1].y + ui * f[1].x};  // u f_-
      const C w1 = {ur * f[0].x + ui * f[0].y, ur * f[0].y - ui * f[0].x};  // u* f_+
      const C g0 = {ct * f[0].x + st * w0.y, ct * f[0].y - st * w0.x};
      const C g1 = {ct * f[1].x + st * w1.y, ct * f[1].y - st * w1.x};
      f[0] = g0;
      f[NC - 1] = g1;
    }
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      C o;
      o.x = scale * (f[q].x * cs + f[q].y * sn);
      o.y = scale * (f[q].y * cs - f[q].x * sn);
      d[q * total + t] = o;
    }
  }
}

// Imaginary time (t -> -i tau, conservative part): real factors
// exp(-(g|psi|^2 + V) tau / hbar) locally and exp(-kappa k^2 tau / hbar) in
// Fourier space.
template <typename R, typename C, int NC>
__global__ void imag_local_kernel(C* psi, Geometry g, const R* V, R cg, R cgx, R cv) {
  const long long sites = (long long)g.nx * g.ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < sites;
       t += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(t / g.nx), i = (int)(t - (long long)j * g.nx);
    const long long off = (long long)(j + HALO) * g.pitch + i + HALO;
    C v[NC];
    R a[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      v[c] = psi[c * g.plane + off];
      a[c] = v[c].x * v[c].x + v[c].y * v[c].y;
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      R e = cg * a[c];
      if (NC == 2) e += cgx * a[NC - 1 - c];
      if (V) e += cv * V[off];
      const R f = exp(-e);
      v[c].x *= f;
      v[c].y *= f;
      psi[c * g.plane + off] = v[c];
    }
  }
}

// exp(-H_k tau / hbar): e^{-c k^2} per component and, for two components,
// cosh(th) - sinh(th) [[0, u], [u*, 0]], th = cd k^2, u = -(k_x - i k_y)^2 / k^2.
template <typename R, typename C, int NC>
__global__ void imag_kinetic_kernel(C* d, int nx, int ny, R dkx, R dky, R c, R cd, R scale) {
  const long long total = (long long)nx * ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(t / nx), i = (int)(t - (long long)j * nx);
    const R kx = dkx * R(fft_index_ssf(i, nx)), ky = dky * R(fft_index_ssf(j, ny));
    const R k2 = ky * ky + kx * kx;
    const R f = scale * exp(-c * k2);
    C v[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) v[q] = d[q * total + t];
    if (NC == 2 && cd != R(0) && k2 > R(0)) {
      const R ch = cosh(cd * k2), sh = sinh(cd * k2);
      const R ur = -(kx * kx - ky * ky) / k2, ui = R(2) * kx * ky / k2;
      const C w0 = {ur * v[1].x - ui * v[1].y, ur * v[1].y + ui * v[1].x};  // u f_-
      const C w1 = {ur * v[0].x + ui * v[0].y, ur * v[0].y - ui * v[0].x};  // u* f_+
      const C g0 = {ch * v[0].x - sh * w0.x, ch * v[0].y - sh * w0.y};
      const C g1 = {ch * v[1].x - sh * w1.x, ch * v[1].y - sh * w1.y};
      v[0] = g0;
      v[NC - 1] = g1;
    }
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      v[q].x *= f;
      v[q].y *= f;
      d[q * total + t] = v[q];
    }
  }
}

constexpr int RED_BLOCKS = 512, RED_THREADS = 256;

// Block partials of sum |psi|^2 (FP64, fixed grid and order: deterministic).
template <typename C>
__global__ void __launch_bounds__(RED_THREADS) sumsq_kernel(const C* psi, Geometry g, int ncomp,
                                                             double* partials) {
  __shared__ double sh[RED_THREADS / 32];
  const long long sites = (long long)g.nx * g.ny;
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < sites;
       t += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(t / g.nx), i = (int)(t - (long long)j * g.nx);
    for (int c = 0; c < ncomp; ++c) {
      const C v = psi[c * g.plane + (long long)(j + HALO) * g.pitch + i + HALO];
      acc += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < RED_THREADS / 32; ++w) s += sh[w];
    partials[blockIdx.x] = s;
  }
}

// Sum of the block partials in a fixed order (every caller the same way).
__device__ __forceinline__ double sum_partials(const double* partials) {
  double s = 0.0;
  for (int b = 0; b < RED_BLOCKS; ++b) s += partials[b];
  return s;
}

__global__ void store_target_kernel(const double* partials, double* target) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *target = sum_partials(partials);
}

// psi *= sqrt(target / sum): the norm back to its value at the start.
template <typename R, typename C>
__global__ void rescale_kernel(C* psi, Geometry g, int ncomp, const double* partials,
                               const double* target) {
  __shared__ R f;
  if (threadIdx.x == 0) f = (R)sqrt(*target / sum_partials(partials));
  __syncthreads();
  const long long sites = (long long)g.nx * g.ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < sites;
       t += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(t / g.nx), i = (int)(t - (long long)j * g.nx);
    const long long off = (long long)(j + HALO) * g.pitch + i + HALO;
    for (int c = 0; c < ncomp; ++c) {
      C v = psi[c * g.plane + off];
      v.x *= f;
      v.y *= f;
      psi[c * g.plane + off] = v;
    }
  }
}

// Local part with the reservoir (no closed form): one classical RK4 step of
// length tau of, per site and component,
//   dpsi_c/dt = (-(i/hbar)(V + g|psi_c|^2 + g_x|psi_o|^2 + g_r n_c) + (R n_c - gamma_c)/2) psi_c,
//   dn_c/dt = P_c - (gamma_r + R|psi_c|^2) n_c,
// in place; with `last` also the step's noise and the clock update.
// Coefficients arrive in the stencil precision (a double-to-float conversion
// per thread would run on the narrow FP64 pipe).
template <typename R>
struct LocalRes {
  R g, gx, gr, ih;    // g/hbar, g_x/hbar, g_r/hbar, 1/hbar (multiplies V)
  R hR, hgc, Rg, gam; // R/2, gamma_c/2, R, gamma_r
  R tau;
};

template <typename R, typename C, int NC>
__global__ void ssf_local_res_kernel(C* psi, R* n, const R* P, long long P_stride, Geometry g,
                                     const R* V, LocalRes<R> q, NoiseKey nz, DevClock* clock,
                                     int parity, int last, double dt64) {
  const long long sites = (long long)g.nx * g.ny;
  const long long step = clock->step[parity];
  if (last && blockIdx.x == 0 && threadIdx.x == 0) {
    clock->step[parity ^ 1] = step + 1;
    clock->t[parity ^ 1] = clock->t[parity] + dt64;
  }
  const R cg = q.g, cgx = q.gx, cgr = q.gr, cih = q.ih;
  const R hR = q.hR, hgc = q.hgc, cR = q.Rg, cgam = q.gam, tau = q.tau;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < sites;
       t += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(t / g.nx), i = (int)(t - (long long)j * g.nx);
    const long long off = (long long)(j + HALO) * g.pitch + i + HALO;
    const R vloc = V ? cih * V[off] : R(0);
    C u0[NC];
    R m0[NC], Pc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      u0[c] = psi[c * g.plane + off];
      m0[c] = n[c * g.plane + off];
      Pc[c] = P[c * P_stride + off];
    }
    C u[NC], au[NC];
    R m[NC], am[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      u[c] = u0[c];
      m[c] = m0[c];
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const R w = (s == 0 || s == 3) ? R(1) : R(2);
      const R cs = (s == 2) ? tau : R(0.5) * tau;
      R a[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) a[c] = u[c].x * u[c].x + u[c].y * u[c].y;
      C ku[NC];
      R km[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        R loc = cg * a[c] + cgr * m[c] + vloc;
        if (NC == 2) loc += cgx * a[NC - 1 - c];
        const R G = hR * m[c] - hgc;
        ku[c].x = loc * u[c].y + G * u[c].x;
        ku[c].y = -loc * u[c].x + G * u[c].y;
        km[c] = Pc[c] - (cgam + cR * a[c]) * m[c];
        if (s == 0) {
          au[c] = ku[c];
          am[c] = km[c];
        } else {
          au[c].x += w * ku[c].x;
          au[c].y += w * ku[c].y;
          am[c] += w * km[c];
        }
      }
      if (s < 3) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          u[c].x = u0[c].x + cs * ku[c].x;
          u[c].y = u0[c].y + cs * ku[c].y;
          m[c] = m0[c] + cs * km[c];
        }
      }
    }
    float2 xi[2];
    if (last && nz.on) nz_site(nz.seed, nz.instance, step, (uint32_t)t, nz.scale, xi[0], xi[1], NC == 2);
    const R t6 = tau / R(6);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      C o;
      o.x = u0[c].x + t6 * au[c].x;
      o.y = u0[c].y + t6 * au[c].y;
      if (last && nz.on) {
        o.x = o.x + R(xi[c].x);
        o.y = o.y + R(xi[c].y);
      }
      psi[c * g.plane + off] = o;
      n[c * g.plane + off] = m0[c] + t6 * am[c];
    }
  }
}

int grid_for(long long n) {
  const long long b = (n + 255) / 256;
  return (int)(b < 8192 ? (b < 1 ? 1 : b) : 8192);
}

template <typename R, typename C, int NC>
const char* ssf_step_t(FftPair& fft, void* psi, const Geometry& g, const void* V,
                       const SsfCoeffs& k, const NoiseKey& nz, DevClock* clock, int parity,
                       cudaStream_t s) {
  C* p = static_cast<C*>(psi);
  const R* v = static_cast<const R*>(V);
  const int blocks = grid_for((long long)g.nx * g.ny);
  ssf_local_kernel<R, C, NC><<<blocks, 256, 0, s>>>(p, g, v, (R)k.gF_half, (R)k.gxF_half,
                                                    (R)k.tau_half_h, (R)k.damp_half, nz, clock,
                                                    parity, 0, k.dt);
  count_launch();
  const char* msg = fft_transform(fft, psi, g, sizeof(R) == 8 ? 64 : 32, true, s);
  if (msg) return msg;
  ssf_kinetic_kernel<R, C, NC><<<blocks, 256, 0, s>>>(static_cast<C*>(fft.scratch), g.nx, g.ny,
                                                      (R)k.dkx, (R)k.dky, (R)k.kin, (R)k.tetm,
                                                      (R)k.scale);
  count_launch();
  msg = fft_transform(fft, psi, g, sizeof(R) == 8 ? 64 : 32, false, s);
  if (msg) return msg;
  ssf_local_kernel<R, C, NC><<<blocks, 256, 0, s>>>(p, g, v, (R)k.gF_half, (R)k.gxF_half,
                                                    (R)k.tau_half_h, (R)k.damp_half, nz, clock,
                                                    parity, 1, k.dt);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? nullptr : "split-step kernel launch failed";
}

template <typename R, typename C, int NC>
const char* imag_steps_t(FftPair& fft, double* red, void* psi, const Geometry& g, const void* V,
                         const phx_params& p, long long nsteps, cudaStream_t s) {
  C* ps = static_cast<C*>(psi);
  const R* v = static_cast<const R*>(V);
  const int blocks = grid_for((long long)g.nx * g.ny);
  const int prec = sizeof(R) == 8 ? 64 : 32;
  const double pi = 3.14159265358979323846;
  const R cg = (R)(p.g * 0.5 * p.dt / HBAR), cgx = (R)(p.g_x * 0.5 * p.dt / HBAR);
  const R cv = (R)(0.5 * p.dt / HBAR);
  const R ck = (R)(p.hbar2_over_2m * p.dt / HBAR), cd = (R)(p.delta_lt * p.dt / HBAR);
  const R dkx = (R)(2.0 * pi / p.lx), dky = (R)(2.0 * pi / p.ly);
  const R scale = (R)(1.0 / ((double)p.nx * p.ny));
  double* partials = red;
  double* target = red + RED_BLOCKS;
  sumsq_kernel<C><<<RED_BLOCKS, RED_THREADS, 0, s>>>(ps, g, NC, partials);
  store_target_kernel<<<1, 32, 0, s>>>(partials, target);
  count_launch(2);
  for (long long k = 0; k < nsteps; ++k) {
    imag_local_kernel<R, C, NC><<<blocks, 256, 0, s>>>(ps, g, v, cg, cgx, cv);
    count_launch();
    const char* msg = fft_transform(fft, psi, g, prec, true, s);
    if (msg) return msg;
    imag_kinetic_kernel<R, C, NC><<<blocks, 256, 0, s>>>(static_cast<C*>(fft.scratch), g.nx,
                                                         g.ny, dkx, dky, ck, cd, scale);
    count_launch();
    msg = fft_transform(fft, psi, g, prec, false, s);
    if (msg) return msg;
    imag_local_kernel<R, C, NC><<<blocks, 256, 0, s>>>(ps, g, v, cg, cgx, cv);
    sumsq_kernel<C><<<RED_BLOCKS, RED_THREADS, 0, s>>>(ps, g, NC, partials);
    rescale_kernel<R, C><<<blocks, 256, 0, s>>>(ps, g, NC, partials, target);
    count_launch(3);
  }
  return cudaGetLastError() == cudaSuccess ? nullptr : "imaginary-time kernel launch failed";
}

template <typename R, typename C, int NC>
const char* ssf_res_step_t(FftPair& fft, void* psi, void* n, const void* P, long long P_stride,
                           const Geometry& g, const void* V, const SsfCoeffs& k,
                           const phx_params& pp_, const NoiseKey& nz, DevClock* clock, int parity,
                           cudaStream_t s) {
  LocalRes<R> q;
  q.g = (R)(pp_.g / HBAR);
  q.gx = (R)(pp_.g_x / HBAR);
  q.gr = (R)(pp_.g_r / HBAR);
  q.ih = (R)(1.0 / HBAR);
  q.hR = (R)(0.5 * pp_.R);
  q.hgc = (R)(0.5 * pp_.gamma_c);
  q.Rg = (R)pp_.R;
  q.gam = (R)pp_.gamma_r;
  q.tau = (R)(0.5 * pp_.dt);
  C* p = static_cast<C*>(psi);
  R* nn = static_cast<R*>(n);
  const R* pp = static_cast<const R*>(P);
  const R* v = static_cast<const R*>(V);
  const int blocks = grid_for((long long)g.nx * g.ny);
  ssf_local_res_kernel<R, C, NC><<<blocks, 256, 0, s>>>(p, nn, pp, P_stride, g, v, q, nz, clock,
                                                        parity, 0, k.dt);
  count_launch();
  const char* msg = fft_transform(fft, psi, g, sizeof(R) == 8 ? 64 : 32, true, s);
  if (msg) return msg;
  ssf_kinetic_kernel<R, C, NC><<<blocks, 256, 0, s>>>(static_cast<C*>(fft.scratch), g.nx, g.ny,
                                                      (R)k.dkx, (R)k.dky, (R)k.kin, (R)k.tetm,
                                                      (R)k.scale);
  count_launch();
  msg = fft_transform(fft, psi, g, sizeof(R) == 8 ? 64 : 32, false, s);
  if (msg) return msg;
  ssf_local_res_kernel<R, C, NC><<<blocks, 256, 0, s>>>(p, nn, pp, P_stride, g, v, q, nz, clock,
                                                        parity, 1, k.dt);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? nullptr : "split-step kernel launch failed";
}

}  // namespace

const char* ssf_step_reservoir(FftPair& fft, void* psi, void* n, const void* P,
                               long long P_stride, const Geometry& g, int precision, int ncomp,
                               const void* V, const phx_params& p, const SsfCoeffs& k,
                               const NoiseKey& nz, DevClock* clock, int parity, cudaStream_t s) {
  if (precision == 64)
    return ncomp == 2 ? ssf_res_step_t<double, double2, 2>(fft, psi, n, P, P_stride, g, V, k, p,
                                                            nz, clock, parity, s)
                      : ssf_res_step_t<double, double2, 1>(fft, psi, n, P, P_stride, g, V, k, p,
                                                            nz, clock, parity, s);
  return ncomp == 2 ? ssf_res_step_t<float, float2, 2>(fft, psi, n, P, P_stride, g, V, k, p, nz,
                                                        clock, parity, s)
                    : ssf_res_step_t<float, float2, 1>(fft, psi, n, P, P_stride, g, V, k, p, nz,
                                                        clock, parity, s);
}

size_t imag_scratch_doubles() { return RED_BLOCKS + 1; }

const char* imag_steps(FftPair& fft, double* red, void* psi, const Geometry& g, int precision,
                       const void* V, const phx_params& p, long long nsteps, cudaStream_t s) {
  const bool two = p.spinor != 0;
  if (precision == 64)
    return two ? imag_steps_t<double, double2, 2>(fft, red, psi, g, V, p, nsteps, s)
               : imag_steps_t<double, double2, 1>(fft, red, psi, g, V, p, nsteps, s);
  return two ? imag_steps_t<float, float2, 2>(fft, red, psi, g, V, p, nsteps, s)
             : imag_steps_t<float, float2, 1>(fft, red, psi, g, V, p, nsteps, s);
}

SsfCoeffs ssf_coeffs(const phx_params& p) {
  SsfCoeffs k;
  const double tau = 0.5 * p.dt;
  const double F = p.gamma_c != 0.0 ? -std::expm1(-p.gamma_c * tau) / p.gamma_c : tau;
  k.gF_half = p.g * F / HBAR;
  k.gxF_half = p.g_x * F / HBAR;
  k.tau_half_h = tau / HBAR;
  k.damp_half = std::exp(-0.5 * p.gamma_c * tau);
  const double pi = 3.14159265358979323846;
  k.dkx = 2.0 * pi / p.lx;
  k.dky = 2.0 * pi / p.ly;
  k.kin = p.hbar2_over_2m * p.dt / HBAR;
  k.tetm = p.delta_lt * p.dt / HBAR;
  k.scale = 1.0 / ((double)p.nx * p.ny);
  k.dt = p.dt;
  return k;
}

const char* ssf_step(FftPair& fft, void* psi, const Geometry& g, int precision, int ncomp,
                     const void* V, const SsfCoeffs& k, const NoiseKey& nz, DevClock* clock,
                     int parity, cudaStream_t s) {
  if (precision == 64)
    return ncomp == 2 ? ssf_step_t<double, double2, 2>(fft, psi, g, V, k, nz, clock, parity, s)
                      : ssf_step_t<double, double2, 1>(fft, psi, g, V, k, nz, clock, parity, s);
  return ncomp == 2 ? ssf_step_t<float, float2, 2>(fft, psi, g, V, k, nz, clock, parity, s)
                    : ssf_step_t<float, float2, 1>(fft, psi, g, V, k, nz, clock, parity, s);
}

}  // namespace phx
