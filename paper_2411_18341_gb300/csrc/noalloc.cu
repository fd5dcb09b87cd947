// Allocation-free FP64 norm and energy: the same quantities as
// phx_norm_energy, computed from caller-owned device arrays in the plain
// (unpadded) layout, with the per-CTA partial sums kept in a fixed,
// file-scope device array instead of memory obtained from cudaMalloc.
//
// This entry point exists for callers that cannot allocate device memory:
// for example a host loop running under a device-memory budget that a
// framework's caching allocator owns completely, or a latency-critical loop
// that must never call into the CUDA allocator (cudaMalloc / cudaFree can
// block on the device).  Such callers cannot create a phx_handle, which
// allocates its state and scratch, but they can still hand in their own
// input and output buffers.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/phx.h"
#include "phx_internal.h"

namespace phx {

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_SITES_PER_THREAD = 16;
constexpr int NA_MAX_BLOCKS = 4096;
// Largest grid the static scratch can reduce: 4096 CTAs x 256 threads x 16
// sites = 2^24 sites (e.g. 4096 x 4096).
constexpr long long NA_MAX_SITES =
    (long long)NA_MAX_BLOCKS * NA_THREADS * NA_SITES_PER_THREAD;
constexpr int NA_MAX_DEVICES = 64;

// Scratch shared by every call on a device: two FP64 partials per CTA plus
// the two final sums (64 KiB + 16 B).  Every slot a call reads is written
// earlier in the same call, so nothing needs clearing between calls; calls
// whose kernels overlap on the GPU (different streams, no ordering) race on
// this array.
__device__ __align__(256) double g_na_scratch[2 * NA_MAX_BLOCKS + 2];

// Device address of the scratch per device, looked up once per device (a
// failed look-up is retried on the next call; the lock keeps threads that
// call at the same time from racing on the slot).
double* g_na_ptr[NA_MAX_DEVICES] = {nullptr};
std::mutex g_na_mu;

__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename R>
struct PlainView {
  const R* psi;  // ncomp planes of ny x nx interleaved complex
  const R* n;
  const R* V;
  int nx, ny, bcx, bcy;
  long long plane;  // nx * ny
  // psi_c at (gx + dx, gy + dy) with the boundary condition; 0 outside a
  // zero-boundary axis
  __device__ double2 ld(int c, int gx, int gy, int dx, int dy) const {
    int x = gx + dx, y = gy + dy;
    if (x < 0 || x >= nx) {
      if (bcx != PHX_BC_PERIODIC) return make_double2(0.0, 0.0);
      x = ((x % nx) + nx) % nx;
    }
    if (y < 0 || y >= ny) {
      if (bcy != PHX_BC_PERIODIC) return make_double2(0.0, 0.0);
      y = ((y % ny) + ny) % ny;
    }
    const R* p = psi + 2 * (c * plane + (long long)y * nx + x);
    return make_double2((double)p[0], (double)p[1]);
  }
};

struct NaPhys {
  double kappa, g, g_x, g_r, delta_lt;
  double idx2, idy2, ixy4;
  int ncomp, reservoir, tetm, has_V;
};

// Per-site norm density sum_c |psi_c|^2 and energy density (the integrand of
// phx_norm_energy's E without the cell area).
template <typename R>
__device__ void na_site(const PlainView<R>& v, const NaPhys& a, int gx, int gy,
                        double& nrm, double& e) {
  double2 pc[2];
  double dens[2], nc[2];
  const long long s = (long long)gy * v.nx + gx;
  for (int c = 0; c < a.ncomp; ++c) {
    pc[c] = v.ld(c, gx, gy, 0, 0);
    dens[c] = pc[c].x * pc[c].x + pc[c].y * pc[c].y;
    nc[c] = a.reservoir ? (double)v.n[c * v.plane + s] : 0.0;
  }
  const double Vs = a.has_V ? (double)v.V[s] : 0.0;
  nrm = 0.0;
  e = 0.0;
  for (int c = 0; c < a.ncomp; ++c) {
    double2 C = pc[c];
    double2 E = v.ld(c, gx, gy, 1, 0), W = v.ld(c, gx, gy, -1, 0);
    double2 N = v.ld(c, gx, gy, 0, 1), S = v.ld(c, gx, gy, 0, -1);
    double lx = (E.x + W.x - 2.0 * C.x) * a.idx2 + (N.x + S.x - 2.0 * C.x) * a.idy2;
    double ly = (E.y + W.y - 2.0 * C.y) * a.idx2 + (N.y + S.y - 2.0 * C.y) * a.idy2;
    // Re(psi^* (-kappa Lap psi)) + (V + g_r n)|psi|^2 + (g/2)|psi|^4
    e += -a.kappa * (C.x * lx + C.y * ly) + (Vs + a.g_r * nc[c]) * dens[c] +
         0.5 * a.g * dens[c] * dens[c];
    nrm += dens[c];
    if (a.tetm) {
      const int o = 1 - c;
      double2 Co = pc[o];
      double2 Eo = v.ld(o, gx, gy, 1, 0), Wo = v.ld(o, gx, gy, -1, 0);
      double2 No = v.ld(o, gx, gy, 0, 1), So = v.ld(o, gx, gy, 0, -1);
      double2 NE = v.ld(o, gx, gy, 1, 1), NW = v.ld(o, gx, gy, -1, 1);
      double2 SE = v.ld(o, gx, gy, 1, -1), SW = v.ld(o, gx, gy, -1, -1);
      double dre = (Eo.x + Wo.x - 2.0 * Co.x) * a.idx2 - (No.x + So.x - 2.0 * Co.x) * a.idy2;
      double dim = (Eo.y + Wo.y - 2.0 * Co.y) * a.idx2 - (No.y + So.y - 2.0 * Co.y) * a.idy2;
      double zx = 2.0 * ((NE.x - SE.x) - (NW.x - SW.x)) * a.ixy4;
      double zy = 2.0 * ((NE.y - SE.y) - (NW.y - SW.y)) * a.ixy4;
      double sgn = (c == 0) ? -1.0 : 1.0;  // J_+ = D - 2i Dxy, J_- = D + 2i Dxy
      double jx = a.delta_lt * (dre - sgn * zy);
      double jy = a.delta_lt * (dim + sgn * zx);
      e += C.x * jx + C.y * jy;  // Re(psi_c^* J_c psi_o)
    }
  }
  if (a.ncomp == 2) e += a.g_x * dens[0] * dens[1];
}

template <typename R>
__global__ void __launch_bounds__(NA_THREADS)
na_partials_kernel(PlainView<R> v, NaPhys a, double* scratch) {
  __shared__ double sh[2][32];
  double acc0 = 0.0, acc1 = 0.0;
  const long long sites = (long long)v.nx * v.ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < sites;
       t += (long long)gridDim.x * blockDim.x) {
    int gy = (int)(t / v.nx), gx = (int)(t - (long long)gy * v.nx);
    double nrm, e;
    na_site(v, a, gx, gy, nrm, e);
    acc0 += nrm;
    acc1 += e;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  acc0 = na_warp_sum(acc0);
  acc1 = na_warp_sum(acc1);
  if (lane == 0) {
    sh[0][wid] = acc0;
    sh[1][wid] = acc1;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    double s0 = lane < nw ? sh[0][lane] : 0.0;
    double s1 = lane < nw ? sh[1][lane] : 0.0;
    s0 = na_warp_sum(s0);
    s1 = na_warp_sum(s1);
    if (lane == 0) {
      scratch[2 * blockIdx.x] = s0;
      scratch[2 * blockIdx.x + 1] = s1;
    }
  }
}

// Fixed-order sum of the CTA partials into scratch[2*NA_MAX_BLOCKS + {0,1}].
__global__ void __launch_bounds__(NA_THREADS)
na_final_kernel(double* scratch, int nblocks) {
  __shared__ double sh[2][32];
  double a0 = 0.0, a1 = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    a0 += scratch[2 * b];
    a1 += scratch[2 * b + 1];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  a0 = na_warp_sum(a0);
  a1 = na_warp_sum(a1);
  if (lane == 0) {
    sh[0][wid] = a0;
    sh[1][wid] = a1;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    double s0 = lane < nw ? sh[0][lane] : 0.0;
    double s1 = lane < nw ? sh[1][lane] : 0.0;
    s0 = na_warp_sum(s0);
    s1 = na_warp_sum(s1);
    if (lane == 0) {
      scratch[2 * NA_MAX_BLOCKS] = s0;
      scratch[2 * NA_MAX_BLOCKS + 1] = s1;
    }
  }
}

// Errors are reported by status code only: recording a message string could
// allocate host memory, which this entry point avoids on every path.
phx_status na_fail(phx_status s, const char* why) {
  (void)why;
  return s;
}

}  // namespace

}  // namespace phx

using namespace phx;

extern "C" phx_status phx_norm_energy_static(const phx_params* p, const void* psi,
                                             const void* n, const void* V,
                                             double* norm, double* energy) {
  if (!p || !psi) return na_fail(PHX_EINVAL, "params and psi must not be NULL");
  if (p->struct_size != sizeof(phx_params))
    return na_fail(PHX_EINVAL, "params.struct_size mismatch (call phx_params_init)");
  if (p->nx < 1 || p->ny < 1) return na_fail(PHX_EINVAL, "nx, ny must be >= 1");
  if (p->precision != 32 && p->precision != 64)
    return na_fail(PHX_EINVAL, "precision must be 32 or 64");
  if ((p->bc_x != PHX_BC_PERIODIC && p->bc_x != PHX_BC_ZERO) ||
      (p->bc_y != PHX_BC_PERIODIC && p->bc_y != PHX_BC_ZERO))
    return na_fail(PHX_EINVAL, "bc_x, bc_y must be PHX_BC_PERIODIC or PHX_BC_ZERO");
  if (!(p->lx > 0) || !(p->ly > 0)) return na_fail(PHX_EINVAL, "lx, ly must be > 0");
  if (p->reservoir && !n) return na_fail(PHX_EINVAL, "reservoir = 1 needs n");
  const long long sites = (long long)p->nx * p->ny;
  if (sites > NA_MAX_SITES)
    return na_fail(PHX_EINVAL,
                   "grid too large for phx_norm_energy_static: nx*ny must be <= "
                   "16777216 (size of its static scratch)");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(PHX_ENODEV, cudaGetErrorString(e));
  if (dev < 0 || dev >= NA_MAX_DEVICES) return na_fail(PHX_ENODEV, "device index too large");
  // Set-up, once per device, with that device current: the device address of
  // the static scratch (its host-side name is only a stand-in).  A look-up
  // that failed leaves the slot empty and is tried again by the next call.
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
      double* ptr = nullptr;
      e = cudaGetSymbolAddress((void**)&ptr, g_na_scratch);
      if (e != cudaSuccess || !ptr) {
        cudaGetLastError();  // clear it: the next call starts clean
        return na_fail(PHX_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
      }
      g_na_ptr[dev] = ptr;
    }
    scratch = g_na_ptr[dev];
  }

  const double dx = p->lx / p->nx, dy = p->ly / p->ny;
  NaPhys a;
  a.kappa = p->hbar2_over_2m;
  a.g = p->g;
  a.g_x = p->g_x;
  a.g_r = p->g_r;
  a.delta_lt = p->delta_lt;
  a.idx2 = 1.0 / (dx * dx);
  a.idy2 = 1.0 / (dy * dy);
  a.ixy4 = 1.0 / (4.0 * dx * dy);
  a.ncomp = p->spinor ? 2 : 1;
  a.reservoir = p->reservoir ? 1 : 0;
  a.tetm = (p->spinor && p->delta_lt != 0.0) ? 1 : 0;
  a.has_V = V != nullptr;

  long long want = (sites + (long long)NA_THREADS * NA_SITES_PER_THREAD - 1) /
                   ((long long)NA_THREADS * NA_SITES_PER_THREAD);
  int nblocks = (int)(want < 1 ? 1 : want);
  cudaStream_t s = static_cast<cudaStream_t>(p->stream);
  if (p->precision == 32) {
    PlainView<float> v{static_cast<const float*>(psi), static_cast<const float*>(n),
                       static_cast<const float*>(V), p->nx, p->ny, p->bc_x, p->bc_y, sites};
    na_partials_kernel<float><<<nblocks, NA_THREADS, 0, s>>>(v, a, scratch);
  } else {
    PlainView<double> v{static_cast<const double*>(psi), static_cast<const double*>(n),
                        static_cast<const double*>(V), p->nx, p->ny, p->bc_x, p->bc_y, sites};
    na_partials_kernel<double><<<nblocks, NA_THREADS, 0, s>>>(v, a, scratch);
  }
  na_final_kernel<<<1, NA_THREADS, 0, s>>>(scratch, nblocks);
  count_launch(2);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(PHX_ECUDA, cudaGetErrorString(e));
  double out[2];
  e = cudaMemcpyAsync(out, scratch + 2 * NA_MAX_BLOCKS, sizeof out,
                      cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return na_fail(PHX_ECUDA, cudaGetErrorString(e));
  const double dV = dx * dy;
  if (norm) *norm = dV * out[0];
  if (energy) *energy = dV * out[1];
  if (!std::isfinite(out[0]) || !std::isfinite(out[1]))
    return na_fail(PHX_ENONFINITE, "state holds NaN or Inf");
  return PHX_OK;
}
