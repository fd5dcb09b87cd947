// Ghost-ring maintenance for host-side uploads and the noise sampler.
#include <atomic>

#include "phx_internal.h"
#include "phx_noise.cuh"

namespace phx {

static std::atomic<unsigned long long> g_launches{0};
static std::atomic<unsigned> g_inject{0};

bool take_injection(unsigned what) {
  unsigned cur = g_inject.load();
  while (cur & what) {
    if (g_inject.compare_exchange_weak(cur, cur & ~what)) return true;
  }
  return false;
}
void arm_injection(unsigned mask) { g_inject.fetch_or(mask); }
void count_launch(unsigned n) { g_launches.fetch_add(n); }
unsigned long long launch_total() { return g_launches.load(); }

// Every padded position outside the domain takes the value of the domain
// site it images (periodic axis) or zero (zero axis, or beyond the ring).
template <int ES>
__global__ void fill_ghosts_kernel(unsigned char* base, int nplanes, Geometry g) {
  long long total = g.plane * nplanes;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long pl = t / g.plane;
    long long r = t - pl * g.plane;
    int py = (int)(r / g.pitch), px = (int)(r - (long long)py * g.pitch);
    int gx = px - HALO, gy = py - HALO;
    bool in_x = gx >= 0 && gx < g.nx, in_y = gy >= 0 && gy < g.ny;
    if (in_x && in_y) continue;
    bool zero = false;
    if (!in_x) {
      if (g.bc_x == BC_PERIODIC && px < g.nx + 2 * HALO)
        gx = ((gx % g.nx) + g.nx) % g.nx;
      else
        zero = true;
    }
    if (!in_y) {
      if (g.bc_y == BC_PERIODIC)
        gy = ((gy % g.ny) + g.ny) % g.ny;
      else
        zero = true;
    }
    unsigned char* dst = base + t * ES;
    if (zero) {
      for (int b = 0; b < ES; ++b) dst[b] = 0;
    } else {
      const unsigned char* src =
          base + (pl * g.plane + (long long)(gy + HALO) * g.pitch + gx + HALO) * ES;
      for (int b = 0; b < ES; ++b) dst[b] = src[b];
    }
  }
}

cudaError_t launch_fill_ghosts(void* base, int esize, int nplanes,
                               const Geometry& g, cudaStream_t s) {
  long long total = g.plane * nplanes;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  auto* b = static_cast<unsigned char*>(base);
  switch (esize) {
    case 4: fill_ghosts_kernel<4><<<blocks, 256, 0, s>>>(b, nplanes, g); break;
    case 8: fill_ghosts_kernel<8><<<blocks, 256, 0, s>>>(b, nplanes, g); break;
    case 16: fill_ghosts_kernel<16><<<blocks, 256, 0, s>>>(b, nplanes, g); break;
    default: return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

// Split nplanes padded planes of interleaved complex values (ghost ring
// included) into a real and an imaginary plane each: plane c of `src` goes
// to dst planes 2c (re) and 2c + 1 (im).
template <typename R, typename C>
__global__ void split_complex_kernel(const C* src, R* dst, int nplanes, long long plane) {
  const long long total = plane * nplanes;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long c = t / plane, r = t - c * plane;
    const C v = src[t];
    dst[(2 * c) * plane + r] = v.x;
    dst[(2 * c + 1) * plane + r] = v.y;
  }
}

cudaError_t launch_split_complex(const void* src, void* dst, int esize, int nplanes,
                                 const Geometry& g, cudaStream_t s) {
  long long total = g.plane * nplanes;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  if (esize == 4)
    split_complex_kernel<float, float2><<<blocks, 256, 0, s>>>(
        static_cast<const float2*>(src), static_cast<float*>(dst), nplanes, g.plane);
  else if (esize == 8)
    split_complex_kernel<double, double2><<<blocks, 256, 0, s>>>(
        static_cast<const double2*>(src), static_cast<double*>(dst), nplanes, g.plane);
  else
    return cudaErrorInvalidValue;
  count_launch();
  return cudaGetLastError();
}

__global__ void noise_sample_kernel(unsigned long long seed, long long step,
                                    unsigned int instance, int ncomp, int nx,
                                    int ny, float scale, float* out) {
  long long sites = (long long)nx * ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < sites;
       t += (long long)gridDim.x * blockDim.x) {
    float2 a, b;
    nz_site(seed, instance, step, (uint32_t)t, scale, a, b, ncomp == 2);
    out[2 * t] = a.x;
    out[2 * t + 1] = a.y;
    if (ncomp == 2) {
      out[2 * (sites + t)] = b.x;
      out[2 * (sites + t) + 1] = b.y;
    }
  }
}

cudaError_t launch_noise_sample(unsigned long long seed, long long step,
                                unsigned int instance, int ncomp, int nx,
                                int ny, float scale, float* out,
                                cudaStream_t s) {
  long long sites = (long long)nx * ny;
  int blocks = (int)((sites + 255) / 256);
  if (blocks > 8192) blocks = 8192;
  if (blocks < 1) blocks = 1;
  noise_sample_kernel<<<blocks, 256, 0, s>>>(seed, step, instance, ncomp, nx,
                                             ny, scale, out);
  count_launch();
  return cudaGetLastError();
}

}  // namespace phx
