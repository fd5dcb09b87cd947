// FP64 reductions over the domain: norm, energy, steady-state residual.
// Each CTA reduces its grid-stride share with warp shuffles and writes one
// FP64 partial per quantity; a single-CTA pass then sums the partials in a
// fixed order, so results are deterministic for a given grid.
#include "phx_internal.h"

namespace phx {

constexpr int RED_THREADS = 256;
constexpr int RED_MAX_BLOCKS = 1216;  // 152 SMs x 8
constexpr int RED_Q = 8;              // quantities per partial record

int reduce_blocks(const Geometry& g) {
  long long sites = (long long)g.nx * g.ny;
  long long b = (sites + RED_THREADS - 1) / RED_THREADS;
  if (b > RED_MAX_BLOCKS) b = RED_MAX_BLOCKS;
  if (b < 1) b = 1;
  return (int)b;
}

size_t reduce_partials_len(const Geometry&) { return (size_t)RED_MAX_BLOCKS * RED_Q; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of NQ values; result valid in thread 0.
template <int NQ>
__device__ void block_sum(double (&v)[NQ], double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double s = warp_sum(v[q]);
    if (lane == 0) sh[q * 32 + wid] = s;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double s = lane < nw ? sh[q * 32 + lane] : 0.0;
      v[q] = warp_sum(s);
    }
  }
  __syncthreads();
}

template <typename R>
struct SiteView {
  const R* psi;  // interleaved complex, padded
  const R* n;
  const R* P;
  const R* V;
  long long plane, pstride;
  int pitch;
  __device__ double2 ld(int c, long long off) const {
    const R* p = psi + 2 * (c * plane + off);
    return make_double2((double)p[0], (double)p[1]);
  }
};

struct LocalOps {
  // (Dxx - Dyy) and (NE - SE - NW + SW) of component c at padded offset off
  template <typename R>
  __device__ static void tetm_parts(const SiteView<R>& v, int c, long long off,
                                    double idx2, double idy2, double2& d,
                                    double2& x) {
    const int P = v.pitch;
    double2 C = v.ld(c, off), E = v.ld(c, off + 1), W = v.ld(c, off - 1);
    double2 N = v.ld(c, off + P), S = v.ld(c, off - P);
    double2 NE = v.ld(c, off + P + 1), NW = v.ld(c, off + P - 1);
    double2 SE = v.ld(c, off - P + 1), SW = v.ld(c, off - P - 1);
    d.x = (E.x + W.x - 2.0 * C.x) * idx2 - (N.x + S.x - 2.0 * C.x) * idy2;
    d.y = (E.y + W.y - 2.0 * C.y) * idx2 - (N.y + S.y - 2.0 * C.y) * idy2;
    x.x = (NE.x - SE.x) - (NW.x - SW.x);
    x.y = (NE.y - SE.y) - (NW.y - SW.y);
  }
};

struct PhysArgs {
  double kappa, g, g_x, g_r, delta_lt, R, gamma_c, gamma_r;
  double idx2, idy2, ixy4;  // 1/dx^2, 1/dy^2, 1/(4 dx dy)
  int ncomp, reservoir, tetm, has_V;
};

// H psi_c (meV, physical units) at a site; returns also |psi_c|^2 and n_c.
template <typename R>
__device__ void site_hamiltonian(const SiteView<R>& v, const PhysArgs& a,
                                 long long off, double2 (&Hc)[2],
                                 double2 (&pc)[2], double (&dens)[2],
                                 double (&nc)[2]) {
  const int P = v.pitch;
  double Vs = a.has_V ? (double)v.V[off] : 0.0;
  for (int c = 0; c < a.ncomp; ++c) {
    pc[c] = v.ld(c, off);
    dens[c] = pc[c].x * pc[c].x + pc[c].y * pc[c].y;
    nc[c] = a.reservoir ? (double)v.n[c * v.plane + off] : 0.0;
  }
  for (int c = 0; c < a.ncomp; ++c) {
    double2 C = pc[c], E = v.ld(c, off + 1), W = v.ld(c, off - 1);
    double2 N = v.ld(c, off + P), S = v.ld(c, off - P);
    double lx = (E.x + W.x - 2.0 * C.x) * a.idx2 + (N.x + S.x - 2.0 * C.x) * a.idy2;
    double ly = (E.y + W.y - 2.0 * C.y) * a.idx2 + (N.y + S.y - 2.0 * C.y) * a.idy2;
    double loc = Vs + a.g * dens[c];
    if (a.ncomp == 2) loc += a.g_x * dens[1 - c];
    if (a.reservoir) loc += a.g_r * nc[c];
    double2 H = make_double2(-a.kappa * lx + loc * C.x, -a.kappa * ly + loc * C.y);
    if (a.tetm) {
      double2 d, x;
      LocalOps::tetm_parts(v, 1 - c, off, a.idx2, a.idy2, d, x);
      double sgn = (c == 0) ? -1.0 : 1.0;  // J_+ = D - 2i Dxy, J_- = D + 2i Dxy
      double2 dxy2 = make_double2(2.0 * x.x * a.ixy4, 2.0 * x.y * a.ixy4);
      // D + sgn * i * (2 Dxy)
      H.x += a.delta_lt * (d.x - sgn * dxy2.y);
      H.y += a.delta_lt * (d.y + sgn * dxy2.x);
    }
    Hc[c] = H;
  }
}

template <typename R>
__global__ void __launch_bounds__(RED_THREADS)
norm_energy_kernel(SiteView<R> v, PhysArgs a, int nx, int ny, double* partials) {
  __shared__ double sh[2 * 32];
  double acc[2] = {0.0, 0.0};
  long long sites = (long long)nx * ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < sites;
       t += (long long)gridDim.x * blockDim.x) {
    int gy = (int)(t / nx), gx = (int)(t - (long long)gy * nx);
    long long off = (long long)(gy + HALO) * v.pitch + gx + HALO;
    double2 H[2], pc[2];
    double dens[2], nc[2];
    // Energy density from H with the interaction terms halved:
    // e = sum_c Re(psi_c^* H psi_c) - (g/2)|psi_c|^4 - (g_x/2)|psi_c|^2|psi_o|^2
    site_hamiltonian(v, a, off, H, pc, dens, nc);
    double e = 0.0, nrm = 0.0;
    for (int c = 0; c < a.ncomp; ++c) {
      nrm += dens[c];
      e += pc[c].x * H[c].x + pc[c].y * H[c].y;
      e -= 0.5 * a.g * dens[c] * dens[c];
    }
    if (a.ncomp == 2) e -= a.g_x * dens[0] * dens[1];
    acc[0] += nrm;
    acc[1] += e;
  }
  block_sum<2>(acc, sh);
  if (threadIdx.x == 0) {
    partials[blockIdx.x * RED_Q + 0] = acc[0];
    partials[blockIdx.x * RED_Q + 1] = acc[1];
  }
}

// Residual pass 1 (mode 0): S_pp, Re/Im S_pK, S_fn, S_nn.
// Pass 2 (mode 1): sum |K + i omega psi|^2 with omega read from out[6].
template <typename R>
__global__ void __launch_bounds__(RED_THREADS)
residual_kernel(SiteView<R> v, PhysArgs a, int nx, int ny, int mode,
                const double* out, double* partials) {
  __shared__ double sh[5 * 32];
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const double omega = mode ? out[6] : 0.0;
  const double ih = 1.0 / HBAR;
  long long sites = (long long)nx * ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < sites;
       t += (long long)gridDim.x * blockDim.x) {
    int gy = (int)(t / nx), gx = (int)(t - (long long)gy * nx);
    long long off = (long long)(gy + HALO) * v.pitch + gx + HALO;
    double2 H[2], pc[2];
    double dens[2], nc[2];
    site_hamiltonian(v, a, off, H, pc, dens, nc);
    for (int c = 0; c < a.ncomp; ++c) {
      double G = -0.5 * a.gamma_c + (a.reservoir ? 0.5 * a.R * nc[c] : 0.0);
      // K = -(i/hbar) H + G psi
      double Kx = H[c].y * ih + G * pc[c].x;
      double Ky = -H[c].x * ih + G * pc[c].y;
      if (mode == 0) {
        acc[0] += dens[c];
        acc[1] += pc[c].x * Kx + pc[c].y * Ky;   // Re conj(psi) K
        acc[2] += pc[c].x * Ky - pc[c].y * Kx;   // Im conj(psi) K
        if (a.reservoir) {
          double Pc = (double)v.P[c * v.pstride + off];
          double fn = Pc - (a.gamma_r + a.R * dens[c]) * nc[c];
          acc[3] += fn * fn;
          acc[4] += nc[c] * nc[c];
        }
      } else {
        double rx = Kx - omega * pc[c].y;  // K + i omega psi
        double ry = Ky + omega * pc[c].x;
        acc[0] += rx * rx + ry * ry;
      }
    }
  }
  block_sum<5>(acc, sh);
  if (threadIdx.x == 0) {
    for (int q = 0; q < 5; ++q) partials[blockIdx.x * RED_Q + q] = acc[q];
  }
}

// Fixed-order sum of the partial records: thread i adds records i, i+256, ...
// then a shuffle tree.  `kind` 0: norm/energy -> out[0..1];
// 1: residual pass 1 -> out[0..4], out[6] = omega;  2: residual pass 2 -> out[5].
__global__ void __launch_bounds__(RED_THREADS)
finalize_kernel(const double* partials, int nblocks, int kind, double* out) {
  __shared__ double sh[5 * 32];
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
    for (int q = 0; q < 5; ++q) acc[q] += partials[b * RED_Q + q];
  block_sum<5>(acc, sh);
  if (threadIdx.x == 0) {
    if (kind == 0) {
      out[0] = acc[0];
      out[1] = acc[1];
    } else if (kind == 1) {
      for (int q = 0; q < 5; ++q) out[q] = acc[q];
      out[6] = acc[0] > 0.0 ? -acc[2] / acc[0] : 0.0;
    } else {
      out[5] = acc[0];
    }
  }
}

static PhysArgs make_phys(const ReduceArgs& r) {
  PhysArgs a;
  a.kappa = r.kappa;
  a.g = r.g;
  a.g_x = r.g_x;
  a.g_r = r.g_r;
  a.delta_lt = r.delta_lt;
  a.R = r.R;
  a.gamma_c = r.gamma_c;
  a.gamma_r = r.gamma_r;
  a.idx2 = r.idx2;
  a.idy2 = r.idy2;
  a.ixy4 = r.ixy4;
  a.ncomp = r.ncomp;
  a.reservoir = r.reservoir;
  a.tetm = r.tetm;
  a.has_V = r.V != nullptr;
  return a;
}

template <typename R>
static SiteView<R> make_view(const ReduceArgs& r) {
  SiteView<R> v;
  v.psi = static_cast<const R*>(r.psi);
  v.n = static_cast<const R*>(r.n);
  v.P = static_cast<const R*>(r.P);
  v.V = static_cast<const R*>(r.V);
  v.plane = r.geo.plane;
  v.pstride = r.P_comp_stride;
  v.pitch = r.geo.pitch;
  return v;
}

cudaError_t launch_norm_energy(const ReduceArgs& r, double* partials,
                               double* out, cudaStream_t s) {
  PhysArgs a = make_phys(r);
  int nb = reduce_blocks(r.geo);
  if (r.precision == 32)
    norm_energy_kernel<float><<<nb, RED_THREADS, 0, s>>>(make_view<float>(r), a,
                                                         r.geo.nx, r.geo.ny, partials);
  else
    norm_energy_kernel<double><<<nb, RED_THREADS, 0, s>>>(make_view<double>(r), a,
                                                          r.geo.nx, r.geo.ny, partials);
  finalize_kernel<<<1, RED_THREADS, 0, s>>>(partials, nb, 0, out);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_residual(const ReduceArgs& r, double* partials, double* out,
                            cudaStream_t s) {
  PhysArgs a = make_phys(r);
  int nb = reduce_blocks(r.geo);
  for (int mode = 0; mode < 2; ++mode) {
    if (r.precision == 32)
      residual_kernel<float><<<nb, RED_THREADS, 0, s>>>(make_view<float>(r), a,
                                                        r.geo.nx, r.geo.ny, mode,
                                                        out, partials);
    else
      residual_kernel<double><<<nb, RED_THREADS, 0, s>>>(make_view<double>(r), a,
                                                         r.geo.nx, r.geo.ny, mode,
                                                         out, partials);
    finalize_kernel<<<1, RED_THREADS, 0, s>>>(partials, nb, mode ? 2 : 1, out);
  }
  count_launch(4);
  return cudaGetLastError();
}

}  // namespace phx
