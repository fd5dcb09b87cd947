// FP64 reductions over the domain: norm, energy, steady-state residual.
// Each CTA reduces its grid-stride share with warp shuffles and writes one
// FP64 partial per quantity; a single-CTA pass then sums the partials in a
// fixed order, so results are deterministic for a given grid.
#include <algorithm>

#include "phx_internal.h"

namespace phx {

constexpr int RED_THREADS = 256;
constexpr int RED_MAX_BLOCKS = 1216;  // 152 SMs x 8
constexpr int RED_Q = 8;              // quantities per partial record
// After the records: an arrival counter (read as unsigned) that the last CTA
// of a reduction resets to zero, and the residual's -hbar omega as a
// double-float; callers zero the whole buffer once when they allocate it.
constexpr int RED_COUNTER = RED_MAX_BLOCKS * RED_Q;

// CTAs of the double-float kernels: their warps take items of 32 x DF_SEG
// columns of one row, about DF_ITEMS items per warp (32 sites per thread),
// so that the double-float warp and CTA sums (about 660 warp instructions
// per warp for six quantities) stay a small part of the work; but at least
// DF_MIN_BLOCKS CTAs (two per SM) while there is an item per warp.
constexpr int DF_SEG = 8;
constexpr int DF_ITEMS = 4;
constexpr int DF_MIN_BLOCKS = 304;
int df_reduce_blocks(const Geometry& g) {
  const long long nseg = (g.nx + 32 * DF_SEG - 1) / (32 * DF_SEG);
  const long long items = nseg * g.ny, wpb = RED_THREADS / 32;
  long long b = (items + wpb * DF_ITEMS - 1) / (wpb * DF_ITEMS);
  if (b < DF_MIN_BLOCKS) b = std::min<long long>(DF_MIN_BLOCKS, (items + wpb - 1) / wpb);
  if (b > RED_MAX_BLOCKS) b = RED_MAX_BLOCKS;
  if (b < 1) b = 1;
  return (int)b;
}

int reduce_blocks(const Geometry& g) {
  long long sites = (long long)g.nx * g.ny;
  long long b = (sites + RED_THREADS - 1) / RED_THREADS;
  if (b > RED_MAX_BLOCKS) b = RED_MAX_BLOCKS;
  if (b < 1) b = 1;
  return (int)b;
}

size_t reduce_partials_len(const Geometry&) { return (size_t)RED_MAX_BLOCKS * RED_Q + 2; }

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

// Called by every CTA after thread 0 wrote its record: the CTA that arrives
// last sums all records in a fixed order (deterministic whatever the arrival
// order) and writes the results.  kind 0: norm/energy -> out[0..1];
// 1: residual pass 1 -> out[0..4], out[6] = omega;  2: residual pass 2 -> out[5].
__device__ void finish_reduction(double* partials, int kind, double* out, double* sh) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();  // this CTA's record visible device-wide before its arrival counts
    unsigned int* cnt = reinterpret_cast<unsigned int*>(partials + RED_COUNTER);
    last = atomicAdd(cnt, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
    for (int q = 0; q < 5; ++q) acc[q] += __ldcg(partials + b * RED_Q + q);
  block_sum<5>(acc, sh);
  if (threadIdx.x == 0) {
    if (kind == 0) {
      out[0] = acc[0];
      out[1] = acc[1];
    } else if (kind == 1) {
      for (int q = 0; q < 5; ++q) out[q] = acc[q];
      const double om = acc[0] > 0.0 ? -acc[2] / acc[0] : 0.0;
      out[6] = om;
      // -hbar omega split into a double-float for the second pass
      const double hw = -HBAR * om;
      const float hi = (float)hw;
      *reinterpret_cast<float2*>(partials + RED_COUNTER + 1) =
          make_float2(hi, (float)(hw - (double)hi));
    } else {
      out[5] = acc[0];
    }
    *reinterpret_cast<unsigned int*>(partials + RED_COUNTER) = 0u;
  }
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
norm_energy_kernel(SiteView<R> v, PhysArgs a, int nx, int ny, double* partials, double* out) {
  __shared__ double sh[5 * 32];
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
  finish_reduction(partials, 0, out, sh);
}

// Residual pass 1 (mode 0): S_pp, Re/Im S_pK, S_fn, S_nn.
// Pass 2 (mode 1): sum |K + i omega psi|^2 with omega read from out[6].
template <typename R>
__global__ void __launch_bounds__(RED_THREADS)
residual_kernel(SiteView<R> v, PhysArgs a, int nx, int ny, int mode,
                double* out, double* partials) {
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
  finish_reduction(partials, mode ? 2 : 1, out, sh);
}

// ---------------------------------------------------------------------------
// FP32 scalar fields: every per-site quantity in double-float arithmetic.
//
// A double-float (hi, lo) is an unevaluated sum of two FP32 numbers carrying
// about 44-48 significant bits.  The error-free transformations are the
// classical ones (Knuth's two-sum, Dekker's fast two-sum, the
// fused-multiply-add two-product), written with explicitly rounded FP32
// operations so that the compiler neither contracts nor reorders them.  The
// FP32 inputs convert exactly; products of two FP32 values and differences of
// neighbours are formed without rounding error in their leading part.
//
// Per thread, each quantity is summed by the cascaded scheme of Ogita, Rump
// and Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 2005,
// Sum2): the running FP32 sum takes every term through a two-sum and the
// rounding errors collect in a second FP32 word, which keeps the result as
// accurate as a sum in twice the working precision.  Warps, CTAs and the
// final pass over the CTA records add double-floats in a fixed order; the FP64
// pipe (about 1/64 of the FP32 pipe on this GPU) is used by one thread of the
// last CTA only, to apply the grid's coefficients to the totals.
//
// Kinetic term.  For ghost cells that hold periodic images or zeros, the
// discrete Green identity
//   sum_sites Re(conj(psi) (E + W - 2C)) = - sum_bonds |psi_b - psi_a|^2
// (bonds: every pair of x neighbours, including the pair between a zero
// ghost and the first site of a zero-BC axis) gives the kinetic energy as a
// sum of non-negative squares of neighbour differences, and
// sum_sites Im(conj(psi) Lap psi) = 0.  Both are identities of the sums, so
// the norm/energy and the residual's first pass read each site's east and
// north neighbour only.
struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_two_sum(float a, float b) {  // a + b exactly
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ DF df_norm(float a, float b) {  // |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// accurate sum of two double-floats (two two-sums)
__device__ __forceinline__ DF df_add(DF x, DF y) {
  const DF s = df_two_sum(x.hi, y.hi);
  const DF t = df_two_sum(x.lo, y.lo);
  const DF u = df_norm(s.hi, __fadd_rn(s.lo, t.hi));
  return df_norm(u.hi, __fadd_rn(u.lo, t.lo));
}
// sum of two double-floats whose low words are added in FP32: the error is of
// the order 2^-48 of the larger operand, which is the accuracy the residual's
// per-site terms need (they are compared with terms of that size)
__device__ __forceinline__ DF df_add_s(DF x, DF y) {
  const DF s = df_two_sum(x.hi, y.hi);
  return df_norm(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ DF df_prod(float a, float b) {  // a * b exactly
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
// x * y, x * b and x^2 with the low word left unnormalised (every consumer
// takes the high words through a two-sum)
__device__ __forceinline__ DF df_mul_s(DF x, DF y) {
  const DF p = df_prod(x.hi, y.hi);
  return {p.hi, __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo))};
}
__device__ __forceinline__ DF df_mulf_s(DF x, float b) {
  const DF p = df_prod(x.hi, b);
  return {p.hi, __fmaf_rn(x.lo, b, p.lo)};
}
__device__ __forceinline__ DF df_sqr_s(DF x) {
  const DF p = df_prod(x.hi, x.hi);
  return {p.hi, __fmaf_rn(__fadd_rn(x.hi, x.hi), x.lo, p.lo)};
}
__device__ __forceinline__ DF df_neg(DF x) { return {-x.hi, -x.lo}; }
constexpr DF DF0 = {0.f, 0.f};

// Running sum of one quantity (Sum2): s + c.
struct Acc {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(DF x) {
    const DF t = df_two_sum(s, x.hi);
    s = t.hi;
    c = __fadd_rn(c, __fadd_rn(t.lo, x.lo));
  }
  __device__ __forceinline__ DF df() const { return df_two_sum(s, c); }
};

// Double-float coefficients, split from their FP64 values on the host (so
// that no thread spends FP64 instructions on them).
struct DfCoeffs {
  DF kx, ky;      // kappa / (hbar dx^2), kappa / (hbar dy^2)
  DF ih;          // 1 / hbar
  DF gh, grh;     // g / hbar, g_r / hbar
  DF hR, hgc;     // R / 2, -gamma_c / 2
  DF gamma_r, R;
};

inline DF df_host(double v) {
  const float hi = (float)v;
  return DF{hi, (float)(v - (double)hi)};
}

// sum of x over the warp, in double-float, in every lane (butterfly order)
__device__ __forceinline__ DF df_warp_sum(DF x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    x = df_add(x, DF{__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)});
  return x;
}

// a + b - 2c for FP32 a, b, c, exact up to the rounding of the low word
__device__ __forceinline__ DF df_second_diff(float a, float b, float c) {
  const DF s = df_two_sum(a, b);
  const DF t = df_two_sum(s.hi, __fmul_rn(-2.0f, c));  // -2c is exact
  return {t.hi, __fadd_rn(t.lo, s.lo)};
}
// |C|^2 of an FP32 complex value, exact up to the rounding of the low word
__device__ __forceinline__ DF df_abs2(float2 c) {
  const DF x = df_prod(c.x, c.x), y = df_prod(c.y, c.y);
  const DF s = df_two_sum(x.hi, y.hi);
  return df_norm(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
// |b - a|^2 of two FP32 complex values (the differences are exact)
__device__ __forceinline__ DF df_bond(float2 a, float2 b) {
  const DF dx = df_two_sum(b.x, -a.x), dy = df_two_sum(b.y, -a.y);
  const DF px = df_sqr_s(dx), py = df_sqr_s(dy);
  const DF s = df_two_sum(px.hi, py.hi);
  return {s.hi, __fadd_rn(s.lo, __fadd_rn(px.lo, py.lo))};
}

// Site loop of the double-float kernels: each warp takes items of
// 32 x DF_SEG consecutive columns of one row (coalesced loads, one integer
// division per item); the grid strides over the items.
template <typename F>
__device__ __forceinline__ void df_sites(int nx, int ny, F&& f) {
  const int lane = threadIdx.x & 31;
  const unsigned nseg = (unsigned)(nx + 32 * DF_SEG - 1) / (32 * DF_SEG);
  const unsigned items = nseg * (unsigned)ny;
  const unsigned wpb = blockDim.x >> 5;
  for (unsigned it = blockIdx.x * wpb + (threadIdx.x >> 5); it < items;
       it += gridDim.x * wpb) {
    const unsigned gy = it / nseg;
    const int x0 = (int)(it - gy * nseg) * (32 * DF_SEG) + lane;
#pragma unroll
    for (int j = 0; j < DF_SEG; ++j) {
      const int gx = x0 + 32 * j;
      if (gx < nx) f(gx, (int)gy);
    }
  }
}

// CTA sum of NQ double-floats, one per thread: warp butterflies, then thread
// q < NQ adds the warps' sums of quantity q in warp order.  The result is
// valid in threads 0..NQ-1 (quantity = thread index).  sh: NQ x 32 float2.
template <int NQ>
__device__ __forceinline__ DF df_block_sum(DF (&v)[NQ], float2* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const DF w = df_warp_sum(v[q]);
    if (lane == 0) sh[q * 32 + wid] = make_float2(w.hi, w.lo);
  }
  __syncthreads();
  DF s = DF0;
  if (threadIdx.x < NQ) {
    const float2* r = sh + threadIdx.x * 32;
    s = DF{r[0].x, r[0].y};
    for (int w = 1; w < nw; ++w) s = df_add(s, DF{r[w].x, r[w].y});
  }
  return s;
}

// The CTA's record: NQ double-floats (as float2 in the record's double
// slots), written by threads 0..NQ-1; then the CTA that arrives last sums all
// records in a fixed order (deterministic whatever the arrival order),
// converts the NQ totals to FP64 (one per thread, so that the narrow FP64
// pipe sees a few warp instructions) and hands them to `fin` in thread 0.
template <int NQ, typename Fin>
__device__ void df_record_and_finish(DF (&v)[NQ], float2* sh, double* partials, Fin&& fin) {
  __shared__ bool last;
  __shared__ double tot[NQ];
  float2* rec = reinterpret_cast<float2*>(partials);
  {
    const DF s = df_block_sum<NQ>(v, sh);
    if (threadIdx.x < NQ) {
      rec[(size_t)blockIdx.x * RED_Q + threadIdx.x] = make_float2(s.hi, s.lo);
      __threadfence();  // the record visible device-wide before the arrival counts
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int* cnt = reinterpret_cast<unsigned int*>(partials + RED_COUNTER);
    last = atomicAdd(cnt, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  DF w[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) w[q] = DF0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const float2 r = __ldcg(rec + (size_t)b * RED_Q + q);
      w[q] = df_add(w[q], DF{r.x, r.y});
    }
  }
  const DF s = df_block_sum<NQ>(w, sh);
  if (threadIdx.x < NQ) tot[threadIdx.x] = (double)s.hi + (double)s.lo;
  __syncthreads();
  if (threadIdx.x == 0) {
    fin(tot);
    *reinterpret_cast<unsigned int*>(partials + RED_COUNTER) = 0u;
  }
}

struct DfField {
  const float2* psi;  // padded, interleaved complex
  const float* n;     // padded planes (nullptr when absent)
  const float* P;
  const float* V;
  int pitch, nx, ny;
  int zx, zy;         // axis with zero boundary condition
};

// Per-site terms shared by the norm/energy and the residual's first pass:
// |C|^2, the x and y bond sums, |C|^4, V|C|^2, n|C|^2.
struct DfSums {
  Acc s0, sbx, sby, sv, sn, s4;
  __device__ __forceinline__ DF site(const DfField& f, const PhysArgs& a, int gx, int gy,
                                     long long off) {
    const float2 C = f.psi[off], E = f.psi[off + 1], N = f.psi[off + f.pitch];
    const DF dens = df_abs2(C);
    s0.add(dens);
    sbx.add(df_bond(C, E));
    sby.add(df_bond(C, N));
    if (f.zx && gx == 0) sbx.add(dens);  // bond from the zero ghost at x = -1
    if (f.zy && gy == 0) sby.add(dens);  // and at y = -1
    s4.add(df_sqr_s(dens));
    if (a.has_V) sv.add(df_mulf_s(dens, f.V[off]));
    if (a.reservoir) sn.add(df_mulf_s(dens, f.n[off]));
    return dens;
  }
};

// Norm and energy of an FP32 scalar field (sums without dV):
//   N = sum |C|^2,
//   E = kappa (S_bx/dx^2 + S_by/dy^2) + sum V|C|^2 + (g/2) sum |C|^4 + g_r sum n|C|^2,
// the kinetic part by the Green identity above (equal to
// sum Re(conj(C) (-kappa Lap C))).
__global__ void __launch_bounds__(RED_THREADS)
df_norm_energy_kernel(DfField f, PhysArgs a, double* partials, double* out) {
  __shared__ float2 sh[6 * 32];
  DfSums t;
  df_sites(f.nx, f.ny, [&](int gx, int gy) {
    t.site(f, a, gx, gy, (long long)(gy + HALO) * f.pitch + gx + HALO);
  });
  DF v[6] = {t.s0.df(), t.sbx.df(), t.sby.df(), t.sv.df(), t.sn.df(), t.s4.df()};
  df_record_and_finish<6>(v, sh, partials, [&](const double* S) {
    out[0] = S[0];
    out[1] = a.kappa * (S[1] * a.idx2 + S[2] * a.idy2) + S[3] + 0.5 * a.g * S[5] +
             a.g_r * S[4];
  });
}

// Residual pass 1 of an FP32 scalar field: S_pp, <psi, K> and the reservoir
// sums.  With K = -(i/hbar) H psi + G psi, G = (R n - gamma_c)/2 and the
// identities above,
//   Re <psi, K> = sum G|C|^2,
//   Im <psi, K> = -(1/hbar) [kinetic + sum (V + g|C|^2 + g_r n)|C|^2],
// omega = -Im<psi, K> / S_pp; f_n = P - (gamma_r + R|C|^2) n per site.
__global__ void __launch_bounds__(RED_THREADS)
df_residual1_kernel(DfField f, PhysArgs a, DfCoeffs k, double* partials, double* out) {
  __shared__ float2 sh[8 * 32];
  DfSums t;
  Acc sfn, snn;
  df_sites(f.nx, f.ny, [&](int gx, int gy) {
    const long long off = (long long)(gy + HALO) * f.pitch + gx + HALO;
    const DF dens = t.site(f, a, gx, gy, off);
    if (a.reservoir) {
      const float nv = f.n[off];
      const DF rate = df_add_s(k.gamma_r, df_mul_s(k.R, dens));
      const DF fn = df_add_s(DF{f.P[off], 0.f}, df_neg(df_mulf_s(rate, nv)));
      sfn.add(df_sqr_s(fn));
      snn.add(df_prod(nv, nv));
    }
  });
  DF v[8] = {t.s0.df(), t.sbx.df(), t.sby.df(), t.sv.df(), t.sn.df(), t.s4.df(),
             sfn.df(),  snn.df()};
  df_record_and_finish<8>(v, sh, partials, [&](const double* S) {
    const double kin = a.kappa * (S[1] * a.idx2 + S[2] * a.idy2);
    const double loc2 = S[3] + a.g * S[5] + a.g_r * S[4];
    out[0] = S[0];
    out[1] = a.reservoir ? 0.5 * (a.R * S[4] - a.gamma_c * S[0]) : -0.5 * a.gamma_c * S[0];
    out[2] = -(kin + loc2) / HBAR;
    out[3] = S[6];
    out[4] = S[7];
    const double om = S[0] > 0.0 ? -out[2] / S[0] : 0.0;
    out[6] = om;
    // -omega as a double-float for the second pass
    const float hi = (float)(-om);
    *reinterpret_cast<float2*>(partials + RED_COUNTER + 1) =
        make_float2(hi, (float)(-om - (double)hi));
  });
}

// Residual pass 2 of an FP32 scalar field: sum |Q|^2 of Q = K + i omega psi,
//   Q.x = G C.x + M C.y - (kx Lx_i + ky Ly_i),
//   Q.y = G C.y - M C.x + (kx Lx_r + ky Ly_r),
//   M = (V + g|C|^2 + g_r n)/hbar - omega,  kx = kappa/(hbar dx^2),
// L the unscaled second differences of Re / Im along x and y; every term in
// double-float (Q is a small difference of terms of the size of K).
__global__ void __launch_bounds__(RED_THREADS)
df_residual2_kernel(DfField f, PhysArgs a, DfCoeffs k, double* partials, double* out) {
  __shared__ float2 sh[32];
  const float2 w2 = __ldcg(reinterpret_cast<const float2*>(partials + RED_COUNTER + 1));
  const DF nom = {w2.x, w2.y};  // -omega, left by the first pass's last CTA
  Acc sq;
  df_sites(f.nx, f.ny, [&](int gx, int gy) {
    const long long off = (long long)(gy + HALO) * f.pitch + gx + HALO;
    const float2 C = f.psi[off], E = f.psi[off + 1], W = f.psi[off - 1];
    const float2 N = f.psi[off + f.pitch], S = f.psi[off - f.pitch];
    const DF dens = df_abs2(C);
    const DF lr = df_add_s(df_mul_s(k.kx, df_second_diff(E.x, W.x, C.x)),
                           df_mul_s(k.ky, df_second_diff(N.x, S.x, C.x)));
    const DF li = df_add_s(df_mul_s(k.kx, df_second_diff(E.y, W.y, C.y)),
                           df_mul_s(k.ky, df_second_diff(N.y, S.y, C.y)));
    DF M = df_add_s(df_mul_s(k.gh, dens), nom);
    if (a.has_V) M = df_add_s(M, df_mulf_s(k.ih, f.V[off]));
    DF G = k.hgc;
    if (a.reservoir) {
      const float nv = f.n[off];
      M = df_add_s(M, df_mulf_s(k.grh, nv));
      G = df_add_s(k.hgc, df_mulf_s(k.hR, nv));
    }
    const DF qx = df_add_s(df_add_s(df_mulf_s(G, C.x), df_mulf_s(M, C.y)), df_neg(li));
    const DF qy = df_add_s(df_add_s(df_mulf_s(G, C.y), df_neg(df_mulf_s(M, C.x))), lr);
    sq.add(df_sqr_s(qx));
    sq.add(df_sqr_s(qy));
  });
  DF v[1] = {sq.df()};
  df_record_and_finish<1>(v, sh, partials, [&](const double* S) { out[5] = S[0]; });
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

static DfField make_df_field(const ReduceArgs& r) {
  DfField f;
  f.psi = static_cast<const float2*>(r.psi);
  f.n = static_cast<const float*>(r.n);
  f.P = static_cast<const float*>(r.P);
  f.V = static_cast<const float*>(r.V);
  f.pitch = r.geo.pitch;
  f.nx = r.geo.nx;
  f.ny = r.geo.ny;
  f.zx = r.geo.bc_x == BC_ZERO;
  f.zy = r.geo.bc_y == BC_ZERO;
  return f;
}

cudaError_t launch_norm_energy(const ReduceArgs& r, double* partials,
                               double* out, cudaStream_t s) {
  PhysArgs a = make_phys(r);
  int nb = reduce_blocks(r.geo);
  if (r.precision == 32 && r.ncomp == 1)
    df_norm_energy_kernel<<<df_reduce_blocks(r.geo), RED_THREADS, 0, s>>>(make_df_field(r), a,
                                                                         partials, out);
  else if (r.precision == 32)
    norm_energy_kernel<float><<<nb, RED_THREADS, 0, s>>>(make_view<float>(r), a,
                                                         r.geo.nx, r.geo.ny, partials, out);
  else
    norm_energy_kernel<double><<<nb, RED_THREADS, 0, s>>>(make_view<double>(r), a,
                                                          r.geo.nx, r.geo.ny, partials, out);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_residual(const ReduceArgs& r, double* partials, double* out,
                            cudaStream_t s) {
  PhysArgs a = make_phys(r);
  if (r.precision == 32 && r.ncomp == 1) {
    DfCoeffs k;
    k.kx = df_host(a.kappa / HBAR * a.idx2);
    k.ky = df_host(a.kappa / HBAR * a.idy2);
    k.ih = df_host(1.0 / HBAR);
    k.gh = df_host(a.g / HBAR);
    k.grh = df_host(a.g_r / HBAR);
    k.hR = df_host(0.5 * a.R);
    k.hgc = df_host(-0.5 * a.gamma_c);
    k.gamma_r = df_host(a.gamma_r);
    k.R = df_host(a.R);
    const DfField f = make_df_field(r);
    const int nb = df_reduce_blocks(r.geo);
    df_residual1_kernel<<<nb, RED_THREADS, 0, s>>>(f, a, k, partials, out);
    df_residual2_kernel<<<nb, RED_THREADS, 0, s>>>(f, a, k, partials, out);
  } else {
    const int nb = reduce_blocks(r.geo);
    for (int mode = 0; mode < 2; ++mode) {
      if (r.precision == 32)
        residual_kernel<float><<<nb, RED_THREADS, 0, s>>>(make_view<float>(r), a, r.geo.nx,
                                                          r.geo.ny, mode, out, partials);
      else
        residual_kernel<double><<<nb, RED_THREADS, 0, s>>>(make_view<double>(r), a, r.geo.nx,
                                                           r.geo.ny, mode, out, partials);
    }
  }
  count_launch(2);
  return cudaGetLastError();
}

}  // namespace phx
