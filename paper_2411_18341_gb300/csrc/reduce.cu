// FP64 reductions over the domain: norm, energy, steady-state residual.
// Each CTA reduces its grid-stride share with warp shuffles and writes one
// FP64 partial per quantity; a single-CTA pass then sums the partials in a
// fixed order, so results are deterministic for a given grid.
#include "phx_internal.h"

namespace phx {

constexpr int RED_THREADS = 256;
constexpr int RED_MAX_BLOCKS = 1216;  // 152 SMs x 8
constexpr int RED_Q = 8;              // quantities per partial record
// After the records: an arrival counter (read as unsigned) that the last CTA
// of a reduction resets to zero, and the residual's -hbar omega as a
// double-float; callers zero the whole buffer once when they allocate it.
constexpr int RED_COUNTER = RED_MAX_BLOCKS * RED_Q;

// CTAs of the double-float kernels: about 16 sites per thread (their
// epilogue sums warps in double-float and leaves FP64 to one lane per warp).
int df_reduce_blocks(const Geometry& g) {
  const long long sites = (long long)g.nx * g.ny;
  long long b = (sites + RED_THREADS * 16 - 1) / (RED_THREADS * 16);
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
// classical ones (Knuth's and Dekker's two-sum, the fused-multiply-add
// two-product), written with explicitly rounded FP32 operations so that the
// compiler neither contracts nor reorders them.  The FP32 inputs convert
// exactly, the stencil's second differences E + W - 2C are formed without
// rounding error in the leading part, and the grid's coefficients (kappa/dx^2,
// g, 1/hbar, ...) are applied once per thread in FP64 to the double-float
// sums, or, where a per-site value is needed (the residual's second pass), as
// double-float constants split from their FP64 values.  The FP64 pipe, about
// 64x slower than the FP32 pipe on this GPU, then only accumulates per-thread
// and per-CTA partials.
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
__device__ __forceinline__ DF df_add(DF x, DF y) {
  const DF s = df_two_sum(x.hi, y.hi);
  const DF t = df_two_sum(x.lo, y.lo);
  const DF u = df_norm(s.hi, __fadd_rn(s.lo, t.hi));
  return df_norm(u.hi, __fadd_rn(u.lo, t.lo));
}
__device__ __forceinline__ DF df_prod(float a, float b) {  // a * b exactly
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ DF df_mul(DF x, DF y) {
  const DF p = df_prod(x.hi, y.hi);
  return df_norm(p.hi, __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo)));
}
__device__ __forceinline__ DF df_mulf(DF x, float b) {
  const DF p = df_prod(x.hi, b);
  return df_norm(p.hi, __fmaf_rn(x.lo, b, p.lo));
}
__device__ __forceinline__ DF df_neg(DF x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ double df_d(DF x) { return (double)x.hi + (double)x.lo; }
constexpr DF DF0 = {0.f, 0.f};

// Double-float coefficients of the residual, split from their FP64 values on
// the host (so that no thread spends FP64 instructions on them).
struct DfCoeffs {
  DF kx, ky;      // kappa / (hbar dx^2), kappa / (hbar dy^2)
  DF ih;          // 1 / hbar
  DF g, g_r;      // meV um^2
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

// CTA sum of NQ FP64 values held by lane 0 of each warp (sh: NQ x 32
// doubles); the result is valid in thread 0.
template <int NQ>
__device__ void warp_leaders_sum(double (&v)[NQ], double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
    for (int q = 0; q < NQ; ++q) sh[q * 32 + wid] = v[q];
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    for (int q = 0; q < NQ; ++q) {
      double s = lane < nw ? sh[q * 32 + lane] : 0.0;
      v[q] = warp_sum(s);
    }
  }
  __syncthreads();
}

// a + b - 2c for FP32 a, b, c: exact up to the last term's rounding
__device__ __forceinline__ DF df_second_diff(float a, float b, float c) {
  const DF s = df_two_sum(a, b);
  const DF t = df_two_sum(s.hi, __fmul_rn(-2.0f, c));  // -2c is exact
  return df_norm(t.hi, __fadd_rn(t.lo, s.lo));
}
// |C|^2 of an FP32 complex value
__device__ __forceinline__ DF df_abs2(float2 c) {
  return df_add(df_prod(c.x, c.x), df_prod(c.y, c.y));
}

struct DfSite {
  float2 C;
  DF lxr, lxi, lyr, lyi;  // second differences of Re and Im along x and y (unscaled)
  DF dens;
};

__device__ __forceinline__ DfSite df_site(const float* psi, long long off, int pitch) {
  auto ld = [&](long long o) { return *reinterpret_cast<const float2*>(psi + 2 * o); };
  DfSite s;
  s.C = ld(off);
  const float2 E = ld(off + 1), W = ld(off - 1), N = ld(off + pitch), S = ld(off - pitch);
  s.lxr = df_second_diff(E.x, W.x, s.C.x);
  s.lxi = df_second_diff(E.y, W.y, s.C.y);
  s.lyr = df_second_diff(N.x, S.x, s.C.x);
  s.lyi = df_second_diff(N.y, S.y, s.C.y);
  s.dens = df_abs2(s.C);
  return s;
}

// Norm and energy of an FP32 scalar field.  Per thread: sums of |C|^2,
// Re(C* Lx C), Re(C* Ly C) (unscaled second differences), V|C|^2, n|C|^2 and
// |C|^4; then e = -kappa (Sx/dx^2 + Sy/dy^2) + S_V + (g/2) S_4 + g_r S_n in FP64.
__global__ void __launch_bounds__(RED_THREADS)
df_norm_energy_kernel(const float* psi, const float* nres, const float* V, int pitch, int nx,
                      int ny, PhysArgs a, double* partials, double* out) {
  __shared__ double sh[5 * 32];
  DF s0 = DF0, sx = DF0, sy = DF0, sv = DF0, sn = DF0, s4 = DF0;
  const long long sites = (long long)nx * ny;
  // 32-bit site index (nx * ny < 2^31 is checked when parameters are validated)
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < (unsigned)sites;
       t += gridDim.x * blockDim.x) {
    const unsigned gy = t / (unsigned)nx, gx = t - gy * (unsigned)nx;
    const long long off = (long long)(gy + HALO) * pitch + gx + HALO;
    const DfSite q = df_site(psi, off, pitch);
    s0 = df_add(s0, q.dens);
    sx = df_add(sx, df_add(df_mulf(q.lxr, q.C.x), df_mulf(q.lxi, q.C.y)));
    sy = df_add(sy, df_add(df_mulf(q.lyr, q.C.x), df_mulf(q.lyi, q.C.y)));
    if (a.has_V) sv = df_add(sv, df_mulf(q.dens, V[off]));
    if (a.reservoir) sn = df_add(sn, df_mulf(q.dens, nres[off]));
    s4 = df_add(s4, df_mul(q.dens, q.dens));
  }
  // warp sums in double-float; FP64 only in each warp's lane 0
  s0 = df_warp_sum(s0);
  sx = df_warp_sum(sx);
  sy = df_warp_sum(sy);
  if (a.has_V) sv = df_warp_sum(sv);
  if (a.reservoir) sn = df_warp_sum(sn);
  s4 = df_warp_sum(s4);
  double acc[2] = {0.0, 0.0};
  if ((threadIdx.x & 31) == 0) {
    acc[0] = df_d(s0);
    acc[1] = -a.kappa * (df_d(sx) * a.idx2 + df_d(sy) * a.idy2) + df_d(sv) +
             0.5 * a.g * df_d(s4) + a.g_r * df_d(sn);
  }
  warp_leaders_sum<2>(acc, sh);
  if (threadIdx.x == 0) {
    partials[blockIdx.x * RED_Q + 0] = acc[0];
    partials[blockIdx.x * RED_Q + 1] = acc[1];
  }
  finish_reduction(partials, 0, out, sh);
}

// Residual of an FP32 scalar field.  Pass 1 (mode 0) accumulates per thread
// |C|^2, Re and Im of C* Lx C and C* Ly C, V|C|^2, n|C|^2, |C|^4, f_n^2 and
// n^2 and forms, in FP64,
//   Re S_pK = -(kappa/hbar) Im(C* Lap C) + sum G|C|^2,  G = (R n - gamma_c)/2
//   Im S_pK =  (kappa/hbar) Re(C* Lap C) - sum loc |C|^2 / hbar,
//   loc = V + g|C|^2 + g_r n  (the terms of K = -(i/hbar) H psi + G psi).
// Pass 2 (mode 1) forms Q = K + i omega psi per site in double-float:
//   Q.x = -(kx Lx_i + ky Ly_i) + (mu/hbar) C.y + G C.x
//   Q.y =  (kx Lx_r + ky Ly_r) - (mu/hbar) C.x + G C.y,
//   kx = kappa/(hbar dx^2), mu = loc - hbar omega,
// and accumulates |Q|^2.
__global__ void __launch_bounds__(RED_THREADS)
df_residual_kernel(const float* psi, const float* nres, const float* P, const float* V,
                   int pitch, int nx, int ny, PhysArgs a, DfCoeffs k, int mode, double* out,
                   double* partials) {
  __shared__ double sh[5 * 32];
  const long long sites = (long long)nx * ny;
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const double ih = 1.0 / HBAR;
  if (mode == 0) {
    DF s0 = DF0, sxr = DF0, syr = DF0, sxi = DF0, syi = DF0, sv = DF0, sn = DF0, s4 = DF0,
       sfn = DF0, snn = DF0;
    const DF gr_ = k.gamma_r, R_ = k.R;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < (unsigned)sites;
         t += gridDim.x * blockDim.x) {
      const unsigned gy = t / (unsigned)nx, gx = t - gy * (unsigned)nx;
      const long long off = (long long)(gy + HALO) * pitch + gx + HALO;
      const DfSite q = df_site(psi, off, pitch);
      s0 = df_add(s0, q.dens);
      // Re(C* L) = C.x L.x + C.y L.y,  Im(C* L) = C.x L.y - C.y L.x
      sxr = df_add(sxr, df_add(df_mulf(q.lxr, q.C.x), df_mulf(q.lxi, q.C.y)));
      syr = df_add(syr, df_add(df_mulf(q.lyr, q.C.x), df_mulf(q.lyi, q.C.y)));
      sxi = df_add(sxi, df_add(df_mulf(q.lxi, q.C.x), df_neg(df_mulf(q.lxr, q.C.y))));
      syi = df_add(syi, df_add(df_mulf(q.lyi, q.C.x), df_neg(df_mulf(q.lyr, q.C.y))));
      if (a.has_V) sv = df_add(sv, df_mulf(q.dens, V[off]));
      s4 = df_add(s4, df_mul(q.dens, q.dens));
      if (a.reservoir) {
        const float nv = nres[off];
        sn = df_add(sn, df_mulf(q.dens, nv));
        // f_n = P - (gamma_r + R|C|^2) n
        const DF rate = df_add(gr_, df_mul(R_, q.dens));
        const DF fn = df_add(df_prod(P[off], 1.0f), df_neg(df_mulf(rate, nv)));
        sfn = df_add(sfn, df_mul(fn, fn));
        snn = df_add(snn, df_prod(nv, nv));
      }
    }
    // warp sums in double-float; FP64 only in each warp's lane 0
    s0 = df_warp_sum(s0);
    sxr = df_warp_sum(sxr);
    syr = df_warp_sum(syr);
    sxi = df_warp_sum(sxi);
    syi = df_warp_sum(syi);
    if (a.has_V) sv = df_warp_sum(sv);
    s4 = df_warp_sum(s4);
    if (a.reservoir) {
      sn = df_warp_sum(sn);
      sfn = df_warp_sum(sfn);
      snn = df_warp_sum(snn);
    }
    if ((threadIdx.x & 31) == 0) {
      const double kh = a.kappa * ih;
      const double re_l = df_d(sxr) * a.idx2 + df_d(syr) * a.idy2;
      const double im_l = df_d(sxi) * a.idx2 + df_d(syi) * a.idy2;
      const double loc2 = df_d(sv) + a.g * df_d(s4) + a.g_r * df_d(sn);  // sum loc |C|^2
      const double g2 = 0.5 * a.R * df_d(sn) - 0.5 * a.gamma_c * df_d(s0);  // sum G |C|^2
      acc[0] = df_d(s0);
      acc[1] = -kh * im_l + g2;
      acc[2] = kh * re_l - loc2 * ih;
      acc[3] = df_d(sfn);
      acc[4] = df_d(snn);
    }
  } else {
    const DF kx = k.kx, ky = k.ky, ihd = k.ih, g_ = k.g, gr_ = k.g_r, hR = k.hR, hgc = k.hgc;
    // -hbar omega as a double-float, left by the first pass's last CTA
    const float2 hw2 = __ldcg(reinterpret_cast<const float2*>(partials + RED_COUNTER + 1));
    const DF hw = {hw2.x, hw2.y};
    DF sq = DF0;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < (unsigned)sites;
         t += gridDim.x * blockDim.x) {
      const unsigned gy = t / (unsigned)nx, gx = t - gy * (unsigned)nx;
      const long long off = (long long)(gy + HALO) * pitch + gx + HALO;
      const DfSite q = df_site(psi, off, pitch);
      DF mu = df_add(df_mul(g_, q.dens), hw);
      if (a.has_V) mu = df_add(mu, df_prod(V[off], 1.0f));
      DF G = hgc;
      if (a.reservoir) {
        const float nv = nres[off];
        mu = df_add(mu, df_mulf(gr_, nv));
        G = df_add(hgc, df_mulf(hR, nv));
      }
      const DF mh = df_mul(mu, ihd);
      const DF lr = df_add(df_mul(kx, q.lxr), df_mul(ky, q.lyr));
      const DF li = df_add(df_mul(kx, q.lxi), df_mul(ky, q.lyi));
      const DF qx = df_add(df_add(df_neg(li), df_mulf(mh, q.C.y)), df_mulf(G, q.C.x));
      const DF qy = df_add(df_add(lr, df_neg(df_mulf(mh, q.C.x))), df_mulf(G, q.C.y));
      sq = df_add(sq, df_add(df_mul(qx, qx), df_mul(qy, qy)));
    }
    sq = df_warp_sum(sq);
    if ((threadIdx.x & 31) == 0) acc[0] = df_d(sq);
  }
  warp_leaders_sum<5>(acc, sh);
  if (threadIdx.x == 0) {
    for (int q = 0; q < 5; ++q) partials[blockIdx.x * RED_Q + q] = acc[q];
  }
  finish_reduction(partials, mode ? 2 : 1, out, sh);
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
  if (r.precision == 32 && r.ncomp == 1)
    df_norm_energy_kernel<<<df_reduce_blocks(r.geo), RED_THREADS, 0, s>>>(
        static_cast<const float*>(r.psi), static_cast<const float*>(r.n),
        static_cast<const float*>(r.V), r.geo.pitch, r.geo.nx, r.geo.ny, a, partials, out);
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
  int nb = reduce_blocks(r.geo);
  DfCoeffs k;
  k.kx = df_host(a.kappa / HBAR * a.idx2);
  k.ky = df_host(a.kappa / HBAR * a.idy2);
  k.ih = df_host(1.0 / HBAR);
  k.g = df_host(a.g);
  k.g_r = df_host(a.g_r);
  k.hR = df_host(0.5 * a.R);
  k.hgc = df_host(-0.5 * a.gamma_c);
  k.gamma_r = df_host(a.gamma_r);
  k.R = df_host(a.R);
  for (int mode = 0; mode < 2; ++mode) {
    if (r.precision == 32 && r.ncomp == 1)
      df_residual_kernel<<<df_reduce_blocks(r.geo), RED_THREADS, 0, s>>>(
          static_cast<const float*>(r.psi), static_cast<const float*>(r.n),
          static_cast<const float*>(r.P), static_cast<const float*>(r.V), r.geo.pitch,
          r.geo.nx, r.geo.ny, a, k, mode, out, partials);
    else if (r.precision == 32)
      residual_kernel<float><<<nb, RED_THREADS, 0, s>>>(make_view<float>(r), a,
                                                        r.geo.nx, r.geo.ny, mode,
                                                        out, partials);
    else
      residual_kernel<double><<<nb, RED_THREADS, 0, s>>>(make_view<double>(r), a,
                                                         r.geo.nx, r.geo.ny, mode,
                                                         out, partials);
  }
  count_launch(2);
  return cudaGetLastError();
}

}  // namespace phx
