// Fused RK4 step, generic over precision and model (scalar / reservoir /
// spinor / TE-TM), one CTA per output tile.
//
// One launch performs one full RK4 step (Eqs. rk4_K1-rk4_final) of
// Eqs. (PULSE_psi)/(PULSE_res) for a TX x TY output tile:
//   1. load psi on the tile plus a depth-4 halo into shared memory (the
//      device layout carries a ghost ring, so the box never wraps);
//   2. evaluate K1..K4 on the tile plus a depth-3 ring; stage values
//      y_k = psi + c_k dt K_{k-1} go to a second shared buffer, the local
//      fields (psi, n, P, V, accumulators) stay in registers.  Every stage is
//      evaluated on the same ring-3 region: values near the region edge go
//      stale one cell per stage, which after four stages reaches exactly the
//      tile border, so the tile itself is exact (Sec. III.B.4's halo
//      argument, with the halo kept on chip);
//   3. psi' = psi + (K1 + 2K2 + 2K3 + K4) dt/6 (likewise n), plus the noise
//      xi, is written to the tile and to its periodic ghost images.
// A coherent drive E_c(r) exp(-i omega t) (when set) is read per site and
// stage from global memory (cached) with the stage time t, t + dt/2,
// t + dt/2, t + dt taken from the FP64 device clock; the four phases are
// evaluated in FP64 by four threads per CTA and shared.
// Only psi', n' leave the SM; the paper's K buffers and two-/five-term sums
// never reach memory.
#pragma once

#include "phx_internal.h"
#include "phx_noise.cuh"

namespace phx {

template <typename R> struct CxOps;
template <> struct CxOps<float> {
  using C = float2;
  __device__ static C mk(float a, float b) { return make_float2(a, b); }
};
template <> struct CxOps<double> {
  using C = double2;
  __device__ static C mk(double a, double b) { return make_double2(a, b); }
};

// Write v at every padded position that images domain site (gx, gy): the
// site itself and, along a periodic axis within HALO of an edge, its ghost
// images.  Interior sites take the single-store path (no division).
template <typename T>
__device__ __forceinline__ void store_with_ghosts(T* plane, const Geometry& g,
                                                  int gx, int gy, T v) {
  const bool near_x = g.bc_x == BC_PERIODIC && (gx < HALO || gx >= g.nx - HALO);
  const bool near_y = g.bc_y == BC_PERIODIC && (gy < HALO || gy >= g.ny - HALO);
  if (!near_x && !near_y) {
    plane[(long long)(gy + HALO) * g.pitch + gx + HALO] = v;
    return;
  }
  if (g.nx >= 2 * HALO && g.ny >= 2 * HALO) {
    // at most one image per axis: the site +-n, no division needed
    const int ix = gx + HALO, iy = gy + HALO;
    const int ix2 = !near_x ? -1 : (gx < HALO ? ix + g.nx : ix - g.nx);
    const int iy2 = !near_y ? -1 : (gy < HALO ? iy + g.ny : iy - g.ny);
    const long long r1 = (long long)iy * g.pitch;
    plane[r1 + ix] = v;
    if (ix2 >= 0) plane[r1 + ix2] = v;
    if (iy2 >= 0) {
      const long long r2 = (long long)iy2 * g.pitch;
      plane[r2 + ix] = v;
      if (ix2 >= 0) plane[r2 + ix2] = v;
    }
    return;
  }
  int mx0 = 0, mx1 = 0, my0 = 0, my1 = 0;
  if (near_x) {
    mx0 = -((gx + HALO) / g.nx);
    mx1 = (g.nx + HALO - 1 - gx) / g.nx;
  }
  if (near_y) {
    my0 = -((gy + HALO) / g.ny);
    my1 = (g.ny + HALO - 1 - gy) / g.ny;
  }
  for (int my = my0; my <= my1; ++my) {
    long long row = (long long)(gy + HALO + my * g.ny) * g.pitch;
    for (int mx = mx0; mx <= mx1; ++mx) plane[row + gx + HALO + mx * g.nx] = v;
  }
}

template <typename R, int NC, bool RES, bool TETM, int TX, int TY, int NT, bool DRV>
__global__ void __launch_bounds__(NT)
rk4_step_generic(const StepArgs<R> a) {
  using C = typename CxOps<R>::C;
  constexpr int LX = TX + 2 * HALO, LY = TY + 2 * HALO;  // loaded box
  constexpr int RXN = TX + 6, RYN = TY + 6;               // computed ring-3 region
  constexpr int NPT = RXN * RYN;
  constexpr int PPT = (NPT + NT - 1) / NT;
  constexpr int LBOX = LX * LY;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* ybuf0 = reinterpret_cast<C*>(smem_raw);
  C* ybuf1 = ybuf0 + NC * LBOX;

  const Geometry& g = a.geo;
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TX;  // domain coords of the tile origin
  const int y0 = blockIdx.y * TY;

  // The loaded box starts at domain (x0-4, y0-4) = padded (x0, y0).
  for (int idx = tid; idx < LBOX; idx += NT) {
    int ly = idx / LX, lx = idx - ly * LX;
    int py = y0 + ly, px = x0 + lx;
    bool ok = (py < g.prow) && (px < g.pitch);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      C v = CxOps<R>::mk(R(0), R(0));
      if (ok) v = a.psi_in[c * g.plane + (long long)py * g.pitch + px];
      ybuf0[c * LBOX + idx] = v;
      ybuf1[c * LBOX + idx] = v;
    }
  }

  // Drive phases exp(-i omega t_s) / hbar of the four stages (FP64 sincos on
  // four threads; published by the barrier below).
  __shared__ R s_dph[4][2];
  if (DRV && tid < 4) {
    const double ts = a.clock->t[a.parity] +
                      (tid == 0 ? 0.0 : (tid == 3 ? a.dt64 : 0.5 * a.dt64));
    double sn, cs;
    sincos(a.omega * ts, &sn, &cs);
    s_dph[tid][0] = R(cs) * a.k.inv_hbar;
    s_dph[tid][1] = R(-sn) * a.k.inv_hbar;
  }

  // Per-point state (fixed ownership across the four stages).
  C psi0[PPT][NC], acc[PPT][NC];
  R n0[PPT][NC], ncur[PPT][NC], nacc[PPT][NC], Pv[PPT][NC], Vv[PPT];
  bool valid[PPT], inside[PPT];
  int sidx[PPT];
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    int idx = tid + k * NT;
    valid[k] = idx < NPT;
    int ry = valid[k] ? idx / RXN : 0;
    int rx = valid[k] ? idx - ry * RXN : 0;
    sidx[k] = (ry + 1) * LX + (rx + 1);
    int gx = x0 - 3 + rx, gy = y0 - 3 + ry;
    inside[k] = (g.bc_x == BC_PERIODIC || (gx >= 0 && gx < g.nx)) &&
                (g.bc_y == BC_PERIODIC || (gy >= 0 && gy < g.ny));
    int py = gy + HALO, px = gx + HALO;
    bool ok = valid[k] && py < g.prow && px < g.pitch;
    long long off = (long long)py * g.pitch + px;
    Vv[k] = (ok && a.V) ? a.V[off] : R(0);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      acc[k][c] = CxOps<R>::mk(R(0), R(0));
      nacc[k][c] = R(0);
      if (RES) {
        n0[k][c] = ok ? a.n_in[c * g.plane + off] : R(0);
        Pv[k][c] = ok ? a.P[c * a.P_comp_stride + off] : R(0);
      } else {
        n0[k][c] = R(0);
        Pv[k][c] = R(0);
      }
      ncur[k][c] = n0[k][c];
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < PPT; ++k)
#pragma unroll
    for (int c = 0; c < NC; ++c) psi0[k][c] = ybuf0[c * LBOX + sidx[k]];

  const CoeffsT<R>& q = a.k;
  const R ax = q.ax, ay = q.ay, a0 = q.a0;
  const R cg = q.g, cgx = q.gx, cgr = q.gr, cih = q.inv_hbar;
  const R hR = q.half_R, hgc = q.half_gc, cR = q.R_, cgr_ = q.gamma_r;
  const R tx = q.tx, ty = q.ty, txy = q.txy;
  const R dt = q.dt;

#pragma unroll 1
  for (int s = 0; s < 4; ++s) {
    const C* yc = (s & 1) ? ybuf1 : ybuf0;
    C* yn = (s & 1) ? ybuf0 : ybuf1;
    const R w = (s == 0 || s == 3) ? R(1) : R(2);
    const R cstep = (s == 2) ? dt : R(0.5) * dt;
    const R dph_re = DRV ? s_dph[s][0] : R(0), dph_im = DRV ? s_dph[s][1] : R(0);
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      if (!valid[k]) continue;
      const int si = sidx[k];
      C cen[NC], lapc[NC];
      R dens[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const C* b = yc + c * LBOX;
        C Cc = b[si], E = b[si + 1], W = b[si - 1], N = b[si + LX], S = b[si - LX];
        cen[c] = Cc;
        // (H_lap / hbar) = ax (E + W) + ay (N + S) + a0 C
        lapc[c].x = ax * (E.x + W.x) + ay * (N.x + S.x) + a0 * Cc.x;
        lapc[c].y = ax * (E.y + W.y) + ay * (N.y + S.y) + a0 * Cc.y;
        dens[c] = Cc.x * Cc.x + Cc.y * Cc.y;
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int o = NC - 1 - c;
        R n_c = ncur[k][c];
        R loc = cg * dens[c] + Vv[k] * cih;
        if (NC == 2) loc += cgx * dens[o];
        if (RES) loc += cgr * n_c;
        C H;
        H.x = lapc[c].x + loc * cen[c].x;
        H.y = lapc[c].y + loc * cen[c].y;
        if (TETM) {
          const C* b = yc + o * LBOX;
          C Co = b[si], E = b[si + 1], W = b[si - 1], N = b[si + LX], S = b[si - LX];
          C NE = b[si + LX + 1], NW = b[si + LX - 1], SE = b[si - LX + 1], SW = b[si - LX - 1];
          // (Dxx - Dyy) psi_o and the mixed difference (4-corner stencil)
          R dre = tx * (E.x + W.x - R(2) * Co.x) - ty * (N.x + S.x - R(2) * Co.x);
          R dim = tx * (E.y + W.y - R(2) * Co.y) - ty * (N.y + S.y - R(2) * Co.y);
          R xre = txy * ((NE.x - SE.x) - (NW.x - SW.x));
          R xim = txy * ((NE.y - SE.y) - (NW.y - SW.y));
          // J_+ (c = 0) = D - 2i Dxy ; J_- (c = 1) = D + 2i Dxy; txy = Delta/(2h dx dy)
          // so 2 Dxy-term = xre + i xim (already includes the factor 2/4).
          if (c == 0) {
            H.x += dre + xim;
            H.y += dim - xre;
          } else {
            H.x += dre - xim;
            H.y += dim + xre;
          }
        }
        if (DRV) {  // + E_c(r) exp(-i omega t_s) / hbar
          // the box position si is padded site (y0 + si / LX, x0 + si % LX)
          const int py = y0 + si / LX, px = x0 + si % LX;
          if (py < g.prow && px < g.pitch) {
            const R* Ec = a.E + c * a.E_comp_stride + (long long)py * g.pitch + px;
            C e;
            e.x = __ldg(Ec);
            e.y = __ldg(Ec + g.plane);
            H.x += e.x * dph_re - e.y * dph_im;
            H.y += e.x * dph_im + e.y * dph_re;
          }
        }
        R G = -hgc;
        if (RES) G += hR * n_c;
        // K = -i H/hbar + G psi   (H already divided by hbar)
        C K;
        K.x = H.y + G * cen[c].x;
        K.y = -H.x + G * cen[c].y;
        acc[k][c].x += w * K.x;
        acc[k][c].y += w * K.y;
        R Kn = R(0);
        if (RES) {
          Kn = Pv[k][c] - (cgr_ + cR * dens[c]) * n_c;
          nacc[k][c] += w * Kn;
        }
        if (s < 3) {
          C y;
          y.x = psi0[k][c].x + cstep * K.x;
          y.y = psi0[k][c].y + cstep * K.y;
          if (!inside[k]) y = CxOps<R>::mk(R(0), R(0));
          yn[c * LBOX + si] = y;
          if (RES) ncur[k][c] = n0[k][c] + cstep * Kn;
        }
      }
    }
    __syncthreads();
  }

  // Final combination and write-back of the output tile.
  const long long step = a.clock->step[a.parity];
  if (blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) {
    a.clock->step[a.parity ^ 1] = step + 1;
    a.clock->t[a.parity ^ 1] = a.clock->t[a.parity] + a.dt64;
  }
  const R dt6 = dt / R(6);
  // Noise is drawn in a grid-uniform branch of its own so that the generator
  // is never issued (predicated off) when noise is disabled.
  float2 xi[PPT][2];
  if (a.noise.on) {
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      int idx = tid + k * NT;
      int ry = idx / RXN, rx = idx - ry * RXN;
      int gx = x0 - 3 + rx, gy = y0 - 3 + ry;
      xi[k][0] = xi[k][1] = make_float2(0.f, 0.f);
      if (valid[k] && gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny) {
        float s0 = a.noise.scale, s1 = a.noise.scale;
        if (a.noise.twa) {  // variance from the reservoir at the step's start
          const NoiseKey& z = a.noise;
          s0 = nz_wigner_scale(z.R, z.gc, z.kw, z.var, RES ? (float)n0[k][0] : 0.f);
          if (NC == 2)
            s1 = nz_wigner_scale(z.R, z.gc, z.kw, z.var, RES ? (float)n0[k][NC - 1] : 0.f);
        }
        nz_site2(a.noise.seed, a.noise.instance, step, (uint32_t)(gy * g.nx + gx),
                 s0, s1, xi[k][0], xi[k][1], NC == 2);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    if (!valid[k]) continue;
    int idx = tid + k * NT;
    int ry = idx / RXN, rx = idx - ry * RXN;
    if (rx < 3 || rx >= 3 + TX || ry < 3 || ry >= 3 + TY) continue;
    int gx = x0 - 3 + rx, gy = y0 - 3 + ry;
    if (gx >= g.nx || gy >= g.ny) continue;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      C out;
      out.x = psi0[k][c].x + acc[k][c].x * dt6;
      out.y = psi0[k][c].y + acc[k][c].y * dt6;
      if (a.noise.on) {
        out.x = out.x + R(xi[k][c].x);
        out.y = out.y + R(xi[k][c].y);
      }
      store_with_ghosts(a.psi_out + c * g.plane, g, gx, gy, out);
      if (RES) {
        R nn = n0[k][c] + nacc[k][c] * dt6;
        store_with_ghosts(a.n_out + c * g.plane, g, gx, gy, nn);
      }
    }
  }
}

template <typename R, int NC, bool RES, bool TETM, int TX, int TY, int NT, bool DRV>
cudaError_t launch_generic_k(const StepArgs<R>& a, cudaStream_t s) {
  using C = typename CxOps<R>::C;
  constexpr int LBOX = (TX + 2 * HALO) * (TY + 2 * HALO);
  size_t smem = 2 * NC * LBOX * sizeof(C);
  auto kern = rk4_step_generic<R, NC, RES, TETM, TX, TY, NT, DRV>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(
        kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  dim3 grid((a.geo.nx + TX - 1) / TX, (a.geo.ny + TY - 1) / TY);
  kern<<<grid, NT, smem, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

// The drive term is compiled in only where a drive is set (a.E != nullptr),
// so undriven steps keep the register budget of the plain equations.
template <typename R, int NC, bool RES, bool TETM, int TX, int TY, int NT>
cudaError_t launch_generic(const StepArgs<R>& a, cudaStream_t s) {
  if (a.E) return launch_generic_k<R, NC, RES, TETM, TX, TY, NT, true>(a, s);
  return launch_generic_k<R, NC, RES, TETM, TX, TY, NT, false>(a, s);
}

}  // namespace phx
