#pragma once
// Persistent, TMA-fed fused RK4 step for the FP32 two-component field with
// reservoirs (Eq. PULSE_psi / PULSE_res, c in {+, -}), with or without the
// TE-TM coupling J_c psi_o and a potential V.
//
// Same scheme as the scalar kernel: one CTA per SM walks a tile list; one
// cp.async.bulk.tensor per field fetches both component planes of the tile
// box (box depth 2) into a double buffer; thread (lane, warp) owns a 2-column
// x MR-row micro-tile of the region for both components, with psi0, the
// stage value, the accumulator and the reservoir values in registers; rows
// above and below cross shared memory, east/west neighbours and the corner
// neighbours of the mixed difference come from the neighbouring lanes by
// warp shuffles (from the loaded box in the first stage).  Per site and
// component, with o the other component:
//   H_c/hbar = ax (E+W) + ay (N+S) + (a0 + V/hbar + g|psi_c|^2 + g_x|psi_o|^2
//              + g_r n_c) psi_c + J_c psi_o,
//   J_c psi_o / hbar = tx (E_o + W_o - 2 psi_o) - ty (N_o + S_o - 2 psi_o)
//                      -/+ i txy (NE_o - NW_o - SE_o + SW_o),
//   K_c = -i H_c/hbar + (R n_c - gamma_c)/2 psi_c,
//   K_n,c = P_c - (gamma_r + R |psi_c|^2) n_c.
#include "rk4_tma_kernel.cuh"

namespace phx {
namespace tma {

template <bool POT, int MR, int WY>
struct SCfg {
  static constexpr int RW = 64;
  static constexpr int RH = MR * WY;
  static constexpr int TX = RW - 6, TY = RH - 6;
  static constexpr int PW = RW + 4;  // psi smem row: 2 alignment cols, ring, region, ring
  static constexpr int PH = RH + 2;
  static constexpr int FW = RW + 4;
  static constexpr int NT = 32 * WY;
  static constexpr int PSI_PLANE = PH * PW;  // float2 elements per component plane
  static constexpr int F_PLANE = RH * FW;    // floats per plane
  static constexpr int PSI_BYTES = ((2 * PSI_PLANE * 8) + 127) / 128 * 128;
  static constexpr int N_BYTES = ((2 * F_PLANE * 4) + 127) / 128 * 128;  // n (or P): two planes
  static constexpr int V_BYTES = ((F_PLANE * 4) + 127) / 128 * 128;
  static constexpr int BUF_BYTES = PSI_BYTES + 2 * N_BYTES + (POT ? V_BYTES : 0);
  static constexpr int TX_BYTES = 2 * PSI_PLANE * 8 + 4 * F_PLANE * 4 + (POT ? F_PLANE * 4 : 0);
  static constexpr int NBUF = 2;
  static constexpr int SMEM = NBUF * BUF_BYTES + PSI_BYTES + 128;
};

template <bool POT, bool PER, bool ONE, bool TETM, int MR, int WY>
__global__ void __launch_bounds__(32 * WY, 1) rk4_f32_tma_spinor(const TileArgs ta) {
  using C = SCfg<POT, MR, WY>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[2];
  unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  float2* Y = reinterpret_cast<float2*>(base + C::NBUF * C::BUF_BYTES);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c0 = 2 * lane;
  const int r0 = MR * warp;
  auto psi_buf = [&](int b) { return reinterpret_cast<float2*>(base + b * C::BUF_BYTES); };
  auto n_buf = [&](int b) {
    return reinterpret_cast<float*>(base + b * C::BUF_BYTES + C::PSI_BYTES);
  };
  auto p_buf = [&](int b) {
    return reinterpret_cast<float*>(base + b * C::BUF_BYTES + C::PSI_BYTES + C::N_BYTES);
  };
  auto v_buf = [&](int b) {
    return reinterpret_cast<float*>(base + b * C::BUF_BYTES + C::PSI_BYTES + 2 * C::N_BYTES);
  };

  for (int i = tid; i < 2 * C::PSI_PLANE; i += C::NT) {
    const int k = i % C::PSI_PLANE;
    const int r = k / C::PW, c = k - r * C::PW;
    if (r == 0 || r == C::PH - 1 || c < 2 || c >= C::RW + 2) Y[i] = f2(0.f, 0.f);
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");

  const int tiles_x1 = ONE ? ta.one.tiles_x : 1;
  struct Coord {
    int inst, kx, ky;
  };
  auto coord_of = [&](int t) {
    Coord c;
    if (ONE) {
      c.inst = 0;
      c.ky = t / tiles_x1;
      c.kx = t - c.ky * tiles_x1;
    } else {
      const int2 v = ta.tile_info[t];
      c.inst = v.x;
      c.kx = v.y & 0xffff;
      c.ky = v.y >> 16;
    }
    return c;
  };
  auto issue = [&](const Coord& c, int b) {
    const TileInst* I = ta.inst + c.inst;
    const int xp = c.kx * C::TX, yp = c.ky * C::TY;
    mbar_arrive_expect_tx(&bar[b], C::TX_BYTES);
    tma_load_3d(psi_buf(b), &I->psi[ta.cur], 2 * (xp - 2), yp, 0, &bar[b]);
    tma_load_3d(n_buf(b), &I->n[ta.cur], xp & ~3, yp + 1, 0, &bar[b]);
    tma_load_3d(p_buf(b), &I->P, xp & ~3, yp + 1, 0, &bar[b]);
    if (POT) tma_load_3d(v_buf(b), &I->V, xp & ~3, yp + 1, 0, &bar[b]);
  };

  const long long step = ta.clock->step[ta.parity];
  if (blockIdx.x == 0 && tid == 0) {
    ta.clock->step[ta.parity ^ 1] = step + 1;
    ta.clock->t[ta.parity ^ 1] = ta.clock->t[ta.parity] + ta.inst[0].dt64;
  }

  int t = blockIdx.x, k = 0;
  if (tid == 0 && t < ta.ntiles && !ta.inject_timeout) issue(coord_of(t), 0);
  for (; t < ta.ntiles; t += gridDim.x, ++k) {
    const int b = k & 1;
    const uint32_t par = (uint32_t)((k >> 1) & 1);
    const int tn = t + (int)gridDim.x;
    const int fail = !mbar_wait_bounded(&bar[b], par);
    if (__syncthreads_or(fail)) {
      if (tid == 0) atomicExch(ta.err, 1);
      return;
    }
    if (tid == 0 && tn < ta.ntiles) {
      fence_proxy_async();
      issue(coord_of(tn), b ^ 1);
    }

    const Coord cc = coord_of(t);
    const TileInst* I = ta.inst + cc.inst;
    const Geometry g = ONE ? ta.one.geo : I->geo;
    float2* const psi_out = ONE ? ta.one.psi_buf[ta.cur ^ 1] : I->psi_buf[ta.cur ^ 1];
    float* const n_out = ONE ? ta.one.n_buf[ta.cur ^ 1] : I->n_buf[ta.cur ^ 1];
    const CoeffsT<float> q = ONE ? ta.one.k : I->k;
    const NoiseKey nz = ONE ? ta.one.noise : I->noise;
    const int p_shared = ONE ? ta.one.p_shared : 0;
    const float2 ax2 = f2(q.ax, q.ax), ay2 = f2(q.ay, q.ay);
    // real coefficients as pairs: the real-valued terms (density, local
    // term, gain, reservoir) of a micro-tile row's two columns go through the
    // packed FP32x2 instructions together
    const float2 cg2 = f2(q.g, q.g), cgx2 = f2(q.gx, q.gx), cgr2 = f2(q.gr, q.gr);
    const float2 cih2 = f2(q.inv_hbar, q.inv_hbar), a02 = f2(q.a0, q.a0);
    const float2 hR2 = f2(q.half_R, q.half_R), nhgc2 = f2(-q.half_gc, -q.half_gc);
    const float2 ncR2 = f2(-q.R_, -q.R_), ncgam2 = f2(-q.gamma_r, -q.gamma_r);
    const float dt = q.dt;
    const float2 tx2 = f2(q.tx, q.tx), nty2 = f2(-q.ty, -q.ty);
    const float2 dg2 = f2(2.f * (q.ty - q.tx), 2.f * (q.ty - q.tx));
    const float2 m12 = f2(-1.f, -1.f);
    const float txy = q.txy;
    const float dt6 = q.dt6;  // dt / 6, divided once on the host
    const int xp = cc.kx * C::TX;
    const int foff = xp & 3;
    float2* P0 = psi_buf(b);
    const float* Nb = n_buf(b);
    const float* Pb = p_buf(b);
    const float* Vb = POT ? v_buf(b) : nullptr;

    // complex values [row][column][component]; real fields as pairs over the
    // row's two columns, [row][component].  n0 and P are read again from the
    // tile's shared n and P boxes (which no stage overwrites) where they are
    // used, which keeps the register budget of 16 warps per CTA.
    float2 p0[MR][2][2], yc[MR][2][2], acc[MR][2][2];
    float2 nc[MR][2], na[MR][2], Vv[MR];
    bool ins[MR][2];
    const int gx0 = xp - HALO + c0;
    const int gy0 = cc.ky * C::TY - 3 + r0;
    // foff + c0 is even and a plane holds an even number of floats: the pair
    // of a row is one 8-byte load
    auto ld2 = [&](const float* p, int j) {
      return *reinterpret_cast<const float2*>(&p[(r0 + j) * C::FW + foff + c0]);
    };
    auto N0 = [&](int j, int c) { return ld2(Nb + c * C::F_PLANE, j); };
    auto PV = [&](int j, int c) { return ld2(Pb + (p_shared ? 0 : c) * C::F_PLANE, j); };
#pragma unroll
    for (int j = 0; j < MR; ++j) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float4 v =
            *reinterpret_cast<const float4*>(&P0[c * C::PSI_PLANE + (r0 + j + 1) * C::PW + c0 + 2]);
        p0[j][0][c] = f2(v.x, v.y);
        p0[j][1][c] = f2(v.z, v.w);
        yc[j][0][c] = p0[j][0][c];
        yc[j][1][c] = p0[j][1][c];
      }
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int gx = gx0 + i, gy = gy0 + j;
        ins[j][i] = PER || ((g.bc_x == BC_PERIODIC || (gx >= 0 && gx < g.nx)) &&
                            (g.bc_y == BC_PERIODIC || (gy >= 0 && gy < g.ny)));
      }
      // the stencil's diagonal a0 rides with the local potential
      Vv[j] = POT ? __ffma2_rn(ld2(Vb, j), cih2, a02) : a02;
#pragma unroll
      for (int c = 0; c < 2; ++c) nc[j][c] = N0(j, c);
    }

#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const float2* src = (s & 1) ? Y : P0;
      float2* dst = (s & 1) ? P0 : Y;
      const float w = (s == 0 || s == 3) ? 1.f : 2.f;
      const float cs = (s == 2) ? dt : 0.5f * dt;
      const float2 w2 = f2(w, w), cs2 = f2(cs, cs);
      // rows above (S) and below (N) of the micro-tile, both components
      float2 Sr[2][2], Nr[2][2];  // [column][component]
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float4 tv =
            *reinterpret_cast<const float4*>(&src[c * C::PSI_PLANE + r0 * C::PW + c0 + 2]);
        const float4 bv = *reinterpret_cast<const float4*>(
            &src[c * C::PSI_PLANE + (r0 + MR + 1) * C::PW + c0 + 2]);
        Sr[0][c] = f2(tv.x, tv.y);
        Sr[1][c] = f2(tv.z, tv.w);
        Nr[0][c] = f2(bv.x, bv.y);
        Nr[1][c] = f2(bv.z, bv.w);
      }
      // west / east neighbours of every row of the micro-tile and of the
      // rows above and below (the corners of the mixed difference):
      // index 0 = row above, 1..MR = own rows, MR+1 = row below
      float2 Wv[MR + 2][2], Ev[MR + 2][2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
#pragma unroll
        for (int j = 0; j < MR + 2; ++j) {
          if (!TETM && (j == 0 || j == MR + 1)) continue;
          if (s == 0) {
            const float2* row = &src[c * C::PSI_PLANE + (r0 + j) * C::PW];
            Wv[j][c] = row[c0 + 1];
            Ev[j][c] = row[c0 + 4];
          } else {
            const float2 lo = j == 0 ? Sr[0][c] : (j == MR + 1 ? Nr[0][c] : yc[j - 1][0][c]);
            const float2 hi = j == 0 ? Sr[1][c] : (j == MR + 1 ? Nr[1][c] : yc[j - 1][1][c]);
            Wv[j][c].x = __shfl_up_sync(0xffffffffu, hi.x, 1);
            Wv[j][c].y = __shfl_up_sync(0xffffffffu, hi.y, 1);
            Ev[j][c].x = __shfl_down_sync(0xffffffffu, lo.x, 1);
            Ev[j][c].y = __shfl_down_sync(0xffffffffu, lo.y, 1);
          }
        }
      }
      // value at (row index jj in 0..MR+1, column ii in -1..2) of component c
      auto at = [&](int jj, int ii, int c) -> float2 {
        if (ii < 0) return Wv[jj][c];
        if (ii > 1) return Ev[jj][c];
        if (jj == 0) return Sr[ii][c];
        if (jj == MR + 1) return Nr[ii][c];
        return yc[jj - 1][ii][c];
      };
      float2 ny[MR][2][2];
      float2 nn[MR][2];
#pragma unroll
      for (int j = 0; j < MR; ++j) {
        const int jj = j + 1;
        // |psi_c|^2 of the row's two sites, per component
        float2 dens[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          dens[c].x = fmaf(yc[j][0][c].x, yc[j][0][c].x, yc[j][0][c].y * yc[j][0][c].y);
          dens[c].y = fmaf(yc[j][1][c].x, yc[j][1][c].x, yc[j][1][c].y * yc[j][1][c].y);
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int o = 1 - c;
          // a0 + V/hbar + g|psi_c|^2 + g_x|psi_o|^2 + g_r n_c and
          // (R n_c - gamma_c)/2 for both sites
          float2 loc = __ffma2_rn(cg2, dens[c], Vv[j]);
          loc = __ffma2_rn(cgx2, dens[o], loc);
          loc = __ffma2_rn(cgr2, nc[j][c], loc);
          const float2 G = __ffma2_rn(hR2, nc[j][c], nhgc2);
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            const float2 Cc = yc[j][i][c];
            const float2 E = at(jj, i + 1, c), W = at(jj, i - 1, c);
            const float2 N = at(jj + 1, i, c), S = at(jj - 1, i, c);
            float2 H = __fmul2_rn(ay2, __fadd2_rn(N, S));
            H = __ffma2_rn(ax2, __fadd2_rn(E, W), H);
            const float li = i ? loc.y : loc.x;
            H = __ffma2_rn(f2(li, li), Cc, H);
            if (TETM) {
              // tx (E+W-2C) - ty (N+S-2C) = tx (E+W) - ty (N+S) + 2 (ty - tx) C
              // of the other component, accumulated into H
              const float2 Co = yc[j][i][o];
              const float2 Eo = at(jj, i + 1, o), Wo = at(jj, i - 1, o);
              const float2 No = at(jj + 1, i, o), So = at(jj - 1, i, o);
              H = __ffma2_rn(tx2, __fadd2_rn(Eo, Wo), H);
              H = __ffma2_rn(nty2, __fadd2_rn(No, So), H);
              H = __ffma2_rn(dg2, Co, H);
              // Q = NE - NW - SE + SW of the other component; J_+ adds
              // -i txy Q, J_- adds +i txy Q
              const float2 NEo = at(jj + 1, i + 1, o), NWo = at(jj + 1, i - 1, o);
              const float2 SEo = at(jj - 1, i + 1, o), SWo = at(jj - 1, i - 1, o);
              const float2 Q = __ffma2_rn(m12, __fadd2_rn(NWo, SEo), __fadd2_rn(NEo, SWo));
              const float sx = c == 0 ? txy : -txy;
              H.x = fmaf(sx, Q.y, H.x);
              H.y = fmaf(-sx, Q.x, H.y);
            }
            const float Gi = i ? G.y : G.x;
            float2 K;
            K.x = fmaf(Gi, Cc.x, H.y);
            K.y = fmaf(Gi, Cc.y, -H.x);
            acc[j][i][c] = s == 0 ? K : __ffma2_rn(w2, K, acc[j][i][c]);
            ny[j][i][c] = __ffma2_rn(cs2, K, p0[j][i][c]);
            if (!PER && !ins[j][i]) ny[j][i][c] = f2(0.f, 0.f);
          }
          // K_n = P - (gamma_r + R|psi_c|^2) n_c for both sites
          const float2 Kn = __ffma2_rn(__ffma2_rn(ncR2, dens[c], ncgam2), nc[j][c], PV(j, c));
          na[j][c] = s == 0 ? Kn : __ffma2_rn(w2, Kn, na[j][c]);
          nn[j][c] = __ffma2_rn(cs2, Kn, N0(j, c));
        }
      }
      if (s < 3) {
#pragma unroll
        for (int j = 0; j < MR; ++j) {
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            yc[j][0][c] = ny[j][0][c];
            yc[j][1][c] = ny[j][1][c];
            nc[j][c] = nn[j][c];
            if (j == 0 || j == MR - 1)
              *reinterpret_cast<float4*>(&dst[c * C::PSI_PLANE + (r0 + j + 1) * C::PW + c0 + 2]) =
                  make_float4(ny[j][0][c].x, ny[j][0][c].y, ny[j][1][c].x, ny[j][1][c].y);
          }
        }
        __syncthreads();
      }
    }

    // psi' = psi0 + (K1 + 2K2 + 2K3 + K4) dt/6 (+ noise), both components
    const float2 d62 = f2(dt6, dt6);
    float2 o[MR][2][2];
    float2 on[MR][2];
#pragma unroll
    for (int j = 0; j < MR; ++j)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
#pragma unroll
        for (int i = 0; i < 2; ++i) o[j][i][c] = __ffma2_rn(d62, acc[j][i][c], p0[j][i][c]);
        on[j][c] = __ffma2_rn(d62, na[j][c], N0(j, c));
      }
    if (nz.on) {
#pragma unroll
      for (int j = 0; j < MR; ++j) {
        const int gy = gy0 + j;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const int gx = gx0 + i;
          const uint32_t site = (uint32_t)(((gy % g.ny + g.ny) % g.ny) * g.nx +
                                           (gx % g.nx + g.nx) % g.nx);
          float2 xp_, xm_;
          float s0 = nz.scale, s1 = nz.scale;
          if (nz.twa) {
            s0 = nz_wigner_scale(nz.R, nz.gc, nz.kw, nz.var, i ? N0(j, 0).y : N0(j, 0).x);
            s1 = nz_wigner_scale(nz.R, nz.gc, nz.kw, nz.var, i ? N0(j, 1).y : N0(j, 1).x);
          }
          nz_site2(nz.seed, nz.instance, step, site, s0, s1, xp_, xm_, true);
          o[j][i][0].x = o[j][i][0].x + xp_.x;
          o[j][i][0].y = o[j][i][0].y + xp_.y;
          o[j][i][1].x = o[j][i][1].x + xm_.x;
          o[j][i][1].y = o[j][i][1].y + xm_.y;
        }
      }
    }
    // Interior tiles (no ghost image, no clipping): 16-byte psi and 8-byte n
    // stores per micro-tile row and component.
    const int ox0 = xp - 1, oy0 = cc.ky * C::TY;
    const bool interior = ox0 >= HALO && ox0 + C::TX <= g.nx - HALO && oy0 >= HALO &&
                          oy0 + C::TY <= g.ny - HALO;
    if (interior) {
      const bool lo = c0 >= 3 && c0 < 3 + C::TX;
      const bool hi = c0 + 1 >= 3 && c0 + 1 < 3 + C::TX;
#pragma unroll
      for (int j = 0; j < MR; ++j) {
        const int r = r0 + j;
        if (r < 3 || r >= 3 + C::TY) continue;  // warp-uniform
        const long long roff = (long long)(gy0 + j + HALO) * g.pitch + gx0 + HALO;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          float2* po = psi_out + c * g.plane + roff;
          float* pn = n_out + c * g.plane + roff;
          if (lo && hi) {
            *reinterpret_cast<float4*>(po) =
                make_float4(o[j][0][c].x, o[j][0][c].y, o[j][1][c].x, o[j][1][c].y);
            *reinterpret_cast<float2*>(pn) = on[j][c];
          } else if (lo || hi) {  // one path for both edge lanes
            const int one = lo ? 0 : 1;
            po[one] = lo ? o[j][0][c] : o[j][1][c];
            pn[one] = lo ? on[j][c].x : on[j][c].y;
          }
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < MR; ++j) {
        const int r = r0 + j;
        const int gy = gy0 + j;
        if (r < 3 || r >= 3 + C::TY || gy >= g.ny) continue;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const int cix = c0 + i, gx = gx0 + i;
          if (cix < 3 || cix >= 3 + C::TX || gx < 0 || gx >= g.nx) continue;
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            store_with_ghosts(psi_out + c * g.plane, g, gx, gy, o[j][i][c]);
            store_with_ghosts(n_out + c * g.plane, g, gx, gy, i ? on[j][c].y : on[j][c].x);
          }
        }
      }
    }
  }
}

template <bool POT, bool PER, bool ONE, bool TETM, int MR, int WY>
cudaError_t launch_spinor_cfg(const TileArgs& ta, cudaStream_t s, int grid) {
  using C = SCfg<POT, MR, WY>;
  auto kern = rk4_f32_tma_spinor<POT, PER, ONE, TETM, MR, WY>;
  static int configured_dev = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_dev != dev) {
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    configured_dev = dev;
  }
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(grid);
  lc.blockDim = dim3(C::NT);
  lc.dynamicSmemBytes = C::SMEM;
  lc.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&lc, kern, ta);
  count_launch();
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int MR, int WY>
cudaError_t launch_spinor_variants(bool pot, bool per, bool one, bool tetm, const TileArgs& ta,
                                   cudaStream_t s, int grid) {
#define PHX_SP_V(ONE_, TETM_)                                                         \
  if (per) {                                                                          \
    if (pot) return launch_spinor_cfg<true, true, ONE_, TETM_, MR, WY>(ta, s, grid);  \
    return launch_spinor_cfg<false, true, ONE_, TETM_, MR, WY>(ta, s, grid);          \
  }                                                                                   \
  if (pot) return launch_spinor_cfg<true, false, ONE_, TETM_, MR, WY>(ta, s, grid);   \
  return launch_spinor_cfg<false, false, ONE_, TETM_, MR, WY>(ta, s, grid);
  if (one) {
    if (tetm) {
      PHX_SP_V(true, true)
    }
    PHX_SP_V(true, false)
  }
  if (tetm) {
    PHX_SP_V(false, true)
  }
  PHX_SP_V(false, false)
#undef PHX_SP_V
}

}  // namespace tma
}  // namespace phx
