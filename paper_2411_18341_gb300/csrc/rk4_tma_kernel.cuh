#pragma once
// Kernel template of the persistent, TMA-fed fused RK4 step for the FP32
// scalar field (Eq. 1 / Eq. PULSE_psi with one component, optionally with the
// reservoir of Eq. PULSE_res or a coherent drive E(r) exp(-i omega t), and a
// potential V).
//
// Per CTA (one or two per SM, 32*WY threads) a loop over output tiles:
//   * the next tiles' psi box (tile + depth-4 halo) and n, P, V boxes are
//     fetched by cp.async.bulk.tensor into a ring of two or three buffers
//     while the current tile is computed (mbarrier completion, bounded waits);
//   * thread (lane, warp) owns a 2-column x MR-row micro-tile of the ring-3
//     region: psi0, the running stage value, the accumulator sum_k w_k K_k and
//     the reservoir values stay in registers across the four stages; between
//     stages only the micro-tile's first and last rows cross shared memory
//     (read by the warps above and below, 16-byte accesses), east/west
//     neighbours come from the neighbouring lanes by warp shuffles;
//   * complex arithmetic uses the packed FP32x2 instructions of sm_100+
//     (__ffma2_rn / __fadd2_rn / __fmul2_rn on (re, im) pairs);
//   * psi' = psi0 + (K1 + 2K2 + 2K3 + K4) dt/6 (+ noise) is stored with
//     16-byte stores, plus the periodic ghost images near the domain edges.
// Tiles are offset by one column (tile kx covers domain columns
// [kx*TX - 1, kx*TX - 1 + TX)) so that every 16-byte alignment rule holds:
// the psi box starts at an even padded column, micro-tile columns are even.
#include <cuda.h>
#include <cuda_runtime.h>

#include "phx_internal.h"
#include "phx_noise.cuh"
#include "rk4_generic.cuh"
#include "rk4_tma.h"

namespace phx {
namespace tma {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for phase `parity` of `bar`, giving up after ~0.25 s; backs off with
// __nanosleep after the first few polls so waiting warps leave issue slots.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (it >= 4) __nanosleep(64);
    if ((it & 63u) == 63u && global_ns() - t0 > 250000000ull) return false;
  }
}

// Completion counters of the multi-step launch: relaxed loads and stores at
// GPU scope; the ordering comes from fence.acq_rel.gpu around them.
__device__ __forceinline__ int ld_relaxed_gpu(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_gpu(int* p, int v) {
  asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_acq_rel_gpu() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}
// orders this thread's generic-proxy view of global memory (data other CTAs
// stored, acquired above) before its following async-proxy (TMA) reads
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y,
                                            int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// MODE: 0 = no reservoir, 1 = reservoir (n and P planes), 2 = coherent
// drive without reservoir (Re E and Im E planes in the n and P slots),
// 3 = reservoir and coherent drive (n, P, Re E, Im E planes).
template <int MODE, bool POT, int MR, int WY, int MINB = 1>
struct Cfg {
  static constexpr int RW = 64;            // region (ring-3) columns: one warp x 2 cols
  static constexpr int RH = MR * WY;       // region rows
  static constexpr int TX = RW - 6, TY = RH - 6;
  static constexpr int PW = RW + 4;        // psi smem row: 2 alignment cols, ring, region, ring
  static constexpr int PH = RH + 2;        // psi smem rows: ring, region, ring
  static constexpr int FW = RW + 4;        // n / P / V smem row (4-float aligned box)
  static constexpr int NT = 32 * WY;
  static constexpr int NF = (MODE == 3 ? 4 : (MODE != 0 ? 2 : 0)) + (POT ? 1 : 0);
  static constexpr int PSI_BYTES = ((PH * PW * 8) + 127) / 128 * 128;
  static constexpr int F_BYTES = ((RH * FW * 4) + 127) / 128 * 128;
  static constexpr int BUF_BYTES = PSI_BYTES + NF * F_BYTES;
  static constexpr int TX_BYTES = PH * PW * 8 + NF * RH * FW * 4;  // bytes one tile brings
  // Input buffers: one per tile in flight (three when shared memory allows,
  // so that a CTA with three tiles has all its loads in flight at once).
  // (Two buffers when two CTAs share an SM.)
  static constexpr int NBUF =
      (MINB == 1 && 3 * BUF_BYTES + PSI_BYTES + 128 <= 227 * 1024) ? 3 : 2;
  static constexpr int SMEM = NBUF * BUF_BYTES + PSI_BYTES + 128;
  // A second stage-exchange buffer, where shared memory allows it (per CTA,
  // and for the CTAs that share an SM): consecutive tiles of a CTA then use
  // different exchange buffers, which lets the kernel drop the barrier at a
  // tile's start (see the kernel).
  static constexpr int SMEM_YY = SMEM + PSI_BYTES;
  static constexpr bool YY_FITS =
      SMEM_YY <= 227 * 1024 && MINB * (SMEM_YY + 1024) <= 228 * 1024;
};

// PER: both axes periodic (every ring cell holds a periodic image, so no
// stage value needs forcing to zero).
// ONE: a single instance, whose scalars come from the kernel parameters
// (ta.one: constant-bank operands, hoisted out of the tile loop) and whose
// tile coordinates advance incrementally; otherwise per-tile instance
// records and precomputed tile coordinates (ta.tile_info).
//
// MS: ta.ms_steps steps in one launch (single instance, no drive).  Work item
// i = s * ntiles + pos is tile pos of step s; CTA c takes items c, c + G,
// c + 2G, ... (G = gridDim.x), so no CTA idles at a step boundary.  Tile
// rows are visited in the folded order 0, ty-1, 1, ty-2, ..., which puts the
// rows a tile depends on (its own and the two next to it, periodic wrap
// included) within two positions of its own, and rows 0 and ty-2 (which
// depend on each other through the ghost rows when the last tile row is thin,
// see dep_axis) within three.  A tile's load for step s is issued once the
// counters done[] of the tiles it exchanges data with reached s: their
// outputs of step s-1 (the input of step s) are stored, and their reads of
// the buffer that step s writes are over.  Warp 0 loads the counters of the
// next item with relaxed loads ahead of time and checks them after the stage
// barriers, so the poll seldom stalls; an item whose neighbours are not done
// when it becomes current is waited for (bounded).  A tile's counter is
// published after the next item's first stage barrier (or at the next item's
// start when that item waits), so the waiting item never depends on an
// unpublished item of its own CTA unless the host's check
// G not in [ntiles - 4 tiles_x, ntiles + 4 tiles_x] fails (the folded order
// keeps every dependency within 4 tiles_x - 1 positions).
template <int MODE, bool POT, bool PER, bool ONE, int MR, int WY, int MINB, bool MS = false>
__global__ void __launch_bounds__(32 * WY, MINB)
rk4_f32_tma(const TileArgs ta) {
  constexpr bool RES = MODE == 1 || MODE == 3, DRV = MODE == 2 || MODE == 3;
  using C = Cfg<MODE, POT, MR, WY, MINB>;
  static_assert(!MS || (ONE && !DRV && C::NBUF == 2), "multi-step: single instance, no drive");
  // YY: two stage-exchange buffers, alternating between consecutive tiles.
  // Then no barrier opens a tile: the first stage barrier also carries the
  // bounded waits' failure vote, and a tile's input buffer is refilled (with
  // the tile NBUF positions later) right after its last stage barrier, the
  // last point that reads it; warps that finish a tile's stores go on to the
  // next tile while others still store.
  constexpr bool YY = !MS && C::YY_FITS;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[3];
  // drive phase exp(-i omega t_s) / hbar per stage: one set for a single
  // instance; for batches the sets of the current and the next tile
  __shared__ float2 s_dph[2][4];
  // 128-byte aligned start, by pointer arithmetic on the shared array so that
  // the compiler keeps every derived access in the shared state space
  unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  float2* const Ybase = reinterpret_cast<float2*>(base + C::NBUF * C::BUF_BYTES);
  constexpr int Y_STRIDE = C::PSI_BYTES / 8;  // float2 elements per exchange buffer

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c0 = 2 * lane;   // region column of the micro-tile's first column
  const int r0 = MR * warp;  // region row of its first row
  auto psi_buf = [&](int b) { return reinterpret_cast<float2*>(base + b * C::BUF_BYTES); };
  auto f_buf = [&](int b, int f) {
    return reinterpret_cast<float*>(base + b * C::BUF_BYTES + C::PSI_BYTES + f * C::F_BYTES);
  };

  // Y ring cells are never written by the stages: give them a defined value.
  for (int yb = 0; yb < (YY ? 2 : 1); ++yb)
    for (int i = tid; i < C::PH * C::PW; i += C::NT) {
      int r = i / C::PW, c = i - r * C::PW;
      if (r == 0 || r == C::PH - 1 || c < 2 || c >= C::RW + 2)
        Ybase[yb * Y_STRIDE + i] = f2(0.f, 0.f);
    }
  if (tid == 0) {
    for (int b = 0; b < C::NBUF; ++b) mbar_init(&bar[b], 1);
    fence_mbar_init();
  }
  __syncthreads();
  // Programmatic dependent launch: this grid may have started while the
  // previous step was still running; everything above touched only shared
  // memory.  Let the next step's grid be scheduled as SMs free up, then wait
  // until the previous grid has completed and its writes are visible.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");

  // Tile coordinates: a running (kx, ky) per stream of tiles for a single
  // instance (one division at the start), a table lookup for batches.
  struct Coord {
    int inst, kx, ky;
  };
  const int tiles_x1 = ONE ? ta.one.tiles_x : 1;
  const int dq = ONE ? (int)gridDim.x / tiles_x1 : 0;
  const int dr = ONE ? (int)gridDim.x - dq * tiles_x1 : 0;
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
  // next tile of this CTA (t + gridDim.x)
  auto advance = [&](Coord& c, int t_next) {
    if (ONE) {
      c.kx += dr;
      c.ky += dq;
      if (c.kx >= tiles_x1) {
        c.kx -= tiles_x1;
        c.ky += 1;
      }
    } else if (t_next < ta.ntiles) {
      c = coord_of(t_next);
    }
  };
  auto issue = [&](const Coord& c, int b, int cur) {
    const TileInst* I = ta.inst + c.inst;
    const int xp = c.kx * C::TX;  // padded column of region column 0
    const int yp = c.ky * C::TY;  // padded row of region row -1
    mbar_arrive_expect_tx(&bar[b], C::TX_BYTES);
    tma_load_3d(psi_buf(b), &I->psi[cur], 2 * (xp - 2), yp, 0, &bar[b]);
    int f = 0;
    if (RES) {
      tma_load_3d(f_buf(b, f++), &I->n[cur], xp & ~3, yp + 1, 0, &bar[b]);
      tma_load_3d(f_buf(b, f++), &I->P, xp & ~3, yp + 1, 0, &bar[b]);
    }
    if (DRV) {
      tma_load_3d(f_buf(b, f++), &I->Er, xp & ~3, yp + 1, 0, &bar[b]);
      tma_load_3d(f_buf(b, f++), &I->Ei, xp & ~3, yp + 1, 0, &bar[b]);
    }
    if (POT) tma_load_3d(f_buf(b, f++), &I->V, xp & ~3, yp + 1, 0, &bar[b]);
  };

  // Drive phases of the four stage times t, t + dt/2, t + dt/2, t + dt of an
  // instance (FP64 sincos on threads 0..3) into set `slot`.  A single
  // instance computes them once, published by the barrier that opens the
  // first tile; a batch computes those of the CTA's next tile while the
  // current one runs, published by the barrier that opens the next tile.
  auto drive_phases = [&](int inst, int slot) {
    const double t0 = ONE ? ta.clock->t[ta.parity] : ta.t_inst[ta.parity * ta.ninst + inst];
    const double dt64 = ta.inst[inst].dt64;
    const double ts = t0 + (tid == 0 ? 0.0 : (tid == 3 ? dt64 : 0.5 * dt64));
    const float ih = ONE ? ta.one.k.inv_hbar : ta.inst[inst].k.inv_hbar;
    if (ONE) {
      double sn, cs;
      sincos(ta.inst[inst].omega * ts, &sn, &cs);
      s_dph[slot][tid] = f2((float)cs * ih, (float)(-sn) * ih);
    } else {
      // once per tile on the critical path of warp 0: the angle is reduced
      // to [-pi, pi] in FP64 (few operations on the narrow FP64 pipe) and
      // its sine and cosine taken in FP32 (error ~1e-7, the stencil's own
      // precision)
      const double a = ta.inst[inst].omega * ts;
      const double r = fma(-rint(a * 0.15915494309189535), 6.283185307179586, a);
      float sn, cs;
      sincosf((float)r, &sn, &cs);
      s_dph[slot][tid] = f2(cs * ih, -sn * ih);
    }
  };
  if (DRV && tid < 4) {
    if (ONE) drive_phases(0, 0);
    else if ((int)blockIdx.x < ta.ntiles) drive_phases(coord_of(blockIdx.x).inst, 0);
  }

  // FP64 simulated time: instance 0 in the clock, all instances in t_inst
  const long long step = ta.clock->step[ta.parity];
  if (!MS && blockIdx.x == 0) {
    if (tid == 0) {
      ta.clock->step[ta.parity ^ 1] = step + 1;
      ta.clock->t[ta.parity ^ 1] = ta.clock->t[ta.parity] + ta.inst[0].dt64;
    }
    if (ta.t_inst)
      for (int i = tid; i < ta.ninst; i += C::NT)
        ta.t_inst[(ta.parity ^ 1) * ta.ninst + i] =
            ta.t_inst[ta.parity * ta.ninst + i] + ta.inst[i].dt64;
  }

  // multi-step items: step s of the launch and tile (kx, ky) of item i
  const int nitems = MS ? ta.ntiles * ta.ms_steps : ta.ntiles;
  const int G = (int)gridDim.x;
  auto ms_coord = [&](int i, Coord& c, int& s) {
    s = i / ta.ntiles;
    const int pos = i - s * ta.ntiles;
    const int rp = pos / tiles_x1;
    c.inst = 0;
    c.kx = pos - rp * tiles_x1;
    c.ky = (rp & 1) ? ta.tiles_y - 1 - (rp >> 1) : (rp >> 1);
  };
  // warp 0 of a multi-step launch: the item whose load waits for its
  // neighbours (or -1; in shared memory, which only warp 0 uses, to spare a
  // register), lanes 0..8 holding the counter of one neighbour each in fv.
  // Coordinates, step and buffer are recomputed from the item.  A counter is
  // published with atomicMax, so that publishing an item twice is harmless.
  __shared__ int s_pend;
  int fv = 0x7fffffff;
  auto set_pend = [&](int v) {
    __syncwarp();
    if (lane == 0) s_pend = v;
    __syncwarp();
  };
  // Along an axis a tile exchanges data with its two neighbours (periodic
  // wrap included) and, when the last tile holds fewer rows (columns) than
  // its box reaches past them, tiles 0 and n-2 exchange too: the box of tile
  // n-2 then reaches the ghost rows that tile 0 writes, and tile 0 writes
  // them from rows that tile n-2 computes.  Candidate c of 0..3 along an axis
  // of n tiles: k-1, k, k+1 (mod n), or that partner (-1: none).
  auto dep_axis = [&](int k, int c, int n, bool thin) {
    if (c < 3) {
      const int v = k + c - 1;
      return v < 0 ? v + n : (v >= n ? v - n : v);
    }
    if (!thin) return -1;
    return k == 0 ? n - 2 : (k == n - 2 ? 0 : -1);
  };
  // (tile kx's box ends at domain column (kx + 1) TX + 3, tile ky's at row
  // (ky + 1) TY + HALO)
  const bool thin_x = (tiles_x1 - 1) * C::TX + 3 > ta.one.geo.nx;
  const bool thin_y = (ta.tiles_y - 1) * C::TY + HALO > ta.one.geo.ny;
  auto ms_load_deps = [&]() {  // warp 0: lanes 0..15 load one candidate each
    fv = 0x7fffffff;
    if (lane < 16) {
      Coord c;
      int sp;
      ms_coord(s_pend, c, sp);
      const int dx = dep_axis(c.kx, lane & 3, tiles_x1, thin_x);
      const int dy = dep_axis(c.ky, lane >> 2, ta.tiles_y, thin_y);
      if (dx >= 0 && dy >= 0) fv = ld_relaxed_gpu(ta.done + dy * tiles_x1 + dx);
    }
  };
  auto ms_issue_pending = [&]() {  // warp 0, after fence.acq_rel.gpu
    __syncwarp();  // every lane's acquire before lane 0's loads
    if (lane == 0) {
      const int pend = s_pend;
      Coord c;
      int sp;
      ms_coord(pend, c, sp);
      fence_proxy_async_global();  // the acquired outputs before the TMA reads
      fence_proxy_async();         // this CTA's generic reads of the buffer before its refill
      issue(c, ((pend - (int)blockIdx.x) / G) % C::NBUF, ta.cur ^ (sp & 1));
    }
    set_pend(-1);
  };
  auto ms_publish = [&](int item) {  // warp 0, after fence.acq_rel.gpu
    if (lane == 0) {
      Coord c;
      int sp;
      ms_coord(item, c, sp);
      atomicMax(ta.done + c.ky * tiles_x1 + c.kx, sp + 1);
    }
  };
  // publish this CTA's previous item (its stores precede a CTA barrier),
  // then check the pending item's neighbours loaded earlier (warp 0)
  auto ms_point = [&](bool publish, int t_now) {
    const int pend = s_pend;
    publish = publish && t_now >= (int)blockIdx.x + G;
    if (!publish && pend < 0) return;
    fence_acq_rel_gpu();
    if (publish) ms_publish(t_now - G);
    if (pend >= 0) {
      if (__all_sync(0xffffffffu, fv >= pend / ta.ntiles)) ms_issue_pending();
      else ms_load_deps();
    }
  };

  int t = blockIdx.x, k = 0, s_cur = 0;
  Coord cc = coord_of(t < ta.ntiles ? t : 0);  // current tile
  Coord cn = cc;                               // next tile to issue (thread 0)
  if (MS) {
    if (warp == 0) {  // prologue: the first item, if it has no dependency
      set_pend(t < nitems ? t : -1);
      if (t < nitems && t < ta.ntiles) {
        if (ta.inject_timeout) set_pend(-1);
        else ms_issue_pending();
      }
    }
  } else if (tid == 0) {  // prologue: the first NBUF-1 tiles (NBUF with YY)
    for (int i = 0; i < C::NBUF - (YY ? 0 : 1); ++i) {
      const int ti = t + i * (int)gridDim.x;
      if (ti < ta.ntiles && !(i == 0 && ta.inject_timeout)) issue(cn, i, ta.cur);
      advance(cn, ti + (int)gridDim.x);
    }
  }
  for (; t < nitems; t += G, ++k) {
    const int b = k % C::NBUF;
    const uint32_t par = (uint32_t)((k / C::NBUF) & 1);
    const int tn = t + (C::NBUF - 1) * (int)gridDim.x;
    int dep_fail = 0;
    if (MS) {
      ms_coord(t, cc, s_cur);
      // the previous item's stores are done by every thread; does this item
      // still wait for its neighbours?
      if (__syncthreads_or(warp == 0 && s_pend == t) && warp == 0) {
        fence_acq_rel_gpu();
        if (k > 0) ms_publish(t - G);
        const int need = t / ta.ntiles;
        const unsigned long long t0 = global_ns();
        for (uint32_t it = 0;; ++it) {
          ms_load_deps();
          if (__all_sync(0xffffffffu, fv >= need)) break;
          if (it >= 4) __nanosleep(128);
          if ((it & 63u) == 63u && global_ns() - t0 > 250000000ull) {
            dep_fail = 1;
            break;
          }
        }
        fence_acq_rel_gpu();
        if (dep_fail) set_pend(-1);
        else ms_issue_pending();
      }
    }
    // every thread waits on the barrier (bounded); the CTA leaves together
    // if any thread gave up, after waiting (bounded) for its other loads:
    // those of the next NBUF-2 tiles (NBUF-1 with YY, whose vote is taken at
    // the first stage barrier).
    const int fail = dep_fail || !mbar_wait_bounded(&bar[b], par);
    auto leave = [&]() {
      if (tid == 0) {
        atomicExch(ta.err, 1);
        for (int j = k + 1; j < k + C::NBUF - (YY ? 0 : 1); ++j)
          if (t + (j - k) * (int)gridDim.x < ta.ntiles)
            mbar_wait_bounded(&bar[j % C::NBUF], (uint32_t)((j / C::NBUF) & 1));
      }
    };
    if (!YY) {
      // This barrier also closes the previous tile: every thread has
      // finished reading its buffers and the shared stage buffer Y.
      if (__syncthreads_or(fail)) {
        leave();
        return;
      }
      if (DRV && !ONE && tid < 4 && t + (int)gridDim.x < ta.ntiles)
        drive_phases(coord_of(t + (int)gridDim.x).inst, (k + 1) & 1);
    }
    // refill the buffer the previous tile used (YY: after this tile's last
    // stage barrier)
    if (YY) {
    } else if (MS) {
      if (warp == 0 && t + G < nitems) {
        set_pend(t + G);
        if (t + G < ta.ntiles) ms_issue_pending();  // step 0 reads the launch's input
        else ms_load_deps();
      }
    } else if (tid == 0 && tn < ta.ntiles) {
      fence_proxy_async();  // its generic reads before the async-proxy write
      issue(cn, (k + C::NBUF - 1) % C::NBUF, ta.cur);
      advance(cn, tn + (int)gridDim.x);
    }

    const int kx = cc.kx, ky = cc.ky;
    const TileInst* I = ta.inst + cc.inst;
    const Geometry g = ONE ? ta.one.geo : I->geo;
    const int cur = MS ? ta.cur ^ (s_cur & 1) : ta.cur;
    float2* const psi_out = ONE ? ta.one.psi_buf[cur ^ 1] : I->psi_buf[cur ^ 1];
    float* const n_out = ONE ? ta.one.n_buf[cur ^ 1] : I->n_buf[cur ^ 1];
    const CoeffsT<float> q = ONE ? ta.one.k : I->k;
    const NoiseKey nz = ONE ? ta.one.noise : I->noise;
    if (!MS) advance(cc, t + (int)gridDim.x);
    const float2 ax2 = f2(q.ax, q.ax), ay2 = f2(q.ay, q.ay);
    // real coefficients as pairs: the thread's two columns go through the
    // real-valued terms (density, local term, gain, reservoir) together
    const float2 cg2 = f2(q.g, q.g), cgr2 = f2(q.gr, q.gr), cih2 = f2(q.inv_hbar, q.inv_hbar);
    const float2 hR2 = f2(q.half_R, q.half_R), nhgc2 = f2(-q.half_gc, -q.half_gc);
    const float2 ncR2 = f2(-q.R_, -q.R_), ncgam2 = f2(-q.gamma_r, -q.gamma_r);
    const float2 a02 = f2(q.a0, q.a0);
    const float dt = q.dt;
    const float dt6 = q.dt6;  // dt / 6, divided once on the host
    const int xp = kx * C::TX;
    const int foff = xp & 3;
    float2* P0 = psi_buf(b);
    const float* Nb = RES ? f_buf(b, 0) : nullptr;
    const float* Pb = RES ? f_buf(b, 1) : nullptr;
    // planes in load order: n, P (reservoir), Re E, Im E (drive), V
    const float* Erb = DRV ? f_buf(b, RES ? 2 : 0) : nullptr;
    const float* Eib = DRV ? f_buf(b, RES ? 3 : 1) : nullptr;
    const float* Vb = POT ? f_buf(b, C::NF - 1) : nullptr;

    // Registers: psi0, current stage value, accumulator (+ reservoir).  Real
    // fields hold the micro-tile row's two columns as one pair (.x, .y).
    float2 p0[MR][2], yc[MR][2], acc[MR][2];
    float2 n0[MR], nc[MR], na[MR], Pv[MR], Vv[MR], Er[MR], Ei[MR];
    bool ins[MR][2];
    const int gx0 = xp - HALO + c0;        // domain column of my first column
    const int gy0 = ky * C::TY - 3 + r0;   // domain row of my first row
    // n0 and P of row j: held in registers, or (multi-step launch, whose
    // bookkeeping needs the registers) read again from the tile's shared
    // n and P boxes, which no stage overwrites
    auto N0 = [&](int j) {
      return (MS && RES) ? *reinterpret_cast<const float2*>(&Nb[(r0 + j) * C::FW + foff + c0])
                         : n0[j];
    };
    auto PV = [&](int j) {
      return (MS && RES) ? *reinterpret_cast<const float2*>(&Pb[(r0 + j) * C::FW + foff + c0])
                         : Pv[j];
    };
#pragma unroll
    for (int j = 0; j < MR; ++j) {
      const float4 v = *reinterpret_cast<const float4*>(&P0[(r0 + j + 1) * C::PW + c0 + 2]);
      p0[j][0] = f2(v.x, v.y);
      p0[j][1] = f2(v.z, v.w);
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        yc[j][i] = p0[j][i];
        acc[j][i] = f2(0.f, 0.f);
        const int gx = gx0 + i, gy = gy0 + j;
        ins[j][i] = PER || ((g.bc_x == BC_PERIODIC || (gx >= 0 && gx < g.nx)) &&
                            (g.bc_y == BC_PERIODIC || (gy >= 0 && gy < g.ny)));
      }
      // foff + c0 is even: the pair of a row is one 8-byte load
      const int fi = (r0 + j) * C::FW + foff + c0;
      auto ld2 = [&](const float* b) { return *reinterpret_cast<const float2*>(&b[fi]); };
      n0[j] = (RES && !MS) ? ld2(Nb) : f2(0.f, 0.f);
      nc[j] = RES ? ld2(Nb) : f2(0.f, 0.f);
      na[j] = f2(0.f, 0.f);
      Pv[j] = (RES && !MS) ? ld2(Pb) : f2(0.f, 0.f);
      Er[j] = DRV ? ld2(Erb) : f2(0.f, 0.f);
      Ei[j] = DRV ? ld2(Eib) : f2(0.f, 0.f);
      // the stencil's diagonal a0 rides with the local potential
      Vv[j] = POT ? __ffma2_rn(ld2(Vb), cih2, a02) : a02;
    }

#pragma unroll
    for (int s = 0; s < 4; ++s) {
      float2* const Y = Ybase + (YY ? (k & 1) * Y_STRIDE : 0);
      const float2* src = (s & 1) ? Y : P0;
      float2* dst = (s & 1) ? P0 : Y;
      const float w = (s == 0 || s == 3) ? 1.f : 2.f;
      const float cs = (s == 2) ? dt : 0.5f * dt;
      const float2 w2 = f2(w, w), cs2 = f2(cs, cs);
      const float2 dph = DRV ? s_dph[ONE ? 0 : (k & 1)][s] : f2(0.f, 0.f);
      // neighbours of the micro-tile
      const float4 tv = *reinterpret_cast<const float4*>(&src[(r0)*C::PW + c0 + 2]);
      const float4 bv = *reinterpret_cast<const float4*>(&src[(r0 + MR + 1) * C::PW + c0 + 2]);
      // West / east neighbours: from the loaded box in the first stage (the
      // ring columns -1 and 64 must be right there), from the neighbouring
      // lanes' registers afterwards (lanes 0 and 31 then see their own
      // values: finite, and only in the ring region that no output needs).
      float2 Wv[MR], Ev[MR];
#pragma unroll
      for (int j = 0; j < MR; ++j) {
        if (s == 0) {
          Wv[j] = src[(r0 + j + 1) * C::PW + c0 + 1];
          Ev[j] = src[(r0 + j + 1) * C::PW + c0 + 4];
        } else {
          Wv[j].x = __shfl_up_sync(0xffffffffu, yc[j][1].x, 1);
          Wv[j].y = __shfl_up_sync(0xffffffffu, yc[j][1].y, 1);
          Ev[j].x = __shfl_down_sync(0xffffffffu, yc[j][0].x, 1);
          Ev[j].y = __shfl_down_sync(0xffffffffu, yc[j][0].y, 1);
        }
      }
      float2 ny[MR][2];
      float2 nn[MR];
#pragma unroll
      for (int j = 0; j < MR; ++j) {
        float2 lap[2];
        float2 dens;  // |psi|^2 of the row's two sites
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const float2 Cc = yc[j][i];
          const float2 W = i ? yc[j][0] : Wv[j];
          const float2 E = i ? Ev[j] : yc[j][1];
          const float2 S = j ? yc[j - 1][i] : (i ? f2(tv.z, tv.w) : f2(tv.x, tv.y));
          const float2 N = (j < MR - 1) ? yc[j + 1][i] : (i ? f2(bv.z, bv.w) : f2(bv.x, bv.y));
          // H/hbar: off-diagonal stencil ax (E+W) + ay (N+S), plus the local
          // term (a0 + V/hbar + g|psi|^2 + g_r n) psi
          lap[i] = __fmul2_rn(ay2, __fadd2_rn(N, S));
          lap[i] = __ffma2_rn(ax2, __fadd2_rn(E, W), lap[i]);
          const float d = fmaf(Cc.x, Cc.x, Cc.y * Cc.y);
          if (i) dens.y = d; else dens.x = d;
        }
        float2 loc = __ffma2_rn(cg2, dens, Vv[j]);
        if (RES) loc = __ffma2_rn(cgr2, nc[j], loc);
        const float2 G = RES ? __ffma2_rn(hR2, nc[j], nhgc2) : nhgc2;  // (R n - gamma_c)/2
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const float2 Cc = yc[j][i];
          const float li = i ? loc.y : loc.x, Gi = i ? G.y : G.x;
          float2 H = __ffma2_rn(f2(li, li), Cc, lap[i]);
          if (DRV) {  // + E exp(-i omega t_s) / hbar
            const float er = i ? Er[j].y : Er[j].x, ei = i ? Ei[j].y : Ei[j].x;
            H = __ffma2_rn(f2(er, er), dph, H);
            H = __ffma2_rn(f2(-ei, ei), f2(dph.y, dph.x), H);
          }
          float2 K;
          K.x = fmaf(Gi, Cc.x, H.y);
          K.y = fmaf(Gi, Cc.y, -H.x);
          acc[j][i] = s == 0 ? K : __ffma2_rn(w2, K, acc[j][i]);
          ny[j][i] = __ffma2_rn(cs2, K, p0[j][i]);
          if (!PER && !ins[j][i]) ny[j][i] = f2(0.f, 0.f);
        }
        if (RES) {  // Kn = P - (gamma_r + R|psi|^2) n for both sites
          const float2 Kn = __ffma2_rn(__ffma2_rn(ncR2, dens, ncgam2), nc[j], PV(j));
          na[j] = s == 0 ? Kn : __ffma2_rn(w2, Kn, na[j]);
          nn[j] = __ffma2_rn(cs2, Kn, N0(j));
        } else {
          nn[j] = f2(0.f, 0.f);
        }
      }
      if (s < 3) {
#pragma unroll
        for (int j = 0; j < MR; ++j) {
          yc[j][0] = ny[j][0];
          yc[j][1] = ny[j][1];
          nc[j] = nn[j];
          // only the micro-tile's first and last rows are read by other warps
          if (j == 0 || j == MR - 1)
            *reinterpret_cast<float4*>(&dst[(r0 + j + 1) * C::PW + c0 + 2]) =
                make_float4(ny[j][0].x, ny[j][0].y, ny[j][1].x, ny[j][1].y);
        }
        // the last stage reads but writes no shared memory
        if (YY && s == 0) {
          // every thread is past the previous tile (whose last stage read
          // the other exchange buffer); the failure vote of this tile's wait
          if (__syncthreads_or(fail)) {
            leave();
            return;
          }
          // the next tile's drive phases (read after this tile's next barrier)
          if (DRV && !ONE && tid < 4 && t + (int)gridDim.x < ta.ntiles)
            drive_phases(coord_of(t + (int)gridDim.x).inst, (k + 1) & 1);
        } else {
          __syncthreads();
        }
        if (YY && s == 2 && tid == 0) {
          // stage 3 reads only Y and registers: this tile's input buffer is
          // free for the tile NBUF positions later
          const int tY = t + C::NBUF * (int)gridDim.x;
          if (tY < ta.ntiles) {
            fence_proxy_async();  // its generic accesses before the async-proxy write
            issue(cn, b, ta.cur);
            advance(cn, tY + (int)gridDim.x);
          }
        }
        if (MS && warp == 0) ms_point(s == 0, t);
      }
    }

    // psi' = psi0 + (K1 + 2K2 + 2K3 + K4) dt/6, written to the output tile
    const float2 d62 = f2(dt6, dt6);
    float2 o[MR][2];
    float2 on[MR];
#pragma unroll
    for (int j = 0; j < MR; ++j) {
#pragma unroll
      for (int i = 0; i < 2; ++i) o[j][i] = __ffma2_rn(d62, acc[j][i], p0[j][i]);
      on[j] = __ffma2_rn(d62, na[j], N0(j));
    }
    if (nz.on) {  // grid-uniform branch: the generator is not issued when off
      // The micro-tile's columns gx0 (even) and gx0 + 1 hold the sites 2p and
      // 2p + 1 of one Philox pair when the row length is even: one call for
      // both; otherwise one call per site.
      const bool paired = (g.nx & 1) == 0;
#pragma unroll
      for (int j = 0; j < MR; ++j) {
        const int gy = gy0 + j;
        const uint32_t row = (uint32_t)(((gy % g.ny + g.ny) % g.ny) * g.nx);
        uint32_t site[2];
        float sc[2];
        float2 xi[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const int gx = gx0 + i;
          site[i] = row + (uint32_t)((gx % g.nx + g.nx) % g.nx);
          sc[i] = nz.twa ? nz_wigner_scale(nz.R, nz.gc, nz.kw, nz.var,
                                           RES ? (i ? N0(j).y : N0(j).x) : 0.f)
                         : nz.scale;
        }
        if (paired) {
          nz_pair(nz.seed, nz.instance, MS ? step + s_cur : step, site[0] >> 1, sc[0], sc[1], xi[0], xi[1]);
        } else {
          float2 unused;
          nz_site(nz.seed, nz.instance, MS ? step + s_cur : step, site[0], sc[0], xi[0], unused, false);
          nz_site(nz.seed, nz.instance, MS ? step + s_cur : step, site[1], sc[1], xi[1], unused, false);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          o[j][i].x = o[j][i].x + xi[i].x;
          o[j][i].y = o[j][i].y + xi[i].y;
        }
      }
    }
    // Interior tiles (no ghost image, no clipping) store whole rows of the
    // micro-tile with one 16-byte psi and one 8-byte n store.
    const int ox0 = xp - 1, oy0 = ky * C::TY;  // domain origin of the output tile
    const bool interior = ox0 >= HALO && ox0 + C::TX <= g.nx - HALO && oy0 >= HALO &&
                          oy0 + C::TY <= g.ny - HALO;
    if (interior) {
      // my two columns inside the output columns [3, 3 + TX) of the region:
      // both (lanes 2..29), one (lanes 1 and 30: column `one`), or none
      const bool lo = c0 >= 3 && c0 < 3 + C::TX;
      const bool hi = c0 + 1 >= 3 && c0 + 1 < 3 + C::TX;
      const int one = lo ? 0 : 1;
#pragma unroll
      for (int j = 0; j < MR; ++j) {
        const int r = r0 + j;
        if (r < 3 || r >= 3 + C::TY) continue;  // warp-uniform
        const long long roff = (long long)(gy0 + j + HALO) * g.pitch + gx0 + HALO;
        if (lo && hi) {
          *reinterpret_cast<float4*>(psi_out + roff) =
              make_float4(o[j][0].x, o[j][0].y, o[j][1].x, o[j][1].y);
          if (RES) *reinterpret_cast<float2*>(n_out + roff) = on[j];
        } else if (lo || hi) {  // one path for both edge lanes
          psi_out[roff + one] = lo ? o[j][0] : o[j][1];
          if (RES) n_out[roff + one] = lo ? on[j].x : on[j].y;
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < MR; ++j) {
        const int r = r0 + j;
        const int gy = gy0 + j;
        if (r < 3 || r >= 3 + C::TY || gy >= g.ny) continue;
        bool ok[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const int c = c0 + i, gx = gx0 + i;
          ok[i] = c >= 3 && c < 3 + C::TX && gx >= 0 && gx < g.nx;
        }
        const bool edge_x = g.bc_x == BC_PERIODIC && (gx0 < HALO || gx0 + 1 >= g.nx - HALO);
        const bool edge_y = g.bc_y == BC_PERIODIC && (gy < HALO || gy >= g.ny - HALO);
        const long long roff = (long long)(gy + HALO) * g.pitch + gx0 + HALO;
        if (ok[0] && ok[1] && !edge_x && !edge_y) {
          *reinterpret_cast<float4*>(psi_out + roff) =
              make_float4(o[j][0].x, o[j][0].y, o[j][1].x, o[j][1].y);
          if (RES) *reinterpret_cast<float2*>(n_out + roff) = on[j];
        } else {
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            if (!ok[i]) continue;
            store_with_ghosts(psi_out, g, gx0 + i, gy, o[j][i]);
            if (RES) store_with_ghosts(n_out, g, gx0 + i, gy, i ? on[j].y : on[j].x);
          }
        }
      }
    }
  }
  if (MS) {  // the last item
    __syncthreads();
    if (warp == 0 && k > 0) {
      fence_acq_rel_gpu();
      ms_publish(t - G);
    }
  }
}

template <int MODE, bool POT, bool PER, bool ONE, int MR, int WY, int MINB>
cudaError_t launch_cfg(const TileArgs& ta, cudaStream_t s, int grid) {
  using C = Cfg<MODE, POT, MR, WY, MINB>;
  auto kern = rk4_f32_tma<MODE, POT, PER, ONE, MR, WY, MINB>;
  constexpr int SMEM = C::YY_FITS ? C::SMEM_YY : C::SMEM;
  static int configured_dev = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_dev != dev) {
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    if (e != cudaSuccess) return e;
    configured_dev = dev;
  }
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(grid);
  lc.blockDim = dim3(C::NT);
  lc.dynamicSmemBytes = SMEM;
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

// Multi-step launch: cooperative, so that every CTA is resident (CTAs wait
// for items of other CTAs).
template <int MODE, bool POT, bool PER, int MR, int WY, int MINB>
cudaError_t launch_cfg_ms(const TileArgs& ta, cudaStream_t s, int grid) {
  using C = Cfg<MODE, POT, MR, WY, MINB>;
  auto kern = rk4_f32_tma<MODE, POT, PER, true, MR, WY, MINB, true>;
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
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&lc, kern, ta);
  count_launch();
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// The multi-step variants of one tile configuration (mode 0 or 1).
template <int MR, int WY, int MINB>
cudaError_t launch_variants_ms(int mode, bool pot, bool per, const TileArgs& ta,
                               cudaStream_t s, int grid) {
#define PHX_TMA_MS(M_)                                                             \
  if (per) {                                                                       \
    if (pot) return launch_cfg_ms<M_, true, true, MR, WY, MINB>(ta, s, grid);      \
    return launch_cfg_ms<M_, false, true, MR, WY, MINB>(ta, s, grid);              \
  }                                                                                \
  if (pot) return launch_cfg_ms<M_, true, false, MR, WY, MINB>(ta, s, grid);       \
  return launch_cfg_ms<M_, false, false, MR, WY, MINB>(ta, s, grid);
  if (mode == 1) {
    PHX_TMA_MS(1)
  }
  if (mode == 0) {
    PHX_TMA_MS(0)
  }
#undef PHX_TMA_MS
  return cudaErrorInvalidValue;
}

// Whether a configuration has the reservoir-and-drive variant (mode 3): one
// CTA per SM (its registers) and two input buffers within shared memory.
template <int MR, int WY, int MINB>
constexpr bool has_mode3() {
  return MINB == 1 && Cfg<3, true, MR, WY, MINB>::SMEM <= 227 * 1024;
}

// All model variants of one tile configuration (mode as in Cfg).
template <int MR, int WY, int MINB>
cudaError_t launch_variants(int mode, bool pot, bool per, bool one, const TileArgs& ta,
                            cudaStream_t s, int grid) {
#define PHX_TMA_V(M_, ONE_)                                                             \
  if (per) {                                                                            \
    if (pot) return launch_cfg<M_, true, true, ONE_, MR, WY, MINB>(ta, s, grid);        \
    return launch_cfg<M_, false, true, ONE_, MR, WY, MINB>(ta, s, grid);                \
  }                                                                                     \
  if (pot) return launch_cfg<M_, true, false, ONE_, MR, WY, MINB>(ta, s, grid);         \
  return launch_cfg<M_, false, false, ONE_, MR, WY, MINB>(ta, s, grid);
  if (one) {
    if (mode == 3) {
      if constexpr (has_mode3<MR, WY, MINB>()) {
        PHX_TMA_V(3, true)
      } else {
        return cudaErrorInvalidValue;
      }
    }
    if (mode == 2) {
      PHX_TMA_V(2, true)
    }
    if (mode == 1) {
      PHX_TMA_V(1, true)
    }
    PHX_TMA_V(0, true)
  }
  if (mode == 3) {
    if constexpr (has_mode3<MR, WY, MINB>()) {
      PHX_TMA_V(3, false)
    } else {
      return cudaErrorInvalidValue;
    }
  }
  if (mode == 2) {
    PHX_TMA_V(2, false)
  }
  if (mode == 1) {
    PHX_TMA_V(1, false)
  }
  PHX_TMA_V(0, false)
#undef PHX_TMA_V
}

}  // namespace tma
}  // namespace phx
