// Batches of independent FP32 scalar instances advanced by one persistent
// kernel launch per RK4 step (the tiles of all members in one work list),
// replayed from a CUDA graph, with a measured choice of tile configuration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/phx.h"
#include "phx_internal.h"
#include "rk4_tma.h"

namespace phx {
unsigned long long launch_total();
}

using namespace phx;

struct phx_batch {
  int count = 0;
  std::vector<phx_params> p;
  std::vector<Geometry> geo;
  std::vector<void*> psi[2], n[2], P, V;
  std::vector<char> has_V;
  std::vector<void*> E;          // per member: Re and Im planes of the drive
  void* E_pool = nullptr;        // every member's drive planes, once any is set
  bool has_E = false;            // the drive variant runs (undriven members: zeros)
  bool reservoir = false;
  bool tile_fixed = false;       // params[0].tile named the configuration
  void* pool = nullptr;          // one allocation for every member's fields
  std::vector<void*> V_owned;    // potentials are allocated on demand
  TileInst* d_inst = nullptr;
  std::vector<TileInst> h_inst;
  int2* d_tile_info = nullptr;   // per tile: (member, kx | ky << 16)
  int ntiles = 0;
  DevClock* clock = nullptr;
  double* t_inst = nullptr;      // [2][count]
  double* partials = nullptr;
  double* red_dev = nullptr;     // [count][8]
  double* red_host = nullptr;    // pinned [count][8]
  int* err_dev = nullptr;
  int cur = 0, parity = 0;
  long long host_step = 0;
  int tile_cfg = 0;
  bool tables_ok = false;
  bool tables_V = false;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  cudaStream_t stream = nullptr;
  int device = 0, num_sms = 0;
  std::string err;
};

namespace {

thread_local std::string g_batch_err = "no error";

phx_status bfail(phx_batch* b, phx_status s, const std::string& m) {
  if (b)
    b->err = m;
  else
    g_batch_err = m;
  return s;
}

phx_status bcuda(phx_batch* b, cudaError_t e, const char* what) {
  return bfail(b, e == cudaErrorMemoryAllocation ? PHX_ENOMEM : PHX_ECUDA,
               std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

#define PHX_BCK(b, expr)                                    \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) return bcuda((b), _e, #expr);    \
  } while (0)

void bfree(phx_batch* b) {
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (void* v : b->V_owned)
    if (v) cudaFree(v);
  if (b->pool) cudaFree(b->pool);
  if (b->E_pool) cudaFree(b->E_pool);
  if (b->d_inst) cudaFree(b->d_inst);
  if (b->d_tile_info) cudaFree(b->d_tile_info);
  if (b->clock) cudaFree(b->clock);
  if (b->t_inst) cudaFree(b->t_inst);
  if (b->partials) cudaFree(b->partials);
  if (b->red_dev) cudaFree(b->red_dev);
  if (b->red_host) cudaFreeHost(b->red_host);
  if (b->err_dev) cudaFree(b->err_dev);
}

bool any_V(const phx_batch* b) {
  return std::any_of(b->has_V.begin(), b->has_V.end(), [](char c) { return c != 0; });
}
bool all_V(const phx_batch* b) {
  return std::all_of(b->has_V.begin(), b->has_V.end(), [](char c) { return c != 0; });
}

// Instance descriptors and the global tile list for configuration cfg.
phx_status build_tables(phx_batch* b, int cfg) {
  std::vector<int2> tile_info;
  int tile0 = 0;
  for (int i = 0; i < b->count; ++i) {
    void* psi[2] = {b->psi[0][i], b->psi[1][i]};
    void* n[2] = {b->n[0][i], b->n[1][i]};
    if (!fill_tile_inst(b->h_inst[i], b->p[i], b->geo[i], psi, n, b->P[i],
                        b->has_V[i] ? b->V[i] : nullptr, cfg, b->has_E ? b->E[i] : nullptr))
      return bfail(b, PHX_ECUDA, "cuTensorMapEncodeTiled failed");
    b->h_inst[i].tile0 = tile0;
    const int tx = b->h_inst[i].tiles_x, ty = b->h_inst[i].tiles_y;
    if (tx > 0xffff || ty > 0x7fff) return bfail(b, PHX_EINVAL, "member grid too large");
    for (int ky = 0; ky < ty; ++ky)
      for (int kx = 0; kx < tx; ++kx) tile_info.push_back(make_int2(i, kx | (ky << 16)));
    tile0 += tx * ty;
  }
  if (b->d_tile_info && b->ntiles < tile0) {
    cudaFree(b->d_tile_info);
    b->d_tile_info = nullptr;
  }
  if (!b->d_tile_info) PHX_BCK(b, cudaMalloc(&b->d_tile_info, sizeof(int2) * tile0));
  b->ntiles = tile0;
  // synchronous copies: the host vectors are temporaries
  PHX_BCK(b, cudaStreamSynchronize(b->stream));
  PHX_BCK(b, cudaMemcpy(b->d_tile_info, tile_info.data(), sizeof(int2) * tile0,
                        cudaMemcpyHostToDevice));
  PHX_BCK(b, cudaMemcpy(b->d_inst, b->h_inst.data(), sizeof(TileInst) * b->count,
                        cudaMemcpyHostToDevice));
  b->tile_cfg = cfg;
  b->tables_ok = true;
  b->tables_V = any_V(b);
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return PHX_OK;
}

TileArgs batch_args(const phx_batch* b, int cur, int parity) {
  TileArgs ta;
  ta.inst = b->d_inst;
  ta.tile_info = b->d_tile_info;
  ta.one = scalars_of(b->h_inst[0]);
  ta.ntiles = b->ntiles;
  ta.ninst = b->count;
  ta.cur = cur;
  ta.clock = b->clock;
  ta.parity = parity;
  ta.t_inst = b->t_inst;
  ta.err = b->err_dev;
  ta.inject_timeout = 0;
  return ta;
}

cudaError_t launch_step(const phx_batch* b, int cur, int parity, cudaStream_t s) {
  const int slots = b->num_sms * tma_ctas_per_sm(b->tile_cfg);
  const int grid = b->ntiles < slots ? b->ntiles : slots;
  bool per = true;
  for (const phx_params& q : b->p)
    per = per && q.bc_x == PHX_BC_PERIODIC && q.bc_y == PHX_BC_PERIODIC;
  const int mode = b->reservoir ? (b->has_E ? 3 : 1) : (b->has_E ? 2 : 0);
  return launch_rk4_tma_f32(b->tile_cfg, mode, b->tables_V, per, batch_args(b, cur, parity), s,
                            grid);
}

// Time each tile configuration on the batch's own state (a step reads buffer
// cur and writes cur ^ 1, so repeating it leaves the state intact).
phx_status autotune(phx_batch* b) {
  const int all_cands[] = {TILE_64x48_M2, TILE_64x64_M2, TILE_64x48, TILE_64x64, TILE_64x32,
                           TILE_64x32_M2_2, TILE_64x32_M4_2};
  // reservoir and drive: the configurations with that variant
  const int drive_res_cands[] = {TILE_64x48, TILE_64x32, TILE_64x48_M2};
  const bool drive_res = b->reservoir && b->has_E;
  const int* cands = drive_res ? drive_res_cands : all_cands;
  cudaEvent_t e0, e1;
  PHX_BCK(b, cudaEventCreate(&e0));
  PHX_BCK(b, cudaEventCreate(&e1));
  // five interleaved rounds of ten launches; each configuration keeps its
  // fastest round
  const int nc = drive_res ? 3 : 7;
  float cfg_ms[7];
  for (int c = 0; c < nc; ++c) cfg_ms[c] = 1e30f;
  for (int round = 0; round < 5; ++round) {
    for (int c = 0; c < nc; ++c) {
      if (build_tables(b, cands[c]) != PHX_OK) continue;
      cudaError_t e = launch_step(b, b->cur, b->parity, b->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
      for (int i = 0; i < 10 && e == cudaSuccess; ++i)
        e = launch_step(b, b->cur, b->parity, b->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      if (ms < cfg_ms[c]) cfg_ms[c] = ms;
    }
  }
  float best_ms = 1e30f;
  int best = cands[0];
  for (int c = 0; c < nc; ++c)
    if (cfg_ms[c] < best_ms) {
      best_ms = cfg_ms[c];
      best = cands[c];
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return build_tables(b, best);
}

// CUDA graph of `steps` (even) launches starting from buffer/parity 0,
// captured on a private stream (the legacy default stream cannot be
// captured) and later launched on the batch's stream.
phx_status build_graph(phx_batch* b, int steps) {
  cudaGraph_t g = nullptr;
  cudaStream_t cs = nullptr;
  PHX_BCK(b, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaError_t e0 = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e0 != cudaSuccess) {
    cudaStreamDestroy(cs);
    return bcuda(b, e0, "cudaStreamBeginCapture");
  }
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < steps && e == cudaSuccess; ++s) e = launch_step(b, s & 1, s & 1, cs);
  cudaError_t e2 = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) return bcuda(b, e, "graph capture launch");
  if (e2 != cudaSuccess) return bcuda(b, e2, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return bcuda(b, e, "cudaGraphInstantiate");
  b->graph_steps = steps;
  return PHX_OK;
}

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DevGuard() {
    int now = -1;
    cudaGetDevice(&now);
    if (prev >= 0 && now != prev) cudaSetDevice(prev);
  }
};

phx_status check_member(phx_batch* b, int32_t i) {
  if (!b) return bfail(nullptr, PHX_EINVAL, "batch is NULL");
  if (i < 0 || i >= b->count) return bfail(b, PHX_EINVAL, "member index out of range");
  return PHX_OK;
}

}  // namespace

extern "C" {

phx_status phx_batch_create(const phx_params* params, int32_t count, phx_batch** out) {
  if (!out) return bfail(nullptr, PHX_EINVAL, "out is NULL");
  *out = nullptr;
  if (!params || count < 1) return bfail(nullptr, PHX_EINVAL, "need count >= 1 params");
  for (int i = 0; i < count; ++i) {
    double dtmax = 0;
    const char* m = check_params(&params[i], &dtmax);
    if (m) return bfail(nullptr, PHX_EINVAL, "member " + std::to_string(i) + ": " + m);
    const phx_params& p = params[i];
    if (p.precision != 32 || p.spinor)
      return bfail(nullptr, PHX_EINVAL, "batches hold FP32 scalar members");
    if (p.reservoir != params[0].reservoir)
      return bfail(nullptr, PHX_EINVAL, "all members need the same reservoir flag");
    if (p.nx < 2 * HALO || p.ny < 2 * HALO)
      return bfail(nullptr, PHX_EINVAL, "batch members need nx, ny >= 8");
    if (!(p.dt > 0.0) || p.dt > dtmax * (1.0 + 1e-12))
      return bfail(nullptr, PHX_EINVAL,
                   "member " + std::to_string(i) + ": dt must be in (0, stability limit]");
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return bfail(nullptr, PHX_ENODEV, cudaGetErrorString(e));
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess || prop.major != 10 || prop.minor != 3)
    return bfail(nullptr, PHX_ENODEV, "kernels are built for sm_103a (GB300)");
  phx_batch* b = new (std::nothrow) phx_batch();
  if (!b) return bfail(nullptr, PHX_ENOMEM, "host allocation failed");
  b->count = count;
  b->device = dev;
  b->num_sms = prop.multiProcessorCount;
  b->stream = static_cast<cudaStream_t>(params[0].stream);
  b->reservoir = params[0].reservoir != 0;
  b->p.assign(params, params + count);
  // params[0].tile fixes the step-kernel configuration (a TMA-fed one);
  // 0 (or any other value) leaves it to the autotuner
  if (params[0].tile >= TILE_64x64 && params[0].tile <= TILE_64x32_M4_2) {
    b->tile_cfg = params[0].tile;
    b->tile_fixed = true;
  }
  b->h_inst.resize(count);
  b->has_V.assign(count, 0);
  b->E.assign(count, nullptr);
  b->V.assign(count, nullptr);
  b->V_owned.assign(count, nullptr);
  size_t total = 0;
  std::vector<size_t> off_psi(count), off_n(count), off_P(count);
  auto take = [&](size_t bytes) {
    size_t o = total;
    total += (bytes + 255) & ~size_t(255);
    return o;
  };
  for (int i = 0; i < count; ++i) {
    Geometry g = padded_geometry(params[i]);
    b->geo.push_back(g);
    off_psi[i] = take(2 * (size_t)g.plane * 8);
    if (b->reservoir) {
      off_n[i] = take(2 * (size_t)g.plane * 4);
      off_P[i] = take((size_t)g.plane * 4);
    }
  }
  auto failc = [&](cudaError_t ce, const char* what) {
    cudaGetLastError();
    std::string m = std::string(what) + ": " + cudaGetErrorString(ce);
    bfree(b);
    delete b;
    return bfail(nullptr, ce == cudaErrorMemoryAllocation ? PHX_ENOMEM : PHX_ECUDA, m);
  };
  if ((e = cudaMalloc(&b->pool, total)) != cudaSuccess) return failc(e, "cudaMalloc pool");
  if ((e = cudaMemsetAsync(b->pool, 0, total, b->stream)) != cudaSuccess) return failc(e, "memset");
  char* base = static_cast<char*>(b->pool);
  for (int k = 0; k < 2; ++k) {
    b->psi[k].resize(count);
    b->n[k].resize(count);
  }
  b->P.resize(count);
  for (int i = 0; i < count; ++i) {
    const Geometry& g = b->geo[i];
    b->psi[0][i] = base + off_psi[i];
    b->psi[1][i] = base + off_psi[i] + (size_t)g.plane * 8;
    b->n[0][i] = b->reservoir ? base + off_n[i] : nullptr;
    b->n[1][i] = b->reservoir ? base + off_n[i] + (size_t)g.plane * 4 : nullptr;
    b->P[i] = b->reservoir ? base + off_P[i] : nullptr;
  }
  if ((e = cudaMalloc(&b->d_inst, sizeof(TileInst) * count)) != cudaSuccess)
    return failc(e, "cudaMalloc descriptors");
  if ((e = cudaMalloc(&b->clock, sizeof(DevClock))) != cudaSuccess) return failc(e, "cudaMalloc clock");
  if ((e = cudaMemsetAsync(b->clock, 0, sizeof(DevClock), b->stream)) != cudaSuccess)
    return failc(e, "memset");
  if ((e = cudaMalloc(&b->t_inst, sizeof(double) * 2 * count)) != cudaSuccess)
    return failc(e, "cudaMalloc times");
  if ((e = cudaMemsetAsync(b->t_inst, 0, sizeof(double) * 2 * count, b->stream)) != cudaSuccess)
    return failc(e, "memset");
  const size_t plen = sizeof(double) * reduce_partials_len(b->geo[0]);
  if ((e = cudaMalloc(&b->partials, plen)) != cudaSuccess)
    return failc(e, "cudaMalloc partials");
  if ((e = cudaMemsetAsync(b->partials, 0, plen, b->stream)) != cudaSuccess)
    return failc(e, "memset");
  if ((e = cudaMalloc(&b->red_dev, sizeof(double) * 8 * count)) != cudaSuccess)
    return failc(e, "cudaMalloc results");
  if ((e = cudaMallocHost(&b->red_host, sizeof(double) * 8 * count)) != cudaSuccess)
    return failc(e, "cudaMallocHost results");
  if ((e = cudaMalloc(&b->err_dev, sizeof(int))) != cudaSuccess) return failc(e, "cudaMalloc err");
  if ((e = cudaMemsetAsync(b->err_dev, 0, sizeof(int), b->stream)) != cudaSuccess)
    return failc(e, "memset");
  if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess) return failc(e, "sync");
  *out = b;
  return PHX_OK;
}

phx_status phx_batch_set_pump(phx_batch* b, int32_t i, const void* P, int on_device) {
  phx_status st = check_member(b, i);
  if (st != PHX_OK) return st;
  if (!b->reservoir) return bfail(b, PHX_ESTATE, "set_pump needs reservoir = 1");
  if (!P) return bfail(b, PHX_EINVAL, "P is NULL");
  DevGuard dg(b->device);
  PHX_BCK(b, upload_field(b->P[i], P, 1, 4, b->geo[i], on_device, b->stream));
  return PHX_OK;
}

phx_status phx_batch_set_potential(phx_batch* b, int32_t i, const void* V, int on_device) {
  phx_status st = check_member(b, i);
  if (st != PHX_OK) return st;
  DevGuard dg(b->device);
  if (!V) {
    b->has_V[i] = 0;
  } else {
    if (!b->V_owned[i]) {
      const size_t bytes = (size_t)b->geo[i].plane * 4;
      PHX_BCK(b, cudaMalloc(&b->V_owned[i], bytes));
      PHX_BCK(b, cudaMemsetAsync(b->V_owned[i], 0, bytes, b->stream));
      b->V[i] = b->V_owned[i];
    }
    PHX_BCK(b, upload_field(b->V[i], V, 1, 4, b->geo[i], on_device, b->stream));
    b->has_V[i] = 1;
  }
  b->tables_ok = false;
  return PHX_OK;
}

phx_status phx_batch_set_drive(phx_batch* b, int32_t i, const void* E, int on_device) {
  phx_status st = check_member(b, i);
  if (st != PHX_OK) return st;
  DevGuard dg(b->device);
  if (!E) {  // a member without drive keeps zero planes
    if (b->has_E)
      PHX_BCK(b, cudaMemsetAsync(b->E[i], 0, 2 * (size_t)b->geo[i].plane * 4, b->stream));
    return PHX_OK;
  }
  if (!b->E_pool) {
    size_t total = 0;
    std::vector<size_t> off(b->count);
    for (int j = 0; j < b->count; ++j) {
      off[j] = total;
      total += (2 * (size_t)b->geo[j].plane * 4 + 255) & ~size_t(255);
    }
    PHX_BCK(b, cudaMalloc(&b->E_pool, total));
    PHX_BCK(b, cudaMemsetAsync(b->E_pool, 0, total, b->stream));
    for (int j = 0; j < b->count; ++j) b->E[j] = static_cast<char*>(b->E_pool) + off[j];
  }
  // stage the interleaved values (ghost ring filled) in the member's idle
  // state buffer -- the next step overwrites it -- and split them into the
  // Re / Im planes the step kernel reads
  void* stage = b->psi[b->cur ^ 1][i];
  PHX_BCK(b, upload_field(stage, E, 1, 8, b->geo[i], on_device, b->stream));
  PHX_BCK(b, launch_split_complex(stage, b->E[i], 4, 1, b->geo[i], b->stream));
  if (!b->has_E) {
    b->has_E = true;
    b->tables_ok = false;
  }
  return PHX_OK;
}

phx_status phx_batch_set_state(phx_batch* b, int32_t i, const void* psi, const void* n,
                               int on_device) {
  phx_status st = check_member(b, i);
  if (st != PHX_OK) return st;
  DevGuard dg(b->device);
  if (psi) PHX_BCK(b, upload_field(b->psi[b->cur][i], psi, 1, 8, b->geo[i], on_device, b->stream));
  if (n && b->reservoir)
    PHX_BCK(b, upload_field(b->n[b->cur][i], n, 1, 4, b->geo[i], on_device, b->stream));
  return PHX_OK;
}

phx_status phx_batch_get_state(phx_batch* b, int32_t i, void* psi, void* n, int on_device) {
  phx_status st = check_member(b, i);
  if (st != PHX_OK) return st;
  DevGuard dg(b->device);
  if (psi) PHX_BCK(b, download_field(psi, b->psi[b->cur][i], 1, 8, b->geo[i], on_device, b->stream));
  if (n) {
    if (!b->reservoir) return bfail(b, PHX_ESTATE, "no reservoir in this batch");
    PHX_BCK(b, download_field(n, b->n[b->cur][i], 1, 4, b->geo[i], on_device, b->stream));
  }
  PHX_BCK(b, cudaStreamSynchronize(b->stream));
  return PHX_OK;
}

phx_status phx_batch_step_n(phx_batch* b, int64_t nsteps) {
  if (!b) return bfail(nullptr, PHX_EINVAL, "batch is NULL");
  if (nsteps < 0) return bfail(b, PHX_EINVAL, "nsteps must be >= 0");
  if (nsteps == 0) return PHX_OK;
  DevGuard dg(b->device);
  if (any_V(b) && !all_V(b))
    return bfail(b, PHX_ESTATE, "either all members or none must have a potential");
  if (b->reservoir && b->has_E && b->tile_cfg != 0 && !tma_has_drive_reservoir(b->tile_cfg)) {
    if (b->tile_fixed)
      return bfail(b, PHX_EINVAL,
                   "reservoir with drive: tile configuration needs to be 2, 3 or 4 (or 0)");
    b->tile_cfg = 0;  // tuned again among the configurations with that variant
  }
  if (b->tile_cfg == 0) {
    phx_status st = autotune(b);
    if (st != PHX_OK) return st;
  } else if (!b->tables_ok || b->tables_V != any_V(b)) {
    phx_status st = build_tables(b, b->tile_cfg);
    if (st != PHX_OK) return st;
  }
  const int G = 20;  // steps per graph replay (even: the state returns to buffer 0)
  int64_t left = nsteps;
  while (left > 0) {
    if (b->cur == 0 && b->parity == 0 && left >= G) {
      if (!b->graph) {
        phx_status st = build_graph(b, G);
        if (st != PHX_OK) return st;
      }
      PHX_BCK(b, cudaGraphLaunch(b->graph, b->stream));
      count_launch(G);
      left -= G;
      b->host_step += G;
    } else {
      PHX_BCK(b, launch_step(b, b->cur, b->parity, b->stream));
      b->cur ^= 1;
      b->parity ^= 1;
      left -= 1;
      b->host_step += 1;
    }
  }
  return PHX_OK;
}

static phx_status batch_reduce(phx_batch* b, bool residual) {
  DevGuard dg(b->device);
  for (int i = 0; i < b->count; ++i) {
    const phx_params& p = b->p[i];
    ReduceArgs r = reduce_args(p, b->geo[i], b->psi[b->cur][i],
                               b->reservoir ? b->n[b->cur][i] : nullptr, b->P[i], 0,
                               b->has_V[i] ? b->V[i] : nullptr);
    cudaError_t e = residual ? launch_residual(r, b->partials, b->red_dev + 8 * i, b->stream)
                             : launch_norm_energy(r, b->partials, b->red_dev + 8 * i, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "reduction launch");
  }
  PHX_BCK(b, cudaMemcpyAsync(b->red_host, b->red_dev, sizeof(double) * 8 * b->count,
                             cudaMemcpyDeviceToHost, b->stream));
  PHX_BCK(b, cudaStreamSynchronize(b->stream));
  int errw = 0;
  PHX_BCK(b, cudaMemcpy(&errw, b->err_dev, sizeof errw, cudaMemcpyDeviceToHost));
  if (errw) {
    PHX_BCK(b, cudaMemset(b->err_dev, 0, sizeof(int)));
    return bfail(b, PHX_ETIMEOUT, "a bounded wait in the step kernel gave up");
  }
  return PHX_OK;
}

phx_status phx_batch_norm_energy(phx_batch* b, double* norms, double* energies) {
  if (!b) return bfail(nullptr, PHX_EINVAL, "batch is NULL");
  phx_status st = batch_reduce(b, false);
  if (st != PHX_OK) return st;
  bool finite = true;
  for (int i = 0; i < b->count; ++i) {
    const phx_params& p = b->p[i];
    const double dV = (p.lx / p.nx) * (p.ly / p.ny);
    const double N = dV * b->red_host[8 * i], E = dV * b->red_host[8 * i + 1];
    if (norms) norms[i] = N;
    if (energies) energies[i] = E;
    finite = finite && std::isfinite(N) && std::isfinite(E);
  }
  if (!finite) return bfail(b, PHX_ENONFINITE, "a member's state holds NaN or Inf");
  return PHX_OK;
}

phx_status phx_batch_residual(phx_batch* b, double* r_psi, double* r_n, double* omega) {
  if (!b) return bfail(nullptr, PHX_EINVAL, "batch is NULL");
  phx_status st = batch_reduce(b, true);
  if (st != PHX_OK) return st;
  bool finite = true;
  for (int i = 0; i < b->count; ++i) {
    const double* o = b->red_host + 8 * i;
    const double rp = o[0] > 0.0 ? std::sqrt(o[5] / o[0]) : 0.0;
    double rn = 0.0;
    if (b->reservoir) rn = o[4] > 0.0 ? std::sqrt(o[3] / o[4]) : (o[3] == 0.0 ? 0.0 : INFINITY);
    if (r_psi) r_psi[i] = rp;
    if (r_n) r_n[i] = rn;
    if (omega) omega[i] = o[6];
    for (int q = 0; q < 7; ++q) finite = finite && std::isfinite(o[q]);
  }
  if (!finite) return bfail(b, PHX_ENONFINITE, "a member's state holds NaN or Inf");
  return PHX_OK;
}

phx_status phx_batch_time(phx_batch* b, int64_t* step, double* t) {
  if (!b) return bfail(nullptr, PHX_EINVAL, "batch is NULL");
  DevGuard dg(b->device);
  DevClock c;
  PHX_BCK(b, cudaMemcpyAsync(&c, b->clock, sizeof c, cudaMemcpyDeviceToHost, b->stream));
  if (t)
    PHX_BCK(b, cudaMemcpyAsync(t, b->t_inst + (size_t)b->parity * b->count,
                               sizeof(double) * b->count, cudaMemcpyDeviceToHost, b->stream));
  PHX_BCK(b, cudaStreamSynchronize(b->stream));
  if (step) *step = c.step[b->parity];
  return PHX_OK;
}

int32_t phx_batch_tile(const phx_batch* b) { return b ? b->tile_cfg : 0; }

const char* phx_batch_last_error(const phx_batch* b) {
  return b ? b->err.c_str() : g_batch_err.c_str();
}

void phx_batch_destroy(phx_batch* b) {
  if (!b) return;
  DevGuard dg(b->device);
  bfree(b);
  delete b;
}

}  // extern "C"
