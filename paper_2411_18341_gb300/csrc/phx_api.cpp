// C ABI of the RK4 dNLSE solver: parameter validation, device buffers,
// uploads with ghost-ring fill, step scheduling and FP64 reductions.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/phx.h"
#include "phx_internal.h"
#include "rk4_tma.h"
#include "kfilter.h"
#include "ssf.h"

namespace phx {
unsigned long long launch_total();
void arm_injection(unsigned mask);
}

using namespace phx;

struct phx_handle {
  phx_params p;
  ModelKey m;
  Geometry geo;
  size_t esize = 0;          // bytes per real
  void* psi[2] = {nullptr, nullptr};
  void* n[2] = {nullptr, nullptr};
  void* P = nullptr;
  long long P_stride = 0;    // elements between P_+ and P_- planes (0 = shared)
  void* V = nullptr;
  bool has_V = false;
  bool owns_state = true;    // psi, n, P allocated here (false: the caller's buffers)
  void* E = nullptr;         // coherent drive amplitude: Re, Im plane per component
  long long E_stride = 0;    // elements between the E_+ and E_- plane pairs (0 = shared)
  bool has_E = false;
  KFilter kf;                // k-space smoothing (off unless set)
  FftPair ssf_fft;           // FFT plans of the split-step integrator (made at first use)
  int ssf_ncomp = 0;         // components the plans were made for
  double* imag_red = nullptr;  // norm scratch of the imaginary-time steps
  DevClock* clock = nullptr;
  double* partials = nullptr;
  double* red_dev = nullptr;
  double* red_host = nullptr;  // pinned
  int cur = 0;                 // buffer holding the current state
  int parity = 0;              // clock slot of the current step
  long long host_step = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  int* err_dev = nullptr;      // set by kernels whose bounded waits gave up (in red_dev)
  double dt_rk4 = 0;           // RK4 stability limit of the grid (phx_stability_dt)
  int tile_cfg = 0;            // chosen tile configuration of the FP32 scalar kernel
  bool tuned = false;          // tile_cfg settled (explicit or autotuned)
  bool maps_ok = false;        // TMA tensor maps encoded for (tile_cfg, has_V)
  bool maps_V = false;
  TileInst h_inst;             // descriptor of this handle for the persistent kernel
  TileInst* d_inst = nullptr;  // its device copy
  int* ms_done = nullptr;      // per-tile step counters of a multi-step launch
  int ms_done_len = 0;
  std::string err;
};

namespace {

thread_local std::string g_err = "no error";

bool periodic(const phx_params& p) {
  return p.bc_x == PHX_BC_PERIODIC && p.bc_y == PHX_BC_PERIODIC;
}

bool spinor_tma_cfg(int cfg) { return cfg >= TILE_SPINOR_64x16 && cfg <= TILE_SPINOR_64x32; }

phx_status fail(phx_handle* h, phx_status s, const std::string& msg) {
  if (h)
    h->err = msg;
  else
    g_err = msg;
  return s;
}

phx_status cuda_fail(phx_handle* h, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" +
                  cudaGetErrorString(e) + ")";
  return fail(h, e == cudaErrorMemoryAllocation ? PHX_ENOMEM : PHX_ECUDA, m);
}

#define PHX_CK(h, expr)                                    \
  do {                                                     \
    cudaError_t _e = (expr);                               \
    if (_e != cudaSuccess) return cuda_fail((h), _e, #expr); \
  } while (0)

bool is_finite(double x) { return std::isfinite(x); }

phx_status validate(const phx_params* p, double* dtmax_out) {
  const char* msg = check_params(p, dtmax_out);
  if (msg) return fail(nullptr, PHX_EINVAL, msg);
  return PHX_OK;
}

void free_all(phx_handle* h) {
  if (!h) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->owns_state) {
    for (int b = 0; b < 2; ++b) {
      if (h->psi[b]) cudaFree(h->psi[b]);
      if (h->n[b]) cudaFree(h->n[b]);
    }
    if (h->P) cudaFree(h->P);
  }
  if (h->V) cudaFree(h->V);
  if (h->E) cudaFree(h->E);
  kfilter_release(h->kf);
  fft_pair_release(h->ssf_fft);
  if (h->imag_red) cudaFree(h->imag_red);
  if (h->clock) cudaFree(h->clock);
  if (h->partials) cudaFree(h->partials);
  if (h->red_dev) cudaFree(h->red_dev);
  if (h->red_host) cudaFreeHost(h->red_host);
  if (h->d_inst) cudaFree(h->d_inst);
  if (h->ms_done) cudaFree(h->ms_done);
  cudaSetDevice(prev);
}

phx_status upload(phx_handle* h, void* dst, const void* src, int nplanes,
                  size_t elem, int on_device) {
  PHX_CK(h, upload_field(dst, src, nplanes, elem, h->geo, on_device, h->stream));
  return PHX_OK;
}

phx_status download(phx_handle* h, void* dst, const void* src, int nplanes,
                    size_t elem, int on_device) {
  PHX_CK(h, download_field(dst, src, nplanes, elem, h->geo, on_device, h->stream));
  return PHX_OK;
}

ReduceArgs make_reduce_args(const phx_handle* h) {
  return reduce_args(h->p, h->geo, h->psi[h->cur], h->m.reservoir ? h->n[h->cur] : nullptr,
                     h->P, h->P_stride, h->has_V ? h->V : nullptr);
}

// Tile configuration of the persistent FP32 scalar kernel: the one with the
// smallest modelled time = (rounds of tiles over the SMs) x (region area).
int choose_tile(const phx_handle* h) {
  if (h->p.tile != 0) return h->p.tile;
  int best = TILE_64x64;
  double best_cost = 1e300;
  for (int cfg : {TILE_64x64, TILE_64x48, TILE_64x32}) {
    TmaBox b = tma_box(cfg);
    long long tx = (h->p.nx + 1 + b.tx - 1) / b.tx, ty = (h->p.ny + b.ty - 1) / b.ty;
    long long rounds = (tx * ty + h->num_sms - 1) / h->num_sms;
    double cost = (double)rounds * (b.tx + 6) * (b.ty + 6);
    if (cost < best_cost) {
      best_cost = cost;
      best = cfg;
    }
  }
  return best;
}

// Process-wide autotune results: (device, nx, ny, bc_x, bc_y, reservoir,
// potential) -> fastest tile configuration.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int, int, int>, int> g_tune;

bool encode_maps(phx_handle* h);
TileArgs tile_args(phx_handle* h, int inj);

// Whether a reservoir handle with a drive steps on the TMA-fed kernel: its
// tile is autotuned (among the configurations with that variant) or fixed to
// one of them.
bool drive_reservoir_tile(const phx_handle* h) {
  return h->p.tile == 0 || tma_has_drive_reservoir(h->p.tile);
}

// One persistent TMA-fed step launch in configuration cfg.
cudaError_t launch_tma(phx_handle* h, int cfg, const TileArgs& ta, int grid) {
  if (spinor_tma_cfg(cfg))
    return launch_rk4_tma_spinor(cfg, h->has_V, periodic(h->p), h->m.tetm, ta, h->stream, grid);
  const int mode = h->m.reservoir ? (h->has_E ? 3 : 1) : (h->has_E ? 2 : 0);
  return launch_rk4_tma_f32(cfg, mode, h->has_V, periodic(h->p), ta, h->stream, grid);
}

// Steps per multi-step launch (configuration 8): long enough that the launch
// and its ramp are negligible, short enough that a chunk is a few ms.
constexpr int MS_CHUNK = 128;

// Steps the next multi-step launch may take out of `want` (0: it does not
// apply, one single-step launch instead).  Needs the tensor maps encoded.
int ms_steps_possible(const phx_handle* h, int64_t want) {
  if (!tma_has_multistep(h->tile_cfg) || h->m.precision != 32 || h->m.ncomp != 1 || h->has_E)
    return 0;
  const int tx = h->h_inst.tiles_x, nt = tx * h->h_inst.tiles_y;
  const int G = h->num_sms * tma_ctas_per_sm(h->tile_cfg);
  // an item must never wait for this CTA's previous item, whose counter is
  // published only after the next item started (see the kernel)
  if (G >= nt - 4 * tx && G <= nt + 4 * tx) return 0;
  int64_t S = want < MS_CHUNK ? want : MS_CHUNK;
  if (h->kf.every > 0) {  // end the chunk where the k-space filter applies
    const int64_t to = h->kf.every - h->host_step % h->kf.every;
    if (S > to) S = to;
  }
  return S >= 2 ? (int)S : 0;
}

// One multi-step launch of S steps on the handle's buffers (the state ends in
// buffer cur ^ (S & 1)); with the clock advanced unless `clock` is false.
cudaError_t launch_ms(phx_handle* h, int S, int inj, bool clock) {
  const int tx = h->h_inst.tiles_x, ty = h->h_inst.tiles_y, nt = tx * ty;
  if (h->ms_done_len < nt) {
    if (h->ms_done) cudaFree(h->ms_done);
    h->ms_done = nullptr;
    h->ms_done_len = 0;
    cudaError_t e = cudaMalloc((void**)&h->ms_done, sizeof(int) * nt);
    if (e != cudaSuccess) return e;
    h->ms_done_len = nt;
  }
  cudaError_t e = cudaMemsetAsync(h->ms_done, 0, sizeof(int) * nt, h->stream);
  if (e != cudaSuccess) return e;
  TileArgs ta = tile_args(h, inj);
  ta.done = h->ms_done;
  ta.ms_steps = S;
  ta.tiles_y = ty;
  const int grid = h->num_sms * tma_ctas_per_sm(h->tile_cfg);
  e = launch_rk4_tma_f32_ms(h->tile_cfg, h->m.reservoir ? 1 : 0, h->has_V, periodic(h->p), ta,
                            h->stream, grid);
  if (e != cudaSuccess || !clock) return e;
  return launch_clock_advance(h->clock, h->parity, S, h->p.dt, h->stream);
}

// Time every tile configuration of the FP32 scalar kernel on this handle's
// own state and keep the fastest.  A step reads the current buffer and writes
// the other one, so repeating it without swapping leaves the state intact.
phx_status autotune(phx_handle* h) {
  const auto key = std::make_tuple(h->device, h->p.nx, h->p.ny, h->p.bc_x, h->p.bc_y,
                                   (int)h->m.reservoir + 2 * h->m.ncomp + 8 * (int)h->m.tetm +
                                       16 * (int)h->has_E,
                                   (int)h->has_V);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      h->tile_cfg = it->second;
      h->maps_ok = false;
      return PHX_OK;
    }
  }
  const int scalar_cands[] = {TILE_64x48_M2, TILE_64x64_M2,   TILE_64x48,
                              TILE_64x64,    TILE_64x32,      TILE_64x32_M2_2,
                              TILE_64x32_M4_2, TILE_64x32_M4_2_MS};
  const int spinor_cands[] = {TILE_SPINOR_64x24, TILE_SPINOR_64x16, TILE_SPINOR_64x32};
  // reservoir and drive: the configurations with that variant
  const int drive_res_cands[] = {TILE_64x48, TILE_64x32, TILE_64x48_M2};
  const bool sp = h->m.ncomp == 2;
  const bool drive_res = !sp && h->m.reservoir && h->has_E;
  const int* cands = sp ? spinor_cands : (drive_res ? drive_res_cands : scalar_cands);
  cudaEvent_t e0, e1;
  PHX_CK(h, cudaEventCreate(&e0));
  PHX_CK(h, cudaEventCreate(&e1));
  // The multi-step configuration advances the state: it runs on the
  // handle's buffers after the current state is saved, which is copied back
  // afterwards (the clock is not advanced while tuning).
  const size_t psi_bytes = (size_t)h->geo.plane * h->m.ncomp * 2 * h->esize;
  const size_t n_bytes = h->m.reservoir ? (size_t)h->geo.plane * h->m.ncomp * h->esize : 0;
  void* saved = nullptr;
  const bool try_ms = !sp && !h->has_E;
  if (try_ms && cudaMalloc(&saved, psi_bytes + n_bytes) != cudaSuccess) {
    cudaGetLastError();
    saved = nullptr;
  }
  if (saved) {
    PHX_CK(h, cudaMemcpyAsync(saved, h->psi[h->cur], psi_bytes, cudaMemcpyDeviceToDevice,
                              h->stream));
    if (n_bytes)
      PHX_CK(h, cudaMemcpyAsync(static_cast<char*>(saved) + psi_bytes, h->n[h->cur], n_bytes,
                                cudaMemcpyDeviceToDevice, h->stream));
  }
  // five interleaved rounds of ten launches (configurations within a few per
  // cent of each other then come out in the same order from run to run);
  // each configuration keeps its fastest round
  // (time per step)
  const int nc = (sp || drive_res) ? 3 : (saved ? 8 : 7);
  float cfg_ms[8];
  for (int c = 0; c < nc; ++c) cfg_ms[c] = 1e30f;
  for (int round = 0; round < 5; ++round) {
    for (int c = 0; c < nc; ++c) {
      const int cfg = cands[c];
      h->tile_cfg = cfg;
      if (!encode_maps(h)) continue;
      // a test hook armed for the real step must not fire here
      const TileArgs ta = tile_args(h, 0);
      const int slots = h->num_sms * tma_ctas_per_sm(cfg);
      const int grid = ta.ntiles < slots ? ta.ntiles : slots;
      const int ms_n = tma_has_multistep(cfg) ? ms_steps_possible(h, 8) : 0;
      if (tma_has_multistep(cfg) && ms_n < 2) continue;
      auto launch = [&]() {
        return ms_n ? launch_ms(h, ms_n, 0, false) : launch_tma(h, cfg, ta, grid);
      };
      const int reps = ms_n ? 4 : 10;
      const int per_rep = ms_n ? ms_n : 1;
      cudaError_t e = cudaSuccess;
      for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = launch();
      if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
      for (int i = 0; i < reps && e == cudaSuccess; ++i) e = launch();
      if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      ms /= (float)(reps * per_rep);
      if (ms < cfg_ms[c]) cfg_ms[c] = ms;
    }
  }
  if (saved) {
    PHX_CK(h, cudaMemcpyAsync(h->psi[h->cur], saved, psi_bytes, cudaMemcpyDeviceToDevice,
                              h->stream));
    if (n_bytes)
      PHX_CK(h, cudaMemcpyAsync(h->n[h->cur], static_cast<char*>(saved) + psi_bytes, n_bytes,
                                cudaMemcpyDeviceToDevice, h->stream));
    PHX_CK(h, cudaStreamSynchronize(h->stream));
    cudaFree(saved);
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
  h->tile_cfg = best;
  h->maps_ok = false;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best;
  return PHX_OK;
}

// Fill the handle's instance descriptor for the current tile configuration
// and queue its upload on the handle's stream.
bool encode_maps(phx_handle* h) {
  // the TMA-fed drive variants: single-component fields
  void* E = (h->has_E && h->m.ncomp == 1) ? h->E : nullptr;
  if (!fill_tile_inst(h->h_inst, h->p, h->geo, h->psi, h->n, h->P, h->has_V ? h->V : nullptr,
                      h->tile_cfg, E))
    return false;
  if (cudaMemcpyAsync(h->d_inst, &h->h_inst, sizeof(TileInst), cudaMemcpyHostToDevice,
                      h->stream) != cudaSuccess)
    return false;
  h->maps_ok = true;
  h->maps_V = h->has_V;
  return true;
}

TileArgs tile_args(phx_handle* h, int inj) {
  TileArgs ta;
  ta.inst = h->d_inst;
  ta.tile_info = nullptr;
  ta.one = scalars_of(h->h_inst);
  ta.one.p_shared = h->P_stride == 0;
  ta.ntiles = h->h_inst.tiles_x * h->h_inst.tiles_y;
  ta.ninst = 1;
  ta.cur = h->cur;
  ta.clock = h->clock;
  ta.parity = h->parity;
  ta.t_inst = nullptr;
  ta.err = h->err_dev;
  ta.inject_timeout = inj;
  ta.tiles_y = h->h_inst.tiles_y;
  return ta;
}

// The device error word copied to the host with the results (slot 8 of
// red_host, already synchronised): clears it on the device when it is set.
phx_status took_device_error(phx_handle* h) {
  int e = 0;
  std::memcpy(&e, h->red_host + 8, sizeof e);
  if (e) {
    PHX_CK(h, cudaMemsetAsync(h->err_dev, 0, sizeof(int), h->stream));
    return fail(h, PHX_ETIMEOUT, "a bounded wait in the step kernel gave up (TMA copy did not complete)");
  }
  return PHX_OK;
}

// Reads and clears the device error word (synchronises the stream).
phx_status check_device_error(phx_handle* h) {
  int e = 0;
  PHX_CK(h, cudaMemcpyAsync(&e, h->err_dev, sizeof e, cudaMemcpyDeviceToHost, h->stream));
  PHX_CK(h, cudaStreamSynchronize(h->stream));
  if (e) {
    PHX_CK(h, cudaMemsetAsync(h->err_dev, 0, sizeof(int), h->stream));
    return fail(h, PHX_ETIMEOUT, "a bounded wait in the step kernel gave up (TMA copy did not complete)");
  }
  return PHX_OK;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int now = -1;
    cudaGetDevice(&now);
    if (prev >= 0 && now != prev) cudaSetDevice(prev);
  }
};

// Bytes of the five state buffers (psi 0/1, n 0/1, P) for parameters p.
void state_sizes(const phx_params& p, size_t sizes[5]) {
  const Geometry g = padded_geometry(p);
  const size_t es = p.precision == 32 ? 4 : 8, nc = p.spinor ? 2 : 1;
  sizes[0] = sizes[1] = nc * (size_t)g.plane * 2 * es;
  sizes[2] = sizes[3] = sizes[4] = p.reservoir ? nc * (size_t)g.plane * es : 0;
}

phx_status create_impl(const phx_params* p, void* const* ext, phx_handle** out);

}  // namespace

extern "C" {

phx_status phx_params_init(phx_params* p) {
  if (!p) return fail(nullptr, PHX_EINVAL, "params is NULL");
  std::memset(p, 0, sizeof(*p));
  p->struct_size = sizeof(phx_params);
  p->nx = 64;
  p->ny = 64;
  p->lx = 1.0;
  p->ly = 1.0;
  p->bc_x = PHX_BC_PERIODIC;
  p->bc_y = PHX_BC_PERIODIC;
  p->precision = 32;
  p->hbar2_over_2m = 0.67;
  return PHX_OK;
}

phx_status phx_stability_dt(const phx_params* p, double* dt_max) {
  if (!dt_max) return fail(nullptr, PHX_EINVAL, "dt_max is NULL");
  return validate(p, dt_max);
}

phx_status phx_create(const phx_params* p, phx_handle** out) {
  return create_impl(p, nullptr, out);
}

phx_status phx_buffer_sizes(const phx_params* p, size_t sizes[5]) {
  if (!sizes) return fail(nullptr, PHX_EINVAL, "sizes is NULL");
  double dtmax = 0;
  phx_status st = validate(p, &dtmax);
  if (st != PHX_OK) return st;
  state_sizes(*p, sizes);
  return PHX_OK;
}

phx_status phx_create_with_buffers(const phx_params* p, void* const buffers[5],
                                   phx_handle** out) {
  if (!out) return fail(nullptr, PHX_EINVAL, "out is NULL");
  *out = nullptr;
  if (!buffers) return fail(nullptr, PHX_EINVAL, "buffers is NULL");
  double dtmax = 0;
  phx_status st = validate(p, &dtmax);
  if (st != PHX_OK) return st;
  size_t sizes[5];
  state_sizes(*p, sizes);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(nullptr, PHX_ENODEV, "no CUDA device");
  for (int i = 0; i < 5; ++i) {
    if (!sizes[i]) continue;
    if (!buffers[i]) return fail(nullptr, PHX_EINVAL, "buffers[" + std::to_string(i) + "] is NULL");
    if (reinterpret_cast<uintptr_t>(buffers[i]) % 256)
      return fail(nullptr, PHX_EINVAL, "buffers[" + std::to_string(i) + "] is not 256-byte aligned");
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, buffers[i]) != cudaSuccess || a.type != cudaMemoryTypeDevice ||
        a.device != dev) {
      cudaGetLastError();
      return fail(nullptr, PHX_EINVAL,
                  "buffers[" + std::to_string(i) + "] is not device memory of the current device");
    }
  }
  return create_impl(p, buffers, out);
}

}  // extern "C"

namespace {

phx_status create_impl(const phx_params* p, void* const* ext, phx_handle** out) {
  if (!out) return fail(nullptr, PHX_EINVAL, "out is NULL");
  *out = nullptr;
  double dtmax = 0;
  phx_status st = validate(p, &dtmax);
  if (st != PHX_OK) return st;
  if (!(p->dt > 0.0)) return fail(nullptr, PHX_EINVAL, "dt must be > 0");
  if (p->integrator == PHX_INTEGRATOR_SPLIT) {
    // split-step: exact linear propagator; the local half steps of the
    // reservoir model are one RK4 step of dt/2 with decay rate gamma_r
    if (p->bc_x != PHX_BC_PERIODIC || p->bc_y != PHX_BC_PERIODIC)
      return fail(nullptr, PHX_EINVAL, "integrator = split-step needs periodic boundaries");
    if (p->wigner_nu > 0.0)
      return fail(nullptr, PHX_EINVAL, "integrator = split-step excludes truncated-Wigner noise");
    if (p->reservoir && 0.5 * p->dt * p->gamma_r > 2.78) {
      char buf[160];
      std::snprintf(buf, sizeof buf,
                    "dt = %.6g ps: the local RK4 half step needs dt/2 * gamma_r <= 2.78", p->dt);
      return fail(nullptr, PHX_EINVAL, buf);
    }
  } else if (p->dt > dtmax * (1.0 + 1e-12)) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "dt = %.6g ps exceeds the RK4 stability limit %.6g ps",
                  p->dt, dtmax);
    return fail(nullptr, PHX_EINVAL, buf);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(nullptr, PHX_ENODEV, std::string("no CUDA device: ") + cudaGetErrorString(e));
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return fail(nullptr, PHX_ENODEV, cudaGetErrorString(e));
  if (prop.major != 10 || prop.minor != 3)
    return fail(nullptr, PHX_ENODEV, "kernels are built for sm_103a (GB300); device is sm_" +
                                         std::to_string(prop.major * 10 + prop.minor));

  phx_handle* h = new (std::nothrow) phx_handle();
  if (!h) return fail(nullptr, PHX_ENOMEM, "host allocation failed");
  h->p = *p;
  h->dt_rk4 = dtmax;
  h->device = dev;
  h->num_sms = prop.multiProcessorCount;
  h->stream = static_cast<cudaStream_t>(p->stream);
  h->m.precision = p->precision;
  h->m.ncomp = p->spinor ? 2 : 1;
  h->m.reservoir = p->reservoir;
  h->m.tetm = (p->spinor && p->delta_lt != 0.0) ? 1 : 0;
  h->esize = p->precision == 32 ? 4 : 8;
  h->geo = padded_geometry(*p);
  h->owns_state = ext == nullptr;
  const Geometry& g = h->geo;

  auto alloc = [&](void** ptr, size_t bytes) -> cudaError_t {
    if (take_injection(INJ_ALLOC)) return cudaErrorMemoryAllocation;
    cudaError_t r = cudaMalloc(ptr, bytes);
    if (r != cudaSuccess) return r;
    return cudaMemsetAsync(*ptr, 0, bytes, h->stream);
  };
  // a state buffer: the caller's (zeroed here) or a new allocation
  auto state = [&](void** ptr, int idx, size_t bytes) -> cudaError_t {
    if (!ext) return alloc(ptr, bytes);
    *ptr = ext[idx];
    return cudaMemsetAsync(*ptr, 0, bytes, h->stream);
  };
  const int nc = h->m.ncomp;
  const size_t cplx = 2 * h->esize, real = h->esize;
  cudaError_t ce = cudaSuccess;
  for (int b = 0; b < 2 && ce == cudaSuccess; ++b) {
    ce = state(&h->psi[b], b, (size_t)nc * g.plane * cplx);
    if (ce == cudaSuccess && h->m.reservoir) ce = state(&h->n[b], 2 + b, (size_t)nc * g.plane * real);
  }
  if (ce == cudaSuccess && h->m.reservoir) {
    ce = state(&h->P, 4, (size_t)nc * g.plane * real);
    h->P_stride = (nc == 2) ? g.plane : 0;
  }
  if (ce == cudaSuccess) ce = alloc((void**)&h->clock, sizeof(DevClock));
  if (ce == cudaSuccess)
    ce = alloc((void**)&h->partials, reduce_partials_len(g) * sizeof(double));
  // 8 results and, in slot 8, the device error word, so that one copy
  // brings both back
  if (ce == cudaSuccess) ce = alloc((void**)&h->red_dev, 9 * sizeof(double));
  if (ce == cudaSuccess) h->err_dev = reinterpret_cast<int*>(h->red_dev + 8);
  if (ce == cudaSuccess) ce = cudaMallocHost((void**)&h->red_host, 9 * sizeof(double));
  if (ce == cudaSuccess) ce = alloc((void**)&h->d_inst, sizeof(TileInst));
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    std::string msg = std::string("device allocation failed: ") + cudaGetErrorString(ce);
    free_all(h);
    delete h;
    return fail(nullptr, ce == cudaErrorMemoryAllocation ? PHX_ENOMEM : PHX_ECUDA, msg);
  }
  if (p->precision == 32 && !p->spinor)
    h->tile_cfg = choose_tile(h);
  else if (p->precision == 32 && p->spinor && p->reservoir &&
           (p->tile == 0 || spinor_tma_cfg(p->tile)))
    h->tile_cfg = p->tile ? p->tile : TILE_SPINOR_64x24;
  else
    h->tile_cfg = TILE_GENERIC;
  *out = h;
  return PHX_OK;
}

}  // namespace

extern "C" {

phx_status phx_set_pump(phx_handle* h, const void* P_plus, const void* P_minus,
                        int on_device) {
  if (!h) return fail(nullptr, PHX_EINVAL, "handle is NULL");
  if (!h->m.reservoir) return fail(h, PHX_ESTATE, "set_pump needs reservoir = 1");
  if (!P_plus) return fail(h, PHX_EINVAL, "P_plus is NULL");
  DeviceGuard dg(h->device);
  const Geometry& g = h->geo;
  phx_status st = upload(h, h->P, P_plus, 1, h->esize, on_device);
  if (st != PHX_OK) return st;
  if (h->m.ncomp == 2) {
    if (P_minus) {
      char* d1 = static_cast<char*>(h->P) + (size_t)g.plane * h->esize;
      st = upload(h, d1, P_minus, 1, h->esize, on_device);
      if (st != PHX_OK) return st;
      h->P_stride = g.plane;
    } else {
      h->P_stride = 0;  // both components read plane 0
    }
  }
  return PHX_OK;
}

phx_status phx_set_potential(phx_handle* h, const void* V, int on_device) {
  if (!h) return fail(nullptr, PHX_EINVAL, "handle is NULL");
  DeviceGuard dg(h->device);
  if (!V) {
    h->has_V = false;
    return PHX_OK;
  }
  if (!h->V) {
    size_t bytes = (size_t)h->geo.plane * h->esize;
    PHX_CK(h, cudaMalloc(&h->V, bytes));
    PHX_CK(h, cudaMemsetAsync(h->V, 0, bytes, h->stream));
  }
  phx_status st = upload(h, h->V, V, 1, h->esize, on_device);
  if (st != PHX_OK) return st;
  h->has_V = true;
  return PHX_OK;
}

phx_status phx_set_drive(phx_handle* h, const void* E_plus, const void* E_minus,
                         int on_device) {
  if (!h) return fail(nullptr, PHX_EINVAL, "handle is NULL");
  DeviceGuard dg(h->device);
  if (!E_plus) {
    if (h->has_E && h->p.tile == 0) h->tuned = false;
    h->has_E = false;
    h->maps_ok = false;
    return PHX_OK;
  }
  const Geometry& g = h->geo;
  const size_t cplx = 2 * h->esize;
  if (!h->E) {
    size_t bytes = (size_t)g.plane * cplx * h->m.ncomp;
    PHX_CK(h, cudaMalloc(&h->E, bytes));
    PHX_CK(h, cudaMemsetAsync(h->E, 0, bytes, h->stream));
  }
  // Stage the interleaved values (ghost ring filled) in the idle half of the
  // state's double buffer -- the next step overwrites it -- and split them
  // into Re / Im planes, the layout the step kernels read.
  void* stage = h->psi[h->cur ^ 1];
  const int planes = (h->m.ncomp == 2 && E_minus) ? 2 : 1;
  phx_status st = upload(h, stage, E_plus, 1, cplx, on_device);
  if (st != PHX_OK) return st;
  if (planes == 2) {
    st = upload(h, static_cast<char*>(stage) + (size_t)g.plane * cplx, E_minus, 1, cplx,
                on_device);
    if (st != PHX_OK) return st;
  }
  PHX_CK(h, launch_split_complex(stage, h->E, (int)h->esize, planes, g, h->stream));
  h->E_stride = planes == 2 ? 2 * g.plane : 0;
  // a drive changes the kernel variant (and, with a reservoir, the tile
  // configurations that have it): an autotuned handle is tuned again
  if (!h->has_E && h->p.tile == 0) h->tuned = false;
  h->has_E = true;
  h->maps_ok = false;
  return PHX_OK;
}

phx_status phx_set_state(phx_handle* h, const void* psi, const void* n, int on_device) {
  if (!h) return fail(nullptr, PHX_EINVAL, "handle is NULL");
  DeviceGuard dg(h->device);
  if (psi) {
    phx_status st = upload(h, h->psi[h->cur], psi, h->m.ncomp, 2 * h->esize, on_device);
    if (st != PHX_OK) return st;
  }
  if (n && h->m.reservoir) {
    phx_status st = upload(h, h->n[h->cur], n, h->m.ncomp, h->esize, on_device);
    if (st != PHX_OK) return st;
  }
  return PHX_OK;
}

phx_status phx_get_state(phx_handle* h, void* psi, void* n, int on_device) {
  if (!h) return fail(nullptr, PHX_EINVAL, "handle is NULL");
  DeviceGuard dg(h->device);
  if (psi) {
    phx_status st = download(h, psi, h->psi[h->cur], h->m.ncomp, 2 * h->esize, on_device);
    if (st != PHX_OK) return st;
  }
  if (n) {
    if (!h->m.reservoir) return fail(h, PHX_ESTATE, "no reservoir in this handle");
    phx_status st = download(h, n, h->n[h->cur], h->m.ncomp, h->esize, on_device);
    if (st != PHX_OK) return st;
  }
  PHX_CK(h, cudaStreamSynchronize(h->stream));
  return check_device_error(h);
}

phx_status phx_step_n(phx_handle* h, int64_t nsteps) {
  if (!h) return fail(nullptr, PHX_EINVAL, "handle is NULL");
  if (nsteps < 0) return fail(h, PHX_EINVAL, "nsteps must be >= 0");
  if (h->p.dt > h->dt_rk4 * (1.0 + 1e-12))
    return fail(h, PHX_ESTATE, "dt exceeds the RK4 stability limit (a split-step handle: use "
                               "phx_step_ssf)");
  DeviceGuard dg(h->device);
  const Coeffs k = make_coeffs(h->p);
  const NoiseKey nz = make_noise_key(h->p);
  for (int64_t s = 0; s < nsteps; ++s) {
    cudaError_t e;
    int taken = 1;  // steps of this launch
    if (take_injection(INJ_LAUNCH))
      return fail(h, PHX_ECUDA, "rk4 step launch: injected launch failure");
    const int inj = take_injection(INJ_TIMEOUT) ? 1 : 0;
    if (h->m.precision == 32) {
      StepArgs<float> a;
      a.geo = h->geo;
      a.psi_in = static_cast<const float2*>(h->psi[h->cur]);
      a.psi_out = static_cast<float2*>(h->psi[h->cur ^ 1]);
      a.n_in = static_cast<const float*>(h->n[h->cur]);
      a.n_out = static_cast<float*>(h->n[h->cur ^ 1]);
      a.P = static_cast<const float*>(h->P);
      a.P_comp_stride = h->P_stride;
      a.V = h->has_V ? static_cast<const float*>(h->V) : nullptr;
      a.E = h->has_E ? static_cast<const float*>(h->E) : nullptr;
      a.E_comp_stride = h->E_stride;
      a.omega = h->p.drive_omega;
      a.k = cast_coeffs<float>(k);
      a.dt64 = k.dt;
      a.noise = nz;
      a.clock = h->clock;
      a.parity = h->parity;
      a.inject_timeout = inj;
      // drive: TMA-fed for a scalar field (with a reservoir only in the
      // configurations that have that variant), else generic
      const bool drive_ok =
          !h->has_E || (h->m.ncomp == 1 && (!h->m.reservoir || drive_reservoir_tile(h)));
      if (h->tile_cfg != TILE_GENERIC && drive_ok &&
          (h->m.ncomp == 1 || spinor_tma_cfg(h->tile_cfg))) {
        if (!h->tuned) {
          if (h->p.tile == 0) {
            phx_status ts = autotune(h);
            if (ts != PHX_OK) return ts;
          }
          h->tuned = true;
        }
        if (!h->maps_ok || h->maps_V != h->has_V) {
          if (!encode_maps(h)) return fail(h, PHX_ECUDA, "cuTensorMapEncodeTiled failed");
        }
        const int ms_n = ms_steps_possible(h, nsteps - s);
        if (ms_n) {
          taken = ms_n;
          e = launch_ms(h, ms_n, inj, true);
        } else {
          const TileArgs ta = tile_args(h, inj);
          const int slots = h->num_sms * tma_ctas_per_sm(h->tile_cfg);
          const int grid = ta.ntiles < slots ? ta.ntiles : slots;
          e = launch_tma(h, h->tile_cfg, ta, grid);
        }
      } else {
        e = launch_rk4_step_f32(h->m, a, h->stream, h->p.tile);
      }
    } else {
      StepArgs<double> a;
      a.geo = h->geo;
      a.psi_in = static_cast<const double2*>(h->psi[h->cur]);
      a.psi_out = static_cast<double2*>(h->psi[h->cur ^ 1]);
      a.n_in = static_cast<const double*>(h->n[h->cur]);
      a.n_out = static_cast<double*>(h->n[h->cur ^ 1]);
      a.P = static_cast<const double*>(h->P);
      a.P_comp_stride = h->P_stride;
      a.V = h->has_V ? static_cast<const double*>(h->V) : nullptr;
      a.E = h->has_E ? static_cast<const double*>(h->E) : nullptr;
      a.E_comp_stride = h->E_stride;
      a.omega = h->p.drive_omega;
      a.k = k;
      a.dt64 = k.dt;
      a.noise = nz;
      a.clock = h->clock;
      a.parity = h->parity;
      a.inject_timeout = 0;
      e = launch_rk4_step_f64(h->m, a, h->stream, h->p.tile);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "rk4 step launch");
    h->cur ^= taken & 1;
    h->parity ^= 1;
    h->host_step += taken;
    s += taken - 1;
    if (h->kf.every > 0 && h->host_step % h->kf.every == 0) {
      const char* msg = kfilter_apply(h->kf, h->psi[h->cur], h->geo, h->m.ncomp,
                                      h->m.precision, h->p.lx, h->p.ly, h->stream);
      if (msg) return fail(h, PHX_ECUDA, msg);
    }
  }
  return PHX_OK;
}

phx_status phx_step_ssf(phx_handle* h, int64_t nsteps) {
  if (!h) return fail(nullptr, PHX_EINVAL, "handle is NULL");
  if (nsteps < 0) return fail(h, PHX_EINVAL, "nsteps must be >= 0");
  if (h->p.bc_x != PHX_BC_PERIODIC || h->p.bc_y != PHX_BC_PERIODIC)
    return fail(h, PHX_ESTATE, "split-step needs periodic boundaries");
  if (h->has_E || h->p.wigner_nu > 0.0)
    return fail(h, PHX_ESTATE, "split-step supports neither a drive nor truncated-Wigner noise");
  if (nsteps == 0) return PHX_OK;
  DeviceGuard dg(h->device);
  if (h->ssf_fft.have_plans && h->ssf_ncomp != h->m.ncomp) fft_pair_release(h->ssf_fft);
  const char* msg = fft_pair_setup(h->ssf_fft, h->geo, h->m.ncomp, h->m.precision);
  if (msg) return fail(h, PHX_ECUDA, msg);
  h->ssf_ncomp = h->m.ncomp;
  const SsfCoeffs k = ssf_coeffs(h->p);
  const NoiseKey nz = make_noise_key(h->p);
  for (int64_t s = 0; s < nsteps; ++s) {
    if (h->m.reservoir)
      msg = ssf_step_reservoir(h->ssf_fft, h->psi[h->cur], h->n[h->cur], h->P, h->P_stride,
                               h->geo, h->m.precision, h->m.ncomp, h->has_V ? h->V : nullptr,
                               h->p, k, nz, h->clock, h->parity, h->stream);
    else
      msg = ssf_step(h->ssf_fft, h->psi[h->cur], h->geo, h->m.precision, h->m.ncomp,
                     h->has_V ? h->V : nullptr, k, nz, h->clock, h->parity, h->stream);
    if (msg) return fail(h, PHX_ECUDA, msg);
    h->parity ^= 1;
    h->host_step += 1;
  }
  PHX_CK(h, launch_fill_ghosts(h->psi[h->cur], (int)(2 * h->esize), h->m.ncomp, h->geo,
                               h->stream));
  if (h->m.reservoir)
    PHX_CK(h, launch_fill_ghosts(h->n[h->cur], (int)h->esize, h->m.ncomp, h->geo, h->stream));
  return PHX_OK;
}

phx_status phx_step_imag(phx_handle* h, int64_t nsteps) {
  if (!h) return fail(nullptr, PHX_EINVAL, "handle is NULL");
  if (nsteps < 0) return fail(h, PHX_EINVAL, "nsteps must be >= 0");
  if (h->m.reservoir) return fail(h, PHX_ESTATE, "imaginary time needs a field without reservoir");
  if (h->p.bc_x != PHX_BC_PERIODIC || h->p.bc_y != PHX_BC_PERIODIC)
    return fail(h, PHX_ESTATE, "imaginary time needs periodic boundaries");
  if (nsteps == 0) return PHX_OK;
  DeviceGuard dg(h->device);
  if (h->ssf_fft.have_plans && h->ssf_ncomp != h->m.ncomp) fft_pair_release(h->ssf_fft);
  const char* msg = fft_pair_setup(h->ssf_fft, h->geo, h->m.ncomp, h->m.precision);
  if (msg) return fail(h, PHX_ECUDA, msg);
  h->ssf_ncomp = h->m.ncomp;
  if (!h->imag_red) PHX_CK(h, cudaMalloc(&h->imag_red, imag_scratch_doubles() * sizeof(double)));
  msg = imag_steps(h->ssf_fft, h->imag_red, h->psi[h->cur], h->geo, h->m.precision,
                   h->has_V ? h->V : nullptr, h->p, nsteps, h->stream);
  if (msg) return fail(h, PHX_ECUDA, msg);
  PHX_CK(h, launch_fill_ghosts(h->psi[h->cur], (int)(2 * h->esize), h->m.ncomp, h->geo,
                               h->stream));
  return PHX_OK;
}

phx_status phx_set_kfilter(phx_handle* h, double k_cut, int32_t order, int64_t every) {
  if (!h) return fail(nullptr, PHX_EINVAL, "handle is NULL");
  if (every < 0) return fail(h, PHX_EINVAL, "every must be >= 0");
  DeviceGuard dg(h->device);
  if (every == 0) {
    h->kf.every = 0;
    return PHX_OK;
  }
  if (!(k_cut > 0) || !is_finite(k_cut)) return fail(h, PHX_EINVAL, "k_cut must be > 0 and finite");
  if (order < 1 || order > 16) return fail(h, PHX_EINVAL, "order must be in 1..16");
  const char* msg = kfilter_setup(h->kf, h->geo, h->m.ncomp, h->m.precision);
  if (msg) {
    h->kf.every = 0;
    return fail(h, PHX_ECUDA, msg);
  }
  h->kf.kc = k_cut;
  h->kf.order = order;
  h->kf.every = every;
  return PHX_OK;
}

phx_status phx_norm_energy(phx_handle* h, double* norm, double* energy) {
  if (!h) return fail(nullptr, PHX_EINVAL, "handle is NULL");
  DeviceGuard dg(h->device);
  ReduceArgs r = make_reduce_args(h);
  PHX_CK(h, launch_norm_energy(r, h->partials, h->red_dev, h->stream));
  PHX_CK(h, cudaMemcpyAsync(h->red_host, h->red_dev, 9 * sizeof(double),
                            cudaMemcpyDeviceToHost, h->stream));
  PHX_CK(h, cudaStreamSynchronize(h->stream));
  {
    phx_status es = took_device_error(h);
    if (es != PHX_OK) return es;
  }
  const double dV = (h->p.lx / h->p.nx) * (h->p.ly / h->p.ny);
  double N = dV * h->red_host[0], E = dV * h->red_host[1];
  if (norm) *norm = N;
  if (energy) *energy = E;
  if (!is_finite(N) || !is_finite(E)) return fail(h, PHX_ENONFINITE, "state holds NaN or Inf");
  return PHX_OK;
}

phx_status phx_residual(phx_handle* h, double* r_psi, double* r_n, double* omega) {
  if (!h) return fail(nullptr, PHX_EINVAL, "handle is NULL");
  DeviceGuard dg(h->device);
  ReduceArgs r = make_reduce_args(h);
  PHX_CK(h, launch_residual(r, h->partials, h->red_dev, h->stream));
  PHX_CK(h, cudaMemcpyAsync(h->red_host, h->red_dev, 9 * sizeof(double),
                            cudaMemcpyDeviceToHost, h->stream));
  PHX_CK(h, cudaStreamSynchronize(h->stream));
  {
    phx_status es = took_device_error(h);
    if (es != PHX_OK) return es;
  }
  const double* o = h->red_host;
  double rp = o[0] > 0.0 ? std::sqrt(o[5] / o[0]) : 0.0;
  double rn = 0.0;
  if (h->m.reservoir) rn = o[4] > 0.0 ? std::sqrt(o[3] / o[4]) : (o[3] == 0.0 ? 0.0 : INFINITY);
  if (r_psi) *r_psi = rp;
  if (r_n) *r_n = rn;
  if (omega) *omega = o[6];
  for (int q = 0; q < 7; ++q)
    if (!is_finite(o[q])) return fail(h, PHX_ENONFINITE, "state holds NaN or Inf");
  return PHX_OK;
}

phx_status phx_time(phx_handle* h, int64_t* step, double* t) {
  if (!h) return fail(nullptr, PHX_EINVAL, "handle is NULL");
  DeviceGuard dg(h->device);
  DevClock c;
  PHX_CK(h, cudaMemcpyAsync(&c, h->clock, sizeof c, cudaMemcpyDeviceToHost, h->stream));
  PHX_CK(h, cudaStreamSynchronize(h->stream));
  if (step) *step = c.step[h->parity];
  if (t) *t = c.t[h->parity];
  return PHX_OK;
}

phx_status phx_set_time(phx_handle* h, int64_t step, double t) {
  if (!h) return fail(nullptr, PHX_EINVAL, "handle is NULL");
  if (step < 0 || !is_finite(t)) return fail(h, PHX_EINVAL, "step must be >= 0 and t finite");
  DeviceGuard dg(h->device);
  DevClock c;
  c.step[0] = c.step[1] = step;
  c.t[0] = c.t[1] = t;
  PHX_CK(h, cudaMemcpyAsync(h->clock, &c, sizeof c, cudaMemcpyHostToDevice, h->stream));
  PHX_CK(h, cudaStreamSynchronize(h->stream));
  h->host_step = step;
  return PHX_OK;
}

phx_status phx_set_stream(phx_handle* h, void* stream) {
  if (!h) return fail(nullptr, PHX_EINVAL, "handle is NULL");
  h->stream = static_cast<cudaStream_t>(stream);
  h->p.stream = stream;
  return PHX_OK;
}

uint64_t phx_launch_count(void) { return phx::launch_total(); }

phx_status phx_debug_inject(uint32_t mask) {
  if (mask & ~7u) return fail(nullptr, PHX_EINVAL, "unknown injection bits");
  phx::arm_injection(mask);
  return PHX_OK;
}

int32_t phx_tile(const phx_handle* h) {
  if (!h) return 0;
  const bool drive_generic =
      h->has_E && (h->m.ncomp == 2 || (h->m.reservoir && !drive_reservoir_tile(h)));
  return (drive_generic && h->m.precision == 32) ? TILE_GENERIC : h->tile_cfg;
}

const char* phx_last_error(const phx_handle* h) {
  if (h) return h->err.c_str();
  return g_err.c_str();
}

const char* phx_status_string(phx_status s) {
  switch (s) {
    case PHX_OK: return "PHX_OK";
    case PHX_EINVAL: return "PHX_EINVAL";
    case PHX_ENOMEM: return "PHX_ENOMEM";
    case PHX_ECUDA: return "PHX_ECUDA";
    case PHX_ENONFINITE: return "PHX_ENONFINITE";
    case PHX_ETIMEOUT: return "PHX_ETIMEOUT";
    case PHX_ESTATE: return "PHX_ESTATE";
    case PHX_ENODEV: return "PHX_ENODEV";
  }
  return "PHX_UNKNOWN";
}

void phx_destroy(phx_handle* h) {
  if (!h) return;
  free_all(h);
  delete h;
}

phx_status phx_noise_sample(uint64_t seed, int64_t step, uint32_t instance,
                            int32_t ncomp, int32_t nx, int32_t ny,
                            double noise_var, float* out_device, void* stream) {
  if (!out_device) return fail(nullptr, PHX_EINVAL, "out_device is NULL");
  if (ncomp != 1 && ncomp != 2) return fail(nullptr, PHX_EINVAL, "ncomp must be 1 or 2");
  if (nx < 1 || ny < 1 || (long long)nx * ny > (1ll << 31) - 1)
    return fail(nullptr, PHX_EINVAL, "bad nx, ny");
  if (!(noise_var >= 0) || !is_finite(noise_var)) return fail(nullptr, PHX_EINVAL, "bad noise_var");
  float scale = (float)std::sqrt(noise_var / 2.0);
  cudaError_t e = launch_noise_sample(seed, step, instance, ncomp, nx, ny, scale,
                                      out_device, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "noise sample launch");
  return PHX_OK;
}

}  // extern "C"
