/*
 * phx.h -- C ABI of the GB300 RK4 solver for the 2D driven-dissipative
 * Gross-Pitaevskii / dissipative nonlinear Schroedinger equation (dNLSE)
 * of PHOENIX (arXiv 2411.18341).
 *
 * What one step computes (all citations are to the paper):
 *   Eq. (PULSE_psi), Sec. V:
 *     dpsi_c/dt = -(i/hbar)[ -(hbar^2/2m) Lap psi_c + (V + g|psi_c|^2
 *                 + g_x|psi_o|^2 + g_r n_c) psi_c + J_c psi_o + E_c ]
 *                 + (1/2)(R n_c - gamma_c) psi_c  (+ dW)
 *     c in {+} (scalar, Eq. 1) or {+,-} (spinor), o = other component,
 *     J_+ = Delta_LT (d_x - i d_y)^2, J_- = Delta_LT (d_x + i d_y)^2,
 *     E_c(r, t) = E_c(r) exp(-i drive_omega t) the coherent drive (zero
 *     until phx_set_drive), t the handle's FP64 simulated time at the RK4
 *     stage (t, t + dt/2, t + dt/2, t + dt).
 *   Eq. (PULSE_res): dn_c/dt = P_c - (gamma_r + R|psi_c|^2) n_c.
 *   Lap: the 5-point central-difference stencil of Sec. III.B.6; the TE-TM
 *   operator uses 3-point second differences and the 4-corner mixed
 *   difference.  Time step: RK4, Eqs. (rk4_K1)-(rk4_final).  Boundary
 *   conditions: x and y independently periodic or zero (Sec. V).
 *   Noise dW: after each deterministic step psi_c += xi_c with xi a complex
 *   Gaussian of E|xi|^2 = noise_var from Philox4x32-10 keyed by
 *   (seed, step, instance, site) (Salmon et al., SC'11), so runs and
 *   resumes are reproducible bit for bit: key = seed, counter = (c, instance,
 *   step lo, step hi) with c = site for two components (words 0,1 -> xi_+,
 *   2,3 -> xi_-) and c = site >> 1 for one component (words 0,1 -> the even,
 *   2,3 -> the odd site of the pair); site = j*nx + i.
 *   Truncated-Wigner mode (Sec. V, Example 4; wigner_nu > 0): the variance
 *   becomes E|xi_c|^2 = noise_var + nu (R n_c + gamma_c) dt / (2 dV) per
 *   site, n_c taken at the start of the step and dV = dx dy, and the Kerr,
 *   cross-Kerr and depletion terms use the renormalised density
 *   |psi|^2 - 1/dV.  Norm, energy and residual stay the plain functionals.
 *
 * Conventions
 *   - Every call returns a phx_status; on error the handle's state is left
 *     as it was and phx_last_error() holds a message.
 *   - Arrays are row-major ny x nx with x fastest; site = j*nx + i.
 *     psi: ncomp planes of interleaved complex (re, im) values; n, P: ncomp
 *     planes of reals; V: one plane.  Element type is float for
 *     precision 32 and double for precision 64.
 *   - `on_device` = 1: the pointer is CUDA device memory of the handle's
 *     device; 0: host memory (pinned or pageable).  Inputs are copied;
 *     the caller keeps ownership of every pointer it passes.  A device
 *     input is read by work queued on params.stream: whatever writes it on
 *     another stream must be complete (or ordered before that stream) when
 *     the call is made.
 *   - Work is queued on params.stream (a cudaStream_t; NULL = legacy default
 *     stream).  Calls that return values to the host synchronise that stream.
 *   - A handle is not thread-safe; distinct handles are independent.
 */
#ifndef PHX_H
#define PHX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PHX_ABI_VERSION 2

typedef enum phx_status {
  PHX_OK = 0,
  PHX_EINVAL = 1,      /* bad argument (null pointer, size, dt above its limit, ...) */
  PHX_ENOMEM = 2,      /* device or host allocation failed */
  PHX_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
  PHX_ENONFINITE = 4,  /* a reduction found NaN or Inf in the state */
  PHX_ETIMEOUT = 5,    /* a bounded device-side wait gave up */
  PHX_ESTATE = 6,      /* call not valid in the handle's current state */
  PHX_ENODEV = 7       /* no CUDA device of compute capability 10.3 (GB300) */
} phx_status;

enum { PHX_BC_PERIODIC = 0, PHX_BC_ZERO = 1 };

/* Parameters of one problem instance (Eqs. PULSE_psi / PULSE_res).
 * Units: lengths um, energies meV, times ps. */
typedef struct phx_params {
  uint32_t struct_size;      /* = sizeof(phx_params); set by phx_params_init */
  int32_t nx, ny;            /* grid points, >= 1 each */
  double lx, ly;             /* domain lengths; dx = lx/nx, dy = ly/ny */
  int32_t bc_x, bc_y;        /* PHX_BC_PERIODIC or PHX_BC_ZERO */
  int32_t precision;         /* 32 or 64: stencil arithmetic and storage */
  int32_t spinor;            /* 0: scalar psi; 1: two components psi_+, psi_- */
  int32_t reservoir;         /* 0/1: evolve n_c with Eq. (PULSE_res) */
  int32_t tile;              /* FP32 scalar step kernel configuration:
                                0 = autotune (the first phx_step_n times each
                                configuration on the handle's own state, without
                                changing it, synchronising the stream once; the
                                choice is cached per grid shape), 1..7 = a fixed
                                shared-memory region and thread shape of the
                                TMA-fed persistent kernel, 8 = configuration 7
                                running up to 128 steps per launch (single
                                handles without drive), 9 = generic kernel;
                                for the generic kernels of the FP32 spinor +
                                reservoir + TE-TM and FP64 scalar reservoir
                                models 10..12 select other tile shapes */
  double hbar2_over_2m;      /* hbar^2/2m, meV um^2 */
  double g, g_x, g_r;        /* meV um^2 */
  double R;                  /* ps^-1 um^2 */
  double gamma_c, gamma_r;   /* ps^-1 */
  double delta_lt;           /* TE-TM splitting Delta_LT, meV um^2 (spinor only) */
  double dt;                 /* time step, ps; rejected above the integrator's limit */
  double noise_var;          /* E|xi|^2 added per site and step; 0 = off */
  double wigner_nu;          /* truncated-Wigner noise intensity nu >= 0; 0 = off */
  double drive_omega;        /* angular frequency of the coherent drive, rad/ps */
  uint64_t seed;             /* Philox key */
  uint32_t instance;         /* Philox counter word 1 (ensemble member id) */
  uint32_t integrator;       /* PHX_INTEGRATOR_RK4 (default): dt must lie within
                                phx_stability_dt; PHX_INTEGRATOR_SPLIT: the handle
                                is stepped by phx_step_ssf, whose linear part is
                                exact, and dt is validated against the split-step
                                scheme's own limit instead (see phx_create) */
  void* stream;              /* cudaStream_t */
} phx_params;

enum { PHX_INTEGRATOR_RK4 = 0, PHX_INTEGRATOR_SPLIT = 1 };

typedef struct phx_handle phx_handle;

/* Fill *p with defaults: 64x64, 1x1 um, periodic, fp32, scalar, no
 * reservoir, hbar^2/2m = 0.67, all other coefficients 0, stream NULL.
 * EINVAL if p is NULL. */
phx_status phx_params_init(phx_params* p);

/* Largest stable RK4 step for the linear Hermitian part of the equations
 * (stencil and TE-TM; nonlinear, potential and loss terms excluded):
 * dt_max = 2 sqrt(2) hbar / lambda_max, 2 sqrt(2) being the extent of the RK4
 * region on the imaginary axis (Eqs. rk4_K1-final).  Host-only; EINVAL on
 * bad parameters. */
phx_status phx_stability_dt(const phx_params* p, double* dt_max);

/* Validate p, allocate the device state on the current CUDA device and
 * zero it (psi = 0, n = 0, P = 0, V absent, step 0, t = 0).
 * EINVAL: bad sizes, BC, precision, spinor-only terms on a scalar problem,
 * dt <= 0, an unknown integrator, or a dt above the integrator's limit:
 *   PHX_INTEGRATOR_RK4   -- dt > phx_stability_dt;
 *   PHX_INTEGRATOR_SPLIT -- the split-step scheme (phx_step_ssf) propagates
 *     the linear part exactly, so the stencil's limit does not apply; the
 *     handle needs periodic boundaries and no truncated-Wigner noise, and with
 *     a reservoir the local half steps (one RK4 step of dt/2 of the local
 *     ODE) need dt/2 x gamma_r within RK4's real-axis extent (2.78).  The
 *     state-dependent local rates (Kerr phase, gain) are not checked.
 *     phx_step_n on such a handle returns ESTATE when dt exceeds
 *     phx_stability_dt.
 * ENODEV: no sm_103 (GB300) device.  ENOMEM / ECUDA on allocation failure.
 * *out is NULL on error. */
phx_status phx_create(const phx_params* p, phx_handle** out);

/* Bytes of the five state buffers a handle with parameters p holds, for
 * callers that own the device memory (a caching allocator, a memory pool):
 * sizes[0], sizes[1] = psi (two buffers, ncomp padded complex planes each),
 * sizes[2], sizes[3] = n, sizes[4] = P (0 without reservoir).  The padded
 * layout carries a ghost ring; use phx_set_state / phx_get_state to move
 * dense arrays in and out.  Host-only; EINVAL on bad parameters. */
phx_status phx_buffer_sizes(const phx_params* p, size_t sizes[5]);

/* As phx_create, but the state buffers are the caller's device memory:
 * buffers[i] of at least sizes[i] bytes (phx_buffer_sizes; entries of size 0
 * are ignored), 256-byte aligned, device memory of the current device.  The
 * handle zeroes them, uses them and never frees them: they must outlive it.
 * The potential, drive, FFT scratch and small work arrays are still
 * allocated by the handle.  EINVAL: a NULL, misaligned or non-device buffer;
 * otherwise as phx_create. */
phx_status phx_create_with_buffers(const phx_params* p, void* const buffers[5],
                                   phx_handle** out);

/* Copy the pump P_+ (and P_-; NULL means P_- = P_+) into the handle
 * (Eq. PULSE_res).  ESTATE if the handle has no reservoir. */
phx_status phx_set_pump(phx_handle* h, const void* P_plus, const void* P_minus,
                        int on_device);

/* Copy the external potential V (Eq. PULSE_psi); V = NULL removes it. */
phx_status phx_set_potential(phx_handle* h, const void* V, int on_device);

/* Copy the coherent drive amplitude E_+(r) (and E_-(r); NULL means
 * E_- = E_+), complex interleaved, meV, one ny x nx plane per component
 * (Eq. PULSE_psi, Sec. V); the step adds E_c(r) exp(-i drive_omega t) to the
 * bracket.  E_plus = NULL removes the drive.  With a drive set, the FP32 scalar
 * field keeps the TMA-fed kernel (with a reservoir: configurations 2, 3 and 4;
 * an autotuned handle is tuned again when a drive is set or removed, a fixed
 * tile without that variant steps on the generic kernel); FP32 fields with two
 * components step on the generic kernel (phx_tile reports 9).  The energy and
 * residual reductions stay those of the undriven equations. */
phx_status phx_set_drive(phx_handle* h, const void* E_plus, const void* E_minus,
                         int on_device);

/* nsteps steps of the split-step Fourier method instead of RK4 (the
 * conventional alternative the paper's conclusions name, without details):
 * Strang splitting psi <- L(dt/2) K(dt) L(dt/2) psi with the exact local
 * propagator L(tau) psi_c = psi_c e^{-gamma_c tau/2}
 * exp(-(i/hbar)(V tau + (g|psi_c|^2 + g_x|psi_o|^2) F)), F = (1 - e^{-gamma_c tau})/gamma_c
 * (tau without loss), and the exact spectral linear propagator
 * K(tau) = exp(-(i/hbar) kappa k^2 tau), k = 2 pi m / L, times, for two
 * components, the exponential of the TE-TM block [[0, a], [a*, 0]],
 * a = -Delta_LT (k_x - i k_y)^2 (cuFFT, loaded at the first call); then the
 * step's noise as in phx_step_n.  With a reservoir, each local half step
 * integrates psi and n together by one RK4 step of dt/2 (the local system
 * has no closed form) and the linear step acts on psi only.  Same dt, clock
 * and state as phx_step_n (the two may alternate).  ESTATE unless the
 * handle is periodic in x and y and has neither a drive nor truncated-Wigner
 * noise; ECUDA if cuFFT is missing. */
phx_status phx_step_ssf(phx_handle* h, int64_t nsteps);

/* (Time steps above the RK4 limit: create the handle with
 * integrator = PHX_INTEGRATOR_SPLIT.) */

/* nsteps imaginary-time steps (t -> -i tau in the conservative part of
 * Eq. PULSE_psi; the conclusions name the method without details), split
 * like phx_step_ssf: psi <- A B A psi with
 * A = exp(-(V + g|psi_c|^2 + g_x|psi_o|^2) dt/(2 hbar)) (densities frozen within
 * the factor) and B = exp(-H_k dt/hbar) in Fourier space (kappa k^2 and, for
 * two components, the TE-TM block), then psi rescaled to the norm it had
 * when the call began.  Converges to the ground state; loss, gain, drive and
 * noise take no part and the clock does not move.  ESTATE unless the handle has no
 * reservoir and is periodic in x and y; ECUDA if cuFFT is missing. */
phx_status phx_step_imag(phx_handle* h, int64_t nsteps);

/* k-space smoothing (Sec. III.B): after every `every`-th step (after the step
 * whose index k, counted as phx_time counts steps, has (k + 1) % every == 0)
 * each component of psi is Fourier transformed, multiplied by the low-pass
 * mask M(k) = exp(-((k_x^2 + k_y^2) / k_cut^2)^order), k = 2 pi m / L with m the
 * FFT index, and transformed back (cuFFT, loaded at the first call).  The
 * paper does not give the mask; this super-Gaussian is this library's.
 * It follows phx_step_n's steps (not phx_step_ssf / phx_step_imag).
 * every = 0 turns smoothing off (k_cut, order ignored).  EINVAL: every < 0,
 * k_cut <= 0 or not finite, order outside 1..16.  ECUDA: cuFFT missing or its
 * plans failed. */
phx_status phx_set_kfilter(phx_handle* h, double k_cut, int32_t order, int64_t every);

/* Copy psi (ncomp planes of complex) and n (ncomp planes; ignored / may be
 * NULL without a reservoir, NULL with a reservoir keeps n) into the handle.
 * psi may be NULL to keep psi. */
phx_status phx_set_state(phx_handle* h, const void* psi, const void* n,
                         int on_device);

/* Copy the current psi and n (either may be NULL) out of the handle;
 * synchronises the stream. */
phx_status phx_get_state(phx_handle* h, void* psi, void* n, int on_device);

/* Queue nsteps >= 0 RK4 steps (Eqs. rk4_K1-final, plus noise when
 * noise_var > 0).  Asynchronous on the stream (except the one-time autotune
 * of tile = 0, see phx_params); advances the step counter and the FP64
 * simulated time t += dt on the device. */
phx_status phx_step_n(phx_handle* h, int64_t nsteps);

/* FP64 norm N = dx dy sum_c |psi_c|^2 and energy
 * E = dx dy sum [ sum_c ( Re psi_c^*(-hbar^2/2m Lap psi_c)
 *     + (V + g_r n_c)|psi_c|^2 + (g/2)|psi_c|^4 ) + g_x|psi_+|^2|psi_-|^2
 *     + Re(psi_+^* J_+ psi_- + psi_-^* J_- psi_+) ],
 * the functional whose derivative dE/dpsi_c^* is the bracket of
 * Eq. (PULSE_psi).  Synchronises; ENONFINITE if the state holds NaN/Inf. */
phx_status phx_norm_energy(phx_handle* h, double* norm, double* energy);

/* Steady-state residual in FP64: K = dpsi/dt of Eq. (PULSE_psi) without
 * noise, omega = -Im<psi,K>/||psi||^2, r_psi = ||K + i omega psi||/||psi||
 * (ps^-1; the global phase rotation of a stationary condensate removed),
 * r_n = ||dn/dt|| / ||n|| (0 without a reservoir).  Any output pointer may be
 * NULL.  Synchronises; ENONFINITE on NaN/Inf. */
phx_status phx_residual(phx_handle* h, double* r_psi, double* r_n,
                        double* omega);

/* Step counter and FP64 simulated time (t accumulated on the device). */
phx_status phx_time(phx_handle* h, int64_t* step, double* t);

/* Overwrite the step counter and time (checkpoint restore). */
phx_status phx_set_time(phx_handle* h, int64_t step, double t);

/* Replace the stream used by later calls. */
phx_status phx_set_stream(phx_handle* h, void* stream);

/* Step-kernel configuration in use (see phx_params.tile; after autotuning,
 * the configuration it chose; 9 = generic kernel), or 0 for NULL. */
int32_t phx_tile(const phx_handle* h);

/* Number of kernels this library has launched in the process so far. */
uint64_t phx_launch_count(void);

/* Measured non-tensor FMA throughput of the current device (no counterpart in
 * the paper; the denominator of the arithmetic roofline of the FP64 step):
 * a kernel of independent fused multiply-add chains in `precision` (32 or
 * 64), 8 CTAs of 256 threads per SM, timed with CUDA events on the legacy
 * default stream after one warm-up launch; *tflops = 2 x FMAs / time, in
 * TFLOP/s.  Allocates and frees a small output buffer; synchronises.
 * Changes no device setting.  EINVAL (bad precision, NULL), ENODEV, ENOMEM,
 * ECUDA. */
phx_status phx_alu_peak_probe(int32_t precision, double* tflops);

/* Failure-injection hook for tests (no counterpart in the paper).  Arms, for
 * the next matching event in this process, one of:
 *   PHX_INJECT_ALLOC   -- the next device allocation in phx_create fails
 *                         (phx_create returns PHX_ENOMEM, nothing leaks);
 *   PHX_INJECT_LAUNCH  -- the next step launch reports failure (PHX_ECUDA);
 *   PHX_INJECT_TIMEOUT -- the next launch of the TMA-fed FP32 step kernel
 *                         leaves its first tile's mbarrier unarmed, so the
 *                         kernel's bounded wait (~0.25 s) gives up, it sets
 *                         the handle's device error word and returns; the
 *                         next synchronising call returns PHX_ETIMEOUT and
 *                         the handle stays usable (state must be reset).
 * No hook faults, traps or hangs the GPU.  EINVAL on unknown bits. */
enum { PHX_INJECT_ALLOC = 1, PHX_INJECT_LAUNCH = 2, PHX_INJECT_TIMEOUT = 4 };
phx_status phx_debug_inject(uint32_t mask);

/* Message of the last error on h (h = NULL: last error of a call without a
 * handle on this thread).  Never NULL. */
const char* phx_last_error(const phx_handle* h);

/* Static name of a status code. */
const char* phx_status_string(phx_status s);

/* Free the handle and its device memory.  NULL-safe. */
void phx_destroy(phx_handle* h);

/* ---- batches: many independent instances, one launch per RK4 step -------
 *
 * A batch holds `count` independent FP32 scalar problems (Eq. 1 /
 * Eq. PULSE_psi with one component; all with or all without reservoir),
 * each with its own grid size, domain, coefficients, dt, seed and instance
 * id.  phx_batch_step_n advances every member by the same number of RK4
 * steps: each step is ONE persistent kernel launch over the tiles of all
 * members (a per-tile instance table), replayed from a CUDA graph, with the
 * tile configuration picked by an autotuner on the first call (which
 * synchronises the stream once) unless params[0].tile names one of the
 * TMA-fed configurations 1..7.  Members are addressed by index 0..count-1;
 * their arrays follow the single-handle conventions above.  params[0].stream
 * is used for all work.  Member i's FP64 simulated time is t0_i + steps*dt_i
 * accumulated on the device. */
typedef struct phx_batch phx_batch;

/* EINVAL: count < 1, any invalid member (see phx_create), precision != 32,
 * spinor != 0, mixed reservoir flags, or a grid smaller than 8 x 8. */
phx_status phx_batch_create(const phx_params* params, int32_t count, phx_batch** out);
phx_status phx_batch_set_pump(phx_batch* b, int32_t i, const void* P, int on_device);
/* V = NULL removes the member's potential; stepping requires that either all
 * members or none have a potential (ESTATE otherwise). */
phx_status phx_batch_set_potential(phx_batch* b, int32_t i, const void* V, int on_device);
/* Copy member i's coherent drive amplitude E(r) (complex interleaved, meV,
 * one ny_i x nx_i plane; Eq. PULSE_psi, Sec. V): the member's step adds
 * E(r) exp(-i drive_omega_i t_i) to the bracket, with its own frequency
 * params[i].drive_omega and its own FP64 time.  Once any member has a drive,
 * every member steps on the drive variant (members without one add a zero
 * plane; the result equals the undriven step).  E = NULL sets member i's
 * drive to zero.  With a reservoir the tile configuration is 2, 3 or 4
 * (autotuned among them; a batch created with another fixed configuration
 * gets EINVAL from phx_batch_step_n).  The drive planes (8 bytes per site of
 * every member) are allocated on the first call. */
phx_status phx_batch_set_drive(phx_batch* b, int32_t i, const void* E, int on_device);
phx_status phx_batch_set_state(phx_batch* b, int32_t i, const void* psi, const void* n,
                               int on_device);
phx_status phx_batch_get_state(phx_batch* b, int32_t i, void* psi, void* n, int on_device);
phx_status phx_batch_step_n(phx_batch* b, int64_t nsteps);
/* Per-member FP64 norm and energy (arrays of count doubles; either may be
 * NULL), same definitions as phx_norm_energy.  Synchronises.  Every member's
 * values are written before PHX_ENONFINITE reports that some member's state
 * holds NaN or Inf (that member's values are then non-finite). */
phx_status phx_batch_norm_energy(phx_batch* b, double* norms, double* energies);
/* Per-member steady-state residuals (arrays of count; any may be NULL);
 * PHX_ENONFINITE as for phx_batch_norm_energy. */
phx_status phx_batch_residual(phx_batch* b, double* r_psi, double* r_n, double* omega);
/* Common step counter and per-member FP64 times (t: count doubles or NULL). */
phx_status phx_batch_time(phx_batch* b, int64_t* step, double* t);
/* Tile configuration in use (0 until the first step), see phx_params.tile. */
int32_t phx_batch_tile(const phx_batch* b);
const char* phx_batch_last_error(const phx_batch* b);
void phx_batch_destroy(phx_batch* b);

/* Generate the noise field xi_c(seed, step, instance, site) that a step
 * with these keys adds, as float32 (re, im) pairs in out_device
 * [ncomp][ny][nx][2] (device memory, caller-owned).  Asynchronous on stream.
 * Lets callers and tests inspect the exact bits the step kernel adds. */
phx_status phx_noise_sample(uint64_t seed, int64_t step, uint32_t instance,
                            int32_t ncomp, int32_t nx, int32_t ny,
                            double noise_var, float* out_device, void* stream);

/* Allocation-free norm and energy (no counterpart in the paper; this is a
 * library convenience).  Computes exactly the quantities of phx_norm_energy
 * -- FP64 N and E, same boundary handling -- from caller-owned device arrays
 * in the plain layout of phx_set_state (psi: ncomp planes of ny x nx complex;
 * n: ncomp planes, required when p->reservoir, else ignored; V: one plane or
 * NULL), in p->precision, on p->stream, without creating a handle.
 *
 * It is meant for callers that may not allocate device memory: code whose
 * device memory is entirely owned by another allocator (a framework's
 * caching pool under a hard budget) or latency-critical loops that must not
 * call cudaMalloc/cudaFree, which can block on the device.  It calls no
 * allocation routine: its scratch (per-CTA FP64 partials and the two final
 * sums) is a fixed file-scope device array of 64 KiB + 16 B, resident on
 * every device that loads this library until the process exits.  Grids with
 * nx*ny > 16777216 (2^24) do not fit that scratch and return PHX_EINVAL.
 *
 * The first call on a device looks up the array's device address (once per
 * device, with that device current; a look-up that failed is tried again by
 * the next call); make that first call before any stream capture.  The
 * address is kept for the life of the process: after cudaDeviceReset of a
 * device this entry point must not be called on that device again (the kept
 * address would be stale).  All calls on a device share the array and leave their partials
 * in it; each call writes every slot it reads, so nothing needs clearing,
 * but calls whose kernels can overlap on the GPU (unordered streams) race.
 * Synchronises p->stream.  Errors (status only; no message is recorded,
 * since storing one could allocate): EINVAL (NULL psi, bad sizes or
 * boundary codes, grid too large, reservoir without n), ENODEV, ECUDA,
 * ENONFINITE. */
phx_status phx_norm_energy_static(const phx_params* p, const void* psi,
                                  const void* n, const void* V, double* norm,
                                  double* energy);

/* ---------------------------------------------------------------------
 * Learned warm start: Fourier neural operator (Li et al., "Fourier Neural
 * Operator for Parametric Partial Differential Equations", 2020) mapping a
 * pump image to an approximate steady state (psi, n), used as the initial
 * condition of the RK4 relaxation.  The paper has no such component; it is
 * an extension of its steady-state workflow (time evolution until the
 * state stops changing, Sec. V).
 *
 *   v0 = a W_lift + b_lift;  v_{l+1} = sigma(K_l v_l + v_l W_l + b_l)
 *   (no sigma after the last layer);  u = sigma(v_L Q1 + q1) Q2 + q2;
 *   K v = irfft2(R . rfft2(v)) on kx in [0, modes_x), ky in
 *   [0, modes_y/2) U [height - modes_y/2, height); sigma = exact GELU;
 *   loss = mean of (u - target)^2 over all output elements.
 *
 * Tensors are channels-last FP32 [batch][height][width][channels] in
 * device memory (caller-owned).  The flat FP32 parameter vector is, in
 * order: W_lift [in, C], b_lift [C]; per layer Rr [modes_y][modes_x][C][C],
 * Ri (same), W [C][C], b [C]; Q1 [C][P], q1 [P], Q2 [P][out], q2 [out]
 * (mode row my < modes_y/2 is ky = my, else ky = height - modes_y + my).
 * Every contraction runs on the tensor cores with BF16 operands and FP32
 * accumulation; activations and parameters are stored in FP32.  Work is
 * queued on config.stream; calls returning host values synchronise it.
 * Errors: EINVAL (NULL pointer, bad configuration, batch outside
 * [1, max_batch]), ENOMEM, ECUDA; message in phx_fno_last_error.
 * --------------------------------------------------------------------- */
typedef struct phx_fno_config {
  uint32_t struct_size;      /* = sizeof(phx_fno_config); set by phx_fno_config_init */
  int32_t height, width;     /* grid (H rows = y, W columns = x) */
  int32_t channels;          /* C, hidden width (<= 256) */
  int32_t layers;            /* spectral layers, 1..8 */
  int32_t modes_x;           /* kept kx modes, <= width/2 */
  int32_t modes_y;           /* kept ky modes (even, <= height), half low and half high */
  int32_t in_channels, out_channels, proj_hidden;  /* out, P <= 256 */
  int32_t max_batch;         /* activations are allocated for this many samples */
  void* stream;              /* cudaStream_t */
} phx_fno_config;

typedef struct phx_fno phx_fno;

/* Defaults: 256 x 256, C = 32, 4 layers, 16 x 32 modes, 3 -> 3 channels,
 * P = 64, max_batch 8, stream NULL. */
phx_status phx_fno_config_init(phx_fno_config* c);
/* Allocates parameters (uninitialised until phx_fno_set_params), Adam
 * moments, DFT tables and activations for max_batch samples. */
phx_status phx_fno_create(const phx_fno_config* c, phx_fno** out);
int64_t phx_fno_num_params(const phx_fno* f);
/* Algorithmic GEMM work issued on f since its creation: the sum over every
 * product of 2 M N K flops (forward, backward and weight-gradient GEMMs,
 * counted when queued), for throughput against the tensor-core roofline.
 * EINVAL if f or flops is NULL. */
phx_status phx_fno_gemm_flops(const phx_fno* f, double* flops);
/* Copies the flat parameters in and resets the Adam moments and step. */
phx_status phx_fno_set_params(phx_fno* f, const float* w, int on_device);
phx_status phx_fno_get_params(phx_fno* f, float* w, int on_device);
/* out [batch][H][W][out] = u(in [batch][H][W][in]); asynchronous. */
phx_status phx_fno_forward(phx_fno* f, const float* in, float* out, int32_t batch);
/* loss (host, may be NULL) and, when grad != NULL, the gradient with
 * respect to the flat parameters into grad (device, num_params floats).
 * Deterministic: fixed-order reductions, no atomics. */
phx_status phx_fno_loss_grad(phx_fno* f, const float* in, const float* target,
                             int32_t batch, double* loss, float* grad);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on the
 * mini-batch; loss (before the update) returned when non-NULL. */
phx_status phx_fno_train_step(phx_fno* f, const float* in, const float* target,
                              int32_t batch, float lr, double* loss);
const char* phx_fno_last_error(const phx_fno* f);
void phx_fno_destroy(phx_fno* f);

/* Network input and output maps (device arrays, caller-owned, asynchronous
 * on `stream`; messages in phx_fno_last_error(NULL)).
 * phx_fno_features: P [batch][height][width] -> out [batch][height][width][3]
 *   = (P / p_thr, x / (lx/2), y / (ly/2)), cell positions -l/2 + i l/n.
 * phx_fno_targets: psi [batch][height][width] complex (re, im) and n (same
 *   shape) -> out [..][3] = (Re, Im of psi e^{-i arg sum psi}) / scale_psi,
 *   n / scale_n: the global phase of a stationary state is arbitrary, so the
 *   target fixes it (sum in FP64, fixed order; batch <= 65535).
 * phx_fno_to_state: u [..][3] -> psi = (u0 + i u1) scale_psi,
 *   n = max(u2, 0) scale_n (n may be NULL). */
phx_status phx_fno_features(const float* P, int32_t batch, int32_t height, int32_t width,
                            double lx, double ly, double p_thr, float* out, void* stream);
phx_status phx_fno_targets(const float* psi, const float* n, int32_t batch, int32_t height,
                           int32_t width, double scale_psi, double scale_n, float* out,
                           void* stream);
phx_status phx_fno_to_state(const float* u, int32_t batch, int32_t height, int32_t width,
                            double scale_psi, double scale_n, float* psi, float* n,
                            void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PHX_H */
