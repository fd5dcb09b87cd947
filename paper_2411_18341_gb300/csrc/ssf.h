// Split-step Fourier integrator for a scalar field without reservoir; see ssf.cu.
#pragma once

#include <cmath>

#include "kfilter.h"
#include "phx_internal.h"

namespace phx {

// Host-computed coefficients of one Strang step (FP64; cast per precision).
struct SsfCoeffs {
  double gF_half;     // g F(dt/2) / hbar
  double gxF_half;    // g_x F(dt/2) / hbar (two components)
  double tau_half_h;  // (dt/2) / hbar, multiplies V
  double damp_half;   // exp(-gamma_c dt/4)
  double dkx, dky;    // 2 pi / L
  double kin;         // kappa dt / hbar
  double tetm;        // Delta_LT dt / hbar (two components)
  double scale;       // 1 / (nx ny), the inverse transform's normalisation
  double dt;
};

SsfCoeffs ssf_coeffs(const phx_params& p);

// One step on the padded state psi (ncomp planes; interior only, the ghost
// ring is left stale),
// queued on stream s.  nullptr on success, else a message.
const char* ssf_step(FftPair& fft, void* psi, const Geometry& g, int precision, int ncomp,
                     const void* V, const SsfCoeffs& k, const NoiseKey& nz, DevClock* clock,
                     int parity, cudaStream_t s);

// One step of the reservoir model: the local half steps integrate psi and n
// together (one RK4 step of dt/2 each), the linear step acts on psi.
const char* ssf_step_reservoir(FftPair& fft, void* psi, void* n, const void* P,
                               long long P_stride, const Geometry& g, int precision, int ncomp,
                               const void* V, const phx_params& p, const SsfCoeffs& k,
                               const NoiseKey& nz, DevClock* clock, int parity, cudaStream_t s);

// Imaginary-time split-step steps with the norm kept at its value at the
// start (the ground state of the conservative scalar Hamiltonian); red is
// device scratch of imag_scratch_doubles() doubles.  The clock does not move.
size_t imag_scratch_doubles();
const char* imag_steps(FftPair& fft, double* red, void* psi, const Geometry& g, int precision,
                       const void* V, const phx_params& p, long long nsteps, cudaStream_t s);

}  // namespace phx
