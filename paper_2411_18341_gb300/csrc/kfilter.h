// k-space smoothing of the state (Sec. III.B) and the FFT pair it shares
// with the split-step Fourier integrator; see kfilter.cu.
#pragma once

#include "phx_internal.h"

namespace phx {

// cuFFT plans between the padded state (ncomp planes, interior only) and a
// dense scratch of ncomp n_x x n_y complex planes.
struct FftPair {
  int plan_fwd = 0, plan_inv = 0;
  bool have_plans = false;
  void* scratch = nullptr;
};

// nullptr on success, else a message.
const char* fft_pair_setup(FftPair& f, const Geometry& g, int ncomp, int precision);
// forward: padded interior -> scratch; else scratch -> padded interior
// (unnormalised, ghost ring untouched).
const char* fft_transform(const FftPair& f, void* psi, const Geometry& g, int precision,
                          bool forward, cudaStream_t s);
void fft_pair_release(FftPair& f);

struct KFilter {
  double kc = 0.0;        // cutoff k_c, 1/um
  int order = 1;          // super-Gaussian order p
  long long every = 0;    // smoothing after every this many steps; 0 = off
  FftPair fft;
};

// setup creates the plans and the scratch for the handle's geometry (once);
// apply smooths the ncomp planes of the padded state psi in place on stream
// s and refills its ghost ring.
const char* kfilter_setup(KFilter& f, const Geometry& g, int ncomp, int precision);
const char* kfilter_apply(const KFilter& f, void* psi, const Geometry& g, int ncomp,
                          int precision, double lx, double ly, cudaStream_t s);
void kfilter_release(KFilter& f);

}  // namespace phx
