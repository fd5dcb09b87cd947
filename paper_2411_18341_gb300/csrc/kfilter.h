// k-space smoothing of the state (Sec. III.B); see kfilter.cu.
#pragma once

#include "phx_internal.h"

namespace phx {

struct KFilter {
  double kc = 0.0;        // cutoff k_c, 1/um
  int order = 1;          // super-Gaussian order p
  long long every = 0;    // smoothing after every this many steps; 0 = off
  int plan_fwd = 0, plan_inv = 0;  // cuFFT plans (padded -> dense, dense -> padded)
  bool have_plans = false;
  void* scratch = nullptr;  // ncomp dense complex planes
};

// nullptr on success, else a message.  setup (re)creates the plans and the
// scratch for the handle's geometry; apply smooths the ncomp planes of the
// padded state psi in place on stream s.
const char* kfilter_setup(KFilter& f, const Geometry& g, int ncomp, int precision);
const char* kfilter_apply(const KFilter& f, void* psi, const Geometry& g, int ncomp,
                          int precision, double lx, double ly, cudaStream_t s);
void kfilter_release(KFilter& f);

}  // namespace phx
