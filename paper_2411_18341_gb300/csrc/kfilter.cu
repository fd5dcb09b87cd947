// k-space smoothing of psi (Sec. III.B): a forward FFT of each component,
// the product with a low-pass mask, and the inverse FFT back into the padded
// state, whose ghost ring is then refilled.  The paper leaves the mask's
// shape open; this library uses the super-Gaussian
//   M(k) = exp(-((k_x^2 + k_y^2) / k_c^2)^p),  k = 2 pi m / L (FFT order),
// with the 1/(nx ny) normalisation of the inverse transform folded in.
//
// The transforms are cuFFT library calls.  cuFFT is loaded with dlopen at
// the first use, so the library itself does not depend on it: a process
// without cuFFT gets PHX_ECUDA from phx_set_kfilter and nothing else changes.
#include <dlfcn.h>
#include <cufft.h>

#include "kfilter.h"

namespace phx {

namespace {

struct FftApi {
  decltype(&cufftPlanMany) plan_many = nullptr;
  decltype(&cufftExecC2C) exec_c2c = nullptr;
  decltype(&cufftExecZ2Z) exec_z2z = nullptr;
  decltype(&cufftSetStream) set_stream = nullptr;
  decltype(&cufftDestroy) destroy = nullptr;
  bool ok = false;
};

const FftApi& fft_api() {
  static FftApi api = [] {
    FftApi a;
    const char* names[] = {"libcufft.so.12", "libcufft.so"};
    void* lib = nullptr;
    for (const char* n : names)
      if ((lib = dlopen(n, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
    if (!lib) return a;
    a.plan_many = reinterpret_cast<decltype(&cufftPlanMany)>(dlsym(lib, "cufftPlanMany"));
    a.exec_c2c = reinterpret_cast<decltype(&cufftExecC2C)>(dlsym(lib, "cufftExecC2C"));
    a.exec_z2z = reinterpret_cast<decltype(&cufftExecZ2Z)>(dlsym(lib, "cufftExecZ2Z"));
    a.set_stream = reinterpret_cast<decltype(&cufftSetStream)>(dlsym(lib, "cufftSetStream"));
    a.destroy = reinterpret_cast<decltype(&cufftDestroy)>(dlsym(lib, "cufftDestroy"));
    a.ok = a.plan_many && a.exec_c2c && a.exec_z2z && a.set_stream && a.destroy;
    return a;
  }();
  return api;
}

// Signed FFT index m of position i on an n-point axis (numpy fftfreq order).
__device__ __forceinline__ int fft_index(int i, int n) { return i <= (n - 1) / 2 ? i : i - n; }

template <typename R, typename C>
__global__ void kfilter_mask_kernel(C* d, int nx, int ny, int ncomp, R dkx, R dky, R inv_kc2,
                                    int order, R scale) {
  const long long total = (long long)nx * ny * ncomp;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long r = t % ((long long)nx * ny);
    const int j = (int)(r / nx), i = (int)(r - (long long)j * nx);
    const R kx = dkx * R(fft_index(i, nx)), ky = dky * R(fft_index(j, ny));
    const R q = (ky * ky + kx * kx) * inv_kc2;
    R qp = q;
    for (int o = 1; o < order; ++o) qp *= q;
    const R m = exp(-qp) * scale;
    C v = d[t];
    v.x *= m;
    v.y *= m;
    d[t] = v;
  }
}

}  // namespace

void fft_pair_release(FftPair& f) {
  const FftApi& api = fft_api();
  if (f.have_plans && api.ok) {
    api.destroy(f.plan_fwd);
    api.destroy(f.plan_inv);
  }
  f.have_plans = false;
  if (f.scratch) cudaFree(f.scratch);
  f.scratch = nullptr;
}

const char* fft_pair_setup(FftPair& f, const Geometry& g, int ncomp, int precision) {
  const FftApi& api = fft_api();
  if (!api.ok) return "cuFFT (libcufft.so.12) could not be loaded";
  if (f.have_plans) return nullptr;
  if (g.plane * ncomp >= (1ll << 31)) return "grid too large for the FFT plans";
  if (!f.scratch) {
    const size_t bytes = (size_t)g.nx * g.ny * ncomp * (precision == 64 ? 16 : 8);
    if (cudaMalloc(&f.scratch, bytes) != cudaSuccess) {
      cudaGetLastError();
      f.scratch = nullptr;
      return "cudaMalloc of the FFT scratch failed";
    }
  }
  int n[2] = {g.ny, g.nx};
  int padded[2] = {g.prow, g.pitch};
  int dense[2] = {g.ny, g.nx};
  const int plane = (int)g.plane, dplane = g.nx * g.ny;
  const cufftType ty = precision == 64 ? CUFFT_Z2Z : CUFFT_C2C;
  if (api.plan_many(&f.plan_fwd, 2, n, padded, 1, plane, dense, 1, dplane, ty, ncomp) !=
      CUFFT_SUCCESS)
    return "cufftPlanMany (forward) failed";
  if (api.plan_many(&f.plan_inv, 2, n, dense, 1, dplane, padded, 1, plane, ty, ncomp) !=
      CUFFT_SUCCESS) {
    api.destroy(f.plan_fwd);
    return "cufftPlanMany (inverse) failed";
  }
  f.have_plans = true;
  return nullptr;
}

const char* fft_transform(const FftPair& f, void* psi, const Geometry& g, int precision,
                          bool forward, cudaStream_t s) {
  const FftApi& api = fft_api();
  if (!f.have_plans) return "FFT plans not set up";
  const int plan = forward ? f.plan_fwd : f.plan_inv;
  if (api.set_stream(plan, s) != CUFFT_SUCCESS) return "cufftSetStream failed";
  const long long origin = (long long)HALO * g.pitch + HALO;
  cufftResult r;
  if (precision == 64) {
    auto* base = static_cast<cufftDoubleComplex*>(psi) + origin;
    auto* sc = static_cast<cufftDoubleComplex*>(f.scratch);
    r = forward ? api.exec_z2z(plan, base, sc, CUFFT_FORWARD)
                : api.exec_z2z(plan, sc, base, CUFFT_INVERSE);
  } else {
    auto* base = static_cast<cufftComplex*>(psi) + origin;
    auto* sc = static_cast<cufftComplex*>(f.scratch);
    r = forward ? api.exec_c2c(plan, base, sc, CUFFT_FORWARD)
                : api.exec_c2c(plan, sc, base, CUFFT_INVERSE);
  }
  return r == CUFFT_SUCCESS ? nullptr : "cuFFT execution failed";
}

void kfilter_release(KFilter& f) {
  fft_pair_release(f.fft);
  f.every = 0;
}

const char* kfilter_setup(KFilter& f, const Geometry& g, int ncomp, int precision) {
  return fft_pair_setup(f.fft, g, ncomp, precision);
}

const char* kfilter_apply(const KFilter& f, void* psi, const Geometry& g, int ncomp,
                          int precision, double lx, double ly, cudaStream_t s) {
  const char* msg = fft_transform(f.fft, psi, g, precision, true, s);
  if (msg) return msg;
  const double pi = 3.14159265358979323846;
  const long long total = (long long)g.nx * g.ny * ncomp;
  const int threads = 256;
  const long long want = (total + threads - 1) / threads;
  const int blocks = (int)(want < 4096 ? want : 4096);
  const double scale = 1.0 / ((double)g.nx * g.ny);
  const double inv_kc2 = 1.0 / (f.kc * f.kc);
  if (precision == 64)
    kfilter_mask_kernel<double, double2><<<blocks, threads, 0, s>>>(
        static_cast<double2*>(f.fft.scratch), g.nx, g.ny, ncomp, 2 * pi / lx, 2 * pi / ly,
        inv_kc2, f.order, scale);
  else
    kfilter_mask_kernel<float, float2><<<blocks, threads, 0, s>>>(
        static_cast<float2*>(f.fft.scratch), g.nx, g.ny, ncomp, (float)(2 * pi / lx),
        (float)(2 * pi / ly), (float)inv_kc2, f.order, (float)scale);
  count_launch();
  if (cudaGetLastError() != cudaSuccess) return "smoothing mask launch failed";
  msg = fft_transform(f.fft, psi, g, precision, false, s);
  if (msg) return msg;
  if (launch_fill_ghosts(psi, precision == 64 ? 16 : 8, ncomp, g, s) != cudaSuccess)
    return "ghost refill after smoothing failed";
  return nullptr;
}

}  // namespace phx
