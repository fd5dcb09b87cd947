// Non-tensor arithmetic peak of the current device, measured: a kernel of
// independent FMA chains (FP64 or FP32) timed with CUDA events.  The step
// kernels are bound by HBM bandwidth (FP32) or by the FP64 pipe (FP64); this
// probe gives the second roofline's denominator as a measured number rather
// than one derived from unit counts and clocks.
#include <cuda_runtime.h>

#include "../../include/phx.h"
#include "phx_internal.h"

namespace phx {
namespace {

constexpr int PR_THREADS = 256;
constexpr int PR_CHAINS = 8;    // independent FMA chains per thread
constexpr int PR_UNROLL = 64;   // FMAs per chain per loop iteration

// Each thread runs PR_CHAINS independent chains x = x * a + b; the result is
// written once (so the chains are not removed) to out[thread].
template <typename T>
__global__ void __launch_bounds__(PR_THREADS) fma_chains_kernel(T a, T b, int iters, T* out) {
  T x[PR_CHAINS];
#pragma unroll
  for (int c = 0; c < PR_CHAINS; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < PR_UNROLL; ++k) {
#pragma unroll
      for (int c = 0; c < PR_CHAINS; ++c) x[c] = fma(x[c], a, b);
    }
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < PR_CHAINS; ++c) s += x[c];
  out[blockIdx.x * (long long)blockDim.x + threadIdx.x] = s;
}

template <typename T>
cudaError_t run_probe(int iters, int blocks, T* out, cudaStream_t s, float* ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  // a is just below 1 and b small, so no chain overflows or underflows
  fma_chains_kernel<T><<<blocks, PR_THREADS, 0, s>>>((T)0.999999, (T)1e-7, iters / 4, out);
  count_launch();
  e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) {
    fma_chains_kernel<T><<<blocks, PR_THREADS, 0, s>>>((T)0.999999, (T)1e-7, iters, out);
    count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

}  // namespace
}  // namespace phx

using namespace phx;

extern "C" phx_status phx_alu_peak_probe(int32_t precision, double* tflops) {
  if (!tflops || (precision != 32 && precision != 64)) return PHX_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PHX_ENODEV;
  const int blocks = sms * 8;  // 8 resident CTAs of 256 threads per SM
  const int iters = precision == 64 ? 64 : 2048;  // a few ms either way
  void* out = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * PR_THREADS * 8) != cudaSuccess) return PHX_ENOMEM;
  float ms = 0.f;
  cudaError_t e = precision == 64
                      ? run_probe<double>(iters, blocks, static_cast<double*>(out), 0, &ms)
                      : run_probe<float>(iters, blocks, static_cast<float*>(out), 0, &ms);
  cudaFree(out);
  if (e != cudaSuccess || ms <= 0.f) {
    cudaGetLastError();
    return PHX_ECUDA;
  }
  const double flops =
      2.0 * (double)blocks * PR_THREADS * PR_CHAINS * PR_UNROLL * (double)iters;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return PHX_OK;
}
