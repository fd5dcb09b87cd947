// Fourier neural operator (Li et al., 2020) for the learned warm start:
// forward, backward and Adam on the GPU.  Every contraction -- the pointwise
// lifting / projection / 1x1 layers, the truncated DFTs along x and y (dense
// cos / sin tables) and the per-mode complex channel mixing -- is a batched,
// strided GEMM on the tensor cores (BF16 operands, FP32 accumulation,
// mma.sync m16n8k16); tensors live in FP32 (channels-last [B, H, W, C]) and
// are rounded to BF16 when a GEMM tile is staged in shared memory.
//
// Parameter layout (flat FP32), shared with the host-side reference:
//   W_lift [Cin, C], b_lift [C],
//   per layer: Rr [MY, MX, C, C], Ri [MY, MX, C, C], W [C, C], b [C],
//   Q1 [C, P], q1 [P], Q2 [P, Cout], q2 [Cout].
// Spectral layer: K(v) = irfft2(R . rfft2(v)) on kx in [0, MX), ky in
// [0, MY/2) U [H - MY/2, H); sigma = exact GELU; loss = mean squared error.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/phx.h"
#include "phx_internal.h"

namespace phx {
namespace {

// ------------------------------------------------------------------ GEMM
struct GemmDesc {
  int M, N, K;
  int K_last;    // K of the last batch entry (split-K tail); = K otherwise
  int nb1, nb2;  // batch = nb1 x nb2
  const float* A;
  long long a_m, a_k, a_b1, a_b2;
  const float* B;
  long long b_k, b_n, b_b1, b_b2;
  float* C;
  long long c_m, c_n, c_b1, c_b2;
  float alpha, beta;
};

constexpr int GM = 64, GN = 64, GK = 32;
constexpr int GT = 128;  // 4 warps, each a 32 x 32 sub-tile

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7},"
      " {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[b] = alpha * A[b] B[b] + beta * C[b] for one 64 x 64 output tile.
// Shared memory holds the A tile row-major [m][k] and the B tile as [n][k],
// both BF16, so each fragment register is one 32-bit shared load.
__global__ void __launch_bounds__(GT) gemm_bf16_kernel(const GemmDesc d) {
  __shared__ __align__(16) __nv_bfloat16 As[GM][GK + 8];
  __shared__ __align__(16) __nv_bfloat16 Bs[GN][GK + 8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m0 = blockIdx.x * GM, n0 = blockIdx.y * GN;
  const int bz = blockIdx.z, b1 = bz / d.nb2, b2 = bz - b1 * d.nb2;
  const int K = bz == (int)gridDim.z - 1 ? d.K_last : d.K;
  const float* A = d.A + b1 * d.a_b1 + b2 * d.a_b2;
  const float* B = d.B + b1 * d.b_b1 + b2 * d.b_b2;
  float* C = d.C + b1 * d.c_b1 + b2 * d.c_b2;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int gid = lane >> 2, tig = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

  for (int k0 = 0; k0 < K; k0 += GK) {
    // stage the tiles (zero outside the matrices), rounding to BF16
    for (int e = tid; e < GM * GK; e += GT) {
      int mm, kk;
      if (d.a_k == 1) {  // consecutive threads walk k
        mm = e / GK;
        kk = e - mm * GK;
      } else {           // consecutive threads walk m
        kk = e / GM;
        mm = e - kk * GM;
      }
      const int m = m0 + mm, k = k0 + kk;
      const float v = (m < d.M && k < K) ? A[m * d.a_m + k * d.a_k] : 0.f;
      As[mm][kk] = __float2bfloat16_rn(v);
    }
    for (int e = tid; e < GN * GK; e += GT) {
      int nn, kk;
      if (d.b_n == 1) {
        kk = e / GN;
        nn = e - kk * GN;
      } else {
        nn = e / GK;
        kk = e - nn * GK;
      }
      const int n = n0 + nn, k = k0 + kk;
      const float v = (n < d.N && k < K) ? B[k * d.b_k + n * d.b_n] : 0.f;
      Bs[nn][kk] = __float2bfloat16_rn(v);
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < GK; ks += 16) {
      uint32_t af[2][4], bfr[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + i * 16 + gid;
        af[i][0] = *reinterpret_cast<const uint32_t*>(&As[r][ks + tig * 2]);
        af[i][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + tig * 2]);
        af[i][2] = *reinterpret_cast<const uint32_t*>(&As[r][ks + tig * 2 + 8]);
        af[i][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + tig * 2 + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = wn + j * 8 + gid;
        bfr[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[c][ks + tig * 2]);
        bfr[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[c][ks + tig * 2 + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j]);
    }
    __syncthreads();
  }
  // epilogue: fragment (row gid / gid+8, columns 2 tig, 2 tig + 1)
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int m = m0 + wm + i * 16 + gid + (r >= 2 ? 8 : 0);
        const int n = n0 + wn + j * 8 + tig * 2 + (r & 1);
        if (m < d.M && n < d.N) {
          float* p = C + m * d.c_m + n * d.c_n;
          const float v = d.alpha * acc[i][j][r];
          *p = d.beta == 0.f ? v : v + d.beta * *p;
        }
      }
}


// ------------------------------------------- tcgen05 GEMM (M-tile 128)
// C[b] = alpha * A[b] B[b] + beta * C[b] on the 5th-generation tensor cores:
// the CTA's 128 threads stage 128 x 64 tiles of A and BN x 64 tiles of B
// (FP32 from global, rounded to BF16) into shared memory in the canonical
// K-major layout without swizzle -- 8-row x 16-byte core matrices, core
// matrix (row group g, k group j) at (g * 8 + j) * 128 bytes, so the
// stride between k groups (LBO) is 128 B and between row groups (SBO)
// 1024 B -- and one elected thread issues four tcgen05.mma (K = 16 each)
// per stage into a 128 x BN FP32 accumulator in tensor memory; a
// tcgen05.commit on an mbarrier releases the stage's buffers.  Two stages
// alternate.  The epilogue reads the accumulator with tcgen05.ld (warp w
// owns TMEM lanes 32w..32w+31 = rows).  Waits are bounded; a CTA that gives
// up raises *err and skips its epilogue.
constexpr int TC_BM = 128, TC_BK = 64, TC_T = 128;

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  const uint64_t lbo = 128 >> 4, sbo = 1024 >> 4;
  return (uint64_t)((saddr >> 4) & 0x3FFF) | (lbo << 16) | (sbo << 32) | (1ull << 46);
}

__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity) {
#pragma unroll 1
  for (uint32_t it = 0; it < (1u << 24); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (it >= 16) __nanosleep(64);
  }
  return false;
}

// byte offset of element (row, k) of a tile in the canonical layout
__device__ __forceinline__ uint32_t tc_off(int row, int k) {
  return (uint32_t)((((row >> 3) << 3) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1);
}

__device__ __forceinline__ uint32_t pack_bf2(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

// Stage rows [r0, r0 + NR) x k [k0, k0 + 64) of a strided FP32 matrix
// (element (r, k) at src[r * s_row + k * s_k], zero outside nrows x K) as
// BF16 in the canonical layout.  One unit = (row, group of 8 k) = one
// 16-byte shared store; consecutive threads take consecutive rows, so each
// quarter-warp's eight stores fill all 32 banks of one core matrix.
template <int NR>
__device__ __forceinline__ void tc_stage(unsigned char* dst, const float* src, int nrows, int r0,
                                         long long s_row, long long s_k, int k0, int K, int tid) {
  constexpr int UNITS = NR * (TC_BK / 8);
  for (int u = tid; u < UNITS; u += TC_T) {
    const int kg = u / NR, row = u - kg * NR;
    const int r = r0 + row, k = k0 + kg * 8;
    float v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = 0.f;
    if (r < nrows && k < K) {
      const float* p = src + r * s_row + (long long)k * s_k;
      if (s_k == 1 && k + 8 <= K && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
        const float4 x = *reinterpret_cast<const float4*>(p);
        const float4 y = *reinterpret_cast<const float4*>(p + 4);
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
        v[4] = y.x; v[5] = y.y; v[6] = y.z; v[7] = y.w;
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (k + i < K) v[i] = p[(long long)i * s_k];
      }
    }
    uint4 q;
    q.x = pack_bf2(v[0], v[1]);
    q.y = pack_bf2(v[2], v[3]);
    q.z = pack_bf2(v[4], v[5]);
    q.w = pack_bf2(v[6], v[7]);
    *reinterpret_cast<uint4*>(dst + tc_off(row, kg * 8)) = q;
  }
}

template <int BN>
__global__ void __launch_bounds__(TC_T) gemm_tc_kernel(const GemmDesc d, int* err) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  constexpr int A_BYTES = TC_BM * TC_BK * 2, B_BYTES = BN * TC_BK * 2;
  auto sA = [&](int st) { return tc_smem + st * A_BYTES; };
  auto sB = [&](int st) { return tc_smem + 2 * A_BYTES + st * B_BYTES; };
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * TC_BM, n0 = blockIdx.y * BN;
  const int bz = blockIdx.z, b1 = bz / d.nb2, b2 = bz - b1 * d.nb2;
  const float* A = d.A + b1 * d.a_b1 + b2 * d.a_b2;
  const float* B = d.B + b1 * d.b_b1 + b2 * d.b_b2;
  float* C = d.C + b1 * d.c_b1 + b2 * d.c_b2;
  const int K = bz == (int)gridDim.z - 1 ? d.K_last : d.K;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&mbar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {  // accumulator: BN columns x 128 lanes of tensor memory
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&tmem_slot)),
                 "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  // instruction descriptor: F32 accumulator, BF16 A and B, both K-major,
  // N >> 3 at bit 17, M >> 4 at bit 24
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                         ((uint32_t)(TC_BM >> 4) << 24);

  const int nk = (K + TC_BK - 1) / TC_BK;
  bool ok = true;
  for (int kc = 0; kc < nk; ++kc) {
    const int st = kc & 1;
    if (kc >= 2 && ok) ok = tc_wait(&mbar[st], (uint32_t)(((kc - 2) >> 1) & 1));
    const int k0 = kc * TC_BK;
    tc_stage<TC_BM>(sA(st), A, d.M, m0, d.a_m, d.a_k, k0, K, tid);
    tc_stage<BN>(sB(st), B, d.N, n0, d.b_n, d.b_k, k0, K, tid);
    // generic-proxy shared stores -> visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0 && ok) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t da = tc_desc(su32(sA(st))), db = tc_desc(su32(sB(st)));
#pragma unroll
      for (int kk = 0; kk < TC_BK / 16; ++kk) {
        const uint32_t acc = (kc > 0 || kk > 0) ? 1u : 0u;
        // K = 16 spans two k groups: advance the start address by 2 * LBO
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da + (uint64_t)(kk * 16)), "l"(db + (uint64_t)(kk * 16)), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              su32(&mbar[st]))
          : "memory");
    }
  }
  // all MMAs done: the last stage's commit covers every earlier one
  if (nk > 0 && ok) ok = tc_wait(&mbar[(nk - 1) & 1], (uint32_t)(((nk - 1) >> 1) & 1));
  if (nk > 1 && ok) ok = tc_wait(&mbar[nk & 1], (uint32_t)(((nk - 2) >> 1) & 1));
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const int m = m0 + 32 * warp + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      uint32_t r[16];
      const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
          "%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
            "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(ta));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m < d.M) {
        float* row = C + m * d.c_m + (long long)(n0 + c0) * d.c_n;
        if (d.c_n == 1 && n0 + c0 + 16 <= d.N && (reinterpret_cast<uintptr_t>(row) & 15) == 0) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float4 o = make_float4(d.alpha * __uint_as_float(r[4 * q]),
                                   d.alpha * __uint_as_float(r[4 * q + 1]),
                                   d.alpha * __uint_as_float(r[4 * q + 2]),
                                   d.alpha * __uint_as_float(r[4 * q + 3]));
            float4* p4 = reinterpret_cast<float4*>(row) + q;
            if (d.beta != 0.f) {
              const float4 c = *p4;
              o.x += d.beta * c.x; o.y += d.beta * c.y; o.z += d.beta * c.z; o.w += d.beta * c.w;
            }
            *p4 = o;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int n = n0 + c0 + j;
            if (n < d.N) {
              float* p = C + m * d.c_m + n * d.c_n;
              const float v = d.alpha * __uint_as_float(r[j]);
              *p = d.beta == 0.f ? v : v + d.beta * *p;
            }
          }
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN)
                 : "memory");
  }
}

// Deterministic split-K reduction: out = alpha * sum_s part[s] + beta * out.
__global__ void splitk_reduce_kernel(const float* part, int S, int M, int N, float* C,
                                     long long c_m, long long c_n, float alpha, float beta) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * N) return;
  float s = 0.f;
  for (int k = 0; k < S; ++k) s += part[(long long)k * M * N + i];
  const int m = i / N, n = i - m * N;
  float* p = C + m * c_m + n * c_n;
  *p = beta == 0.f ? alpha * s : alpha * s + beta * *p;
}

// ---------------------------------------------------------- elementwise
__device__ __forceinline__ float gelu_f(float z) {
  return 0.5f * z * (1.f + erff(z * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) +
         z * 0.3989422804014327f * expf(-0.5f * z * z);
}

// x[r][c] += bias[c]; optionally y = GELU(x) (x keeps the pre-activation)
__global__ void bias_act_kernel(float* x, const float* bias, long long rows, int cols, float* y) {
  const long long n = rows * cols;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float z = x[i] + bias[i % cols];
    x[i] = z;
    if (y) y[i] = gelu_f(z);
  }
}

// dz = dy * GELU'(z)  (in place on dy)
__global__ void gelu_back_kernel(float* dy, const float* z, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dy[i] *= gelu_grad(z[i]);
}

// Per-block partial column sums of x [rows x cols] (cols <= 256).
__global__ void colsum_partial_kernel(const float* x, long long rows, int cols, float* part) {
  extern __shared__ float sh[];
  const int c = threadIdx.x % cols, lanes = blockDim.x / cols, l = threadIdx.x / cols;
  float s = 0.f;
  if (threadIdx.x < lanes * cols)
    for (long long r = (long long)blockIdx.x * lanes + l; r < rows; r += (long long)gridDim.x * lanes)
      s += x[r * cols + c];
  sh[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x < cols) {
    float t = 0.f;
    for (int k = 0; k < lanes; ++k) t += sh[k * cols + threadIdx.x];
    part[blockIdx.x * cols + threadIdx.x] = t;
  }
}

__global__ void colsum_final_kernel(const float* part, int nblocks, int cols, float* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float t = 0.f;
  for (int b = 0; b < nblocks; ++b) t += part[b * cols + c];
  out[c] = t;
}

// du = (2 / count)(u - t); per-block partial sums of (u - t)^2 in FP64
__global__ void mse_kernel(const float* u, const float* t, float* du, long long n, double* part) {
  __shared__ double sh[256];
  double s = 0.0;
  const float sc = 2.f / (float)n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float e = u[i] - t[i];
    s += (double)e * e;
    if (du) du[i] = sc * e;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// Adam (Kingma & Ba 2015) with bias correction; b1t = beta1^step, b2t = beta2^step.
__global__ void adam_kernel(float* w, const float* g, float* m, float* v, long long n, float lr,
                            float beta1, float beta2, float eps, float b1t, float b2t) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = beta1 * m[i] + (1.f - beta1) * gi;
    const float vi = beta2 * v[i] + (1.f - beta2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.f - b1t), vh = vi / (1.f - b2t);
    w[i] -= lr * mh / (sqrtf(vh) + eps);
  }
}

// ------------------------------------------- network input / output maps
// Input features of one pump image: (P / P_thr, x / (lx/2), y / (ly/2)) at
// the cell positions -l/2 + i l/n.
__global__ void features_kernel(const float* P, long long total, int H, int W, double lx,
                                double ly, double p_thr, float* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i % ((long long)H * W);
    const int y = (int)(r / W), x = (int)(r - (long long)y * W);
    out[3 * i + 0] = (float)((double)P[i] / p_thr);
    out[3 * i + 1] = (float)((-0.5 * lx + x * (lx / W)) / (0.5 * lx));
    out[3 * i + 2] = (float)((-0.5 * ly + y * (ly / H)) / (0.5 * ly));
  }
}

// Per-sample sum of psi (FP64, fixed order: strided per-thread sums, then a
// shared-memory tree), stored as the unit phase factor exp(-i arg sum).
__global__ void __launch_bounds__(512) phase_kernel(const float2* psi, long long hw, double2* ph) {
  __shared__ double sr[512], si[512];
  const float2* p = psi + blockIdx.x * hw;
  double a = 0.0, b = 0.0;
  for (long long i = threadIdx.x; i < hw; i += blockDim.x) {
    a += p[i].x;
    b += p[i].y;
  }
  sr[threadIdx.x] = a;
  si[threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sr[threadIdx.x] += sr[threadIdx.x + o];
      si[threadIdx.x] += si[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double m = sqrt(sr[0] * sr[0] + si[0] * si[0]);
    ph[blockIdx.x] = m > 0.0 ? make_double2(sr[0] / m, -si[0] / m) : make_double2(1.0, 0.0);
  }
}

// Network target: (Re, Im) of psi rotated by the sample's phase factor, over
// scale_psi, and n over scale_n.
__global__ void targets_kernel(const float2* psi, const float* n, long long total, long long hw,
                               const double2* ph, double scale_psi, double scale_n, float* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 e = ph[i / hw];
    const double re = psi[i].x, im = psi[i].y;
    out[3 * i + 0] = (float)((re * e.x - im * e.y) / scale_psi);
    out[3 * i + 1] = (float)((re * e.y + im * e.x) / scale_psi);
    out[3 * i + 2] = (float)((double)n[i] / scale_n);
  }
}

// Network output back to a solver state: psi = (u0 + i u1) scale_psi,
// n = max(u2, 0) scale_n (a reservoir density is non-negative).
__global__ void to_state_kernel(const float* u, long long total, double scale_psi, double scale_n,
                                float2* psi, float* n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    psi[i] = make_float2((float)(u[3 * i] * scale_psi), (float)(u[3 * i + 1] * scale_psi));
    if (n) n[i] = (float)(fmax((double)u[3 * i + 2], 0.0) * scale_n);
  }
}

int blocks_for(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

}  // namespace
}  // namespace phx

using namespace phx;

struct phx_fno {
  phx_fno_config cfg;
  cudaStream_t stream = nullptr;
  long long nparams = 0;
  // parameter offsets
  long long o_Wl, o_bl, o_Rr[8], o_Ri[8], o_W[8], o_b[8], o_Q1, o_q1, o_Q2, o_q2;
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // params, grads, Adam moments
  long long step = 0;
  // DFT tables
  float *Fx = nullptr, *Gx = nullptr, *Cy = nullptr, *Sy = nullptr;
  // activations (max_batch)
  std::vector<float*> act;  // v_0 .. v_L
  std::vector<float*> zl;   // pre-activations z_0 .. z_{L-1}
  float *Vx = nullptr, *Vxy = nullptr, *Sh = nullptr, *gy = nullptr;  // per-layer spectral temps
  std::vector<float*> Vxy_l;  // Vxy kept per layer for the weight gradients
  float *z1 = nullptr, *h1 = nullptr, *u = nullptr;
  float *dv = nullptr, *dv2 = nullptr, *dz = nullptr, *dh = nullptr, *du = nullptr;
  float *dVx = nullptr, *dVxy = nullptr, *dSh = nullptr, *dgy = nullptr;
  float* splitk = nullptr;
  long long splitk_len = 0;
  float* colpart = nullptr;
  int* tc_err = nullptr;  // set by a tensor-core GEMM whose bounded wait gave up
  double gemm_flops = 0;  // algorithmic GEMM flops issued since creation (2 M N K per product)
  double* lpart = nullptr;
  double* lpart_host = nullptr;
  int device = 0;
  std::string err;
};

namespace {

thread_local std::string g_fno_err = "no error";

phx_status ffail(phx_fno* f, phx_status s, const std::string& msg) {
  if (f)
    f->err = msg;
  else
    g_fno_err = msg;
  return s;
}

#define PHX_FCK(f, expr)                                                                   \
  do {                                                                                     \
    cudaError_t _e = (expr);                                                               \
    if (_e != cudaSuccess)                                                                 \
      return ffail((f), _e == cudaErrorMemoryAllocation ? PHX_ENOMEM : PHX_ECUDA,          \
                   std::string(#expr) + ": " + cudaGetErrorString(_e));                    \
  } while (0)

GemmDesc gd(int M, int N, int K, int nb1, int nb2, const float* A, long long a_m,
            long long a_k, long long a_b1, long long a_b2, const float* B, long long b_k,
            long long b_n, long long b_b1, long long b_b2, float* C, long long c_m,
            long long c_n, long long c_b1, long long c_b2, float alpha, float beta) {
  GemmDesc d;
  d.M = M; d.N = N; d.K = K; d.K_last = K; d.nb1 = nb1; d.nb2 = nb2;
  d.A = A; d.a_m = a_m; d.a_k = a_k; d.a_b1 = a_b1; d.a_b2 = a_b2;
  d.B = B; d.b_k = b_k; d.b_n = b_n; d.b_b1 = b_b1; d.b_b2 = b_b2;
  d.C = C; d.c_m = c_m; d.c_n = c_n; d.c_b1 = c_b1; d.c_b2 = c_b2;
  d.alpha = alpha; d.beta = beta;
  return d;
}

template <int BN>
cudaError_t run_gemm_tc(phx_fno* f, const GemmDesc& d) {
  const int smem = 2 * TC_BM * TC_BK * 2 + 2 * BN * TC_BK * 2;
  static int configured = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured != dev) {
    cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<BN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured = dev;
  }
  dim3 grid((d.M + TC_BM - 1) / TC_BM, (d.N + BN - 1) / BN, d.nb1 * d.nb2);
  gemm_tc_kernel<BN><<<grid, TC_T, smem, f->stream>>>(d, f->tc_err);
  count_launch();
  return cudaGetLastError();
}

// Tall products (M >= 128: the pointwise layers over batch x H x W rows and
// the inverse DFTs over H or W rows) run on tcgen05 with a 128-row tile;
// short ones (the forward truncated DFTs, the per-mode mixing, the split-K
// weight gradients) on the mma.sync kernel, whose 64-row tile wastes less.
cudaError_t run_gemm(phx_fno* f, const GemmDesc& d) {
  // every product of the batch has K columns except the last, which has K_last
  f->gemm_flops += 2.0 * d.M * d.N * ((double)d.K * (d.nb1 * d.nb2 - 1) + d.K_last);
  if (d.M >= TC_BM && d.N <= 256) {
    if (d.N <= 32) return run_gemm_tc<32>(f, d);
    if (d.N <= 64) return run_gemm_tc<64>(f, d);
    if (d.N <= 128) return run_gemm_tc<128>(f, d);
  }
  dim3 grid((d.M + GM - 1) / GM, (d.N + GN - 1) / GN, d.nb1 * d.nb2);
  gemm_bf16_kernel<<<grid, GT, 0, f->stream>>>(d);
  count_launch();
  return cudaGetLastError();
}

// Unbatched GEMM with a long K (the weight gradients, K = batch x H x W):
// split K into S chunks of kc (the last one shorter) written to a workspace,
// then a fixed-order reduction (deterministic, no atomics).
cudaError_t run_gemm_splitk(phx_fno* f, const GemmDesc& d) {
  const int S_MAX = 128;
  if (d.K < 4096 || (long long)S_MAX * d.M * d.N > f->splitk_len) return run_gemm(f, d);
  const int kc = ((d.K + S_MAX - 1) / S_MAX + GK - 1) / GK * GK;
  const int S = (d.K + kc - 1) / kc;
  GemmDesc p = d;
  p.K = kc;
  p.K_last = d.K - kc * (S - 1);
  p.nb1 = 1;
  p.nb2 = S;
  p.a_b1 = 0;
  p.a_b2 = (long long)kc * d.a_k;
  p.b_b1 = 0;
  p.b_b2 = (long long)kc * d.b_k;
  p.C = f->splitk;
  p.c_m = d.N;
  p.c_n = 1;
  p.c_b1 = 0;
  p.c_b2 = (long long)d.M * d.N;
  p.alpha = 1.f;
  p.beta = 0.f;
  cudaError_t e = run_gemm(f, p);
  if (e != cudaSuccess) return e;
  splitk_reduce_kernel<<<(d.M * d.N + 255) / 256, 256, 0, f->stream>>>(
      f->splitk, S, d.M, d.N, d.C, d.c_m, d.c_n, d.alpha, d.beta);
  count_launch();
  return cudaGetLastError();
}

cudaError_t bias_act(phx_fno* f, float* x, const float* b, long long rows, int cols, float* y) {
  bias_act_kernel<<<blocks_for(rows * cols), 256, 0, f->stream>>>(x, b, rows, cols, y);
  count_launch();
  return cudaGetLastError();
}

cudaError_t gelu_back(phx_fno* f, float* dy, const float* z, long long n) {
  gelu_back_kernel<<<blocks_for(n), 256, 0, f->stream>>>(dy, z, n);
  count_launch();
  return cudaGetLastError();
}

// out[c] = sum_r x[r][c] (deterministic two-pass)
cudaError_t colsum(phx_fno* f, const float* x, long long rows, int cols, float* out) {
  const int nb = 512;
  colsum_partial_kernel<<<nb, 256, 256 * sizeof(float), f->stream>>>(x, rows, cols, f->colpart);
  colsum_final_kernel<<<(cols + 127) / 128, 128, 0, f->stream>>>(f->colpart, nb, cols, out);
  count_launch(2);
  return cudaGetLastError();
}

// Spectral branch of layer l: s = K_l(v) written into z (beta = 0).
cudaError_t spectral_forward(phx_fno* f, int l, int B, const float* v, float* z) {
  const phx_fno_config& c = f->cfg;
  const int H = c.height, W = c.width, C = c.channels, MX = c.modes_x, MY = c.modes_y;
  const long long HWC = (long long)H * W * C;
  const long long XM = 2LL * MX * C;    // Vx row (one y) length
  const long long HX = (long long)H * XM;
  const long long MM = (long long)MY * MX * C;  // one part of Vxy
  float* Vxy = f->Vxy_l[l];
  const float* Rr = f->w + f->o_Rr[l];
  const float* Ri = f->w + f->o_Ri[l];
  cudaError_t e;
  // 1. Vx[b,y] = Fx [2MX x W] . v[b,y] [W x C]
  e = run_gemm(f, gd(2 * MX, C, W, B, H, f->Fx, W, 1, 0, 0, v, C, 1, HWC, (long long)W * C,
                     f->Vx, C, 1, HX, XM, 1.f, 0.f));
  if (e) return e;
  // 2. Vxy_re = Cy Vx_re + Sy Vx_im ; Vxy_im = Cy Vx_im - Sy Vx_re   (per b)
  const float* Vre = f->Vx;
  const float* Vim = f->Vx + (long long)MX * C;
  float* Yre = Vxy;
  float* Yim = Vxy + MM;
  const int NY = MX * C;
  e = run_gemm(f, gd(MY, NY, H, B, 1, f->Cy, H, 1, 0, 0, Vre, XM, 1, HX, 0, Yre, NY, 1, 2 * MM, 0, 1.f, 0.f));
  if (e) return e;
  e = run_gemm(f, gd(MY, NY, H, B, 1, f->Sy, H, 1, 0, 0, Vim, XM, 1, HX, 0, Yre, NY, 1, 2 * MM, 0, 1.f, 1.f));
  if (e) return e;
  e = run_gemm(f, gd(MY, NY, H, B, 1, f->Cy, H, 1, 0, 0, Vim, XM, 1, HX, 0, Yim, NY, 1, 2 * MM, 0, 1.f, 0.f));
  if (e) return e;
  e = run_gemm(f, gd(MY, NY, H, B, 1, f->Sy, H, 1, 0, 0, Vre, XM, 1, HX, 0, Yim, NY, 1, 2 * MM, 0, -1.f, 1.f));
  if (e) return e;
  // 3. per mode (my, kx): S_re = Vr Rr - Vi Ri ; S_im = Vr Ri + Vi Rr   [B x C] x [C x C]
  float* Sre = f->Sh;
  float* Sim = f->Sh + MM;
  const long long CC = (long long)C * C;
  auto mix = [&](const float* Ain, const float* Wt, float* Out, float alpha, float beta) {
    return run_gemm(f, gd(B, C, C, MY, MX, Ain, 2 * MM, 1, (long long)MX * C, C, Wt, C, 1,
                          (long long)MX * CC, CC, Out, 2 * MM, 1, (long long)MX * C, C, alpha, beta));
  };
  if ((e = mix(Yre, Rr, Sre, 1.f, 0.f))) return e;
  if ((e = mix(Yim, Ri, Sre, -1.f, 1.f))) return e;
  if ((e = mix(Yre, Ri, Sim, 1.f, 0.f))) return e;
  if ((e = mix(Yim, Rr, Sim, 1.f, 1.f))) return e;
  // 4. g_re[y] = sum_my cos S_re - sin S_im ; g_im = sin S_re + cos S_im  (Cy^T views)
  float* Gre = f->gy;
  float* Gim = f->gy + (long long)MX * C;
  e = run_gemm(f, gd(H, NY, MY, B, 1, f->Cy, 1, H, 0, 0, Sre, NY, 1, 2 * MM, 0, Gre, XM, 1, HX, 0, 1.f, 0.f));
  if (e) return e;
  e = run_gemm(f, gd(H, NY, MY, B, 1, f->Sy, 1, H, 0, 0, Sim, NY, 1, 2 * MM, 0, Gre, XM, 1, HX, 0, -1.f, 1.f));
  if (e) return e;
  e = run_gemm(f, gd(H, NY, MY, B, 1, f->Sy, 1, H, 0, 0, Sre, NY, 1, 2 * MM, 0, Gim, XM, 1, HX, 0, 1.f, 0.f));
  if (e) return e;
  e = run_gemm(f, gd(H, NY, MY, B, 1, f->Cy, 1, H, 0, 0, Sim, NY, 1, 2 * MM, 0, Gim, XM, 1, HX, 0, 1.f, 1.f));
  if (e) return e;
  // 5. s[b,y] = Gx [W x 2MX] . g[b,y] [2MX x C]
  return run_gemm(f, gd(W, C, 2 * MX, B, H, f->Gx, 2 * MX, 1, 0, 0, f->gy, C, 1, HX, XM, z, C, 1,
                        HWC, (long long)W * C, 1.f, 0.f));
}

// Adjoint of spectral_forward: given dz (= ds), accumulate dv += K^T dz and
// the gradients of Rr, Ri (written, beta = 0).
cudaError_t spectral_backward(phx_fno* f, int l, int B, const float* dz, float* dv) {
  const phx_fno_config& c = f->cfg;
  const int H = c.height, W = c.width, C = c.channels, MX = c.modes_x, MY = c.modes_y;
  const long long HWC = (long long)H * W * C;
  const long long XM = 2LL * MX * C, HX = (long long)H * XM, MM = (long long)MY * MX * C;
  const int NY = MX * C;
  const long long CC = (long long)C * C;
  const float* Rr = f->w + f->o_Rr[l];
  const float* Ri = f->w + f->o_Ri[l];
  float* gRr = f->g + f->o_Rr[l];
  float* gRi = f->g + f->o_Ri[l];
  const float* Vxy = f->Vxy_l[l];
  cudaError_t e;
  // 5'. dg[b,y] = Gx^T [2MX x W] . dz[b,y]
  e = run_gemm(f, gd(2 * MX, C, W, B, H, f->Gx, 1, 2 * MX, 0, 0, dz, C, 1, HWC, (long long)W * C,
                     f->dgy, C, 1, HX, XM, 1.f, 0.f));
  if (e) return e;
  // 4'. dS_re = Cy dg_re + Sy dg_im ; dS_im = -Sy dg_re + Cy dg_im
  const float* dGre = f->dgy;
  const float* dGim = f->dgy + (long long)MX * C;
  float* dSre = f->dSh;
  float* dSim = f->dSh + MM;
  e = run_gemm(f, gd(MY, NY, H, B, 1, f->Cy, H, 1, 0, 0, dGre, XM, 1, HX, 0, dSre, NY, 1, 2 * MM, 0, 1.f, 0.f));
  if (e) return e;
  e = run_gemm(f, gd(MY, NY, H, B, 1, f->Sy, H, 1, 0, 0, dGim, XM, 1, HX, 0, dSre, NY, 1, 2 * MM, 0, 1.f, 1.f));
  if (e) return e;
  e = run_gemm(f, gd(MY, NY, H, B, 1, f->Sy, H, 1, 0, 0, dGre, XM, 1, HX, 0, dSim, NY, 1, 2 * MM, 0, -1.f, 0.f));
  if (e) return e;
  e = run_gemm(f, gd(MY, NY, H, B, 1, f->Cy, H, 1, 0, 0, dGim, XM, 1, HX, 0, dSim, NY, 1, 2 * MM, 0, 1.f, 1.f));
  if (e) return e;
  // 3'. per mode: dVr = dSr Rr^T + dSi Ri^T ; dVi = -dSr Ri^T + dSi Rr^T
  //             dRr = Vr^T dSr + Vi^T dSi ; dRi = -Vi^T dSr + Vr^T dSi
  const float* Vr = Vxy;
  const float* Vi = Vxy + MM;
  float* dVr = f->dVxy;
  float* dVi = f->dVxy + MM;
  auto mixT = [&](const float* Ain, const float* Wt, float* Out, float alpha, float beta) {
    // Out [B x C] = Ain [B x C] . Wt^T
    return run_gemm(f, gd(B, C, C, MY, MX, Ain, 2 * MM, 1, (long long)MX * C, C, Wt, 1, C,
                          (long long)MX * CC, CC, Out, 2 * MM, 1, (long long)MX * C, C, alpha, beta));
  };
  if ((e = mixT(dSre, Rr, dVr, 1.f, 0.f))) return e;
  if ((e = mixT(dSim, Ri, dVr, 1.f, 1.f))) return e;
  if ((e = mixT(dSre, Ri, dVi, -1.f, 0.f))) return e;
  if ((e = mixT(dSim, Rr, dVi, 1.f, 1.f))) return e;
  auto wgrad = [&](const float* X, const float* dS, float* Out, float alpha, float beta) {
    // Out [C x C] = X^T [C x B] . dS [B x C]
    return run_gemm(f, gd(C, C, B, MY, MX, X, 1, 2 * MM, (long long)MX * C, C, dS, 2 * MM, 1,
                          (long long)MX * C, C, Out, C, 1, (long long)MX * CC, CC, alpha, beta));
  };
  if ((e = wgrad(Vr, dSre, gRr, 1.f, 0.f))) return e;
  if ((e = wgrad(Vi, dSim, gRr, 1.f, 1.f))) return e;
  if ((e = wgrad(Vi, dSre, gRi, -1.f, 0.f))) return e;
  if ((e = wgrad(Vr, dSim, gRi, 1.f, 1.f))) return e;
  // 2'. dVx_re = Cy^T dVr - Sy^T dVi ; dVx_im = Sy^T dVr + Cy^T dVi
  float* dXre = f->dVx;
  float* dXim = f->dVx + (long long)MX * C;
  e = run_gemm(f, gd(H, NY, MY, B, 1, f->Cy, 1, H, 0, 0, dVr, NY, 1, 2 * MM, 0, dXre, XM, 1, HX, 0, 1.f, 0.f));
  if (e) return e;
  e = run_gemm(f, gd(H, NY, MY, B, 1, f->Sy, 1, H, 0, 0, dVi, NY, 1, 2 * MM, 0, dXre, XM, 1, HX, 0, -1.f, 1.f));
  if (e) return e;
  e = run_gemm(f, gd(H, NY, MY, B, 1, f->Sy, 1, H, 0, 0, dVr, NY, 1, 2 * MM, 0, dXim, XM, 1, HX, 0, 1.f, 0.f));
  if (e) return e;
  e = run_gemm(f, gd(H, NY, MY, B, 1, f->Cy, 1, H, 0, 0, dVi, NY, 1, 2 * MM, 0, dXim, XM, 1, HX, 0, 1.f, 1.f));
  if (e) return e;
  // 1'. dv[b,y] += Fx^T [W x 2MX] . dVx[b,y]
  return run_gemm(f, gd(W, C, 2 * MX, B, H, f->Fx, 1, W, 0, 0, f->dVx, C, 1, HX, XM, dv, C, 1, HWC,
                        (long long)W * C, 1.f, 1.f));
}

cudaError_t forward(phx_fno* f, const float* in, int B) {
  const phx_fno_config& c = f->cfg;
  const long long R = (long long)B * c.height * c.width;
  const int C = c.channels;
  cudaError_t e;
  // lift: v0 = a W_lift + b_lift
  e = run_gemm(f, gd((int)R, C, c.in_channels, 1, 1, in, c.in_channels, 1, 0, 0, f->w + f->o_Wl, C, 1,
                     0, 0, f->act[0], C, 1, 0, 0, 1.f, 0.f));
  if (e) return e;
  if ((e = bias_act(f, f->act[0], f->w + f->o_bl, R, C, nullptr))) return e;
  for (int l = 0; l < c.layers; ++l) {
    float* z = f->zl[l];
    if ((e = spectral_forward(f, l, B, f->act[l], z))) return e;
    e = run_gemm(f, gd((int)R, C, C, 1, 1, f->act[l], C, 1, 0, 0, f->w + f->o_W[l], C, 1, 0, 0, z,
                       C, 1, 0, 0, 1.f, 1.f));
    if (e) return e;
    const bool last = l == c.layers - 1;
    if (last) {
      if ((e = bias_act(f, z, f->w + f->o_b[l], R, C, nullptr))) return e;
      if ((e = cudaMemcpyAsync(f->act[l + 1], z, sizeof(float) * R * C, cudaMemcpyDeviceToDevice,
                               f->stream)))
        return e;
    } else {
      if ((e = bias_act(f, z, f->w + f->o_b[l], R, C, f->act[l + 1]))) return e;
    }
  }
  // projection: h = GELU(v_L Q1 + q1) ; u = h Q2 + q2
  const int P = c.proj_hidden;
  e = run_gemm(f, gd((int)R, P, C, 1, 1, f->act[c.layers], C, 1, 0, 0, f->w + f->o_Q1, P, 1, 0, 0,
                     f->z1, P, 1, 0, 0, 1.f, 0.f));
  if (e) return e;
  if ((e = bias_act(f, f->z1, f->w + f->o_q1, R, P, f->h1))) return e;
  e = run_gemm(f, gd((int)R, c.out_channels, P, 1, 1, f->h1, P, 1, 0, 0, f->w + f->o_Q2,
                     c.out_channels, 1, 0, 0, f->u, c.out_channels, 1, 0, 0, 1.f, 0.f));
  if (e) return e;
  return bias_act(f, f->u, f->w + f->o_q2, R, c.out_channels, nullptr);
}

// Loss and full gradient into f->g (forward must have run on `in`).
cudaError_t backward(phx_fno* f, const float* in, const float* target, int B, double* loss) {
  const phx_fno_config& c = f->cfg;
  const long long R = (long long)B * c.height * c.width;
  const int C = c.channels, P = c.proj_hidden, CO = c.out_channels;
  cudaError_t e;
  const int nb = 512;
  mse_kernel<<<nb, 256, 0, f->stream>>>(f->u, target, f->du, R * CO, f->lpart);
  count_launch();
  if ((e = cudaGetLastError())) return e;
  if ((e = cudaMemcpyAsync(f->lpart_host, f->lpart, sizeof(double) * nb, cudaMemcpyDeviceToHost,
                           f->stream)))
    return e;
  // projection
  if ((e = run_gemm_splitk(f, gd(P, CO, (int)R, 1, 1, f->h1, 1, P, 0, 0, f->du, CO, 1, 0, 0,
                                 f->g + f->o_Q2, CO, 1, 0, 0, 1.f, 0.f))))
    return e;
  if ((e = colsum(f, f->du, R, CO, f->g + f->o_q2))) return e;
  if ((e = run_gemm(f, gd((int)R, P, CO, 1, 1, f->du, CO, 1, 0, 0, f->w + f->o_Q2, 1, CO, 0, 0, f->dh,
                          P, 1, 0, 0, 1.f, 0.f))))
    return e;
  if ((e = gelu_back(f, f->dh, f->z1, R * P))) return e;
  if ((e = run_gemm_splitk(f, gd(C, P, (int)R, 1, 1, f->act[c.layers], 1, C, 0, 0, f->dh, P, 1, 0, 0,
                                 f->g + f->o_Q1, P, 1, 0, 0, 1.f, 0.f))))
    return e;
  if ((e = colsum(f, f->dh, R, P, f->g + f->o_q1))) return e;
  // dv_L = dh Q1^T
  float* dv = f->dv;
  float* dvn = f->dv2;
  if ((e = run_gemm(f, gd((int)R, C, P, 1, 1, f->dh, P, 1, 0, 0, f->w + f->o_Q1, 1, P, 0, 0, dv, C, 1,
                          0, 0, 1.f, 0.f))))
    return e;
  for (int l = c.layers - 1; l >= 0; --l) {
    // dz = dv * GELU'(z) (identity on the last layer); dz lives in dv
    if (l < c.layers - 1)
      if ((e = gelu_back(f, dv, f->zl[l], R * C))) return e;
    // local branch
    if ((e = run_gemm_splitk(f, gd(C, C, (int)R, 1, 1, f->act[l], 1, C, 0, 0, dv, C, 1, 0, 0,
                                   f->g + f->o_W[l], C, 1, 0, 0, 1.f, 0.f))))
      return e;
    if ((e = colsum(f, dv, R, C, f->g + f->o_b[l]))) return e;
    if ((e = run_gemm(f, gd((int)R, C, C, 1, 1, dv, C, 1, 0, 0, f->w + f->o_W[l], 1, C, 0, 0, dvn, C,
                            1, 0, 0, 1.f, 0.f))))
      return e;
    // spectral branch (accumulates into dvn)
    if ((e = spectral_backward(f, l, B, dv, dvn))) return e;
    std::swap(dv, dvn);
  }
  // lift
  if ((e = run_gemm_splitk(f, gd(c.in_channels, C, (int)R, 1, 1, in, 1, c.in_channels, 0, 0, dv, C, 1,
                                 0, 0, f->g + f->o_Wl, C, 1, 0, 0, 1.f, 0.f))))
    return e;
  if ((e = colsum(f, dv, R, C, f->g + f->o_bl))) return e;
  if ((e = cudaStreamSynchronize(f->stream))) return e;
  double s = 0.0;
  for (int i = 0; i < nb; ++i) s += f->lpart_host[i];
  if (loss) *loss = s / (double)(R * CO);
  return cudaSuccess;
}

void free_fno(phx_fno* f) {
  if (f->stream) cudaStreamSynchronize(f->stream);
  float* bufs[] = {f->w, f->g, f->m, f->v, f->Fx, f->Gx, f->Cy, f->Sy, f->Vx, f->Vxy, f->Sh, f->gy,
                   f->z1, f->h1, f->u, f->dv, f->dv2, f->dz, f->dh, f->du, f->dVx, f->dVxy, f->dSh,
                   f->dgy, f->splitk, f->colpart};
  for (float* p : bufs)
    if (p) cudaFree(p);
  for (float* p : f->act)
    if (p) cudaFree(p);
  for (float* p : f->zl)
    if (p) cudaFree(p);
  for (float* p : f->Vxy_l)
    if (p) cudaFree(p);
  if (f->lpart) cudaFree(f->lpart);
  if (f->tc_err) cudaFree(f->tc_err);
  if (f->lpart_host) cudaFreeHost(f->lpart_host);
}

}  // namespace

extern "C" {

phx_status phx_fno_config_init(phx_fno_config* c) {
  if (!c) return ffail(nullptr, PHX_EINVAL, "config is NULL");
  std::memset(c, 0, sizeof *c);
  c->struct_size = sizeof(phx_fno_config);
  c->height = 256;
  c->width = 256;
  c->channels = 32;
  c->layers = 4;
  c->modes_x = 16;
  c->modes_y = 32;
  c->in_channels = 3;
  c->out_channels = 3;
  c->proj_hidden = 64;
  c->max_batch = 8;
  return PHX_OK;
}

phx_status phx_fno_create(const phx_fno_config* cfg, phx_fno** out) {
  if (!out) return ffail(nullptr, PHX_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfg || cfg->struct_size != sizeof(phx_fno_config))
    return ffail(nullptr, PHX_EINVAL, "config missing or struct_size mismatch");
  const phx_fno_config& c = *cfg;
  if (c.height < 2 || c.width < 2 || c.channels < 1 || c.layers < 1 || c.layers > 8 ||
      c.modes_x < 1 || c.modes_x > c.width / 2 || c.modes_y < 2 || (c.modes_y & 1) ||
      c.modes_y > c.height || c.in_channels < 1 || c.out_channels < 1 || c.proj_hidden < 1 ||
      c.max_batch < 1 || c.channels > 256 || c.proj_hidden > 256 || c.out_channels > 256)
    return ffail(nullptr, PHX_EINVAL, "invalid FNO configuration");
  phx_fno* f = new (std::nothrow) phx_fno();
  if (!f) return ffail(nullptr, PHX_ENOMEM, "host allocation failed");
  f->cfg = c;
  f->stream = static_cast<cudaStream_t>(c.stream);
  cudaGetDevice(&f->device);
  const long long C = c.channels, MX = c.modes_x, MY = c.modes_y;
  long long o = 0;
  auto take = [&](long long n) {
    long long r = o;
    o += n;
    return r;
  };
  f->o_Wl = take(c.in_channels * C);
  f->o_bl = take(C);
  for (int l = 0; l < c.layers; ++l) {
    f->o_Rr[l] = take(MY * MX * C * C);
    f->o_Ri[l] = take(MY * MX * C * C);
    f->o_W[l] = take(C * C);
    f->o_b[l] = take(C);
  }
  f->o_Q1 = take(C * c.proj_hidden);
  f->o_q1 = take(c.proj_hidden);
  f->o_Q2 = take((long long)c.proj_hidden * c.out_channels);
  f->o_q2 = take(c.out_channels);
  f->nparams = o;
  const long long Bm = c.max_batch, H = c.height, W = c.width;
  const long long R = Bm * H * W;
  auto fail_alloc = [&](cudaError_t e) {
    std::string m = std::string("allocation failed: ") + cudaGetErrorString(e);
    free_fno(f);
    delete f;
    return ffail(nullptr, e == cudaErrorMemoryAllocation ? PHX_ENOMEM : PHX_ECUDA, m);
  };
  auto alloc = [&](float** p, long long n) { return cudaMalloc(p, sizeof(float) * (n > 0 ? n : 1)); };
  cudaError_t e = cudaSuccess;
  for (float** p : {&f->w, &f->g, &f->m, &f->v})
    if (e == cudaSuccess) e = alloc(p, f->nparams);
  if (e == cudaSuccess) e = cudaMemsetAsync(f->m, 0, sizeof(float) * f->nparams, f->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(f->v, 0, sizeof(float) * f->nparams, f->stream);
  if (e == cudaSuccess) e = alloc(&f->Fx, 2 * MX * W);
  if (e == cudaSuccess) e = alloc(&f->Gx, 2 * MX * W);
  if (e == cudaSuccess) e = alloc(&f->Cy, MY * H);
  if (e == cudaSuccess) e = alloc(&f->Sy, MY * H);
  f->act.assign(c.layers + 1, nullptr);
  f->zl.assign(c.layers, nullptr);
  f->Vxy_l.assign(c.layers, nullptr);
  for (int l = 0; l <= c.layers && e == cudaSuccess; ++l) e = alloc(&f->act[l], R * C);
  for (int l = 0; l < c.layers && e == cudaSuccess; ++l) e = alloc(&f->zl[l], R * C);
  for (int l = 0; l < c.layers && e == cudaSuccess; ++l) e = alloc(&f->Vxy_l[l], Bm * 2 * MY * MX * C);
  if (e == cudaSuccess) e = alloc(&f->Vx, Bm * H * 2 * MX * C);
  if (e == cudaSuccess) e = alloc(&f->Sh, Bm * 2 * MY * MX * C);
  if (e == cudaSuccess) e = alloc(&f->gy, Bm * H * 2 * MX * C);
  if (e == cudaSuccess) e = alloc(&f->dVx, Bm * H * 2 * MX * C);
  if (e == cudaSuccess) e = alloc(&f->dVxy, Bm * 2 * MY * MX * C);
  if (e == cudaSuccess) e = alloc(&f->dSh, Bm * 2 * MY * MX * C);
  if (e == cudaSuccess) e = alloc(&f->dgy, Bm * H * 2 * MX * C);
  if (e == cudaSuccess) e = alloc(&f->z1, R * c.proj_hidden);
  if (e == cudaSuccess) e = alloc(&f->h1, R * c.proj_hidden);
  if (e == cudaSuccess) e = alloc(&f->dh, R * c.proj_hidden);
  if (e == cudaSuccess) e = alloc(&f->u, R * c.out_channels);
  if (e == cudaSuccess) e = alloc(&f->du, R * c.out_channels);
  if (e == cudaSuccess) e = alloc(&f->dv, R * C);
  if (e == cudaSuccess) e = alloc(&f->dv2, R * C);
  long long maxmn = std::max({C * C, C * (long long)c.proj_hidden,
                              (long long)c.proj_hidden * c.out_channels, c.in_channels * C});
  f->splitk_len = 128 * maxmn;
  if (e == cudaSuccess) e = alloc(&f->splitk, f->splitk_len);
  if (e == cudaSuccess) e = alloc(&f->colpart, 512LL * 256);
  if (e == cudaSuccess) e = cudaMalloc(&f->lpart, sizeof(double) * 512);
  if (e == cudaSuccess) e = cudaMalloc(&f->tc_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(f->tc_err, 0, sizeof(int), f->stream);
  if (e == cudaSuccess) e = cudaMallocHost(&f->lpart_host, sizeof(double) * 512);
  if (e != cudaSuccess) return fail_alloc(e);
  // DFT tables (FP64 angles, FP32 values)
  const double pi = 3.14159265358979323846;
  std::vector<float> Fx(2 * MX * W), Gx(2 * MX * W), Cy(MY * H), Sy(MY * H);
  for (int k = 0; k < MX; ++k)
    for (int x = 0; x < W; ++x) {
      const double a = 2.0 * pi * (double)k * x / W;
      const double wk = (k == 0 ? 1.0 : 2.0) / ((double)H * W);
      Fx[k * W + x] = (float)std::cos(a);
      Fx[(MX + k) * W + x] = (float)(-std::sin(a));
      Gx[x * 2 * MX + k] = (float)(wk * std::cos(a));
      Gx[x * 2 * MX + MX + k] = (float)(-wk * std::sin(a));
    }
  for (int m = 0; m < MY; ++m) {
    const long long ky = m < MY / 2 ? m : (long long)H - MY + m;
    for (int y = 0; y < H; ++y) {
      const double a = 2.0 * pi * (double)((ky * y) % H) / H;
      Cy[m * H + y] = (float)std::cos(a);
      Sy[m * H + y] = (float)std::sin(a);
    }
  }
  e = cudaMemcpy(f->Fx, Fx.data(), sizeof(float) * Fx.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(f->Gx, Gx.data(), sizeof(float) * Gx.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(f->Cy, Cy.data(), sizeof(float) * Cy.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(f->Sy, Sy.data(), sizeof(float) * Sy.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
  if (e != cudaSuccess) return fail_alloc(e);
  *out = f;
  return PHX_OK;
}

int64_t phx_fno_num_params(const phx_fno* f) { return f ? f->nparams : 0; }

phx_status phx_fno_gemm_flops(const phx_fno* f, double* flops) {
  if (!f || !flops) return PHX_EINVAL;
  *flops = f->gemm_flops;
  return PHX_OK;
}

phx_status phx_fno_set_params(phx_fno* f, const float* w, int on_device) {
  if (!f || !w) return ffail(f, PHX_EINVAL, "NULL argument");
  PHX_FCK(f, cudaMemcpyAsync(f->w, w, sizeof(float) * f->nparams,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, f->stream));
  PHX_FCK(f, cudaMemsetAsync(f->m, 0, sizeof(float) * f->nparams, f->stream));
  PHX_FCK(f, cudaMemsetAsync(f->v, 0, sizeof(float) * f->nparams, f->stream));
  PHX_FCK(f, cudaStreamSynchronize(f->stream));
  f->step = 0;
  return PHX_OK;
}

phx_status phx_fno_get_params(phx_fno* f, float* w, int on_device) {
  if (!f || !w) return ffail(f, PHX_EINVAL, "NULL argument");
  PHX_FCK(f, cudaMemcpyAsync(w, f->w, sizeof(float) * f->nparams,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, f->stream));
  PHX_FCK(f, cudaStreamSynchronize(f->stream));
  return PHX_OK;
}

phx_status phx_fno_forward(phx_fno* f, const float* in, float* out, int32_t batch) {
  if (!f || !in || !out) return ffail(f, PHX_EINVAL, "NULL argument");
  if (batch < 1 || batch > f->cfg.max_batch) return ffail(f, PHX_EINVAL, "batch out of range");
  PHX_FCK(f, forward(f, in, batch));
  const long long n = (long long)batch * f->cfg.height * f->cfg.width * f->cfg.out_channels;
  PHX_FCK(f, cudaMemcpyAsync(out, f->u, sizeof(float) * n, cudaMemcpyDeviceToDevice, f->stream));
  return PHX_OK;
}

phx_status phx_fno_loss_grad(phx_fno* f, const float* in, const float* target, int32_t batch,
                             double* loss, float* grad) {
  if (!f || !in || !target) return ffail(f, PHX_EINVAL, "NULL argument");
  if (batch < 1 || batch > f->cfg.max_batch) return ffail(f, PHX_EINVAL, "batch out of range");
  PHX_FCK(f, forward(f, in, batch));
  PHX_FCK(f, backward(f, in, target, batch, loss));
  int tc_err = 0;
  PHX_FCK(f, cudaMemcpy(&tc_err, f->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (tc_err) return ffail(f, PHX_ETIMEOUT, "a tensor-core GEMM wait timed out");
  if (grad) {
    PHX_FCK(f, cudaMemcpyAsync(grad, f->g, sizeof(float) * f->nparams, cudaMemcpyDeviceToDevice,
                               f->stream));
    PHX_FCK(f, cudaStreamSynchronize(f->stream));
  }
  return PHX_OK;
}

phx_status phx_fno_train_step(phx_fno* f, const float* in, const float* target, int32_t batch,
                              float lr, double* loss) {
  phx_status st = phx_fno_loss_grad(f, in, target, batch, loss, nullptr);
  if (st != PHX_OK) return st;
  f->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float b1t = (float)std::pow((double)b1, (double)f->step);
  const float b2t = (float)std::pow((double)b2, (double)f->step);
  adam_kernel<<<blocks_for(f->nparams), 256, 0, f->stream>>>(f->w, f->g, f->m, f->v, f->nparams, lr,
                                                             b1, b2, 1e-8f, b1t, b2t);
  count_launch();
  PHX_FCK(f, cudaGetLastError());
  return PHX_OK;
}

phx_status phx_fno_features(const float* P, int32_t batch, int32_t height, int32_t width, double lx,
                            double ly, double p_thr, float* out, void* stream) {
  if (!P || !out || batch < 1 || height < 1 || width < 1 || !(lx > 0) || !(ly > 0) || !(p_thr > 0))
    return ffail(nullptr, PHX_EINVAL, "phx_fno_features: bad argument");
  const long long total = (long long)batch * height * width;
  features_kernel<<<blocks_for(total), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      P, total, height, width, lx, ly, p_thr, out);
  count_launch();
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PHX_OK : ffail(nullptr, PHX_ECUDA, cudaGetErrorString(e));
}

phx_status phx_fno_targets(const float* psi, const float* n, int32_t batch, int32_t height,
                           int32_t width, double scale_psi, double scale_n, float* out,
                           void* stream) {
  if (!psi || !n || !out || batch < 1 || batch > 65535 || height < 1 || width < 1 ||
      !(scale_psi > 0) || !(scale_n > 0))
    return ffail(nullptr, PHX_EINVAL, "phx_fno_targets: bad argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long hw = (long long)height * width, total = batch * hw;
  double2* ph = nullptr;
  cudaError_t e = cudaMallocAsync(&ph, sizeof(double2) * batch, st);
  if (e != cudaSuccess) return ffail(nullptr, PHX_ENOMEM, cudaGetErrorString(e));
  phase_kernel<<<batch, 512, 0, st>>>(reinterpret_cast<const float2*>(psi), hw, ph);
  targets_kernel<<<blocks_for(total), 256, 0, st>>>(reinterpret_cast<const float2*>(psi), n,
                                                     total, hw, ph, scale_psi, scale_n, out);
  count_launch(2);
  e = cudaGetLastError();
  cudaFreeAsync(ph, st);
  return e == cudaSuccess ? PHX_OK : ffail(nullptr, PHX_ECUDA, cudaGetErrorString(e));
}

phx_status phx_fno_to_state(const float* u, int32_t batch, int32_t height, int32_t width,
                            double scale_psi, double scale_n, float* psi, float* n, void* stream) {
  if (!u || !psi || batch < 1 || height < 1 || width < 1)
    return ffail(nullptr, PHX_EINVAL, "phx_fno_to_state: bad argument");
  const long long total = (long long)batch * height * width;
  to_state_kernel<<<blocks_for(total), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      u, total, scale_psi, scale_n, reinterpret_cast<float2*>(psi), n);
  count_launch();
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PHX_OK : ffail(nullptr, PHX_ECUDA, cudaGetErrorString(e));
}

const char* phx_fno_last_error(const phx_fno* f) { return f ? f->err.c_str() : g_fno_err.c_str(); }

void phx_fno_destroy(phx_fno* f) {
  if (!f) return;
  free_fno(f);
  delete f;
}

}  // extern "C"
