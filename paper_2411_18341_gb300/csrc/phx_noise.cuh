// Counter-based complex Gaussian noise for the dW term of Eq. (PULSE_psi).
//
// Philox4x32-10 as published by Salmon, Moraes, Dror and Shaw, "Parallel
// random numbers: as easy as 1, 2, 3" (SC'11), keyed by
// key = (seed lo, seed hi), counter = (c, instance, step lo, step hi): for two
// components c = site and words (w0, w1) give xi_+, (w2, w3) xi_-; for one
// component c = site >> 1 and words (w0, w1) give the even, (w2, w3) the odd
// site of the pair, so one call serves two sites.
// The Box-Muller transform uses this project's own ln and cos/sin built
// from textbook series and only separately rounded float32 +, -, *, / and
// sqrt (explicit __f*_rn intrinsics, never contracted into FMA), so a CPU
// program that performs the same operations in the same order obtains the
// same bits:
//   u      = (2*(w >> 9) + 1) * 2^-24                         (exact)
//   ln u   = e*ln2_hi + (2(s + s z P(z)) + e*ln2_lo),  s = (m-1)/(m+1),
//            z = s^2, P(z) = 1/3 + z/5 + ... + z^4/11 (Horner),
//            m in [sqrt(1/2), sqrt(2)), ln2 split into a 16-bit head.
//   cos/sin(2 pi u): q = floor(4u), r = 4u - q (exact), phi = r*(pi/2),
//            Taylor series with coefficients 1/k! (sin to phi^13, cos to
//            phi^14), then the quadrant rotation.
//   xi     = scale * (rho cos, rho sin),  rho = sqrt(-2 ln u1).
#pragma once

#include <stdint.h>

namespace phx {

struct U4 {
  uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ void mulhilo32(uint32_t a, uint32_t b,
                                                   uint32_t& hi, uint32_t& lo) {
#ifdef __CUDA_ARCH__
  lo = a * b;
  hi = __umulhi(a, b);
#else
  uint64_t p = (uint64_t)a * (uint64_t)b;
  lo = (uint32_t)p;
  hi = (uint32_t)(p >> 32);
#endif
}

__host__ __device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0,
                                                     uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(M0, c.x, hi0, lo0);
    mulhilo32(M1, c.z, hi1, lo1);
    U4 n;
    n.x = hi1 ^ c.y ^ k0;
    n.y = lo1;
    n.z = hi0 ^ c.w ^ k1;
    n.w = lo0;
    c = n;
    k0 += W0;
    k1 += W1;
  }
  return c;
}

#ifdef __CUDACC__

__device__ __forceinline__ float nz_uniform(uint32_t w) {
  // integer 2*(w>>9)+1 < 2^24 converts exactly; the power-of-two scale is exact
  return __fmul_rn(__uint2float_rn(2u * (w >> 9) + 1u), 5.9604644775390625e-08f);
}

__device__ __forceinline__ float nz_ln(float u) {
  uint32_t bits = __float_as_uint(u);
  int e = (int)((bits >> 23) & 0xFFu) - 127;
  float m = __uint_as_float((bits & 0x7FFFFFu) | 0x3F800000u);
  if (m > 0x1.6a09e6p+0f) {  // sqrt(2) rounded to float
    m = __fmul_rn(m, 0.5f);
    e += 1;
  }
  float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
  float z = __fmul_rn(s, s);
  float p = 0x1.745d18p-4f;                              // 1/11
  p = __fadd_rn(__fmul_rn(p, z), 0x1.c71c72p-4f);        // 1/9
  p = __fadd_rn(__fmul_rn(p, z), 0x1.24924ap-3f);        // 1/7
  p = __fadd_rn(__fmul_rn(p, z), 0x1.99999ap-3f);        // 1/5
  p = __fadd_rn(__fmul_rn(p, z), 0x1.555556p-2f);        // 1/3
  float t = __fmul_rn(__fmul_rn(s, z), p);
  float lnm = __fmul_rn(2.0f, __fadd_rn(s, t));
  float ef = (float)e;  // |e| <= 25, exact
  return __fadd_rn(__fmul_rn(ef, 0x1.62e4p-1f),
                   __fadd_rn(lnm, __fmul_rn(ef, 0x1.7f7d1cp-20f)));
}

__device__ __forceinline__ void nz_cos_sin_2pi(float u, float& co, float& si) {
  float t = __fmul_rn(u, 4.0f);
  float fq = floorf(t);
  int q = ((int)fq) & 3;
  float r = __fsub_rn(t, fq);
  float phi = __fmul_rn(r, 0x1.921fb6p+0f);  // pi/2 rounded to float
  float z = __fmul_rn(phi, phi);
  float ps = 0x1.612462p-33f;                           //  1/13!
  ps = __fadd_rn(__fmul_rn(ps, z), -0x1.ae6456p-26f);   // -1/11!
  ps = __fadd_rn(__fmul_rn(ps, z), 0x1.71de3ap-19f);    //  1/9!
  ps = __fadd_rn(__fmul_rn(ps, z), -0x1.a01a02p-13f);   // -1/7!
  ps = __fadd_rn(__fmul_rn(ps, z), 0x1.111112p-7f);     //  1/5!
  ps = __fadd_rn(__fmul_rn(ps, z), -0x1.555556p-3f);    // -1/3!
  float s = __fadd_rn(phi, __fmul_rn(__fmul_rn(phi, z), ps));
  float pc = -0x1.93974ap-37f;                          // -1/14!
  pc = __fadd_rn(__fmul_rn(pc, z), 0x1.1eed8ep-29f);    //  1/12!
  pc = __fadd_rn(__fmul_rn(pc, z), -0x1.27e4fcp-22f);   // -1/10!
  pc = __fadd_rn(__fmul_rn(pc, z), 0x1.a01a02p-16f);    //  1/8!
  pc = __fadd_rn(__fmul_rn(pc, z), -0x1.6c16c2p-10f);   // -1/6!
  pc = __fadd_rn(__fmul_rn(pc, z), 0x1.555556p-5f);     //  1/4!
  pc = __fadd_rn(__fmul_rn(pc, z), -0.5f);              // -1/2!
  float c = __fadd_rn(1.0f, __fmul_rn(z, pc));
  switch (q) {
    case 0: co = c; si = s; break;
    case 1: co = -s; si = c; break;
    case 2: co = -c; si = -s; break;
    default: co = s; si = -c; break;
  }
}

// Two words -> one complex Gaussian sample (re, im) times scale.
__device__ __forceinline__ float2 nz_box_muller(uint32_t wa, uint32_t wb,
                                                float scale) {
  float u1 = nz_uniform(wa);
  float u2 = nz_uniform(wb);
  float lg = nz_ln(u1);
  float rho = __fsqrt_rn(__fmul_rn(-2.0f, lg));
  float c, s;
  nz_cos_sin_2pi(u2, c, s);
  float z1 = __fmul_rn(rho, c);
  float z2 = __fmul_rn(rho, s);
  return make_float2(__fmul_rn(scale, z1), __fmul_rn(scale, z2));
}

__device__ __forceinline__ U4 nz_words(unsigned long long seed, unsigned int instance,
                                       long long step, uint32_t ctr) {
  U4 c;
  c.x = ctr;
  c.y = instance;
  c.z = (uint32_t)((unsigned long long)step & 0xFFFFFFFFull);
  c.w = (uint32_t)((unsigned long long)step >> 32);
  return philox4x32_10(c, (uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32));
}

// Noise of site `site` at step `step`: xi_+ and, for two components, xi_-,
// each component with its own per-quadrature standard deviation.
__device__ __forceinline__ void nz_site2(unsigned long long seed,
                                         unsigned int instance,
                                         long long step, uint32_t site,
                                         float scale0, float scale1,
                                         float2& xi0, float2& xi1, bool two) {
  if (two) {
    const U4 w = nz_words(seed, instance, step, site);
    xi0 = nz_box_muller(w.x, w.y, scale0);
    xi1 = nz_box_muller(w.z, w.w, scale1);
  } else {
    const U4 w = nz_words(seed, instance, step, site >> 1);
    xi0 = (site & 1u) ? nz_box_muller(w.z, w.w, scale0) : nz_box_muller(w.x, w.y, scale0);
  }
}

// One-component noise of the even site 2p and the odd site 2p + 1 from one
// Philox call.
__device__ __forceinline__ void nz_pair(unsigned long long seed, unsigned int instance,
                                        long long step, uint32_t pair, float scale_even,
                                        float scale_odd, float2& xi_even, float2& xi_odd) {
  const U4 w = nz_words(seed, instance, step, pair);
  xi_even = nz_box_muller(w.x, w.y, scale_even);
  xi_odd = nz_box_muller(w.z, w.w, scale_odd);
}

__device__ __forceinline__ void nz_site(unsigned long long seed,
                                        unsigned int instance,
                                        long long step, uint32_t site,
                                        float scale, float2& xi0, float2& xi1,
                                        bool two) {
  nz_site2(seed, instance, step, site, scale, scale, xi0, xi1, two);
}

// Truncated-Wigner per-quadrature standard deviation (Sec. V, Example 4):
// E|xi|^2 = nu (R n + gamma_c) dt / (2 dV) + noise_var, evaluated in float32
// as v = ((R n + gamma_c) kw) + var with kw = nu dt / (2 dV), each operation
// separately rounded, then sqrt(max(v, 0) / 2).
__device__ __forceinline__ float nz_wigner_scale(float R, float gc, float kw,
                                                 float var, float n) {
  float v = __fadd_rn(__fmul_rn(__fadd_rn(__fmul_rn(R, n), gc), kw), var);
  v = fmaxf(v, 0.0f);
  return __fsqrt_rn(__fmul_rn(v, 0.5f));
}

#endif  // __CUDACC__

}  // namespace phx
