"""Oracle for the additive complex noise dW of Eq. (PULSE_psi).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper names a complex Wiener term dW (Sec. V, Eq. PULSE_psi) but not its
generator.  The reading used here (fixed variance per step, added after each
full deterministic RK4 step) draws, for every grid site, component and step,
one complex Gaussian from a counter-based generator so that any site of any
step can be regenerated independently:

* Philox4x32-10 exactly as published by Salmon, Moraes, Dror and Shaw,
  "Parallel random numbers: as easy as 1, 2, 3" (SC'11): a 4x32-bit counter,
  a 2x32-bit key, ten rounds; each round multiplies counter words 0 and 2 by
  the two published multipliers (full 64-bit products split into hi/lo
  words), permutes and XORs with the round key; the key is bumped by the two
  published Weyl constants between rounds.
* key = (seed lo 32 bits, seed hi 32 bits);
  two components: counter = (site = j*nx + i, instance, step lo 32 bits,
  step hi 32 bits), words (w0, w1) feed component +, (w2, w3) component -;
  one component: counter word 0 = site >> 1, words (w0, w1) feed the even and
  (w2, w3) the odd site of the pair (one Philox call per two sites).
* uniform: u = (2*(w >> 9) + 1) * 2**-24, exact in FP32, u in (0, 1).
* Box-Muller: rho = sqrt(-2 ln u1), theta = 2 pi u2, z1 = rho cos theta,
  z2 = rho sin theta, xi = s*(z1 + i z2) with s = float32(sqrt(var/2)) so that
  E|xi|^2 = var.
* ln and cos/sin are this project's own, from textbook series:
  ln(u) = e ln2 + 2 atanh((m-1)/(m+1)) with m in [sqrt(1/2), sqrt(2)) and the
  atanh Taylor series through s^11; ln2 is split Cody-Waite style into a
  16-bit head and a float tail.  cos/sin(2 pi u) use the exact quadrant split
  of 4u and Taylor polynomials with coefficients 1/k! through degree 13/14.
  Every operation is a separately rounded float32 +, -, *, / or sqrt (no
  fused multiply-add), evaluated here with numpy float32 arrays.

Parity: pinned by (i) Triton's independent Philox4x32-10 run in its CPU
interpreter, (ii) libm log/sin/cos within stated error bounds, (iii) sample
statistics of the Gaussians (tests/test_oracle_noise.py).
"""
import numpy as np

U32 = np.uint32
U64 = np.uint64
F32 = np.float32

# Philox4x32 multipliers and Weyl key increments (Salmon et al., SC'11).
PHILOX_M0 = U64(0xD2511F53)
PHILOX_M1 = U64(0xCD9E8D57)
PHILOX_W0 = U32(0x9E3779B9)
PHILOX_W1 = U32(0xBB67AE85)
MASK32 = U64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds.  c0..c3: uint32 arrays (broadcastable),
    k0, k1: uint32 scalars.  Returns four uint32 arrays."""
    c0 = np.asarray(c0, dtype=U32)
    c1 = np.asarray(c1, dtype=U32)
    c2 = np.asarray(c2, dtype=U32)
    c3 = np.asarray(c3, dtype=U32)
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = U32(k0)
    k1 = U32(k1)
    with np.errstate(over="ignore"):
        for rnd in range(10):
            p0 = c0.astype(U64) * PHILOX_M0
            p1 = c2.astype(U64) * PHILOX_M1
            hi0 = (p0 >> U64(32)).astype(U32)
            lo0 = (p0 & MASK32).astype(U32)
            hi1 = (p1 >> U64(32)).astype(U32)
            lo1 = (p1 & MASK32).astype(U32)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
            if rnd != 9:
                k0 = U32((int(k0) + int(PHILOX_W0)) & 0xFFFFFFFF)
                k1 = U32((int(k1) + int(PHILOX_W1)) & 0xFFFFFFFF)
    return c0, c1, c2, c3


def uniform_open01(w):
    """uint32 word -> float32 in (0, 1): (2*(w>>9)+1) * 2^-24, exact."""
    m = (np.asarray(w, dtype=U32) >> U32(9)).astype(np.int64)
    return (2 * m + 1).astype(F32) * F32(2.0 ** -24)


# float32 constants (correctly rounded values of the stated rationals).
_INV_ODD = [F32(float.fromhex(h)) for h in (
    "0x1.745d18p-4",   # 1/11
    "0x1.c71c72p-4",   # 1/9
    "0x1.24924ap-3",   # 1/7
    "0x1.99999ap-3",   # 1/5
    "0x1.555556p-2",   # 1/3
)]
_LN2_HI = F32(float.fromhex("0x1.62e4p-1"))      # 45426/65536, 16 significant bits
_LN2_LO = F32(float.fromhex("0x1.7f7d1cp-20"))   # float32(ln 2 - LN2_HI)
_SQRT2 = F32(float.fromhex("0x1.6a09e6p+0"))     # float32(sqrt 2)
_PIO2 = F32(float.fromhex("0x1.921fb6p+0"))      # float32(pi/2)
# 1/k! for the sine (k = 13, 11, 9, 7, 5, 3) and cosine (k = 14, ..., 2) series
_SIN_C = [F32(float.fromhex(h)) for h in (
    "0x1.612462p-33", "-0x1.ae6456p-26", "0x1.71de3ap-19",
    "-0x1.a01a02p-13", "0x1.111112p-7", "-0x1.555556p-3")]
_COS_C = [F32(float.fromhex(h)) for h in (
    "-0x1.93974ap-37", "0x1.1eed8ep-29", "-0x1.27e4fcp-22", "0x1.a01a02p-16",
    "-0x1.6c16c2p-10", "0x1.555556p-5", "-0x1.0p-1")]


def ln_f32(u):
    """Natural log of float32 u > 0 (normal), separately rounded float32 ops."""
    u = np.asarray(u, dtype=F32)
    bits = u.view(U32)
    e = ((bits >> U32(23)) & U32(0xFF)).astype(np.int32) - 127
    m = ((bits & U32(0x7FFFFF)) | U32(0x3F800000)).view(F32)
    big = m > _SQRT2
    m = np.where(big, m * F32(0.5), m).astype(F32)
    e = np.where(big, e + 1, e)
    s = (m - F32(1.0)) / (m + F32(1.0))
    z = s * s
    poly = _INV_ODD[0]
    for c in _INV_ODD[1:]:
        poly = poly * z + c
    p = (s * z) * poly
    lnm = F32(2.0) * (s + p)
    ef = e.astype(F32)
    return (ef * _LN2_HI + (lnm + ef * _LN2_LO)).astype(F32)


def cos_sin_2pi_f32(u):
    """(cos 2 pi u, sin 2 pi u) for float32 u in [0, 1)."""
    u = np.asarray(u, dtype=F32)
    t = u * F32(4.0)
    q = np.floor(t).astype(np.int32) & 3
    r = t - np.floor(t).astype(F32)
    phi = r * _PIO2
    z = phi * phi
    ps = _SIN_C[0]
    for c in _SIN_C[1:]:
        ps = ps * z + c
    s = phi + (phi * z) * ps
    pc = _COS_C[0]
    for c in _COS_C[1:]:
        pc = pc * z + c
    c = F32(1.0) + z * pc
    cos_t = np.select([q == 0, q == 1, q == 2], [c, -s, -c], s).astype(F32)
    sin_t = np.select([q == 0, q == 1, q == 2], [s, c, -s], -c).astype(F32)
    return cos_t, sin_t


def box_muller_f32(wa, wb, scale):
    """Two uint32 words -> complex Gaussian (re, im) in float32 times scale."""
    u1 = uniform_open01(wa)
    u2 = uniform_open01(wb)
    lg = ln_f32(u1)
    rho = np.sqrt(F32(-2.0) * lg).astype(F32)
    c, s = cos_sin_2pi_f32(u2)
    z1 = rho * c
    z2 = rho * s
    sc = np.asarray(scale, F32)
    return (sc * z1).astype(F32), (sc * z2).astype(F32)


def noise_scale(var):
    """float32(sqrt(var/2)): per-quadrature standard deviation for E|xi|^2=var."""
    return F32(np.sqrt(np.float64(var) / 2.0))


def _words(sites, ncomp, instance, step, seed):
    """Philox words of each site: two components use the counter `site` and
    words (w0, w1) for xi_+ and (w2, w3) for xi_-; one component uses the
    counter site >> 1 and words (w0, w1) for the even and (w2, w3) for the
    odd site of the pair, so that one Philox call serves two sites."""
    sites = np.asarray(sites).astype(np.uint64)
    ctr = (sites if ncomp == 2 else sites >> np.uint64(1)).astype(U32)
    w0, w1, w2, w3 = philox4x32_10(ctr, U32(instance), U32(step & 0xFFFFFFFF),
                                   U32(step >> 32), seed & 0xFFFFFFFF, seed >> 32)
    if ncomp == 2:
        return (w0, w1), (w2, w3)
    odd = (sites & np.uint64(1)).astype(bool)
    return (np.where(odd, w2, w0), np.where(odd, w3, w1)), None


def noise_field(seed, step, instance, ncomp, ny, nx, var):
    """Noise xi_c(site) added after RK4 step `step` (0-based): float32 arrays
    re, im of shape (ncomp, ny, nx)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    step = int(step) & 0xFFFFFFFFFFFFFFFF
    site = np.arange(ny * nx, dtype=np.uint64).reshape(ny, nx)
    a, b = _words(site, ncomp, instance, step, seed)
    sc = noise_scale(var)
    re = np.empty((ncomp, ny, nx), F32)
    im = np.empty((ncomp, ny, nx), F32)
    re[0], im[0] = box_muller_f32(a[0], a[1], sc)
    if ncomp == 2:
        re[1], im[1] = box_muller_f32(b[0], b[1], sc)
    return re, im


def noise_field_scaled(seed, step, instance, ncomp, ny, nx, scale):
    """As noise_field with a per-site, per-component float32 scale array of
    shape (ncomp, ny, nx) (the per-quadrature standard deviation)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    step = int(step) & 0xFFFFFFFFFFFFFFFF
    site = np.arange(ny * nx, dtype=np.uint64).reshape(ny, nx)
    a, b = _words(site, ncomp, instance, step, seed)
    scale = np.asarray(scale, F32)
    re = np.empty((ncomp, ny, nx), F32)
    im = np.empty((ncomp, ny, nx), F32)
    re[0], im[0] = box_muller_f32(a[0], a[1], scale[0])
    if ncomp == 2:
        re[1], im[1] = box_muller_f32(b[0], b[1], scale[1])
    return re, im


def noise_at_scaled(seed, step, instance, sites, ncomp, scale):
    """As noise_at with a per-site, per-component float32 scale array of
    shape (ncomp,) + sites.shape."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    step = int(step) & 0xFFFFFFFFFFFFFFFF
    sites = np.asarray(sites).astype(np.uint64)
    a, b = _words(sites, ncomp, instance, step, seed)
    scale = np.asarray(scale, F32).reshape((ncomp,) + sites.shape)
    re = np.empty((ncomp,) + sites.shape, F32)
    im = np.empty((ncomp,) + sites.shape, F32)
    re[0], im[0] = box_muller_f32(a[0], a[1], scale[0])
    if ncomp == 2:
        re[1], im[1] = box_muller_f32(b[0], b[1], scale[1])
    return re, im


def noise_at(seed, step, instance, sites, ncomp, var):
    """Noise for arbitrary global site indices (uint32 array): float32 arrays
    re, im of shape (ncomp,) + sites.shape."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    step = int(step) & 0xFFFFFFFFFFFFFFFF
    sites = np.asarray(sites).astype(np.uint64)
    a, b = _words(sites, ncomp, instance, step, seed)
    sc = noise_scale(var)
    re = np.empty((ncomp,) + sites.shape, F32)
    im = np.empty((ncomp,) + sites.shape, F32)
    re[0], im[0] = box_muller_f32(a[0], a[1], sc)
    if ncomp == 2:
        re[1], im[1] = box_muller_f32(b[0], b[1], sc)
    return re, im
