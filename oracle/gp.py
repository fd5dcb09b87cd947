"""FP64 oracle for the RK4 time step of the extended dNLSE (PHOENIX).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``): never imported by the
product path.

What it computes, in the paper's order and notation:

* Eq. (PULSE_psi), Sec. V, with coherent drive E = 0 and the noise dW applied
  separately after each step (``noise``):
      dpsi_c/dt = -(i/hbar) [ -(hbar^2/2m) Lap psi_c + (V + g|psi_c|^2
                  + g_x|psi_o|^2 + g_r n_c) psi_c + J_c psi_o ]
                  + (1/2)(R n_c - gamma_c) psi_c
  for c in {+} (scalar) or {+, -} (spinor; o is the other component), with
  J_+ = Delta_LT (d_x - i d_y)^2 and J_- = Delta_LT (d_x + i d_y)^2.
  Eq. (1) is the case without reservoir and spinor.
* Eq. (PULSE_res): dn_c/dt = P_c - (gamma_r + R|psi_c|^2) n_c.
* Laplacian: the 5-point central-difference stencil of Sec. III.B.6
  (performance-modelling subsection).  (d_x -/+ i d_y)^2 = Dxx - Dyy -/+ 2i Dxy,
  with 3-point Dxx, Dyy and the 4-corner Dxy (reading: the paper gives no
  discretisation for the TE-TM term).
* RK4: Eqs. (rk4_K1)-(rk4_final) applied to the joint state (psi, n); the
  time derivative f is read as dpsi/dt (the printed "f = -(i/hbar) d_t psi"
  is garbled; Listing 2 adds g|psi|^2 (-i psi)/hbar and -gamma psi/2 to it).
* Boundary conditions (Sec. V, symbols paragraph): x and y independently
  periodic (wrap) or zero (psi = 0 outside the grid).

Arrays: psi (ncomp, ny, nx) complex128, n / P (ncomp, ny, nx) float64,
V (ny, nx) float64; x is the fastest index, site = j*nx + i.
"""
from dataclasses import dataclass, field, replace
import numpy as np

from . import noise as _noise

HBAR = 0.6582119569  # meV ps (CODATA 2018 value of hbar in these units)

PERIODIC = 0
ZERO = 1


@dataclass
class Params:
    nx: int
    ny: int
    lx: float                 # um
    ly: float                 # um
    bc_x: int = PERIODIC
    bc_y: int = PERIODIC
    spinor: bool = False
    reservoir: bool = False
    kappa: float = 0.67       # hbar^2/2m, meV um^2
    g: float = 0.0            # meV um^2
    g_x: float = 0.0
    g_r: float = 0.0
    R: float = 0.0            # ps^-1 um^2
    gamma_c: float = 0.0      # ps^-1
    gamma_r: float = 0.0      # ps^-1
    delta_lt: float = 0.0     # meV um^2
    dt: float = 0.0           # ps
    noise_var: float = 0.0    # E|xi|^2 added per site per step
    wigner_nu: float = 0.0    # truncated-Wigner noise intensity nu (0: off)
    drive_omega: float = 0.0  # angular frequency of the coherent drive, rad/ps
    kfilter_kc: float = 0.0   # k-space smoothing cutoff k_c, 1/um (0: off)
    kfilter_order: int = 1    # super-Gaussian order p of the smoothing mask
    kfilter_every: int = 0    # smoothing after every this many steps (0: off)
    seed: int = 0
    instance: int = 0

    @property
    def dx(self):
        return self.lx / self.nx

    @property
    def dy(self):
        return self.ly / self.ny

    @property
    def ncomp(self):
        return 2 if self.spinor else 1

    def with_(self, **kw):
        return replace(self, **kw)


def shift(a, di, dj, p):
    """b[..., j, i] = a[..., j+dj, i+di] with the boundary condition of p."""
    b = a
    if di:
        if p.bc_x == PERIODIC:
            b = np.roll(b, -di, axis=-1)
        else:
            c = np.zeros_like(b)
            if di > 0:
                c[..., :, :-di] = b[..., :, di:]
            else:
                c[..., :, -di:] = b[..., :, :di]
            b = c
    if dj:
        if p.bc_y == PERIODIC:
            b = np.roll(b, -dj, axis=-2)
        else:
            c = np.zeros_like(b)
            if dj > 0:
                c[..., :-dj, :] = b[..., dj:, :]
            else:
                c[..., -dj:, :] = b[..., :dj, :]
            b = c
    return b


def d_xx(a, p):
    return (shift(a, 1, 0, p) + shift(a, -1, 0, p) - 2.0 * a) / p.dx ** 2


def d_yy(a, p):
    return (shift(a, 0, 1, p) + shift(a, 0, -1, p) - 2.0 * a) / p.dy ** 2


def laplacian(a, p):
    """5-point stencil (Sec. III.B.6):
    [a(i+1,j)+a(i-1,j)-2a(i,j)]/dx^2 + [a(i,j+1)+a(i,j-1)-2a(i,j)]/dy^2."""
    return d_xx(a, p) + d_yy(a, p)


def d_xy(a, p):
    """[a(i+1,j+1) - a(i+1,j-1) - a(i-1,j+1) + a(i-1,j-1)] / (4 dx dy)."""
    return (shift(a, 1, 1, p) - shift(a, 1, -1, p) - shift(a, -1, 1, p)
            + shift(a, -1, -1, p)) / (4.0 * p.dx * p.dy)


def tetm(a, sign, p):
    """(d_x + sign*i d_y)^2 a = Dxx a - Dyy a + sign*2i Dxy a."""
    return d_xx(a, p) - d_yy(a, p) + sign * 2j * d_xy(a, p)


def hamiltonian_apply(psi, n, V, p):
    """H psi_c of Eq. (PULSE_psi), the bracket multiplied by -(i/hbar)
    (including the coupling J_c psi_o), per component."""
    out = np.empty_like(psi)
    dens = np.abs(psi) ** 2
    for c in range(p.ncomp):
        loc = p.g * dens[c]
        if V is not None:
            loc = loc + V
        if p.spinor:
            loc = loc + p.g_x * dens[1 - c]
        if p.reservoir:
            loc = loc + p.g_r * n[c]
        h = -p.kappa * laplacian(psi[c], p) + loc * psi[c]
        if p.spinor and p.delta_lt != 0.0:
            # J_+ = Delta_LT (d_x - i d_y)^2 acts on psi_-;
            # J_- = Delta_LT (d_x + i d_y)^2 acts on psi_+.
            sign = -1.0 if c == 0 else 1.0
            h = h + p.delta_lt * tetm(psi[1 - c], sign, p)
        out[c] = h
    return out


def rhs(psi, n, P, V, p, E=None, t=0.0):
    """Time derivatives (f_psi, f_n) of Eqs. (PULSE_psi)/(PULSE_res) at time
    t, without dW.  f_n is None without a reservoir.

    Coherent drive (Sec. V): E is None (E = 0) or the complex amplitude
    E_c(r) (meV) per component, and the drive term inside the bracket of
    Eq. (PULSE_psi) is E_c(r) exp(-i drive_omega t).

    Truncated-Wigner mode (Sec. V, Example 4; wigner_nu > 0): the equations
    are solved for the renormalised density |psi|^2 - 1/dV (dV the cell
    area) in the Kerr, cross-Kerr and reservoir-depletion terms."""
    h = hamiltonian_apply(psi, n, V, p)
    w = 1.0 / (p.dx * p.dy) if p.wigner_nu > 0.0 else 0.0
    if w:
        gsum = p.g + (p.g_x if p.spinor else 0.0)
        h = h - (gsum * w) * psi
    if E is not None:
        h = h + np.asarray(E) * np.exp(-1j * p.drive_omega * t)
    f_psi = -1j / HBAR * h
    for c in range(p.ncomp):
        gain = -0.5 * p.gamma_c
        if p.reservoir:
            gain = gain + 0.5 * p.R * n[c]
        f_psi[c] = f_psi[c] + gain * psi[c]
    f_n = None
    if p.reservoir:
        f_n = np.empty_like(n)
        dens = np.abs(psi) ** 2
        for c in range(p.ncomp):
            f_n[c] = P[c] - (p.gamma_r + p.R * (dens[c] - w)) * n[c]
    return f_psi, f_n


def rk4_step(psi, n, P, V, p, E=None, t=0.0):
    """One deterministic RK4 step from time t, Eqs. (rk4_K1)-(rk4_final):
    K1 = f(t, y), K2 = f(t + dt/2, y + dt/2 K1), K3 = f(t + dt/2, y + dt/2 K2),
    K4 = f(t + dt, y + dt K3), y' = y + (K1 + 2K2 + 2K3 + K4) dt / 6, on
    y = (psi, n); the only explicit time dependence is the drive's phase."""
    dt = p.dt
    th = t + 0.5 * dt
    k1p, k1n = rhs(psi, n, P, V, p, E, t)
    k2p, k2n = rhs(psi + 0.5 * dt * k1p,
                   None if n is None else n + 0.5 * dt * k1n, P, V, p, E, th)
    k3p, k3n = rhs(psi + 0.5 * dt * k2p,
                   None if n is None else n + 0.5 * dt * k2n, P, V, p, E, th)
    k4p, k4n = rhs(psi + dt * k3p,
                   None if n is None else n + dt * k3n, P, V, p, E, t + dt)
    psi_new = psi + (k1p + 2.0 * k2p + 2.0 * k3p + k4p) * dt / 6.0
    n_new = None
    if n is not None:
        n_new = n + (k1n + 2.0 * k2n + 2.0 * k3n + k4n) * dt / 6.0
    return psi_new, n_new


def wigner_scale(n_start, p):
    """Per-site, per-quadrature standard deviation of the truncated-Wigner
    increment, float32: E|xi_c|^2 = noise_var + nu (R n_c + gamma_c) dt / (2 dV)
    (<dW dW*> = (R n + gamma_c) delta / (2 dV) per unit time, Sec. V,
    Example 4; Ito: n_c at the start of the step), evaluated as
    v = ((R n + gamma_c) kw) + noise_var with kw = nu dt / (2 dV), each
    operation rounded to float32, then sqrt(max(v, 0) / 2)."""
    F = np.float32
    kw = F(p.wigner_nu * p.dt / (2.0 * p.dx * p.dy))
    n32 = (np.zeros((p.ncomp, p.ny, p.nx)) if n_start is None else np.asarray(n_start)).astype(F)
    a = (F(p.R) * n32).astype(F)
    b = (a + F(p.gamma_c)).astype(F)
    c = (b * kw).astype(F)
    v = (c + F(p.noise_var)).astype(F)
    v = np.maximum(v, F(0.0))
    return np.sqrt((v * F(0.5)).astype(F)).astype(F)


def add_noise(psi, step, p, fp32_state=False, n_start=None):
    """psi_c += xi_c(seed, step, instance, site) after the deterministic step
    (reading: operator splitting; fixed variance per step, or the
    truncated-Wigner variance of wigner_scale)."""
    if p.noise_var == 0.0 and p.wigner_nu == 0.0:
        return psi
    if p.wigner_nu > 0.0:
        re, im = _noise.noise_field_scaled(p.seed, step, p.instance, p.ncomp, p.ny, p.nx,
                                           wigner_scale(n_start, p))
    else:
        re, im = _noise.noise_field(p.seed, step, p.instance, p.ncomp, p.ny, p.nx,
                                    p.noise_var)
    if fp32_state:
        return (psi.real.astype(np.float32) + re) + 1j * (
            psi.imag.astype(np.float32) + im)
    return psi + (re.astype(np.float64) + 1j * im.astype(np.float64))


def kfilter_mask(p):
    """Smoothing mask of Sec. III.B (shape not given; reading: a
    super-Gaussian low-pass) M(k) = exp(-((k_x^2 + k_y^2) / k_c^2)^p) on the
    grid's angular wavenumbers k = 2 pi m / L, m in FFT order."""
    kx = 2.0 * np.pi * np.fft.fftfreq(p.nx, p.dx)
    ky = 2.0 * np.pi * np.fft.fftfreq(p.ny, p.dy)
    k2 = ky[:, None] ** 2 + kx[None, :] ** 2
    return np.exp(-((k2 / p.kfilter_kc ** 2) ** int(p.kfilter_order)))


def kfilter(psi, p):
    """k-space smoothing (Sec. III.B): FFT of each component, product with
    the mask, inverse FFT (numpy's FFT as the library step)."""
    M = kfilter_mask(p)
    return np.stack([np.fft.ifft2(M * np.fft.fft2(psi[c])) for c in range(psi.shape[0])])


def ssf_local(psi, V, p, tau):
    """Exact solution over time tau of the local part of Eq. (PULSE_psi)
    without reservoir, dpsi_c/dt = (-(i/hbar)(V + g|psi_c|^2 + g_x|psi_o|^2)
    - gamma_c/2) psi_c: every |psi_c|^2 decays as e^{-gamma_c t}, so
    psi_c(tau) = psi_c e^{-gamma_c tau/2} exp(-(i/hbar)(V tau + (g|psi_c|^2 + g_x|psi_o|^2) F)),
    F = (1 - e^{-gamma_c tau})/gamma_c (F = tau without loss)."""
    a = np.abs(psi) ** 2
    if p.gamma_c != 0.0:
        F = -np.expm1(-p.gamma_c * tau) / p.gamma_c
    else:
        F = tau
    out = np.empty_like(psi)
    for c in range(psi.shape[0]):
        dens = p.g * a[c]
        if psi.shape[0] == 2:
            dens = dens + p.g_x * a[1 - c]
        phase = dens * F
        if V is not None:
            phase = phase + V * tau
        out[c] = psi[c] * np.exp(-0.5 * p.gamma_c * tau) * np.exp(-1j / HBAR * phase)
    return out


def ssf_kinetic(psi, p, tau):
    """Exact propagation by the linear part in Fourier space (spectral,
    k = 2 pi m / L, periodic): exp(-(i/hbar) kappa k^2 tau) per component; for
    two components with TE-TM splitting the 2x2 block per k,
    H_k = [[kappa k^2, a], [a*, kappa k^2]], a = -Delta_LT (k_x - i k_y)^2
    (J_+ = Delta_LT (d_x - i d_y)^2 on psi_-), whose exponential is
    e^{-i kappa k^2 tau/hbar} (cos th - i sin th [[0, u], [u*, 0]]),
    th = Delta_LT k^2 tau / hbar, u = a / |a|."""
    kx = 2.0 * np.pi * np.fft.fftfreq(p.nx, p.dx)
    ky = 2.0 * np.pi * np.fft.fftfreq(p.ny, p.dy)
    k2 = ky[:, None] ** 2 + kx[None, :] ** 2
    U = np.exp(-1j / HBAR * p.kappa * k2 * tau)
    f = [np.fft.fft2(psi[c]) for c in range(psi.shape[0])]
    if psi.shape[0] == 2 and p.delta_lt != 0.0:
        kc = kx[None, :] - 1j * ky[:, None]
        with np.errstate(invalid="ignore", divide="ignore"):
            u = np.where(k2 > 0, -(kc ** 2) / k2, 0.0)
        th = p.delta_lt * k2 * tau / HBAR
        c, s = np.cos(th), np.sin(th)
        f = [c * f[0] - 1j * s * u * f[1], c * f[1] - 1j * s * np.conj(u) * f[0]]
    return np.stack([np.fft.ifft2(U * fc) for fc in f])


def run_ssf(psi, V, p, nsteps, step0=0):
    """The split-step Fourier method (conclusions: the conventional
    alternative to RK4 the paper's code also offers; no details given).
    Reading: Strang splitting of a field without reservoir (scalar, or two
    components with cross-Kerr and TE-TM coupling), psi <- L(dt/2) K(dt)
    L(dt/2) psi per step with the exact local (ssf_local) and linear
    (ssf_kinetic) propagators, then the same per-step noise as run().
    Periodic boundaries only."""
    psi = np.array(psi, dtype=np.complex128)
    V = None if V is None else np.asarray(V, dtype=np.float64)
    for k in range(nsteps):
        psi = ssf_local(psi, V, p, 0.5 * p.dt)
        psi = ssf_kinetic(psi, p, p.dt)
        psi = ssf_local(psi, V, p, 0.5 * p.dt)
        psi = add_noise(psi, step0 + k, p)
    return psi


def ssf_local_reservoir(psi, n, P, V, p, tau):
    """Local part of Eqs. (PULSE_psi)/(PULSE_res) with the reservoir (no
    spatial coupling): per site and component
    dpsi_c/dt = (-(i/hbar)(V + g|psi_c|^2 + g_x|psi_o|^2 + g_r n_c) + (R n_c - gamma_c)/2) psi_c,
    dn_c/dt = P_c - (gamma_r + R|psi_c|^2) n_c,
    advanced by one classical RK4 step of length tau (the system has no
    closed form; reading of the split-step method for the reservoir model)."""
    nc = psi.shape[0]

    def f(u, m):
        a = np.abs(u) ** 2
        fu = np.empty_like(u)
        fm = np.empty_like(m)
        for c in range(nc):
            loc = p.g * a[c] + p.g_r * m[c]
            if nc == 2:
                loc = loc + p.g_x * a[1 - c]
            if V is not None:
                loc = loc + V
            fu[c] = -1j / HBAR * loc * u[c] + 0.5 * (p.R * m[c] - p.gamma_c) * u[c]
            fm[c] = P[c] - (p.gamma_r + p.R * a[c]) * m[c]
        return fu, fm

    k1 = f(psi, n)
    k2 = f(psi + 0.5 * tau * k1[0], n + 0.5 * tau * k1[1])
    k3 = f(psi + 0.5 * tau * k2[0], n + 0.5 * tau * k2[1])
    k4 = f(psi + tau * k3[0], n + tau * k3[1])
    return (psi + tau * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0]) / 6,
            n + tau * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1]) / 6)


def run_ssf_reservoir(psi, n, P, V, p, nsteps, step0=0):
    """Split-step Fourier for the reservoir model (reading): Strang splitting
    (psi, n) <- L(dt/2) K(dt) L(dt/2) with the local RK4 step of
    ssf_local_reservoir and the exact spectral linear propagator of
    ssf_kinetic acting on psi (n has no linear spatial part), then the
    per-step noise of run().  Returns (psi, n)."""
    psi = np.array(psi, dtype=np.complex128)
    n = np.array(n, dtype=np.float64)
    P = np.broadcast_to(np.asarray(P, dtype=np.float64), n.shape)
    V = None if V is None else np.asarray(V, dtype=np.float64)
    for k in range(nsteps):
        n_start = n
        psi, n = ssf_local_reservoir(psi, n, P, V, p, 0.5 * p.dt)
        psi = ssf_kinetic(psi, p, p.dt)
        psi, n = ssf_local_reservoir(psi, n, P, V, p, 0.5 * p.dt)
        psi = add_noise(psi, step0 + k, p, n_start=n_start)
    return psi, n


def run_imag(psi, V, p, nsteps):
    """Imaginary-time propagation (named in the conclusions; no details
    given).  Reading: t -> -i tau in the conservative part of Eq. (PULSE_psi)
    without reservoir, split like run_ssf --
    psi_c <- exp(-(V + g|psi_c|^2 + g_x|psi_o|^2) dt/(2 hbar)) psi_c (densities
    frozen within the factor), the linear factor exp(-H_k dt/hbar) in Fourier
    space (kappa k^2, and for two components the TE-TM block of ssf_kinetic:
    e^{-kappa k^2 tau/hbar} (cosh th - sinh th [[0, u], [u*, 0]])), the local
    factor again -- then rescaled to the norm N = dV sum |psi|^2 it had at the
    start.  Loss, gain and noise take no part.  Converges to the ground state
    of the (spectral) Hamiltonian."""
    psi = np.array(psi, dtype=np.complex128)
    V = None if V is None else np.asarray(V, dtype=np.float64)
    N0 = norm(psi, p)
    nc = psi.shape[0]

    def local(u):
        a = np.abs(u) ** 2
        out = np.empty_like(u)
        for c in range(nc):
            ph = p.g * a[c]
            if nc == 2:
                ph = ph + p.g_x * a[1 - c]
            if V is not None:
                ph = ph + V
            out[c] = u[c] * np.exp(-0.5 * p.dt / HBAR * ph)
        return out

    kx = 2.0 * np.pi * np.fft.fftfreq(p.nx, p.dx)
    ky = 2.0 * np.pi * np.fft.fftfreq(p.ny, p.dy)
    k2 = ky[:, None] ** 2 + kx[None, :] ** 2
    K = np.exp(-p.kappa * k2 * p.dt / HBAR)
    mix = nc == 2 and p.delta_lt != 0.0
    if mix:
        kc = kx[None, :] - 1j * ky[:, None]
        with np.errstate(invalid="ignore", divide="ignore"):
            uu = np.where(k2 > 0, -(kc ** 2) / k2, 0.0)
        th = p.delta_lt * k2 * p.dt / HBAR
        ch, sh = np.cosh(th), np.sinh(th)
    for _ in range(nsteps):
        psi = local(psi)
        f = [np.fft.fft2(psi[c]) for c in range(nc)]
        if mix:
            f = [ch * f[0] - sh * uu * f[1], ch * f[1] - sh * np.conj(uu) * f[0]]
        psi = np.stack([np.fft.ifft2(K * fc) for fc in f])
        psi = local(psi)
        psi = psi * np.sqrt(N0 / norm(psi, p))
    return psi


def run(psi, n, P, V, p, nsteps, step0=0, E=None, t0=0.0):
    """nsteps RK4 steps (with noise after each) starting at step index step0
    and time t0 (the time advances by t += dt per step, in FP64).  With
    kfilter_every > 0 the smoothing follows every step k (0-based index)
    with (k + 1) % kfilter_every == 0.
    Returns (psi, n) in FP64."""
    psi = np.array(psi, dtype=np.complex128)
    n = None if n is None else np.array(n, dtype=np.float64)
    P = None if P is None else np.asarray(P, dtype=np.float64)
    V = None if V is None else np.asarray(V, dtype=np.float64)
    if p.reservoir:
        if n is None:
            n = np.zeros((p.ncomp, p.ny, p.nx))
        if P is None:
            P = np.zeros((p.ncomp, p.ny, p.nx))
        elif P.shape[0] != p.ncomp:
            P = np.broadcast_to(P, (p.ncomp, p.ny, p.nx))
    if E is not None:
        E = np.broadcast_to(np.asarray(E, dtype=np.complex128), (p.ncomp, p.ny, p.nx))
    t = t0
    for k in range(nsteps):
        n_start = n
        psi, n = rk4_step(psi, n, P, V, p, E, t)
        psi = add_noise(psi, step0 + k, p, n_start=n_start)
        if p.kfilter_every > 0 and (step0 + k + 1) % p.kfilter_every == 0:
            psi = kfilter(psi, p)
        t = t + p.dt
    return psi, n


# ---------------------------------------------------------------- reductions

def norm(psi, p):
    """N = dV sum_c sum_sites |psi_c|^2."""
    return p.dx * p.dy * float(np.sum(np.abs(psi) ** 2))


def energy(psi, n, V, p):
    """Discrete energy functional whose derivative d E / d psi_c^* is
    dV * (H psi_c) of ``hamiltonian_apply`` (reservoir treated as a frozen
    potential g_r n_c):
    E = dV sum [ sum_c ( Re(psi_c^* (-kappa Lap psi_c)) + (V + g_r n_c)|psi_c|^2
                 + (g/2)|psi_c|^4 ) + g_x |psi_+|^2 |psi_-|^2
                 + Re(psi_+^* J_+ psi_- + psi_-^* J_- psi_+) ]."""
    dens = np.abs(psi) ** 2
    tot = 0.0
    for c in range(p.ncomp):
        kin = np.real(np.conj(psi[c]) * (-p.kappa * laplacian(psi[c], p)))
        loc = 0.5 * p.g * dens[c] ** 2
        if V is not None:
            loc = loc + V * dens[c]
        if p.reservoir:
            loc = loc + p.g_r * n[c] * dens[c]
        tot += float(np.sum(kin + loc))
    if p.spinor:
        tot += float(np.sum(p.g_x * dens[0] * dens[1]))
        if p.delta_lt != 0.0:
            cross = (np.conj(psi[0]) * p.delta_lt * tetm(psi[1], -1.0, p)
                     + np.conj(psi[1]) * p.delta_lt * tetm(psi[0], 1.0, p))
            tot += float(np.sum(np.real(cross)))
    return p.dx * p.dy * tot


def residual(psi, n, P, V, p):
    """Steady-state residual (reading: a stationary condensate rotates as
    exp(-i mu t / hbar), so the global phase rotation is removed):
        K = f_psi(psi, n),  omega* = -Im<psi, K> / ||psi||^2,
        r_psi = ||K + i omega* psi|| / ||psi||   (ps^-1),
        r_n   = ||f_n|| / ||n||.
    <a, b> = sum_c sum_sites conj(a) b.  Returns (r_psi, r_n, omega*)."""
    K, fn = rhs(psi, n, P, V, p)
    spp = float(np.sum(np.abs(psi) ** 2))
    if spp == 0.0:
        r_psi, omega = 0.0, 0.0
    else:
        omega = -float(np.imag(np.sum(np.conj(psi) * K))) / spp
        r_psi = float(np.sqrt(np.sum(np.abs(K + 1j * omega * psi) ** 2) / spp))
    r_n = 0.0
    if p.reservoir:
        snn = float(np.sum(n ** 2))
        sff = float(np.sum(fn ** 2))
        r_n = (float(np.sqrt(sff / snn)) if snn > 0.0
               else (0.0 if sff == 0.0 else float("inf")))
    return r_psi, r_n, omega


# ------------------------------------------------------------------ stability

def linear_spectral_radius(p):
    """Largest |eigenvalue| (meV) of the linear Hermitian part
    -kappa Lap (+ Delta_LT J) on the grid's Fourier modes (brute force).
    Periodic axes: k = 2 pi m / N; zero axes: Dirichlet modes k = pi m/(N+1)
    (reading: for TE-TM with zero BC the Dirichlet modes are used as an
    approximation).  K^2 = (2 - 2 cos k d)/d^2, s = sin(k d)/d; the TE-TM
    block at k has eigenvalues kappa(Kx^2+Ky^2) +- Delta_LT *
    sqrt((Kx^2 - Ky^2)^2 + 4 sx^2 sy^2)."""
    def modes(N, bc):
        if bc == PERIODIC:
            return 2.0 * np.pi * np.arange(N) / N
        return np.pi * np.arange(1, N + 1) / (N + 1)
    # kx, ky below are the dimensionless phases k*dx, k*dy of each mode
    kx = modes(p.nx, p.bc_x)[None, :]
    ky = modes(p.ny, p.bc_y)[:, None]
    Kx2 = (2.0 - 2.0 * np.cos(kx)) / p.dx ** 2
    Ky2 = (2.0 - 2.0 * np.cos(ky)) / p.dy ** 2
    lam = p.kappa * (Kx2 + Ky2)
    if p.spinor and p.delta_lt != 0.0:
        sx = np.sin(kx) / p.dx
        sy = np.sin(ky) / p.dy
        off = abs(p.delta_lt) * np.sqrt((Kx2 - Ky2) ** 2 + 4.0 * sx ** 2 * sy ** 2)
        lam = np.maximum(np.abs(lam + off), np.abs(lam - off))
    return float(np.max(np.abs(lam)))


RK4_IMAG_AXIS_LIMIT = 2.0 * np.sqrt(2.0)  # |R(iy)| <= 1 iff |y| <= 2 sqrt 2


def stability_dt_max(p):
    """Largest dt for which RK4 is stable on the linear Hermitian part:
    dt_max = 2 sqrt(2) hbar / lambda_max (reading: the nonlinear, potential
    and loss terms are excluded)."""
    lam = linear_spectral_radius(p)
    if lam == 0.0:
        return float("inf")
    return RK4_IMAG_AXIS_LIMIT * HBAR / lam


def pump_threshold(p):
    """Homogeneous condensation threshold P_thr = gamma_c gamma_r / R from
    Eq. (PULSE_res) at psi -> 0 (n = P/gamma_r) and Eq. (PULSE_psi) gain
    R n = gamma_c."""
    return p.gamma_c * p.gamma_r / p.R


def step_at_sites(psi, n, P, V, p, sites_ji, step, radius=5, E=None, t=0.0):
    """One RK4 step (plus noise) evaluated only at the given (j, i) sites of
    a large grid.  A step's output at a site depends on the inputs within
    distance 4 (one cell per stage), so each site is computed on its own
    window of radius `radius` >= 5 evolved with zero boundaries: along a
    periodic axis the window wraps; along a zero axis it is cut at the domain
    edge (cells outside the domain stay zero at every stage).
    Returns (psi_c[sites], n_c[sites]) with shape (ncomp, nsites)."""
    nc = p.ncomp
    out_psi = np.empty((nc, len(sites_ji)), complex)
    out_n = np.empty((nc, len(sites_ji))) if p.reservoir else None
    Pb = np.broadcast_to(P, (nc, p.ny, p.nx)) if p.reservoir else None
    Eb = np.broadcast_to(E, (nc, p.ny, p.nx)) if E is not None else None

    def axis(c, N, bc):
        if bc == PERIODIC:
            return np.arange(c - radius, c + radius + 1) % N, radius
        lo, hi = max(c - radius, 0), min(c + radius, N - 1)
        return np.arange(lo, hi + 1), c - lo

    for k, (j, i) in enumerate(sites_ji):
        jj, cj = axis(j, p.ny, p.bc_y)
        ii, ci = axis(i, p.nx, p.bc_x)
        q = p.with_(nx=len(ii), ny=len(jj), lx=len(ii) * p.dx, ly=len(jj) * p.dy,
                    bc_x=ZERO, bc_y=ZERO, noise_var=0.0)
        win = lambda a: a[..., jj[:, None], ii[None, :]]
        a, b = rk4_step(win(psi), win(n) if p.reservoir else None,
                        win(Pb) if p.reservoir else None,
                        win(V) if V is not None else None, q,
                        win(Eb) if E is not None else None, t)
        out_psi[:, k] = a[:, cj, ci]
        if p.reservoir:
            out_n[:, k] = b[:, cj, ci]
    sites = np.array([j * p.nx + i for j, i in sites_ji])
    if p.wigner_nu > 0.0:
        js = np.array([j for j, _ in sites_ji])
        is_ = np.array([i for _, i in sites_ji])
        n_s = n[:, js, is_] if p.reservoir else np.zeros((nc, len(sites_ji)))
        row = p.with_(nx=len(sites_ji), ny=1, lx=len(sites_ji) * p.dx, ly=p.dy)  # same dV
        re, im = _noise.noise_at_scaled(p.seed, step, p.instance, sites, nc,
                                        wigner_scale(n_s, row))
        out_psi = out_psi + (re.astype(np.float64) + 1j * im.astype(np.float64))
    elif p.noise_var != 0.0:
        re, im = _noise.noise_at(p.seed, step, p.instance, sites, nc, p.noise_var)
        out_psi = out_psi + (re.astype(np.float64) + 1j * im.astype(np.float64))
    return out_psi, out_n
