"""Pins of the oracle's split-step Fourier method (Strang splitting with
exact local and spectral kinetic propagators)."""
import numpy as np

from oracle import gp

HB = gp.HBAR


def test_plane_wave_kinetic_phase_is_exact():
    """Free field: exp(i k.r) only acquires exp(-i kappa k^2 t / hbar), for
    any dt (the kinetic propagator is exact in Fourier space)."""
    p = gp.Params(nx=16, ny=10, lx=8.0, ly=5.0, kappa=0.67, dt=0.37)
    x = np.arange(16) * p.dx
    y = np.arange(10) * p.dy
    kx, ky = 2 * np.pi * 3 / 8.0, -2 * np.pi * 2 / 5.0
    w = np.exp(1j * (kx * x[None, :] + ky * y[:, None]))[None]
    out = gp.run_ssf(w, None, p, 7)
    want = w * np.exp(-1j * 0.67 * (kx ** 2 + ky ** 2) * 7 * 0.37 / HB)
    assert np.abs(out - want).max() < 1e-12


def test_uniform_nonlinear_lossy_state_is_exact():
    """Uniform psi: the kinetic step is the identity and the local step solves
    psi' = (-(i/hbar) g |psi|^2 - gamma/2) psi exactly:
    psi(t) = psi0 e^{-gamma t/2} exp(-(i/hbar) g |psi0|^2 (1 - e^{-gamma t})/gamma)."""
    g, gam, dt, n = 0.4, 0.3, 0.21, 13
    p = gp.Params(nx=6, ny=4, lx=3.0, ly=2.0, g=g, gamma_c=gam, dt=dt)
    psi0 = 1.3 - 0.4j
    out = gp.run_ssf(np.full((1, 4, 6), psi0), None, p, n)
    t = n * dt
    want = psi0 * np.exp(-gam * t / 2) * np.exp(-1j / HB * g * abs(psi0) ** 2 * (1 - np.exp(-gam * t)) / gam)
    assert np.abs(out - want).max() < 1e-13


def spectral_rk4(psi, V, p, T, dt):
    """Independent reference: RK4 with small dt on the same PDE, Laplacian
    evaluated spectrally (FFT derivative)."""
    kx = 2 * np.pi * np.fft.fftfreq(p.nx, p.dx)
    ky = 2 * np.pi * np.fft.fftfreq(p.ny, p.dy)
    k2 = ky[:, None] ** 2 + kx[None, :] ** 2

    def f(u):
        kin = np.fft.ifft2(k2 * np.fft.fft2(u))  # -Lap u
        return -1j / HB * (p.kappa * kin + (V + p.g * np.abs(u) ** 2) * u) - 0.5 * p.gamma_c * u

    u = psi.copy()
    for _ in range(int(round(T / dt))):
        a = f(u)
        b = f(u + 0.5 * dt * a)
        c = f(u + 0.5 * dt * b)
        d = f(u + dt * c)
        u = u + dt * (a + 2 * b + 2 * c + d) / 6
    return u


def test_second_order_against_spectral_rk4():
    """Against an independent spectral RK4 reference of the same equation the
    split-step error falls about 4x per halving of dt (Strang: 2nd order)."""
    nx, ny, L = 32, 24, 8.0
    p = gp.Params(nx=nx, ny=ny, lx=L, ly=L * ny / nx, kappa=0.67, g=0.3, gamma_c=0.2)
    x = np.arange(nx) * p.dx
    y = np.arange(ny) * p.dy
    psi = (np.exp(-((x[None, :] - 4) ** 2 + (y[:, None] - 3) ** 2) / 2.0)
           * np.exp(1j * 2 * np.pi * x[None, :] / L)).astype(complex)
    V = 0.5 * np.cos(2 * np.pi * x[None, :] / L) * np.cos(2 * np.pi * y[:, None] / p.ly)
    T = 0.8
    ref = spectral_rk4(psi, V, p, T, 0.0005)
    errs = []
    for dt in (0.04, 0.02, 0.01):
        out = gp.run_ssf(psi[None], V, p.with_(dt=dt), int(round(T / dt)))[0]
        errs.append(np.linalg.norm(out - ref) / np.linalg.norm(ref))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs
    assert errs[2] < 1e-3


def test_conservative_steps_keep_the_norm():
    rng = np.random.default_rng(5)
    p = gp.Params(nx=20, ny=14, lx=6.0, ly=4.2, g=0.5, dt=0.05)
    psi = rng.normal(size=(1, 14, 20)) + 1j * rng.normal(size=(1, 14, 20))
    V = rng.uniform(-1, 1, (14, 20))
    out = gp.run_ssf(psi, V, p, 40)
    assert abs(np.linalg.norm(out) / np.linalg.norm(psi) - 1) < 1e-13


def spinor_plane(p, mx, my, sign):
    """Eigen-spinor (1, sign u*) e^{i k.r} of the spectral TE-TM block."""
    kx, ky = 2 * np.pi * mx / p.lx, 2 * np.pi * my / p.ly
    x = np.arange(p.nx) * p.dx
    y = np.arange(p.ny) * p.dy
    w = np.exp(1j * (kx * x[None, :] + ky * y[:, None]))
    k2 = kx * kx + ky * ky
    u = -((kx - 1j * ky) ** 2) / k2
    return np.stack([w, sign * np.conj(u) * w]), k2


def test_tetm_eigen_spinors_rotate_at_their_energies():
    """Free spinor field with TE-TM splitting: (1, +-u*) e^{ik.r} acquires
    exp(-i (kappa +- Delta_LT) k^2 t / hbar) exactly -- the two TE and TM
    branches of the splitting; a wrong sign or conjugation of J mixes them."""
    p = gp.Params(nx=16, ny=12, lx=8.0, ly=6.0, spinor=True, kappa=0.67, delta_lt=0.2, dt=0.21)
    for mx, my in [(2, 1), (-3, 2), (1, -4)]:
        for sign in (1, -1):
            v, k2 = spinor_plane(p, mx, my, sign)
            out = gp.run_ssf(v, None, p, 5)
            want = v * np.exp(-1j * (0.67 + sign * 0.2) * k2 * 5 * 0.21 / HB)
            assert np.abs(out - want).max() < 1e-12, (mx, my, sign)


def test_spinor_local_step_is_exact():
    """Uniform spinor, g, g_x and loss: each component keeps its density
    ratio and rotates by (g|psi_c|^2 + g_x|psi_o|^2)(1 - e^{-gamma t})/(gamma hbar)."""
    g, gx, gam, dt, n = 0.4, 0.15, 0.3, 0.2, 9
    p = gp.Params(nx=4, ny=4, lx=2.0, ly=2.0, spinor=True, g=g, g_x=gx, gamma_c=gam, dt=dt)
    a, b = 1.1 + 0.2j, -0.5 + 0.7j
    psi = np.stack([np.full((4, 4), a), np.full((4, 4), b)])
    out = gp.run_ssf(psi, None, p, n)
    t = n * dt
    F = (1 - np.exp(-gam * t)) / gam
    for c, (z, o) in enumerate(((a, b), (b, a))):
        want = z * np.exp(-gam * t / 2) * np.exp(-1j / HB * (g * abs(z) ** 2 + gx * abs(o) ** 2) * F)
        assert np.abs(out[c] - want).max() < 1e-13


def test_spinor_split_step_agrees_with_the_rk4_path():
    """A smooth spinor packet with TE-TM splitting, cross-Kerr and loss: the
    split-step (spectral) and the RK4 (finite-difference) paths agree to
    their discretisation errors, which ties the spectral J to the stencil's
    sign conventions."""
    n, L = 64, 16.0
    p = gp.Params(nx=n, ny=n, lx=L, ly=L, spinor=True, kappa=0.67, g=0.05, g_x=0.02,
                  gamma_c=0.1, delta_lt=0.5)
    p = p.with_(dt=0.2 * gp.stability_dt_max(p))
    x = (np.arange(n) - n // 2) * p.dx
    env = np.exp(-(x[None, :] ** 2 + x[:, None] ** 2) / 8.0)
    psi = np.stack([env * np.exp(0.6j * x[None, :]), 0.5 * env * np.exp(-0.4j * x[:, None])])
    steps = int(1.0 / p.dt)  # 1 ps: the TE-TM coupling turns the state by O(1)
    a = gp.run_ssf(psi, None, p, steps)
    b, _ = gp.run(psi, None, None, None, p, steps)
    nb = np.linalg.norm(b)
    assert np.linalg.norm(a - b) / nb < 0.02
    # the coupling matters at this scale (with it switched off they differ by O(1);
    # with its sign flipped, by ~0.9)
    a0 = gp.run_ssf(psi, None, p.with_(delta_lt=0.0), steps)
    assert np.linalg.norm(a0 - b) / nb > 0.3
    # and the spinor split-step keeps the norm without loss
    q = p.with_(gamma_c=0.0)
    c = gp.run_ssf(psi, None, q, 40)
    assert abs(np.linalg.norm(c) / np.linalg.norm(psi) - 1) < 1e-12


def test_reservoir_split_step_relaxes_to_the_uniform_condensate():
    """Uniform pump above threshold: the reservoir split-step relaxes to
    n = gamma_c / R and |psi|^2 = (P/n - gamma_r)/R (the closed-form stationary
    state of Eqs. PULSE_psi/res), like the RK4 path."""
    p = gp.Params(nx=4, ny=4, lx=2.0, ly=2.0, reservoir=True, g=6e-3, g_r=1.2e-2,
                  R=0.01, gamma_c=0.15, gamma_r=0.225, dt=0.05)
    Pv = 2.0 * gp.pump_threshold(p)
    P = np.full((1, 4, 4), Pv)
    psi, n = gp.run_ssf_reservoir(np.full((1, 4, 4), 1.5 + 0j), np.zeros((1, 4, 4)), P, None,
                                  p, 12000)
    n_s = p.gamma_c / p.R
    assert np.allclose(n, n_s, rtol=1e-6)
    assert np.allclose(np.abs(psi) ** 2, (Pv / n_s - p.gamma_r) / p.R, rtol=1e-6)


def spectral_rk4_reservoir(psi, n, P, V, p, T, dt):
    """Independent reference: RK4 with small dt, spectral Laplacian."""
    kx = 2 * np.pi * np.fft.fftfreq(p.nx, p.dx)
    ky = 2 * np.pi * np.fft.fftfreq(p.ny, p.dy)
    k2 = ky[:, None] ** 2 + kx[None, :] ** 2

    def f(u, m):
        kin = np.fft.ifft2(k2 * np.fft.fft2(u))
        fu = -1j / HB * (p.kappa * kin + (V + p.g * np.abs(u) ** 2 + p.g_r * m) * u) \
            + 0.5 * (p.R * m - p.gamma_c) * u
        fm = P - (p.gamma_r + p.R * np.abs(u) ** 2) * m
        return fu, fm

    u, m = psi.copy(), n.copy()
    for _ in range(int(round(T / dt))):
        a = f(u, m)
        b = f(u + 0.5 * dt * a[0], m + 0.5 * dt * a[1])
        c = f(u + 0.5 * dt * b[0], m + 0.5 * dt * b[1])
        d = f(u + dt * c[0], m + dt * c[1])
        u = u + dt * (a[0] + 2 * b[0] + 2 * c[0] + d[0]) / 6
        m = m + dt * (a[1] + 2 * b[1] + 2 * c[1] + d[1]) / 6
    return u, m


def test_reservoir_split_step_is_second_order():
    nx, ny, L = 32, 24, 8.0
    p = gp.Params(nx=nx, ny=ny, lx=L, ly=L * ny / nx, reservoir=True, kappa=0.67, g=0.3,
                  g_r=0.5, R=0.3, gamma_c=0.2, gamma_r=0.4)
    x = np.arange(nx) * p.dx
    y = np.arange(ny) * p.dy
    psi = (np.exp(-((x[None, :] - 4) ** 2 + (y[:, None] - 3) ** 2) / 2.0)
           * np.exp(1j * 2 * np.pi * x[None, :] / L)).astype(complex)
    n = 0.5 + 0.3 * np.cos(2 * np.pi * y[:, None] / p.ly) * np.ones((ny, nx))
    P = 0.8 + 0.4 * np.sin(2 * np.pi * x[None, :] / L) * np.ones((ny, nx))
    V = 0.5 * np.cos(2 * np.pi * x[None, :] / L) * np.cos(2 * np.pi * y[:, None] / p.ly)
    T = 0.8
    ref_u, ref_m = spectral_rk4_reservoir(psi, n, P, V, p, T, 0.0005)
    errs = []
    for dt in (0.04, 0.02, 0.01):
        u, m = gp.run_ssf_reservoir(psi[None], n[None], P[None], V, p.with_(dt=dt),
                                    int(round(T / dt)))
        errs.append(np.linalg.norm(u[0] - ref_u) / np.linalg.norm(ref_u)
                    + np.linalg.norm(m[0] - ref_m) / np.linalg.norm(ref_m))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs
