"""Pins of the oracle's coherent drive E_c(r) exp(-i omega t) (Eq. PULSE_psi,
Sec. V) against closed forms of the linear driven, damped equation."""
import numpy as np

from oracle import gp

HB = gp.HBAR


def uniform_exact(E0, gam, om, t):
    """psi' = -(i/hbar) E0 e^{-i om t} - (gam/2) psi, psi(0) = 0:
    psi(t) = A (e^{-i om t} - e^{-gam t/2}), A = -(i/hbar) E0 / (gam/2 - i om)."""
    A = -1j / HB * E0 / (0.5 * gam - 1j * om)
    return A * (np.exp(-1j * om * t) - np.exp(-0.5 * gam * t))


def test_uniform_drive_fourth_order_to_closed_form():
    """A uniform drive on a periodic grid (the Laplacian of a uniform field is
    zero): the RK4 error against the closed form falls 16-fold when dt
    halves -- which fixes the stage times t, t + dt/2, t + dt/2, t + dt of the
    drive's phase -- and the sign of the phase and the -i/hbar factor."""
    E0, gam, om, T = 0.3 - 0.1j, 0.4, -1.7, 6.0
    errs = []
    for dt in (0.1, 0.05):
        p = gp.Params(nx=6, ny=5, lx=3.0, ly=2.5, kappa=0.67, gamma_c=gam, dt=dt,
                      drive_omega=om)
        E = np.full((1, 5, 6), E0)
        psi, _ = gp.run(np.zeros((1, 5, 6), complex), None, None, None, p,
                        int(round(T / dt)), E=E)
        assert np.allclose(psi, psi[0, 0, 0], rtol=0, atol=1e-14)
        errs.append(abs(psi[0, 0, 0] - uniform_exact(E0, gam, om, T)))
    assert errs[1] < 2e-6 * abs(uniform_exact(E0, gam, om, T))
    assert 13.0 < errs[0] / errs[1] < 19.0, errs


def test_plane_wave_drive_steady_state():
    """E = E0 exp(i k.r) with k on the grid drives the single discrete mode:
    psi -> a e^{-i om t} e^{i k.r}, a = -(i/hbar) E0 / (gam/2 + i(eps_k/hbar - om)),
    eps_k = kappa (4 sin^2(k_x dx/2)/dx^2 + 4 sin^2(k_y dy/2)/dy^2).  A
    transposed or mis-placed E, or a drive at the wrong frequency, fails."""
    nx, ny, lx, ly = 12, 9, 6.0, 4.5
    dx, dy = lx / nx, ly / ny
    kx, ky = 2 * np.pi * 2 / lx, 2 * np.pi * 1 / ly
    gam, om, E0 = 1.2, 0.8, 0.05
    p = gp.Params(nx=nx, ny=ny, lx=lx, ly=ly, kappa=0.67, gamma_c=gam, drive_omega=om)
    p = p.with_(dt=0.2 * gp.stability_dt_max(p))
    x = np.arange(nx) * dx
    y = np.arange(ny) * dy
    wave = np.exp(1j * (kx * x[None, :] + ky * y[:, None]))
    steps = int(np.ceil(30.0 / p.dt))  # 36 decay times of the amplitude
    psi, _ = gp.run(np.zeros((1, ny, nx), complex), None, None, None, p, steps,
                    E=(E0 * wave)[None])
    eps = 0.67 * (4 * np.sin(kx * dx / 2) ** 2 / dx ** 2 + 4 * np.sin(ky * dy / 2) ** 2 / dy ** 2)
    a = -1j / HB * E0 / (0.5 * gam + 1j * (eps / HB - om))
    want = a * np.exp(-1j * om * steps * p.dt) * wave
    assert np.abs(psi[0] - want).max() < 1e-6 * abs(a), np.abs(psi[0] - want).max() / abs(a)


def test_spinor_drive_acts_on_its_component():
    """E_- alone drives psi_- by the scalar closed form and leaves psi_+ at
    zero (no cross-Kerr, no TE-TM)."""
    E0, gam, om, dt, T = 0.2, 0.5, 2.3, 0.02, 4.0
    p = gp.Params(nx=4, ny=4, lx=2.0, ly=2.0, spinor=True, gamma_c=gam, dt=dt,
                  drive_omega=om)
    E = np.zeros((2, 4, 4), complex)
    E[1] = E0
    psi, _ = gp.run(np.zeros((2, 4, 4), complex), None, None, None, p, int(round(T / dt)), E=E)
    assert np.all(psi[0] == 0)
    assert abs(psi[1, 2, 3] - uniform_exact(E0, gam, om, T)) < 1e-7


def test_time_origin_carries_over():
    """Two runs of k steps, the second from t0 = k dt and step k, equal one
    run of 2k steps: the drive's phase follows the accumulated time."""
    p = gp.Params(nx=7, ny=6, lx=3.5, ly=3.0, g=0.2, gamma_c=0.3, dt=0.03, drive_omega=3.0)
    rng = np.random.default_rng(1)
    E = (rng.normal(size=(1, 6, 7)) + 1j * rng.normal(size=(1, 6, 7))) * 0.1
    psi0 = rng.normal(size=(1, 6, 7)) + 0j
    a, _ = gp.run(psi0, None, None, None, p, 20, E=E)
    b1, _ = gp.run(psi0, None, None, None, p, 10, E=E)
    t = 0.0
    for _ in range(10):
        t = t + p.dt
    b, _ = gp.run(b1, None, None, None, p, 10, step0=10, E=E, t0=t)
    assert np.array_equal(a, b)


def test_windowed_step_with_drive_equals_full_grid_step():
    """oracle.gp.step_at_sites (the full-size sampled parity) with a drive and
    a time origin equals the full-grid step at every sampled site."""
    import synth
    p = gp.Params(nx=23, ny=19, lx=7.0, ly=6.0, g=0.2, gamma_c=0.1, drive_omega=1.7,
                  noise_var=1e-3, seed=5)
    p = p.with_(dt=0.4 * gp.stability_dt_max(p))
    psi, _, _, V = synth.random_state(1, 19, 23, 11, reservoir=False)
    rng = np.random.default_rng(6)
    E = (rng.normal(size=(1, 19, 23)) + 1j * rng.normal(size=(1, 19, 23))) * 0.2
    t0 = 2.35
    full, _ = gp.run(psi, None, None, V, p, 1, step0=4, E=E, t0=t0)
    sites = [(0, 0), (18, 22), (0, 22), (9, 11), (5, 0)]
    sp, _ = gp.step_at_sites(psi, None, None, V, p, sites, step=4, E=E, t=t0)
    for k, (j, i) in enumerate(sites):
        assert abs(sp[0, k] - full[0, j, i]) < 1e-13
