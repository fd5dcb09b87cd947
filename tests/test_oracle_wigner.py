"""Pins of the oracle's truncated-Wigner mode (Sec. V, Example 4): noise
with <dW dW*> = nu (R n + gamma_c) delta / (2 dV) per unit time, and the
renormalised density |psi|^2 - 1/dV in the Kerr and depletion terms."""
import numpy as np

from oracle import gp, noise

HB = gp.HBAR


def rk4_amplification(z):
    """RK4 stability polynomial of y' = lambda y at z = lambda dt."""
    return 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24


def test_vacuum_noise_is_half_a_particle_per_mode():
    """Pure loss gamma_c plus Wigner noise (nu = 1, no coupling between sites):
    psi_{k+1} = A psi_k + xi_k with E|xi|^2 = gamma dt / (2 dV), so the
    stationary <|psi|^2> is E|xi|^2 / (1 - A^2), which tends to 1/(2 dV) --
    the half quantum of the Wigner representation's vacuum -- as dt -> 0;
    and <psi^2> = 0 (no preferred phase)."""
    gam, dt = 0.5, 0.05
    p = gp.Params(nx=32, ny=32, lx=32.0, ly=32.0, kappa=0.0, gamma_c=gam, dt=dt,
                  wigner_nu=1.0, seed=3)
    dV = p.dx * p.dy
    psi = np.zeros((1, 32, 32), complex)
    acc, acc2, cnt = 0.0, 0.0, 0
    for k in range(3000):
        psi, _ = gp.run(psi, None, None, None, p, 1, step0=k)
        if k >= 1000:
            acc += float(np.mean(np.abs(psi) ** 2))
            acc2 += complex(np.mean(psi ** 2))
            cnt += 1
    A = rk4_amplification(-0.5 * gam * dt)
    exact = gam * dt / (2 * dV) / (1 - A * A)
    assert abs(acc / cnt - exact) < 0.03 * exact, (acc / cnt, exact)
    assert abs(exact - 1 / (2 * dV)) < 0.02 / (2 * dV)  # O(gamma dt) from 1/(2 dV)
    assert abs(acc2 / cnt) < 0.03 * exact


def test_noise_variance_follows_density():
    """The per-site increment variance is nu (R n + gamma_c) dt / (2 dV) (+ the
    fixed noise_var): checked on the sample variance of one step from psi = 0
    with kappa = 0, on a reservoir that is uniform in each half of the grid."""
    p = gp.Params(nx=64, ny=64, lx=32.0, ly=32.0, kappa=0.0, reservoir=True, R=0.2,
                  gamma_c=0.1, dt=0.02, wigner_nu=2.0, noise_var=1e-4, seed=9)
    n = np.zeros((1, 64, 64))
    n[0, :, 32:] = 3.0
    sc = gp.wigner_scale(n, p)
    dV = p.dx * p.dy
    for half, nv in ((slice(0, 32), 0.0), (slice(32, 64), 3.0)):
        want = p.wigner_nu * (p.R * nv + p.gamma_c) * p.dt / (2 * dV) + p.noise_var
        assert abs(2 * float(sc[0, 0, half][0]) ** 2 - want) < 1e-6 * want
    # a step from psi = 0 with P = 0: psi = xi exactly, so its sample variance
    re, im = noise.noise_field_scaled(p.seed, 0, 0, 1, 64, 64, sc)
    psi, _ = gp.run(np.zeros((1, 64, 64), complex), n, np.zeros((1, 64, 64)), None, p, 1)
    assert np.array_equal(psi.real, re.astype(np.float64))
    assert np.array_equal(psi.imag, im.astype(np.float64))
    for half, nv in ((slice(0, 32), 0.0), (slice(32, 64), 3.0)):
        want = p.wigner_nu * (p.R * nv + p.gamma_c) * p.dt / (2 * dV) + p.noise_var
        got = float(np.mean(np.abs(psi[0, :, half]) ** 2))
        assert abs(got - want) < 0.06 * want, (got, want)


def test_renormalised_uniform_condensate():
    """Deterministic part with the renormalised density: a uniform pump
    above threshold relaxes to n = gamma_c/R and
    |psi|^2 - 1/dV = (P/n - gamma_r)/R, rotating at (g (|psi|^2 - 1/dV) + g_r n)/hbar."""
    p = gp.Params(nx=4, ny=4, lx=2.0, ly=2.0, reservoir=True, g=6e-3, g_r=1.2e-2,
                  R=0.01, gamma_c=0.15, gamma_r=0.225, dt=0.05, wigner_nu=1.0)
    dV = p.dx * p.dy
    Pv = 2.0 * gp.pump_threshold(p)
    P = np.full((1, 4, 4), Pv)
    psi, n = np.full((1, 4, 4), 1.5 + 0j), np.zeros((1, 4, 4))
    for _ in range(12000):
        psi, n = gp.rk4_step(psi, n, P, None, p)  # no noise: the deterministic map
    n_s = p.gamma_c / p.R
    d_s = (Pv / n_s - p.gamma_r) / p.R + 1.0 / dV
    assert np.allclose(n, n_s, rtol=1e-6)
    assert np.allclose(np.abs(psi) ** 2, d_s, rtol=1e-6)
    # one more step rotates the phase by the renormalised frequency
    psi2, _ = gp.rk4_step(psi, n, P, None, p)
    om = -np.angle(psi2[0, 0, 0] / psi[0, 0, 0]) / p.dt
    assert abs(om - (p.g * (d_s - 1 / dV) + p.g_r * n_s) / HB) < 1e-5


def test_wigner_off_is_the_plain_equation():
    p = gp.Params(nx=6, ny=5, lx=3.0, ly=2.5, reservoir=True, g=0.1, g_r=0.2, R=0.3,
                  gamma_c=0.2, gamma_r=0.4, dt=0.01)
    rng = np.random.default_rng(0)
    psi = rng.normal(size=(1, 5, 6)) + 1j * rng.normal(size=(1, 5, 6))
    n = rng.uniform(0, 1, (1, 5, 6))
    P = rng.uniform(0, 1, (1, 5, 6))
    a = gp.rhs(psi, n, P, None, p)
    b = gp.rhs(psi, n, P, None, p.with_(wigner_nu=0.0))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    c = gp.rhs(psi, n, P, None, p.with_(wigner_nu=0.5))
    # the renormalisation is independent of nu's value (only its sign)
    d = gp.rhs(psi, n, P, None, p.with_(wigner_nu=2.0))
    assert np.array_equal(c[0], d[0]) and not np.array_equal(a[0], c[0])
