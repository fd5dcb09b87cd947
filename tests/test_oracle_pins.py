"""Pins of the FP64 oracle (oracle/gp.py) against what the paper and the
mathematics fix: closed forms, invariants, special cases and printed
coefficients.  CPU only."""
import os

import numpy as np
import pytest

from oracle import gp
import synth

HB = gp.HBAR
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def P_(**kw):
    base = dict(nx=16, ny=16, lx=8.0, ly=8.0)
    base.update(kw)
    return gp.Params(**base)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


# ------------------------------------------------------------------ stencil

def test_stencil_matches_printed_weights():
    """Apply the oracle Laplacian to unit impulses and compare with the
    printed 5-point weights (tests/golden/stencil_5pt.txt)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "stencil_5pt.txt"))
            if l.strip() and not l.startswith("#")]
    p = P_(nx=7, ny=9, lx=7 * 0.3, ly=9 * 0.7)
    a = np.zeros((9, 7), complex)
    a[4, 3] = 1.0
    lap = gp.laplacian(a, p)
    expect = np.zeros((9, 7))
    for di, dj, wx, wy in rows:
        # lap(i,j) receives weight from a(i+di, j+dj); with a the impulse at
        # (3,4), lap at (3-di, 4-dj) gets the weight
        expect[4 - int(dj), 3 - int(di)] += float(wx) / p.dx ** 2 + float(wy) / p.dy ** 2
    assert np.allclose(lap.real, expect, rtol=0, atol=1e-12)
    assert np.all(lap.imag == 0)


@pytest.mark.parametrize("nx,ny,lx,ly,mx,my", [(16, 16, 8.0, 8.0, 3, 5),
                                               (24, 10, 5.0, 9.0, 7, 2),
                                               (64, 64, 20.0, 20.0, 32, 31)])
def test_laplacian_plane_wave_eigenvalue(nx, ny, lx, ly, mx, my):
    """Lap_h e^{i k.r} = -[(2-2cos kx dx)/dx^2 + (2-2cos ky dy)/dy^2] e^{i k.r}."""
    p = P_(nx=nx, ny=ny, lx=lx, ly=ly)
    kx, ky = 2 * np.pi * mx / lx, 2 * np.pi * my / ly
    X, Y = np.meshgrid(np.arange(nx) * p.dx, np.arange(ny) * p.dy)
    psi = np.exp(1j * (kx * X + ky * Y))
    lam = -((2 - 2 * np.cos(kx * p.dx)) / p.dx ** 2 + (2 - 2 * np.cos(ky * p.dy)) / p.dy ** 2)
    assert rel(gp.laplacian(psi, p), lam * psi) < 1e-12


def test_zero_bc_laplacian_dirichlet_sine_modes():
    """With zero BC the sine modes sin(pi m (i+1)/(N+1)) are eigenvectors with
    eigenvalue -(2-2cos(pi m/(N+1)))/dx^2 (textbook Dirichlet result)."""
    p = P_(nx=11, ny=6, lx=3.3, ly=2.4, bc_x=gp.ZERO, bc_y=gp.ZERO)
    i = np.arange(11)[None, :]
    j = np.arange(6)[:, None]
    mx, my = 4, 2
    psi = np.sin(np.pi * mx * (i + 1) / 12) * np.sin(np.pi * my * (j + 1) / 7) + 0j
    lam = -((2 - 2 * np.cos(np.pi * mx / 12)) / p.dx ** 2 + (2 - 2 * np.cos(np.pi * my / 7)) / p.dy ** 2)
    assert rel(gp.laplacian(psi, p), lam * psi) < 1e-12


# ------------------------------------------------------------------ RK4

def rk4_poly_from_printed():
    """Stability polynomial of RK4 built from the printed coefficients:
    for y' = z y (dt = 1): K1 = z, K2 = z(1 + c1 K1), ...; returns poly
    coefficients in z."""
    rows = {l.split()[0]: [float(v) for v in l.split()[1:]]
            for l in open(os.path.join(GOLDEN, "rk4_listing1.txt"))
            if l.strip() and not l.startswith("#")}
    c, w = rows["stage_factor"], rows["final_weight"]
    P = np.polynomial.Polynomial
    z = P([0, 1])
    K = [z]
    for ck in c:
        K.append(z * (1 + ck * K[-1]))
    R = 1 + sum(wk * Kk for wk, Kk in zip(w, K))
    return R.coef


def test_rk4_polynomial_from_listing1_is_taylor():
    coef = rk4_poly_from_printed()
    assert np.allclose(coef, [1, 1, 1 / 2, 1 / 6, 1 / 24], atol=1e-15)


def lin_symbol(p, V0=0.0):
    """Per-mode generator (ps^-1) of the linear scalar problem."""
    mx = np.fft.fftfreq(p.nx) * p.nx
    my = np.fft.fftfreq(p.ny) * p.ny
    ax = 2 * np.pi * mx / p.nx
    ay = 2 * np.pi * my / p.ny
    K2 = ((2 - 2 * np.cos(ax)) / p.dx ** 2)[None, :] + ((2 - 2 * np.cos(ay)) / p.dy ** 2)[:, None]
    return -1j / HB * (p.kappa * K2 + V0) - 0.5 * p.gamma_c


def test_linear_rk4_closed_form_fft():
    """Noise-free periodic linear case (g=0, V=const, loss): every Fourier
    mode is multiplied per step by R(z) = 1+z+z^2/2+z^3/6+z^4/24, z = dt*lam_k."""
    p = P_(nx=16, ny=12, lx=6.0, ly=5.0, gamma_c=0.3)
    p = p.with_(dt=0.4 * gp.stability_dt_max(p))
    V0 = 0.7
    V = np.full((12, 16), V0)
    rng = np.random.default_rng(0)
    psi0 = (rng.normal(size=(1, 12, 16)) + 1j * rng.normal(size=(1, 12, 16)))
    steps = 25
    psi, _ = gp.run(psi0, None, None, V, p, steps)
    z = p.dt * lin_symbol(p, V0)
    R = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
    expect = np.fft.ifft2(np.fft.fft2(psi0[0]) * R ** steps)
    assert rel(psi[0], expect) < 1e-12


def naive_dft2(a):
    ny, nx = a.shape
    Fx = np.exp(-2j * np.pi * np.outer(np.arange(nx), np.arange(nx)) / nx)
    Fy = np.exp(-2j * np.pi * np.outer(np.arange(ny), np.arange(ny)) / ny)
    return Fy @ a @ Fx.T


def test_linear_rk4_closed_form_naive_dft_8x8():
    """Same pin with an O(N^4) naive DFT on 8x8 (no FFT library)."""
    p = P_(nx=8, ny=8, lx=4.0, ly=4.0, gamma_c=0.1)
    p = p.with_(dt=0.5 * gp.stability_dt_max(p))
    rng = np.random.default_rng(1)
    psi0 = rng.normal(size=(1, 8, 8)) + 1j * rng.normal(size=(1, 8, 8))
    psi, _ = gp.run(psi0, None, None, None, p, 10)
    z = p.dt * lin_symbol(p)
    R = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
    hat = naive_dft2(psi0[0]) * R ** 10
    inv = np.conj(naive_dft2(np.conj(hat))) / 64
    assert rel(psi[0], inv) < 1e-12


def test_tetm_linear_rk4_block_closed_form():
    """Spinor with TE-TM: per k a 2x2 block A_k; psi_hat advances by the
    matrix polynomial R(dt A_k).  J_+ = Delta (d_x - i d_y)^2 has symbol
    Delta(-Kx^2 + Ky^2 + 2i sx sy) (continuum (i kx + ky)^2 discretised)."""
    nx, ny = 12, 10
    p = P_(nx=nx, ny=ny, lx=5.0, ly=4.0, spinor=True, delta_lt=0.3, gamma_c=0.05)
    p = p.with_(dt=0.45 * gp.stability_dt_max(p))
    rng = np.random.default_rng(2)
    psi0 = rng.normal(size=(2, ny, nx)) + 1j * rng.normal(size=(2, ny, nx))
    steps = 12
    psi, _ = gp.run(psi0, None, None, None, p, steps)
    ax = (2 * np.pi * np.fft.fftfreq(nx))[None, :] * np.ones((ny, 1))
    ay = (2 * np.pi * np.fft.fftfreq(ny))[:, None] * np.ones((1, nx))
    Kx2 = (2 - 2 * np.cos(ax)) / p.dx ** 2
    Ky2 = (2 - 2 * np.cos(ay)) / p.dy ** 2
    sx = np.sin(ax) / p.dx
    sy = np.sin(ay) / p.dy
    Jp = p.delta_lt * (-Kx2 + Ky2 + 2j * sx * sy)
    Jm = p.delta_lt * (-Kx2 + Ky2 - 2j * sx * sy)
    h = p.kappa * (Kx2 + Ky2)
    hat = np.stack([np.fft.fft2(psi0[0]), np.fft.fft2(psi0[1])])
    out = np.empty_like(hat)
    for j in range(ny):
        for i in range(nx):
            A = -1j / HB * np.array([[h[j, i], Jp[j, i]], [Jm[j, i], h[j, i]]]) - 0.5 * p.gamma_c * np.eye(2)
            Z = p.dt * A
            R = np.eye(2) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24
            out[:, j, i] = np.linalg.matrix_power(R, steps) @ hat[:, j, i]
    expect = np.stack([np.fft.ifft2(out[0]), np.fft.ifft2(out[1])])
    assert rel(psi, expect) < 1e-11


def test_exact_nonlinear_plane_wave():
    """psi0 = A e^{ik.r} stays a plane wave: every site equals a_k e^{ik.r}
    where a follows scalar RK4 for a' = -(i/hbar)(kappa K^2 + g|a|^2) a.
    Against the continuum omega = (kappa k^2 + g|A|^2)/hbar the phase error
    is O(dt^4) + O((k dx)^2)."""
    p = P_(nx=32, ny=32, lx=16.0, ly=16.0, g=0.05)
    p = p.with_(dt=0.3 * gp.stability_dt_max(p))
    A = 1.7
    kx, ky = 2 * np.pi * 2 / 16.0, 2 * np.pi * 1 / 16.0
    X, Y = np.meshgrid(np.arange(32) * p.dx, np.arange(32) * p.dy)
    e = np.exp(1j * (kx * X + ky * Y))
    steps = 60
    psi, _ = gp.run((A * e)[None], None, None, None, p, steps)
    K2 = (2 - 2 * np.cos(kx * p.dx)) / p.dx ** 2 + (2 - 2 * np.cos(ky * p.dy)) / p.dy ** 2
    a = complex(A)

    def f(a):
        return -1j / HB * (p.kappa * K2 + p.g * abs(a) ** 2) * a
    for _ in range(steps):
        k1 = f(a)
        k2 = f(a + 0.5 * p.dt * k1)
        k3 = f(a + 0.5 * p.dt * k2)
        k4 = f(a + p.dt * k3)
        a = a + (k1 + 2 * k2 + 2 * k3 + k4) * p.dt / 6
    assert rel(psi[0], a * e) < 1e-12
    # continuum frequency
    t = steps * p.dt
    omega = (p.kappa * (kx ** 2 + ky ** 2) + p.g * A ** 2) / HB
    phase_num = np.angle(psi[0, 0, 0] / A)
    dphi = np.angle(np.exp(1j * (phase_num + omega * t)))
    assert abs(dphi) < 0.02 * omega * t  # (k dx)^2 ~ 0.2 -> ~1.7% phase error
    assert abs(abs(psi[0, 0, 0]) - A) < 1e-3 * A


def gaussian_packet(X, Y, t, A, s2, hbar_over_m):
    q = s2 + 1j * hbar_over_m * t
    return A * s2 / q * np.exp(-(X ** 2 + Y ** 2) / (2 * q))


def test_free_gaussian_packet_second_order_in_dx():
    """g = 0 free packet: psi(r,t) = A s^2/(s^2 + i hbar t/m)
    exp(-r^2/(2(s^2 + i hbar t/m))), hbar/m = 2 kappa/hbar.  Error O(dx^2):
    halving dx divides the error by ~4."""
    errs = []
    t_end = 1.0
    s = 1.0
    for n in (24, 48):
        L = 16.0
        p = P_(nx=n, ny=n, lx=L, ly=L)
        dt0 = 0.25 * gp.stability_dt_max(p)
        steps = int(np.ceil(t_end / dt0))
        p = p.with_(dt=t_end / steps)
        X, Y = synth.mesh(n, n, L, L)
        hm = 2 * p.kappa / HB
        psi0 = gaussian_packet(X, Y, 0.0, 1.0, s * s, hm)
        psi, _ = gp.run(psi0[None], None, None, None, p, steps)
        ex = gaussian_packet(X, Y, t_end, 1.0, s * s, hm)
        errs.append(np.max(np.abs(psi[0] - ex)))
    ratio = errs[0] / errs[1]
    assert 3.5 < ratio < 4.5, (errs, ratio)
    assert errs[1] < 1e-2


def test_conservation_hermitian():
    """R = gamma = P = 0, noise off, smooth state: N and E constant to 1e-10."""
    cfg = synth.conservative_64()
    p = gp.Params(**{k: v for k, v in cfg["params"].items()})
    p = p.with_(dt=p.dt / 10)
    X, Y = synth.mesh(64, 64, 20.0, 20.0)
    psi0 = (5.0 * np.exp(-(X ** 2 + Y ** 2) / 9.0) * np.exp(0.3j * X))[None]
    N0, E0 = gp.norm(psi0, p), gp.energy(psi0, None, None, p)
    psi, _ = gp.run(psi0, None, None, None, p, 300)
    N1, E1 = gp.norm(psi, p), gp.energy(psi, None, None, p)
    assert abs(N1 - N0) / N0 < 1e-10
    assert abs(E1 - E0) / abs(E0) < 1e-10


def test_conservation_hermitian_spinor_tetm():
    p = gp.Params(nx=24, ny=24, lx=12.0, ly=12.0, spinor=True, g=0.02,
                  g_x=0.01, delta_lt=0.1)
    p = p.with_(dt=0.05 * gp.stability_dt_max(p))
    X, Y = synth.mesh(24, 24, 12.0, 12.0)
    psi0 = np.stack([2.0 * np.exp(-(X ** 2 + Y ** 2) / 4.0),
                     1.5j * np.exp(-((X - 1) ** 2 + Y ** 2) / 5.0) * np.exp(0.4j * Y)])
    N0, E0 = gp.norm(psi0, p), gp.energy(psi0, None, None, p)
    psi, _ = gp.run(psi0, None, None, None, p, 200)
    assert abs(gp.norm(psi, p) - N0) / N0 < 1e-10
    assert abs(gp.energy(psi, None, None, p) - E0) / abs(E0) < 1e-10


def test_fourth_order_in_dt():
    """Reservoir and gain on, smooth data on 16x16: the error ratio for
    dt -> dt/2 against a dt/64 reference is 16 within 15%."""
    p = gp.Params(nx=16, ny=16, lx=8.0, ly=8.0, reservoir=True, g=0.3, g_r=0.5,
                  R=0.4, gamma_c=0.2, gamma_r=0.3)
    psi0, n0, P, V = synth.random_state(1, 16, 16, 7, amp=0.5, smooth=True)
    n0 = np.abs(n0) * 0.5
    T = 0.8
    # asymptotic regime: |lambda dt| well inside the RK4 region
    dt = 0.15 * gp.stability_dt_max(p)
    steps = int(np.ceil(T / dt))

    def sol(m):
        q = p.with_(dt=T / (steps * m))
        return gp.run(psi0, n0, P, V, q, steps * m)
    ref_psi, ref_n = sol(64)
    e = []
    for m in (1, 2):
        psi, n = sol(m)
        e.append(np.linalg.norm(psi - ref_psi) + np.linalg.norm(n - ref_n))
    ratio = e[0] / e[1]
    assert 16 * 0.85 < ratio < 16 * 1.15, ratio


# ------------------------------------------------------------ special cases

def test_pure_decay_uniform():
    p = gp.Params(nx=6, ny=5, lx=3.0, ly=2.5, gamma_c=0.4, kappa=0.67, dt=0.3)
    psi0 = np.full((1, 5, 6), 0.8 - 0.3j)
    psi, _ = gp.run(psi0, None, None, None, p, 17)
    z = -0.5 * p.gamma_c * p.dt
    R = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
    assert rel(psi, psi0 * R ** 17) < 1e-13


def test_reservoir_with_zero_field():
    """psi = 0: n_{k+1} = R(z) n_k + dt P (1 + z/2 + z^2/6 + z^3/24),
    z = -gamma_r dt (RK4 of a linear ODE with constant source), -> P/gamma_r."""
    p = gp.Params(nx=5, ny=4, lx=2.0, ly=2.0, reservoir=True, R=0.01,
                  gamma_c=0.15, gamma_r=0.225, g_r=0.012, dt=0.9)
    rng = np.random.default_rng(3)
    P = rng.uniform(1, 5, size=(1, 4, 5))
    n0 = rng.uniform(0, 2, size=(1, 4, 5))
    psi0 = np.zeros((1, 4, 5), complex)
    psi, n = gp.run(psi0, n0, P, None, p, 40)
    z = -p.gamma_r * p.dt
    R = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
    S = p.dt * (1 + z / 2 + z ** 2 / 6 + z ** 3 / 24)
    nk = n0.copy()
    for _ in range(40):
        nk = R * nk + S * P
    assert rel(n, nk) < 1e-13
    assert np.all(psi == 0)
    psi, n = gp.run(psi0, n0, P, None, p, 400)
    assert rel(n, P / p.gamma_r) < 1e-10


def test_uniform_condensate_relaxes_to_stationary_state():
    """Uniform pump above threshold: n -> gamma_c/R, |psi|^2 -> (P/n - gamma_r)/R."""
    p = gp.Params(nx=4, ny=4, lx=2.0, ly=2.0, reservoir=True, g=6e-3, g_r=1.2e-2,
                  R=0.01, gamma_c=0.15, gamma_r=0.225, dt=0.05)
    Pv = 2.0 * gp.pump_threshold(p)
    P = np.full((1, 4, 4), Pv)
    psi0 = np.full((1, 4, 4), 0.1 + 0j)
    psi, n = gp.run(psi0, np.zeros((1, 4, 4)), P, None, p, 12000)
    n_s = p.gamma_c / p.R
    d_s = (Pv / n_s - p.gamma_r) / p.R
    assert np.allclose(n, n_s, rtol=1e-6)
    assert np.allclose(np.abs(psi) ** 2, d_s, rtol=1e-6)
    r_psi, r_n, om = gp.residual(psi, n, P, None, p)
    assert r_psi < 1e-6 and r_n < 1e-6
    # stationary frequency of a uniform state: (g |psi|^2 + g_r n)/hbar
    assert abs(om - (p.g * d_s + p.g_r * n_s) / HB) < 1e-6


# ------------------------------------------------------- energy / residual

@pytest.mark.parametrize("bc", [gp.PERIODIC, gp.ZERO])
def test_energy_derivative_is_hamiltonian(bc):
    """dE/dpsi_c^* (Wirtinger, central differences) = dV (H psi)_c, which also
    checks the discrete TE-TM operator is Hermitian (J_-^dagger = J_+)."""
    p = gp.Params(nx=7, ny=6, lx=3.5, ly=2.4, bc_x=bc, bc_y=bc, spinor=True,
                  reservoir=True, g=0.3, g_x=0.17, g_r=0.2, delta_lt=0.11)
    psi, n, P, V = synth.random_state(2, 6, 7, 11)
    H = gp.hamiltonian_apply(psi, n, V, p)
    dV = p.dx * p.dy
    h = 1e-6
    for (c, j, i) in [(0, 0, 0), (1, 3, 4), (0, 5, 6), (1, 2, 0)]:
        d = np.zeros_like(psi)
        d[c, j, i] = h
        dEr = (gp.energy(psi + d, n, V, p) - gp.energy(psi - d, n, V, p)) / (2 * h)
        dEi = (gp.energy(psi + 1j * d, n, V, p) - gp.energy(psi - 1j * d, n, V, p)) / (2 * h)
        wirt = 0.5 * (dEr + 1j * dEi)
        assert abs(wirt - dV * H[c, j, i]) < 1e-6 * max(1.0, abs(dV * H[c, j, i]))


def test_residual_plane_wave_is_zero_and_omega_exact():
    p = P_(nx=16, ny=16, lx=8.0, ly=8.0, g=0.04)
    X, Y = np.meshgrid(np.arange(16) * p.dx, np.arange(16) * p.dy)
    kx = 2 * np.pi * 3 / 8.0
    A = 1.3
    psi = (A * np.exp(1j * kx * X))[None]
    r_psi, r_n, om = gp.residual(psi, None, None, None, p)
    K2 = (2 - 2 * np.cos(kx * p.dx)) / p.dx ** 2
    assert r_psi < 1e-12
    assert abs(om - (p.kappa * K2 + p.g * A * A) / HB) < 1e-10 * abs(om)


def test_residual_omega_minimises():
    p = gp.Params(nx=9, ny=8, lx=4.0, ly=4.0, reservoir=True, g=0.2, g_r=0.1,
                  R=0.05, gamma_c=0.2, gamma_r=0.3)
    psi, n, P, V = synth.random_state(1, 8, 9, 5)
    r, rn, om = gp.residual(psi, n, P, V, p)
    K, fn = gp.rhs(psi, n, P, V, p)
    nrm = np.linalg.norm(psi)
    for d in (1e-3, -1e-3, 0.1, -0.1):
        assert np.linalg.norm(K + 1j * (om + d) * psi) / nrm > r
    assert abs(rn - np.linalg.norm(fn) / np.linalg.norm(n)) < 1e-12 * rn


def test_norm_of_gaussian():
    """N of A exp(-r^2/w^2) on a fine periodic grid -> A^2 pi w^2 / 2."""
    n, L = 128, 40.0
    p = gp.Params(nx=n, ny=n, lx=L, ly=L)
    psi = synth.gaussian(n, n, L, L, 2.0, 3.0)[None] + 0j
    assert abs(gp.norm(psi, p) - 4.0 * np.pi * 9.0 / 2) < 1e-9


# ------------------------------------------------------------- stability

def test_stability_scalar_closed_form_and_empirical():
    """dt_max = 2 sqrt(2) hbar / (kappa (4/dx^2 + 4/dy^2)) for even periodic
    grids; RK4 on the Nyquist mode is bounded just below, grows just above."""
    p = gp.Params(nx=16, ny=16, lx=5.0, ly=5.0)
    lam = p.kappa * (4 / p.dx ** 2 + 4 / p.dy ** 2)
    dtm = gp.stability_dt_max(p)
    assert abs(dtm - 2 * np.sqrt(2) * HB / lam) < 1e-14 * dtm
    i = np.arange(16)
    psi0 = ((-1.0) ** (i[None, :] + i[:, None]) + 0j)[None]
    for f, grows in ((0.999, False), (1.01, True)):
        psi, _ = gp.run(psi0, None, None, None, p.with_(dt=f * dtm), 400)
        amp = np.max(np.abs(psi))
        assert (amp > 1.0 + 1e-3) == grows, (f, amp)


def test_stability_tetm_brute_force():
    p = gp.Params(nx=10, ny=10, lx=3.0, ly=3.0, spinor=True, delta_lt=0.5)
    lam = gp.linear_spectral_radius(p)
    # brute force: build the dense 2N x 2N Hermitian operator and take eigvals
    N = 100
    M = np.zeros((2 * N, 2 * N), complex)
    for c in range(2):
        for s in range(N):
            e = np.zeros((2, 10, 10), complex)
            e[c].flat[s] = 1.0
            M[:, c * N + s] = gp.hamiltonian_apply(e, None, None, p).reshape(-1)
    assert np.allclose(M, M.conj().T, atol=1e-12)
    ev = np.linalg.eigvalsh(M)
    assert abs(np.max(np.abs(ev)) - lam) < 1e-9 * lam


def test_derived_constants_file_matches_oracle():
    c = synth.load_constants()
    p = gp.Params(**synth.conservative_64()["params"])
    assert abs(c["conservative_64"]["dt"] - 0.5 * gp.stability_dt_max(p)) < 1e-15
    # dx = 0.3125, lambda = 0.67 * 8 / dx^2 meV
    assert abs(c["conservative_64"]["dt"] - 0.5 * 2 * np.sqrt(2) * HB / (0.67 * 8 / 0.3125 ** 2)) < 1e-15
    assert c["pump_threshold"] == pytest.approx(0.15 * 0.225 / 0.01)


@pytest.mark.parametrize("factor,grows", [(0.9, False), (1.1, True), (0.97, False),
                                           (1.03, True)])
def test_pump_threshold_from_the_dynamics(factor, grows):
    """gp.pump_threshold pinned by the equations' own dynamics rather than by
    its formula: a uniform pump factor * P_thr on a periodic grid, the
    reservoir started at its psi = 0 value P / gamma_r, a weak uniform psi.
    Below the threshold the condensate amplitude decays, above it grows (the
    amplitude stays far below saturation, so depletion plays no part); the
    net rate is (R P / gamma_r - gamma_c) / 2 for |psi|^2, i.e. the sign
    flips exactly at P = P_thr."""
    p = gp.Params(nx=2, ny=2, lx=4.0, ly=4.0, **{k: v for k, v in synth.reservoir_physics().items()})
    p = p.with_(dt=0.25)
    Pv = factor * gp.pump_threshold(p)
    psi0 = np.full((1, 2, 2), 1e-4 + 0j)
    n0 = np.full((1, 2, 2), Pv / p.gamma_r)
    P = np.full((1, 2, 2), Pv)
    steps = 2400 if abs(factor - 1) > 0.05 else 4800   # 600 / 1200 ps
    psi, n = gp.run(psi0, n0, P, None, p, steps)
    ratio = float(np.mean(np.abs(psi) ** 2) / np.mean(np.abs(psi0) ** 2))
    expected = np.exp((p.R * Pv / p.gamma_r - p.gamma_c) * steps * p.dt)
    assert (ratio > 1.0) == grows, ratio
    # and at the rate the linear analysis gives (RK4 error at dt = 0.25 ps
    # is far below 1 %)
    assert ratio == pytest.approx(expected, rel=1e-2)


@pytest.mark.parametrize("bc,nu", [(gp.PERIODIC, 0.0), (gp.ZERO, 0.0), (gp.PERIODIC, 1.5)])
def test_windowed_step_equals_full_grid_step(bc, nu):
    """oracle.gp.step_at_sites (used for sampled parity at full size) equals
    the full-grid step at every sampled site, including edges and corners,
    also in truncated-Wigner mode (renormalised density, per-site variance)."""
    p = gp.Params(nx=23, ny=19, lx=7.0, ly=6.0, bc_x=bc, bc_y=gp.PERIODIC,
                  spinor=True, reservoir=True, g=0.2, g_x=0.05, g_r=0.1, R=0.05,
                  gamma_c=0.1, gamma_r=0.2, delta_lt=0.07, noise_var=1e-3, seed=4,
                  wigner_nu=nu)
    p = p.with_(dt=0.4 * gp.stability_dt_max(p))
    psi, n, P, V = synth.random_state(2, 19, 23, 9)
    full_psi, full_n = gp.run(psi, n, P, V, p, 1, step0=3)
    sites = [(0, 0), (18, 22), (0, 22), (9, 11), (5, 0), (18, 3)]
    sp, sn = gp.step_at_sites(psi, n, P, V, p, sites, step=3)
    for k, (j, i) in enumerate(sites):
        assert np.allclose(sp[:, k], full_psi[:, j, i], rtol=0, atol=1e-13)
        assert np.allclose(sn[:, k], full_n[:, j, i], rtol=0, atol=1e-13)
