"""Pins of the oracle's imaginary-time propagation (split-step, norm kept)."""
import numpy as np

from oracle import gp

HB = gp.HBAR


def spectral_energy(psi, V, p):
    """<psi| kappa k^2 + V |psi> / <psi|psi> with the spectral kinetic energy."""
    kx = 2 * np.pi * np.fft.fftfreq(p.nx, p.dx)
    ky = 2 * np.pi * np.fft.fftfreq(p.ny, p.dy)
    k2 = ky[:, None] ** 2 + kx[None, :] ** 2
    f = np.fft.fft2(psi)
    kin = p.kappa * np.sum(k2 * np.abs(f) ** 2) / np.sum(np.abs(f) ** 2)
    pot = np.sum(V * np.abs(psi) ** 2) / np.sum(np.abs(psi) ** 2)
    return kin + pot


def test_harmonic_ground_state():
    """V = m w^2 r^2 / 2 with m = hbar^2 / (2 kappa): the ground state is the
    Gaussian exp(-r^2 / (2 l^2)), l^2 = 2 kappa / (hbar w), of energy hbar w
    (2D); a displaced, tilted start relaxes to it."""
    n, L, w = 64, 20.0, 1.0
    p = gp.Params(nx=n, ny=n, lx=L, ly=L, kappa=0.67, dt=0.01)
    x = (np.arange(n) - n // 2) * p.dx
    r2 = x[None, :] ** 2 + x[:, None] ** 2
    m = HB ** 2 / (2 * 0.67)
    V = 0.5 * m * w ** 2 * r2
    psi0 = (np.exp(-((x[None, :] - 1.5) ** 2 + (x[:, None] + 0.7) ** 2) / 3.0)
            * np.exp(0.8j * x[None, :]))[None]
    out = gp.run_imag(psi0, V, p, 2000)[0]
    assert abs(spectral_energy(out, V, p) / (HB * w) - 1) < 1e-4
    l2 = 2 * 0.67 / (HB * w)
    gs = np.exp(-r2 / (2 * l2))
    ov = abs(np.vdot(gs, out)) / (np.linalg.norm(gs) * np.linalg.norm(out))
    assert ov > 1 - 1e-6
    assert abs(gp.norm(out[None], p) / gp.norm(psi0, p) - 1) < 1e-12


def test_two_plane_waves_decay_by_their_kinetic_energy():
    """Free field: the amplitude ratio of two plane waves falls by
    exp(-kappa (k2^2 - k1^2) tau / hbar), exactly, whatever the dt."""
    p = gp.Params(nx=24, ny=16, lx=12.0, ly=8.0, kappa=0.67, dt=0.3)
    x = np.arange(24) * p.dx
    y = np.arange(16) * p.dy
    k1 = (2 * np.pi / 12.0, 0.0)
    k2 = (2 * np.pi * 2 / 12.0, 2 * np.pi / 8.0)
    w1 = np.exp(1j * (k1[0] * x[None, :] + k1[1] * y[:, None]))
    w2 = np.exp(1j * (k2[0] * x[None, :] + k2[1] * y[:, None]))
    out = gp.run_imag((w1 + 0.5 * w2)[None], None, p, 5)[0]
    a = np.vdot(w1, out) / w1.size
    b = np.vdot(w2, out) / w2.size
    tau = 5 * 0.3
    want = 0.5 * np.exp(-0.67 * ((k2[0] ** 2 + k2[1] ** 2) - (k1[0] ** 2 + k1[1] ** 2)) * tau / HB)
    assert abs(b / a - want) < 1e-12


def test_tetm_branches_decay_by_their_energies():
    """Free spinor field with TE-TM splitting in imaginary time: the TM-like
    eigen-spinor (1, -u*) e^{ik.r} (energy (kappa - Delta) k^2) gains on the
    TE-like (1, u*) e^{ik.r} by exactly exp(2 Delta k^2 tau / hbar)."""
    p = gp.Params(nx=16, ny=12, lx=8.0, ly=6.0, spinor=True, kappa=0.67, delta_lt=0.2, dt=0.1)
    mx, my = 2, -1
    kx, ky = 2 * np.pi * mx / p.lx, 2 * np.pi * my / p.ly
    x = np.arange(p.nx) * p.dx
    y = np.arange(p.ny) * p.dy
    w = np.exp(1j * (kx * x[None, :] + ky * y[:, None]))
    k2 = kx * kx + ky * ky
    u = -((kx - 1j * ky) ** 2) / k2
    vp = np.stack([w, np.conj(u) * w])
    vm = np.stack([w, -np.conj(u) * w])
    out = gp.run_imag(vp + 0.3 * vm, None, p, 6)
    cp = np.vdot(vp, out) / np.vdot(vp, vp)
    cm = np.vdot(vm, out) / np.vdot(vm, vm)
    want = 0.3 * np.exp(2 * 0.2 * k2 * 6 * 0.1 / HB)
    assert abs(cm / cp - want) < 1e-10 * want
