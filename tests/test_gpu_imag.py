"""Imaginary-time steps (phx_step_imag) through the C ABI against the
oracle's run_imag, and the harmonic-oscillator ground state reached on the
GPU."""
import numpy as np
import pytest

from oracle import gp
import synth
from gpu_util import phx, get_state, rel_l2, rounded, TOL

pytestmark = pytest.mark.gpu
HB = gp.HBAR


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("size", [(131, 77), (64, 64)])
def test_imag_parity(prec, size):
    m = phx()
    real, cplx = (np.float64, np.complex128) if prec == 64 else (np.float32, np.complex64)
    d = synth.base_params(*size, 0.3 * size[0], 0.3 * size[1], g=0.3, gamma_c=0.2,
                          noise_var=1e-3, dt=0.02)
    psi0, _, _, V = synth.random_state(1, size[1], size[0], 7, amp=0.7, reservoir=False,
                                       smooth=True)
    psi0, V = rounded(psi0, prec), rounded(V, prec)
    h = m.phx_create(m.params_from_dict(d, precision=prec))
    m.phx_set_potential(h, np.ascontiguousarray(V, real))
    m.phx_set_state(h, np.ascontiguousarray(psi0, cplx))
    m.phx_step_imag(h, 25)
    g_psi, _ = get_state(h, prec)
    o_psi = gp.run_imag(psi0, V, gp.Params(**d), 25)
    assert rel_l2(g_psi, o_psi) <= TOL[prec], rel_l2(g_psi, o_psi)
    s, t = m.phx_time(h)
    assert s == 0 and t == 0.0  # imaginary time does not move the clock


def test_harmonic_ground_state_on_gpu():
    m = phx()
    n, L, w = 64, 20.0, 1.0
    d = synth.base_params(n, n, L, L, dt=0.01)
    x = (np.arange(n) - n // 2) * (L / n)
    r2 = x[None, :] ** 2 + x[:, None] ** 2
    mass = HB ** 2 / (2 * d["kappa"])
    V = 0.5 * mass * w ** 2 * r2
    psi0 = (np.exp(-((x[None, :] - 1.5) ** 2 + (x[:, None] + 0.7) ** 2) / 3.0)
            * np.exp(0.8j * x[None, :]))[None]
    h = m.phx_create(m.params_from_dict(d, precision=64))
    m.phx_set_potential(h, np.ascontiguousarray(V))
    m.phx_set_state(h, np.ascontiguousarray(psi0))
    N0, _ = m.phx_norm_energy(h)
    m.phx_step_imag(h, 2000)
    out, _ = get_state(h, 64)
    N1, _ = m.phx_norm_energy(h)
    assert abs(N1 / N0 - 1) < 1e-12
    l2 = 2 * d["kappa"] / (HB * w)
    gs = np.exp(-r2 / (2 * l2))
    ov = abs(np.vdot(gs, out[0])) / (np.linalg.norm(gs) * np.linalg.norm(out[0]))
    assert ov > 1 - 1e-6


def test_imag_refuses_unsupported_states():
    m = phx()
    for kw in (dict(reservoir=True, R=0.1, gamma_r=0.2), dict(bc_y=1)):
        d = synth.base_params(40, 36, 12.0, 10.8, dt=0.01, **kw)
        h = m.phx_create(m.params_from_dict(d, precision=64))
        with pytest.raises(m.PhxError) as e:
            m.phx_step_imag(h, 1)
        assert e.value.status == 6, kw


@pytest.mark.parametrize("prec", [64, 32])
def test_imag_spinor_parity(prec):
    """Two components with cross-Kerr and TE-TM in imaginary time."""
    m = phx()
    real, cplx = (np.float64, np.complex128) if prec == 64 else (np.float32, np.complex64)
    d = synth.base_params(97, 66, 29.1, 19.8, spinor=True, g=0.3, g_x=0.1, delta_lt=0.2, dt=0.02)
    psi0, _, _, V = synth.random_state(2, 66, 97, 13, amp=0.7, reservoir=False, smooth=True)
    psi0, V = rounded(psi0, prec), rounded(V, prec)
    h = m.phx_create(m.params_from_dict(d, precision=prec))
    m.phx_set_potential(h, np.ascontiguousarray(V, real))
    m.phx_set_state(h, np.ascontiguousarray(psi0, cplx))
    m.phx_step_imag(h, 25)
    g_psi, _ = get_state(h, prec)
    o_psi = gp.run_imag(psi0, V, gp.Params(**d), 25)
    assert rel_l2(g_psi, o_psi) <= TOL[prec], rel_l2(g_psi, o_psi)
