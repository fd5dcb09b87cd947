"""Split-step Fourier steps (phx_step_ssf) through the C ABI against the
oracle's run_ssf: FP64 (1e-11) and FP32 (1e-4), prime and power-of-two,
non-square grids, potential, loss, Kerr term and per-step noise; RK4 and
split-step steps alternating on one handle; the states it refuses."""
import numpy as np
import pytest

from oracle import gp
import synth
from gpu_util import phx, get_state, rel_l2, rounded, TOL

pytestmark = pytest.mark.gpu


def params(nx, ny, **kw):
    d = synth.base_params(nx, ny, 0.3 * nx, 0.3 * ny, g=0.3, gamma_c=0.1)
    d.update(kw)
    d["dt"] = min(0.45 * gp.stability_dt_max(gp.Params(**d)), 0.05)
    return d


def start(d, prec, seed=3, with_V=True):
    m = phx()
    real, cplx = (np.float64, np.complex128) if prec == 64 else (np.float32, np.complex64)
    psi0, _, _, V = synth.random_state(1, d["ny"], d["nx"], seed, amp=0.7, reservoir=False,
                                       smooth=True)
    V = V if with_V else None
    psi0, V = rounded(psi0, prec), rounded(V, prec)
    h = m.phx_create(m.params_from_dict(d, precision=prec))
    if V is not None:
        m.phx_set_potential(h, np.ascontiguousarray(V, real))
    m.phx_set_state(h, np.ascontiguousarray(psi0, cplx))
    return h, psi0, V


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("size", [(131, 77), (64, 48), (45, 90)])
@pytest.mark.parametrize("noise_var", [0.0, 1e-4])
def test_ssf_parity(prec, size, noise_var):
    d = params(*size, noise_var=noise_var, seed=41)
    h, psi0, V = start(d, prec)
    phx().phx_set_time(h, 17, 0.0)
    phx().phx_step_ssf(h, 12)
    g_psi, _ = get_state(h, prec)
    o_psi = gp.run_ssf(psi0, V, gp.Params(**d), 12, step0=17)
    assert rel_l2(g_psi, o_psi) <= TOL[prec], rel_l2(g_psi, o_psi)
    s, t = phx().phx_time(h)
    assert s == 29 and abs(t - 12 * d["dt"]) < 1e-12


@pytest.mark.parametrize("prec", [64, 32])
def test_ssf_conservative_keeps_norm_and_alternates_with_rk4(prec):
    """gamma_c = 0: the split-step is unitary (norm kept to rounding); then
    RK4 steps continue from the split-step state (ghost ring refilled) and
    match the oracle doing the same."""
    m = phx()
    d = params(96, 70, gamma_c=0.0)
    h, psi0, V = start(d, prec, seed=5)
    N0, _ = m.phx_norm_energy(h)
    m.phx_step_ssf(h, 20)
    N1, _ = m.phx_norm_energy(h)
    assert abs(N1 / N0 - 1) < (1e-12 if prec == 64 else 2e-5)
    m.phx_step_n(h, 5)
    m.phx_step_ssf(h, 3)
    g_psi, _ = get_state(h, prec)
    p = gp.Params(**d)
    o = gp.run_ssf(psi0, V, p, 20)
    o, _ = gp.run(o, None, None, V, p, 5, step0=20)
    o = gp.run_ssf(o, V, p, 3, step0=25)
    assert rel_l2(g_psi, o) <= TOL[prec], rel_l2(g_psi, o)


def test_ssf_refuses_unsupported_states():
    m = phx()
    for kw in (dict(bc_x=1), dict(wigner_nu=1.0)):
        d = params(40, 36, **kw)
        h = m.phx_create(m.params_from_dict(d, precision=64))
        with pytest.raises(m.PhxError) as e:
            m.phx_step_ssf(h, 1)
        assert e.value.status == 6, kw  # PHX_ESTATE
    d = params(40, 36)
    h = m.phx_create(m.params_from_dict(d, precision=64))
    m.phx_set_drive(h, np.ones((36, 40), np.complex128))
    with pytest.raises(m.PhxError) as e:
        m.phx_step_ssf(h, 1)
    assert e.value.status == 6


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("tetm", [0.0, 0.2])
def test_ssf_spinor_parity(prec, tetm):
    """Two components: cross-Kerr in the local step, the spectral TE-TM block
    in the linear step, per-step noise on both components."""
    m = phx()
    real, cplx = (np.float64, np.complex128) if prec == 64 else (np.float32, np.complex64)
    d = synth.base_params(97, 66, 29.1, 19.8, spinor=True, g=0.3, g_x=0.1, gamma_c=0.05,
                          delta_lt=tetm, noise_var=1e-4, seed=43)
    d["dt"] = min(0.45 * gp.stability_dt_max(gp.Params(**d)), 0.05)
    psi0, _, _, V = synth.random_state(2, 66, 97, 9, amp=0.7, reservoir=False, smooth=True)
    psi0, V = rounded(psi0, prec), rounded(V, prec)
    h = m.phx_create(m.params_from_dict(d, precision=prec))
    m.phx_set_potential(h, np.ascontiguousarray(V, real))
    m.phx_set_state(h, np.ascontiguousarray(psi0, cplx))
    m.phx_step_ssf(h, 10)
    g_psi, _ = get_state(h, prec)
    o_psi = gp.run_ssf(psi0, V, gp.Params(**d), 10)
    assert rel_l2(g_psi, o_psi) <= TOL[prec], rel_l2(g_psi, o_psi)


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("spinor", [False, True])
def test_ssf_reservoir_parity(prec, spinor):
    """Reservoir model: local half steps integrate psi and n together (one RK4
    step each), the spectral linear step acts on psi; separate pump planes
    for two components; noise."""
    m = phx()
    real, cplx = (np.float64, np.complex128) if prec == 64 else (np.float32, np.complex64)
    kw = dict(spinor=True, g_x=0.1, delta_lt=0.2) if spinor else {}
    d = synth.base_params(83, 58, 24.9, 17.4, g=0.3, g_r=0.5, R=0.3, gamma_c=0.15, gamma_r=0.4,
                          reservoir=True, noise_var=1e-4, seed=47, **kw)
    d["dt"] = min(0.45 * gp.stability_dt_max(gp.Params(**d)), 0.05)
    nc = 2 if spinor else 1
    psi0, n0, P, V = synth.random_state(nc, 58, 83, 15, amp=0.7, smooth=True)
    psi0, n0, P, V = (rounded(x, prec) for x in (psi0, n0, P, V))
    h = m.phx_create(m.params_from_dict(d, precision=prec))
    m.phx_set_pump(h, *[np.ascontiguousarray(P[c], real) for c in range(nc)])
    m.phx_set_potential(h, np.ascontiguousarray(V, real))
    m.phx_set_state(h, np.ascontiguousarray(psi0, cplx), np.ascontiguousarray(n0, real))
    m.phx_set_time(h, 7, 0.0)
    m.phx_step_ssf(h, 9)
    g_psi, g_n = get_state(h, prec)
    o_psi, o_n = gp.run_ssf_reservoir(psi0, n0, P, V, gp.Params(**d), 9, step0=7)
    assert rel_l2(g_psi, o_psi) <= TOL[prec], rel_l2(g_psi, o_psi)
    assert rel_l2(g_n, o_n) <= TOL[prec], rel_l2(g_n, o_n)
    # RK4 steps continue from the split-step state (ghost rings refilled)
    m.phx_step_n(h, 3)
    g_psi, g_n = get_state(h, prec)
    o_psi, o_n = gp.run(o_psi, o_n, P, V, gp.Params(**d), 3, step0=16)
    assert rel_l2(g_psi, o_psi) <= TOL[prec], rel_l2(g_psi, o_psi)
    assert rel_l2(g_n, o_n) <= TOL[prec], rel_l2(g_n, o_n)


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("factor", [4.0, 12.0])
@pytest.mark.parametrize("kind", ["loss", "reservoir", "spinor_tetm"])
def test_ssf_time_step_above_the_rk4_limit(prec, factor, kind):
    """A split-step handle (integrator = split) steps at dt = factor x the RK4
    stability limit: the exact linear propagator is stable there; parity with
    the oracle's split-step at the same dt (reservoir model: local RK4 half
    steps, still well inside their own limit).  phx_step_n refuses the
    handle's dt."""
    m = phx()
    real, cplx = (np.float64, np.complex128) if prec == 64 else (np.float32, np.complex64)
    if kind == "reservoir":
        d = synth.base_params(96, 64, 28.8, 19.2, g=0.3, g_r=0.5, R=0.3, gamma_c=0.15,
                              gamma_r=0.4, reservoir=True, noise_var=1e-4, seed=49)
        nc, res = 1, True
    elif kind == "spinor_tetm":
        d = synth.base_params(96, 64, 28.8, 19.2, g=0.3, g_x=0.1, gamma_c=0.1, spinor=True,
                              delta_lt=0.2, noise_var=1e-4, seed=51)
        nc, res = 2, False
    else:
        d = synth.base_params(96, 64, 28.8, 19.2, g=0.3, gamma_c=0.1, noise_var=1e-4, seed=53)
        nc, res = 1, False
    lim = gp.stability_dt_max(gp.Params(**d))
    d.update(dt=factor * lim, integrator=1)
    psi0, n0, P, V = synth.random_state(nc, 64, 96, 17, amp=0.5, reservoir=res, smooth=True)
    psi0, n0, P, V = (rounded(x, prec) for x in (psi0, n0, P, V))
    h = m.phx_create(m.params_from_dict(d, precision=prec))
    if res:
        m.phx_set_pump(h, np.ascontiguousarray(P[0], real))
    m.phx_set_potential(h, np.ascontiguousarray(V, real))
    m.phx_set_state(h, np.ascontiguousarray(psi0, cplx),
                    None if n0 is None else np.ascontiguousarray(n0, real))
    m.phx_step_ssf(h, 10)
    g_psi, g_n = get_state(h, prec)
    p = gp.Params(**{k: v for k, v in d.items() if k != "integrator"})
    if res:
        o_psi, o_n = gp.run_ssf_reservoir(psi0, n0, P, V, p, 10)
        assert rel_l2(g_n, o_n) <= TOL[prec], rel_l2(g_n, o_n)
    else:
        o_psi = gp.run_ssf(psi0, V, p, 10)
    assert rel_l2(g_psi, o_psi) <= TOL[prec], rel_l2(g_psi, o_psi)
    assert np.all(np.isfinite(g_psi))
    s, t = m.phx_time(h)
    assert s == 10 and abs(t - 10 * d["dt"]) <= 1e-12 * t
    with pytest.raises(m.PhxError) as e:
        m.phx_step_n(h, 1)
    assert e.value.status == 6  # PHX_ESTATE
