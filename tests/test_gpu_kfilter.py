"""k-space smoothing (Sec. III.B) through the C ABI against the oracle: the
step schedule, the mask on non-square, prime and power-of-two grids, both
precisions, scalar and spinor states, periodic and zero boundaries, and the
TMA-fed FP32 kernel reading the refilled ghost ring afterwards."""
import numpy as np
import pytest

from oracle import gp
import synth
from gpu_util import phx, get_state, rel_l2, rounded, TOL, TMA_SCALAR_TILES

pytestmark = pytest.mark.gpu


def model(kind, nx, ny, bc):
    d = synth.base_params(nx, ny, 0.3 * nx, 0.3 * ny, bc_x=bc[0], bc_y=bc[1])
    if kind == "reservoir":
        d.update(synth.reservoir_physics())
        d.update(g=0.3, g_r=0.5, R=0.3, gamma_r=0.4)
    elif kind == "spinor_res_tetm":
        d.update(synth.reservoir_physics())
        d.update(spinor=True, g=0.3, g_x=0.1, g_r=0.4, R=0.3, delta_lt=0.2)
    d["dt"] = min(0.45 * gp.stability_dt_max(gp.Params(**d)), 0.05)
    return d


def run_filtered(d, prec, kc, order, every, steps, step0=4, tile=0):
    m = phx()
    real, cplx = (np.float64, np.complex128) if prec == 64 else (np.float32, np.complex64)
    nc = 2 if d["spinor"] else 1
    # rough initial state, so that the mask removes a visible part of it
    psi0, n0, P, V = synth.random_state(nc, d["ny"], d["nx"], 21, amp=0.6, smooth=False)
    psi0, n0, P, V = (rounded(x, prec) for x in (psi0, n0, P, V))
    h = m.phx_create(m.params_from_dict(d, precision=prec, tile=tile))
    m.phx_set_pump(h, *[np.ascontiguousarray(P[c], real) for c in range(nc)])
    m.phx_set_potential(h, np.ascontiguousarray(V, real))
    m.phx_set_state(h, np.ascontiguousarray(psi0, cplx), np.ascontiguousarray(n0, real))
    m.phx_set_kfilter(h, kc, order, every)
    m.phx_set_time(h, step0, 0.0)
    m.phx_step_n(h, steps)
    g_psi, g_n = get_state(h, prec)
    p = gp.Params(**d).with_(kfilter_kc=kc, kfilter_order=order, kfilter_every=every)
    o_psi, o_n = gp.run(psi0, n0, P, V, p, steps, step0=step0)
    u_psi, _ = gp.run(psi0, n0, P, V, p.with_(kfilter_every=0), steps, step0=step0)
    return h, (g_psi, g_n), (o_psi, o_n), u_psi


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("kind", ["reservoir", "spinor_res_tetm"])
@pytest.mark.parametrize("size", [(131, 77), (64, 48), (97, 128)])
@pytest.mark.parametrize("bc", [(0, 0), (1, 0)])
def test_kfilter_parity(prec, kind, size, bc):
    d = model(kind, *size, bc)
    h, (g_psi, g_n), (o_psi, o_n), u_psi = run_filtered(d, prec, kc=4.0, order=2, every=3,
                                                        steps=8)
    assert rel_l2(g_psi, o_psi) <= TOL[prec], rel_l2(g_psi, o_psi)
    assert rel_l2(g_n, o_n) <= TOL[prec], rel_l2(g_n, o_n)
    # the smoothing acted (steps 5 and 8 of 4..11 are followed by it)
    assert rel_l2(u_psi, o_psi) > 1e3 * TOL[prec]


@pytest.mark.parametrize("tile", [0, 3, 6])
def test_kfilter_with_tma_scalar_kernel(tile):
    d = model("reservoir", 131, 77, (0, 0))
    h, (g_psi, g_n), (o_psi, o_n), _ = run_filtered(d, 32, kc=3.0, order=1, every=2,
                                                    steps=9, tile=tile)
    assert rel_l2(g_psi, o_psi) <= 1e-4
    assert rel_l2(g_n, o_n) <= 1e-4
    assert phx().phx_tile(h) in TMA_SCALAR_TILES


def test_kfilter_off_and_invalid_arguments():
    m = phx()
    d = model("reservoir", 40, 36, (0, 0))
    h, (g_psi, _), (o_psi, _), u_psi = run_filtered(d, 64, kc=1e9, order=1, every=1, steps=3)
    # a cutoff far above the grid's wavenumbers leaves the run unchanged
    assert rel_l2(g_psi, u_psi) <= 1e-12
    for kc, order, every in [(0.0, 1, 1), (-1.0, 1, 1), (float("nan"), 1, 1), (1.0, 0, 1),
                             (1.0, 17, 1), (1.0, 1, -1)]:
        with pytest.raises(m.PhxError) as e:
            m.phx_set_kfilter(h, kc, order, every)
        assert e.value.status == 1
    m.phx_set_kfilter(h, 0.0, 0, 0)  # off: the other arguments are ignored
